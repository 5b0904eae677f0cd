// The tensor-core complex GEMM of the mixed path (tpf_gemm.cu).
#pragma once

#include <cuda.h>

#include "tpf_internal.h"

namespace tpf {

// What the GEMM epilogue does with D = A B^T (one 128 x 128 tile per accumulator stage).
struct GemmEpi {
    int mode;  // 0 = store D (FP32), 1 = fixed-point update of V (complex only), 2 = bias and
               // activation of a network layer (real only)
    int cplx;  // 1: A, B, D complex (four real-plane MMAs per K step); 0: real (one MMA)
    int bf16;  // operand format: 0 = fp16, 1 = bf16
    int *err;  // set to 1 when a bounded wait expires
    // Limit of every wait for work (0: the default 2 s).  The waits that drain a stopped CTA's own
    // copies and MMAs keep the default.
    uint64_t wait_ns;
    // Self-test of the bounded waits only: the producer issues no copies, so the MMA and epilogue
    // waits run out after wait_ns and the kernel takes its error path (flag, drain, free TMEM).
    int withhold_loads;
    // mode 0: D[n][m] in two FP32 planes with leading dimension ldD (= M)
    float *Dr, *Di;
    int ldD;
    // mode 1: V += 2^-(k_exp + rexp[col]) D for iterating columns, max |dV| per column into delta
    int n, n_pad, k_exp;
    const int *flags, *rexp, *tile_active;
    float2 *Vhi, *Vlo;
    unsigned *delta;
    // mode 2: z = D + bias[m] for rows m < real (z = 0 beyond); Dr[n][m] = z when Dr is set, and
    // Ab[n][m] = bf16(gelu(z)) (gelu != 0) or bf16(z) when Ab is set (16-bit words), both with
    // leading dimension ldD
    const float *bias;
    int real, gelu;
    unsigned short *Ab;
};

// Tensor maps of the four fp16 operand planes: A (K) [M][K] and B (rho) [N][K], K fastest.
struct GemmMaps {
    CUtensorMap ar, ai, br, bi;
};

// A [rows][inner] BF16 matrix read in (128 rows x 64 elements) boxes with the 128-byte swizzle.
bool make_bf16_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows);
// A [rows][inner] FP64 matrix (row stride inner * 8 bytes, a multiple of 16) read in unswizzled
// (box_rows x box_inner) boxes; elements outside the matrix read as zero.
bool make_f64_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint32_t box_inner,
                  uint32_t box_rows);

// Ai, Bi may be null for a real product.  bf16 selects the element type of the maps.
bool make_gemm_maps(GemmMaps *maps, const void *Ar, const void *Ai, int M, int K, const void *Br, const void *Bi,
                    int64_t N, bool bf16 = false);

// D = A B^T (complex or real, per ep.cplx) for all (m_tiles x n_tiles) tiles of 128 x 128,
// K = 64 n_chunks, by one persistent CTA per SM.  In mode 1, tiles whose tile_active entry is 0
// are skipped.
tpf_status launch_gemm(const GemmMaps &maps, int m_tiles, int64_t n_tiles, int n_chunks, const GemmEpi &ep,
                       cudaStream_t st);

}  // namespace tpf
