// Tensor-core complex GEMM of the mixed path: D = K rho for all iterating columns (the dense step
// of Eq. 12 in residual form), fp16 operands, FP32 accumulation in TMEM.
//
// A complex product becomes four real-plane MMAs per 16-wide K step:
//     Re D = Kr rr - Ki ri,   Im D = Kr ri + Ki rr
// (the minus sign by the instruction descriptor's negate-A bit).  Tiles are 128 buses x 128
// columns with both accumulators (Re, Im) in TMEM; the K loop runs over 64-element chunks
// streamed by TMA in the 128-byte swizzle that the MMA descriptors read.
//
// One persistent CTA per SM walks the tiles.  Warp 0 issues the TMA loads into a 3-slot ring,
// warp 1 issues the MMAs, and warps 2-9 drain the accumulators (two warps per TMEM lane quarter,
// each taking half of the tile's columns).  TMEM holds two accumulator stages (2 x 256 columns),
// so the epilogue of one tile overlaps the main loop of the next.
// Every wait is bounded (2 s on %globaltimer by default): on expiry the CTA raises an error flag,
// stops, waits for its own copies and MMAs (again bounded, 2 s), frees TMEM and returns.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "tpf_gemm.h"
#include "tpf_tc.cuh"

namespace tpf {

namespace {

using namespace tc;

constexpr uint32_t kTileBytes = kTileM * kChunkK * 2;  // 16 KB: 128 rows x 64 16-bit elements
constexpr int kEpiWarps = 8;                            // two per TMEM lane quarter
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kGemmThreads = 64 + kEpiThreads;          // TMA, MMA, epilogue warps
constexpr size_t kGemmSmem = 1024 + 192 * 1024 + 2048;  // align slack + operand ring + barriers

// Complex products stream four planes per K chunk (Ar, Ai, Br, Bi) into 3 slots and keep two
// accumulators (Re, Im) per TMEM stage; real products stream two planes into 6 slots.
template <bool CPLX>
struct Cfg {
    static constexpr int kStages = CPLX ? 3 : 6;
    static constexpr uint32_t kStageBytes = (CPLX ? 4 : 2) * kTileBytes;
    static constexpr uint32_t kAccCols = CPLX ? 256 : 128;  // one stage: Re [0,128), Im [128,256)
    static constexpr uint32_t kTmemCols = 2 * kAccCols;     // two stages
};

__device__ __forceinline__ float pow2f_g(int e) {
    e = e < -126 ? -126 : (e > 127 ? 127 : e);
    return __int_as_float((127 + e) << 23);
}

// Barrier of the epilogue warps alone.
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }

// Maximum over the 32 lanes of a warp, returned to every lane (redux.sync on FP32).
__device__ __forceinline__ float warp_max_f(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ bool tile_live(const GemmEpi &ep, int64_t n_tile) {
    return ep.mode != 1 || ep.tile_active[n_tile] != 0;
}

template <bool CPLX>
__global__ void __launch_bounds__(kGemmThreads, 1)
    tc_gemm(const __grid_constant__ CUtensorMap tmAr, const __grid_constant__ CUtensorMap tmAi,
            const __grid_constant__ CUtensorMap tmBr, const __grid_constant__ CUtensorMap tmBi, int m_tiles,
            int64_t n_tiles, int n_chunks, GemmEpi ep) {
    using C = Cfg<CPLX>;
    constexpr int kStages = C::kStages;
    constexpr uint32_t kStageBytes = C::kStageBytes, kAccCols = C::kAccCols, kTmemCols = C::kTmemCols;
    extern __shared__ uint8_t smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + kStages * kStageBytes);  // [kStages]  TMA -> MMA
    uint64_t *empty = full + kStages;                              // [kStages]  MMA -> TMA
    uint64_t *tfull = empty + kStages;                             // [2]        MMA -> epilogue
    uint64_t *tempty = tfull + 2;                                  // [2]        epilogue -> MMA
    uint64_t *done = tempty + 2;                                   // [1]        all MMAs retired
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    int *abort_flag = (int *)(tmem_slot + 1);
    // Per column of the current tile (mode 1): the update's scale, 0 for a column that does not
    // iterate and negative for an anchored one (whose offset from V_ref is updated); the largest
    // |dV| over the tile's rows.
    float *col_scale = (float *)(abort_flag + 1);                  // [128]
    unsigned *col_dmax = (unsigned *)(col_scale + kTileN);         // [128]

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&tfull[a]), 1);
            mbar_init(smem_u32(&tempty[a]), kEpiWarps);  // lane 0 of each epilogue warp
        }
        mbar_init(smem_u32(done), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int64_t total = (int64_t)m_tiles * n_tiles;
    volatile int *vabort = abort_flag;
    const uint64_t lim = ep.wait_ns ? ep.wait_ns : kWaitNs;  // waits for work; drains use kWaitNs

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        const uint32_t sbase = smem_u32(smem);
        int64_t g = 0;  // chunks issued by this CTA
        for (int64_t tile = blockIdx.x; tile < total && !*vabort && !ep.withhold_loads; tile += gridDim.x) {
            const int64_t n_tile = tile / m_tiles;
            const int m_tile = (int)(tile % m_tiles);
            if (!tile_live(ep, n_tile)) continue;
            const int m0 = m_tile * kTileM;
            const int n0 = (int)(n_tile * kTileN);
            for (int c = 0; c < n_chunks; ++c, ++g) {
                const int slot = (int)(g % kStages);
                const uint32_t use = (uint32_t)(g / kStages);
                if (!mbar_wait(smem_u32(&empty[slot]), (use & 1) ^ 1, lim)) {
                    *vabort = 1;
                    atomicExch(ep.err, 1);
                    break;
                }
                const uint32_t st = sbase + slot * kStageBytes;
                const uint32_t bar = smem_u32(&full[slot]);
                mbar_expect_tx(bar, kStageBytes);
                const int k = c * kChunkK;
                if constexpr (CPLX) {
                    tma_load_2d(st, &tmAr, bar, k, m0);
                    tma_load_2d(st + kTileBytes, &tmAi, bar, k, m0);
                    tma_load_2d(st + 2 * kTileBytes, &tmBr, bar, k, n0);
                    tma_load_2d(st + 3 * kTileBytes, &tmBi, bar, k, n0);
                } else {
                    tma_load_2d(st, &tmAr, bar, k, m0);
                    tma_load_2d(st + kTileBytes, &tmBr, bar, k, n0);
                }
            }
        }
        if (*vabort) {  // let this CTA's copies in flight land before it leaves (bounded)
            for (int64_t q = g - 1; q >= 0 && q >= g - kStages; --q)
                mbar_wait(smem_u32(&full[q % kStages]), (uint32_t)(q / kStages) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t sbase = smem_u32(smem);
        const uint32_t fmt = ep.bf16 ? 1u : 0u;
        const uint32_t id_pos = idesc_f16(kTileM, kTileN, 0, fmt), id_neg = idesc_f16(kTileM, kTileN, 1, fmt);
        int64_t g = 0;
        uint32_t j = 0;  // tiles processed by this CTA
        for (int64_t tile = blockIdx.x; tile < total && !*vabort; tile += gridDim.x) {
            if (!tile_live(ep, tile / m_tiles)) continue;
            const uint32_t a = j & 1, u = j >> 1;
            if (!mbar_wait(smem_u32(&tempty[a]), (u & 1) ^ 1, lim)) {
                *vabort = 1;
                atomicExch(ep.err, 1);
                break;
            }
            tc_fence_after();
            const uint32_t tDr = tmem + a * kAccCols, tDi = tDr + kTileN;
            bool ok = true;
            for (int c = 0; c < n_chunks; ++c, ++g) {
                const int slot = (int)(g % kStages);
                if (!mbar_wait(smem_u32(&full[slot]), (uint32_t)(g / kStages) & 1, lim)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t st = sbase + slot * kStageBytes;
#pragma unroll
                for (int kk = 0; kk < kChunkK / 16; ++kk) {
                    const uint32_t first = (c | kk) != 0;
                    if constexpr (CPLX) {
                        const uint64_t ar = sw128_desc(st + kk * 32), ai = sw128_desc(st + kTileBytes + kk * 32);
                        const uint64_t br = sw128_desc(st + 2 * kTileBytes + kk * 32);
                        const uint64_t bi = sw128_desc(st + 3 * kTileBytes + kk * 32);
                        umma_f16(tDr, ar, br, id_pos, first);  // Re += Kr rr
                        umma_f16(tDr, ai, bi, id_neg, 1u);     // Re -= Ki ri
                        umma_f16(tDi, ar, bi, id_pos, first);  // Im += Kr ri
                        umma_f16(tDi, ai, br, id_pos, 1u);     // Im += Ki rr
                    } else {
                        (void)id_neg;
                        (void)tDi;
                        umma_f16(tDr, sw128_desc(st + kk * 32), sw128_desc(st + kTileBytes + kk * 32), id_pos, first);
                    }
                }
                umma_commit(smem_u32(&empty[slot]));
            }
            umma_commit(smem_u32(&tfull[a]));
            ++j;
            if (!ok) {
                *vabort = 1;
                atomicExch(ep.err, 1);
                break;
            }
        }
        umma_commit(smem_u32(done));
        mbar_wait(smem_u32(done), 0);  // every MMA of this CTA has retired (bounded)
    } else if (warp >= 2) {
        // ---------------- epilogue (256 threads: one TMEM lane each, two per lane) ----------------
        const int et = tid - 64;
        const int quarter = warp & 3;  // TMEM lanes this warp may access
        const int row = quarter * 32 + lane;
        const int half = (warp - 2) >> 2;  // the tile's columns 64 half .. 64 half + 63
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        __shared__ int s_fail;
        if (et == 0) s_fail = 0;
        epi_sync();
        uint32_t j = 0;
        for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
            const int64_t n_tile = tile / m_tiles;
            const int m_tile = (int)(tile % m_tiles);
            if (!tile_live(ep, n_tile)) continue;
            const uint32_t a = j & 1, u = j >> 1;
            if (ep.mode == 1 && et < kTileN) {
                const int64_t t = n_tile * kTileN + et;
                const int f = ep.flags[t];
                const float sc = pow2f_g(-ep.k_exp - ep.rexp[t]);
                col_scale[et] = (f & kActive) ? ((f & kAnchored) ? -sc : sc) : 0.0f;
                col_dmax[et] = 0u;
            }
            if (!mbar_wait(smem_u32(&tfull[a]), u & 1, lim)) atomicOr(&s_fail, 1);
            epi_sync();
            if (s_fail) {
                *vabort = 1;
                atomicExch(ep.err, 1);
                break;
            }
            tc_fence_after();
            const int m = m_tile * kTileM + row;
            const uint32_t tacc = tmem + a * kAccCols + lane_off;
            for (int cb = half * (kTileN / 64); cb < (half + 1) * (kTileN / 64); ++cb) {
                uint32_t vr[32], vi[32];
                tmem_ld32(tacc + cb * 32, vr);
                if constexpr (CPLX) tmem_ld32(tacc + kTileN + cb * 32, vi);
                tmem_wait_ld();
                if (ep.mode == 0) {
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int64_t nn = n_tile * kTileN + cb * 32 + q;
                        ep.Dr[nn * ep.ldD + m] = __uint_as_float(vr[q]);
                        if constexpr (CPLX) ep.Di[nn * ep.ldD + m] = __uint_as_float(vi[q]);
                    }
                } else if constexpr (!CPLX) {
                    // Layer output of this lane's unit m for 32 columns: bias, then GELU (erf form).
                    const bool live = m < ep.real;
                    const float bm = live ? ep.bias[m] : 0.0f;
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int64_t k = (n_tile * kTileN + cb * 32 + q) * ep.ldD + m;
                        const float z = live ? __uint_as_float(vr[q]) + bm : 0.0f;
                        if (ep.Dr) ep.Dr[k] = z;
                        if (ep.Ab) {
                            const float a = ep.gelu ? 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)) : z;
                            ep.Ab[k] = __bfloat16_as_ushort(__float2bfloat16_rn(a));
                        }
                    }
                } else {
                    // Update V of this lane's bus for the block's 32 columns, 16 at a time (loads
                    // first, then stores); the largest |dV|^2 of each column over the warp's rows by
                    // one warp-wide reduction, kept by lane q for column q, its square root taken
                    // once (the square root is monotonic, so this is the largest |dV|).
                    const bool row_ok = m < ep.n;
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const int c0 = cb * 32 + hh * 16;
                        float2 old[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const float sc = col_scale[c0 + q];
                            const int64_t k = (n_tile * kTileN + c0 + q) * ep.n_pad + m;
                            const float2 *src = sc < 0.0f ? ep.Vlo : ep.Vhi;  // anchored: V_ref fixed
                            old[q] = (sc != 0.0f && row_ok) ? src[k] : make_float2(0.0f, 0.0f);
                        }
                        float mine = 0.0f;
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const float sc = col_scale[c0 + q], s = fabsf(sc);
                            const float dr = __uint_as_float(vr[hh * 16 + q]) * s, di = __uint_as_float(vi[hh * 16 + q]) * s;
                            float d2 = 0.0f;
                            if (sc != 0.0f && row_ok) {
                                const int64_t k = (n_tile * kTileN + c0 + q) * ep.n_pad + m;
                                float2 *dst = sc < 0.0f ? ep.Vlo : ep.Vhi;
                                dst[k] = make_float2(old[q].x + dr, old[q].y + di);
                                d2 = __fmaf_rn(dr, dr, __fmul_rn(di, di));
                                if (d2 != d2) d2 = __int_as_float(0x7f800000);  // NaN -> +inf
                            }
                            const float mx = warp_max_f(d2);
                            if (lane == q) mine = mx;
                        }
                        if (lane < 16 && mine > 0.0f) atomicMax(&col_dmax[c0 + lane], __float_as_uint(sqrtf(mine)));
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[a]));  // accumulator stage a is free again
            epi_sync();
            if (ep.mode == 1 && et < kTileN) {
                const unsigned d = col_dmax[et];
                if (d) atomicMax(&ep.delta[n_tile * kTileN + et], d);
            }
            epi_sync();  // column info is rewritten by the next tile
            ++j;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// A [rows][inner] 16-bit matrix read in (128 rows x 64 elements) boxes, 128-byte swizzle.
bool make_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, bool bf16) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)kChunkK, (cuuint32_t)kTileM};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool make_bf16_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows) {
    return make_map(map, base, inner, rows, true);
}

bool make_f64_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows, uint32_t box_inner,
                  uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 8};
    cuuint32_t box[2] = {box_inner, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_gemm_maps(GemmMaps *maps, const void *Ar, const void *Ai, int M, int K, const void *Br, const void *Bi,
                    int64_t N, bool bf16) {
    std::memset(maps, 0, sizeof(*maps));
    if (!make_map(&maps->ar, Ar, K, M, bf16) || !make_map(&maps->br, Br, K, N, bf16)) return false;
    if (Ai && !make_map(&maps->ai, Ai, K, M, bf16)) return false;
    if (Bi && !make_map(&maps->bi, Bi, K, N, bf16)) return false;
    return true;
}

tpf_status launch_gemm(const GemmMaps &maps, int m_tiles, int64_t n_tiles, int n_chunks, const GemmEpi &ep,
                       cudaStream_t st) {
    static std::atomic<uint64_t> attr{0};
    if (!once_per_device(attr, [] {
            return cudaFuncSetAttribute(tc_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem) ==
                       cudaSuccess &&
                   cudaFuncSetAttribute(tc_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem) ==
                       cudaSuccess;
        }))
        return TPF_ECUDA;
    if (ep.cplx ? ep.mode == 2 : ep.mode == 1) return TPF_EINVAL;
    if (ep.mode == 2 && (!ep.bias || (!ep.Dr && !ep.Ab))) return TPF_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    const int64_t total = (int64_t)m_tiles * n_tiles;
    const unsigned grid = (unsigned)(total < sms ? total : sms);
    if (ep.cplx)
        tc_gemm<true><<<grid, kGemmThreads, kGemmSmem, st>>>(maps.ar, maps.ai, maps.br, maps.bi, m_tiles, n_tiles,
                                                             n_chunks, ep);
    else
        tc_gemm<false><<<grid, kGemmThreads, kGemmSmem, st>>>(maps.ar, maps.ai, maps.br, maps.bi, m_tiles, n_tiles,
                                                              n_chunks, ep);
    if (cudaGetLastError() != cudaSuccess) return TPF_ECUDA;
    return TPF_OK;
}

}  // namespace tpf
