// The fused inference kernel of the learned warm start (tpf_mlp_infer.cu).
#pragma once

#include <cuda.h>

#include "tpf_internal.h"

namespace tpf {

constexpr int kMaxInferLayers = 8;  // weight layers the fused kernel takes (up to 7 hidden layers)

struct InferArgs {
    CUtensorMap map_w[kMaxInferLayers];     // W_l [out][in] BF16, box 64 x 128: W_0 with interleaved inputs,
                                            // W_{L-1} with interleaved output rows
    const float *bias[kMaxInferLayers];     // FP32 biases of the hidden layers
    CUtensorMap map_s;                      // S [T][n] complex128 as FP64 [T][2n], box 64 x 32, no swizzle
    const float4 *xnorm;                    // [P0 / 2] per bus: 1 / sd_P, -mean_P / sd_P, 1 / sd_Q, -mean_Q / sd_Q
                                            // (zero for padding buses and constant features)
    const float *bias_out;                  // [PL] last layer's bias, interleaved
    const float *out_mean, *out_std;        // [PL] target statistics, interleaved
    int L, H, P0, PL, n;                    // weight layers, hidden width (128 or 256), padded widths, buses
    int64_t T, tiles;                       // columns and 128-column tiles
    float lo2, hi2;                         // guard: |V_0|^2 must lie in [lo2, hi2]
    void *V0;                               // [T][n] complex64, or complex128 when v0_64
    int v0_64;
    int guard;                              // apply the |V| guard here (else the reader checks)
    int v0_half;                            // V0 holds half2 deviations (Re V - 1, Im V) instead
    int64_t pitch;                          // complex values per column of V0 (>= n; n for [T][n])
    int *fallback;                          // columns that failed the guard (given the flat start)
    int *err;                               // set when a bounded wait expired
};

// Whether the fused kernel takes a network of this shape.
bool infer_supported(int L, int H, int P0, int PL);

// One launch over g.tiles tiles (one persistent CTA per SM).
tpf_status launch_infer(const InferArgs &g, cudaStream_t st);

}  // namespace tpf
