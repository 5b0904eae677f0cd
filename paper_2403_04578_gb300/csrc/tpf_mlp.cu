// Learned warm start: a multilayer perceptron that maps a column's loads to a starting voltage
// for the fixed-point iteration (not in the paper; it only changes V_0 of Algorithm 1, whose
// iterates then converge to the same high-voltage solution from any start).
//
// Features of a column: P_1..P_n, Q_1..Q_n of the demand buses (Re/Im of S), z-scored per feature;
// targets: Re V_i - 1 and Im V_i, z-scored.  Layers z_l = W_l a_{l-1} + b_l, a_l = gelu(z_l)
// (erf form), linear output, mean squared error, Adam.  Every matrix product runs on the
// tcgen05 tensor cores in BF16 with FP32 accumulation (tpf_gemm.cu, real mode):
//   forward   Z_l  = A_{l-1} W_l^T          (A = W_l,     B = A_{l-1})
//   weights   dW_l = dZ_l^T A_{l-1}         (A = dZ_l^T,  B = A_{l-1}^T; D comes out transposed)
//   inputs    dA   = dZ_l W_l               (A = W_l^T,   B = dZ_l)
// FP32 master weights, BF16 copies (W and W^T) for the products.  Feature dimensions are padded
// to multiples of 128 and the batch to a multiple of 128; padded units stay exactly zero.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "tpf_gemm.h"
#include "tpf_mlp_infer.h"

using bf16 = __nv_bfloat16;

struct tpf_mlp {
    int device = 0;
    int n = 0;                 // demand buses of the feeder
    int L = 0;                 // weight layers
    std::vector<int> dim, pad; // real and padded widths, L + 1 entries
    int max_batch = 0;
    int64_t step = 0;          // Adam step counter
    // device parameters, per layer
    std::vector<float *> W, b, mW, vW, mb, vb, gWT, gb;
    std::vector<bf16 *> Wb, WTb;
    // normalisation (device, FP32): features and targets
    float *in_mean = nullptr, *in_std = nullptr, *out_mean = nullptr, *out_std = nullptr;
    // activations for max_batch columns
    bf16 *X0 = nullptr, *X0T = nullptr;
    std::vector<float *> Z;          // pre-activations [B][pad_l]
    std::vector<bf16 *> A, AT;       // activations and transposes (hidden layers)
    std::vector<bf16 *> dZ, dZT;     // gradients of the pre-activations
    float *dA = nullptr;             // [B][max pad]
    float *target = nullptr;         // [B][pad_L]
    double *loss = nullptr;          // [1]
    int *err = nullptr;              // GEMM wait-expiry flag
    int *fallback = nullptr;         // [1] columns whose prediction failed the guard
    // Fused inference (tpf_mlp_infer.cu): the first and last layers with interleaved inputs /
    // outputs, the last bias and the statistics in the same order, rebuilt when stale.
    bool infer_fresh = false;
    bf16 *Wi0 = nullptr, *WiL = nullptr;   // [pad1][pad0] and [padL][pad(L-1)]
    float *bi_out = nullptr, *om_i = nullptr, *os_i = nullptr;  // [padL]
    float4 *xn_i = nullptr;  // [pad0 / 2] per bus: 1 / sd_P, -mean_P / sd_P, 1 / sd_Q, -mean_Q / sd_Q
    __half2 *V0c = nullptr;                // predicted deviations (Re V - 1, Im V) of tpf_solve_learned
    int64_t v0_cap = 0;                    // complex values allocated in V0c
};

namespace tpf {
namespace {

#define MLP_CK(call)                 \
    do {                             \
        if ((call) != cudaSuccess) { \
            cudaGetLastError();      \
            return TPF_ECUDA;        \
        }                            \
    } while (0)

constexpr int kThreads = 256;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// The elementwise kernels run on a 2-D grid: x over the features (or units) of a column, y over
// the columns b of the batch (grid-stride), so that no thread divides an index.
//
// Features of columns t0..t0+B-1 (rows beyond T are zero): x = (f - mean) / std, feature j < n
// is Re S_j and feature n + j is Im S_j; features 2n .. P-1 are padding (zero).  Thread j reads
// S_j once and writes both of its features, and zeroes padding feature 2n + j.
__global__ void k_features(const double2 *__restrict__ S, int64_t T, int64_t t0, int B, int n, int P,
                           const float *__restrict__ mean, const float *__restrict__ sd, bf16 *X, bf16 *XT) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool feat = j < n, pad = j < P - 2 * n;
    if (!feat && !pad) return;
    const float mr = feat ? mean[j] : 0.0f, dr = feat ? sd[j] : 0.0f;
    const float mi = feat ? mean[n + j] : 0.0f, di = feat ? sd[n + j] : 0.0f;
    const bf16 zero = __float2bfloat16_rn(0.0f);
    for (int b = blockIdx.y; b < B; b += gridDim.y) {
        const int64_t t = t0 + b;
        if (feat) {
            float xr = 0.0f, xi = 0.0f;
            if (t < T) {
                const double2 s = S[t * n + j];
                xr = dr > 0.0f ? ((float)s.x - mr) / dr : 0.0f;
                xi = di > 0.0f ? ((float)s.y - mi) / di : 0.0f;
            }
            const bf16 vr = __float2bfloat16_rn(xr), vi = __float2bfloat16_rn(xi);
            X[(int64_t)b * P + j] = vr;
            X[(int64_t)b * P + n + j] = vi;
            if (XT) {
                XT[(int64_t)j * B + b] = vr;
                XT[(int64_t)(n + j) * B + b] = vi;
            }
        }
        if (pad) {
            X[(int64_t)b * P + 2 * n + j] = zero;
            if (XT) XT[(int64_t)(2 * n + j) * B + b] = zero;
        }
    }
}

// Normalised targets: (Re V - 1, Im V).
__global__ void k_targets(const double2 *__restrict__ V, int64_t T, int64_t t0, int B, int n, int P,
                          const float *__restrict__ mean, const float *__restrict__ sd, float *Y) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * P) return;
    const int b = (int)(idx / P), j = (int)(idx % P);
    const int64_t t = t0 + b;
    float y = 0.0f;
    if (t < T && j < 2 * n) {
        const double2 v = V[t * n + (j < n ? j : j - n)];
        const float f = j < n ? (float)(v.x - 1.0) : (float)v.y;
        y = sd[j] > 0.0f ? (f - mean[j]) / sd[j] : 0.0f;
    }
    Y[idx] = y;
}

// z += b; a = gelu(z) (hidden) or z (output); padded units forced to zero.  AT (the transposed
// activations, for the weight gradients) may be null.
__global__ void k_act_fwd(float *Z, const float *__restrict__ bias, int B, int P, int real, int hidden, bf16 *A,
                          bf16 *AT) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= P) return;
    const float bo = o < real ? bias[o] : 0.0f;
    for (int b = blockIdx.y; b < B; b += gridDim.y) {
        const int64_t idx = (int64_t)b * P + o;
        const float z = o < real ? Z[idx] + bo : 0.0f;
        Z[idx] = z;
        if (hidden) {
            const bf16 a = __float2bfloat16_rn(o < real ? gelu(z) : 0.0f);
            A[idx] = a;
            if (AT) AT[(int64_t)o * B + b] = a;
        }
    }
}

// dL/dy of the mean squared error over B x real outputs, and the loss.
__global__ void k_loss_grad(const float *__restrict__ Y, const float *__restrict__ T, int B, int P, int real,
                            bf16 *dZ, bf16 *dZT, double *loss) {
    __shared__ float red[kThreads / 32];
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float sq = 0.0f;
    if (idx < (int64_t)B * P) {
        const int b = (int)(idx / P), o = (int)(idx % P);
        float g = 0.0f;
        if (o < real) {
            const float d = Y[idx] - T[idx];
            sq = d * d;
            g = 2.0f * d / ((float)B * (float)real);
        }
        const bf16 v = __float2bfloat16_rn(g);
        dZ[idx] = v;
        dZT[(int64_t)o * B + b] = v;
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        atomicAdd(loss, (double)s / ((double)B * (double)real));
    }
}

// dz = da * gelu'(z) for a hidden layer.
__global__ void k_act_bwd(const float *__restrict__ dA, const float *__restrict__ Z, int B, int P, int real,
                          bf16 *dZ, bf16 *dZT) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * P) return;
    const int b = (int)(idx / P), o = (int)(idx % P);
    const float g = o < real ? dA[idx] * gelu_grad(Z[idx]) : 0.0f;
    const bf16 v = __float2bfloat16_rn(g);
    dZ[idx] = v;
    dZT[(int64_t)o * B + b] = v;
}

// db[o] = sum_b dZ[b][o] (one warp per output unit, rows of dZ^T are contiguous).
__global__ void k_bias_grad(const bf16 *__restrict__ dZT, int B, int P, float *db) {
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (o >= P) return;
    float s = 0.0f;
    for (int b = lane; b < B; b += 32) s += __bfloat162float(dZT[(int64_t)o * B + b]);
    for (int k = 16; k > 0; k >>= 1) s += __shfl_xor_sync(0xffffffffu, s, k);
    if (lane == 0) db[o] = s;
}

// Adam on W (gradient given transposed, gWT[k][o]) and b; then the BF16 copies W and W^T.
__global__ void k_adam(float *W, const float *__restrict__ gWT, float *m, float *v, float *b, const float *__restrict__ gb,
                       float *mb, float *vb, bf16 *Wb, bf16 *WTb, int Pout, int Pin, int real_out, int real_in, float lr,
                       float b1, float b2, float eps, float c1, float c2, int update) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx < (int64_t)Pout * Pin) {
        const int o = (int)(idx / Pin), k = (int)(idx % Pin);
        float w = W[idx];
        if (update && o < real_out && k < real_in) {
            const float g = gWT[(int64_t)k * Pout + o];
            const float mm = b1 * m[idx] + (1.0f - b1) * g;
            const float vv = b2 * v[idx] + (1.0f - b2) * g * g;
            m[idx] = mm;
            v[idx] = vv;
            w -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
            W[idx] = w;
        }
        const bf16 wb = __float2bfloat16_rn(w);
        Wb[idx] = wb;
        WTb[(int64_t)k * Pout + o] = wb;
    }
    if (update && idx < real_out) {
        const float g = gb[idx];
        const float mm = b1 * mb[idx] + (1.0f - b1) * g;
        const float vv = b2 * vb[idx] + (1.0f - b2) * g * g;
        mb[idx] = mm;
        vb[idx] = vv;
        b[idx] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// Mean and standard deviation of each feature (f < 2n: Re/Im of S) and target (Re V - 1, Im V)
// over T columns; one block per quantity, double accumulation.
__global__ void k_norm_stats(const double2 *__restrict__ S, const double2 *__restrict__ V, int64_t T, int n,
                             float *in_mean, float *in_std, float *out_mean, float *out_std) {
    __shared__ double r1[kThreads], r2[kThreads];
    const int q = blockIdx.x;  // [0, 2n): features, [2n, 4n): targets
    const bool is_in = q < 2 * n;
    const int j = is_in ? q : q - 2 * n;
    const int bus = j < n ? j : j - n;
    double s1 = 0.0, s2 = 0.0;
    for (int64_t t = threadIdx.x; t < T; t += blockDim.x) {
        double f;
        if (is_in) {
            const double2 s = S[t * n + bus];
            f = j < n ? s.x : s.y;
        } else {
            const double2 v = V[t * n + bus];
            f = j < n ? v.x - 1.0 : v.y;
        }
        s1 += f;
        s2 += f * f;
    }
    r1[threadIdx.x] = s1;
    r2[threadIdx.x] = s2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            r1[threadIdx.x] += r1[threadIdx.x + w];
            r2[threadIdx.x] += r2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mu = r1[0] / (double)T;
        const double var = r2[0] / (double)T - mu * mu;
        const float sd = var > 0.0 ? (float)sqrt(var) : 0.0f;
        if (is_in) {
            in_mean[j] = (float)mu;
            in_std[j] = sd;
        } else {
            out_mean[j] = (float)mu;
            out_std[j] = sd;
        }
    }
}

// Denormalise the prediction of columns t0..t0+B-1 into V_0; one warp per column.  A column
// whose predicted |V_i| leaves [lo, hi] anywhere (or is not finite) gets the flat start instead.
// The prediction is an approximate start: it is formed in FP32 (the iteration refines it).
__global__ void k_predict_out(const float *__restrict__ Y, int B, int P, int n, int64_t T, int64_t t0,
                              const float *__restrict__ mean, const float *__restrict__ sd, float lo, float hi,
                              double2 *V0, int *fallback) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (b >= B || t0 + b >= T) return;
    const int64_t t = t0 + b;
    bool ok = true;
    for (int i = lane; i < n; i += 32) {
        const float re = 1.0f + (Y[(int64_t)b * P + i] * sd[i] + mean[i]);
        const float im = Y[(int64_t)b * P + n + i] * sd[n + i] + mean[n + i];
        const float mag2 = re * re + im * im;
        if (!(mag2 >= lo * lo && mag2 <= hi * hi)) ok = false;
        V0[t * n + i] = make_double2((double)re, (double)im);
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
        for (int i = lane; i < n; i += 32) V0[t * n + i] = make_double2(1.0, 0.0);
        if (lane == 0) atomicAdd(fallback, 1);
    }
}

// The inference copies: W_0 with its inputs interleaved (column 2j <- j, 2j + 1 <- n + j), W_{L-1},
// its bias and the target statistics with their outputs interleaved (row 2i <- i, 2i + 1 <- n + i),
// and per bus the feature z-score as a scale and a shift (x = s * scale + shift; both zero where
// the standard deviation is, as in the training features).  One thread per element of the largest.
__global__ void k_infer_weights(const float *__restrict__ W0, const float *__restrict__ WL, const float *__restrict__ bL,
                                const float *__restrict__ im, const float *__restrict__ is,
                                const float *__restrict__ om, const float *__restrict__ os, int n, int P0, int H0,
                                int PL, int HL, bf16 *Wi0, bf16 *WiL, float *bi, float4 *xn, float *omi, float *osi) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    auto src = [n](int k) { return (k & 1) ? n + (k >> 1) : (k >> 1); };  // interleaved -> blocked index
    if (idx < (int64_t)H0 * P0) {  // W_0 [H0][P0]
        const int o = (int)(idx / P0), k = (int)(idx % P0);
        Wi0[idx] = __float2bfloat16_rn(k < 2 * n ? W0[(int64_t)o * P0 + src(k)] : 0.0f);
    }
    if (idx < (int64_t)PL * HL) {  // W_{L-1} [PL][HL]
        const int o = (int)(idx / HL), k = (int)(idx % HL);
        WiL[idx] = __float2bfloat16_rn(o < 2 * n ? WL[(int64_t)src(o) * HL + k] : 0.0f);
    }
    if (idx < PL) {
        const int o = (int)idx;
        bi[o] = o < 2 * n ? bL[src(o)] : 0.0f;
        omi[o] = o < 2 * n ? om[src(o)] : 0.0f;
        osi[o] = o < 2 * n ? os[src(o)] : 0.0f;
    }
    if (idx < P0 / 2) {
        const int j = (int)idx;
        float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (j < n) {
            const float dp = is[j], dq = is[n + j];
            if (dp > 0.0f) z.x = 1.0f / dp, z.y = -im[j] / dp;
            if (dq > 0.0f) z.z = 1.0f / dq, z.w = -im[n + j] / dq;
        }
        xn[j] = z;
    }
}

unsigned blocks(int64_t work) { return (unsigned)((work + kThreads - 1) / kThreads); }

// D[N][M] (FP32) = sum_k A[M][K] B[N][K] on the tensor cores, BF16 operands.
tpf_status gemm_bf16(const void *A, int M, int K, const void *B, int N, float *D, int *err, cudaStream_t st) {
    GemmMaps maps;
    if (!make_gemm_maps(&maps, A, nullptr, M, K, B, nullptr, N, true)) return TPF_ECUDA;
    GemmEpi ep{};
    ep.mode = 0;
    ep.cplx = 0;
    ep.bf16 = 1;
    ep.err = err;
    ep.Dr = D;
    ep.ldD = M;
    return launch_gemm(maps, M / kTileM, N / kTileN, K / kChunkK, ep, st);
}

// The same product with the layer's bias and activation in the epilogue: z = D + bias for the
// first `real` rows; Z (FP32, may be null) receives z, Ab (may be null) bf16(gelu(z)) or bf16(z).
tpf_status gemm_bf16_layer(const void *A, int M, int K, const void *B, int N, const float *bias, int real, bool gelu,
                           float *Z, bf16 *Ab, int *err, cudaStream_t st) {
    GemmMaps maps;
    if (!make_gemm_maps(&maps, A, nullptr, M, K, B, nullptr, N, true)) return TPF_ECUDA;
    GemmEpi ep{};
    ep.mode = 2;
    ep.cplx = 0;
    ep.bf16 = 1;
    ep.err = err;
    ep.Dr = Z;
    ep.ldD = M;
    ep.bias = bias;
    ep.real = real;
    ep.gelu = gelu ? 1 : 0;
    ep.Ab = reinterpret_cast<unsigned short *>(Ab);
    return launch_gemm(maps, M / kTileM, N / kTileN, K / kChunkK, ep, st);
}

void free_mlp(tpf_mlp *h) {
    auto F = [](auto &v) {
        for (auto p : v) cudaFree(p);
        v.clear();
    };
    F(h->W); F(h->b); F(h->mW); F(h->vW); F(h->mb); F(h->vb); F(h->gWT); F(h->gb); F(h->Wb); F(h->WTb);
    F(h->Z); F(h->A); F(h->AT); F(h->dZ); F(h->dZT);
    cudaFree(h->in_mean); cudaFree(h->in_std); cudaFree(h->out_mean); cudaFree(h->out_std);
    cudaFree(h->X0); cudaFree(h->X0T); cudaFree(h->dA); cudaFree(h->target); cudaFree(h->loss); cudaFree(h->err);
    cudaFree(h->fallback);
    cudaFree(h->Wi0); cudaFree(h->WiL); cudaFree(h->bi_out); cudaFree(h->om_i); cudaFree(h->os_i);
    cudaFree(h->xn_i); cudaFree(h->V0c);
    cudaGetLastError();
}

template <typename T>
bool dalloc(T **p, size_t count) {
    if (cudaMalloc((void **)p, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    cudaMemset(*p, 0, sizeof(T) * (count ? count : 1));
    return true;
}

// Rewrite the BF16 copies of every layer from the FP32 masters (no update).
tpf_status publish(tpf_mlp *h, cudaStream_t st) {
    h->infer_fresh = false;
    for (int l = 0; l < h->L; ++l) {
        const int Po = h->pad[l + 1], Pi = h->pad[l];
        k_adam<<<blocks((int64_t)Po * Pi), kThreads, 0, st>>>(h->W[l], h->gWT[l], h->mW[l], h->vW[l], h->b[l], h->gb[l],
                                                              h->mb[l], h->vb[l], h->Wb[l], h->WTb[l], Po, Pi,
                                                              h->dim[l + 1], h->dim[l], 0.f, 0.f, 0.f, 0.f, 1.f, 1.f, 0);
    }
    MLP_CK(cudaGetLastError());
    return TPF_OK;
}

// 2-D grid of the elementwise kernels for B columns of P features or units.
dim3 grid2(int P, int B) { return dim3((unsigned)((P + kThreads - 1) / kThreads), (unsigned)std::min(B, 4096)); }

// Forward pass of B columns whose features are in X0; leaves Z[L-1] = normalised prediction.
// Training also keeps every layer's Z and writes the transposed activations that the weight
// gradients read (a pass of its own); inference takes bias and GELU in the product's epilogue.
tpf_status forward(tpf_mlp *h, int B, cudaStream_t st, bool train) {
    const bf16 *in = h->X0;
    for (int l = 0; l < h->L; ++l) {
        const int Po = h->pad[l + 1], Pi = h->pad[l];
        const bool hidden = l < h->L - 1;
        if (!train) {
            tpf_status rs = gemm_bf16_layer(h->Wb[l], Po, Pi, in, B, h->b[l], h->dim[l + 1], hidden,
                                            hidden ? nullptr : h->Z[l], hidden ? h->A[l] : nullptr, h->err, st);
            if (rs != TPF_OK) return rs;
            in = hidden ? h->A[l] : nullptr;
            continue;
        }
        tpf_status rs = gemm_bf16(h->Wb[l], Po, Pi, in, B, h->Z[l], h->err, st);
        if (rs != TPF_OK) return rs;
        k_act_fwd<<<grid2(Po, B), kThreads, 0, st>>>(h->Z[l], h->b[l], B, Po, h->dim[l + 1], hidden,
                                                     hidden ? h->A[l] : nullptr,
                                                     hidden && train ? h->AT[l] : nullptr);
        MLP_CK(cudaGetLastError());
        in = hidden ? h->A[l] : nullptr;
    }
    return TPF_OK;
}

// Backward pass after forward() with targets in h->target: fills gWT and gb of every layer.
tpf_status backward(tpf_mlp *h, int B, cudaStream_t st) {
    const int L = h->L;
    MLP_CK(cudaMemsetAsync(h->loss, 0, sizeof(double), st));
    k_loss_grad<<<blocks((int64_t)B * h->pad[L]), kThreads, 0, st>>>(h->Z[L - 1], h->target, B, h->pad[L], h->dim[L],
                                                                      h->dZ[L - 1], h->dZT[L - 1], h->loss);
    MLP_CK(cudaGetLastError());
    for (int l = L - 1; l >= 0; --l) {
        const int Po = h->pad[l + 1], Pi = h->pad[l];
        const bf16 *inT = l > 0 ? h->AT[l - 1] : h->X0T;
        tpf_status rs = gemm_bf16(h->dZT[l], Po, B, inT, Pi, h->gWT[l], h->err, st);  // dW^T [Pi][Po]
        if (rs != TPF_OK) return rs;
        k_bias_grad<<<(Po * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(h->dZT[l], B, Po, h->gb[l]);
        MLP_CK(cudaGetLastError());
        if (l > 0) {
            rs = gemm_bf16(h->WTb[l], Pi, Po, h->dZ[l], B, h->dA, h->err, st);  // dA [B][Pi]
            if (rs != TPF_OK) return rs;
            k_act_bwd<<<blocks((int64_t)B * Pi), kThreads, 0, st>>>(h->dA, h->Z[l - 1], B, Pi, h->dim[l], h->dZ[l - 1],
                                                                    h->dZT[l - 1]);
            MLP_CK(cudaGetLastError());
        }
    }
    return TPF_OK;
}

tpf_status load_batch(tpf_mlp *h, int B, const void *S, const void *V, int64_t T, int64_t t0, bool transpose,
                      cudaStream_t st) {
    k_features<<<grid2(std::max(h->n, h->pad[0] - 2 * h->n), B), kThreads, 0, st>>>(
        (const double2 *)S, T, t0, B, h->n, h->pad[0], h->in_mean, h->in_std, h->X0, transpose ? h->X0T : nullptr);
    if (V)
        k_targets<<<blocks((int64_t)B * h->pad[h->L]), kThreads, 0, st>>>(
            (const double2 *)V, T, t0, B, h->n, h->pad[h->L], h->out_mean, h->out_std, h->target);
    MLP_CK(cudaGetLastError());
    return TPF_OK;
}

tpf_status check_err(tpf_mlp *h, cudaStream_t st) {
    int e = 0;
    MLP_CK(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MLP_CK(cudaStreamSynchronize(st));
    return e ? TPF_ETIMEOUT : TPF_OK;
}

bool fused_ok(const tpf_mlp *h) {
    const int L = h->L, H = h->pad[1];
    for (int l = 1; l < L; ++l)
        if (h->pad[l] != H) return false;
    return infer_supported(L, H, h->pad[0], h->pad[L]);
}

// Predicted V_0 of T columns with the fused kernel (one launch; it reads S itself): complex128
// (v0_64) or complex64 into V0, or with v0_half the half-precision deviations (Re V - 1, Im V);
// with guard, a column whose prediction leaves the |V| band gets the flat start here (otherwise
// its reader, the learned-start solve, checks the band).  V0 holds pitch (default n) values per
// column.
tpf_status infer_fused(tpf_mlp *h, int64_t T, const void *S, void *V0, bool v0_64, cudaStream_t st,
                       bool guard = true, int64_t pitch = 0, int64_t *launches = nullptr, bool v0_half = false) {
    const int L = h->L, H = h->pad[1], P0 = h->pad[0], PL = h->pad[L];
    // S is read by TMA: a 16-byte aligned base, and column indices within its 32-bit coordinates.
    if (reinterpret_cast<uintptr_t>(S) % 16 || T > ((int64_t)1 << 31) - 256) return TPF_EINVAL;
    if (!h->infer_fresh) {
        if (!h->Wi0 && !(dalloc(&h->Wi0, (size_t)H * P0) && dalloc(&h->WiL, (size_t)PL * h->pad[L - 1]) &&
                         dalloc(&h->bi_out, PL) && dalloc(&h->om_i, PL) && dalloc(&h->os_i, PL) &&
                         dalloc(&h->xn_i, P0 / 2)))
            return TPF_ENOMEM;
        const int64_t work = std::max<int64_t>((int64_t)H * P0, (int64_t)PL * h->pad[L - 1]);
        k_infer_weights<<<blocks(work), kThreads, 0, st>>>(h->W[0], h->W[L - 1], h->b[L - 1], h->in_mean, h->in_std,
                                                           h->out_mean, h->out_std, h->n, P0, H, PL, h->pad[L - 1],
                                                           h->Wi0, h->WiL, h->bi_out, h->xn_i, h->om_i, h->os_i);
        MLP_CK(cudaGetLastError());
        h->infer_fresh = true;
        if (launches) ++*launches;
    }
    if (T <= 0) return TPF_OK;
    InferArgs g{};
    bool maps = make_bf16_map(&g.map_w[0], h->Wi0, P0, H) && make_bf16_map(&g.map_w[L - 1], h->WiL, H, PL);
    for (int l = 1; l < L - 1 && maps; ++l) maps = make_bf16_map(&g.map_w[l], h->Wb[l], H, H);
    if (!maps) return TPF_ECUDA;
    for (int l = 0; l < L - 1; ++l) g.bias[l] = h->b[l];
    if (!make_f64_map(&g.map_s, S, 2 * (uint64_t)h->n, (uint64_t)T, 64, 32)) return TPF_ECUDA;
    g.xnorm = h->xn_i;
    g.bias_out = h->bi_out;
    g.out_mean = h->om_i;
    g.out_std = h->os_i;
    g.L = L;
    g.H = H;
    g.P0 = P0;
    g.PL = PL;
    g.n = h->n;
    g.lo2 = 0.7f * 0.7f;
    g.hi2 = 1.1f * 1.1f;
    g.v0_64 = v0_64 ? 1 : 0;
    g.guard = guard ? 1 : 0;
    g.v0_half = v0_half ? 1 : 0;
    g.pitch = pitch ? pitch : h->n;
    g.fallback = h->fallback;
    g.err = h->err;
    g.V0 = V0;
    g.T = T;
    g.tiles = (T + 127) / 128;
    tpf_status rs = launch_infer(g, st);
    if (rs == TPF_OK && launches) ++*launches;
    return rs;
}

}  // namespace
}  // namespace tpf

using namespace tpf;

extern "C" {

tpf_status tpf_mlp_create(int n_pq, int hidden, int n_hidden_layers, int max_batch, uint64_t seed, tpf_mlp **out) {
    if (!out) return TPF_EINVAL;
    *out = nullptr;
    if (n_pq < 1 || hidden < 1 || n_hidden_layers < 1 || n_hidden_layers > 16 || max_batch < 128 ||
        max_batch % 128 || 2 * n_pq > 65536 || hidden > 65536)
        return TPF_EINVAL;
    tpf_mlp *h = new (std::nothrow) tpf_mlp();
    if (!h) return TPF_ENOMEM;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return TPF_ECUDA;
    }
    h->n = n_pq;
    h->L = n_hidden_layers + 1;
    h->max_batch = max_batch;
    h->dim.push_back(2 * n_pq);
    for (int l = 0; l < n_hidden_layers; ++l) h->dim.push_back(hidden);
    h->dim.push_back(2 * n_pq);
    for (int d : h->dim) h->pad.push_back((int)round_up(d, 128));
    int maxpad = 0;
    for (int p : h->pad) maxpad = p > maxpad ? p : maxpad;
    const int L = h->L, B = max_batch;
    bool ok = true;
    h->W.resize(L); h->b.resize(L); h->mW.resize(L); h->vW.resize(L); h->mb.resize(L); h->vb.resize(L);
    h->gWT.resize(L); h->gb.resize(L); h->Wb.resize(L); h->WTb.resize(L); h->Z.resize(L); h->dZ.resize(L);
    h->dZT.resize(L); h->A.resize(L - 1); h->AT.resize(L - 1);
    for (int l = 0; l < L && ok; ++l) {
        const size_t wsz = (size_t)h->pad[l + 1] * h->pad[l];
        ok = dalloc(&h->W[l], wsz) && dalloc(&h->mW[l], wsz) && dalloc(&h->vW[l], wsz) && dalloc(&h->gWT[l], wsz) &&
             dalloc(&h->Wb[l], wsz) && dalloc(&h->WTb[l], wsz) && dalloc(&h->b[l], h->pad[l + 1]) &&
             dalloc(&h->mb[l], h->pad[l + 1]) && dalloc(&h->vb[l], h->pad[l + 1]) && dalloc(&h->gb[l], h->pad[l + 1]) &&
             dalloc(&h->Z[l], (size_t)B * h->pad[l + 1]) && dalloc(&h->dZ[l], (size_t)B * h->pad[l + 1]) &&
             dalloc(&h->dZT[l], (size_t)B * h->pad[l + 1]);
        if (ok && l < L - 1) ok = dalloc(&h->A[l], (size_t)B * h->pad[l + 1]) && dalloc(&h->AT[l], (size_t)B * h->pad[l + 1]);
    }
    ok = ok && dalloc(&h->in_mean, h->pad[0]) && dalloc(&h->in_std, h->pad[0]) && dalloc(&h->out_mean, h->pad[L]) &&
         dalloc(&h->out_std, h->pad[L]) && dalloc(&h->X0, (size_t)B * h->pad[0]) &&
         dalloc(&h->X0T, (size_t)B * h->pad[0]) && dalloc(&h->dA, (size_t)B * maxpad) &&
         dalloc(&h->target, (size_t)B * h->pad[L]) && dalloc(&h->loss, 1) && dalloc(&h->err, 1) &&
         dalloc(&h->fallback, 1);
    if (!ok) {
        free_mlp(h);
        delete h;
        return TPF_ENOMEM;
    }
    // Xavier-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)), zero biases; splitmix64.
    uint64_t state = seed;
    auto next_u01 = [&state]() {
        uint64_t z = (state += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < L && ok; ++l) {
        const int Po = h->pad[l + 1], Pi = h->pad[l], ro = h->dim[l + 1], ri = h->dim[l];
        const double a = std::sqrt(6.0 / (double)(ri + ro));
        std::vector<float> w((size_t)Po * Pi, 0.0f);
        for (int o = 0; o < ro; ++o)
            for (int k = 0; k < ri; ++k) w[(size_t)o * Pi + k] = (float)((2.0 * next_u01() - 1.0) * a);
        ok = cudaMemcpy(h->W[l], w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    }
    std::vector<float> ones((size_t)maxpad, 1.0f);
    ok = ok && cudaMemcpy(h->in_std, ones.data(), sizeof(float) * h->pad[0], cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(h->out_std, ones.data(), sizeof(float) * h->pad[L], cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok || publish(h, nullptr) != TPF_OK || cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        free_mlp(h);
        delete h;
        return TPF_ECUDA;
    }
    *out = h;
    return TPF_OK;
}

void tpf_mlp_destroy(tpf_mlp *h) {
    if (!h) return;
    tpf::DeviceScope dscope(h->device);
    free_mlp(h);
    delete h;
}

int64_t tpf_mlp_param_count(const tpf_mlp *h) {
    if (!h) return -1;
    int64_t c = 0;
    for (int l = 0; l < h->L; ++l) c += (int64_t)h->dim[l + 1] * h->dim[l] + h->dim[l + 1];
    return c;
}

// Copy parameters between the device masters and a flat host array: for each layer W [out][in]
// row-major, then b [out].
static tpf_status params_io(tpf_mlp *h, float *host, bool to_host, bool grads) {
    if (!h || !host) return TPF_EINVAL;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok || cudaDeviceSynchronize() != cudaSuccess) return TPF_ECUDA;
    size_t off = 0;
    for (int l = 0; l < h->L; ++l) {
        const int Po = h->pad[l + 1], Pi = h->pad[l], ro = h->dim[l + 1], ri = h->dim[l];
        std::vector<float> w((size_t)Po * Pi);
        if (to_host) {
            if (cudaMemcpy(w.data(), grads ? h->gWT[l] : h->W[l], sizeof(float) * w.size(), cudaMemcpyDeviceToHost) !=
                cudaSuccess)
                return TPF_ECUDA;
            for (int o = 0; o < ro; ++o)
                for (int k = 0; k < ri; ++k)
                    host[off + (size_t)o * ri + k] = grads ? w[(size_t)k * Po + o] : w[(size_t)o * Pi + k];
        } else {
            std::fill(w.begin(), w.end(), 0.0f);
            for (int o = 0; o < ro; ++o)
                for (int k = 0; k < ri; ++k) w[(size_t)o * Pi + k] = host[off + (size_t)o * ri + k];
            if (cudaMemcpy(h->W[l], w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice) != cudaSuccess)
                return TPF_ECUDA;
        }
        off += (size_t)ro * ri;
        std::vector<float> bb((size_t)Po, 0.0f);
        if (to_host) {
            if (cudaMemcpy(bb.data(), grads ? h->gb[l] : h->b[l], sizeof(float) * Po, cudaMemcpyDeviceToHost) !=
                cudaSuccess)
                return TPF_ECUDA;
            std::memcpy(host + off, bb.data(), sizeof(float) * ro);
        } else {
            std::memcpy(bb.data(), host + off, sizeof(float) * ro);
            if (cudaMemcpy(h->b[l], bb.data(), sizeof(float) * Po, cudaMemcpyHostToDevice) != cudaSuccess)
                return TPF_ECUDA;
        }
        off += ro;
    }
    if (!to_host) {
        tpf_status rs = publish(h, nullptr);
        if (rs != TPF_OK) return rs;
        if (cudaDeviceSynchronize() != cudaSuccess) return TPF_ECUDA;
    }
    return TPF_OK;
}

tpf_status tpf_mlp_get_params(tpf_mlp *h, float *host) { return params_io(h, host, true, false); }
tpf_status tpf_mlp_set_params(tpf_mlp *h, const float *host) { return params_io(h, const_cast<float *>(host), false, false); }

tpf_status tpf_mlp_fit_normalization(tpf_mlp *h, int64_t T, const void *S_dev, const void *V_dev, void *stream) {
    if (!h || T < 1 || !S_dev || !V_dev) return TPF_EINVAL;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    h->infer_fresh = false;
    k_norm_stats<<<4 * h->n, kThreads, 0, st>>>((const double2 *)S_dev, (const double2 *)V_dev, T, h->n, h->in_mean,
                                                h->in_std, h->out_mean, h->out_std);
    MLP_CK(cudaGetLastError());
    MLP_CK(cudaStreamSynchronize(st));
    return TPF_OK;
}

tpf_status tpf_mlp_get_normalization(tpf_mlp *h, float *in_mean, float *in_std, float *out_mean, float *out_std) {
    if (!h || !in_mean || !in_std || !out_mean || !out_std) return TPF_EINVAL;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    const size_t a = sizeof(float) * 2 * h->n;
    if (cudaMemcpy(in_mean, h->in_mean, a, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(in_std, h->in_std, a, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(out_mean, h->out_mean, a, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(out_std, h->out_std, a, cudaMemcpyDeviceToHost) != cudaSuccess)
        return TPF_ECUDA;
    return TPF_OK;
}

tpf_status tpf_mlp_gradients(tpf_mlp *h, int B, const void *S_dev, const void *V_dev, double *loss_out,
                             float *grads_host, void *stream) {
    if (!h || B < 128 || B % 128 || B > h->max_batch || !S_dev || !V_dev) return TPF_EINVAL;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    MLP_CK(cudaMemsetAsync(h->err, 0, sizeof(int), st));
    tpf_status rs = load_batch(h, B, S_dev, V_dev, B, 0, true, st);
    if (rs == TPF_OK) rs = forward(h, B, st, true);
    if (rs == TPF_OK) rs = backward(h, B, st);
    if (rs == TPF_OK) rs = check_err(h, st);
    if (rs != TPF_OK) return rs;
    if (loss_out) MLP_CK(cudaMemcpy(loss_out, h->loss, sizeof(double), cudaMemcpyDeviceToHost));
    if (grads_host) return params_io(h, grads_host, true, true);
    return TPF_OK;
}

tpf_status tpf_mlp_train_step(tpf_mlp *h, int B, const void *S_dev, const void *V_dev, double lr, double *loss_out,
                              void *stream) {
    if (!h || B < 128 || B % 128 || B > h->max_batch || !S_dev || !V_dev || !(lr > 0.0)) return TPF_EINVAL;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    MLP_CK(cudaMemsetAsync(h->err, 0, sizeof(int), st));
    tpf_status rs = load_batch(h, B, S_dev, V_dev, B, 0, true, st);
    if (rs == TPF_OK) rs = forward(h, B, st, true);
    if (rs == TPF_OK) rs = backward(h, B, st);
    if (rs != TPF_OK) return rs;
    const int64_t k = ++h->step;
    h->infer_fresh = false;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - (float)std::pow(0.9, (double)k), c2 = 1.0f - (float)std::pow(0.999, (double)k);
    for (int l = 0; l < h->L; ++l) {
        const int Po = h->pad[l + 1], Pi = h->pad[l];
        k_adam<<<blocks((int64_t)Po * Pi), kThreads, 0, st>>>(h->W[l], h->gWT[l], h->mW[l], h->vW[l], h->b[l], h->gb[l],
                                                              h->mb[l], h->vb[l], h->Wb[l], h->WTb[l], Po, Pi,
                                                              h->dim[l + 1], h->dim[l], (float)lr, b1, b2, eps, c1, c2,
                                                              1);
    }
    MLP_CK(cudaGetLastError());
    if (loss_out) {
        MLP_CK(cudaMemcpyAsync(loss_out, h->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        return check_err(h, st);
    }
    return TPF_OK;
}

tpf_status tpf_mlp_predict(tpf_mlp *h, int64_t T, const void *S_dev, void *V0_dev, int64_t *fallback_out,
                           void *stream) {
    if (!h || T < 0) return TPF_EINVAL;
    if (T == 0) {
        if (fallback_out) *fallback_out = 0;
        return TPF_OK;
    }
    if (!S_dev || !V0_dev) return TPF_EINVAL;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    MLP_CK(cudaMemsetAsync(h->err, 0, sizeof(int), st));
    MLP_CK(cudaMemsetAsync(h->fallback, 0, sizeof(int), st));
    const int B = h->max_batch;
    if (fused_ok(h)) {
        tpf_status rs = infer_fused(h, T, S_dev, V0_dev, true, st);
        if (rs != TPF_OK) return rs;
        T = 0;  // done: skip the layer-by-layer path below
    }
    for (int64_t t0 = 0; t0 < T; t0 += B) {
        tpf_status rs = load_batch(h, B, S_dev, nullptr, T, t0, false, st);
        if (rs == TPF_OK) rs = forward(h, B, st, false);
        if (rs != TPF_OK) return rs;
        k_predict_out<<<(B * 32 + kThreads - 1) / kThreads, kThreads, 0, st>>>(
            h->Z[h->L - 1], B, h->pad[h->L], h->n, T, t0, h->out_mean, h->out_std, 0.7f, 1.1f, (double2 *)V0_dev,
            h->fallback);
        MLP_CK(cudaGetLastError());
    }
    int fb = 0;
    MLP_CK(cudaMemcpyAsync(&fb, h->fallback, sizeof(int), cudaMemcpyDeviceToHost, st));
    tpf_status rs = check_err(h, st);
    if (fallback_out) *fallback_out = fb;
    return rs;
}

tpf_status tpf_solve_learned(tpf_handle *hd, tpf_mlp *net, int64_t T, const void *S_dev, void *V_dev,
                             int32_t *iters_dev, double *mismatch_dev, const tpf_opts *opts, int64_t *fallback_out,
                             void *stream) {
    if (!hd || !net || T < 0) return TPF_EINVAL;
    tpf_opts o;
    tpf_default_opts(&o);
    if (opts) o = *opts;
    if (!(o.tol >= 0.0) || o.max_iter < 1 || o.max_iter > 100000 || !(o.switch_tol >= 0.0)) return TPF_EINVAL;
    if (o.method != TPF_METHOD_SPARSE || o.precision != TPF_PREC_MIXED) return TPF_EUNSUPPORTED;
    if (net->n != hd->net.n_pq || net->device != hd->device) return TPF_EINVAL;
    if (fallback_out) *fallback_out = 0;
    hd->stats = tpf_stats{};
    hd->stats.columns = T;
    if (T == 0) return TPF_OK;
    if (!S_dev || !V_dev) return TPF_EINVAL;
    if (!fused_ok(net)) return TPF_EUNSUPPORTED;
    tpf::DeviceScope dscope(hd->device);
    if (!dscope.ok) return TPF_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    // Prediction and solve in equal chunks of at most 1,048,576 columns: the predicted deviations
    // from the flat start (half2 per bus) of one chunk live in a buffer of the network, grown on
    // demand.
    constexpr int64_t kLearnedChunk = 1 << 20;
    const int64_t n_ch = (T + kLearnedChunk - 1) / kLearnedChunk;
    const int64_t chunk = std::min<int64_t>(T, round_up((T + n_ch - 1) / n_ch, 128));
    const int64_t cap = round_up(chunk, 128);
    const int n = net->n;
    // Columns of the prediction buffer start on 64-byte boundaries: a warp's 32 consecutive
    // half-precision outputs of one column then fill two whole 32-byte sectors.
    const int64_t pitch = round_up(n, 16);
    if (net->v0_cap < cap * pitch) {
        cudaFree(net->V0c);
        net->V0c = nullptr;
        net->v0_cap = 0;
        if (!dalloc(&net->V0c, (size_t)(cap * pitch))) return TPF_ENOMEM;
        net->v0_cap = cap * pitch;
    }
    MLP_CK(cudaMemsetAsync(net->err, 0, sizeof(int), st));
    MLP_CK(cudaMemsetAsync(net->fallback, 0, sizeof(int), st));
    tpf_stats total{};
    tpf_status result = TPF_OK;
    int64_t fallback = 0;
    for (int64_t c0 = 0; c0 < T; c0 += chunk) {
        const int64_t Tc = std::min(chunk, T - c0);
        const double2 *Sc = static_cast<const double2 *>(S_dev) + (size_t)c0 * n;
        int64_t predict_launches = 0;
        tpf_status rs = infer_fused(net, Tc, Sc, net->V0c, false, st, false, pitch, &predict_launches, true);
        if (rs != TPF_OK) return rs;
        rs = tpf::solve_sparse_ex(hd, Tc, Sc, static_cast<double2 *>(V_dev) + (size_t)c0 * n,
                                  iters_dev ? iters_dev + c0 : nullptr, mismatch_dev ? mismatch_dev + c0 : nullptr,
                                  nullptr, o, st, net->V0c, pitch);
        if (rs != TPF_OK && rs != TPF_ENOCONV) return rs;
        if (rs == TPF_ENOCONV) result = TPF_ENOCONV;
        fallback += hd->start_fallback;
        const tpf_stats &p = hd->stats;
        total.sweeps = std::max(total.sweeps, p.sweeps);
        total.precise_sweeps = std::max(total.precise_sweeps, p.precise_sweeps);
        total.converged += p.converged;
        total.kernel_launches += p.kernel_launches + predict_launches;
        total.residual_ms += p.residual_ms;
    }
    const tpf_status rs = check_err(net, st);
    total.columns = T;
    hd->stats = total;
    if (fallback_out) *fallback_out = fallback;
    return rs != TPF_OK ? rs : result;
}

}  // extern "C"
