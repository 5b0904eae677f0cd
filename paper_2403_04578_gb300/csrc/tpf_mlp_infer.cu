// Fused inference of the learned warm start: every layer of the network for a tile of 128
// columns in one persistent tcgen05 kernel, the hidden activations kept in shared memory.
//
// The network maps a column's loads to a starting voltage (features P_j, Q_j z-scored; targets
// Re V_i - 1, Im V_i z-scored; hidden layers z = W a + b, a = gelu(z)).  For inference the input
// features and the outputs are taken in interleaved order (P_1, Q_1, P_2, Q_2, ... and
// Re V_1 - 1, Im V_1, ...), so that a tile of features is a contiguous run of buses and an
// output tile is a contiguous run of complex voltages; the first and last weight matrices are
// permuted to match once per change of the parameters.
//
// Per CTA tile (M = 128 columns):
//   layer 0       D = X W_0^T        A = X (written from S by the converter warps), B = W_0 (TMA), K = P0
//   layers 1..    D = H W_l^T        A = H (shared memory), B = W_l (TMA), K = hidden
//   last layer    D = W_L H^T        in M tiles of 128 outputs, A = rows of W_L (TMA), B = H
// with the FP32 accumulator in TMEM (two stages of 256 columns).  The last layer is taken
// transposed (outputs on the TMEM lanes, the tile's columns along TMEM), so that a warp's 32
// threads hold 32 consecutive outputs of one column and its stores to V_0 are contiguous.  Warp 0
// issues the TMA loads of the weights into a 3-slot ring, warp 1 the MMAs (one thread); 8 converter
// warps read the loads S of the tile's columns straight from the complex128 tensor, z-score them
// and write the layer-0 operand (BF16, the 128-byte swizzled layout TMA would have written) into
// a 3-slot ring of their own, so that the feature matrix never exists in memory (each ring has its
// own full / empty barriers: a parity wait is exact only for a waiter that takes part in every
// phase of its barrier); 8 warps run the epilogues:
// bias and GELU (tanh form, half precision) of a hidden layer written as BF16 into the
// shared-memory operand of the next layer
// (128-byte swizzle, the layout TMA would have written), and for the last layer the
// denormalisation into V_0 with the |V| guard.  Every wait is bounded; on expiry the CTA flags the
// error, drains its own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "tpf_gemm.h"
#include "tpf_mlp_infer.h"
#include "tpf_tc.cuh"

namespace tpf {

namespace {

using namespace tc;

constexpr int kEpiGroups = 2;  // epilogue warps per TMEM lane quarter
constexpr int kEpiThreads = 128 * kEpiGroups;
constexpr int kConvWarps = 8;  // feature converters: 16 rows of each layer-0 chunk per warp
constexpr int kConvRows = 128 / kConvWarps;
constexpr int kEpiWarp0 = 2 + kConvWarps;
constexpr int kThreads = 64 + 32 * kConvWarps + kEpiThreads;  // TMA, MMA, converters, epilogues
constexpr int kStages = 3;
constexpr uint32_t kATile = 128 * 64 * 2;  // 16 KB: 128 rows x 64 BF16 (one K chunk of A)
constexpr uint32_t kBMax = 256 * 64 * 2;   // 32 KB: up to 256 rows x 64 BF16 (one K chunk of B)
constexpr uint32_t kStageBytes = kBMax;    // weight ring slot: a K chunk of W_0 or W_l, or 128 rows of W_L
constexpr uint32_t kHBytes = 128 * 256 * 2;  // hidden activations of the tile, 4 K chunks of 16 KB
constexpr uint32_t kBiasBytes = (kMaxInferLayers - 1) * 256 * 4;  // hidden biases, staged once
constexpr size_t kSmem = 1024 + kStages * (kStageBytes + kATile) + kHBytes + 1024 + kBiasBytes;
constexpr int kOutTile = 128;  // outputs per last-layer accumulator job

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// GELU of a pair of pre-activations for the next layer's BF16 operand, in packed half precision
// with its tanh form, 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))): one tanh.approx.f16x2 and
// a few f16x2 FMAs per pair.  The tanh form differs from the erf form z Phi(z) (which training
// uses) by at most about 3e-4, and the half-precision evaluation by about 1e-3 relative, both
// below the BF16 rounding (2^-9 relative) of the activation they produce.
__device__ __forceinline__ uint32_t gelu_pair_bf16(float z0, float z1) {
    const __half2 z = __floats2half2_rn(z0, z1);
    const __half2 k0 = __float2half2_rn(0.7978845608f), k1 = __float2half2_rn(0.0356774081f);  // sqrt(2/pi), *0.044715
    const __half2 half = __float2half2_rn(0.5f);
    const __half2 u = __hmul2(z, __hfma2(__hmul2(z, z), k1, k0));
    __half2 t;
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(*reinterpret_cast<uint32_t *>(&t)) : "r"(*reinterpret_cast<const uint32_t *>(&u)));
    const __half2 hz = __hmul2(half, z);
    const float2 g = __half22float2(__hfma2(hz, t, hz));
    return pack_bf16(g.x, g.y);
}

// FP64 -> FP32 from the high word alone (sign, 11-bit exponent rebiased from 1023 to 127, the
// top 20 mantissa bits; truncated), by the IEEE-754 field layout: plain integer arithmetic instead
// of the FP64 pipe, exact enough for a feature rounded to BF16 (8 mantissa bits).  Magnitudes below
// FP32's normal range flush to zero, those above it (and NaN) become infinity.
__device__ __forceinline__ float f64_hi_to_f32(uint32_t hi) {
    const uint32_t mag = min(hi & 0x7fffffffu, 0x47f00000u);
    const uint32_t f = mag >= 0x38100000u ? (mag - 0x38000000u) << 3 : 0u;
    return __uint_as_float(f | (hi & 0x80000000u));
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }


__global__ void __launch_bounds__(kThreads, 1) mlp_infer(const __grid_constant__ InferArgs g) {
    extern __shared__ uint8_t smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *Xs = smem + kStages * kStageBytes;  // [kStages] layer-0 A tiles written by the converters
    uint8_t *Hs = Xs + kStages * kATile;
    uint64_t *full = (uint64_t *)(Hs + kHBytes);  // [kStages] TMA -> MMA
    uint64_t *empty = full + kStages;              // [kStages] MMA -> TMA
    uint64_t *tfull = empty + kStages;             // [2] MMA -> epilogue
    uint64_t *tempty = tfull + 2;                  // [2] epilogue -> MMA
    uint64_t *hready = tempty + 2;                 // [1] epilogue -> MMA: the activations are written
    uint64_t *done = hready + 1;                   // [1] every MMA of this CTA retired
    uint64_t *xfull = done + 1;                    // [kStages] converters -> MMA: a layer-0 A tile is written
    uint64_t *xempty = xfull + kStages;            // [kStages] MMA -> converters
    uint32_t *tmem_slot = (uint32_t *)(xempty + kStages);
    int *abort_flag = (int *)(tmem_slot + 1);
    float *s_bias = (float *)(Hs + kHBytes + 1024);  // [L-1][H] biases of the hidden layers
    __shared__ int s_fail;
    __shared__ unsigned s_badm[4];  // bit c: column c of the tile left the guard band somewhere

    const int L = g.L, H = g.H;
    const int k0 = g.P0 / 64, kh = H / 64, n_out = g.PL / kOutTile;
    constexpr uint32_t kTmemCols = 512;
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
            mbar_init(smem_u32(&xfull[s]), kConvWarps);  // lane 0 of each converter warp
            mbar_init(smem_u32(&xempty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&tfull[a]), 1);
            mbar_init(smem_u32(&tempty[a]), kEpiThreads / 32);  // lane 0 of each epilogue warp
        }
        mbar_init(smem_u32(hready), 1);
        mbar_init(smem_u32(done), 1);
        *abort_flag = 0;
        s_fail = 0;
        for (int c = 0; c < 4; ++c) s_badm[c] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int k = tid; k < (L - 1) * H; k += blockDim.x) s_bias[k] = __ldg(g.bias[k / H] + k % H);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    volatile int *vabort = abort_flag;

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer: the operand chunks of every job, in job order ----------------
        const uint32_t sbase = smem_u32(smem);
        int64_t q = 0;  // chunks issued by this CTA
        auto slot_ready = [&](uint32_t &st) -> bool {
            const int slot = (int)(q % kStages);
            if (!mbar_wait(smem_u32(&empty[slot]), ((uint32_t)(q / kStages) & 1) ^ 1)) {
                *vabort = 1;
                atomicExch(g.err, 1);
                return false;
            }
            st = sbase + slot * kStageBytes;
            return true;
        };
        for (int64_t tile = blockIdx.x; tile < g.tiles && !*vabort; tile += gridDim.x) {
            bool ok = true;
            for (int c = 0; c < k0 && ok; ++c, ++q) {  // layer 0: W_0 (the converters write X)
                uint32_t st;
                if (!(ok = slot_ready(st))) break;
                const uint32_t bar = smem_u32(&full[q % kStages]);
                mbar_expect_tx(bar, (uint32_t)H * 128);
                for (int r = 0; r < H / 128; ++r) tma_load_2d(st + r * 16384, &g.map_w[0], bar, c * 64, r * 128);
            }
            for (int l = 1; l < L - 1 && ok; ++l)  // hidden layers: W_l
                for (int c = 0; c < kh && ok; ++c, ++q) {
                    uint32_t st;
                    if (!(ok = slot_ready(st))) break;
                    const uint32_t bar = smem_u32(&full[q % kStages]);
                    mbar_expect_tx(bar, (uint32_t)H * 128);
                    for (int r = 0; r < H / 128; ++r)
                        tma_load_2d(st + r * 16384, &g.map_w[l], bar, c * 64, r * 128);
                }
            for (int nt = 0; nt < n_out && ok; ++nt)  // last layer: 128 output rows of W_L at a time
                for (int c = 0; c < kh && ok; ++c, ++q) {
                    uint32_t st;
                    if (!(ok = slot_ready(st))) break;
                    const uint32_t bar = smem_u32(&full[q % kStages]);
                    mbar_expect_tx(bar, 16384);
                    tma_load_2d(st, &g.map_w[L - 1], bar, c * 64, nt * kOutTile);
                }
            if (!ok) break;
        }
        if (*vabort) {  // the copies in flight land before the CTA leaves (bounded)
            for (int64_t r = q - 1; r >= 0 && r >= q - kStages; --r)
                mbar_wait(smem_u32(&full[r % kStages]), (uint32_t)(r / kStages) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t sbase = smem_u32(smem), xbase = smem_u32(Xs), hbase = smem_u32(Hs);
        const uint32_t id_hidden = idesc_f16(128, H, 0, 1), id_out = idesc_f16(128, kOutTile, 0, 1);
        int64_t q = 0;   // chunks consumed
        uint32_t jq = 0; // accumulator jobs
        uint32_t hq = 0; // activation tiles waited for
        uint32_t xq = 0; // layer-0 A tiles consumed
        bool ok = true;
        // One accumulator job: wait for the stage, optionally for fresh activations, then n_k chunks.
        // from_h: A = the activations, B = the ring's weights; out: A = the ring's weights, B = the
        // activations (the transposed last layer); otherwise layer 0: A = the converters' features.
        auto job = [&](int n_k, bool from_h, bool wait_h, uint32_t idesc, bool out = false) -> bool {
            const uint32_t a = jq & 1, u = jq >> 1;
            if (!mbar_wait(smem_u32(&tempty[a]), (u & 1) ^ 1)) return false;
            if (wait_h) {
                if (!mbar_wait(smem_u32(hready), hq & 1)) return false;
                ++hq;
            }
            tc_fence_after();
            const uint32_t acc = tmem + a * 256;
            for (int c = 0; c < n_k; ++c, ++q) {
                const int slot = (int)(q % kStages);
                if (!mbar_wait(smem_u32(&full[slot]), (uint32_t)(q / kStages) & 1)) return false;
                const bool x_in = !from_h && !out;
                const uint32_t xslot = xq % kStages;
                if (x_in && !mbar_wait(smem_u32(&xfull[xslot]), (xq / kStages) & 1)) return false;
                tc_fence_after();
                const uint32_t st = sbase + slot * kStageBytes;
                const uint32_t abase = out ? st : (from_h ? hbase + c * kATile : xbase + xslot * kATile);
                const uint32_t bbase = out ? hbase + c * kATile : st;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma_f16(acc, sw128_desc(abase + kk * 32), sw128_desc(bbase + kk * 32), idesc, (c | kk) != 0);
                umma_commit(smem_u32(&empty[slot]));
                if (x_in) {
                    umma_commit(smem_u32(&xempty[xslot]));
                    ++xq;
                }
            }
            umma_commit(smem_u32(&tfull[a]));
            ++jq;
            return true;
        };
        for (int64_t tile = blockIdx.x; tile < g.tiles && ok && !*vabort; tile += gridDim.x) {
            ok = job(k0, false, false, id_hidden);
            for (int l = 1; l < L - 1 && ok; ++l) ok = job(kh, true, true, id_hidden);
            for (int nt = 0; nt < n_out && ok; ++nt) ok = job(kh, false, nt == 0, id_out, true);
        }
        if (!ok) {
            *vabort = 1;
            atomicExch(g.err, 1);
        }
        umma_commit(smem_u32(done));
        mbar_wait(smem_u32(done), 0);  // every MMA of this CTA has retired (bounded)
    } else if (warp >= 2 && warp < kEpiWarp0) {
        // ---------------- feature converters ----------------
        // Layer-0 chunk c of a tile is features 64 c .. 64 c + 63 = buses 32 c .. 32 c + 31, (P, Q)
        // interleaved.  Lane l takes bus 32 c + l; warp w rows (columns t) 16 w .. 16 w + 15, one
        // coalesced 512-byte load of S per row.  The chunk's loads go out in two halves of 8 rows,
        // each half of the next chunk issued as soon as this chunk's half is converted, so that
        // one to two halves per warp stay in flight.
        const int cw = warp - 2;
        const int64_t my_tiles = g.tiles > blockIdx.x ? (g.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
        const int64_t steps = my_tiles * k0;
        const uint8_t *Sb = reinterpret_cast<const uint8_t *>(g.S);
        auto load_half = [&](uint4 (&v)[8], int64_t s, int half) {
            const int64_t tile = blockIdx.x + (s / k0) * gridDim.x;
            const int j = (int)(s % k0) * 32 + lane;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t t = tile * 128 + cw * kConvRows + half * 8 + i;
                v[i] = (j < g.n && t < g.T) ? __ldg(reinterpret_cast<const uint4 *>(Sb + (t * g.n + j) * 16))
                                            : make_uint4(0u, 0u, 0u, 0u);
            }
        };
        auto store_half = [&](const uint4 (&v)[8], uint8_t *a, float4 nm, int half) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int r = cw * kConvRows + half * 8 + i;
                const float xr = fmaf(f64_hi_to_f32(v[i].y), nm.x, nm.y);
                const float xi = fmaf(f64_hi_to_f32(v[i].w), nm.z, nm.w);
                *reinterpret_cast<uint32_t *>(a + (r >> 3) * 1024 + (r & 7) * 128 + (((lane >> 2) ^ (r & 7)) << 4) +
                                              ((lane & 3) << 2)) = pack_bf16(xr, xi);
            }
        };
        uint4 va[8], vb[8];
        if (steps > 0) {
            load_half(va, 0, 0);
            load_half(vb, 0, 1);
        }
        for (int64_t s = 0; s < steps; ++s) {  // s: this A tile's place in the converters' ring
            const int c = (int)(s % k0);
            const int slot = (int)(s % kStages);
            const int j = c * 32 + lane;
            const float4 nm = j < g.n ? __ldg(g.xnorm + j) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (*vabort || !mbar_wait(smem_u32(&xempty[slot]), ((uint32_t)(s / kStages) & 1) ^ 1)) {
                *vabort = 1;
                atomicExch(g.err, 1);
                break;
            }
            uint8_t *a = Xs + slot * kATile;
            store_half(va, a, nm, 0);
            if (s + 1 < steps) load_half(va, s + 1, 0);
            store_half(vb, a, nm, 1);
            if (s + 1 < steps) load_half(vb, s + 1, 1);
            fence_async_smem();  // the MMAs (async proxy) read this tile next
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&xfull[slot]));
        }
    } else if (warp >= kEpiWarp0) {
        // ---------------- epilogue: kEpiGroups warps per TMEM lane quarter ----------------
        // Hidden layers: thread = column row of the tile, `part` splits the units.  Last layer:
        // thread = output row of the accumulator, `part` splits the tile's columns.
        const int quarter = warp & 3;  // TMEM lanes this warp may access
        const int part = (warp - kEpiWarp0) >> 2;
        const int row = quarter * 32 + lane;
        const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
        const int et = tid - 32 * kEpiWarp0;
        // This row's 128-byte line inside each 16 KB K chunk of the activations (SW128 layout).
        uint8_t *hrow = Hs + (row >> 3) * 1024 + (row & 7) * 128;
        const int hp = H / 32 / kEpiGroups;  // pieces of 32 units per part
        uint32_t jq = 0;
        for (int64_t tile = blockIdx.x; tile < g.tiles; tile += gridDim.x) {
            const int64_t t = tile * 128 + row;  // this thread's column (hidden layers)
            bool failed = false;
            const int jobs = L - 1 + n_out;
            for (int j = 0; j < jobs; ++j, ++jq) {
                const uint32_t a = jq & 1, u = jq >> 1;
                if (!mbar_wait(smem_u32(&tfull[a]), u & 1)) atomicOr(&s_fail, 1);
                epi_sync();
                if (s_fail) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + a * 256 + lane_off;
                if (j < L - 1) {
                    // Hidden activations of layer j: bias, GELU, BF16 into the next layer's A operand.
                    const float *bias = s_bias + j * H;
                    for (int p = part * hp; p < (part + 1) * hp; ++p) {
                        uint32_t v[32];
                        tmem_ld32(acc + p * 32, v);
                        tmem_wait_ld();
                        uint32_t w[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const float2 b2 = *reinterpret_cast<const float2 *>(bias + p * 32 + 2 * e);
                            w[e] = gelu_pair_bf16(__uint_as_float(v[2 * e]) + b2.x,
                                                  __uint_as_float(v[2 * e + 1]) + b2.y);
                        }
                        // Units p*32 .. p*32+31: K chunk p/2, 16-byte groups 4 (p&1) .. +3, swizzled by row.
                        uint8_t *chunk = hrow + (p >> 1) * kATile;
#pragma unroll
                        for (int gq = 0; gq < 4; ++gq) {
                            const int grp = ((p & 1) * 4 + gq) ^ (row & 7);
                            *reinterpret_cast<uint4 *>(chunk + grp * 16) =
                                make_uint4(w[4 * gq], w[4 * gq + 1], w[4 * gq + 2], w[4 * gq + 3]);
                        }
                    }
                    fence_async_smem();  // the MMAs (async proxy) read these activations next
                    tc_fence_before();
                    epi_sync();
                    if (et == 0) mbar_arrive(smem_u32(hready));
                } else {
                    // Transposed last layer: this thread's lane is output o = 128 nt + row (interleaved:
                    // bus o / 2, Re V - 1 for even o, Im V for odd o), the accumulator columns are the
                    // tile's 128 columns.  The even and odd lanes of a pair see both parts of a bus.
                    const int o = (j - (L - 1)) * kOutTile + row, i = o >> 1;
                    // value = (d + b) s + m (+ 1 for Re V) = d s + c
                    const float so = __ldg(g.out_std + o);
                    const float cd = __ldg(g.bias_out + o) * so + __ldg(g.out_mean + o);  // deviation: Re V - 1, Im V
                    const float co = cd + ((o & 1) ? 0.0f : 1.0f);
                    const int64_t stride = 2 * g.pitch;  // floats (or doubles) per column of V0
                    for (int p = part * (4 / kEpiGroups); p < (part + 1) * (4 / kEpiGroups); ++p) {
                        uint32_t v[32];
                        tmem_ld32(acc + p * 32, v);
                        tmem_wait_ld();
                        const int64_t c0 = tile * 128 + p * 32;  // first column of this piece
                        const int valid = i < g.n ? (int)min((int64_t)32, g.T - c0) : 0;
                        if (g.v0_half) {
                            // The deviation from the flat start in half precision (the reader adds 1
                            // to the real part and checks the |V| band).
                            __half *dst = static_cast<__half *>(g.V0) + c0 * stride + o;
                            if (valid == 32) {
#pragma unroll
                                for (int e = 0; e < 32; ++e)
                                    dst[e * stride] = __float2half_rn(fmaf(__uint_as_float(v[e]), so, cd));
                            } else {
#pragma unroll
                                for (int e = 0; e < 32; ++e)
                                    if (e < valid) dst[e * stride] = __float2half_rn(fmaf(__uint_as_float(v[e]), so, cd));
                            }
                            continue;
                        }
                        float val[32];
#pragma unroll
                        for (int e = 0; e < 32; ++e) val[e] = fmaf(__uint_as_float(v[e]), so, co);
                        if (g.guard) {
                            uint32_t bad = 0;  // bit e: column c0 + e left the guard band at this bus
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                const float other = __shfl_xor_sync(0xffffffffu, val[e], 1);
                                const float m2 = fmaf(val[e], val[e], other * other);
                                bad |= (m2 >= g.lo2 && m2 <= g.hi2) ? 0u : (1u << e);
                            }
                            bad &= valid >= 32 ? 0xffffffffu : (valid <= 0 ? 0u : (1u << valid) - 1u);
                            bad = __reduce_or_sync(0xffffffffu, bad);
                            if (lane == 0 && bad) atomicOr(&s_badm[p], bad);
                        }
                        if (g.v0_64) {
                            double *dst = static_cast<double *>(g.V0) + c0 * stride + o;
                            if (valid == 32) {
#pragma unroll
                                for (int e = 0; e < 32; ++e) dst[e * stride] = (double)val[e];
                            } else {
#pragma unroll
                                for (int e = 0; e < 32; ++e)
                                    if (e < valid) dst[e * stride] = (double)val[e];
                            }
                        } else {
                            float *dst = static_cast<float *>(g.V0) + c0 * stride + o;
                            if (valid == 32) {
#pragma unroll
                                for (int e = 0; e < 32; ++e) dst[e * stride] = val[e];
                            } else {
#pragma unroll
                                for (int e = 0; e < 32; ++e)
                                    if (e < valid) dst[e * stride] = val[e];
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[a]));
            }
            if (failed) {
                *vabort = 1;
                atomicExch(g.err, 1);
                break;
            }
            epi_sync();  // every output of the tile has been checked
            const bool bad = (s_badm[row >> 5] >> (row & 31)) & 1u;
            epi_sync();  // every thread has read its bit
            if (et < 4) s_badm[et] = 0;  // (set again only after the next tile's first job barrier)
            if (part == 0) {
                if (t < g.T && bad) {  // outside the guard band: the flat start for this column
                    for (int i = 0; i < g.n; ++i) {
                        const int64_t k = t * g.pitch + i;
                        if (g.v0_64)
                            static_cast<double2 *>(g.V0)[k] = make_double2(1.0, 0.0);
                        else
                            static_cast<float2 *>(g.V0)[k] = make_float2(1.0f, 0.0f);
                    }
                    atomicAdd(g.fallback, 1);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace

bool infer_supported(int L, int H, int P0, int PL) {
    return L >= 2 && L <= kMaxInferLayers && (H == 128 || H == 256) && P0 % 128 == 0 && PL % kOutTile == 0;
}

tpf_status launch_infer(const InferArgs &g, cudaStream_t st) {
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem) != cudaSuccess) {
            cudaGetLastError();
            return TPF_ECUDA;
        }
        attr = true;
    }
    if (g.tiles <= 0) return TPF_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    const unsigned grid = (unsigned)(g.tiles < sms ? g.tiles : sms);
    mlp_infer<<<grid, kThreads, kSmem, st>>>(g);
    if (cudaGetLastError() != cudaSuccess) return TPF_ECUDA;
    return TPF_OK;
}

}  // namespace tpf
