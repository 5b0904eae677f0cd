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
//   layer 0       D = X W_0^T        A = X (converted from S on chip), B = W_0 (TMA), K = P0
//   layers 1..    D = H W_l^T        A = H (shared memory), B = W_l (TMA), K = hidden
//   last layer    D = W_L H^T        in M tiles of 128 outputs, A = rows of W_L (TMA), B = H
// with FP32 accumulators in TMEM: layer 0 in columns 0..255, the hidden layers in 256..511, the
// last layer's jobs in alternating halves of 256..511.  The last layer is taken transposed
// (outputs on the TMEM lanes, the tile's columns along TMEM), so that a warp's 32 threads hold 32
// consecutive outputs of one column and its stores to V_0 are contiguous.
//
// Warps: 0 issues the TMA loads of the weights into a ring of 16 KB slots (128 rows x 64 BF16;
// a 256-row operand takes two slots and two N = 128 MMAs); 1 issues the MMAs (one thread); 2
// issues the TMA loads of the loads S themselves (complex128 read as FP64 pairs, boxes of 32
// columns x 32 buses) into a staging ring; 3-10 convert the staged loads into the layer-0 operand
// (z-scored, BF16, in the 128-byte swizzled layout TMA would have written) in a ring of their own,
// so that no feature matrix exists in memory; 11-18 run the epilogues: bias and GELU (tanh form,
// half precision) of a hidden layer written as BF16 into the shared-memory operand of the next
// layer, and for the last layer the denormalisation into V_0 with the |V| guard.  The next
// tile's layer-0 chunks are issued between this tile's hidden and output jobs, so that reading S
// overlaps the output epilogue.  Each ring has its own full / empty barriers (a parity wait is
// exact only for a waiter that takes part in every phase of its barrier).  Every wait is bounded;
// on expiry the CTA flags the error, drains its own copies and MMAs, frees TMEM and returns.
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
constexpr int kConvWarps = 8;                      // feature converters
constexpr int kSRows = 32;                         // columns (rows of S) per staged box
constexpr int kConvRows = kSRows / kConvWarps;     // rows of a box per converter warp
constexpr int kBoxes = 128 / kSRows;               // staged boxes per layer-0 chunk
constexpr int kConvWarp0 = 3;
constexpr int kEpiWarp0 = kConvWarp0 + kConvWarps;
constexpr int kThreads = 32 * kEpiWarp0 + kEpiThreads;  // TMA W, MMA, TMA S, converters, epilogues
constexpr int kWSlots = 4;                         // weight ring: 16 KB slots
constexpr int kXSlots = 2;                         // layer-0 operand ring: 16 KB slots
constexpr int kSSlots = 4;                         // staged S: 16 KB slots
constexpr uint32_t kSlot = 128 * 64 * 2;           // 16 KB: 128 rows x 64 BF16 (one K chunk of 128 rows)
constexpr uint32_t kSBox = kSRows * 32 * 16;       // 16 KB: 32 columns x 32 complex128 loads
constexpr uint32_t kHBytes = 128 * 256 * 2;        // hidden activations of the tile, 4 K chunks of 16 KB
constexpr size_t kSmem = 1024 + (kWSlots + kXSlots) * kSlot + kSSlots * kSBox + kHBytes + 1024;
constexpr int kOutTile = 128;  // outputs per last-layer accumulator job
static_assert(kSmem <= 232448, "shared memory");

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

// The next tile's layer-0 chunks that go after job jj of this tile's J jobs: spread evenly over
// the jobs, the last one after the last job.
__device__ __forceinline__ int l0_target(int jj, int J, int k0) {
    return jj + 1 >= J ? k0 : min(k0 - 1, (jj + 1) * k0 / J);
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads) : "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__global__ void __launch_bounds__(kThreads, 1) mlp_infer(const __grid_constant__ InferArgs g) {
    extern __shared__ uint8_t smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *Ws = smem;                    // [kWSlots] weight boxes (TMA)
    uint8_t *Xs = Ws + kWSlots * kSlot;    // [kXSlots] layer-0 A tiles (converters)
    uint8_t *Ss = Xs + kXSlots * kSlot;    // [kSSlots] staged boxes of S (TMA)
    uint8_t *Hs = Ss + kSSlots * kSBox;    // activations of the tile
    uint64_t *wfull = (uint64_t *)(Hs + kHBytes);  // [kWSlots] TMA -> MMA
    uint64_t *wempty = wfull + kWSlots;            // [kWSlots] MMA -> TMA
    uint64_t *xfull = wempty + kWSlots;            // [kXSlots] converters -> MMA
    uint64_t *xempty = xfull + kXSlots;            // [kXSlots] MMA -> converters
    uint64_t *sfull = xempty + kXSlots;            // [kSSlots] TMA -> converters
    uint64_t *sempty = sfull + kSSlots;            // [kSSlots] converters -> TMA
    // Accumulators in TMEM: columns 0..255 take layer 0 (region 1); columns 256..511 (region 2)
    // take the hidden layers (both halves) and the last layer's jobs (alternating halves of 128).
    uint64_t *tfull1 = sempty + kSSlots;           // [1] MMA -> epilogue: layer 0 accumulated
    uint64_t *tempty1 = tfull1 + 1;                // [1] epilogue -> MMA: region 1 read
    uint64_t *tfull2 = tempty1 + 1;                // [2] per half of region 2
    uint64_t *tempty2 = tfull2 + 2;                // [2]
    uint64_t *hready = tempty2 + 2;                // [1] epilogue -> MMA: the activations are written
    uint64_t *done = hready + 1;                   // [1] every MMA of this CTA retired
    uint32_t *tmem_slot = (uint32_t *)(done + 1);
    int *abort_flag = (int *)(tmem_slot + 1);
    __shared__ int s_fail;
    __shared__ unsigned s_badm[4];  // bit c: column c of the tile left the guard band somewhere

    const int L = g.L, H = g.H;
    const int k0 = g.P0 / 64, kh = H / 64, n_out = g.PL / kOutTile, hr = H / 128;
    constexpr uint32_t kTmemCols = 512;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < kWSlots; ++s) {
            mbar_init(smem_u32(&wfull[s]), 1);
            mbar_init(smem_u32(&wempty[s]), 1);
        }
        for (int s = 0; s < kXSlots; ++s) {
            mbar_init(smem_u32(&xfull[s]), kConvWarps);  // lane 0 of each converter warp
            mbar_init(smem_u32(&xempty[s]), 1);
        }
        for (int s = 0; s < kSSlots; ++s) {
            mbar_init(smem_u32(&sfull[s]), 1);
            mbar_init(smem_u32(&sempty[s]), kConvWarps);
        }
        mbar_init(smem_u32(tfull1), 1);
        mbar_init(smem_u32(tempty1), kEpiThreads / 32);  // lane 0 of each epilogue warp
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&tfull2[a]), 1);
            mbar_init(smem_u32(&tempty2[a]), kEpiThreads / 32);
        }
        mbar_init(smem_u32(hready), 1);
        mbar_init(smem_u32(done), 1);
        *abort_flag = 0;
        s_fail = 0;
        for (int c = 0; c < 4; ++c) s_badm[c] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    volatile int *vabort = abort_flag;
    // This CTA's tiles, and the jobs of one tile after its layer 0: the hidden layers, then the
    // last layer's output tiles.
    const int64_t my_tiles = g.tiles > blockIdx.x ? (g.tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int J = (L - 2) + n_out;
    auto fail = [&]() {
        *vabort = 1;
        atomicExch(g.err, 1);
    };

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer of the weights, in the MMA's order ----------------
        // One 16 KB box per ring slot: 128 rows x one K chunk of 64.
        const uint32_t wbase = smem_u32(Ws);
        int64_t q = 0;  // boxes issued by this CTA
        auto box = [&](const CUtensorMap *map, int x, int y) -> bool {
            const int slot = (int)(q % kWSlots);
            if (!mbar_wait(smem_u32(&wempty[slot]), ((uint32_t)(q / kWSlots) & 1) ^ 1)) {
                fail();
                return false;
            }
            const uint32_t bar = smem_u32(&wfull[slot]);
            mbar_expect_tx(bar, kSlot);
            tma_load_2d(wbase + slot * kSlot, map, bar, x, y);
            ++q;
            return true;
        };
        auto w0_chunk = [&](int c) -> bool {  // layer 0: K chunk c of W_0, H / 128 boxes
            for (int r = 0; r < hr; ++r)
                if (!box(&g.map_w[0], c * 64, r * 128)) return false;
            return true;
        };
        auto job_chunks = [&](int jj) -> bool {
            for (int c = 0; c < kh; ++c) {
                if (jj < L - 2) {  // hidden layer jj + 1: K chunk c of W_l
                    for (int r = 0; r < hr; ++r)
                        if (!box(&g.map_w[jj + 1], c * 64, r * 128)) return false;
                } else if (!box(&g.map_w[L - 1], c * 64, (jj - (L - 2)) * kOutTile)) {  // 128 rows of W_L
                    return false;
                }
            }
            return true;
        };
        bool ok = true;
        for (int c = 0; c < k0 && ok && my_tiles > 0; ++c) ok = w0_chunk(c);
        for (int64_t it = 0; it < my_tiles && ok && !*vabort; ++it) {
            const bool next = it + 1 < my_tiles;
            int cn = 0;  // the next tile's layer-0 chunks issued so far
            for (int jj = 0; jj < J && ok; ++jj) {
                ok = job_chunks(jj);
                for (const int tgt = next ? l0_target(jj, J, k0) : 0; cn < tgt && ok; ++cn) ok = w0_chunk(cn);
            }
        }
        if (*vabort) {  // the copies in flight land before the CTA leaves (bounded)
            for (int64_t r = q - 1; r >= 0 && r >= q - kWSlots; --r)
                mbar_wait(smem_u32(&wfull[r % kWSlots]), (uint32_t)(r / kWSlots) & 1);
        }
    } else if (warp == 2 && lane == 0) {
        // ---------------- TMA producer of the loads S ----------------
        // Per tile and layer-0 chunk c: kBoxes boxes of 32 columns x 32 buses (64 FP64 values:
        // P, Q of buses 32 c .. 32 c + 31); buses beyond n and columns beyond T read as zero.
        const uint32_t sbase = smem_u32(Ss);
        int64_t k = 0;  // boxes issued
        bool ok = true;
        for (int64_t it = 0; it < my_tiles && ok && !*vabort; ++it) {
            const int64_t tile = blockIdx.x + it * gridDim.x;
            for (int c = 0; c < k0 && ok; ++c)
                for (int b = 0; b < kBoxes; ++b, ++k) {
                    const int slot = (int)(k % kSSlots);
                    if (!mbar_wait(smem_u32(&sempty[slot]), ((uint32_t)(k / kSSlots) & 1) ^ 1)) {
                        fail();
                        ok = false;
                        break;
                    }
                    const uint32_t bar = smem_u32(&sfull[slot]);
                    mbar_expect_tx(bar, kSBox);
                    tma_load_2d(sbase + slot * kSBox, &g.map_s, bar, c * 64, (int)(tile * 128 + b * kSRows));
                }
        }
        if (*vabort) {
            for (int64_t r = k - 1; r >= 0 && r >= k - kSSlots; --r)
                mbar_wait(smem_u32(&sfull[r % kSSlots]), (uint32_t)(r / kSSlots) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        // Per tile: layer 0 into region 1 (A = the converters' features), the hidden layers into
        // region 2 (A = the activations), the last layer's output tiles into the halves of region 2
        // (A = rows of W_L, B = the activations); a 256-unit layer is two N = 128 halves, one
        // weight box each.  The next tile's layer-0 chunks are interleaved between this tile's
        // jobs (l0_target), the last of them after the last output job, so that layer 0's
        // completion also retires every MMA that reads this tile's activations.
        const uint32_t wbase = smem_u32(Ws), xbase = smem_u32(Xs), hbase = smem_u32(Hs);
        const uint32_t id128 = idesc_f16(128, 128, 0, 1);
        int64_t q = 0;              // weight boxes consumed
        uint32_t xq = 0;            // layer-0 A tiles consumed
        uint32_t hq = 0;            // activation tiles waited for
        uint32_t u1 = 0;            // uses of region 1
        uint32_t u20 = 0, u21 = 0;  // uses of the halves of region 2
        uint32_t jo = 0;            // output jobs
        auto next_w = [&](uint32_t &st) -> bool {
            const int slot = (int)(q % kWSlots);
            if (!mbar_wait(smem_u32(&wfull[slot]), (uint32_t)(q / kWSlots) & 1)) return false;
            tc_fence_after();
            st = wbase + slot * kSlot;
            return true;
        };
        auto release_w = [&]() {
            umma_commit(smem_u32(&wempty[q % kWSlots]));
            ++q;
        };
        auto mma4 = [&](uint32_t acc, uint32_t a, uint32_t b, bool accumulate) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                umma_f16(acc, sw128_desc(a + kk * 32), sw128_desc(b + kk * 32), id128, accumulate || kk != 0);
        };
        auto l0_chunk = [&](int c) -> bool {
            if (c == 0 && !mbar_wait(smem_u32(tempty1), (u1 & 1) ^ 1)) return false;
            const uint32_t xslot = xq % kXSlots;
            if (!mbar_wait(smem_u32(&xfull[xslot]), (xq / kXSlots) & 1)) return false;
            tc_fence_after();
            for (int r = 0; r < hr; ++r) {
                uint32_t st;
                if (!next_w(st)) return false;
                mma4(tmem + r * 128, xbase + xslot * kSlot, st, c != 0);
                release_w();
            }
            umma_commit(smem_u32(&xempty[xslot]));
            ++xq;
            if (c == k0 - 1) {
                umma_commit(smem_u32(tfull1));
                ++u1;
            }
            return true;
        };
        auto job = [&](int jj) -> bool {
            const bool hidden = jj < L - 2;
            const uint32_t h = jo & 1, uh = h ? u21 : u20;
            if (hidden) {
                if (!mbar_wait(smem_u32(&tempty2[0]), (u20 & 1) ^ 1) || !mbar_wait(smem_u32(&tempty2[1]), (u21 & 1) ^ 1))
                    return false;
            } else if (!mbar_wait(smem_u32(&tempty2[h]), (uh & 1) ^ 1)) {
                return false;
            }
            if (hidden || jj == L - 2) {  // the activations this job reads are written
                if (!mbar_wait(smem_u32(hready), hq & 1)) return false;
                ++hq;
            }
            tc_fence_after();
            for (int c = 0; c < kh; ++c) {
                if (hidden) {
                    for (int r = 0; r < hr; ++r) {
                        uint32_t st;
                        if (!next_w(st)) return false;
                        mma4(tmem + 256 + r * 128, hbase + c * kSlot, st, c != 0);
                        release_w();
                    }
                } else {
                    uint32_t st;
                    if (!next_w(st)) return false;
                    mma4(tmem + 256 + h * kOutTile, st, hbase + c * kSlot, c != 0);
                    release_w();
                }
            }
            if (hidden) {
                umma_commit(smem_u32(&tfull2[0]));
                umma_commit(smem_u32(&tfull2[1]));
                ++u20;
                ++u21;
            } else {
                umma_commit(smem_u32(&tfull2[h]));
                if (h) ++u21; else ++u20;
                ++jo;
            }
            return true;
        };
        bool ok = true;
        for (int c = 0; c < k0 && ok && my_tiles > 0; ++c) ok = l0_chunk(c);
        for (int64_t it = 0; it < my_tiles && ok && !*vabort; ++it) {
            const bool next = it + 1 < my_tiles;
            int cn = 0;
            for (int jj = 0; jj < J && ok; ++jj) {
                ok = job(jj);
                for (const int tgt = next ? l0_target(jj, J, k0) : 0; cn < tgt && ok; ++cn) ok = l0_chunk(cn);
            }
        }
        if (!ok) fail();
        umma_commit(smem_u32(done));
        mbar_wait(smem_u32(done), 0);  // every MMA of this CTA has retired (bounded)
    } else if (warp >= kConvWarp0 && warp < kEpiWarp0) {
        // ---------------- feature converters ----------------
        // Layer-0 chunk c of a tile is features 64 c .. 64 c + 63 = buses 32 c .. 32 c + 31, (P, Q)
        // interleaved.  Lane l takes bus 32 c + l; warp w rows 4 w .. 4 w + 3 of each staged box
        // (one 16-byte shared-memory read per row, 512 contiguous bytes per warp), converted from
        // the FP64 high words and written as one BF16 pair into the swizzled A tile.
        const int cw = warp - kConvWarp0;
        const int64_t steps = my_tiles * k0;
        int64_t k = 0;  // staged boxes consumed
        for (int64_t s = 0; s < steps; ++s) {
            const int xslot = (int)(s % kXSlots);
            const int j = (int)(s % k0) * 32 + lane;
            const float4 nm = j < g.n ? __ldg(g.xnorm + j) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (*vabort || !mbar_wait(smem_u32(&xempty[xslot]), ((uint32_t)(s / kXSlots) & 1) ^ 1)) {
                fail();
                break;
            }
            uint8_t *a = Xs + xslot * kSlot;
            bool ok = true;
            for (int b = 0; b < kBoxes; ++b, ++k) {
                const int sslot = (int)(k % kSSlots);
                if (!mbar_wait(smem_u32(&sfull[sslot]), (uint32_t)(k / kSSlots) & 1)) {
                    ok = false;
                    break;
                }
                const uint8_t *src = Ss + sslot * kSBox;
#pragma unroll
                for (int i = 0; i < kConvRows; ++i) {
                    const int rl = cw * kConvRows + i, r = b * kSRows + rl;
                    const uint4 v = *reinterpret_cast<const uint4 *>(src + rl * 512 + lane * 16);
                    const float xr = fmaf(f64_hi_to_f32(v.y), nm.x, nm.y);
                    const float xi = fmaf(f64_hi_to_f32(v.w), nm.z, nm.w);
                    *reinterpret_cast<uint32_t *>(a + (r >> 3) * 1024 + (r & 7) * 128 + (((lane >> 2) ^ (r & 7)) << 4) +
                                                  ((lane & 3) << 2)) = pack_bf16(xr, xi);
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&sempty[sslot]));
            }
            if (!ok) {
                fail();
                break;
            }
            fence_async_smem();  // the MMAs (async proxy) read this tile next
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&xfull[xslot]));
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
        uint32_t e1 = 0, e20 = 0, e21 = 0, eo = 0;  // uses of region 1, of the halves of region 2; output jobs
        for (int64_t tile = blockIdx.x; tile < g.tiles; tile += gridDim.x) {
            const int64_t t = tile * 128 + row;  // this thread's column (hidden layers)
            bool failed = false;
            const int jobs = L - 1 + n_out;
            for (int j = 0; j < jobs; ++j) {
                // Job j: layer 0 (region 1), hidden layer j (region 2), or output tile j - (L - 1)
                // (half eo & 1 of region 2).
                const uint32_t h = eo & 1, eh = h ? e21 : e20;
                bool got;
                if (j == 0)
                    got = mbar_wait(smem_u32(tfull1), e1 & 1);
                else if (j < L - 1)
                    got = mbar_wait(smem_u32(&tfull2[0]), e20 & 1) && mbar_wait(smem_u32(&tfull2[1]), e21 & 1);
                else
                    got = mbar_wait(smem_u32(&tfull2[h]), eh & 1);
                if (!got) atomicOr(&s_fail, 1);
                epi_sync();
                if (s_fail) {
                    failed = true;
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (j == 0 ? 0u : 256u + (j < L - 1 ? 0u : h * kOutTile)) + lane_off;
                if (j < L - 1) {
                    // Hidden activations of layer j: bias, GELU, BF16 into the next layer's A operand.
                    const float *bias = g.bias[j];
                    for (int p = part * hp; p < (part + 1) * hp; ++p) {
                        uint32_t v[32];
                        tmem_ld32(acc + p * 32, v);
                        tmem_wait_ld();
                        uint32_t w[16];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const float2 b2 = __ldg(reinterpret_cast<const float2 *>(bias + p * 32 + 2 * e));
                            w[e] = gelu_pair_bf16(__uint_as_float(v[2 * e]) + b2.x,
                                                  __uint_as_float(v[2 * e + 1]) + b2.y);
                        }
                        // Units p*32 .. p*32+31: K chunk p/2, 16-byte groups 4 (p&1) .. +3, swizzled by row.
                        uint8_t *chunk = hrow + (p >> 1) * kSlot;
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
                if (j == 0) {
                    if (lane == 0) mbar_arrive(smem_u32(tempty1));
                    ++e1;
                } else if (j < L - 1) {
                    if (lane == 0) {
                        mbar_arrive(smem_u32(&tempty2[0]));
                        mbar_arrive(smem_u32(&tempty2[1]));
                    }
                    ++e20;
                    ++e21;
                } else {
                    if (lane == 0) mbar_arrive(smem_u32(&tempty2[h]));
                    if (h) ++e21; else ++e20;
                    ++eo;
                }
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
    static std::atomic<uint64_t> attr{0};
    if (!once_per_device(attr, [] {
            return cudaFuncSetAttribute(mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem) == cudaSuccess;
        }))
        return TPF_ECUDA;
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
