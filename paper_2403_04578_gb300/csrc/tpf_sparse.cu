// Sparse tensor formulation (Sec. IV-B, Eq. 13-14, Algorithm 2) on radial feeders.
//
// Algorithm 2 replaces the dense product with K = -Y_dd^{-1} by a sparse solve with Y_dd, factored
// once; the sequence of iterates is the one of the dense form.  On a radial feeder Y_dd factors
// without fill-in and the solve is a substitution over the tree.  Expanding the fixed-point step
// V_{k+1} = K conj(S ./ V_k) + W that way gives, for every demand bus c with parent p(c) and
// branch impedance z_c (V_slack = v_s),
//
//     L_c      = sum over the subtree of c of I_i,   I_i = conj(S_i / V_i)      (leaves -> slack)
//     V_new_c  = V_new_p(c) - z_c L_c  =  v_s - sum over the path slack..c of z_b L_b   (slack -> leaves)
//
// Both passes become prefix sums once the buses are numbered in depth-first preorder: the subtree
// of the bus at position q is the position range [q, end_q), so L_q = P[end_q - 1] - P[q - 1]
// with P the inclusive prefix sum of I; and the path sum at q is the prefix sum at q of E, where
// E_q = x_q minus the x_b of every b whose range ends at q (x_b = z_b L_b).  A sweep is then two
// block-wide scans and no level-by-level walk.
//
// Precision follows the mixed dense path: far from convergence the sweep runs in FP32 on V
// itself.  Once the step is small the column is anchored at V_ref = fl32(V): the first step from
// V_ref, D = BFS(V_ref) - V_ref, is computed once in double-float, and every later sweep only
// carries FP32 corrections:  delta_new = D - sum over the path of z_b dL_b, with dL the subtree
// sums of conj(S ./ (V_ref + delta)) - conj(S ./ V_ref), which are small near the solution.
// The iterate is V_ref + delta; results reach the FP64 solution.
//
// One block owns one column for its whole solve.  Each thread owns kBPT consecutive depth-first
// positions and keeps their V_ref, delta and ends-list bounds in registers; shared memory holds S
// and z, the prefix-sum arrays, D and the tree's range / parent / ends-index arrays, all indexed
// by slot (j * threads + k for the j-th position of thread k) so that a warp's accesses to its own
// positions fall in consecutive banks.  Device memory is read for S once (again at a second
// anchor) and written once for V.  Feeders of 4,097 to 6,144 demand buses take 16 positions per
// thread and keep D, S and z in a device scratch slice per block instead (see mx_tree).
#include <algorithm>
#include <cstdlib>
#include <limits>
#include <new>
#include <tuple>
#include <vector>

#include "tpf_dd.cuh"

namespace tpf {

namespace {

constexpr int kMaxThreads = kTreeMaxThreads;  // so at most 8 * 512 = 4096 demand buses
constexpr int kMaxWarps = kMaxThreads / 32;
constexpr unsigned kFull = 0xffffffffu;
constexpr int kGather = 4;  // ends-list entries per position gathered without a loop

// One feeder's share of a launch: its network arrays (slot layout) and its tensors.
struct TreeWork {
    int n, n_ends;
    float2 vs_f;
    c2 vs_dd;
    const int *col, *end, *par, *ecnt, *ends, *kidx;
    const float4 *z;
    const float4 *zip_hi, *zip_lo;  // ZIP coefficients (alpha_P, alpha_I, alpha_Z, 0) per slot, or null
    // Polyphase: positions per phase block, v_s per phase, per slot the rows of the branch's
    // impedance (double-float) and admittance blocks, [slot][phase].
    int nbp;
    float2 vs_fp[3];
    c2 vs_ddp[3];
    const float4 *zrow;
    const float2 *yrow;
    const float2 *zrow_f;  // FP32 impedance rows for the sweeps, read through the cache
    const void *S;       // complex128 or, with s32, complex64 [T][n]
    const void *V0;      // given start, same type as V_out
    void *V_out;         // complex128 or, with v32, complex64 [T][n]; may be null
    int32_t *iters_out;  // [T] or null
    double *mismatch_out;  // [T] or null
    int s32, v32;
    int v0_pred;         // V0 is the learned start's prediction, half2 deviations (Re V - 1, Im V)
                         // per bus (V_out complex128): a column with some |V_i| outside
                         // [0.7, 1.1] starts flat instead
    int64_t v0_pitch;    // complex values per column of that prediction
    int64_t col0;        // first launch column of this feeder
    int64_t T;
    int *conv;           // converged columns of this feeder (accumulated)
    // Voltage-band statistics (each may be null): per column min / max |V| and the number of buses
    // outside [v_min, v_max]; per bus the number of columns below / above the band.
    float *col_vmin, *col_vmax;
    int32_t *col_viol, *bus_under, *bus_over;
    float v_min2, v_max2;
};

struct TreeArgs {
    const TreeWork *works;  // n_works entries, sorted by col0; null: the single feeder `one`
    TreeWork one;
    int n_works;
    int max_iter;
    int given;  // V_0 is read from V0 (a given or warm start)
    int blind;  // ... and anchored at once, its low words kept (a given start)
    float tol2, switch_tol, switch_tol2;  // squared tolerances compare with squared steps
    int *counters;                        // [5] largest per-column sweep count, [6] largest anchor count
    // Large-feeder kernel (16 buses per thread): per block (launch column), (kZip ? 3 : 2) * ns
    // float4 of device scratch for D, (S_hi, z) and the ZIP coefficients.
    float4 *scratch;
};

// Packed per-position word: ends-list start (bits 0-15), count (16-29), phase (30-31).
__device__ __forceinline__ int ends_cnt(int ec) { return (int)(((unsigned)ec >> 16) & 0x3fffu); }
__device__ __forceinline__ int phase_of(int ec) { return (int)((unsigned)ec >> 30); }

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// The FP32 products below are written with explicitly rounded intrinsics, so that the compiler
// cannot contract them differently in different instantiations of the kernel: every kernel then
// rounds a given formula the same way, whatever code surrounds it (ZIP loads with alpha_P = 1 then
// round their currents exactly as constant power does).
__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
    return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float abs2(float2 a) { return __fmaf_rn(a.x, a.x, __fmul_rn(a.y, a.y)); }
// max(a, b) that returns NaN if either is NaN (fmaxf returns the other operand).
__device__ __forceinline__ float fmax_nan(float a, float b) {
    float r;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}
// Maximum over the 32 lanes of a warp, returned to every lane, in one warp-wide reduction
// (redux.sync on FP32, sm_100 family): the NaN-propagating form, and the form that ignores NaN.
__device__ __forceinline__ float warp_max_nan(float v) {
    float r;
    asm volatile("redux.sync.max.NaN.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float warp_max(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float4 pack(c2 v) { return make_float4(v.re.h, v.re.l, v.im.h, v.im.l); }
__device__ __forceinline__ c2 unpack(float4 v) { return {{v.x, v.y}, {v.z, v.w}}; }

// conj(s / v) in FP32 with the hardware reciprocal (sweeps: their rounding is far below what the
// FP32 phase resolves, and the anchored corrections are small differences).
__device__ __forceinline__ float2 current_fast(float2 v, float2 s) {
    const float inv = __fdividef(1.0f, abs2(v));
    return make_float2(__fmul_rn(__fmaf_rn(s.x, v.x, __fmul_rn(s.y, v.y)), inv),
                       __fmul_rn(__fmaf_rn(s.x, v.y, -__fmul_rn(s.y, v.x)), inv));
}
// conj(s / (v + d)) - conj(s / v) = -conj(s d / ((v + d) v)), FP32 with the hardware reciprocal.
__device__ __forceinline__ float2 delta_current_fast(float2 v, float2 d, float2 s) {
    const float2 w = cmul2(s, d);
    const float2 q = cmul2(add2(v, d), v);
    const float inv = __fdividef(1.0f, abs2(q));
    return make_float2(-__fmul_rn(__fmaf_rn(w.x, q.x, __fmul_rn(w.y, q.y)), inv),
                       __fmul_rn(__fmaf_rn(w.y, q.x, -__fmul_rn(w.x, q.y)), inv));
}

// Demand current of Eq. 3 with ZIP loads, i_d = alpha_P conj(s / v) + alpha_I conj(s) +
// alpha_Z conj(s) v, and its change when v moves from v to v + d (the constant-current part
// cancels, the constant-impedance part is linear).  al = (alpha_P, alpha_I, alpha_Z, -).
template <bool kZip>
__device__ __forceinline__ float2 demand_current(float2 v, float2 s, float4 al) {
    const float2 c = current_fast(v, s);
    if (!kZip) return c;
    const float2 cs_v = cmul2(make_float2(s.x, -s.y), v);  // conj(s) v
    return make_float2(__fmaf_rn(al.x, c.x, __fmaf_rn(al.y, s.x, __fmul_rn(al.z, cs_v.x))),
                       __fmaf_rn(al.x, c.y, __fmaf_rn(-al.y, s.y, __fmul_rn(al.z, cs_v.y))));
}
template <bool kZip>
__device__ __forceinline__ float2 demand_change(float2 v, float2 d, float2 s, float4 al) {
    const float2 c = delta_current_fast(v, d, s);
    if (!kZip) return c;
    const float2 cs_d = cmul2(make_float2(s.x, -s.y), d);  // conj(s) d
    return make_float2(__fmaf_rn(al.x, c.x, __fmul_rn(al.z, cs_d.x)), __fmaf_rn(al.x, c.y, __fmul_rn(al.z, cs_d.y)));
}

// Sum of the warp totals of the warps before `warp`: lane l holds the total of warp l (lanes past
// the block's nw warps are zero), a shuffle scan over the lanes, then the entry of lane warp - 1.
__device__ __forceinline__ float2 warps_before(float2 t, int lane, int warp, int nw) {
    if (lane >= nw) t = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int o = 1; o < nw; o <<= 1) {
        const float ux = __shfl_up_sync(kFull, t.x, o), uy = __shfl_up_sync(kFull, t.y, o);
        if (lane >= o) t = add2(make_float2(ux, uy), t);
    }
    const float px = __shfl_sync(kFull, t.x, warp ? warp - 1 : 0), py = __shfl_sync(kFull, t.y, warp ? warp - 1 : 0);
    return warp ? make_float2(px, py) : make_float2(0.0f, 0.0f);
}

// Exclusive scan over the threads of the block (thread order) of one complex FP32 value.
__device__ __forceinline__ float2 block_scan(float2 v, float2 *wt, int lane, int warp, int nw) {
    float2 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float ux = __shfl_up_sync(kFull, inc.x, o), uy = __shfl_up_sync(kFull, inc.y, o);
        if (lane >= o) inc = add2(make_float2(ux, uy), inc);
    }
    // The lane's exclusive value as its inclusive value minus its own (one rounding, one shuffle
    // fewer than taking the neighbour's inclusive value).
    const float2 off = lane ? make_float2(inc.x - v.x, inc.y - v.y) : make_float2(0.0f, 0.0f);
    if (lane == 31) wt[warp] = inc;
    __syncthreads();
    return add2(warps_before(wt[lane < kMaxWarps ? lane : 0], lane, warp, nw), off);
}

// Double-float arithmetic of the anchor.  Each result carries an absolute error of a few units
// of 2^-44 times the larger operand, which is what the anchor needs (D to about 1e-13 pu against
// terms of order 0.1 pu); the products are exact in their high parts through FMA.
__device__ __forceinline__ f2 qadd(f2 a, f2 b) {
    const f2 s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ f2 qneg(f2 a) { return {-a.h, -a.l}; }
// The sum without the final renormalisation: the high part is the rounded sum of the high parts,
// the low part collects their exact rounding error and the low parts.  Inside a scan, where a
// handful of such sums follow one another, the low part stays within a few ulp of the high part;
// cqnorm restores |l| <= ulp(h) / 2 at the end.
__device__ __forceinline__ f2 qadd_lazy(f2 a, f2 b) {
    const f2 s = two_sum(a.h, b.h);
    return {s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l))};
}
__device__ __forceinline__ c2 cqadd_lazy(c2 a, c2 b) { return {qadd_lazy(a.re, b.re), qadd_lazy(a.im, b.im)}; }
__device__ __forceinline__ c2 cqnorm(c2 a) { return {fast_two_sum(a.re.h, a.re.l), fast_two_sum(a.im.h, a.im.l)}; }
__device__ __forceinline__ c2 cqadd(c2 a, c2 b) { return {qadd(a.re, b.re), qadd(a.im, b.im)}; }
__device__ __forceinline__ c2 cqsub(c2 a, c2 b) { return {qadd(a.re, qneg(b.re)), qadd(a.im, qneg(b.im))}; }
// a * b, both double-float complex.
__device__ __forceinline__ c2 cqmul(c2 a, c2 b) {
    const float p = __fmul_rn(a.re.h, b.re.h), pe = __fmaf_rn(a.re.h, b.re.h, -p);
    const float q = __fmul_rn(a.im.h, b.im.h), qe = __fmaf_rn(a.im.h, b.im.h, -q);
    const f2 sr = two_sum(p, -q);
    const float lr = (pe - qe) + (a.re.h * b.re.l + a.re.l * b.re.h) - (a.im.h * b.im.l + a.im.l * b.im.h);
    const float u = __fmul_rn(a.re.h, b.im.h), ue = __fmaf_rn(a.re.h, b.im.h, -u);
    const float v = __fmul_rn(a.im.h, b.re.h), ve = __fmaf_rn(a.im.h, b.re.h, -v);
    const f2 si = two_sum(u, v);
    const float li = (ue + ve) + (a.re.h * b.im.l + a.re.l * b.im.h) + (a.im.h * b.re.l + a.im.l * b.re.h);
    return {fast_two_sum(sr.h, __fadd_rn(sr.l, lr)), fast_two_sum(si.h, __fadd_rn(si.l, li))};
}
// conj(S / V) for a double-float S and an FP32 V: w_h = S / V in FP32, then the residual
// r = S - w_h V from exact products and w_l = r / V, so that w_h + w_l carries S / V to about
// 2^-44 relative.
__device__ __forceinline__ c2 current_q(c2 S, float2 V) {
    const float inv = __fdividef(1.0f, V.x * V.x + V.y * V.y);
    const float2 wh = make_float2((S.re.h * V.x + S.im.h * V.y) * inv, (S.im.h * V.x - S.re.h * V.y) * inv);
    // r.re = S.re - (wh.x V.x - wh.y V.y)
    const float a1 = __fmul_rn(wh.x, V.x), a1e = __fmaf_rn(wh.x, V.x, -a1);
    const float a2 = __fmul_rn(wh.y, V.y), a2e = __fmaf_rn(wh.y, V.y, -a2);
    const f2 t = two_sum(S.re.h, -a1);
    const float rr = __fadd_rn(__fadd_rn(t.h, a2), __fadd_rn(t.l, __fadd_rn(S.re.l, __fsub_rn(a2e, a1e))));
    // r.im = S.im - (wh.x V.y + wh.y V.x)
    const float b1 = __fmul_rn(wh.x, V.y), b1e = __fmaf_rn(wh.x, V.y, -b1);
    const float b2 = __fmul_rn(wh.y, V.x), b2e = __fmaf_rn(wh.y, V.x, -b2);
    const f2 u = two_sum(S.im.h, -b2);
    const float ri = __fadd_rn(__fsub_rn(u.h, b1), __fadd_rn(u.l, __fsub_rn(S.im.l, __fadd_rn(b1e, b2e))));
    const float2 wl = make_float2((rr * V.x + ri * V.y) * inv, (ri * V.x - rr * V.y) * inv);
    return {fast_two_sum(wh.x, wl.x), fast_two_sum(-wh.y, -wl.y)};
}

// Exclusive block scan in double-float.
__device__ __forceinline__ c2 block_scan_dd(c2 v, float4 *wt, int lane, int warp, int nw) {
    c2 inc = v;
#pragma unroll 1
    for (int o = 1; o < 32; o <<= 1) {
        float4 u = pack(inc);
        u.x = __shfl_up_sync(kFull, u.x, o);
        u.y = __shfl_up_sync(kFull, u.y, o);
        u.z = __shfl_up_sync(kFull, u.z, o);
        u.w = __shfl_up_sync(kFull, u.w, o);
        if (lane >= o) inc = cqadd_lazy(unpack(u), inc);
    }
    inc = cqnorm(inc);
    float4 e = pack(inc);
    e.x = __shfl_up_sync(kFull, e.x, 1);
    e.y = __shfl_up_sync(kFull, e.y, 1);
    e.z = __shfl_up_sync(kFull, e.z, 1);
    e.w = __shfl_up_sync(kFull, e.w, 1);
    const c2 off = lane ? unpack(e) : c2{{0.0f, 0.0f}, {0.0f, 0.0f}};
    if (lane == 31) wt[warp] = pack(inc);
    __syncthreads();
    // Lane l scans the warp totals up to warp l; each warp takes lane warp - 1's sum.
    float4 tw = lane < nw ? wt[lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 1
    for (int o = 1; o < nw; o <<= 1) {
        float4 u;
        u.x = __shfl_up_sync(kFull, tw.x, o);
        u.y = __shfl_up_sync(kFull, tw.y, o);
        u.z = __shfl_up_sync(kFull, tw.z, o);
        u.w = __shfl_up_sync(kFull, tw.w, o);
        if (lane >= o) tw = pack(cqadd_lazy(unpack(u), unpack(tw)));
    }
    tw = pack(cqnorm(unpack(tw)));
    const int src = warp ? warp - 1 : 0;
    tw.x = __shfl_sync(kFull, tw.x, src);
    tw.y = __shfl_sync(kFull, tw.y, src);
    tw.z = __shfl_sync(kFull, tw.z, src);
    tw.w = __shfl_sync(kFull, tw.w, src);
    return warp ? cqadd(unpack(tw), off) : off;
}

// Slot of depth-first position p for blocks of th threads with kBPT positions each.
template <int kBPT>
__device__ __forceinline__ int slot_of(int p, int th) {
    return (p & (kBPT - 1)) * th + p / kBPT;
}
// Slot of the position after the one in slot s.
template <int kBPT>
__device__ __forceinline__ int next_slot(int s, int th) {
    return s < (kBPT - 1) * th ? s + th : s - (kBPT - 1) * th + 1;
}

// First part of an anchor, in double-float.  On entry A[s] = (S_hi) and B[s] = (V_ref, S_lo) for
// the thread's own slots.  Leaves in B the inclusive prefix sums of the path terms and returns the
// thread's exclusive scan offset.  ecnt holds the thread's ends-list bounds, s_rk the subtree
// ranges (as in the kernel).
// The loops run over shared memory only and are not unrolled: the anchor runs once or twice per
// column and its code stays small; the unrolled staging in the kernel keeps the device-memory
// loads in flight together.
template <int kBPT, bool kZip, int kPh>
__device__ __forceinline__ c2 anchor_dd(const TreeWork &a, float4 *A, float4 *B, const int *s_rk,
                                        const float4 *Zs, const int *ecnt, float4 *wtd,
                                        int tid, int th, int lane, int warp) {
    const int n = a.n, base = tid * kBPT;
    // Load currents at V_ref and their inclusive prefix sums.
    c2 run = {{0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll 1
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        if (q < n) {
            const float4 sh = A[s], v = B[s];
            const c2 Sd = {{sh.x, v.z}, {sh.y, v.w}};
            c2 I = current_q(Sd, make_float2(v.x, v.y));
            if (kZip) {
                // alpha_P conj(s / v) + alpha_I conj(s) + alpha_Z conj(s) v with double-float alphas
                const float4 ah = Zs[s], al = a.zip_lo[s];
                const c2 cs = {Sd.re, qneg(Sd.im)};
                I = cqadd(cqadd(cqmul(c2{{ah.x, al.x}, {0.0f, 0.0f}}, I), cqmul(c2{{ah.y, al.y}, {0.0f, 0.0f}}, cs)),
                          cqmul(c2{{ah.z, al.z}, {0.0f, 0.0f}}, cqmul(cs, c2{{v.x, 0.0f}, {v.y, 0.0f}})));
            }
            run = cqadd(run, I);
            A[s] = pack(run);
        }
    }
    c2 off = block_scan_dd(run, wtd, lane, warp, th >> 5);
#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const int s = j * th + tid;
        A[s] = pack(cqadd(off, unpack(A[s])));
        if (kPh == 1) B[s] = a.z[s];  // (re_hi, im_hi, re_lo, im_lo)
    }
    __syncthreads();
    // Branch terms x_q = z_q (P[end_q - 1] - P[q - 1]); polyphase: x = sum over phases p' of
    // Z[p][p'] L_{p'}, the subtree sums of the same buses in the other phase blocks.
#pragma unroll 1
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        if (q < n) {
            if (kPh == 1) {
                c2 L = unpack(A[s_rk[s] & 0xffff]);
                if (q > 0) L = cqsub(L, unpack(A[j ? s - th : (kBPT - 1) * th + tid - 1]));
                const float4 zq = B[s];
                B[s] = pack(cqmul(c2{{zq.x, zq.z}, {zq.y, zq.w}}, L));
            } else {
                const int p = q / a.nbp, qb = q - p * a.nbp, eb = (s_rk[s] & 0xffff) - p * a.nbp;
                c2 x = {{0.0f, 0.0f}, {0.0f, 0.0f}};
                for (int pp = 0; pp < kPh; ++pp) {
                    c2 L = unpack(A[slot_of<kBPT>(pp * a.nbp + eb - 1, th)]);
                    const int prev = pp * a.nbp + qb - 1;
                    if (prev >= 0) L = cqsub(L, unpack(A[slot_of<kBPT>(prev, th)]));
                    const float4 zq = a.zrow[(size_t)s * kPh + pp];
                    x = cqadd(x, cqmul(c2{{zq.x, zq.z}, {zq.y, zq.w}}, L));
                }
                B[s] = pack(x);
            }
        }
    }
    __syncthreads();
    // The branch terms in ends-list order (A is free now), so that each position's list is
    // contiguous.
#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const int s = j * th + tid, k = s_rk[s] >> 16;
        if (k >= 0) A[k] = B[s];
    }
    __syncthreads();
    // Inclusive prefix sums of E_q = x_q - (x_b of every b whose range ends at q), into B.
    run = c2{{0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll 1
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        if (q < n) {
            int ec = ecnt[0];  // ecnt[j] by selects: the array stays in registers
#pragma unroll
            for (int i = 1; i < kBPT; ++i)
                if (j == i) ec = ecnt[i];
            const int st = ec & 0xffff, cnt = ends_cnt(ec);
            c2 e = unpack(B[s]);
#pragma unroll 1
            for (int k = 0; k < cnt; ++k) e = cqsub(e, unpack(A[st + k]));
            run = cqadd(run, e);
            B[s] = pack(run);
        }
    }
    return block_scan_dd(run, wtd, lane, warp, th >> 5);
}

// kTh > 0 fixes the block size at compile time (it must equal blockDim.x): the slot arithmetic
// and the scans then run on constants.  kTh = 0 takes it from blockDim.x.
//
// kBPT == 16 is the large-feeder kernel (4,097 to 6,144 demand buses): the prefix array and the tree
// indices stay in shared memory, D, (S_hi, z) and the ZIP coefficients go to the block's slice of
// device scratch (through the cache), and the block has up to 384 threads of 168 registers.
template <int kBPT, bool kZip, int kPh, int kTh>
__global__ void __maxnreg__(kBPT == 16 ? 168 : (kBPT == 8 ? 128 : (kBPT == 4 && (kZip || kPh > 1) ? 80 : 64)))
    mx_tree(const __grid_constant__ TreeArgs g) {
    constexpr bool kBig = kBPT == 16;
    extern __shared__ float4 tsm[];
    __shared__ int s_work;
    const int th = kTh ? kTh : (int)blockDim.x, ns = th * kBPT;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = th >> 5;
    if (tid == 0) {
        // The feeder of this block's column: the last work whose first column is <= blockIdx.x.
        int lo = 0, hi = g.works ? g.n_works - 1 : 0;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (g.works[mid].col0 <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_work = lo;
    }
    __syncthreads();
    const TreeWork &a = g.works ? g.works[s_work] : g.one;
    const int n = a.n;
    // Arrays indexed by slot s = j th + k of position q = kBPT k + j.
    float4 *const A = tsm;       // [ns] double-float prefix sums (anchor); float2 P and X in the sweeps
    float4 *const big = kBig ? g.scratch + (size_t)blockIdx.x * (kZip ? 3 : 2) * ns : nullptr;
    float4 *const B = kBig ? big : tsm + ns;  // [ns] V_ref (anchor input), x (anchor), then D = BFS(V_ref) - V_ref
    float4 *const C = kBig ? big + ns : tsm + 2 * ns;  // [ns] (S_hi, z_hi) of each position
    float4 *const Zs = kBig ? big + 2 * ns : tsm + 3 * ns;  // [ns] ZIP coefficients (kZip only)
    // [ns] the subtree's range [q, end_q): one phase, the slot of its last position end_q - 1 (the
    // slot itself for a leaf); polyphase, end_q.  (The polyphase impedance rows stay in device
    // memory, read through the cache: in shared memory they would halve the resident blocks.)
    // [ns] per slot, bits 0-15: the subtree's range [q, end_q): one phase, the slot of its last
    // position end_q - 1 (the slot itself for a leaf); polyphase, end_q.  Bits 16-31: where the
    // position's branch term goes in the ends-ordered copy of X (-1: nowhere).  One word, so that a
    // sweep reads both with one shared-memory load.  (The polyphase impedance rows stay in device
    // memory, read through the cache: in shared memory they would halve the resident blocks.)
    int *const s_rk = reinterpret_cast<int *>(tsm + (kBig ? 1 : (kZip ? 4 : 3)) * ns);
    short *const s_par = reinterpret_cast<short *>(s_rk + ns);  // [ns] parent slot, -1 = the slack
    float2 *P = reinterpret_cast<float2 *>(A);  // [ns] inclusive prefix sums of the load currents
    float2 *X = P + ns;                           // [ns] branch terms z_q L_q; the residual's x at the end
    __shared__ float2 wt2[kMaxWarps];
    __shared__ float4 wtd[kMaxWarps];
    __shared__ float4 wtm[kMaxWarps];
    __shared__ float4 wm[kMaxWarps];
    const int64_t t = (int64_t)blockIdx.x - a.col0;  // column within the feeder
    const int base = tid * kBPT;
    // S and V of this column: complex128 (double2) or complex64 (float2).
    const double2 *S64 = static_cast<const double2 *>(a.S) + t * n;
    const float2 *S32 = static_cast<const float2 *>(a.S) + t * n;

#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        const int rng = kPh > 1 ? a.end[s] : (q < n ? slot_of<kBPT>(a.end[s] - 1, th) : s);
        s_rk[s] = (rng & 0xffff) | (a.kidx[s] << 16);
        s_par[s] = (short)a.par[s];
    }
    // Per position: V_ref (or V before anchoring) and delta = V - V_ref in registers, the ends-list
    // bounds in registers, S and z in C.
    float2 vr[kBPT], dl[kBPT];
    int ecnt[kBPT];
#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        vr[j] = make_float2(1.0f, 0.0f);
        dl[j] = make_float2(0.0f, 0.0f);
        ecnt[j] = 0;
        float2 sh = make_float2(0.0f, 0.0f), zh = sh, sl = sh;
        if (q < n) {
            const int i = a.col[s];
            if (a.s32) {
                sh = S32[i];
            } else {
                const double2 sv = S64[i];
                sh = make_float2(__double2float_rn(sv.x), __double2float_rn(sv.y));
                sl = make_float2(__double2float_rn(sv.x - (double)sh.x), __double2float_rn(sv.y - (double)sh.y));
            }
            const float4 zq = a.z[s];
            zh = make_float2(zq.x, zq.y);
            ecnt[j] = a.ecnt[s];
        }
        C[s] = make_float4(sh.x, sh.y, zh.x, zh.y);
        B[s] = make_float4(sl.x, sl.y, 0.0f, 0.0f);  // S_lo until the first anchor replaces it by D
        if (kZip) Zs[s] = q < n ? a.zip_hi[s] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    if (g.given) {  // a loop of its own: fewer loads in flight at once, fewer registers
        bool off_band = false;
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            const int q = base + j, s = j * th + tid;
            if (q < n) {
                const int64_t k = t * n + a.col[s];
                if (a.v0_pred) {
                    const float2 d = __half22float2(static_cast<const __half2 *>(a.V0)[t * a.v0_pitch + a.col[s]]);
                    vr[j] = make_float2(1.0f + d.x, d.y);
                    const float m2 = abs2(vr[j]);
                    off_band |= !(m2 >= 0.49f && m2 <= 1.21f);
                } else if (a.v32) {
                    vr[j] = static_cast<const float2 *>(a.V0)[k];
                } else {
                    const double2 v = static_cast<const double2 *>(a.V0)[k];
                    vr[j] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
                    if (g.blind)  // a warm start runs FP32 sweeps on fl32(V_0) first
                        dl[j] = make_float2(__double2float_rn(v.x - (double)vr[j].x),
                                            __double2float_rn(v.y - (double)vr[j].y));
                }
            }
        }
        // A predicted V_0 with |V_i| outside [0.7, 1.1] at any bus is not trusted: the flat start.
        if (a.v0_pred && __syncthreads_or(off_band)) {
#pragma unroll
            for (int j = 0; j < kBPT; ++j) vr[j] = make_float2(1.0f, 0.0f);
            if (tid == 0) atomicAdd(&g.counters[7], 1);
        }
    }
    __syncthreads();
    // A given start is anchored at once ("blind"), and anchored again when the step is small; a
    // warm start (an approximate V_0) takes FP32 sweeps first, like the flat start.
    bool anchored = g.blind != 0, blind = anchored, anchor_now = anchored, done = false, conv = false;
    int it = 0, anchors = 0;
    float dprev2 = 0.0f;
    // Each sweep's block-wide max |step| (and max |delta|) is reduced within the warp at the end
    // of the sweep and finished at the first barrier of the next one (its first scan's), where
    // the decision is taken; a sweep whose predecessor turns out to end the column or to call for
    // an anchor is abandoned before it changes any state.
    bool pending = false;
    float2 wmx = make_float2(0.0f, 0.0f);
    // Every thread takes the same decision from the same block max.  A step is only trusted to be
    // below tol on an anchored column whose offset from V_ref is small: in FP32 on V itself (or on
    // a large offset) a tiny step can round to zero.
    auto decide = [&](float2 dm) {
        const float d2 = dm.x;
        ++it;
        if (d2 <= g.tol2 && anchored && (!blind || dm.y < g.switch_tol2)) {
            done = conv = true;
        } else if (it >= g.max_iter || !(d2 < 1e30f)) {
            done = true;
        } else if (!anchored || blind) {
            // Anchor once the step is small, or is predicted (geometric rate) to fall below 3e-6
            // in the next sweep: d^2 < 3e-6 d_prev, squared.
            if (d2 < g.switch_tol2 || (dprev2 > 0.0f && d2 * d2 < 9e-12f * dprev2)) {
                anchor_now = true;
                blind = false;
            }
        }
        dprev2 = d2;
    };
    for (;;) {
        // The first sweep after an anchor taken from the FP32 phase starts at delta = 0 exactly:
        // every load-current change is zero, so the path sums are zero and the sweep returns
        // delta = D.  Its scans are skipped (the result is the same bit for bit).
        bool zero_sweep = false;
        if (anchor_now) {
            zero_sweep = !anchored;
            anchor_now = false;
            anchored = true;
            ++anchors;
            if (anchors > 1) {
                // B holds the previous anchor's D: S_lo again, one position at a time (rare).
#pragma unroll 1
                for (int j = 0; j < kBPT; ++j) {
                    const int q = base + j, s = j * th + tid;
                    float2 slo = make_float2(0.0f, 0.0f);
                    if (q < n && !a.s32) {
                        const double2 sv = S64[a.col[s]];
                        const float4 cs = C[s];
                        slo = make_float2(__double2float_rn(sv.x - (double)cs.x), __double2float_rn(sv.y - (double)cs.y));
                    }
                    B[s] = make_float4(slo.x, slo.y, 0.0f, 0.0f);
                }
            }
            // V_ref <- fl32(V); the remainder stays in delta.  D = BFS(V_ref) - V_ref goes to B.
#pragma unroll
            for (int j = 0; j < kBPT; ++j) {
                const int s = j * th + tid;
                const f2 re = two_sum(vr[j].x, dl[j].x), im = two_sum(vr[j].y, dl[j].y);
                vr[j] = make_float2(re.h, im.h);
                dl[j] = make_float2(re.l, im.l);
                const float4 cs = C[s], b = B[s];  // b = (S_lo, -)
                A[s] = make_float4(cs.x, cs.y, 0.0f, 0.0f);
                B[s] = make_float4(re.h, im.h, b.x, b.y);
            }
            const c2 off = anchor_dd<kBPT, kZip, kPh>(a, A, B, s_rk, Zs, ecnt, wtd, tid, th, lane, warp);
#pragma unroll
            for (int j = 0; j < kBPT; ++j) {
                const int q = base + j, s = j * th + tid;
                if (q < n) {
                    const c2 ps = cqadd(off, unpack(B[s]));
                    const c2 vs = kPh == 1 ? a.vs_dd : a.vs_ddp[phase_of(ecnt[j])];
                    const c2 D = cqsub(cqsub(vs, c2{{vr[j].x, 0.0f}, {vr[j].y, 0.0f}}), ps);
                    B[s] = make_float4(D.re.h, D.im.h, D.re.l, D.im.l);
                }
            }
            __syncthreads();  // the sweep reuses A
        }
        if (done) break;

        // --- one sweep ---
        float2 loc[kBPT], off = make_float2(0.0f, 0.0f);  // path sums: off + loc[j]
#pragma unroll
        for (int j = 0; j < kBPT; ++j) loc[j] = off;
        if (!zero_sweep) {
            // Load currents (or their change from V_ref) and their inclusive prefix sums P.
            // (Two loops behind one block-uniform branch, so that only one of the two current
            // formulas is evaluated.)
            float2 run = make_float2(0.0f, 0.0f);
            if (anchored) {
#pragma unroll
                for (int j = 0; j < kBPT; ++j) {
                    const float4 cs = C[j * th + tid];
                    const float4 al = kZip ? Zs[j * th + tid] : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
                    run = add2(run, demand_change<kZip>(vr[j], dl[j], make_float2(cs.x, cs.y), al));
                    loc[j] = run;  // positions past n have S = 0 and add nothing
                }
            } else {
#pragma unroll
                for (int j = 0; j < kBPT; ++j) {
                    const float4 cs = C[j * th + tid];
                    const float4 al = kZip ? Zs[j * th + tid] : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
                    run = add2(run, demand_current<kZip>(vr[j], make_float2(cs.x, cs.y), al));
                    loc[j] = run;
                }
            }
            {
                // First scan; its barrier also finishes the previous sweep's block max.
                float2 inc = run;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float ux = __shfl_up_sync(kFull, inc.x, o), uy = __shfl_up_sync(kFull, inc.y, o);
                    if (lane >= o) inc = add2(make_float2(ux, uy), inc);
                }
                const float ex = inc.x - run.x, ey = inc.y - run.y;  // exclusive: inclusive minus own
                if (lane == 31) wtm[warp] = make_float4(inc.x, inc.y, wmx.x, wmx.y);
                __syncthreads();
                const float4 tw = lane < nwarps ? wtm[lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (pending) {
                    pending = false;
                    // Max over lanes 0 .. nwarps - 1 (the warps' maxima; a NaN stays NaN), one warp-wide
                    // reduction whose result every lane receives: the decision below must be the same
                    // in every thread of the block, or threads would leave the sweep loop while others
                    // wait at a barrier.  Lanes past nwarps hold 0, below every squared step, so the
                    // reduction runs over all 32 lanes.  max |delta| only counts on a blind anchor.
                    decide(make_float2(warp_max_nan(tw.z), warp_max(tw.w)));
                    if (done || anchor_now) continue;
                }
                off = add2(warps_before(make_float2(tw.x, tw.y), lane, warp, nwarps),
                           lane ? make_float2(ex, ey) : make_float2(0.0f, 0.0f));
            }
#pragma unroll
            for (int j = 0; j < kBPT; ++j) {
                loc[j] = add2(off, loc[j]);  // the thread's own prefix values, also kept in registers
                P[j * th + tid] = loc[j];
            }
            __syncthreads();
            // Branch terms x_q = z_q (P[end_q - 1] - P[q - 1]).
            // Descending j: loc[j - 1] still holds the prefix value of position q - 1.
#pragma unroll
            for (int j = kBPT - 1; j >= 0; --j) {
                const int q = base + j, s = j * th + tid, rk = s_rk[s];
                float2 xq = make_float2(0.0f, 0.0f);  // positions past n contribute nothing
                if (q < n) {
                    if (kPh == 1) {
                        const int ls = rk & 0xffff;  // slot of the subtree's last position (s for a leaf)
                        float2 L = ls == s ? loc[j] : P[ls];
                        if (j) L = sub2(L, loc[j - 1]);
                        else if (q > 0) L = sub2(L, P[(kBPT - 1) * th + tid - 1]);
                        const float4 cs = C[s];
                        xq = cmul2(make_float2(cs.z, cs.w), L);
                    } else {
                        // x = sum over phases p' of Z[p][p'] L_{p'}
                        const int p = phase_of(ecnt[j]), qb = q - p * a.nbp, eb = (rk & 0xffff) - p * a.nbp;
#pragma unroll
                        for (int pp = 0; pp < kPh; ++pp) {
                            float2 L = P[slot_of<kBPT>(pp * a.nbp + eb - 1, th)];
                            const int prev = pp * a.nbp + qb - 1;
                            if (prev >= 0) L = sub2(L, P[slot_of<kBPT>(prev, th)]);
                            xq = add2(xq, cmul2(__ldg(&a.zrow_f[(size_t)s * kPh + pp]), L));
                        }
                    }
                }
                // The branch term goes where the position that closes its range gathers it: X
                // holds the terms in ends-list order, so each position's list is contiguous.
                const int k = rk >> 16;
                if (k >= 0) X[k] = xq;
                loc[j] = xq;
            }
            __syncthreads();
            // Path sums: prefix sums of E_q = x_q - (x_b of every b whose subtree range ends at
            // q).  Up to kGather entries per position unrolled and predicated; longer lists (rare:
            // a drop of more than kGather levels between neighbouring positions) finish in a loop.
            bool longer = false;
#pragma unroll
            for (int j = 0; j < kBPT; ++j) {
                const int st = ecnt[j] & 0xffff, cnt = ends_cnt(ecnt[j]);
                float2 e = loc[j];
#pragma unroll
                for (int k = 0; k < kGather; ++k)
                    if (k < cnt) e = sub2(e, X[st + k]);
                longer |= cnt > kGather;
                loc[j] = e;
            }
            if (longer) {
#pragma unroll
                for (int j = 0; j < kBPT; ++j) {
                    const int st = ecnt[j] & 0xffff, cnt = ends_cnt(ecnt[j]);
                    for (int k = kGather; k < cnt; ++k) loc[j] = sub2(loc[j], X[st + k]);
                }
            }
            run = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int j = 0; j < kBPT; ++j) {
                run = add2(run, loc[j]);  // positions past n have x = 0 and no ends
                loc[j] = run;
            }
            off = block_scan(run, wt2, lane, warp, nwarps);
        }
        // max |step|^2 (NaN if any step is NaN), and on a blind anchor max |delta|^2
        float2 mx = make_float2(0.0f, 0.0f);
        if (anchored) {
#pragma unroll
            for (int j = 0; j < kBPT; ++j) {
                const int q = base + j, s = j * th + tid;
                if (q < n) {
                    const float4 D = B[s];
                    const float2 nd = add2(sub2(make_float2(D.x, D.y), add2(off, loc[j])), make_float2(D.z, D.w));
                    mx.x = fmax_nan(mx.x, abs2(sub2(nd, dl[j])));
                    dl[j] = nd;
                    mx.y = fmaxf(mx.y, abs2(nd));
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < kBPT; ++j) {
                const int q = base + j;
                if (q < n) {
                    const float2 nv = sub2(kPh == 1 ? a.vs_f : a.vs_fp[phase_of(ecnt[j])], add2(off, loc[j]));
                    mx.x = fmax_nan(mx.x, abs2(sub2(nv, vr[j])));
                    vr[j] = nv;
                }
            }
        }
        wmx = make_float2(warp_max_nan(mx.x), warp_max(mx.y));
        pending = true;
    }

    // Outputs: V, iteration count and the mismatch max_i |V_i| |rho_i| at the returned V, with
    // rho = Y_dd x + c:
    //   anchored:   x = delta - D, x_slack = 0,   c = conj(S ./ V) - conj(S ./ V_ref)
    //               (from rho(V_ref) = -Y_dd D, as D = K rho(V_ref) with K = -Y_dd^{-1});
    //   otherwise:  x = V,         x_slack = v_s, c = conj(S ./ V).
    // On the tree (Y_dd x)_q = -J_q + sum over the children k of J_k with the branch currents
    // J_k = y_k (x_parent(k) - x_k); the children of q are q + 1 and then each next sibling, the
    // end of the previous one's range, while inside q's range.
    float2 *J = reinterpret_cast<float2 *>(B);
    float2 xs[kBPT];
#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        if (anchored) {
            const float4 D = B[s];
            xs[j] = sub2(sub2(dl[j], make_float2(D.x, D.y)), make_float2(D.z, D.w));
        } else {
            xs[j] = vr[j];
        }
        if (q < n) {
            if (a.V_out) {
                const int64_t k = t * n + a.col[s];
                if (a.v32)
                    static_cast<float2 *>(a.V_out)[k] = add2(vr[j], dl[j]);
                else
                    static_cast<double2 *>(a.V_out)[k] =
                        make_double2((double)vr[j].x + (double)dl[j].x, (double)vr[j].y + (double)dl[j].y);
            }
            X[s] = xs[j];
        }
    }
    __syncthreads();  // X complete; B (D) no longer read
    const float2 x_slack = anchored ? make_float2(0.0f, 0.0f) : a.vs_f;
#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        if (q < n) {
            const int p = s_par[s];
            if (kPh == 1) {
                const float4 cs = C[s];
                const float2 zq = make_float2(cs.z, cs.w);
                const float inv = __fdividef(1.0f, abs2(zq));
                const float2 yk = make_float2(zq.x * inv, -zq.y * inv);
                J[s] = cmul2(yk, sub2(p >= 0 ? X[p] : x_slack, xs[j]));
            } else {
                // J = sum over phases p' of Y[ph][p'] (x_parent,p' - x_q,p'): the parent's
                // position comes back from its slot (position = (slot % th) kBPT + slot / th).
                const int ph = phase_of(ecnt[j]), qb = q - ph * a.nbp;
                const int pb = p >= 0 ? (p % th) * kBPT + p / th - ph * a.nbp : -1;
                float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int pp = 0; pp < kPh; ++pp) {
                    const float2 xp = pb >= 0 ? X[slot_of<kBPT>(pp * a.nbp + pb, th)]
                                              : (anchored ? make_float2(0.0f, 0.0f) : a.vs_fp[pp]);
                    const float2 xq = X[slot_of<kBPT>(pp * a.nbp + qb, th)];
                    acc = add2(acc, cmul2(a.yrow[(size_t)s * kPh + pp], sub2(xp, xq)));
                }
                J[s] = acc;
            }
        }
    }
    __syncthreads();
    // Mismatch, |V| band statistics: (max mismatch, -min |V|^2, max |V|^2, buses outside the band).
    float4 red = make_float4(0.0f, -__int_as_float(0x7f800000), 0.0f, 0.0f);
#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        if (q < n) {
            const float4 cs = C[s];
            const float2 sh = make_float2(cs.x, cs.y);
            const float4 al = kZip ? Zs[s] : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
            float2 r = anchored ? demand_change<kZip>(vr[j], dl[j], sh, al) : demand_current<kZip>(vr[j], sh, al);
            r = sub2(r, J[s]);
            if (kPh == 1) {
                // The first child is q + 1, each next one follows the previous one's last position;
                // the child whose subtree ends where q's ends is the last.
                const int lq = s_rk[s] & 0xffff;
                for (int ks = lq == s ? -1 : next_slot<kBPT>(s, th); ks >= 0;) {
                    r = add2(r, J[ks]);
                    const int lc = s_rk[ks] & 0xffff;
                    ks = lc == lq ? -1 : next_slot<kBPT>(lc, th);
                }
            } else {
                const int e = s_rk[s] & 0xffff;
                for (int k = q + 1; k < e;) {
                    const int ks = slot_of<kBPT>(k, th);
                    r = add2(r, J[ks]);
                    k = s_rk[ks] & 0xffff;
                }
            }
            const float v2 = abs2(add2(vr[j], dl[j]));
            float mv = sqrtf(v2 * abs2(r));
            if (mv != mv) mv = __int_as_float(0x7f800000);  // a NaN mismatch reports as +inf
            red.x = fmaxf(red.x, mv);
            red.y = fmaxf(red.y, -v2);
            red.z = fmaxf(red.z, v2);
            const bool under = v2 < a.v_min2, over = v2 > a.v_max2;
            red.w += (under || over) ? 1.0f : 0.0f;
            if (under && a.bus_under) atomicAdd(&a.bus_under[a.col[s]], 1);
            if (over && a.bus_over) atomicAdd(&a.bus_over[a.col[s]], 1);
        }
    }
    red = make_float4(warp_max(red.x), warp_max(red.y), warp_max(red.z),
                      (float)__reduce_add_sync(kFull, (unsigned)red.w));
    if (lane == 0) wm[warp] = red;
    __syncthreads();
    if (tid == 0) {
        float4 r = wm[0];
        for (int w = 1; w < nwarps; ++w)
            r = make_float4(fmaxf(r.x, wm[w].x), fmaxf(r.y, wm[w].y), fmaxf(r.z, wm[w].z), r.w + wm[w].w);
        if (a.mismatch_out) a.mismatch_out[t] = (double)r.x;
        if (a.iters_out) a.iters_out[t] = conv ? it : -g.max_iter;
        if (a.col_vmin) a.col_vmin[t] = sqrtf(-r.y);
        if (a.col_vmax) a.col_vmax[t] = sqrtf(r.z);
        if (a.col_viol) a.col_viol[t] = (int32_t)r.w;
        if (conv) atomicAdd(a.conv, 1);
        atomicMax(&g.counters[5], it);
        atomicMax(&g.counters[6], anchors);
    }
}

}  // namespace

int tree_bpt(int n) {
    if (const char *e = std::getenv("TPF_TREE_BPT")) {
        const int b = std::atoi(e);
        if (b == 2 || b == 4 || b == 8 || b == kTreeBigBPT) return tree_threads(n, b) ? b : 0;
    }
    for (int b : {4, 8, kTreeBigBPT})
        if (tree_threads(n, b)) return b;
    return 0;
}

namespace {

// The network part of a feeder's work entry.
TreeWork work_of(const tpf_handle *h) {
    const DeviceNet &d = h->dev;
    TreeWork w{};
    w.n = d.n;
    w.n_ends = d.t_n_ends;
    w.vs_f = make_float2((float)h->net.vs_re, (float)h->net.vs_im);
    const float rh = (float)h->net.vs_re, ih = (float)h->net.vs_im;
    w.vs_dd = c2{{rh, (float)(h->net.vs_re - (double)rh)}, {ih, (float)(h->net.vs_im - (double)ih)}};
    w.col = d.t_col;
    w.end = d.t_end;
    w.par = d.t_par;
    w.ecnt = d.t_ecnt;
    w.ends = d.t_ends;
    w.kidx = d.t_kidx;
    w.z = d.t_z;
    w.zip_hi = d.t_zip_hi;
    w.zip_lo = d.t_zip_lo;
    w.nbp = d.nbp;
    w.zrow = d.t_zrow;
    w.zrow_f = d.t_zrow_f;
    w.yrow = d.t_yrow;
    for (int p = 0; p < 3; ++p) {
        const bool has = p < h->net.phases && (int)h->net.vs.size() >= 2 * (p + 1);
        const double re = has ? h->net.vs[2 * p] : h->net.vs_re, im = has ? h->net.vs[2 * p + 1] : h->net.vs_im;
        const float fr = (float)re, fi = (float)im;
        w.vs_fp[p] = make_float2(fr, fi);
        w.vs_ddp[p] = c2{{fr, (float)(re - (double)fr)}, {fi, (float)(im - (double)fi)}};
    }
    w.v_min2 = 0.0f;
    w.v_max2 = std::numeric_limits<float>::infinity();
    return w;
}

size_t tree_smem(int threads, int bpt, bool zip, int phases) {
    (void)phases;
    const size_t ns = (size_t)threads * bpt;
    // A, B, C (and the ZIP coefficients); range, parent, ends index.  The large-feeder kernel
    // keeps only A and the indices on chip.
    if (bpt == kTreeBigBPT) return ns * sizeof(float4) + sizeof(short) * 3 * ns;
    return (zip ? 4 : 3) * ns * sizeof(float4) + sizeof(short) * 3 * ns;
}

// Device scratch per launch column of the large-feeder kernel.
size_t tree_scratch_per_col(int threads, int bpt, bool zip) {
    return bpt == kTreeBigBPT ? (size_t)(zip ? 3 : 2) * threads * bpt * sizeof(float4) : 0;
}

// cols == 0 only sets the kernel's shared-memory attribute.
template <int kBPT, bool kZip, int kPh, int kTh = 0>
cudaError_t launch_tree_t(int threads, int64_t cols, size_t smem, const TreeArgs &g, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(mx_tree<kBPT, kZip, kPh, kTh>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess && cols > 0) mx_tree<kBPT, kZip, kPh, kTh><<<(unsigned)cols, threads, smem, st>>>(g);
    return e;
}

// The single-phase constant-power kernel has compile-time block sizes for the power-of-two shapes
// of the default bus-per-thread choice (4 buses per thread at 64-512 threads, 8 at 512); other
// block sizes and the ZIP and polyphase kernels take the block size at run time.
template <int kBPT>
cudaError_t launch_tree_b(int threads, bool zip, int phases, int64_t cols, size_t smem, const TreeArgs &g,
                          cudaStream_t st) {
    if (phases == 3) return launch_tree_t<kBPT, false, 3>(threads, cols, smem, g, st);
    if (zip) return launch_tree_t<kBPT, true, 1>(threads, cols, smem, g, st);
    if constexpr (kBPT == 4) {
        switch (threads) {
        case 64: return launch_tree_t<kBPT, false, 1, 64>(threads, cols, smem, g, st);
        case 128: return launch_tree_t<kBPT, false, 1, 128>(threads, cols, smem, g, st);
        case 256: return launch_tree_t<kBPT, false, 1, 256>(threads, cols, smem, g, st);
        case 512: return launch_tree_t<kBPT, false, 1, 512>(threads, cols, smem, g, st);
        default: break;
        }
    }
    if constexpr (kBPT == 8)
        if (threads == 512) return launch_tree_t<kBPT, false, 1, 512>(threads, cols, smem, g, st);
    return launch_tree_t<kBPT, false, 1>(threads, cols, smem, g, st);
}

// prepare: set the kernel's attributes only (before a stream capture), launch nothing.
tpf_status launch_tree(int bpt, int threads, bool zip, int phases, int64_t cols, const TreeArgs &g, cudaStream_t st,
                       bool prepare = false) {
    if (cols <= 0 && !prepare) return TPF_OK;
    if (cols > 0x7fffffff) return TPF_EUNSUPPORTED;  // one block per column
    if (phases != 1 && (phases != 3 || zip)) return TPF_EUNSUPPORTED;
    const size_t smem = tree_smem(threads, bpt, zip, phases);
    if (smem > 227 * 1024) return TPF_EUNSUPPORTED;
    cudaError_t e;
    const int64_t c = prepare ? 0 : cols;
    if (bpt == kTreeBigBPT)
        e = launch_tree_b<kTreeBigBPT>(threads, zip, phases, c, smem, g, st);
    else if (bpt == 8)
        e = launch_tree_b<8>(threads, zip, phases, c, smem, g, st);
    else if (bpt == 4)
        e = launch_tree_b<4>(threads, zip, phases, c, smem, g, st);
    else
        e = launch_tree_b<2>(threads, zip, phases, c, smem, g, st);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return TPF_ECUDA;
    return TPF_OK;
}

TreeArgs args_of(const tpf_opts &o) {
    TreeArgs g{};
    g.max_iter = o.max_iter;
    g.given = o.start != TPF_START_FLAT;
    g.blind = o.start == TPF_START_GIVEN;
    const float tol = (float)o.tol, sw = (float)o.switch_tol;
    g.tol2 = tol * tol;
    g.switch_tol = sw;
    g.switch_tol2 = sw * sw;
    return g;
}

}  // namespace

tpf_status solve_sparse_ex(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters, double *mismatch,
                           const tpf_outputs *out, const tpf_opts &o, cudaStream_t st, const void *V0_pred,
                           int64_t v0_pitch) {
    const DeviceNet &d = h->dev;
    if (!d.radial || o.precision != TPF_PREC_MIXED || d.t_threads == 0) return TPF_EUNSUPPORTED;
    if (T > 0x7fffffff) return TPF_EUNSUPPORTED;
    tpf_status rs = ensure_workspace(h, T, kWsState);  // counters
    if (rs != TPF_OK) return rs;
    Workspace &w = h->ws;
    if (cudaMemsetAsync(w.counters, 0, sizeof(int) * 8, st) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    TreeArgs g = args_of(o);
    g.counters = w.counters;
    g.one = work_of(h);
    TreeWork &wk = g.one;
    wk.S = S;
    wk.V0 = V;
    wk.V_out = V;
    if (V0_pred) {  // a warm start read from a separate predicted V_0
        wk.V0 = V0_pred;
        wk.v0_pred = 1;
        wk.v0_pitch = v0_pitch > 0 ? v0_pitch : h->dev.n;
        g.given = 1;
        g.blind = 0;
    }
    wk.iters_out = iters;
    wk.mismatch_out = mismatch;
    wk.T = T;
    wk.conv = w.counters + kCntConverged;
    if (out) {
        wk.s32 = out->s_complex64 != 0;
        wk.v32 = out->v_complex64 != 0;
        wk.col_vmin = out->col_vmin;
        wk.col_vmax = out->col_vmax;
        wk.col_viol = out->col_viol;
        wk.bus_under = out->bus_under;
        wk.bus_over = out->bus_over;
        wk.v_min2 = (float)(out->v_min * out->v_min);
        wk.v_max2 = (float)(out->v_max * out->v_max);
    }
    // The large-feeder kernel keeps part of each column's state in device scratch: its columns go
    // in chunks of at most 8,192 launch columns, each with its slice.
    const bool zip = d.t_zip_hi != nullptr;
    const size_t per_col = tree_scratch_per_col(d.t_threads, d.t_bpt, zip);
    const int64_t chunk = per_col ? std::min<int64_t>(T, 8192) : T;
    if (per_col && w.tree_scratch_bytes < per_col * chunk) {
        cudaFree(w.tree_scratch);
        w.tree_scratch = nullptr;
        w.tree_scratch_bytes = 0;
        if (cudaMalloc(&w.tree_scratch, per_col * chunk) != cudaSuccess) {
            cudaGetLastError();
            return TPF_ENOMEM;
        }
        w.tree_scratch_bytes = per_col * chunk;
    }
    g.scratch = w.tree_scratch;
    KernelTimer timer(o.profile != 0, st);
    int launches = 0;
    const int n = d.n;
    const size_t s_size = wk.s32 ? sizeof(float2) : sizeof(double2), v_size = wk.v32 ? sizeof(float2) : sizeof(double2);
    for (int64_t c0 = 0; c0 < T && rs == TPF_OK; c0 += chunk) {
        TreeArgs gc = g;
        TreeWork &wc = gc.one;
        wc.T = std::min(chunk, T - c0);
        wc.S = static_cast<const char *>(S) + (size_t)c0 * n * s_size;
        if (V) wc.V0 = wc.V_out = static_cast<char *>(V) + (size_t)c0 * n * v_size;
        if (V0_pred) wc.V0 = static_cast<const char *>(V0_pred) + (size_t)c0 * wk.v0_pitch * sizeof(__half2);
        if (iters) wc.iters_out = iters + c0;
        if (mismatch) wc.mismatch_out = mismatch + c0;
        if (wk.col_vmin) wc.col_vmin = wk.col_vmin + c0;
        if (wk.col_vmax) wc.col_vmax = wk.col_vmax + c0;
        if (wk.col_viol) wc.col_viol = wk.col_viol + c0;
        timer.begin(KernelTimer::kResidual);
        rs = launch_tree(d.t_bpt, d.t_threads, zip, d.phases, wc.T, gc, st);
        timer.end();
        ++launches;
    }
    if (rs != TPF_OK) return rs;
    if (cudaMemcpyAsync(w.counters_host, w.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    const int64_t conv = w.counters_host[kCntConverged];
    h->stats.sweeps = w.counters_host[5];
    h->start_fallback = V0_pred ? w.counters_host[7] : 0;
    h->stats.precise_sweeps = w.counters_host[6];
    h->stats.kernel_launches = launches;
    h->stats.converged = conv;
    h->stats.residual_ms = timer.total_ms(KernelTimer::kResidual);
    return conv == T ? TPF_OK : TPF_ENOCONV;
}

tpf_status solve_sparse(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters, double *mismatch,
                        const tpf_opts &o, cudaStream_t st) {
    return solve_sparse_ex(h, T, S, V, iters, mismatch, nullptr, o, st);
}

tpf_status autotune_sparse(tpf_handle *h, int64_t T, const void *S, const tpf_opts &o, cudaStream_t st,
                           int *bpt_out) {
    DeviceNet &d = h->dev;
    if (!d.radial || d.t_threads == 0) return TPF_EUNSUPPORTED;
    const int n = d.n;
    // The ZIP coefficients live in the slot layout too: keep a host copy to lay them out again.
    std::vector<double> zip;
    if (d.zip64) {
        zip.resize(3 * (size_t)n);
        if (cudaMemcpy(zip.data(), d.zip64, sizeof(double) * zip.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            return TPF_ECUDA;
        }
    }
    auto relayout = [&](int bpt) -> tpf_status {
        tpf_status rs = layout_tree(h, bpt);
        if (rs == TPF_OK && !zip.empty()) rs = set_zip(h, zip.data());
        return rs;
    };
    void *V = nullptr;
    if (cudaMalloc(&V, sizeof(double) * 2 * (size_t)T * n) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ENOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    tpf_opts ot = o;
    ot.start = TPF_START_FLAT;
    ot.profile = 0;
    const int current = d.t_bpt;
    int best = 0;
    float best_ms = 0.0f;
    tpf_status rs = TPF_OK;
    for (int bpt : {2, 4, 8}) {
        if (!tree_threads(n, bpt)) continue;
        rs = relayout(bpt);
        if (rs != TPF_OK) break;
        if (d.t_threads == 0) continue;  // the layout does not fit this shape
        rs = solve_sparse(h, T, S, V, nullptr, nullptr, ot, st);  // warm-up
        if (rs != TPF_OK && rs != TPF_ENOCONV) {
            if (rs == TPF_EUNSUPPORTED) { rs = TPF_OK; continue; }  // too much shared memory
            break;
        }
        cudaEventRecord(e0, st);
        for (int r = 0; r < 2 && (rs == TPF_OK || rs == TPF_ENOCONV); ++r) rs = solve_sparse(h, T, S, V, nullptr, nullptr, ot, st);
        cudaEventRecord(e1, st);
        if (rs != TPF_OK && rs != TPF_ENOCONV) break;
        rs = TPF_OK;
        float ms = 0.0f;
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (best == 0 || ms < best_ms) {
            best = bpt;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(V);
    const tpf_status rs2 = relayout(best ? best : current);
    if (rs != TPF_OK) return rs;
    if (rs2 != TPF_OK) return rs2;
    if (bpt_out) *bpt_out = d.t_bpt;
    return TPF_OK;
}

namespace {

// The work table of a batch: feeders grouped by launch shape (buses per thread, threads, ZIP,
// phases), each group one launch over the concatenated columns of its feeders (col0 relative to
// the group), and the feeder behind each entry.
struct BatchLayout {
    std::vector<TreeWork> works;
    std::vector<std::pair<int, int>> groups;  // [first, last) in works
    std::vector<int> order;                   // works[k] belongs to feeder order[k]
};

BatchLayout batch_layout(int F, tpf_handle *const *hs, const int64_t *T, const void *const *S, void *const *V,
                         int32_t *const *iters, double *const *mismatch) {
    BatchLayout L;
    L.order.resize(F);
    for (int f = 0; f < F; ++f) L.order[f] = f;
    auto key = [&](int f) {
        const DeviceNet &d = hs[f]->dev;
        return std::make_tuple(d.t_zip_hi != nullptr, d.phases, d.t_bpt, d.t_threads);
    };
    std::sort(L.order.begin(), L.order.end(), [&](int x, int y) {
        const auto kx = key(x), ky = key(y);
        return kx != ky ? kx < ky : x < y;
    });
    L.works.resize(F);
    for (int k = 0; k < F; ++k) {
        const int f = L.order[k];
        TreeWork w = work_of(hs[f]);
        w.S = S[f];
        w.V0 = V[f];
        w.V_out = V[f];
        w.iters_out = iters ? iters[f] : nullptr;
        w.mismatch_out = mismatch ? mismatch[f] : nullptr;
        w.T = T[f];
        L.works[k] = w;
    }
    for (int k = 0; k < F;) {
        int e = k + 1;
        while (e < F && key(L.order[e]) == key(L.order[k])) ++e;
        int64_t c = 0;
        for (int i = k; i < e; ++i) {
            L.works[i].col0 = c;
            c += L.works[i].T;
        }
        L.groups.push_back({k, e});
        k = e;
    }
    return L;
}

int64_t group_cols(const BatchLayout &L, const std::pair<int, int> &gr) {
    int64_t cols = 0;
    for (int i = gr.first; i < gr.second; ++i) cols += L.works[i].T;
    return cols;
}

// Per-feeder converged counts (the first F entries of hconv), the largest sweep and anchor counts
// (entries F + 5 and F + 6) into the caller's outputs; TPF_OK when every column converged.
tpf_status batch_results(int F, const int64_t *T, const int *hconv, int launches, double kernel_ms,
                         int64_t *conv_out, tpf_stats *stats) {
    bool all = true;
    int64_t conv = 0, cols = 0;
    for (int f = 0; f < F; ++f) {
        if (conv_out) conv_out[f] = hconv[f];
        conv += hconv[f];
        cols += T[f];
        all = all && hconv[f] == T[f];
    }
    if (stats) {
        *stats = tpf_stats{};
        stats->sweeps = hconv[F + 5];
        stats->precise_sweeps = hconv[F + 6];
        stats->converged = conv;
        stats->columns = cols;
        stats->kernel_launches = launches;
        stats->residual_ms = kernel_ms;
    }
    return all ? TPF_OK : TPF_ENOCONV;
}

}  // namespace

tpf_status solve_batch_sparse(int F, tpf_handle *const *hs, const int64_t *T, const void *const *S, void *const *V,
                              int32_t *const *iters, double *const *mismatch, const tpf_opts &o, int64_t *conv_out,
                              tpf_stats *stats, cudaStream_t st) {
    BatchLayout L = batch_layout(F, hs, T, S, V, iters, mismatch);
    // Device copies: the work table and the per-feeder converged counts, plus the counters.
    const size_t wbytes = sizeof(TreeWork) * F, cbytes = sizeof(int) * ((size_t)F + 8);
    char *dbuf = nullptr;
    if (cudaMalloc(&dbuf, wbytes + cbytes) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ENOMEM;
    }
    TreeWork *dworks = reinterpret_cast<TreeWork *>(dbuf);
    int *dconv = reinterpret_cast<int *>(dbuf + wbytes), *dcnt = dconv + F;
    for (int k = 0; k < F; ++k) L.works[k].conv = dconv + L.order[k];
    tpf_status rs = TPF_OK;
    KernelTimer timer(o.profile != 0, st);
    int launches = 0;
    if (cudaMemsetAsync(dconv, 0, cbytes, st) != cudaSuccess ||
        cudaMemcpyAsync(dworks, L.works.data(), wbytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rs = TPF_ECUDA;
    TreeArgs g = args_of(o);
    g.counters = dcnt;
    for (auto &gr : L.groups) {
        if (rs != TPF_OK) break;
        const DeviceNet &d = hs[L.order[gr.first]]->dev;
        g.works = dworks + gr.first;
        g.n_works = gr.second - gr.first;
        timer.begin(KernelTimer::kResidual);
        rs = launch_tree(d.t_bpt, d.t_threads, d.t_zip_hi != nullptr, d.phases, group_cols(L, gr), g, st);
        timer.end();
        ++launches;
    }
    std::vector<int> hconv(F + 8, 0);
    if (rs == TPF_OK && (cudaMemcpyAsync(hconv.data(), dconv, cbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess))
        rs = TPF_ECUDA;
    if (rs != TPF_OK) cudaStreamSynchronize(st);
    cudaFree(dbuf);
    if (rs != TPF_OK) {
        cudaGetLastError();
        return rs;
    }
    return batch_results(F, T, hconv.data(), launches, timer.total_ms(KernelTimer::kResidual), conv_out, stats);
}

}  // namespace tpf

// A prepared batch: the work table stays on the device, and one solve of every feeder (reset of
// the counters, one launch per launch shape, copy of the counts to pinned host memory) is a CUDA
// graph, replayed by tpf_batch_launch.
struct tpf_batch {
    int F = 0, device = 0, launches = 0;
    std::vector<tpf_handle *> hs;
    std::vector<int> gens;      // each handle's layout generation when the graph was captured
    std::vector<int64_t> T;
    char *dbuf = nullptr;       // work table, converged counts [F], counters [8]
    int *hcnt = nullptr;        // pinned: the counts and counters of the last replay
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    bool pending = false;
};

namespace tpf {

int batch_device(const tpf_batch *b) { return b->device; }

void batch_plan_destroy(tpf_batch *b) {
    if (!b) return;
    DeviceScope dscope(b->device);
    if (b->pending && b->done) cudaEventSynchronize(b->done);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->done) cudaEventDestroy(b->done);
    cudaFree(b->dbuf);
    if (b->hcnt) cudaFreeHost(b->hcnt);
    cudaGetLastError();
    delete b;
}

tpf_status batch_plan_create(int F, tpf_handle *const *hs, const int64_t *T, const void *const *S, void *const *V,
                             int32_t *const *iters, double *const *mismatch, const tpf_opts &o, tpf_batch **out) {
    tpf_batch *b = new (std::nothrow) tpf_batch;
    if (!b) return TPF_ENOMEM;
    b->F = F;
    b->device = hs[0]->device;
    b->hs.assign(hs, hs + F);
    b->T.assign(T, T + F);
    for (int f = 0; f < F; ++f) b->gens.push_back(hs[f]->dev.layout_gen);
    BatchLayout L = batch_layout(F, hs, T, S, V, iters, mismatch);
    const size_t wbytes = sizeof(TreeWork) * F, cbytes = sizeof(int) * ((size_t)F + 8);
    if (cudaMalloc(&b->dbuf, wbytes + cbytes) != cudaSuccess || cudaMallocHost(&b->hcnt, cbytes) != cudaSuccess) {
        batch_plan_destroy(b);
        return TPF_ENOMEM;
    }
    TreeWork *dworks = reinterpret_cast<TreeWork *>(b->dbuf);
    int *dconv = reinterpret_cast<int *>(b->dbuf + wbytes), *dcnt = dconv + F;
    for (int k = 0; k < F; ++k) L.works[k].conv = dconv + L.order[k];
    tpf_status rs = TPF_OK;
    if (cudaMemcpy(dworks, L.works.data(), wbytes, cudaMemcpyHostToDevice) != cudaSuccess) rs = TPF_ECUDA;
    TreeArgs g = args_of(o);
    g.counters = dcnt;
    // Kernel attributes first: they are not stream work, so they stay out of the capture.
    for (auto &gr : L.groups) {
        if (rs != TPF_OK) break;
        const DeviceNet &d = hs[L.order[gr.first]]->dev;
        rs = launch_tree(d.t_bpt, d.t_threads, d.t_zip_hi != nullptr, d.phases, 0, g, nullptr, true);
    }
    cudaStream_t cs = nullptr;
    if (rs == TPF_OK && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rs = TPF_ECUDA;
    if (rs == TPF_OK && cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        if (cudaMemsetAsync(dconv, 0, cbytes, cs) != cudaSuccess) rs = TPF_ECUDA;
        for (auto &gr : L.groups) {
            if (rs != TPF_OK) break;
            const DeviceNet &d = hs[L.order[gr.first]]->dev;
            g.works = dworks + gr.first;
            g.n_works = gr.second - gr.first;
            const int64_t cols = group_cols(L, gr);
            rs = launch_tree(d.t_bpt, d.t_threads, d.t_zip_hi != nullptr, d.phases, cols, g, cs);
            if (cols > 0) ++b->launches;
        }
        if (rs == TPF_OK && cudaMemcpyAsync(b->hcnt, dconv, cbytes, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
            rs = TPF_ECUDA;
        // The capture always ends, so that the stream leaves capture mode whatever happened.
        if (cudaStreamEndCapture(cs, &b->graph) != cudaSuccess && rs == TPF_OK) rs = TPF_ECUDA;
    } else if (rs == TPF_OK) {
        rs = TPF_ECUDA;
    }
    if (rs == TPF_OK && (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess ||
                         cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess))
        rs = TPF_ECUDA;
    if (cs) cudaStreamDestroy(cs);
    if (rs != TPF_OK) {
        cudaGetLastError();
        batch_plan_destroy(b);
        return rs;
    }
    *out = b;
    return TPF_OK;
}

tpf_status batch_plan_launch(tpf_batch *b, cudaStream_t st) {
    for (int f = 0; f < b->F; ++f)
        if (b->hs[f]->dev.layout_gen != b->gens[f]) return TPF_EINVAL;  // a re-laid-out feeder
    if (b->pending && cudaEventSynchronize(b->done) != cudaSuccess) return TPF_ECUDA;  // one replay at a time
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess || cudaEventRecord(b->done, st) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    b->pending = true;
    return TPF_OK;
}

tpf_status batch_plan_wait(tpf_batch *b, int64_t *conv_out, tpf_stats *stats) {
    if (!b->pending) return TPF_EINVAL;
    if (cudaEventSynchronize(b->done) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    b->pending = false;
    return batch_results(b->F, b->T.data(), b->hcnt, b->launches, 0.0, conv_out, stats);
}

}  // namespace tpf
