// Mixed-precision solve path: fp16 tensor-core sweeps (tcgen05, FP32 accumulation in TMEM) in
// residual form, with V and the residual carried in double-float.
//
// The fixed point of Eq. 2 / Eq. 12, V = K conj(S ./ V) + W with K = -Y_dd^{-1} and
// W = K Y_ds v_s, is the zero of the residual
//
//     rho(V) = (Y_dd V + Y_ds v_s) + conj(S ./ V)      (Eq. 1 with i_d = conj(S ./ V))
//
// and the fixed-point step is exactly  V_{k+1} = V_k + K rho(V_k)  (expand K rho with
// K Y_dd = -I).  Written this way the dense product only carries the correction: the fp16 error
// of K and rho scales with |rho| -> 0 instead of with |V|, so the iterates converge to the
// double-precision solution while the O(n^2) work per column runs on fp16 tensor cores.
// rho itself is O(n) per column: for a shunt-free network (Y V)_i = sum_j y_ij (V_i - V_j) over
// the branches at bus i (V_slack = v_s).
//
// Per sweep:  mx_prologue  (one warp per column) decides convergence from the last step,
//                          forms rho (FP32 while the column's step is above switch_tol,
//                          double-float after), scales it by a per-column power of two and
//                          writes the fp16 B operand;
//             tc_gemm      (one CTA per 128 buses x 128 columns) computes K rho with four
//                          real-plane MMAs per K step (Re = Kr rr - Ki ri, Im = Kr ri + Ki rr),
//                          then its epilogue adds the update to V and folds max |dV| per column.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <cstdlib>
#include <cstring>

#include "tpf_internal.h"

namespace tpf {

#define TPF_CK(call)                  \
    do {                              \
        if ((call) != cudaSuccess) {  \
            cudaGetLastError();       \
            return TPF_ECUDA;         \
        }                             \
    } while (0)

namespace {

// ------------------------------------------------------------------------------------------
// Double-float arithmetic (a value is hi + lo with |lo| <= ulp(hi)/2).  Every operation uses the
// explicitly rounded intrinsics so that the compiler cannot fuse or reorder the error terms.
// ------------------------------------------------------------------------------------------
struct f2 {
    float h, l;
};

__device__ __forceinline__ f2 two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}
__device__ __forceinline__ f2 dd_add(f2 a, f2 b) {
    f2 s = two_sum(a.h, b.h);
    f2 t = two_sum(a.l, b.l);
    s = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(s.h, __fadd_rn(s.l, t.l));
}
__device__ __forceinline__ f2 dd_sub(f2 a, f2 b) { return dd_add(a, f2{-b.h, -b.l}); }
__device__ __forceinline__ f2 dd_mul(f2 a, f2 b) {
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ f2 dd_rcp(f2 b) {
    float q1 = __frcp_rn(b.h);
    f2 r = dd_sub(f2{1.0f, 0.0f}, dd_mul(b, f2{q1, 0.0f}));
    return fast_two_sum(q1, __fmul_rn(r.h, q1));
}

struct c2 {
    f2 re, im;
};
__device__ __forceinline__ c2 c_add(c2 a, c2 b) { return {dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ c2 c_sub(c2 a, c2 b) { return {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
__device__ __forceinline__ c2 c_mul(c2 a, c2 b) {
    return {dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}

// conj(s / v) = conj(s) v / |v|^2 in double-float.
__device__ __forceinline__ c2 load_current_dd(c2 s, c2 v) {
    f2 inv = dd_rcp(dd_add(dd_mul(v.re, v.re), dd_mul(v.im, v.im)));
    f2 nr = dd_add(dd_mul(s.re, v.re), dd_mul(s.im, v.im));
    f2 ni = dd_sub(dd_mul(s.re, v.im), dd_mul(s.im, v.re));
    return {dd_mul(nr, inv), dd_mul(ni, inv)};
}

// hi[k] + lo[k] as a normalised double-float (lo == nullptr reads as zero).
__device__ __forceinline__ c2 load_c2(const float2 *hi, const float2 *lo, int64_t k) {
    float2 a = hi[k];
    if (!lo) return {{a.x, 0.0f}, {a.y, 0.0f}};
    float2 b = lo[k];
    return {two_sum(a.x, b.x), two_sum(a.y, b.y)};
}

// rho_i in double-float for bus i of the column whose V planes start at vh / vl.
__device__ __forceinline__ c2 residual_dd(int i, const float2 *vh, const float2 *vl, const float2 *sh,
                                          const float2 *sl, const int *row_ptr, const int *nbr, const float4 *y,
                                          c2 vs) {
    c2 v = load_c2(vh, vl, i);
    c2 acc = load_current_dd(load_c2(sh, sl, i), v);
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        int j = nbr[e];
        c2 vj = j >= 0 ? load_c2(vh, vl, j) : vs;
        float4 ye = y[e];
        c2 yy = {{ye.x, ye.z}, {ye.y, ye.w}};
        acc = c_add(acc, c_mul(yy, c_sub(v, vj)));
    }
    return acc;
}

// conj(s / v) = conj(s) v / |v|^2 in FP32.
__device__ __forceinline__ float2 load_current_f32(float2 v, float2 s) {
    float inv = 1.0f / (v.x * v.x + v.y * v.y);
    return make_float2((s.x * v.x + s.y * v.y) * inv, (s.x * v.y - s.y * v.x) * inv);
}

// conj(s / (v + d)) - conj(s / v) = -conj(s d / ((v + d) v)) in FP32 (small when d is small).
__device__ __forceinline__ float2 delta_current(float2 v, float2 d, float2 s) {
    float2 w = make_float2(s.x * d.x - s.y * d.y, s.x * d.y + s.y * d.x);
    float2 vp = make_float2(v.x + d.x, v.y + d.y);
    float2 q = make_float2(vp.x * v.x - vp.y * v.y, vp.x * v.y + vp.y * v.x);
    float inv = 1.0f / (q.x * q.x + q.y * q.y);
    float wr = (w.x * q.x + w.y * q.y) * inv, wi = (w.y * q.x - w.x * q.y) * inv;  // w / q
    return make_float2(-wr, wi);                                                    // -conj(w / q)
}

// rho_i in FP32 from the high words only (the sweeps far from convergence).
__device__ __forceinline__ float2 residual_f32(int i, const float2 *vh, const float2 *sh, const int *row_ptr,
                                               const int *nbr, const float4 *y, float2 vs) {
    float2 v = vh[i];
    float2 cur = load_current_f32(v, sh[i]);
    float ar = cur.x, ai = cur.y;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        int j = nbr[e];
        float2 vj = j >= 0 ? vh[j] : vs;
        float dr = v.x - vj.x, di = v.y - vj.y;
        float4 ye = y[e];
        ar += ye.x * dr - ye.y * di;
        ai += ye.x * di + ye.y * dr;
    }
    return make_float2(ar, ai);
}

// rho(V_ref + d) - rho(V_ref) in FP32 for an anchored column (V_ref = vh, d = vl):
//   sum_j y_ij (d_i - d_j)                       (the network part is linear in V)
//   + conj(S/(V_ref + d)) - conj(S/V_ref) = -conj(S d / ((V_ref + d) V_ref)).
// Both terms are proportional to |d|, so their FP32 rounding error is ~6e-8 |d| |y|.
__device__ __forceinline__ float2 residual_corr(int i, const float2 *vh, const float2 *vl, const float2 *sh,
                                                const int *row_ptr, const int *nbr, const float4 *y) {
    const float2 d = vl[i];
    const float2 dc = delta_current(vh[i], d, sh[i]);
    float ar = dc.x, ai = dc.y;
    for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
        int j = nbr[e];
        float2 dj = j >= 0 ? vl[j] : make_float2(0.0f, 0.0f);
        float dr = d.x - dj.x, di = d.y - dj.y;
        float4 ye = y[e];
        ar += ye.x * dr - ye.y * di;
        ai += ye.x * di + ye.y * dr;
    }
    return make_float2(ar, ai);
}

__device__ __forceinline__ float pow2f(int e) {
    e = e < -126 ? -126 : (e > 127 ? 127 : e);
    return __int_as_float((127 + e) << 23);
}

// ------------------------------------------------------------------------------------------
// Elementwise kernels
// ------------------------------------------------------------------------------------------

// Split S (and V_0) into double-float planes with padded rows; one block per column.
__global__ void mx_pack(int64_t T, int n, int n_pad, const double2 *__restrict__ S, const double2 *__restrict__ V0,
                        float2 *Shi, float2 *Slo, float2 *Vhi, float2 *Vlo, int *flags, int *iters,
                        unsigned *delta, unsigned *dprev) {
    const int64_t t = blockIdx.x;
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x) {
        float2 sh = make_float2(0.f, 0.f), sl = sh, vh = make_float2(1.f, 0.f), vl = make_float2(0.f, 0.f);
        if (t < T && i < n) {
            double2 s = S[t * n + i];
            sh = make_float2(__double2float_rn(s.x), __double2float_rn(s.y));
            sl = make_float2(__double2float_rn(s.x - (double)sh.x), __double2float_rn(s.y - (double)sh.y));
            if (V0) {
                double2 v = V0[t * n + i];
                vh = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
                vl = make_float2(__double2float_rn(v.x - (double)vh.x), __double2float_rn(v.y - (double)vh.y));
            }
        }
        const int64_t k = t * n_pad + i;
        Shi[k] = sh;
        Slo[k] = sl;
        Vhi[k] = vh;
        Vlo[k] = vl;
    }
    if (threadIdx.x == 0) {
        flags[t] = t < T ? kActive : 0;
        iters[t] = 0;
        delta[t] = 0u;
        dprev[t] = 0u;
    }
}

struct PrologueArgs {
    int64_t cols;
    int n, n_pad, sweep, max_iter;
    float tol, switch_tol;
    float2 vs_f;
    c2 vs_dd;
    float2 *Vhi, *Vlo;
    const float2 *Shi, *Slo;
    float2 *RefHi, *RefLo;
    const int *row_ptr, *nbr;
    const float4 *y;
    int *flags, *iters, *rexp, *tile_active, *counters;
    unsigned *delta, *dprev;
    int given;  // the solve started from a given V_0: anchor every column at sweep 0
    int radial;
    const int *par, *ch_ptr, *ch;
    const float2 *ypar;
    __half *Rr, *Ri;
};

// One warp per column.  (1) Convergence decision for the step the last sweep applied (stop at
// max |dV| <= tol, give up at max_iter or on a non-finite step) and the anchoring decision.
// (2) rho for every bus: FP32 before anchoring; at the anchoring sweep V is re-based
// (Vhi + Vlo -> two-sum) and rho(V_ref) is evaluated once in double-float and stored; after it,
// rho = rho(V_ref) + FP32 correction in Vlo = V - V_ref.  (3) The fp16 operand 2^rexp * rho with
// max |component| in [2^13, 2^14).  BPL = buses per lane (n_pad / 32).
template <int BPL>
__global__ void __launch_bounds__(512, 1) mx_prologue(PrologueArgs a) {
    __shared__ int blk_active, blk_conv, blk_anch;
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (threadIdx.x == 0) {
        blk_active = 0;
        blk_conv = 0;
        blk_anch = 0;
    }
    __syncthreads();
    int f = 0;
    bool anchor = false;
    if (t < a.cols) {
        f = a.flags[t];
        if (a.sweep > 0 && (f & kActive)) {
            const float d = __uint_as_float(a.delta[t]);
            const float dp = __uint_as_float(a.dprev[t]);
            const int it = a.iters[t] + 1;
            if (d <= a.tol) {
                f = kDone;
            } else if (it >= a.max_iter || !(d < 1e30f)) {
                f = 0;
            } else if (!(f & kAnchored) || (f & kBlind)) {
                // Anchor once the step is small, or is predicted (geometric rate) to fall below
                // 3e-6 in the next sweep, while FP32 rounding (~1e-7) is still far below it.
                if (d < a.switch_tol || (dp > 0.0f && d * d < 3e-6f * dp)) {
                    anchor = true;
                    f = (f | kAnchored) & ~kBlind;
                }
            }
            __syncwarp();
            if (lane == 0) {
                a.iters[t] = it;
                a.flags[t] = f;
                a.delta[t] = 0u;
                a.dprev[t] = __float_as_uint(d);
                if (f & kDone) atomicAdd(&blk_conv, 1);
            }
        } else if (a.sweep == 0 && a.given && (f & kActive)) {
            anchor = true;
            f |= kAnchored | kBlind;
            __syncwarp();
            if (lane == 0) a.flags[t] = f;
        }
    }
    if (t < a.cols && (f & kActive)) {
        const int64_t base = t * a.n_pad;
        float2 *vh = a.Vhi + base;
        const float2 *sh = a.Shi + base;
        float rr[BPL], ri[BPL];
        float m = 0.0f;
        const bool anchored = (f & kAnchored) != 0;
        float2 *vl = a.Vlo + base;
        float2 *rh = a.RefHi + base, *rl = a.RefLo + base;
        if (anchor) {  // re-base: Vhi <- fl(Vhi + Vlo), Vlo <- the exact remainder
#pragma unroll
            for (int b = 0; b < BPL; ++b) {
                int i = lane + 32 * b;
                if (i < a.n) {
                    float2 h = vh[i], l = vl[i];
                    f2 re = two_sum(h.x, l.x), im = two_sum(h.y, l.y);
                    vh[i] = make_float2(re.h, im.h);
                    vl[i] = make_float2(re.l, im.l);
                }
            }
            __syncwarp();
        }
        if (a.radial && !anchor) {
            // Radial feeder: rho_i = local_i - J_i + sum_{children c} J_c with the branch current
            // J_c = y_c (V_parent(c) - V_c).  The column's V (or V - V_ref once anchored) is staged
            // in shared memory so the parent gathers and the children sums stay on chip.
            extern __shared__ float2 psm[];
            float2 *vb = psm + (size_t)(threadIdx.x >> 5) * 2 * a.n_pad;
            float2 *jb = vb + a.n_pad;
            const float2 *src = anchored ? vl : vh;
            const float2 vsrc = anchored ? make_float2(0.0f, 0.0f) : a.vs_f;
#pragma unroll
            for (int b = 0; b < BPL; ++b) {
                int i = lane + 32 * b;
                vb[i] = i < a.n ? src[i] : make_float2(0.0f, 0.0f);
            }
            __syncwarp();
#pragma unroll
            for (int b = 0; b < BPL; ++b) {
                int i = lane + 32 * b;
                rr[b] = 0.f;
                ri[b] = 0.f;
                if (i < a.n) {
                    const float2 v = vb[i];
                    const int p = a.par[i];
                    const float2 vp = p >= 0 ? vb[p] : vsrc;
                    const float2 y = a.ypar[i];
                    const float dr = vp.x - v.x, di = vp.y - v.y;
                    const float2 J = make_float2(y.x * dr - y.y * di, y.x * di + y.y * dr);
                    jb[i] = J;
                    const float2 loc = anchored ? delta_current(vh[i], v, sh[i]) : load_current_f32(v, sh[i]);
                    rr[b] = loc.x - J.x;
                    ri[b] = loc.y - J.y;
                }
            }
            __syncwarp();
#pragma unroll
            for (int b = 0; b < BPL; ++b) {
                int i = lane + 32 * b;
                if (i < a.n) {
                    for (int e = a.ch_ptr[i]; e < a.ch_ptr[i + 1]; ++e) {
                        const float2 J = jb[a.ch[e]];
                        rr[b] += J.x;
                        ri[b] += J.y;
                    }
                    if (anchored) {
                        const float2 h = rh[i], l = rl[i];
                        const f2 sr = two_sum(h.x, rr[b]), si = two_sum(h.y, ri[b]);
                        rr[b] = sr.h + (sr.l + l.x);
                        ri[b] = si.h + (si.l + l.y);
                    }
                }
                m = fmaxf(m, fmaxf(fabsf(rr[b]), fabsf(ri[b])));
            }
        } else if (anchored) {
#pragma unroll
            for (int b = 0; b < BPL; ++b) {
                int i = lane + 32 * b;
                rr[b] = 0.f;
                ri[b] = 0.f;
                if (i < a.n) {
                    c2 ref;
                    if (anchor) {
                        ref = residual_dd(i, vh, nullptr, sh, a.Slo + base, a.row_ptr, a.nbr, a.y, a.vs_dd);
                        rh[i] = make_float2(ref.re.h, ref.im.h);
                        rl[i] = make_float2(ref.re.l, ref.im.l);
                    } else {
                        float2 h = rh[i], l = rl[i];
                        ref = {{h.x, l.x}, {h.y, l.y}};
                    }
                    float2 c = residual_corr(i, vh, vl, sh, a.row_ptr, a.nbr, a.y);
                    f2 sr = two_sum(ref.re.h, c.x), si = two_sum(ref.im.h, c.y);
                    rr[b] = sr.h + (sr.l + ref.re.l);
                    ri[b] = si.h + (si.l + ref.im.l);
                }
                m = fmaxf(m, fmaxf(fabsf(rr[b]), fabsf(ri[b])));
            }
        } else {
#pragma unroll
            for (int b = 0; b < BPL; ++b) {
                int i = lane + 32 * b;
                rr[b] = 0.f;
                ri[b] = 0.f;
                if (i < a.n) {
                    float2 r = residual_f32(i, vh, sh, a.row_ptr, a.nbr, a.y, a.vs_f);
                    rr[b] = r.x;
                    ri[b] = r.y;
                }
                m = fmaxf(m, fmaxf(fabsf(rr[b]), fabsf(ri[b])));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        int e = 0;
        if (m > 0.0f) {
            frexpf(m, &e);
            e = 14 - e;
        }
        if (e > 120) e = 120;
        const float sc = pow2f(e);
        __half *Rr = a.Rr + base, *Ri = a.Ri + base;
#pragma unroll
        for (int b = 0; b < BPL; ++b) {
            int i = lane + 32 * b;
            if (i < a.n_pad) {
                Rr[i] = __float2half_rn(rr[b] * sc);
                Ri[i] = __float2half_rn(ri[b] * sc);
            }
        }
        if (lane == 0) {
            a.rexp[t] = e;
            a.tile_active[t / kTileN] = 1;
            atomicAdd(&blk_active, 1);
            if (anchor) atomicAdd(&blk_anch, 1);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (blk_active) atomicAdd(&a.counters[kCntActive], blk_active);
        if (blk_conv) atomicAdd(&a.counters[kCntConverged], blk_conv);
        if (blk_anch) atomicAdd(&a.counters[kCntPrecise], blk_anch);
    }
}

// Final outputs: V (complex128) from double-float, iteration counts, and the power mismatch
// max_i |V_i conj((Y v)_i) + S_i| = max_i |V_i| |rho_i| evaluated in double-float.
__global__ void __launch_bounds__(256) mx_finish(int64_t T, int n, int n_pad, int max_iter, const int *flags,
                                                 const int *it_state, const float2 *Vhi, const float2 *Vlo,
                                                 const float2 *Shi, const float2 *Slo, const int *row_ptr,
                                                 const int *nbr, const float4 *y, c2 vs, double2 *V_out,
                                                 int32_t *iters_out, double *mismatch_out) {
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= T) return;
    const int64_t base = t * n_pad;
    if (lane == 0 && iters_out) iters_out[t] = (flags[t] & kDone) ? it_state[t] : -max_iter;
    float worst = 0.0f;
    for (int i = lane; i < n; i += 32) {
        float2 h = Vhi[base + i], l = Vlo[base + i];
        V_out[t * n + i] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
        if (mismatch_out) {
            c2 r = residual_dd(i, Vhi + base, Vlo + base, Shi + base, Slo + base, row_ptr, nbr, y, vs);
            float mv = sqrtf(h.x * h.x + h.y * h.y) * sqrtf(r.re.h * r.re.h + r.im.h * r.im.h);
            if (!(mv <= worst)) worst = mv;
        }
    }
    if (!mismatch_out) return;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float other = __shfl_xor_sync(0xffffffffu, worst, o);
        if (!(other <= worst)) worst = other;
    }
    if (lane == 0) mismatch_out[t] = (double)worst;
}

// ------------------------------------------------------------------------------------------
// tcgen05 / TMA / mbarrier primitives (inline PTX)
// ------------------------------------------------------------------------------------------
constexpr int kStages = 3;
constexpr uint32_t kTileBytes = kTileM * kChunkK * 2;  // 16 KB: 128 rows x 64 fp16
constexpr uint32_t kStageBytes = 4 * kTileBytes;        // Ar, Ai, Br, Bi
constexpr uint64_t kWaitNs = 2000000000ull;             // bounded waits: 2 s
constexpr uint32_t kTmemCols = 256;                     // Dr: cols [0,128), Di: [128,256)
constexpr size_t kGemmSmem = 1024 + kStages * kStageBytes + 2048;  // align slack + stages + barriers/column info

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase with the given parity to complete; false if kWaitNs passed first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle layout written by
// TMA: rows of 64 fp16 (128 B), 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16 with fp16 A and B, FP32 accumulation, both K-major.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int negA) {
    return (1u << 4) | ((uint32_t)negA << 13) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct GemmEpi {
    int mode;  // 0 = store D (self-test), 1 = fixed-point update
    int *err;  // set to 1 when a bounded wait expires
    // mode 0
    float *Dr, *Di;
    int ldD;  // = M
    // mode 1
    int n, n_pad, k_exp;
    const int *flags, *rexp, *tile_active;
    float2 *Vhi, *Vlo;
    unsigned *delta;
};

// D[m][n] = sum_k A[m][k] B[n][k] over complex numbers for one 128 x 128 tile, with the K loop
// pipelined over kStages shared-memory slots.  Thread 0 issues both the TMA loads and the MMAs;
// all four warps then drain the two TMEM accumulators (Re, Im) in the epilogue.
__global__ void __launch_bounds__(128, 1)
    tc_gemm(const __grid_constant__ CUtensorMap tmAr, const __grid_constant__ CUtensorMap tmAi,
            const __grid_constant__ CUtensorMap tmBr, const __grid_constant__ CUtensorMap tmBi, int n_chunks,
            GemmEpi ep) {
    extern __shared__ uint8_t smem_raw[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m_tile = blockIdx.x, n_tile = blockIdx.y;
    if (ep.mode == 1 && ep.tile_active[n_tile] == 0) return;  // every column of this tile is done

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *extra = smem + kStages * kStageBytes;
    uint64_t *full = (uint64_t *)extra;          // [kStages]
    uint64_t *empty = full + kStages;            // [kStages]
    uint64_t *accb = empty + kStages;            // [1]
    uint32_t *tmem_slot = (uint32_t *)(accb + 1);
    int *abort_flag = (int *)(tmem_slot + 1);
    float *col_scale = (float *)(abort_flag + 1);  // [128]
    int *col_flag = (int *)(col_scale + kTileN);   // [128]
    unsigned *col_dmax = (unsigned *)(col_flag + kTileN);  // [128]

    if (warp == 0) {
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
        mbar_init(smem_u32(accb), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (ep.mode == 1) {
        const int64_t t = (int64_t)n_tile * kTileN + tid;
        int f = ep.flags[t];
        col_flag[tid] = f;
        col_scale[tid] = (f & kActive) ? pow2f(-ep.k_exp - ep.rexp[t]) : 0.0f;
        col_dmax[tid] = 0u;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t tDr = tmem, tDi = tmem + kTileN;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t sbase = smem_u32(smem);
            const int m0 = m_tile * kTileM, n0 = n_tile * kTileN;
            auto issue = [&](int chunk, int slot) {
                const uint32_t st = sbase + slot * kStageBytes;
                const uint32_t bar = smem_u32(&full[slot]);
                mbar_expect_tx(bar, kStageBytes);
                const int k = chunk * kChunkK;
                tma_load_2d(st, &tmAr, bar, k, m0);
                tma_load_2d(st + kTileBytes, &tmAi, bar, k, m0);
                tma_load_2d(st + 2 * kTileBytes, &tmBr, bar, k, n0);
                tma_load_2d(st + 3 * kTileBytes, &tmBi, bar, k, n0);
            };
            const uint32_t id_pos = idesc_f16(kTileM, kTileN, 0), id_neg = idesc_f16(kTileM, kTileN, 1);
            int issued = 0, consumed = 0;
            for (; issued < kStages && issued < n_chunks; ++issued) issue(issued, issued);
            bool ok = true;
            for (int c = 0; c < n_chunks && ok; ++c) {
                const int s = c % kStages;
                if (!mbar_wait(smem_u32(&full[s]), (c / kStages) & 1)) {
                    ok = false;
                    break;
                }
                consumed = c + 1;
                tc_fence_after();
                const uint32_t st = sbase + s * kStageBytes;
#pragma unroll
                for (int kk = 0; kk < kChunkK / 16; ++kk) {
                    const uint64_t ar = sw128_desc(st + kk * 32), ai = sw128_desc(st + kTileBytes + kk * 32);
                    const uint64_t br = sw128_desc(st + 2 * kTileBytes + kk * 32);
                    const uint64_t bi = sw128_desc(st + 3 * kTileBytes + kk * 32);
                    const uint32_t first = (c | kk) != 0;
                    umma_f16(tDr, ar, br, id_pos, first);  // Re += Kr rr
                    umma_f16(tDr, ai, bi, id_neg, 1u);     // Re -= Ki ri
                    umma_f16(tDi, ar, bi, id_pos, first);  // Im += Kr ri
                    umma_f16(tDi, ai, br, id_pos, 1u);     // Im += Ki rr
                }
                umma_commit(smem_u32(&empty[s]));
                const int refill = c - 1 + kStages;  // reuse the slot of chunk c-1
                if (c >= 1 && refill < n_chunks) {
                    const int sp = (c - 1) % kStages;
                    if (!mbar_wait(smem_u32(&empty[sp]), ((c - 1) / kStages) & 1)) {
                        ok = false;
                        break;
                    }
                    issue(refill, sp);
                    ++issued;
                }
            }
            umma_commit(smem_u32(accb));
            if (!ok) {
                *abort_flag = 1;
                atomicExch(ep.err, 1);
                // Let copies still in flight land before the CTA leaves (bounded).
                for (int c = consumed; c < issued; ++c) mbar_wait(smem_u32(&full[c % kStages]), (c / kStages) & 1);
            }
        }
        __syncwarp();
    }
    const bool acc_ok = mbar_wait(smem_u32(accb), 0);
    if (!acc_ok) atomicExch(ep.err, 1);
    tc_fence_after();
    __syncthreads();
    const bool run = acc_ok && *(volatile int *)abort_flag == 0;
    if (run) {
        const int row = warp * 32 + lane;  // TMEM lane = row of the tile
        const uint32_t lane_off = (uint32_t)(warp * 32) << 16;
        const int m = m_tile * kTileM + row;
        for (int cb = 0; cb < kTileN / 32; ++cb) {
            uint32_t vr[32], vi[32];
            tmem_ld32(tDr + lane_off + cb * 32, vr);
            tmem_ld32(tDi + lane_off + cb * 32, vi);
            tmem_wait_ld();
            if (ep.mode == 0) {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int64_t nn = (int64_t)n_tile * kTileN + cb * 32 + q;
                    ep.Dr[nn * ep.ldD + m] = __uint_as_float(vr[q]);
                    ep.Di[nn * ep.ldD + m] = __uint_as_float(vi[q]);
                }
            } else {
                // Update V of this lane's bus for the 32 columns (all loads first, then the
                // stores), then a transposed butterfly max over the warp: after 31 shuffles lane l
                // holds max_rows |dV| of column cb*32 + l.
                float2 old[32];
                float mag[32];
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int c = cb * 32 + q;
                    const int f = col_flag[c];
                    const bool act = (f & kActive) && m < ep.n;
                    const int64_t k = ((int64_t)n_tile * kTileN + c) * ep.n_pad + m;
                    const float2 *src = (f & kAnchored) ? ep.Vlo : ep.Vhi;  // anchored: V_ref stays fixed
                    old[q] = act ? src[k] : make_float2(0.0f, 0.0f);
                }
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int c = cb * 32 + q;
                    const int f = col_flag[c];
                    const bool act = (f & kActive) && m < ep.n;
                    const float sc = col_scale[c];
                    const float dr = __uint_as_float(vr[q]) * sc, di = __uint_as_float(vi[q]) * sc;
                    float dmag = 0.0f;
                    if (act) {
                        const int64_t k = ((int64_t)n_tile * kTileN + c) * ep.n_pad + m;
                        float2 *dst = (f & kAnchored) ? ep.Vlo : ep.Vhi;
                        dst[k] = make_float2(old[q].x + dr, old[q].y + di);
                        dmag = sqrtf(dr * dr + di * di);
                        if (dmag != dmag) dmag = __int_as_float(0x7f800000);  // NaN -> +inf
                    }
                    mag[q] = dmag;
                }
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) {
                    const bool upper = (lane & off) != 0;
#pragma unroll
                    for (int j = 0; j < off; ++j) {
                        const float send = upper ? mag[j] : mag[j + off];
                        const float keep = upper ? mag[j + off] : mag[j];
                        mag[j] = fmaxf(keep, __shfl_xor_sync(0xffffffffu, send, off));
                    }
                }
                if (mag[0] > 0.0f) atomicMax(&col_dmax[cb * 32 + lane], __float_as_uint(mag[0]));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (run && ep.mode == 1) {
        const unsigned d = col_dmax[tid];
        if (d) atomicMax(&ep.delta[(int64_t)n_tile * kTileN + tid], d);
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// ------------------------------------------------------------------------------------------
// Host helpers
// ------------------------------------------------------------------------------------------
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

// A [rows][inner] fp16 matrix read in (128 rows x 64 elements) boxes, 128-byte swizzle.
bool make_map(CUtensorMap *map, const void *base, uint64_t inner, uint64_t rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {inner * 2};
    cuuint32_t box[2] = {(cuuint32_t)kChunkK, (cuuint32_t)kTileM};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool gemm_attr_set = false;
tpf_status prepare_gemm() {
    if (!gemm_attr_set) {
        TPF_CK(cudaFuncSetAttribute(tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGemmSmem));
        gemm_attr_set = true;
    }
    return TPF_OK;
}

// Radial feeders stage two n_pad-long float2 rows per warp in shared memory; the block takes as
// many warps (columns) as fit in ~96 KB so that two blocks share an SM.
template <int BPL>
tpf_status launch_prologue(const PrologueArgs &a, cudaStream_t st) {
    static bool attr = false;
    const size_t per_warp = a.radial ? (size_t)2 * a.n_pad * sizeof(float2) : 0;
    int warps = per_warp ? (int)((96 * 1024) / per_warp) : 16;
    warps = warps < 1 ? 1 : (warps > 16 ? 16 : warps);
    const size_t smem = per_warp * warps;
    if (!attr) {
        TPF_CK(cudaFuncSetAttribute(mx_prologue<BPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
    }
    const int64_t blocks = (a.cols + warps - 1) / warps;
    mx_prologue<BPL><<<(unsigned)blocks, 32 * warps, smem, st>>>(a);
    return TPF_OK;
}

}  // namespace

tpf_status selftest_gemm(int M, int N, int K, const void *Ar, const void *Ai, const void *Br, const void *Bi, float *Dr,
                         float *Di, cudaStream_t st) {
    tpf_status rs = prepare_gemm();
    if (rs != TPF_OK) return rs;
    CUtensorMap m[4];
    if (!make_map(&m[0], Ar, K, M) || !make_map(&m[1], Ai, K, M) || !make_map(&m[2], Br, K, N) ||
        !make_map(&m[3], Bi, K, N))
        return TPF_ECUDA;
    int *err = nullptr;
    TPF_CK(cudaMalloc(&err, sizeof(int)));
    TPF_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    GemmEpi ep{};
    ep.mode = 0;
    ep.err = err;
    ep.Dr = Dr;
    ep.Di = Di;
    ep.ldD = M;
    tc_gemm<<<dim3(M / kTileM, N / kTileN), 128, kGemmSmem, st>>>(m[0], m[1], m[2], m[3], K / kChunkK, ep);
    cudaError_t e = cudaGetLastError();
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(err);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    return herr ? TPF_ETIMEOUT : TPF_OK;
}

tpf_status solve_mixed(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters, double *mismatch,
                       const tpf_opts &o, cudaStream_t st) {
    const int n = h->dev.n, n_pad = h->dev.n_pad;
    if (n_pad > 2048) return TPF_EUNSUPPORTED;
    tpf_status rs = ensure_workspace(h, T, true);
    if (rs != TPF_OK) return rs;
    rs = prepare_gemm();
    if (rs != TPF_OK) return rs;
    Workspace &w = h->ws;
    const int64_t cols = round_up(T, kTileN);
    CUtensorMap maps[4];
    if (!make_map(&maps[0], h->dev.Kr16, n_pad, n_pad) || !make_map(&maps[1], h->dev.Ki16, n_pad, n_pad) ||
        !make_map(&maps[2], w.Rr16, n_pad, cols) || !make_map(&maps[3], w.Ri16, n_pad, cols))
        return TPF_ECUDA;
    int64_t launches = 0, gemm_cols = 0;
    KernelTimer timer(o.profile != 0, st);
    TPF_CK(cudaMemsetAsync(w.counters, 0, sizeof(int) * 8, st));
    timer.begin(KernelTimer::kOther);
    mx_pack<<<(unsigned)cols, 256, 0, st>>>(T, n, n_pad, (const double2 *)S,
                                             o.start == TPF_START_GIVEN ? (const double2 *)V : nullptr, w.Shi, w.Slo,
                                             w.Vhi, w.Vlo, w.flags, w.iters, w.delta_bits, w.dprev);
    timer.end();
    ++launches;
    TPF_CK(cudaGetLastError());

    PrologueArgs pa{};
    pa.cols = cols;
    pa.n = n;
    pa.n_pad = n_pad;
    pa.max_iter = o.max_iter;
    pa.tol = (float)o.tol;
    pa.switch_tol = (float)o.switch_tol;
    pa.vs_f = make_float2((float)h->net.vs_re, (float)h->net.vs_im);
    {
        float rh = (float)h->net.vs_re, ih = (float)h->net.vs_im;
        pa.vs_dd = c2{{rh, (float)(h->net.vs_re - (double)rh)}, {ih, (float)(h->net.vs_im - (double)ih)}};
    }
    pa.Vhi = w.Vhi;
    pa.Vlo = w.Vlo;
    pa.Shi = w.Shi;
    pa.Slo = w.Slo;
    pa.RefHi = w.RefHi;
    pa.RefLo = w.RefLo;
    pa.dprev = w.dprev;
    pa.given = o.start == TPF_START_GIVEN;
    pa.radial = h->dev.radial ? 1 : 0;
    pa.par = h->dev.par;
    pa.ch_ptr = h->dev.ch_ptr;
    pa.ch = h->dev.ch;
    pa.ypar = h->dev.ypar;
    pa.row_ptr = h->dev.row_ptr;
    pa.nbr = h->dev.nbr;
    pa.y = h->dev.y2f;
    pa.flags = w.flags;
    pa.iters = w.iters;
    pa.rexp = w.rexp;
    pa.tile_active = w.tile_active;
    pa.counters = w.counters;
    pa.delta = w.delta_bits;
    pa.Rr = (__half *)w.Rr16;
    pa.Ri = (__half *)w.Ri16;

    GemmEpi ep{};
    ep.mode = 1;
    ep.err = w.counters + kCntError;
    ep.n = n;
    ep.n_pad = n_pad;
    ep.k_exp = h->dev.k_exp;
    ep.flags = w.flags;
    ep.rexp = w.rexp;
    ep.tile_active = w.tile_active;
    ep.Vhi = w.Vhi;
    ep.Vlo = w.Vlo;
    ep.delta = w.delta_bits;
    const dim3 ggrid(n_pad / kTileM, (unsigned)(cols / kTileN));

    int sweeps = 0, precise_sweeps = 0;
    for (int s = 0; s <= o.max_iter; ++s) {
        TPF_CK(cudaMemsetAsync(w.tile_active, 0, sizeof(int) * (cols / kTileN), st));
        TPF_CK(cudaMemsetAsync(w.counters, 0, sizeof(int) * 2, st));  // active, precise
        pa.sweep = s;
        const int bpl = n_pad / 32;
        timer.begin(KernelTimer::kResidual);
        if (bpl <= 4) rs = launch_prologue<4>(pa, st);
        else if (bpl <= 8) rs = launch_prologue<8>(pa, st);
        else if (bpl <= 16) rs = launch_prologue<16>(pa, st);
        else if (bpl <= 32) rs = launch_prologue<32>(pa, st);
        else rs = launch_prologue<64>(pa, st);
        timer.end();
        if (rs != TPF_OK) return rs;
        ++launches;
        TPF_CK(cudaGetLastError());
        TPF_CK(cudaMemcpyAsync(w.counters_host, w.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
        TPF_CK(cudaStreamSynchronize(st));
        if (w.counters_host[kCntError]) return TPF_ETIMEOUT;
        if (w.counters_host[kCntActive] == 0) break;
        if (w.counters_host[kCntPrecise] > 0) ++precise_sweeps;
        gemm_cols += w.counters_host[kCntActive];
        timer.begin(KernelTimer::kGemm);
        tc_gemm<<<ggrid, 128, kGemmSmem, st>>>(maps[0], maps[1], maps[2], maps[3], n_pad / kChunkK, ep);
        timer.end();
        ++launches;
        ++sweeps;
        TPF_CK(cudaGetLastError());
    }
    timer.begin(KernelTimer::kOther);
    mx_finish<<<(unsigned)((T * 32 + 255) / 256), 256, 0, st>>>(T, n, n_pad, o.max_iter, w.flags, w.iters, w.Vhi,
                                                               w.Vlo, w.Shi, w.Slo, h->dev.row_ptr, h->dev.nbr,
                                                               h->dev.y2f, pa.vs_dd, (double2 *)V, iters, mismatch);
    timer.end();
    ++launches;
    TPF_CK(cudaGetLastError());
    TPF_CK(cudaMemcpyAsync(w.counters_host, w.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
    TPF_CK(cudaStreamSynchronize(st));
    h->stats.sweeps = sweeps;
    h->stats.precise_sweeps = precise_sweeps;
    h->stats.kernel_launches = launches;
    h->stats.converged = w.counters_host[kCntConverged];
    h->stats.gemm_launches = sweeps;
    h->stats.gemm_columns = gemm_cols;
    h->stats.gemm_ms = timer.total_ms(KernelTimer::kGemm);
    h->stats.residual_ms = timer.total_ms(KernelTimer::kResidual);
    h->stats.other_ms = timer.total_ms(KernelTimer::kOther);
    if (w.counters_host[kCntError]) return TPF_ETIMEOUT;
    return h->stats.converged == T ? TPF_OK : TPF_ENOCONV;
}

}  // namespace tpf
