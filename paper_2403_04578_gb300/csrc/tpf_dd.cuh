// Device helpers of the mixed-precision path: double-float arithmetic and the residual
// rho(V) = (Y_dd V + Y_ds v_s) + conj(S ./ V) of Eq. 1 in its three precisions.
#pragma once

#include <cuda_fp16.h>

#include "tpf_internal.h"

namespace tpf {

// A double-float value is hi + lo with |lo| <= ulp(hi)/2.  The arithmetic is the classical
// error-free-transformation method: Knuth's TwoSum (and Dekker's FastTwoSum when |a| >= |b|) for
// the exact rounding error of a sum, the FMA-based TwoProduct (p = fl(a b), e = fma(a, b, -p)) for
// that of a product, and one Newton step q1 + q1 (1 - b q1) for a reciprocal; the double-float
// operations combine them as in Dekker's and Shewchuk's double-length arithmetic.  Every operation
// uses explicitly rounded intrinsics so that the compiler cannot fuse or reorder the error terms.
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

// rho_i in double-float for bus i of the column whose V planes start at vh / vl, any network:
// (Y v)_i = sum_j y_ij (V_i - V_j) over the branches at bus i, V_slack = vs.
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

// conj(s / v) in FP32.
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

// rho_i in FP32 from the high words only (sweeps far from convergence), any network.
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

// rho(V_ref + d) - rho(V_ref) in FP32 for an anchored column (V_ref = vh, d = vl), any network:
//   sum_j y_ij (d_i - d_j)  +  conj(S/(V_ref + d)) - conj(S/V_ref).
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

// Arguments of the per-sweep residual kernel.
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

// Launch the residual kernel of one sweep (tpf_residual.cu).
tpf_status launch_residual(const PrologueArgs &a, cudaStream_t st);
// Final outputs of a solve: V (complex128 [T][n]), iteration counts, mismatch, and the converged
// columns counted per 128-column tile into tile_done (zeroed by the caller).
tpf_status launch_final(const PrologueArgs &a, int64_t T, void *V_out, int32_t *iters_out, double *mismatch_out,
                        int *tile_done, cudaStream_t st);

}  // namespace tpf
