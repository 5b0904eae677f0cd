// The per-sweep residual kernel of the mixed path (Eq. 1 residual, Algorithm 1 loop control).
//
// One 128-thread block per column.  Thread 0 first takes the column's decision for the step the
// last sweep applied: stop at max |dV| <= tol (the per-column form of Algorithm 1's test), give
// up at max_iter or on a non-finite step, and anchor the column once its step is small (see
// below).  The block then forms rho_i for every bus i:
//
//   before anchoring   rho = conj(S ./ V) + (Y v)         FP32, from the high words of V
//   anchoring sweep    V_ref <- fl(V), rho(V_ref) in double-float, stored
//   after anchoring    rho = rho(V_ref) + [rho(V_ref + d) - rho(V_ref)], the bracket in FP32
//
// with (Y v)_i = sum_j y_ij (V_i - V_j) over the branches at i (V_slack = v_s).  On a radial
// feeder this is conj(S_i/V_i) - J_i + sum_{children c} J_c with J_c = y_c (V_parent(c) - V_c);
// the column's V (or d = V - V_ref) is staged in shared memory so the parent and children
// gathers stay on chip.  Finally rho is written as the fp16 B operand 2^e rho with the column's
// largest component in [2^13, 2^14) (e per column, exact to undo).
#include "tpf_dd.cuh"

namespace tpf {

namespace {

constexpr int kResThreads = 128;

__global__ void __launch_bounds__(kResThreads) mx_residual(PrologueArgs a) {
    extern __shared__ float2 rsm[];
    float2 *vb = rsm;            // [n_pad] staged V or d (radial feeders)
    float2 *rb = rsm + a.n_pad;  // [n_pad] rho
    __shared__ int s_f, s_anchor;
    __shared__ float s_red[kResThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t = blockIdx.x;
    if (tid == 0) {
        int f = a.flags[t], anchor = 0;
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
                    anchor = 1;
                    f = (f | kAnchored) & ~kBlind;
                }
            }
            a.iters[t] = it;
            a.flags[t] = f;
            a.delta[t] = 0u;
            a.dprev[t] = __float_as_uint(d);
        } else if (a.sweep == 0 && a.given && (f & kActive)) {
            anchor = 1;
            f |= kAnchored | kBlind;
            a.flags[t] = f;
        }
        s_f = f;
        s_anchor = anchor;
    }
    __syncthreads();
    const int f = s_f;
    const bool anchor = s_anchor != 0;
    if (!(f & kActive)) return;
    const bool anchored = (f & kAnchored) != 0;
    const int64_t base = t * a.n_pad;
    float2 *vh = a.Vhi + base, *vl = a.Vlo + base;
    const float2 *sh = a.Shi + base;
    float2 *rh = a.RefHi + base, *rl = a.RefLo + base;
    if (anchor) {  // re-base: Vhi <- fl(Vhi + Vlo), Vlo <- the exact remainder
        for (int i = tid; i < a.n; i += kResThreads) {
            const float2 h = vh[i], l = vl[i];
            const f2 re = two_sum(h.x, l.x), im = two_sum(h.y, l.y);
            vh[i] = make_float2(re.h, im.h);
            vl[i] = make_float2(re.l, im.l);
        }
        __syncthreads();
    }
    float m = 0.0f;
    if (a.radial && !anchor) {
        const float2 *src = anchored ? vl : vh;
        const float2 vsrc = anchored ? make_float2(0.0f, 0.0f) : a.vs_f;
        for (int i = tid; i < a.n_pad; i += kResThreads) vb[i] = i < a.n ? src[i] : make_float2(0.0f, 0.0f);
        __syncthreads();
#pragma unroll 2
        for (int i = tid; i < a.n; i += kResThreads) {
            const float2 v = vb[i];
            const int p = a.par[i];
            const float2 vp = p >= 0 ? vb[p] : vsrc;
            const float2 y = a.ypar[i];
            float dr = vp.x - v.x, di = vp.y - v.y;
            const float2 loc = anchored ? delta_current(vh[i], v, sh[i]) : load_current_f32(v, sh[i]);
            float ar = loc.x - (y.x * dr - y.y * di);  // - J_i
            float ai = loc.y - (y.x * di + y.y * dr);
            for (int e = a.ch_ptr[i]; e < a.ch_ptr[i + 1]; ++e) {  // + J_c = y_c (V_i - V_c)
                const int c = a.ch[e];
                const float2 yc = a.ypar[c], vc = vb[c];
                dr = v.x - vc.x;
                di = v.y - vc.y;
                ar += yc.x * dr - yc.y * di;
                ai += yc.x * di + yc.y * dr;
            }
            if (anchored) {
                const float2 h = rh[i], l = rl[i];
                const f2 sr = two_sum(h.x, ar), si = two_sum(h.y, ai);
                ar = sr.h + (sr.l + l.x);
                ai = si.h + (si.l + l.y);
            }
            rb[i] = make_float2(ar, ai);
            m = fmaxf(m, fmaxf(fabsf(ar), fabsf(ai)));
        }
    } else if (anchored) {
        for (int i = tid; i < a.n; i += kResThreads) {
            c2 ref;
            if (anchor) {
                ref = residual_dd(i, vh, nullptr, sh, a.Slo + base, a.row_ptr, a.nbr, a.y, a.vs_dd);
                rh[i] = make_float2(ref.re.h, ref.im.h);
                rl[i] = make_float2(ref.re.l, ref.im.l);
            } else {
                const float2 h = rh[i], l = rl[i];
                ref = {{h.x, l.x}, {h.y, l.y}};
            }
            const float2 c = residual_corr(i, vh, vl, sh, a.row_ptr, a.nbr, a.y);
            const f2 sr = two_sum(ref.re.h, c.x), si = two_sum(ref.im.h, c.y);
            const float ar = sr.h + (sr.l + ref.re.l), ai = si.h + (si.l + ref.im.l);
            rb[i] = make_float2(ar, ai);
            m = fmaxf(m, fmaxf(fabsf(ar), fabsf(ai)));
        }
    } else {
        for (int i = tid; i < a.n; i += kResThreads) {
            const float2 r = residual_f32(i, vh, sh, a.row_ptr, a.nbr, a.y, a.vs_f);
            rb[i] = r;
            m = fmaxf(m, fmaxf(fabsf(r.x), fabsf(r.y)));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_red[warp] = m;
    __syncthreads();
    m = s_red[0];
#pragma unroll
    for (int w = 1; w < kResThreads / 32; ++w) m = fmaxf(m, s_red[w]);
    int e = 0;
    if (m > 0.0f) {
        frexpf(m, &e);
        e = 14 - e;
    }
    if (e > 120) e = 120;
    const float sc = pow2f(e);
    __half *Rr = a.Rr + base, *Ri = a.Ri + base;
    for (int i = tid; i < a.n_pad; i += kResThreads) {
        const float2 r = i < a.n ? rb[i] : make_float2(0.0f, 0.0f);
        Rr[i] = __float2half_rn(r.x * sc);
        Ri[i] = __float2half_rn(r.y * sc);
    }
    if (tid == 0) {
        a.rexp[t] = e;
        atomicAdd(&a.tile_active[t / kTileN], 1);  // iterating columns of this 128-column tile
        if (anchor && a.counters[kCntPrecise] == 0) atomicExch(&a.counters[kCntPrecise], 1);
    }
}

}  // namespace

tpf_status launch_residual(const PrologueArgs &a, cudaStream_t st) {
    static bool attr = false;
    const size_t smem = (size_t)2 * a.n_pad * sizeof(float2);
    if (!attr) {
        if (cudaFuncSetAttribute(mx_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess) {
            cudaGetLastError();
            return TPF_ECUDA;
        }
        attr = true;
    }
    mx_residual<<<(unsigned)a.cols, kResThreads, smem, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return TPF_ECUDA;
    return TPF_OK;
}

}  // namespace tpf
