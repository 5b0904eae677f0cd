// The per-sweep residual kernel of the mixed path (Eq. 1 residual, Algorithm 1 loop control), and
// its final-output variant.
//
// One block of 128 kCPB threads handles kCPB consecutive columns, so the per-bus network data
// (parent, branch admittance, children) is loaded once and used for all of them.  In a sweep, thread c
// (c < kCPB) first takes column c's decision for the step the last sweep applied: stop at
// max |dV| <= tol (the per-column form of Algorithm 1's test), give up at max_iter or on a
// non-finite step, and anchor the column once its step is small.  The block then forms rho_i:
//
//   before anchoring   rho = conj(S ./ V) + (Y v)         FP32, from the high words of V
//   anchoring sweep    V_ref <- fl(V), rho(V_ref) in double-float, stored
//   after anchoring    rho = rho(V_ref) + [rho(V_ref + d) - rho(V_ref)], the bracket in FP32
//
// with (Y v)_i = sum_j y_ij (V_i - V_j) over the branches at i (V_slack = v_s).  On a radial
// feeder this is conj(S_i/V_i) - J_i + sum_{children c} J_c with J_c = y_c (V_parent(c) - V_c);
// the columns' V (or d = V - V_ref) are staged in shared memory so the parent and children
// gathers stay on chip.  Finally rho is written as the fp16 B operand 2^e rho with the column's
// largest component in [2^13, 2^14) (e per column, exact to undo).
//
// The final variant evaluates rho once more at the returned V (same formulas, no decision) and
// writes V as complex128, the iteration counts and the mismatch max_i |V_i| |rho_i|
// (= max_i |V_i conj((Y v)_i) + S_i|).
#include "tpf_dd.cuh"

namespace tpf {

namespace {

// Columns per block (the per-bus network data is loaded once for all of them); 128 threads per
// column.
#ifndef TPF_RES_CPB
#define TPF_RES_CPB 1
#endif
constexpr int kCPB = TPF_RES_CPB;
constexpr int kResThreads = 128 * kCPB;

struct FinalArgs {
    int64_t T;
    double2 *V_out;
    int32_t *iters_out;
    double *mismatch_out;
    int *tile_done;
};

template <bool FINAL>
__global__ void __launch_bounds__(kResThreads) mx_residual(PrologueArgs a, FinalArgs fo) {
    extern __shared__ float2 rsm[];
    float2 *vb = rsm;                      // [kCPB][n_pad] staged V or d (radial feeders)
    float2 *rb = rsm + kCPB * a.n_pad;     // [kCPB][n_pad] rho
    __shared__ int s_f[kCPB], s_anchor[kCPB];
    __shared__ float s_red[kResThreads / 32][kCPB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * kCPB;
    const int64_t tlim = FINAL ? fo.T : a.cols;
    if (tid < kCPB) {
        const int64_t t = t0 + tid;
        int f = t < tlim ? a.flags[t] : 0, anchor = 0;
        if (FINAL) {
            // Every real column gets outputs; the residual uses the column's current mode.
            if (t < tlim) f |= kActive;
        } else if (a.sweep > 0 && (f & kActive)) {
            const float d = __uint_as_float(a.delta[t]);
            const float dp = __uint_as_float(a.dprev[t]);
            const int it = a.iters[t] + 1;
            // A column that stops keeps kAnchored: the final pass evaluates its residual at
            // V_ref + (V - V_ref) with the stored rho(V_ref).
            if (d <= a.tol) {
                f = kDone | (f & kAnchored);
            } else if (it >= a.max_iter || !(d < 1e30f)) {
                f &= kAnchored;
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
        s_f[tid] = f;
        s_anchor[tid] = anchor;
    }
    __syncthreads();
    int fl[kCPB];
    bool anch[kCPB], live = false, any_anchor = false;
#pragma unroll
    for (int c = 0; c < kCPB; ++c) {
        fl[c] = s_f[c];
        anch[c] = s_anchor[c] != 0;
        live |= (fl[c] & kActive) != 0;
        any_anchor |= anch[c];
    }
    if (!live) return;

    // Columns anchored in this sweep: re-base V, then rho(V_ref) in double-float (any network).
    if (any_anchor) {
#pragma unroll 1
        for (int c = 0; c < kCPB; ++c) {
            if (!anch[c]) continue;
            const int64_t base = (t0 + c) * a.n_pad;
            float2 *vh = a.Vhi + base, *vl = a.Vlo + base;
            for (int i = tid; i < a.n; i += kResThreads) {
                const float2 h = vh[i], l = vl[i];
                const f2 re = two_sum(h.x, l.x), im = two_sum(h.y, l.y);
                vh[i] = make_float2(re.h, im.h);
                vl[i] = make_float2(re.l, im.l);
            }
        }
        __syncthreads();
#pragma unroll 1
        for (int c = 0; c < kCPB; ++c) {
            if (!anch[c]) continue;
            const int64_t base = (t0 + c) * a.n_pad;
            float2 *vh = a.Vhi + base, *vl = a.Vlo + base;
            const float2 *sh = a.Shi + base;
            for (int i = tid; i < a.n; i += kResThreads) {
                const c2 ref = residual_dd(i, vh, nullptr, sh, a.Slo + base, a.row_ptr, a.nbr, a.y, a.vs_dd);
                a.RefHi[base + i] = make_float2(ref.re.h, ref.im.h);
                a.RefLo[base + i] = make_float2(ref.re.l, ref.im.l);
                const float2 cr = residual_corr(i, vh, vl, sh, a.row_ptr, a.nbr, a.y);
                const f2 sr = two_sum(ref.re.h, cr.x), si = two_sum(ref.im.h, cr.y);
                rb[c * a.n_pad + i] = make_float2(sr.h + (sr.l + ref.re.l), si.h + (si.l + ref.im.l));
            }
        }
    }

    // All other live columns.
    bool tree_col[kCPB];
#pragma unroll
    for (int c = 0; c < kCPB; ++c) tree_col[c] = (fl[c] & kActive) && !anch[c];
    if (a.radial) {
#pragma unroll
        for (int c = 0; c < kCPB; ++c) {
            if (!tree_col[c]) continue;
            const int64_t base = (t0 + c) * a.n_pad;
            const float2 *src = (fl[c] & kAnchored) ? a.Vlo + base : a.Vhi + base;
            float2 *dst = vb + c * a.n_pad;
            for (int i = tid; i < a.n; i += kResThreads) dst[i] = src[i];
        }
        __syncthreads();
        for (int i = tid; i < a.n; i += kResThreads) {
            const int p = a.par[i];
            const float2 y = a.ypar[i];
            const int cb = a.ch_ptr[i], ce = a.ch_ptr[i + 1];
            float2 v[kCPB], acc[kCPB];
#pragma unroll
            for (int c = 0; c < kCPB; ++c) {
                acc[c] = make_float2(0.0f, 0.0f);
                v[c] = make_float2(0.0f, 0.0f);
                if (!tree_col[c]) continue;
                const bool anchored = (fl[c] & kAnchored) != 0;
                const int64_t base = (t0 + c) * a.n_pad;
                const float2 *v_c = vb + c * a.n_pad;
                v[c] = v_c[i];
                const float2 vp = p >= 0 ? v_c[p] : (anchored ? make_float2(0.0f, 0.0f) : a.vs_f);
                const float dr = vp.x - v[c].x, di = vp.y - v[c].y;
                const float2 s = a.Shi[base + i];
                const float2 loc = anchored ? delta_current(a.Vhi[base + i], v[c], s) : load_current_f32(v[c], s);
                acc[c] = make_float2(loc.x - (y.x * dr - y.y * di), loc.y - (y.x * di + y.y * dr));  // - J_i
            }
            for (int e = cb; e < ce; ++e) {  // + J_k = y_k (V_i - V_k) for the children k
                const int k = a.ch[e];
                const float2 yk = a.ypar[k];
#pragma unroll
                for (int c = 0; c < kCPB; ++c) {
                    if (!tree_col[c]) continue;
                    const float2 vk = vb[c * a.n_pad + k];
                    const float dr = v[c].x - vk.x, di = v[c].y - vk.y;
                    acc[c].x += yk.x * dr - yk.y * di;
                    acc[c].y += yk.x * di + yk.y * dr;
                }
            }
#pragma unroll
            for (int c = 0; c < kCPB; ++c) {
                if (!tree_col[c]) continue;
                float ar = acc[c].x, ai = acc[c].y;
                if (fl[c] & kAnchored) {
                    const int64_t base = (t0 + c) * a.n_pad;
                    const float2 h = a.RefHi[base + i], l = a.RefLo[base + i];
                    const f2 sr = two_sum(h.x, ar), si = two_sum(h.y, ai);
                    ar = sr.h + (sr.l + l.x);
                    ai = si.h + (si.l + l.y);
                }
                rb[c * a.n_pad + i] = make_float2(ar, ai);
            }
        }
    } else {
#pragma unroll 1
        for (int c = 0; c < kCPB; ++c) {
            if (!tree_col[c]) continue;
            const int64_t base = (t0 + c) * a.n_pad;
            const float2 *vh = a.Vhi + base, *vl = a.Vlo + base, *sh = a.Shi + base;
            for (int i = tid; i < a.n; i += kResThreads) {
                float2 r;
                if (fl[c] & kAnchored) {
                    const float2 cr = residual_corr(i, vh, vl, sh, a.row_ptr, a.nbr, a.y);
                    const float2 h = a.RefHi[base + i], l = a.RefLo[base + i];
                    const f2 sr = two_sum(h.x, cr.x), si = two_sum(h.y, cr.y);
                    r = make_float2(sr.h + (sr.l + l.x), si.h + (si.l + l.y));
                } else {
                    r = residual_f32(i, vh, sh, a.row_ptr, a.nbr, a.y, a.vs_f);
                }
                rb[c * a.n_pad + i] = r;
            }
        }
    }
    __syncthreads();

    if constexpr (FINAL) {
        // Outputs: V = Vhi + Vlo as complex128, iteration counts, mismatch max_i |V_i| |rho_i|.
        float m[kCPB];
#pragma unroll
        for (int c = 0; c < kCPB; ++c) {
            m[c] = 0.0f;
            const int64_t t = t0 + c;
            if (!(fl[c] & kActive)) continue;
            const int64_t base = t * a.n_pad;
            for (int i = tid; i < a.n; i += kResThreads) {
                const float2 h = a.Vhi[base + i], l = a.Vlo[base + i];
                fo.V_out[t * a.n + i] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
                const float2 r = rb[c * a.n_pad + i];
                const float vm = sqrtf((h.x + l.x) * (h.x + l.x) + (h.y + l.y) * (h.y + l.y));
                float mv = vm * sqrtf(r.x * r.x + r.y * r.y);
                if (mv != mv) mv = __int_as_float(0x7f800000);  // a NaN mismatch reports as +inf
                m[c] = fmaxf(m[c], mv);
            }
        }
#pragma unroll
        for (int c = 0; c < kCPB; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m[c] = fmaxf(m[c], __shfl_xor_sync(0xffffffffu, m[c], o));
            if (lane == 0) s_red[warp][c] = m[c];
        }
        __syncthreads();
        if (tid < kCPB) {
            const int64_t t = t0 + tid;
            if (t < fo.T) {
                float mm = s_red[0][tid];
                for (int w = 1; w < kResThreads / 32; ++w) mm = fmaxf(mm, s_red[w][tid]);
                const bool done = (s_f[tid] & kDone) != 0;
                if (fo.mismatch_out) fo.mismatch_out[t] = (double)mm;
                if (fo.iters_out) fo.iters_out[t] = done ? a.iters[t] : -a.max_iter;
                if (done) atomicAdd(&fo.tile_done[t / kTileN], 1);
            }
        }
    } else {
    // Per-column scale and the fp16 operand.
    float m[kCPB];
#pragma unroll
    for (int c = 0; c < kCPB; ++c) {
        m[c] = 0.0f;
        if (!(fl[c] & kActive)) continue;
        for (int i = tid; i < a.n; i += kResThreads) {
            const float2 r = rb[c * a.n_pad + i];
            m[c] = fmaxf(m[c], fmaxf(fabsf(r.x), fabsf(r.y)));
        }
    }
#pragma unroll
    for (int c = 0; c < kCPB; ++c) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[c] = fmaxf(m[c], __shfl_xor_sync(0xffffffffu, m[c], o));
        if (lane == 0) s_red[warp][c] = m[c];
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kCPB; ++c) {
        if (!(fl[c] & kActive)) continue;
        float mm = s_red[0][c];
#pragma unroll
        for (int w = 1; w < kResThreads / 32; ++w) mm = fmaxf(mm, s_red[w][c]);
        int e = 0;
        if (mm > 0.0f) {
            frexpf(mm, &e);
            e = 14 - e;
        }
        if (e > 120) e = 120;
        const float sc = pow2f(e);
        const int64_t t = t0 + c, base = t * a.n_pad;
        __half *Rr = a.Rr + base, *Ri = a.Ri + base;
        for (int i = tid; i < a.n_pad; i += kResThreads) {
            const float2 r = i < a.n ? rb[c * a.n_pad + i] : make_float2(0.0f, 0.0f);
            Rr[i] = __float2half_rn(r.x * sc);
            Ri[i] = __float2half_rn(r.y * sc);
        }
        if (tid == 0) {
            a.rexp[t] = e;
            atomicAdd(&a.tile_active[t / kTileN], 1);  // iterating columns of this 128-column tile
            if (anch[c] && a.counters[kCntPrecise] == 0) atomicExch(&a.counters[kCntPrecise], 1);
        }
    }
    }  // FINAL
}

template <bool FINAL>
tpf_status launch(const PrologueArgs &a, const FinalArgs &fo, int64_t cols, cudaStream_t st) {
    static std::atomic<uint64_t> attr{0};
    const size_t smem = (size_t)2 * kCPB * a.n_pad * sizeof(float2);
    if (!once_per_device(attr, [] {
            return cudaFuncSetAttribute(mx_residual<FINAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
                   cudaSuccess;
        }))
        return TPF_ECUDA;
    const int64_t blocks = (cols + kCPB - 1) / kCPB;
    mx_residual<FINAL><<<(unsigned)blocks, kResThreads, smem, st>>>(a, fo);
    if (cudaGetLastError() != cudaSuccess) return TPF_ECUDA;
    return TPF_OK;
}

}  // namespace

tpf_status launch_residual(const PrologueArgs &a, cudaStream_t st) {
    return launch<false>(a, FinalArgs{}, a.cols, st);
}

tpf_status launch_final(const PrologueArgs &a, int64_t T, void *V_out, int32_t *iters_out, double *mismatch_out,
                        int *tile_done, cudaStream_t st) {
    FinalArgs fo{T, (double2 *)V_out, iters_out, mismatch_out, tile_done};
    return launch<true>(a, fo, T, st);
}

}  // namespace tpf
