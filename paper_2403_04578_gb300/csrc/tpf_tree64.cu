// Sparse tensor formulation in plain double precision (Sec. IV-B, Eq. 13-14, Algorithm 2).
//
// The same iterate as the mixed tree kernel and as Algorithm 1, V_{k+1} = K conj(S ./ V_k) + W,
// evaluated without K: on a radial feeder Y_dd factors without fill-in, and with the demand buses
// in depth-first preorder the substitution is two prefix sums per sweep,
//
//     L_q      = P[end_q - 1] - P[q - 1],     P = inclusive prefix sum of I = conj(S ./ V)
//     V_new,q  = v_s - (prefix sum at q of E),  E_q = z_q L_q - sum of z_b L_b over the b whose
//                                                   subtree range [b, end_b) ends at q
//
// (the path sum of the branch drops from the slack to q).  Every operation is FP64: this is the
// plain double-precision fixed-point iteration of the sparse form, with Algorithm 1's per-column
// stopping rule (max_i |V_{k+1,i} - V_{k,i}| <= tol, the first iterate that meets it is returned),
// so that it can stand beside the mixed-precision sparse path as a like-for-like FP64 reference.
//
// One block owns one column for its whole solve, with the slot layout of the mixed kernel
// (thread k owns depth-first positions k*bpt .. k*bpt + bpt - 1, position q at slot
// (q % bpt) * threads + q / bpt).  V and the thread's prefix values live in registers; shared
// memory holds S, z and one prefix array per slot (P in the first half of a sweep, the branch
// terms in ends-list order in the second), plus the range, ends-index and parent slots.  GB300
// issues FP64 at 1/64 of its FP32 rate, so this kernel is bound by the FP64 pipe.
#include <cstdint>

#include "tpf_internal.h"

namespace tpf {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxWarps64 = kTreeMaxThreads / 32;

struct Tree64Args {
    int n, max_iter;
    double tol2;     // tol squared: a step is compared squared
    double2 vs;      // slack voltage
    const int *col, *end, *par, *ecnt, *kidx;
    const double2 *z;      // [slot] branch impedance to the parent
    const double *zip;     // [3][n] (alpha_P, alpha_I, alpha_Z) by column, or null
    const double2 *S;      // [T][n]
    double2 *V;            // [T][n]; read first as V_0 when given
    int given;
    int32_t *iters_out;    // [T] or null
    double *mismatch_out;  // [T] or null
    int *counters;         // [kCntConverged] converged columns, [5] largest sweep count
};

__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double dabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
// max that returns NaN if either operand is NaN
__device__ __forceinline__ double dmax_nan(double m, double x) { return (m != m || x <= m) ? m : x; }

// Demand current of Eq. 3 in FP64: alpha_P conj(s / v) + alpha_I conj(s) + alpha_Z conj(s) v for
// the bus in column i (constant power, conj(s / v), without ZIP coefficients).
template <bool kZip>
__device__ __forceinline__ double2 demand64(double2 v, double2 s, const Tree64Args &g, int slot) {
    const double inv = 1.0 / dabs2(v);
    const double2 csv = make_double2(fma(s.x, v.x, s.y * v.y), fma(s.x, v.y, -s.y * v.x));  // conj(s) v
    const double2 c = make_double2(csv.x * inv, csv.y * inv);                             // conj(s / v)
    if (!kZip) return c;
    const int i = __ldg(g.col + slot), n = g.n;
    const double ap = __ldg(g.zip + i), ai = __ldg(g.zip + n + i), az = __ldg(g.zip + 2 * n + i);
    return make_double2(ap * c.x + ai * s.x + az * csv.x, ap * c.y - ai * s.y + az * csv.y);
}

// Exclusive scan over the block's threads (thread order) of one complex FP64 value; ends with all
// warp totals read, after one barrier.
__device__ __forceinline__ double2 block_scan64(double2 v, double2 *wt, int lane, int warp, int nw) {
    double2 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double ux = __shfl_up_sync(kFull, inc.x, o), uy = __shfl_up_sync(kFull, inc.y, o);
        if (lane >= o) inc = dadd(make_double2(ux, uy), inc);
    }
    const double ex = __shfl_up_sync(kFull, inc.x, 1), ey = __shfl_up_sync(kFull, inc.y, 1);
    if (lane == 31) wt[warp] = inc;
    __syncthreads();
    // Lane l scans the warp totals of warps 0..l; warp w takes lane w-1's sum.
    double2 t = lane < nw ? wt[lane] : make_double2(0.0, 0.0);
    for (int o = 1; o < nw; o <<= 1) {
        const double ux = __shfl_up_sync(kFull, t.x, o), uy = __shfl_up_sync(kFull, t.y, o);
        if (lane >= o) t = dadd(make_double2(ux, uy), t);
    }
    const int src = warp ? warp - 1 : 0;
    const double px = __shfl_sync(kFull, t.x, src), py = __shfl_sync(kFull, t.y, src);
    const double2 before = warp ? make_double2(px, py) : make_double2(0.0, 0.0);
    return dadd(before, lane ? make_double2(ex, ey) : make_double2(0.0, 0.0));
}

template <int kBPT>
__device__ __forceinline__ int next_slot64(int s, int th) {
    return s < (kBPT - 1) * th ? s + th : s - (kBPT - 1) * th + 1;
}

template <int kBPT, bool kZip>
__global__ void __launch_bounds__(kTreeMaxThreads) __maxnreg__(kBPT == 4 ? 80 : (kBPT == 2 ? 64 : 128)) f64_tree(const __grid_constant__ Tree64Args g) {
    extern __shared__ double2 dsm[];
    const int th = (int)blockDim.x, ns = th * kBPT, n = g.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = th >> 5;
    double2 *const Ss = dsm;        // [ns] S of each position
    double2 *const Zs = dsm + ns;   // [ns] z of each position; branch currents J at the end
    double2 *const PX = dsm + 2 * ns;  // [ns] prefix sums P, then branch terms in ends-list order
    short *const s_rng = reinterpret_cast<short *>(dsm + 3 * ns);  // slot of the subtree's last position
    short *const s_kidx = s_rng + ns;  // where the position's branch term goes in ends-list order (-1: nowhere)
    short *const s_par = s_kidx + ns;  // parent slot, -1 = the slack
    __shared__ double2 wt[kMaxWarps64];
    __shared__ double wm[kMaxWarps64];
    const int64_t t = blockIdx.x;
    const int base = tid * kBPT;
    const double2 *S = g.S + t * n;
    double2 *Vc = g.V + t * n;

    double2 V[kBPT];
    int ecnt[kBPT];
#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        double2 sv = make_double2(0.0, 0.0), zv = sv;
        V[j] = make_double2(1.0, 0.0);  // flat start (Algorithm 1)
        ecnt[j] = 0;
        int rng = s;
        if (q < n) {
            const int i = g.col[s];
            sv = S[i];
            zv = g.z[s];
            ecnt[j] = g.ecnt[s];
            const int e = g.end[s] - 1;  // last position of the subtree
            rng = (e % kBPT) * th + e / kBPT;
            if (g.given) V[j] = Vc[i];
        }
        Ss[s] = sv;
        Zs[s] = zv;
        s_rng[s] = (short)rng;
        s_kidx[s] = (short)g.kidx[s];
        s_par[s] = (short)g.par[s];
    }
    __syncthreads();

    int it = 0;
    bool conv = false;
    for (;;) {
        // Load currents and their inclusive prefix sums P.
        double2 loc[kBPT], run = make_double2(0.0, 0.0);
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            const int q = base + j, s = j * th + tid;
            if (q < n) run = dadd(run, demand64<kZip>(V[j], Ss[s], g, s));
            loc[j] = run;
        }
        double2 off = block_scan64(run, wt, lane, warp, nw);
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            loc[j] = dadd(off, loc[j]);
            PX[j * th + tid] = loc[j];
        }
        __syncthreads();
        // Branch terms x_q = z_q (P[end_q - 1] - P[q - 1]); descending j keeps loc[j - 1] = P[q - 1].
#pragma unroll
        for (int j = kBPT - 1; j >= 0; --j) {
            const int q = base + j, s = j * th + tid;
            double2 x = make_double2(0.0, 0.0);
            if (q < n) {
                const int ls = s_rng[s];
                double2 L = ls == s ? loc[j] : PX[ls];
                if (j) L = dsub(L, loc[j - 1]);
                else if (q > 0) L = dsub(L, PX[(kBPT - 1) * th + tid - 1]);
                x = dmul(Zs[s], L);
            }
            loc[j] = x;
        }
        __syncthreads();  // every read of P is done: PX takes the branch terms in ends-list order
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            const int k = s_kidx[j * th + tid];
            if (k >= 0) PX[k] = loc[j];
        }
        __syncthreads();
        // Path sums: prefix sums of E_q = x_q - (x_b of every b whose range ends at q).
        run = make_double2(0.0, 0.0);
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            const int st = ecnt[j] & 0xffff, cnt = (int)(((unsigned)ecnt[j] >> 16) & 0x3fffu);
            double2 e = loc[j];
            for (int k = 0; k < cnt; ++k) e = dsub(e, PX[st + k]);
            run = dadd(run, e);
            loc[j] = run;
        }
        off = block_scan64(run, wt, lane, warp, nw);
        double m = 0.0;
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            const int q = base + j;
            if (q < n) {
                const double2 vn = dsub(g.vs, dadd(off, loc[j]));
                m = dmax_nan(m, dabs2(dsub(vn, V[j])));
                V[j] = vn;
            }
        }
        // Block max of |step|^2 (a NaN stays NaN); every thread reads the same warp maxima and so
        // takes the same decision.
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = dmax_nan(m, __shfl_xor_sync(kFull, m, o));
        if (lane == 0) wm[warp] = m;
        __syncthreads();
        m = wm[0];
        for (int w = 1; w < nw; ++w) m = dmax_nan(m, wm[w]);
        ++it;
        if (m <= g.tol2) {
            conv = true;
            break;
        }
        if (it >= g.max_iter || !(m < 1e60)) break;
    }

    // Outputs: V, the iteration count, and the power mismatch max_i |V_i conj((Y v)_i) + S_i| at
    // the returned V (ZIP: |V_i| |(Y v)_i + i_d,i|).  On the tree (Y v)_q = -J_q + sum over the
    // children k of J_k with the branch currents J_k = y_k (V_parent(k) - V_k), y_k = 1 / z_k.
#pragma unroll
    for (int j = 0; j < kBPT; ++j) {
        const int q = base + j, s = j * th + tid;
        if (q < n) Vc[g.col[s]] = V[j];
        PX[s] = V[j];
    }
    __syncthreads();
    if (g.mismatch_out) {
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            const int q = base + j, s = j * th + tid;
            if (q < n) {
                const int p = s_par[s];
                const double2 zq = Zs[s];
                const double inv = 1.0 / dabs2(zq);
                const double2 y = make_double2(zq.x * inv, -zq.y * inv);
                Zs[s] = dmul(y, dsub(p >= 0 ? PX[p] : g.vs, V[j]));  // the slot's own z is read first
            }
        }
        __syncthreads();
        double worst = 0.0;
#pragma unroll
        for (int j = 0; j < kBPT; ++j) {
            const int q = base + j, s = j * th + tid;
            if (q < n) {
                double2 acc = make_double2(-Zs[s].x, -Zs[s].y);
                // The first child is q + 1; each next one follows the previous one's last position;
                // the child whose subtree ends where q's ends is the last.
                const int lq = s_rng[s];
                for (int ks = lq == s ? -1 : next_slot64<kBPT>(s, th); ks >= 0;) {
                    acc = dadd(acc, Zs[ks]);
                    const int lc = s_rng[ks];
                    ks = lc == lq ? -1 : next_slot64<kBPT>(lc, th);
                }
                const double2 v = V[j], sv = Ss[s];
                double mm;
                if (kZip) {
                    const double2 i_d = demand64<kZip>(v, sv, g, s);
                    mm = sqrt(dabs2(v) * dabs2(dadd(acc, i_d)));
                } else {
                    // V conj(acc) + S
                    mm = sqrt(dabs2(make_double2(v.x * acc.x + v.y * acc.y + sv.x, v.y * acc.x - v.x * acc.y + sv.y)));
                }
                worst = dmax_nan(worst, mm);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) worst = dmax_nan(worst, __shfl_xor_sync(kFull, worst, o));
        if (lane == 0) wm[warp] = worst;  // (the last sweep's maxima were read before two barriers)
        __syncthreads();
        if (tid == 0) {
            double r = wm[0];
            for (int w = 1; w < nw; ++w) r = dmax_nan(r, wm[w]);
            g.mismatch_out[t] = r != r ? __longlong_as_double(0x7ff0000000000000ll) : r;  // NaN reports as +inf
        }
    }
    if (tid == 0) {
        if (g.iters_out) g.iters_out[t] = conv ? it : -g.max_iter;
        if (conv) atomicAdd(&g.counters[kCntConverged], 1);
        atomicMax(&g.counters[5], it);
    }
}

template <int kBPT, bool kZip>
cudaError_t launch64_t(int threads, int64_t cols, size_t smem, const Tree64Args &g, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(f64_tree<kBPT, kZip>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && cols > 0) f64_tree<kBPT, kZip><<<(unsigned)cols, threads, smem, st>>>(g);
    return e;
}
template <int kBPT>
cudaError_t launch64(int threads, int64_t cols, size_t smem, const Tree64Args &g, cudaStream_t st) {
    return g.zip ? launch64_t<kBPT, true>(threads, cols, smem, g, st) : launch64_t<kBPT, false>(threads, cols, smem, g, st);
}

}  // namespace

size_t tree64_smem(int threads, int bpt) {
    const size_t ns = (size_t)threads * bpt;
    return 3 * ns * sizeof(double2) + 3 * ns * sizeof(short);
}

tpf_status solve_tree64(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters, double *mismatch,
                        const tpf_opts &o, cudaStream_t st) {
    const DeviceNet &d = h->dev;
    if (!d.radial || d.phases != 1 || d.t_threads == 0 || d.t_bpt == kTreeBigBPT || !d.t_z64) return TPF_EUNSUPPORTED;
    if (T > 0x7fffffff) return TPF_EUNSUPPORTED;  // one block per column
    const size_t smem = tree64_smem(d.t_threads, d.t_bpt);
    if (smem > 227 * 1024) return TPF_EUNSUPPORTED;
    tpf_status rs = ensure_workspace(h, T, kWsState);  // counters
    if (rs != TPF_OK) return rs;
    Workspace &w = h->ws;
    if (cudaMemsetAsync(w.counters, 0, sizeof(int) * 8, st) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    Tree64Args g{};
    g.n = d.n;
    g.max_iter = o.max_iter;
    g.tol2 = o.tol * o.tol;
    g.vs = make_double2(h->net.vs_re, h->net.vs_im);
    g.col = d.t_col;
    g.end = d.t_end;
    g.par = d.t_par;
    g.ecnt = d.t_ecnt;
    g.kidx = d.t_kidx;
    g.z = d.t_z64;
    g.zip = d.zip64;
    g.S = static_cast<const double2 *>(S);
    g.V = static_cast<double2 *>(V);
    g.given = o.start != TPF_START_FLAT;
    g.iters_out = iters;
    g.mismatch_out = mismatch;
    g.counters = w.counters;
    KernelTimer timer(o.profile != 0, st);
    timer.begin(KernelTimer::kGemm);
    cudaError_t e;
    switch (d.t_bpt) {
        case 2: e = launch64<2>(d.t_threads, T, smem, g, st); break;
        case 4: e = launch64<4>(d.t_threads, T, smem, g, st); break;
        case 8: e = launch64<8>(d.t_threads, T, smem, g, st); break;
        default: return TPF_EUNSUPPORTED;
    }
    timer.end();
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    if (cudaMemcpyAsync(w.counters_host, w.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    const int64_t conv = w.counters_host[kCntConverged];
    h->stats.sweeps = w.counters_host[5];
    h->stats.kernel_launches = 1;
    h->stats.converged = conv;
    h->stats.gemm_ms = timer.total_ms(KernelTimer::kGemm);
    return conv == T ? TPF_OK : TPF_ENOCONV;
}

}  // namespace tpf
