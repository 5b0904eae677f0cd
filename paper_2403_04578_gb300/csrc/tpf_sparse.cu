// Sparse tensor formulation (Sec. IV-B, Eq. 13-14, Algorithm 2) on radial feeders.
//
// Algorithm 2 replaces the dense product with K by a sparse solve with Y_dd, factored once.  On a
// radial feeder Y_dd factors without fill-in and its solve is a two-pass tree substitution, so a
// sweep costs O(n) per column instead of the dense O(n^2).  The iterate is the same as in the
// dense form (Algorithm 2's text: the voltage sequence does not change).  Written in residual form
// like the mixed dense path,
//
//     Y_dd dV = -rho(V),   V <- V + dV,
//
// the solve is: branch currents J_c = rho_c + sum_{children k} J_k from the leaves up (the current
// each subtree draws), then dV_c = dV_parent(c) - z_c J_c from the slack down (dV = 0 at the slack).
// rho uses the anchored precision scheme of the mixed path (FP32 far from convergence, then
// rho(V_ref) in double-float plus FP32 corrections), and the solve itself runs in FP32 on the small
// correction, so results reach the FP64 solution.
//
// One 128-thread block owns one column for the whole solve: S, V, rho(V_ref) and the work vector
// stay in shared memory across all sweeps, so device memory is touched once to read S and once to
// write V.  Each tree pass walks the depth levels with one barrier per level.
#include "tpf_dd.cuh"

namespace tpf {

namespace {

constexpr int kTreeThreads = 128;

struct TreeArgs {
    int64_t T;
    int n, depth, max_iter, given;
    float tol, switch_tol;
    float2 vs_f;
    c2 vs_dd;
    const double2 *S;
    const double2 *V0;
    double2 *V_out;
    int32_t *iters_out;
    double *mismatch_out;
    int *tile_done;   // converged columns per 128-column tile
    int *max_sweeps;  // largest per-column sweep count
    const int *par, *ch_ptr, *ch, *lvl_ptr, *lvl_bus, *row_ptr, *nbr;
    const float2 *ypar, *zpar;
    const float4 *y;
};

// rho_i (FP32 or anchored) from the staged column: vh = V (or V_ref), vl = V - V_ref.
__device__ __forceinline__ float2 tree_rho(const TreeArgs &a, int i, bool anchored, const float2 *vh,
                                           const float2 *vl, const float2 *sh, const float2 *rh, const float2 *rl) {
    const float2 *v = anchored ? vl : vh;
    const float2 vi = v[i];
    const int p = a.par[i];
    const float2 vp = p >= 0 ? v[p] : (anchored ? make_float2(0.0f, 0.0f) : a.vs_f);
    const float2 y = a.ypar[i];
    float dr = vp.x - vi.x, di = vp.y - vi.y;
    const float2 loc = anchored ? delta_current(vh[i], vi, sh[i]) : load_current_f32(vi, sh[i]);
    float ar = loc.x - (y.x * dr - y.y * di), ai = loc.y - (y.x * di + y.y * dr);
    for (int e = a.ch_ptr[i]; e < a.ch_ptr[i + 1]; ++e) {
        const int k = a.ch[e];
        const float2 yk = a.ypar[k], vk = v[k];
        dr = vi.x - vk.x;
        di = vi.y - vk.y;
        ar += yk.x * dr - yk.y * di;
        ai += yk.x * di + yk.y * dr;
    }
    if (anchored) {
        const f2 sr = two_sum(rh[i].x, ar), si = two_sum(rh[i].y, ai);
        ar = sr.h + (sr.l + rl[i].x);
        ai = si.h + (si.l + rl[i].y);
    }
    return make_float2(ar, ai);
}

__global__ void __launch_bounds__(kTreeThreads) mx_tree(TreeArgs a) {
    extern __shared__ float2 tsm[];
    const int n = a.n;
    float2 *vh = tsm, *vl = vh + n, *sh = vl + n, *sl = sh + n, *rh = sl + n, *rl = rh + n, *w = rl + n;
    __shared__ float s_red[kTreeThreads / 32];
    __shared__ int s_state;  // bit 0 done, 1 converged, 2 anchored, 3 blind, 4 anchor now
    __shared__ int s_it;
    __shared__ float s_dprev;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t t = blockIdx.x;
    if (t >= a.T) return;
    const double2 *S = a.S + t * n;
    for (int i = tid; i < n; i += kTreeThreads) {
        const double2 s = S[i];
        const float2 h = make_float2(__double2float_rn(s.x), __double2float_rn(s.y));
        sh[i] = h;
        sl[i] = make_float2(__double2float_rn(s.x - (double)h.x), __double2float_rn(s.y - (double)h.y));
        float2 v0h = make_float2(1.0f, 0.0f), v0l = make_float2(0.0f, 0.0f);
        if (a.given) {
            const double2 v = a.V0[t * n + i];
            v0h = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
            v0l = make_float2(__double2float_rn(v.x - (double)v0h.x), __double2float_rn(v.y - (double)v0h.y));
        }
        vh[i] = v0h;
        vl[i] = v0l;
    }
    if (tid == 0) {
        s_state = a.given ? (4 | 8 | 16) : 0;  // a given start is anchored at once (blind)
        s_it = 0;
        s_dprev = 0.0f;
    }
    __syncthreads();
    for (;;) {
        int state = s_state;
        if (state & 16) {  // (re-)anchor: V_ref <- fl(V), rho(V_ref) in double-float
            for (int i = tid; i < n; i += kTreeThreads) {
                const f2 re = two_sum(vh[i].x, vl[i].x), im = two_sum(vh[i].y, vl[i].y);
                vh[i] = make_float2(re.h, im.h);
                vl[i] = make_float2(re.l, im.l);
            }
            __syncthreads();
            for (int i = tid; i < n; i += kTreeThreads) {
                const c2 r = residual_dd(i, vh, nullptr, sh, sl, a.row_ptr, a.nbr, a.y, a.vs_dd);
                rh[i] = make_float2(r.re.h, r.im.h);
                rl[i] = make_float2(r.re.l, r.im.l);
            }
            __syncthreads();
            if (tid == 0) s_state = state & ~16;
            state &= ~16;
        }
        if (state & 1) break;
        const bool anchored = (state & 4) != 0;
        // rho -> w
        for (int i = tid; i < n; i += kTreeThreads) w[i] = tree_rho(a, i, anchored, vh, vl, sh, rh, rl);
        __syncthreads();
        // leaves to slack: J_c = rho_c + sum_{children} J_k
        for (int d = a.depth; d >= 1; --d) {
            for (int q = a.lvl_ptr[d - 1] + tid; q < a.lvl_ptr[d]; q += kTreeThreads) {
                const int c = a.lvl_bus[q];
                float2 J = w[c];
                for (int e = a.ch_ptr[c]; e < a.ch_ptr[c + 1]; ++e) {
                    const float2 Jk = w[a.ch[e]];
                    J.x += Jk.x;
                    J.y += Jk.y;
                }
                w[c] = J;
            }
            __syncthreads();
        }
        // slack to leaves: dV_c = dV_parent - z_c J_c
        for (int d = 1; d <= a.depth; ++d) {
            for (int q = a.lvl_ptr[d - 1] + tid; q < a.lvl_ptr[d]; q += kTreeThreads) {
                const int c = a.lvl_bus[q];
                const int p = a.par[c];
                const float2 dp = p >= 0 ? w[p] : make_float2(0.0f, 0.0f);
                const float2 J = w[c], z = a.zpar[c];
                w[c] = make_float2(dp.x - (z.x * J.x - z.y * J.y), dp.y - (z.x * J.y + z.y * J.x));
            }
            __syncthreads();
        }
        // V += dV and max |dV|
        float m = 0.0f;
        for (int i = tid; i < n; i += kTreeThreads) {
            const float2 dv = w[i];
            if (anchored) {
                vl[i] = make_float2(vl[i].x + dv.x, vl[i].y + dv.y);
            } else {
                vh[i] = make_float2(vh[i].x + dv.x, vh[i].y + dv.y);
            }
            float mag = sqrtf(dv.x * dv.x + dv.y * dv.y);
            if (mag != mag) mag = __int_as_float(0x7f800000);
            m = fmaxf(m, mag);
        }
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) s_red[warp] = m;
        __syncthreads();
        if (tid == 0) {
            float d = s_red[0];
            for (int k = 1; k < kTreeThreads / 32; ++k) d = fmaxf(d, s_red[k]);
            const int it = ++s_it;
            int st = s_state;
            if (d <= a.tol) {
                st |= 1 | 2;
            } else if (it >= a.max_iter || !(d < 1e30f)) {
                st |= 1;
            } else if (!(st & 4) || (st & 8)) {
                if (d < a.switch_tol || (s_dprev > 0.0f && d * d < 3e-6f * s_dprev)) st = (st | 4 | 16) & ~8;
            }
            s_dprev = d;
            s_state = st;
        }
        __syncthreads();
    }
    // Outputs: V, iteration count, mismatch max_i |V_i| |rho_i| at the returned V.
    const int state = s_state;
    const bool anchored = (state & 4) != 0;
    float m = 0.0f;
    for (int i = tid; i < n; i += kTreeThreads) {
        const float2 r = tree_rho(a, i, anchored, vh, vl, sh, rh, rl);
        const float2 h = vh[i], l = vl[i];
        a.V_out[t * n + i] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
        const float vr = h.x + l.x, vi = h.y + l.y;
        float mv = sqrtf(vr * vr + vi * vi) * sqrtf(r.x * r.x + r.y * r.y);
        if (mv != mv) mv = __int_as_float(0x7f800000);
        m = fmaxf(m, mv);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __syncthreads();
    if (lane == 0) s_red[warp] = m;
    __syncthreads();
    if (tid == 0) {
        float mm = s_red[0];
        for (int k = 1; k < kTreeThreads / 32; ++k) mm = fmaxf(mm, s_red[k]);
        const bool conv = (state & 2) != 0;
        if (a.mismatch_out) a.mismatch_out[t] = (double)mm;
        if (a.iters_out) a.iters_out[t] = conv ? s_it : -a.max_iter;
        if (conv) atomicAdd(&a.tile_done[t / kTileN], 1);
        atomicMax(a.max_sweeps, s_it);
    }
}

}  // namespace

tpf_status solve_sparse(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters, double *mismatch,
                        const tpf_opts &o, cudaStream_t st) {
    const DeviceNet &d = h->dev;
    if (!d.radial || o.precision != TPF_PREC_MIXED) return TPF_EUNSUPPORTED;
    const int n = d.n;
    const size_t smem = (size_t)7 * n * sizeof(float2);
    if (smem > 200 * 1024) return TPF_EUNSUPPORTED;
    tpf_status rs = ensure_workspace(h, T, kWsState);  // counters and per-tile counts
    if (rs != TPF_OK) return rs;
    Workspace &w = h->ws;
    if (T > 0x7fffffff) return TPF_EUNSUPPORTED;  // one block per column
    if (cudaFuncSetAttribute(mx_tree, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    const int64_t n_tiles = round_up(T, kTileN) / kTileN;
    if (cudaMemsetAsync(w.tile_active, 0, sizeof(int) * n_tiles, st) != cudaSuccess ||
        cudaMemsetAsync(w.counters, 0, sizeof(int) * 8, st) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    TreeArgs a{};
    a.T = T;
    a.n = n;
    a.depth = d.depth;
    a.max_iter = o.max_iter;
    a.given = o.start == TPF_START_GIVEN;
    a.tol = (float)o.tol;
    a.switch_tol = (float)o.switch_tol;
    a.vs_f = make_float2((float)h->net.vs_re, (float)h->net.vs_im);
    {
        const float rh = (float)h->net.vs_re, ih = (float)h->net.vs_im;
        a.vs_dd = c2{{rh, (float)(h->net.vs_re - (double)rh)}, {ih, (float)(h->net.vs_im - (double)ih)}};
    }
    a.S = (const double2 *)S;
    a.V0 = (const double2 *)V;
    a.V_out = (double2 *)V;
    a.iters_out = iters;
    a.mismatch_out = mismatch;
    a.tile_done = w.tile_active;
    a.max_sweeps = w.counters + 5;
    a.par = d.par;
    a.ch_ptr = d.ch_ptr;
    a.ch = d.ch;
    a.lvl_ptr = d.lvl_ptr;
    a.lvl_bus = d.lvl_bus;
    a.row_ptr = d.row_ptr;
    a.nbr = d.nbr;
    a.ypar = d.ypar;
    a.zpar = d.zpar;
    a.y = d.y2f;
    KernelTimer timer(o.profile != 0, st);
    timer.begin(KernelTimer::kResidual);
    mx_tree<<<(unsigned)T, kTreeThreads, smem, st>>>(a);
    timer.end();
    if (cudaGetLastError() != cudaSuccess) return TPF_ECUDA;
    std::vector<int> tiles(n_tiles);
    if (cudaMemcpyAsync(w.counters_host, w.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(tiles.data(), w.tile_active, sizeof(int) * n_tiles, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    int64_t conv = 0;
    for (int x : tiles) conv += x;
    h->stats.sweeps = w.counters_host[5];
    h->stats.kernel_launches = 1;
    h->stats.converged = conv;
    h->stats.residual_ms = timer.total_ms(KernelTimer::kResidual);
    return conv == T ? TPF_OK : TPF_ENOCONV;
}

}  // namespace tpf
