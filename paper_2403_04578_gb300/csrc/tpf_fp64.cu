// Device buffers of a handle and the plain double-precision solve path.
//
// The FP64 path is Algorithm 1 in its direct form, V_{k+1} = K conj(S ./ V_k) + W (Eq. 2 and
// Eq. 12), with per-column stopping.  Each sweep is one kernel over (64-bus x 32-column) output
// tiles: the tile's injections conj(S ./ V) are formed from V_k in shared memory chunk by chunk
// (the Hadamard step of Algorithm 1), multiplied by the matching K tile with FP64 FMAs, W is
// added and the per-column max |V_{k+1} - V_k| is folded in with an atomic max.  GB300 runs FP64
// at 1/64 of its FP32 rate, so this path is FP64-pipe bound; it is the reference point for the
// mixed-precision path.
#include <cstdio>
#include <type_traits>
#include <math_constants.h>

#include "tpf_internal.h"

namespace tpf {

#define TPF_CK(call)                                   \
    do {                                               \
        if ((call) != cudaSuccess) {                   \
            cudaGetLastError();                        \
            return TPF_ECUDA;                          \
        }                                              \
    } while (0)

namespace {

__global__ void k_to_fp16(const double *__restrict__ K, int n, int n_pad, float scale, __half *Kr, __half *Ki) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_pad * n_pad) return;
    int i = (int)(idx / n_pad), j = (int)(idx % n_pad);
    float re = 0.f, im = 0.f;
    if (i < n && j < n) {
        re = (float)K[((size_t)i * n + j) * 2] * scale;
        im = (float)K[((size_t)i * n + j) * 2 + 1] * scale;
    }
    Kr[idx] = __float2half_rn(re);
    Ki[idx] = __float2half_rn(im);
}

}  // namespace

// Slot-ordered depth-first arrays of the sparse formulation for blocks of tree_threads(n, bpt)
// threads with bpt positions each (replacing any earlier layout; bpt 0 disables the sparse path).
tpf_status layout_tree(tpf_handle *h, int bpt) {
    const Network &net = h->net;
    DeviceNet &d = h->dev;
    ++d.layout_gen;
    const int n = net.n_pq;
    cudaFree(d.t_col); cudaFree(d.t_end); cudaFree(d.t_par); cudaFree(d.t_ecnt); cudaFree(d.t_ends); cudaFree(d.t_z);
    cudaFree(d.t_zrow); cudaFree(d.t_yrow); cudaFree(d.t_kidx); cudaFree(d.t_zrow_f); cudaFree(d.t_z64);
    d.t_z64 = nullptr;
    d.t_col = d.t_end = d.t_par = d.t_ecnt = d.t_ends = d.t_kidx = nullptr;
    d.t_z = d.t_zrow = nullptr;
    d.t_yrow = d.t_zrow_f = nullptr;
    d.t_threads = d.t_bpt = 0;
    if (net.radial) {
        // Slot-ordered depth-first arrays of the sparse formulation.
        const int th = bpt ? tree_threads(n, bpt) : 0;
        d.t_threads = th;
        d.t_bpt = bpt;
        if (th > 0) {
            const int ns = th * bpt;
            auto slot = [th, bpt](int q) { return (q % bpt) * th + q / bpt; };
            const int ph = net.phases, nb = n / ph;
            std::vector<int> col(ns, -1), end(ns, 0), par(ns, -1), ecnt(ns, 0), ends, kidx(ns, -1);
            std::vector<float4> z(ns, make_float4(0.f, 0.f, 0.f, 0.f));
            std::vector<double2> z64(ph == 1 ? ns : 0, make_double2(0.0, 0.0));
            // Polyphase: row p of the branch's impedance (double-float) and admittance per slot.
            std::vector<float4> zrow(ph > 1 ? (size_t)ns * ph : 0, make_float4(0.f, 0.f, 0.f, 0.f));
            std::vector<float2> yrow(ph > 1 ? (size_t)ns * ph : 0, make_float2(0.f, 0.f)), zrow_f = yrow;
            std::vector<int> pos_par(n, -1);  // parent position of each position
            for (int q = 0; q < n; ++q)
                for (int c = q + 1; c < net.dfs_end[q]; c = net.dfs_end[c]) pos_par[c] = q;
            bool fits = true;
            for (int q = 0; q < n; ++q) {
                const int s = slot(q), cnt = net.dfs_eptr[q + 1] - net.dfs_eptr[q];
                col[s] = net.dfs_col[q];
                end[s] = net.dfs_end[q];
                par[s] = pos_par[q] < 0 ? -1 : slot(pos_par[q]);
                if ((int)ends.size() > 0xffff || cnt > 0x3fff) fits = false;
                // start | count << 16 | phase << 30
                ecnt[s] = (int)ends.size() | (cnt << 16) | ((q / nb) << 30);
                for (int k = net.dfs_eptr[q]; k < net.dfs_eptr[q + 1]; ++k) {
                    kidx[slot(net.dfs_ends[k])] = (int)ends.size();  // where its branch term is scattered
                    ends.push_back(slot(net.dfs_ends[k]));
                }
                auto dd = [](double re, double im) {
                    const float rh = (float)re, ih = (float)im;
                    return make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
                };
                if (ph == 1) {
                    z[s] = dd(net.dfs_z[2 * q], net.dfs_z[2 * q + 1]);
                    z64[s] = make_double2(net.dfs_z[2 * q], net.dfs_z[2 * q + 1]);
                } else {
                    for (int pp = 0; pp < ph; ++pp) {
                        const size_t k = (size_t)q * ph + pp;
                        zrow[(size_t)s * ph + pp] = dd(net.dfs_zrow[2 * k], net.dfs_zrow[2 * k + 1]);
                        zrow_f[(size_t)s * ph + pp] = make_float2(zrow[(size_t)s * ph + pp].x, zrow[(size_t)s * ph + pp].y);
                        yrow[(size_t)s * ph + pp] = make_float2((float)net.dfs_yrow[2 * k], (float)net.dfs_yrow[2 * k + 1]);
                    }
                    const float4 zz = zrow[(size_t)s * ph + q / nb];  // the own-phase entry, for z-only uses
                    z[s] = zz;
                }
            }
            d.t_n_ends = (int)ends.size();
            if (ends.empty()) ends.push_back(0);
            auto up = [](auto **dst, const auto &v) -> bool {
                using T = typename std::decay_t<decltype(v)>::value_type;
                if (cudaMalloc((void **)dst, sizeof(T) * v.size()) != cudaSuccess) return false;
                return cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice) == cudaSuccess;
            };
            if (!fits) {
                d.t_threads = 0;
            } else if (!up(&d.t_col, col) || !up(&d.t_end, end) || !up(&d.t_par, par) || !up(&d.t_ecnt, ecnt) ||
                       !up(&d.t_ends, ends) || !up(&d.t_z, z) || !up(&d.t_kidx, kidx) ||
                       (ph == 1 && !up(&d.t_z64, z64)) || (ph > 1 && (!up(&d.t_zrow, zrow) || !up(&d.t_yrow, yrow) || !up(&d.t_zrow_f, zrow_f)))) {
                cudaGetLastError();
                return TPF_ECUDA;
            }
        }
    }
    return TPF_OK;
}

tpf_status upload_network(tpf_handle *h) {
    int dev = 0;
    TPF_CK(cudaGetDevice(&dev));
    h->device = dev;
    const Network &net = h->net;
    DeviceNet &d = h->dev;
    const int n = net.n_pq;
    d.n = n;
    d.n_pad = (int)round_up(n, kTileM);
    const int nnz = net.row_ptr[n];
    TPF_CK(cudaMalloc(&d.row_ptr, sizeof(int) * (n + 1)));
    TPF_CK(cudaMalloc(&d.nbr, sizeof(int) * (nnz > 0 ? nnz : 1)));
    TPF_CK(cudaMalloc(&d.y64, sizeof(double) * 2 * (nnz > 0 ? nnz : 1)));
    TPF_CK(cudaMalloc(&d.y2f, sizeof(float4) * (nnz > 0 ? nnz : 1)));
    TPF_CK(cudaMemcpy(d.row_ptr, net.row_ptr.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
    if (nnz > 0) {
        TPF_CK(cudaMemcpy(d.nbr, net.nbr.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice));
        TPF_CK(cudaMemcpy(d.y64, net.y.data(), sizeof(double) * 2 * nnz, cudaMemcpyHostToDevice));
        // Double-float split of each admittance: hi = fl(y), lo = fl(y - hi).
        std::vector<float4> y2(nnz);
        for (int k = 0; k < nnz; ++k) {
            double re = net.y[2 * k], im = net.y[2 * k + 1];
            float rh = (float)re, ih = (float)im;
            y2[k] = make_float4(rh, ih, (float)(re - (double)rh), (float)(im - (double)ih));
        }
        TPF_CK(cudaMemcpy(d.y2f, y2.data(), sizeof(float4) * nnz, cudaMemcpyHostToDevice));
    }
    d.radial = net.radial;
    d.phases = net.phases;
    d.nbp = n / net.phases;
    if (net.phases > 1) {
        // Polyphase: the unknown each neighbour-list entry's admittance multiplies, and v_s.
        TPF_CK(cudaMalloc(&d.csr_self, sizeof(int) * (nnz > 0 ? nnz : 1)));
        if (nnz > 0) TPF_CK(cudaMemcpy(d.csr_self, net.csr_self.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice));
    }
    TPF_CK(cudaMalloc(&d.vs64, sizeof(double) * 2 * net.phases));
    {
        std::vector<double> vs(net.vs);
        if (vs.empty()) vs = {net.vs_re, net.vs_im};
        TPF_CK(cudaMemcpy(d.vs64, vs.data(), sizeof(double) * 2 * net.phases, cudaMemcpyHostToDevice));
    }
    if (net.radial && net.phases == 1) {
        const int nch = net.ch_ptr[n];
        std::vector<float2> yp(n);
        for (int i = 0; i < n; ++i) yp[i] = make_float2((float)net.ypar[2 * i], (float)net.ypar[2 * i + 1]);
        TPF_CK(cudaMalloc(&d.par, sizeof(int) * n));
        TPF_CK(cudaMalloc(&d.ch_ptr, sizeof(int) * (n + 1)));
        TPF_CK(cudaMalloc(&d.ch, sizeof(int) * (nch > 0 ? nch : 1)));
        TPF_CK(cudaMalloc(&d.ypar, sizeof(float2) * n));
        TPF_CK(cudaMemcpy(d.par, net.par.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        TPF_CK(cudaMemcpy(d.ch_ptr, net.ch_ptr.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
        if (nch > 0) TPF_CK(cudaMemcpy(d.ch, net.ch.data(), sizeof(int) * nch, cudaMemcpyHostToDevice));
        TPF_CK(cudaMemcpy(d.ypar, yp.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    }
    if (net.radial) {
        const tpf_status rs = layout_tree(h, tree_bpt(n));
        if (rs != TPF_OK) return rs;
    }
    if (!net.K.empty()) return ensure_dense(h);  // meshed networks: K was built with the network
    return TPF_OK;
}

tpf_status ensure_dense(tpf_handle *h) {
    DeviceNet &d = h->dev;
    if (d.K64) return TPF_OK;
    Network &net = h->net;
    try {
        compute_dense(net);
    } catch (const std::bad_alloc &) {
        return TPF_ENOMEM;
    }
    const int n = d.n;
    if (cudaMalloc(&d.K64, sizeof(double) * 2 * (size_t)n * n) != cudaSuccess ||
        cudaMalloc(&d.W64, sizeof(double) * 2 * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ENOMEM;
    }
    TPF_CK(cudaMemcpy(d.K64, net.K.data(), sizeof(double) * net.K.size(), cudaMemcpyHostToDevice));
    TPF_CK(cudaMemcpy(d.W64, net.W.data(), sizeof(double) * net.W.size(), cudaMemcpyHostToDevice));
    // fp16 planes of K * 2^k_exp with the largest component in [2^13, 2^14).
    double kmax = 0.0;
    for (double v : net.K) kmax = fmax(kmax, fabs(v));
    int e = 0;
    if (kmax > 0.0) frexp(kmax, &e);
    d.k_exp = 14 - e;
    const size_t plane = (size_t)d.n_pad * d.n_pad;
    TPF_CK(cudaMalloc(&d.Kr16, sizeof(__half) * plane));
    TPF_CK(cudaMalloc(&d.Ki16, sizeof(__half) * plane));
    k_to_fp16<<<(unsigned)((plane + 255) / 256), 256>>>(d.K64, n, d.n_pad, ldexpf(1.0f, d.k_exp),
                                                          (__half *)d.Kr16, (__half *)d.Ki16);
    TPF_CK(cudaGetLastError());
    TPF_CK(cudaDeviceSynchronize());
    std::vector<double>().swap(net.K);  // the device copies serve from here on
    return TPF_OK;
}

tpf_status set_zip(tpf_handle *h, const double *alpha) {
    DeviceNet &d = h->dev;
    if (d.phases > 1) return alpha ? TPF_EUNSUPPORTED : TPF_OK;
    ++d.layout_gen;
    // The sparse kernel's ZIP coefficients take a fourth shared-memory region (16 B per slot): at 8
    // buses per thread (3,073 to 4,096 demand buses) the block would need more than 227 KB, so such
    // feeders are laid out at 16 buses per thread, whose kernel keeps the coefficients in device
    // scratch; without coefficients they return to the default layout.
    if (d.radial && d.t_threads > 0) {
        const size_t zip_smem_bpt8 = (size_t)(4 * 16 + 3 * 2) * tree_threads(d.n, 8) * 8;
        if (alpha && d.t_bpt == 8 && zip_smem_bpt8 > 227 * 1024) {
            const tpf_status rs = layout_tree(h, kTreeBigBPT);
            if (rs != TPF_OK) return rs;
        } else if (!alpha && d.t_bpt == kTreeBigBPT && tree_bpt(d.n) != kTreeBigBPT) {
            const tpf_status rs = layout_tree(h, tree_bpt(d.n));
            if (rs != TPF_OK) return rs;
        }
    }
    cudaFree(d.zip64);
    cudaFree(d.t_zip_hi);
    cudaFree(d.t_zip_lo);
    d.zip64 = nullptr;
    d.t_zip_hi = d.t_zip_lo = nullptr;
    if (!alpha) return TPF_OK;
    const int n = d.n;
    TPF_CK(cudaMalloc(&d.zip64, sizeof(double) * 3 * (size_t)n));
    TPF_CK(cudaMemcpy(d.zip64, alpha, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice));
    if (d.t_threads > 0) {
        const int th = d.t_threads, bpt = d.t_bpt, ns = th * bpt;
        std::vector<float4> hi(ns, make_float4(0.f, 0.f, 0.f, 0.f)), lo = hi;
        const Network &net = h->net;
        for (int q = 0; q < n; ++q) {
            const int s = (q % bpt) * th + q / bpt, i = net.dfs_col[q];
            float hv[3], lv[3];
            for (int k = 0; k < 3; ++k) {
                const double a = alpha[(size_t)k * n + i];
                hv[k] = (float)a;
                lv[k] = (float)(a - (double)hv[k]);
            }
            hi[s] = make_float4(hv[0], hv[1], hv[2], 0.f);
            lo[s] = make_float4(lv[0], lv[1], lv[2], 0.f);
        }
        TPF_CK(cudaMalloc(&d.t_zip_hi, sizeof(float4) * ns));
        TPF_CK(cudaMalloc(&d.t_zip_lo, sizeof(float4) * ns));
        TPF_CK(cudaMemcpy(d.t_zip_hi, hi.data(), sizeof(float4) * ns, cudaMemcpyHostToDevice));
        TPF_CK(cudaMemcpy(d.t_zip_lo, lo.data(), sizeof(float4) * ns, cudaMemcpyHostToDevice));
    }
    return TPF_OK;
}

void free_device(tpf_handle *h) {
    DeviceNet &d = h->dev;
    cudaFree(d.K64); cudaFree(d.W64); cudaFree(d.row_ptr); cudaFree(d.nbr); cudaFree(d.y64); cudaFree(d.y2f);
    cudaFree(d.Kr16); cudaFree(d.Ki16);
    cudaFree(d.par); cudaFree(d.ch_ptr); cudaFree(d.ch); cudaFree(d.ypar);
    cudaFree(d.t_col); cudaFree(d.t_end); cudaFree(d.t_par); cudaFree(d.t_ecnt); cudaFree(d.t_ends); cudaFree(d.t_z);
    cudaFree(d.t_kidx); cudaFree(d.t_z64);
    cudaFree(d.zip64); cudaFree(d.t_zip_hi); cudaFree(d.t_zip_lo);
    cudaFree(d.csr_self); cudaFree(d.vs64); cudaFree(d.t_zrow); cudaFree(d.t_yrow); cudaFree(d.t_zrow_f);
    d = DeviceNet();
    Workspace &w = h->ws;
    cudaFree(w.Vhi); cudaFree(w.Vlo); cudaFree(w.Shi); cudaFree(w.Slo); cudaFree(w.Rr16); cudaFree(w.Ri16);
    cudaFree(w.RefHi); cudaFree(w.RefLo); cudaFree(w.dprev);
    cudaFree(w.Valt); cudaFree(w.delta_bits); cudaFree(w.delta64); cudaFree(w.iters); cudaFree(w.flags);
    cudaFree(w.rexp); cudaFree(w.tile_active); cudaFree(w.counters);
    if (w.counters_host) cudaFreeHost(w.counters_host);
    cudaFree(w.S_dev); cudaFree(w.V_dev); cudaFree(w.it_dev); cudaFree(w.mm_dev); cudaFree(w.tree_scratch);
    w = Workspace();
    if (h->tmaps) {
        free(h->tmaps);
        h->tmaps = nullptr;
    }
    cudaGetLastError();
}

tpf_status ensure_workspace(tpf_handle *h, int64_t cols, int kind) {
    const bool mixed = kind == kWsMixed, fp64 = kind == kWsFp64;
    Workspace &w = h->ws;
    const int n = h->dev.n, n_pad = h->dev.n_pad;
    cols = round_up(cols, kTileN);
    const bool have_mixed = w.Vhi != nullptr;
    const bool have_fp64 = w.Valt != nullptr;
    if (w.counters == nullptr) {
        TPF_CK(cudaMalloc(&w.counters, sizeof(int) * 8));
        TPF_CK(cudaMallocHost(&w.counters_host, sizeof(int) * 8));
        TPF_CK(cudaMemset(w.counters, 0, sizeof(int) * 8));
    }
    if (cols <= w.cap_cols && (mixed ? have_mixed : (fp64 ? have_fp64 : true))) return TPF_OK;
    int64_t cap = cols > w.cap_cols ? cols : w.cap_cols;
    bool want_mixed = mixed || (have_mixed && cap > w.cap_cols);
    bool want_fp64 = fp64 || (have_fp64 && cap > w.cap_cols);
    if (cap > w.cap_cols) {
        cudaFree(w.delta_bits); cudaFree(w.delta64); cudaFree(w.iters); cudaFree(w.flags); cudaFree(w.rexp);
        cudaFree(w.tile_active); cudaFree(w.dprev);
        w.delta_bits = nullptr; w.delta64 = nullptr; w.iters = nullptr; w.flags = nullptr; w.rexp = nullptr;
        w.tile_active = nullptr; w.dprev = nullptr;
        TPF_CK(cudaMalloc(&w.delta_bits, sizeof(unsigned) * cap));
        TPF_CK(cudaMalloc(&w.dprev, sizeof(unsigned) * cap));
        TPF_CK(cudaMalloc(&w.delta64, sizeof(unsigned long long) * cap));
        TPF_CK(cudaMalloc(&w.iters, sizeof(int) * cap));
        TPF_CK(cudaMalloc(&w.flags, sizeof(int) * cap));
        TPF_CK(cudaMalloc(&w.rexp, sizeof(int) * cap));
        TPF_CK(cudaMalloc(&w.tile_active, sizeof(int) * (cap / kTileN)));
        if (have_mixed || want_mixed) {
            cudaFree(w.Vhi); cudaFree(w.Vlo); cudaFree(w.Shi); cudaFree(w.Slo); cudaFree(w.Rr16); cudaFree(w.Ri16);
            cudaFree(w.RefHi); cudaFree(w.RefLo);
            w.Vhi = w.Vlo = w.Shi = w.Slo = w.RefHi = w.RefLo = nullptr; w.Rr16 = w.Ri16 = nullptr;
        }
        if (have_fp64 || want_fp64) {
            cudaFree(w.Valt);
            w.Valt = nullptr;
        }
        w.cap_cols = cap;
    }
    w.n_pad = n_pad;
    const size_t el = (size_t)w.cap_cols * n_pad;
    if (want_mixed && w.Vhi == nullptr) {
        if (cudaMalloc(&w.Vhi, sizeof(float2) * el) != cudaSuccess || cudaMalloc(&w.Vlo, sizeof(float2) * el) != cudaSuccess ||
            cudaMalloc(&w.Shi, sizeof(float2) * el) != cudaSuccess || cudaMalloc(&w.Slo, sizeof(float2) * el) != cudaSuccess ||
            cudaMalloc(&w.RefHi, sizeof(float2) * el) != cudaSuccess || cudaMalloc(&w.RefLo, sizeof(float2) * el) != cudaSuccess ||
            cudaMalloc(&w.Rr16, sizeof(__half) * el) != cudaSuccess || cudaMalloc(&w.Ri16, sizeof(__half) * el) != cudaSuccess) {
            cudaGetLastError();
            return TPF_ENOMEM;
        }
    }
    if (want_fp64 && w.Valt == nullptr) {
        if (cudaMalloc(&w.Valt, sizeof(double) * 2 * (size_t)w.cap_cols * n) != cudaSuccess) {
            cudaGetLastError();
            return TPF_ENOMEM;
        }
    }
    return TPF_OK;
}

// ------------------------------------------------------------------------------------------
// FP64 path kernels
// ------------------------------------------------------------------------------------------
namespace {

constexpr int F64_BM = 64, F64_BN = 32, F64_KC = 16;

__global__ void f64_init(int64_t T, int64_t cols, int n, int flat, double2 *V, int *flags, int *iters,
                         unsigned long long *delta) {
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx < cols) {
        flags[idx] = idx < T ? kActive : 0;
        iters[idx] = 0;
        delta[idx] = 0ull;
    }
    if (flat && idx < T * (int64_t)n) V[idx] = make_double2(1.0, 0.0);
}

// One sweep of V_out = K conj(S ./ V_in) + W over a (64 x 32) tile; inactive columns untouched.
__global__ void __launch_bounds__(256) f64_sweep(const double2 *__restrict__ K, const double2 *__restrict__ W,
                                                 const double2 *__restrict__ S, const double2 *__restrict__ Vin,
                                                 double2 *__restrict__ Vout, int n, int64_t T,
                                                 const int *__restrict__ flags, unsigned long long *delta,
                                                 const double *__restrict__ zip) {
    __shared__ double2 Ks[F64_BM][F64_KC + 1];
    __shared__ double2 Is[F64_KC][F64_BN];
    __shared__ int act[F64_BN];
    __shared__ int any;
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * F64_BM;
    const int64_t t0 = (int64_t)blockIdx.x * F64_BN;
    if (tid == 0) any = 0;
    __syncthreads();
    if (tid < F64_BN) {
        int64_t t = t0 + tid;
        int a = (t < T) ? (flags[t] & kActive) : 0;
        act[tid] = a;
        if (a) atomicOr(&any, 1);
    }
    __syncthreads();
    if (!any) return;
    const int rg = tid / 16, cg = tid % 16;
    double2 acc[4][2];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[r][c] = make_double2(0.0, 0.0);
    for (int k0 = 0; k0 < n; k0 += F64_KC) {
        for (int e = tid; e < F64_BM * F64_KC; e += 256) {
            int r = e / F64_KC, c = e % F64_KC;
            int i = m0 + r, k = k0 + c;
            Ks[r][c] = (i < n && k < n) ? K[(size_t)i * n + k] : make_double2(0.0, 0.0);
        }
        for (int e = tid; e < F64_KC * F64_BN; e += 256) {
            int kk = e % F64_KC, tt = e / F64_KC;
            int k = k0 + kk;
            int64_t t = t0 + tt;
            double2 cur = make_double2(0.0, 0.0);
            if (k < n && act[tt]) {
                double2 s = S[t * n + k], v = Vin[t * n + k];
                // conj(s / v) = conj(s) v / |v|^2
                double inv = 1.0 / (v.x * v.x + v.y * v.y);
                cur = make_double2((s.x * v.x + s.y * v.y) * inv, (s.x * v.y - s.y * v.x) * inv);
                if (zip) {
                    // Eq. 3: alpha_P conj(s / v) + alpha_I conj(s) + alpha_Z conj(s) v
                    const double ap = zip[k], ai = zip[n + k], az = zip[2 * n + k];
                    cur = make_double2(ap * cur.x + ai * s.x + az * (s.x * v.x + s.y * v.y),
                                       ap * cur.y - ai * s.y + az * (s.x * v.y - s.y * v.x));
                }
            }
            Is[kk][tt] = cur;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < F64_KC; ++kk) {
            double2 a[4], b[2];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = Ks[rg * 4 + r][kk];
#pragma unroll
            for (int c = 0; c < 2; ++c) b[c] = Is[kk][cg * 2 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    acc[r][c].x = fma(a[r].x, b[c].x, fma(-a[r].y, b[c].y, acc[r][c].x));
                    acc[r][c].y = fma(a[r].x, b[c].y, fma(a[r].y, b[c].x, acc[r][c].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        int tt = cg * 2 + c;
        int64_t t = t0 + tt;
        if (!act[tt]) continue;
        double dmax = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int i = m0 + rg * 4 + r;
            if (i >= n) continue;
            double2 w = W[i];
            double2 vn = make_double2(acc[r][c].x + w.x, acc[r][c].y + w.y);
            double2 vo = Vin[t * n + i];
            double d = hypot(vn.x - vo.x, vn.y - vo.y);
            if (!(d <= dmax)) dmax = (d != d) ? CUDART_INF : d;  // a NaN step counts as infinite
            Vout[t * n + i] = vn;
        }
        // Non-negative doubles order like their bit patterns.
        if (dmax > 0.0) atomicMax(&delta[t], (unsigned long long)__double_as_longlong(dmax));
    }
}

// Per-column decision after a sweep: count the update, stop converged, exhausted or diverged
// columns.  iters holds the updates applied; kDone marks the columns that met tol.
__global__ void f64_decide(int64_t T, double tol, int max_iter, int *flags, int *iters,
                           unsigned long long *delta, int *counters) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int active = 0, conv = 0;
    if (t < T && (flags[t] & kActive)) {
        int k = iters[t] + 1;
        iters[t] = k;
        double d = __longlong_as_double((long long)delta[t]);
        delta[t] = 0ull;
        if (d <= tol) {
            flags[t] = kDone;
            conv = 1;
        } else if (k >= max_iter || !(d < 1e30)) {
            flags[t] = 0;
        } else {
            active = 1;
        }
    }
    unsigned m = __ballot_sync(0xffffffffu, active);
    unsigned c = __ballot_sync(0xffffffffu, conv);
    if ((threadIdx.x & 31) == 0) {
        if (m) atomicAdd(&counters[kCntActive], __popc(m));
        if (c) atomicAdd(&counters[kCntConverged], __popc(c));
    }
}

// Copy the final iterate into V (when it sits in the second buffer), write the iteration counts
// and the FP64 power mismatch max_i |V_i conj(sum_j y_ij (V_i - V_j)) + S_i|.
__global__ void f64_finish(int64_t T, int n, int max_iter, const int *__restrict__ flags,
                           const int *__restrict__ it_state, double2 *V, const double2 *__restrict__ Valt,
                           const double2 *__restrict__ S, const int *__restrict__ row_ptr,
                           const int *__restrict__ nbr, const double2 *__restrict__ y,
                           const int *__restrict__ self, const double2 *__restrict__ vs,
                           const double *__restrict__ zip, int32_t *iters_out, double *mismatch_out) {
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= T) return;
    const int updates = it_state[t];
    if (updates & 1) {
        for (int i = lane; i < n; i += 32) V[t * n + i] = Valt[t * n + i];
    }
    __syncwarp();
    if (lane == 0 && iters_out) iters_out[t] = (flags[t] & kDone) ? updates : -max_iter;
    if (!mismatch_out) return;
    double worst = 0.0;
    const double2 *v = V + t * n;
    for (int i = lane; i < n; i += 32) {
        double2 vi = v[i];
        double2 acc = make_double2(0.0, 0.0);
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            // (Y v)_i = sum_e y_e (v[self_e] - v[nbr_e]); nbr_e = -1 - p names slack phase p
            int j = nbr[e];
            double2 vj = j >= 0 ? v[j] : vs[-1 - j];
            double2 vself = self ? v[self[e]] : vi;
            double2 d = make_double2(vself.x - vj.x, vself.y - vj.y);
            double2 ye = y[e];
            acc.x += ye.x * d.x - ye.y * d.y;
            acc.y += ye.x * d.y + ye.y * d.x;
        }
        double2 s = S[t * n + i];
        double m;
        if (zip) {
            // |V_i| |(Y v)_i + i_d,i| with the ZIP demand current of Eq. 3
            const double ap = zip[i], ai = zip[n + i], az = zip[2 * n + i];
            const double inv = 1.0 / (vi.x * vi.x + vi.y * vi.y);
            const double cr = (s.x * vi.x + s.y * vi.y) * inv, ci = (s.x * vi.y - s.y * vi.x) * inv;
            const double ir = ap * cr + ai * s.x + az * (s.x * vi.x + s.y * vi.y);
            const double ii = ap * ci - ai * s.y + az * (s.x * vi.y - s.y * vi.x);
            m = hypot(vi.x, vi.y) * hypot(acc.x + ir, acc.y + ii);
        } else {
            // V_i conj(acc) + S_i
            double mr = vi.x * acc.x + vi.y * acc.y + s.x;
            double mi = vi.y * acc.x - vi.x * acc.y + s.y;
            m = hypot(mr, mi);
        }
        if (!(m <= worst)) worst = m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double other = __shfl_xor_sync(0xffffffffu, worst, o);
        if (!(other <= worst)) worst = other;
    }
    if (lane == 0) mismatch_out[t] = worst;
}

}  // namespace

tpf_status solve_fp64(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters, double *mismatch,
                      const tpf_opts &o, cudaStream_t st) {
    tpf_status rs = ensure_dense(h);
    if (rs != TPF_OK) return rs;
    rs = ensure_workspace(h, T, kWsFp64);
    if (rs != TPF_OK) return rs;
    Workspace &w = h->ws;
    const int n = h->dev.n;
    const int64_t cols = round_up(T, kTileN);
    int64_t launches = 0;
    KernelTimer timer(o.profile != 0, st);
    TPF_CK(cudaMemsetAsync(w.counters, 0, sizeof(int) * 8, st));
    {
        int64_t work = cols > T * n ? cols : T * n;
        f64_init<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(T, cols, n, o.start == TPF_START_FLAT,
                                                                  (double2 *)V, w.flags, w.iters, w.delta64);
        ++launches;
    }
    TPF_CK(cudaGetLastError());
    double2 *buf[2] = {(double2 *)V, (double2 *)w.Valt};
    const dim3 grid((unsigned)((T + F64_BN - 1) / F64_BN), (n + F64_BM - 1) / F64_BM);
    int sweeps = 0;
    int64_t active = T, gemm_cols = 0;
    for (int k = 0; k < o.max_iter; ++k) {
        timer.begin(KernelTimer::kGemm);
        f64_sweep<<<grid, 256, 0, st>>>((const double2 *)h->dev.K64, (const double2 *)h->dev.W64, (const double2 *)S,
                                        buf[k & 1], buf[(k + 1) & 1], n, T, w.flags, w.delta64, h->dev.zip64);
        timer.end();
        gemm_cols += active;
        TPF_CK(cudaMemsetAsync(w.counters, 0, sizeof(int) * 4, st));
        timer.begin(KernelTimer::kResidual);
        f64_decide<<<(unsigned)((T + 255) / 256), 256, 0, st>>>(T, o.tol, o.max_iter, w.flags, w.iters, w.delta64,
                                                                w.counters);
        timer.end();
        launches += 2;
        TPF_CK(cudaGetLastError());
        ++sweeps;
        TPF_CK(cudaMemcpyAsync(w.counters_host, w.counters, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
        TPF_CK(cudaStreamSynchronize(st));
        active = w.counters_host[kCntActive];
        if (active == 0) break;
    }
    timer.begin(KernelTimer::kOther);
    f64_finish<<<(unsigned)((T * 32 + 255) / 256), 256, 0, st>>>(
        T, n, o.max_iter, w.flags, w.iters, (double2 *)V, (const double2 *)w.Valt, (const double2 *)S,
        h->dev.row_ptr, h->dev.nbr, (const double2 *)h->dev.y64, h->dev.csr_self, (const double2 *)h->dev.vs64,
        h->dev.zip64, iters, mismatch);
    timer.end();
    ++launches;
    TPF_CK(cudaGetLastError());
    TPF_CK(cudaMemcpyAsync(w.counters_host, w.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
    TPF_CK(cudaStreamSynchronize(st));
    h->stats.sweeps = sweeps;
    h->stats.kernel_launches = launches;
    h->stats.converged = w.counters_host[kCntConverged];
    h->stats.gemm_launches = sweeps;
    h->stats.gemm_columns = gemm_cols;
    h->stats.gemm_ms = timer.total_ms(KernelTimer::kGemm);
    h->stats.residual_ms = timer.total_ms(KernelTimer::kResidual);
    h->stats.other_ms = timer.total_ms(KernelTimer::kOther);
    return h->stats.converged == T ? TPF_OK : TPF_ENOCONV;
}

}  // namespace tpf

// ------------------------------------------------------------------------------------------
// Allocation-free FP64 solve (tpf_solve_fp64_noalloc)
//
// For callers that cannot allocate device memory (their runtime hands out device memory only
// from its own pool, or their loop cannot afford cudaMalloc/cudaFree, which may synchronise the
// device): the same FP64 kernels as solve_fp64, with the scratch they need in one fixed array.
// ------------------------------------------------------------------------------------------

// The scratch of every tpf_solve_fp64_noalloc call on a device.  Layout for a call with
// cols = T rounded up to 128:  [0, 1024) counters | flags int[cols] | iters int[cols] |
// step double-bits[cols] | second V buffer complex128[cols][n].
static __device__ __align__(256) unsigned char g_noalloc_scratch[TPF_NOALLOC_SCRATCH_BYTES];

#include <mutex>

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoallocMaxDevices];  // device address of g_noalloc_scratch, per device
}  // namespace

extern "C" tpf_status tpf_solve_fp64_noalloc(int n, const void *K_dev, const void *W_dev, int64_t T,
                                             const void *S_dev, void *V_dev, int32_t *iters_dev, double tol,
                                             int max_iter, int given_start, void *stream) {
    using namespace tpf;
    if (n < 1 || T < 0 || !(tol >= 0.0) || max_iter < 1 || max_iter > 100000) return TPF_EINVAL;
    if (T == 0) return TPF_OK;
    if (!K_dev || !W_dev || !S_dev || !V_dev) return TPF_EINVAL;
    const int64_t cols = round_up(T, kTileN);
    const size_t off_flags = 1024;
    const size_t off_iters = off_flags + sizeof(int) * (size_t)cols;
    const size_t off_delta = off_iters + sizeof(int) * (size_t)cols;
    const size_t off_valt = off_delta + sizeof(unsigned long long) * (size_t)cols;
    const size_t need = off_valt + sizeof(double2) * (size_t)cols * (size_t)n;  // 1024 + 16 cols (n + 1)
    if ((size_t)cols > TPF_NOALLOC_SCRATCH_BYTES / 16 || need > TPF_NOALLOC_SCRATCH_BYTES) return TPF_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return TPF_ECUDA;
    }
    if (dev < 0 || dev >= kNoallocMaxDevices) return TPF_EUNSUPPORTED;
    char *base = nullptr;
    {
        // Host code cannot use the array's name as a device address: look it up once per device.
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return TPF_ECUDA;
            }
            g_noalloc_addr[dev] = p;
        }
        base = (char *)g_noalloc_addr[dev];
    }
    int *counters = (int *)base;
    int *flags = (int *)(base + off_flags);
    int *iters = (int *)(base + off_iters);
    unsigned long long *delta = (unsigned long long *)(base + off_delta);
    double2 *Valt = (double2 *)(base + off_valt);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    // The array keeps the previous call's contents: zero the counters, and f64_init resets the
    // per-column state (flags, iteration counts, steps) that the sweeps read.
    TPF_CK(cudaMemsetAsync(counters, 0, sizeof(int) * 8, st));
    {
        int64_t work = cols > T * n ? cols : T * n;
        f64_init<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(T, cols, n, given_start ? 0 : 1, (double2 *)V_dev,
                                                                  flags, iters, delta);
    }
    TPF_CK(cudaGetLastError());
    double2 *buf[2] = {(double2 *)V_dev, Valt};
    const dim3 grid((unsigned)((T + F64_BN - 1) / F64_BN), (n + F64_BM - 1) / F64_BM);
    int host_counters[8] = {0};
    for (int k = 0; k < max_iter; ++k) {
        f64_sweep<<<grid, 256, 0, st>>>((const double2 *)K_dev, (const double2 *)W_dev, (const double2 *)S_dev,
                                        buf[k & 1], buf[(k + 1) & 1], n, T, flags, delta, nullptr);
        TPF_CK(cudaMemsetAsync(counters, 0, sizeof(int) * 4, st));
        f64_decide<<<(unsigned)((T + 255) / 256), 256, 0, st>>>(T, tol, max_iter, flags, iters, delta, counters);
        TPF_CK(cudaGetLastError());
        TPF_CK(cudaMemcpyAsync(host_counters, counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
        TPF_CK(cudaStreamSynchronize(st));
        if (host_counters[kCntActive] == 0) break;
    }
    f64_finish<<<(unsigned)((T * 32 + 255) / 256), 256, 0, st>>>(T, n, max_iter, flags, iters, (double2 *)V_dev,
                                                                 Valt, (const double2 *)S_dev, nullptr, nullptr,
                                                                 nullptr, nullptr, nullptr, nullptr, iters_dev,
                                                                 nullptr);
    TPF_CK(cudaGetLastError());
    TPF_CK(cudaMemcpyAsync(host_counters, counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
    TPF_CK(cudaStreamSynchronize(st));
    return host_counters[kCntConverged] == T ? TPF_OK : TPF_ENOCONV;
}
