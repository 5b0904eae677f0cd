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
// Per sweep:  mx_residual  (tpf_residual.cu, one block per column) decides convergence from the
//                          last step, forms rho (FP32 far from convergence, then against a
//                          double-float anchor), scales it by a per-column power of two and
//                          writes the fp16 B operand;
//             tc_gemm      (tpf_gemm.cu, persistent, warp-specialised) computes K rho with four
//                          real-plane MMAs per K step (Re = Kr rr - Ki ri, Im = Kr ri + Ki rr)
//                          over 128 x 128 tiles; its epilogue adds the update to V and folds
//                          max |dV| per column.
// This file holds the packing and output kernels and the host loop of a solve.
#include <cuda_fp16.h>

#include <cstdlib>
#include <cstring>

#include "tpf_dd.cuh"
#include "tpf_gemm.h"

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
// Elementwise kernels
// ------------------------------------------------------------------------------------------

// Split S (and V_0) into double-float planes with padded rows; one block per column.  A warm start
// (v0_lo == 0) keeps only fl32(V_0): its FP32 sweeps run on the high plane.
__global__ void mx_pack(int64_t T, int n, int n_pad, const double2 *__restrict__ S, const double2 *__restrict__ V0,
                        int v0_lo, float2 *Shi, float2 *Slo, float2 *Vhi, float2 *Vlo, int *flags, int *iters,
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
                if (v0_lo)
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

}  // namespace

tpf_status selftest_gemm(int M, int N, int K, const void *Ar, const void *Ai, const void *Br, const void *Bi, float *Dr,
                         float *Di, cudaStream_t st, uint64_t wait_ns, int withhold_loads) {
    GemmMaps maps;
    if (!make_gemm_maps(&maps, Ar, Ai, M, K, Br, Bi, N)) return TPF_ECUDA;
    int *err = nullptr;
    TPF_CK(cudaMalloc(&err, sizeof(int)));
    TPF_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    GemmEpi ep{};
    ep.mode = 0;
    ep.cplx = 1;
    ep.err = err;
    ep.Dr = Dr;
    ep.Di = Di;
    ep.ldD = M;
    ep.wait_ns = wait_ns;
    ep.withhold_loads = withhold_loads;
    tpf_status rs = launch_gemm(maps, M / kTileM, N / kTileN, K / kChunkK, ep, st);
    int herr = 0;
    cudaError_t e = cudaSuccess;
    if (rs == TPF_OK) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (rs == TPF_OK && e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(err);
    if (rs != TPF_OK) return rs;
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
    if (h->dev.zip64) return TPF_EUNSUPPORTED;    // ZIP loads: sparse formulation or FP64 path
    if (h->dev.phases > 1) return TPF_EUNSUPPORTED;  // polyphase: sparse formulation or FP64 path
    tpf_status rs = ensure_dense(h);
    if (rs != TPF_OK) return rs;
    rs = ensure_workspace(h, T, kWsMixed);
    if (rs != TPF_OK) return rs;
    Workspace &w = h->ws;
    const int64_t cols = round_up(T, kTileN);
    GemmMaps maps;
    if (!make_gemm_maps(&maps, h->dev.Kr16, h->dev.Ki16, n_pad, n_pad, w.Rr16, w.Ri16, cols)) return TPF_ECUDA;
    int64_t launches = 0, gemm_cols = 0;
    KernelTimer timer(o.profile != 0, st);
    TPF_CK(cudaMemsetAsync(w.counters, 0, sizeof(int) * 8, st));
    timer.begin(KernelTimer::kOther);
    mx_pack<<<(unsigned)cols, 256, 0, st>>>(T, n, n_pad, (const double2 *)S,
                                             o.start != TPF_START_FLAT ? (const double2 *)V : nullptr,
                                             o.start == TPF_START_GIVEN, w.Shi, w.Slo,
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
    ep.cplx = 1;
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

    int sweeps = 0, precise_sweeps = 0;
    const int64_t n_tiles = cols / kTileN;
    std::vector<int> tile_host(n_tiles);
    for (int s = 0; s <= o.max_iter; ++s) {
        TPF_CK(cudaMemsetAsync(w.tile_active, 0, sizeof(int) * (cols / kTileN), st));
        TPF_CK(cudaMemsetAsync(w.counters, 0, sizeof(int) * 2, st));  // active, precise
        pa.sweep = s;
        timer.begin(KernelTimer::kResidual);
        rs = launch_residual(pa, st);
        timer.end();
        if (rs != TPF_OK) return rs;
        ++launches;
        TPF_CK(cudaMemcpyAsync(w.counters_host, w.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
        TPF_CK(cudaMemcpyAsync(tile_host.data(), w.tile_active, sizeof(int) * n_tiles, cudaMemcpyDeviceToHost, st));
        TPF_CK(cudaStreamSynchronize(st));
        if (w.counters_host[kCntError]) return TPF_ETIMEOUT;
        int64_t active = 0;
        for (int64_t k = 0; k < n_tiles; ++k) active += tile_host[k];
        if (active == 0) break;
        if (w.counters_host[kCntPrecise] > 0) ++precise_sweeps;
        gemm_cols += active;
        timer.begin(KernelTimer::kGemm);
        rs = launch_gemm(maps, n_pad / kTileM, cols / kTileN, n_pad / kChunkK, ep, st);
        timer.end();
        if (rs != TPF_OK) return rs;
        ++launches;
        ++sweeps;
        TPF_CK(cudaGetLastError());
    }
    TPF_CK(cudaMemsetAsync(w.tile_active, 0, sizeof(int) * n_tiles, st));  // reused: converged per tile
    timer.begin(KernelTimer::kOther);
    rs = launch_final(pa, T, V, iters, mismatch, w.tile_active, st);
    timer.end();
    if (rs != TPF_OK) return rs;
    ++launches;
    TPF_CK(cudaMemcpyAsync(w.counters_host, w.counters, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
    TPF_CK(cudaMemcpyAsync(tile_host.data(), w.tile_active, sizeof(int) * n_tiles, cudaMemcpyDeviceToHost, st));
    TPF_CK(cudaStreamSynchronize(st));
    int64_t converged = 0;
    for (int64_t k = 0; k < n_tiles; ++k) converged += tile_host[k];
    h->stats.sweeps = sweeps;
    h->stats.precise_sweeps = precise_sweeps;
    h->stats.kernel_launches = launches;
    h->stats.converged = converged;
    h->stats.gemm_launches = sweeps;
    h->stats.gemm_columns = gemm_cols;
    h->stats.gemm_ms = timer.total_ms(KernelTimer::kGemm);
    h->stats.residual_ms = timer.total_ms(KernelTimer::kResidual);
    h->stats.other_ms = timer.total_ms(KernelTimer::kOther);
    if (w.counters_host[kCntError]) return TPF_ETIMEOUT;
    return h->stats.converged == T ? TPF_OK : TPF_ENOCONV;
}

}  // namespace tpf
