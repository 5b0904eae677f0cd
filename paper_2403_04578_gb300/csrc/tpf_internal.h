// Internal declarations shared by the host and device translation units of libtpf.
#pragma once

#include <atomic>
#include <cstdint>
#include <vector>

#include "../../include/tpf.h"

#ifdef __CUDACC__
#include <cuda_fp16.h>
#endif
#include <cuda_runtime.h>

namespace tpf {

// Row padding of the tensor-core operands: the bus dimension is padded to a multiple of the
// 64-element (128-byte) K chunk and of the 128-row M tile.
constexpr int kChunkK = 64;
constexpr int kTileM = 128;
constexpr int kTileN = 128;

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Runs set() (a kernel attribute, which is per device) once for the current device: `done` holds
// one bit per device, devices past the 64th run it every time.  False when set() or the device
// query fails (the CUDA error is cleared).
template <class F>
bool once_per_device(std::atomic<uint64_t> &done, F set) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const uint64_t bit = dev >= 0 && dev < 64 ? 1ull << dev : 0;
    if (bit && (done.load(std::memory_order_relaxed) & bit)) return true;
    if (!set()) {
        cudaGetLastError();
        return false;
    }
    done.fetch_or(bit, std::memory_order_relaxed);
    return true;
}

// Sparse formulation: demand buses per thread (2, 4 or 8; 16 for the large-feeder kernel, whose
// D, S and z live in a device scratch), largest block, and the block size for n demand buses with
// bpt buses per thread: the fewest whole warps that hold them (0 when n does not fit one block).
constexpr int kTreeMaxThreads = 512;
constexpr int kTreeBigBPT = 16;
constexpr int kTreeBigMaxThreads = 384;  // 168 registers per thread
int tree_bpt(int n);  // the choice for n demand buses (TPF_TREE_BPT overrides it)
inline int tree_threads(int n, int bpt) {
    const int t = ((n + bpt - 1) / bpt + 31) / 32 * 32;
    const int cap = bpt == kTreeBigBPT ? kTreeBigMaxThreads : kTreeMaxThreads;
    return t < 32 ? 32 : (t <= cap ? t : 0);
}

// Host-side result of the network preprocessing (Eq. 1 and Eq. 3).
struct Network {
    int n_bus = 0, n_pq = 0, slack = 0;
    double vs_re = 1.0, vs_im = 0.0;
    bool radial = false;
    std::vector<int> pq;          // column position -> bus
    std::vector<int> pos;         // bus -> column position, -1 for the slack
    std::vector<double> K;        // complex [n_pq][n_pq], K = -Y_dd^{-1} (radial: built on demand)
    // Radial networks: breadth-first bus order from the slack, each bus's parent and the complex
    // impedance of the branch to it (bus-indexed), from which compute_dense builds K.
    std::vector<int> bfs_order, bus_parent;
    std::vector<double> bus_z;
    std::vector<double> W;        // complex [n_pq], W = K Y_ds v_s
    // Neighbour lists of the demand buses (CSR over column positions): for each bus i, the
    // other end j of every branch at i (-1 = the slack) and that branch's admittance y = 1/z.
    std::vector<int> row_ptr, nbr;
    std::vector<double> y;        // complex [nnz]
    // Radial networks only: the parent of each demand bus (column position, -1 = the slack), the
    // admittance of the branch to it, and each bus's children (CSR over column positions).
    std::vector<int> par, ch_ptr, ch;
    std::vector<double> ypar;     // complex [n_pq]
    // Radial networks only, in depth-first preorder positions q of the demand buses: the column
    // of each position, the end of its subtree's position range [q, dfs_end[q]), the impedance of
    // the branch to its parent and the positions whose range ends at q (CSR dfs_eptr / dfs_ends).
    // Polyphase networks repeat the positions once per phase (position p n_bus_pq + q for phase p)
    // and carry, per position, the row p of the branch's impedance and admittance blocks.
    std::vector<int> dfs_col, dfs_end, dfs_eptr, dfs_ends;
    std::vector<double> dfs_z;  // complex [positions]
    // Polyphase networks (phases > 1): unknowns are (demand bus, phase), index i*phases + p; the
    // slack holds vs[p]; the neighbour lists above run over unknowns and also name, per entry, the
    // unknown of the own bus whose voltage the entry's admittance multiplies (csr_self), so that
    // (Y v)_u = sum_e y_e (v[csr_self_e] - v[nbr_e]) with nbr_e = -1 - p' for slack phase p'.
    int phases = 1;
    std::vector<double> vs;       // complex [phases]
    std::vector<int> csr_self;    // [nnz] (phases > 1)
    std::vector<double> dfs_zrow, dfs_yrow;  // complex [positions][phases]
};

// Build K (radial networks build it here, on first need; a no-op when it exists).
void compute_dense(Network &net);

// The same for a polyphase network (phases x phases branch blocks, interleaved complex).
tpf_status build_network_poly(int n_bus, int n_branch, int phases, const int32_t *from, const int32_t *to,
                              const double *z_pu, int slack, const double *v0, int n_pq, const int32_t *pq_bus,
                              Network &net);

// Build the network arrays; returns TPF_OK or the status to report.
tpf_status build_network(int n_bus, int n_branch, const int32_t *from, const int32_t *to,
                         const double *z_pu, int slack, double v0_re, double v0_im, int n_pq,
                         const int32_t *pq_bus, Network &net);

// Device copies owned by a handle.
struct DeviceNet {
    int n = 0;           // n_pq
    int n_pad = 0;       // n rounded up to kTileM (and hence to kChunkK)
    // FP64 path
    double *K64 = nullptr;   // complex [n][n]
    double *W64 = nullptr;   // complex [n]
    int *row_ptr = nullptr, *nbr = nullptr;
    double *y64 = nullptr;   // complex [nnz]
    float4 *y2f = nullptr;   // double-float complex admittance (re_hi, im_hi, re_lo, im_lo) [nnz]
    bool radial = false;
    int *par = nullptr, *ch_ptr = nullptr, *ch = nullptr;  // radial only
    float2 *ypar = nullptr;  // FP32 admittance of the branch to the parent [n]
    // Sparse formulation (radial only).  Block of t_threads threads per column; thread k owns the
    // t_bpt consecutive depth-first positions q = t_bpt k + j, stored at slot
    // s = j t_threads + k (so that a warp touches consecutive words).  Per slot: the column (-1
    // past n), the end of the subtree's position range, the parent's slot (-1 = the slack), the
    // start and count (start | count << 16) in t_ends of the slots of the positions whose
    // subtree range ends at q, and the double-float z of the branch to the parent
    // (re_hi, im_hi, re_lo, im_lo).
    int t_threads = 0, t_bpt = 0, t_n_ends = 0;
    int *t_col = nullptr, *t_end = nullptr, *t_par = nullptr, *t_ecnt = nullptr, *t_ends = nullptr;
    int *t_kidx = nullptr;  // per slot: the index in t_ends at which its position appears, or -1
    float4 *t_z = nullptr;
    double2 *t_z64 = nullptr;  // FP64 z per slot (single phase), for the FP64 sparse kernel
    // ZIP load coefficients (Eq. 3), set by tpf_set_zip; null for constant power.  zip64: double
    // [3][n] in column order (FP64 path); t_zip_hi / t_zip_lo: float4 (alpha_P, alpha_I, alpha_Z, 0)
    // per slot, high and low words (sparse path).
    double *zip64 = nullptr;
    float4 *t_zip_hi = nullptr, *t_zip_lo = nullptr;
    // Polyphase networks: phases, demand buses per phase block (n = nbp * phases unknowns), the
    // unknown each neighbour-list entry's admittance multiplies (null when phases == 1), v_s per
    // phase (complex, also for phases == 1), and per slot the rows p of the branch's impedance
    // (double-float, [ns][phases]) and admittance (FP32) blocks.
    int phases = 1, nbp = 0;
    int *csr_self = nullptr;
    double *vs64 = nullptr;
    float4 *t_zrow = nullptr;
    float2 *t_yrow = nullptr;
    float2 *t_zrow_f = nullptr;  // the high words of t_zrow (the sweeps' FP32 impedance rows)
    // Mixed path: fp16 planes of K * 2^k_exp, [n_pad][n_pad], zero padded
    void *Kr16 = nullptr, *Ki16 = nullptr;
    int k_exp = 0;
    // Incremented whenever the sparse layout or the ZIP coefficients are replaced: a prepared
    // batch (tpf_batch) that captured the old device arrays then refuses to launch.
    int layout_gen = 0;
};

// Workspaces of a solve, grown on demand.
struct Workspace {
    int64_t cap_cols = 0;     // columns allocated (multiple of kTileN)
    int n_pad = 0;
    // mixed path
    // V = Vhi + Vlo: before a column is anchored Vhi carries V and Vlo = 0; after, Vhi is the
    // frozen anchor V_ref and Vlo the offset from it.  S = Shi + Slo.  RefHi + RefLo hold
    // rho(V_ref) in double-float.
    float2 *Vhi = nullptr, *Vlo = nullptr, *Shi = nullptr, *Slo = nullptr;  // [cols][n_pad]
    float2 *RefHi = nullptr, *RefLo = nullptr;                              // [cols][n_pad]
    void *Rr16 = nullptr, *Ri16 = nullptr;                                  // fp16 [cols][n_pad]
    unsigned int *dprev = nullptr;        // float bits of the step before the last (mixed)
    // FP64 path: second V buffer, complex128 [cols][n]
    double *Valt = nullptr;
    // per-column state
    unsigned int *delta_bits = nullptr;   // float bits (mixed) of the last max|dV|
    unsigned long long *delta64 = nullptr;// double bits (FP64 path)
    int *iters = nullptr;
    int *flags = nullptr;
    int *rexp = nullptr;
    int *tile_active = nullptr;           // [cols / kTileN]
    int *counters = nullptr;              // [8] device counters
    int *counters_host = nullptr;         // pinned mirror
    // large-feeder sparse kernel: per-block slices of D, (S_hi, z) and the ZIP coefficients
    float4 *tree_scratch = nullptr;
    size_t tree_scratch_bytes = 0;
    // host-solve staging
    int64_t host_cap = 0;
    void *S_dev = nullptr, *V_dev = nullptr;
    int32_t *it_dev = nullptr;
    double *mm_dev = nullptr;
};

// kAnchored: the column's residual is rho(V_ref) + FP32 corrections in V - V_ref.
// kBlind: anchored at a given starting point (not yet at a small step); re-anchored once the step
// falls below switch_tol.
enum ColFlags : int { kActive = 1, kAnchored = 2, kDone = 4, kBlind = 8 };
enum Counter : int { kCntActive = 0, kCntPrecise = 1, kCntError = 2, kCntConverged = 4 };

// Makes `dev` the current device for the lifetime of the scope and then gives the caller's current
// device back, so that an entry point of the library never changes which device its caller uses.
struct DeviceScope {
    int prev = -1;
    bool ok = false;
    explicit DeviceScope(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        ok = (prev == dev) || cudaSetDevice(dev) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    ~DeviceScope() {
        if (prev >= 0) {
            int cur = -1;
            if (cudaGetDevice(&cur) != cudaSuccess || cur != prev) cudaSetDevice(prev);
            cudaGetLastError();
        }
    }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;
};

// CUDA-event timing of kernel launches by category (only when a solve asks for it).
struct KernelTimer {
    enum { kGemm = 0, kResidual = 1, kOther = 2 };
    bool on = false;
    cudaStream_t st = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[3];
    int cur = -1;
    KernelTimer(bool enable, cudaStream_t s) : on(enable), st(s) {}
    void begin(int cat) {
        if (!on) return;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
        ev[cat].push_back({a, b});
        cur = cat;
    }
    void end() {
        if (!on || cur < 0) return;
        cudaEventRecord(ev[cur].back().second, st);
        cur = -1;
    }
    // Call after the stream has been synchronised.
    double total_ms(int cat) const {
        double s = 0.0;
        for (auto &p : ev[cat]) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) s += ms;
        }
        return s;
    }
    ~KernelTimer() {
        for (auto &v : ev)
            for (auto &p : v) {
                cudaEventDestroy(p.first);
                cudaEventDestroy(p.second);
            }
    }
};

}  // namespace tpf

struct tpf_handle {
    int device = 0;
    tpf::Network net;
    tpf::DeviceNet dev;
    tpf::Workspace ws;
    tpf_stats stats{};
    int64_t start_fallback = 0;  // columns of the last learned-start solve that started flat
    void *tmaps = nullptr;  // tensor maps of the fp16 K planes (opaque, allocated by the mixed path)
};

namespace tpf {
// Upload the network to the device (tpf_create).
tpf_status upload_network(tpf_handle *h);
// Upload K, W and the fp16 planes of K on first use by a dense solve.
tpf_status ensure_dense(tpf_handle *h);
// (Re)build the sparse formulation's slot layout for bpt positions per thread (0: none).
tpf_status layout_tree(tpf_handle *h, int bpt);
// Time the sparse kernel's block shapes on T sample columns and keep the fastest.
tpf_status autotune_sparse(tpf_handle *h, int64_t T, const void *S, const tpf_opts &o, cudaStream_t st,
                           int *bpt_out);
// Upload (alpha != null, host [3][n]) or drop the ZIP coefficients.
tpf_status set_zip(tpf_handle *h, const double *alpha);
void free_device(tpf_handle *h);
// Ensure workspaces for `cols` columns: kind 0 = FP64 path, 1 = mixed path, 2 = per-column state only.
enum WorkspaceKind : int { kWsFp64 = 0, kWsMixed = 1, kWsState = 2 };
tpf_status ensure_workspace(tpf_handle *h, int64_t cols, int kind);
// The two solve paths.  Return TPF_OK / TPF_ENOCONV / errors.
tpf_status solve_fp64(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters,
                      double *mismatch, const tpf_opts &o, cudaStream_t st);
tpf_status solve_mixed(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters,
                       double *mismatch, const tpf_opts &o, cudaStream_t st);
tpf_status solve_sparse(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters,
                        double *mismatch, const tpf_opts &o, cudaStream_t st);
// V0_pred (optional, device half2 deviations (Re V - 1, Im V) per bus, column t at
// V0_pred + t * v0_pitch, v0_pitch >= n; 0 = n): a warm start read from a prediction instead of
// from V; a column whose prediction has some |V_i| outside [0.7, 1.1] starts flat (counted in
// h->start_fallback).
tpf_status solve_sparse_ex(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters,
                           double *mismatch, const tpf_outputs *out, const tpf_opts &o, cudaStream_t st,
                           const void *V0_pred = nullptr, int64_t v0_pitch = 0);
// The sparse formulation in plain FP64 (radial, single phase, up to 4,096 demand buses).
tpf_status solve_tree64(tpf_handle *h, int64_t T, const void *S, void *V, int32_t *iters,
                        double *mismatch, const tpf_opts &o, cudaStream_t st);
size_t tree64_smem(int threads, int bpt);
tpf_status solve_batch_sparse(int F, tpf_handle *const *hs, const int64_t *T, const void *const *S,
                              void *const *V, int32_t *const *iters, double *const *mismatch,
                              const tpf_opts &o, int64_t *conv_out, tpf_stats *stats, cudaStream_t st);
// A prepared batch of radial feeders under the sparse method (arguments checked by the caller):
// its work table on the device and a CUDA graph of one solve of all of them.
tpf_status batch_plan_create(int F, tpf_handle *const *hs, const int64_t *T, const void *const *S,
                             void *const *V, int32_t *const *iters, double *const *mismatch,
                             const tpf_opts &o, tpf_batch **out);
tpf_status batch_plan_launch(tpf_batch *b, cudaStream_t st);
tpf_status batch_plan_wait(tpf_batch *b, int64_t *conv_out, tpf_stats *stats);
void batch_plan_destroy(tpf_batch *b);
int batch_device(const tpf_batch *b);
tpf_status selftest_gemm(int M, int N, int K, const void *Ar, const void *Ai, const void *Br,
                         const void *Bi, float *Dr, float *Di, cudaStream_t st, uint64_t wait_ns = 0,
                         int withhold_loads = 0);
}  // namespace tpf
