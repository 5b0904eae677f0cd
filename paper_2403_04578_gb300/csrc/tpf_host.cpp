// Host side of libtpf: network preprocessing (Eq. 1 and Eq. 3), handle lifetime and the public
// entry points that dispatch to the FP64 and mixed solve paths.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <queue>

#include "tpf_internal.h"

using cplx = std::complex<double>;

namespace tpf {

namespace {

// Dense inverse by LU with partial pivoting (used for networks that are not trees).
bool lu_inverse(int n, std::vector<cplx> &A /* in: A, out: A^{-1}, row-major */) {
    std::vector<int> piv(n);
    double scale = 0.0;
    for (const cplx &v : A) scale = std::max(scale, std::abs(v));
    for (int c = 0; c < n; ++c) {
        int p = c;
        double best = std::abs(A[(size_t)c * n + c]);
        for (int r = c + 1; r < n; ++r) {
            double v = std::abs(A[(size_t)r * n + c]);
            if (v > best) { best = v; p = r; }
        }
        if (!(best > 0.0) || best < 1e-14 * scale) return false;
        piv[c] = p;
        if (p != c)
            for (int j = 0; j < n; ++j) std::swap(A[(size_t)c * n + j], A[(size_t)p * n + j]);
        cplx inv = 1.0 / A[(size_t)c * n + c];
        for (int r = c + 1; r < n; ++r) {
            cplx f = A[(size_t)r * n + c] * inv;
            A[(size_t)r * n + c] = f;
            if (f == cplx(0.0)) continue;
            for (int j = c + 1; j < n; ++j) A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
        }
    }
    // Solve A X = P^T I column by column.
    std::vector<cplx> X((size_t)n * n), col(n);
    for (int j = 0; j < n; ++j) {
        std::fill(col.begin(), col.end(), cplx(0.0));
        col[j] = 1.0;
        for (int c = 0; c < n; ++c) std::swap(col[c], col[piv[c]]);  // apply row swaps in order
        for (int r = 0; r < n; ++r) {  // forward (unit lower)
            cplx s = col[r];
            for (int k = 0; k < r; ++k) s -= A[(size_t)r * n + k] * col[k];
            col[r] = s;
        }
        for (int r = n - 1; r >= 0; --r) {  // backward
            cplx s = col[r];
            for (int k = r + 1; k < n; ++k) s -= A[(size_t)r * n + k] * col[k];
            col[r] = s / A[(size_t)r * n + r];
        }
        for (int r = 0; r < n; ++r) X[(size_t)r * n + j] = col[r];
    }
    A.swap(X);
    return true;
}

}  // namespace

tpf_status build_network(int n_bus, int n_branch, const int32_t *from, const int32_t *to,
                         const double *z_pu, int slack, double v0_re, double v0_im, int n_pq,
                         const int32_t *pq_bus, Network &net) {
    if (n_bus < 2 || n_branch < n_bus - 1 || n_pq != n_bus - 1) return TPF_EINVAL;
    if (!from || !to || !z_pu || !pq_bus) return TPF_EINVAL;
    if (slack < 0 || slack >= n_bus) return TPF_EINVAL;
    if (!std::isfinite(v0_re) || !std::isfinite(v0_im)) return TPF_EINVAL;
    net = Network();
    net.n_bus = n_bus;
    net.n_pq = n_pq;
    net.slack = slack;
    net.vs_re = v0_re;
    net.vs_im = v0_im;
    net.pos.assign(n_bus, -2);
    net.pos[slack] = -1;
    net.pq.assign(pq_bus, pq_bus + n_pq);
    for (int i = 0; i < n_pq; ++i) {
        int b = pq_bus[i];
        if (b < 0 || b >= n_bus || net.pos[b] != -2) return TPF_EINVAL;  // out of range, slack or repeated
        net.pos[b] = i;
    }
    // Adjacency with branch admittances y = 1/z (Eq. 1 without shunts).
    std::vector<std::vector<std::pair<int, cplx>>> adj(n_bus);
    for (int e = 0; e < n_branch; ++e) {
        int a = from[e], b = to[e];
        if (a < 0 || b < 0 || a >= n_bus || b >= n_bus || a == b) return TPF_EINVAL;
        cplx z(z_pu[2 * e], z_pu[2 * e + 1]);
        if (!std::isfinite(z.real()) || !std::isfinite(z.imag()) || std::abs(z) == 0.0) return TPF_EINVAL;
        cplx y = 1.0 / z;
        adj[a].push_back({b, y});
        adj[b].push_back({a, y});
    }
    // Connectivity from the slack.
    std::vector<int> parent(n_bus, -2), order;
    std::vector<cplx> zpar(n_bus, 0.0);
    order.reserve(n_bus);
    parent[slack] = -1;
    order.push_back(slack);
    for (size_t q = 0; q < order.size(); ++q) {
        int u = order[q];
        for (auto &nb : adj[u]) {
            if (parent[nb.first] == -2) {
                parent[nb.first] = u;
                zpar[nb.first] = 1.0 / nb.second;
                order.push_back(nb.first);
            }
        }
    }
    if ((int)order.size() != n_bus) return TPF_ESINGULAR;
    net.radial = (n_branch == n_bus - 1);

    const int n = n_pq;
    if (net.radial) {
        // K is built on demand (compute_dense): the sparse formulation never needs it.
        net.bfs_order = order;
        net.bus_parent = parent;
        net.bus_z.assign(2 * (size_t)n_bus, 0.0);
        for (int b = 0; b < n_bus; ++b) {
            net.bus_z[2 * b] = zpar[b].real();
            net.bus_z[2 * b + 1] = zpar[b].imag();
        }
    } else {
        net.K.assign((size_t)2 * n * n, 0.0);
        std::vector<cplx> Ydd((size_t)n * n, 0.0);
        for (int i = 0; i < n; ++i) {
            int b = net.pq[i];
            for (auto &nb : adj[b]) {
                Ydd[(size_t)i * n + i] += nb.second;
                if (nb.first != slack) Ydd[(size_t)i * n + net.pos[nb.first]] -= nb.second;
            }
        }
        if (!lu_inverse(n, Ydd)) return TPF_ESINGULAR;
        for (size_t k = 0; k < (size_t)n * n; ++k) {
            net.K[2 * k] = -Ydd[k].real();
            net.K[2 * k + 1] = -Ydd[k].imag();
        }
    }
    // W = K Y_ds v_s.  Without shunts every row of Y sums to zero, so Y_dd 1 = -Y_ds and
    // W = -Y_dd^{-1} Y_ds v_s = v_s at every demand bus.
    net.W.assign((size_t)2 * n, 0.0);
    for (int i = 0; i < n; ++i) {
        net.W[2 * i] = v0_re;
        net.W[2 * i + 1] = v0_im;
    }
    // Tree arrays in column positions (radial networks).
    if (net.radial) {
        net.par.assign(n, -1);
        net.ypar.assign((size_t)2 * n, 0.0);
        std::vector<int> nch(n, 0);
        for (int i = 0; i < n; ++i) {
            int b = net.pq[i], p = parent[b];
            net.par[i] = net.pos[p];  // -1 for the slack
            cplx y = 1.0 / zpar[b];
            net.ypar[2 * i] = y.real();
            net.ypar[2 * i + 1] = y.imag();
            if (net.par[i] >= 0) ++nch[net.par[i]];
        }
        net.ch_ptr.assign(n + 1, 0);
        for (int i = 0; i < n; ++i) net.ch_ptr[i + 1] = net.ch_ptr[i] + nch[i];
        net.ch.assign(net.ch_ptr[n], 0);
        std::vector<int> fill(net.ch_ptr.begin(), net.ch_ptr.end() - 1);
        for (int i = 0; i < n; ++i)
            if (net.par[i] >= 0) net.ch[fill[net.par[i]]++] = i;
        // Depth-first preorder of the demand buses: the subtree of the bus at position q is the
        // position range [q, dfs_end[q]).
        net.dfs_col.clear();
        net.dfs_col.reserve(n);
        std::vector<int> stack, posdfs(n_bus, -1);
        std::vector<std::vector<int>> kids(n_bus);
        for (size_t q = 1; q < order.size(); ++q) kids[parent[order[q]]].push_back(order[q]);
        for (auto it = kids[slack].rbegin(); it != kids[slack].rend(); ++it) stack.push_back(*it);
        while (!stack.empty()) {
            const int u = stack.back();
            stack.pop_back();
            posdfs[u] = (int)net.dfs_col.size();
            net.dfs_col.push_back(net.pos[u]);
            for (auto it = kids[u].rbegin(); it != kids[u].rend(); ++it) stack.push_back(*it);
        }
        std::vector<int> size(n_bus, 1);
        for (size_t q = order.size() - 1; q >= 1; --q) size[parent[order[q]]] += size[order[q]];
        net.dfs_end.assign(n, 0);
        net.dfs_z.assign((size_t)2 * n, 0.0);
        std::vector<int> nend(n + 1, 0);
        for (int i = 0; i < n; ++i) {
            const int b = net.pq[i], q = posdfs[b];
            net.dfs_end[q] = q + size[b];
            net.dfs_z[2 * q] = zpar[b].real();
            net.dfs_z[2 * q + 1] = zpar[b].imag();
            ++nend[net.dfs_end[q]];
        }
        // For each position q < n, the positions whose subtree range ends at q.
        net.dfs_eptr.assign(n + 1, 0);
        for (int q = 0; q < n; ++q) net.dfs_eptr[q + 1] = net.dfs_eptr[q] + nend[q];
        net.dfs_ends.assign(net.dfs_eptr[n], 0);
        std::vector<int> fill_e(net.dfs_eptr.begin(), net.dfs_eptr.end() - 1);
        for (int q = 0; q < n; ++q)
            if (net.dfs_end[q] < n) net.dfs_ends[fill_e[net.dfs_end[q]]++] = q;
    }
    // Neighbour lists in column positions.
    net.row_ptr.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) net.row_ptr[i + 1] = net.row_ptr[i] + (int)adj[net.pq[i]].size();
    net.nbr.resize(net.row_ptr[n]);
    net.y.resize((size_t)2 * net.row_ptr[n]);
    for (int i = 0; i < n; ++i) {
        int k = net.row_ptr[i];
        for (auto &nb : adj[net.pq[i]]) {
            net.nbr[k] = net.pos[nb.first];  // -1 for the slack
            net.y[2 * k] = nb.second.real();
            net.y[2 * k + 1] = nb.second.imag();
            ++k;
        }
    }
    return TPF_OK;
}

tpf_status build_network_poly(int n_bus, int n_branch, int phases, const int32_t *from, const int32_t *to,
                              const double *z_pu, int slack, const double *v0, int n_pq, const int32_t *pq_bus,
                              Network &net) {
    const int ph = phases;
    if (ph < 2 || ph > 3) return TPF_EINVAL;
    if (n_bus < 2 || n_branch < n_bus - 1 || n_pq != n_bus - 1) return TPF_EINVAL;
    if (!from || !to || !z_pu || !pq_bus || !v0) return TPF_EINVAL;
    if (slack < 0 || slack >= n_bus) return TPF_EINVAL;
    for (int p = 0; p < 2 * ph; ++p)
        if (!std::isfinite(v0[p])) return TPF_EINVAL;
    net = Network();
    net.n_bus = n_bus;
    net.phases = ph;
    net.n_pq = n_pq * ph;
    net.slack = slack;
    net.vs.assign(v0, v0 + 2 * ph);
    net.vs_re = v0[0];
    net.vs_im = v0[1];
    net.pos.assign(n_bus, -2);
    net.pos[slack] = -1;
    net.pq.assign(pq_bus, pq_bus + n_pq);
    for (int i = 0; i < n_pq; ++i) {
        const int b = pq_bus[i];
        if (b < 0 || b >= n_bus || net.pos[b] != -2) return TPF_EINVAL;
        net.pos[b] = i;
    }
    // Branch admittance blocks Y_e = Z_e^{-1} (phases x phases, by LU).
    std::vector<std::vector<std::pair<int, int>>> adj(n_bus);  // (other bus, branch)
    std::vector<cplx> Yb((size_t)n_branch * ph * ph), Zb((size_t)n_branch * ph * ph);
    for (int e = 0; e < n_branch; ++e) {
        const int a = from[e], b = to[e];
        if (a < 0 || b < 0 || a >= n_bus || b >= n_bus || a == b) return TPF_EINVAL;
        std::vector<cplx> blk(ph * ph);
        for (int k = 0; k < ph * ph; ++k) {
            const cplx z(z_pu[2 * ((size_t)e * ph * ph + k)], z_pu[2 * ((size_t)e * ph * ph + k) + 1]);
            if (!std::isfinite(z.real()) || !std::isfinite(z.imag())) return TPF_EINVAL;
            blk[k] = z;
            Zb[(size_t)e * ph * ph + k] = z;
        }
        if (!lu_inverse(ph, blk)) return TPF_EINVAL;  // a singular branch matrix
        std::copy(blk.begin(), blk.end(), Yb.begin() + (size_t)e * ph * ph);
        adj[a].push_back({b, e});
        adj[b].push_back({a, e});
    }
    std::vector<int> parent(n_bus, -2), pbranch(n_bus, -1), order;
    order.reserve(n_bus);
    parent[slack] = -1;
    order.push_back(slack);
    for (size_t q = 0; q < order.size(); ++q) {
        const int u = order[q];
        for (auto &nb : adj[u])
            if (parent[nb.first] == -2) {
                parent[nb.first] = u;
                pbranch[nb.first] = nb.second;
                order.push_back(nb.first);
            }
    }
    if ((int)order.size() != n_bus) return TPF_ESINGULAR;
    net.radial = (n_branch == n_bus - 1);
    // W = v_s phase by phase: with every bus at v_s no branch carries current, so
    // Y_dd (1 x v_s) + Y_ds v_s = 0 without shunts.
    net.W.assign(2 * (size_t)net.n_pq, 0.0);
    for (int i = 0; i < n_pq; ++i)
        for (int p = 0; p < ph; ++p) {
            net.W[2 * ((size_t)i * ph + p)] = v0[2 * p];
            net.W[2 * ((size_t)i * ph + p) + 1] = v0[2 * p + 1];
        }
    // Neighbour lists over unknowns u = i*ph + p: for each branch at bus i and each phase p',
    // y = Y_e[p][p'] multiplying (v_{i,p'} - v_{j,p'}).
    net.row_ptr.assign(net.n_pq + 1, 0);
    net.nbr.clear();
    net.y.clear();
    net.csr_self.clear();
    for (int i = 0; i < n_pq; ++i) {
        const int b = net.pq[i];
        for (int p = 0; p < ph; ++p) {
            for (auto &nb : adj[b]) {
                const cplx *Y = &Yb[(size_t)nb.second * ph * ph];
                for (int pp = 0; pp < ph; ++pp) {
                    net.csr_self.push_back(i * ph + pp);
                    net.nbr.push_back(nb.first == slack ? -1 - pp : net.pos[nb.first] * ph + pp);
                    net.y.push_back(Y[p * ph + pp].real());
                    net.y.push_back(Y[p * ph + pp].imag());
                }
            }
            net.row_ptr[i * ph + p + 1] = (int)net.nbr.size();
        }
    }
    if (net.radial) {
        // Depth-first positions of the demand buses, repeated per phase block (position
        // p*n_pq + q); a block's first position also closes the previous block's open path.
        std::vector<int> posdfs(n_bus, -1), dcol;
        std::vector<std::vector<int>> kids(n_bus);
        for (size_t q = 1; q < order.size(); ++q) kids[parent[order[q]]].push_back(order[q]);
        std::vector<int> stack;
        for (auto it = kids[slack].rbegin(); it != kids[slack].rend(); ++it) stack.push_back(*it);
        while (!stack.empty()) {
            const int u = stack.back();
            stack.pop_back();
            posdfs[u] = (int)dcol.size();
            dcol.push_back(u);
            for (auto it = kids[u].rbegin(); it != kids[u].rend(); ++it) stack.push_back(*it);
        }
        std::vector<int> size(n_bus, 1);
        for (size_t q = order.size() - 1; q >= 1; --q) size[parent[order[q]]] += size[order[q]];
        const int n = n_pq, P = n * ph;
        net.dfs_col.assign(P, 0);
        net.dfs_end.assign(P, 0);
        net.dfs_zrow.assign(2 * (size_t)P * ph, 0.0);
        net.dfs_yrow.assign(2 * (size_t)P * ph, 0.0);
        std::vector<std::vector<int>> ends_at(P + 1);
        std::vector<int> open_last;  // positions of block 0 whose range ends at n
        for (int q = 0; q < n; ++q) {
            const int b = dcol[q], e = pbranch[b];
            for (int p = 0; p < ph; ++p) {
                const int Q = p * n + q;
                net.dfs_col[Q] = net.pos[b] * ph + p;
                net.dfs_end[Q] = p * n + q + size[b];
                if (q + size[b] < n) ends_at[p * n + q + size[b]].push_back(Q);
                for (int pp = 0; pp < ph; ++pp) {
                    const cplx z = Zb[(size_t)e * ph * ph + p * ph + pp], y = Yb[(size_t)e * ph * ph + p * ph + pp];
                    net.dfs_zrow[2 * ((size_t)Q * ph + pp)] = z.real();
                    net.dfs_zrow[2 * ((size_t)Q * ph + pp) + 1] = z.imag();
                    net.dfs_yrow[2 * ((size_t)Q * ph + pp)] = y.real();
                    net.dfs_yrow[2 * ((size_t)Q * ph + pp) + 1] = y.imag();
                }
            }
            if (q + size[b] == n) open_last.push_back(q);
        }
        for (int p = 1; p < ph; ++p)
            for (int q : open_last) ends_at[p * n].push_back((p - 1) * n + q);
        net.dfs_eptr.assign(P + 1, 0);
        net.dfs_ends.clear();
        for (int Q = 0; Q < P; ++Q) {
            for (int b : ends_at[Q]) net.dfs_ends.push_back(b);
            net.dfs_eptr[Q + 1] = (int)net.dfs_ends.size();
        }
    }
    return TPF_OK;
}

void compute_dense(Network &net) {
    if (!net.K.empty()) return;
    if (net.phases > 1) {
        // Y_dd over unknowns from the neighbour lists (diagonal blocks from csr_self), then K by LU.
        const int N = net.n_pq;
        std::vector<cplx> Ydd((size_t)N * N, 0.0);
        for (int u = 0; u < N; ++u)
            for (int e = net.row_ptr[u]; e < net.row_ptr[u + 1]; ++e) {
                const cplx y(net.y[2 * e], net.y[2 * e + 1]);
                Ydd[(size_t)u * N + net.csr_self[e]] += y;
                if (net.nbr[e] >= 0) Ydd[(size_t)u * N + net.nbr[e]] -= y;
            }
        if (!lu_inverse(N, Ydd)) return;  // connected networks are nonsingular
        net.K.assign((size_t)2 * N * N, 0.0);
        for (size_t k = 0; k < (size_t)N * N; ++k) {
            net.K[2 * k] = -Ydd[k].real();
            net.K[2 * k + 1] = -Ydd[k].imag();
        }
        return;
    }
    if (!net.radial) return;
    // (Y_dd^{-1})_{ij} = impedance of the branches shared by the slack-to-i and slack-to-j paths.
    // For each j: mark j's ancestors with their path impedance, then a top-down pass gives every
    // bus the path impedance of its deepest marked ancestor.
    const int n = net.n_pq, n_bus = net.n_bus, slack = net.slack;
    const std::vector<int> &order = net.bfs_order, &parent = net.bus_parent;
    net.K.assign((size_t)2 * n * n, 0.0);
    std::vector<cplx> zpath(n_bus, 0.0), val(n_bus);
    for (size_t q = 1; q < order.size(); ++q) {
        const int u = order[q];
        zpath[u] = zpath[parent[u]] + cplx(net.bus_z[2 * u], net.bus_z[2 * u + 1]);
    }
    std::vector<char> mark(n_bus);
    for (int jc = 0; jc < n; ++jc) {
        std::fill(mark.begin(), mark.end(), 0);
        for (int u = net.pq[jc]; u != slack; u = parent[u]) mark[u] = 1;
        val[slack] = 0.0;
        for (size_t q = 1; q < order.size(); ++q) {
            const int u = order[q];
            val[u] = mark[u] ? zpath[u] : val[parent[u]];
        }
        for (int ic = 0; ic < n; ++ic) {
            const cplx k = -val[net.pq[ic]];
            net.K[((size_t)ic * n + jc) * 2] = k.real();
            net.K[((size_t)ic * n + jc) * 2 + 1] = k.imag();
        }
    }
}

}  // namespace tpf

namespace {

// The host-buffer solve: columns are independent, so it runs chunk by chunk on the device
// workspace (see the comment inside); solve(cols, S_dev, V_dev, iters_dev, mismatch_dev) solves one
// chunk on `stream` and leaves its statistics in h->stats.  v_in: V_host holds a start to copy in.
template <class Solve>
tpf_status host_chunks(tpf_handle *h, int64_t T, const void *S_host, void *V_host, int32_t *iters_host,
                       double *mismatch_host, const tpf_opts &o, void *stream, bool v_in, Solve solve) {
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    tpf::Workspace &w = h->ws;
    const size_t col_bytes = (size_t)h->net.n_pq * 16;
    if (T > w.host_cap) {
        cudaFree(w.S_dev); cudaFree(w.V_dev); cudaFree(w.it_dev); cudaFree(w.mm_dev);
        w.S_dev = w.V_dev = nullptr; w.it_dev = nullptr; w.mm_dev = nullptr; w.host_cap = 0;
        if (cudaMalloc(&w.S_dev, col_bytes * T) != cudaSuccess || cudaMalloc(&w.V_dev, col_bytes * T) != cudaSuccess ||
            cudaMalloc(&w.it_dev, sizeof(int32_t) * T) != cudaSuccess ||
            cudaMalloc(&w.mm_dev, sizeof(double) * T) != cudaSuccess) {
            cudaGetLastError();
            return TPF_ENOMEM;
        }
        w.host_cap = T;
    }
    // Columns are independent, so the solve runs chunk by chunk: every host-to-device copy is queued
    // at once on an input stream, each chunk's solve waits only for its own copy, and its results go
    // back on an output stream while the next chunk is solved (pinned host memory overlaps; pageable
    // memory still works, with the copies serialised by the driver).
    // The sparse solve is one short launch per chunk, so it takes finer chunks (less fill and drain
    // around the copies); the dense solve's per-sweep host loop prefers fewer.
    const int64_t max_chunks = o.method == TPF_METHOD_SPARSE ? 32 : 8;  // the learned start is sparse
    const int64_t n_chunks = T >= 65536 ? std::min<int64_t>(max_chunks, T / 16384) : 1;
    const int64_t chunk = tpf::round_up((T + n_chunks - 1) / n_chunks, tpf::kTileN);
    cudaStream_t sin = nullptr, sout = nullptr;
    std::vector<cudaEvent_t> ev;
    auto cleanup = [&]() {
        if (sout) cudaStreamSynchronize(sout);
        if (sin) cudaStreamSynchronize(sin);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
        if (sin) cudaStreamDestroy(sin);
        if (sout) cudaStreamDestroy(sout);
        cudaGetLastError();
    };
    if (cudaStreamCreateWithFlags(&sin, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sout, cudaStreamNonBlocking) != cudaSuccess) {
        cleanup();
        return TPF_ECUDA;
    }
    ev.assign(2 * n_chunks, nullptr);
    for (cudaEvent_t &e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cleanup();
            return TPF_ECUDA;
        }
    const char *Sh = static_cast<const char *>(S_host);
    char *Vh = static_cast<char *>(V_host);
    char *Sd = static_cast<char *>(w.S_dev), *Vd = static_cast<char *>(w.V_dev);
    for (int64_t c = 0; c < n_chunks; ++c) {
        const int64_t a = c * chunk, b = std::min(T, a + chunk);
        if (a >= b) break;
        if (cudaMemcpyAsync(Sd + a * col_bytes, Sh + a * col_bytes, (b - a) * col_bytes, cudaMemcpyHostToDevice, sin) !=
                cudaSuccess ||
            (v_in && cudaMemcpyAsync(Vd + a * col_bytes, Vh + a * col_bytes, (b - a) * col_bytes,
                                                           cudaMemcpyHostToDevice, sin) != cudaSuccess) ||
            cudaEventRecord(ev[2 * c], sin) != cudaSuccess) {
            cleanup();
            return TPF_ECUDA;
        }
    }
    tpf_stats total{};
    tpf_status result = TPF_OK;
    for (int64_t c = 0; c < n_chunks; ++c) {
        const int64_t a = c * chunk, b = std::min(T, a + chunk);
        if (a >= b) break;
        if (cudaStreamWaitEvent(s, ev[2 * c], 0) != cudaSuccess) {
            cleanup();
            return TPF_ECUDA;
        }
        tpf_status st = solve(b - a, Sd + a * col_bytes, Vd + a * col_bytes, iters_host ? w.it_dev + a : nullptr,
                              mismatch_host ? w.mm_dev + a : nullptr);
        if (st != TPF_OK && st != TPF_ENOCONV) {
            cleanup();
            return st;
        }
        if (st == TPF_ENOCONV) result = TPF_ENOCONV;
        const tpf_stats &p = h->stats;
        total.sweeps = std::max(total.sweeps, p.sweeps);
        total.precise_sweeps = std::max(total.precise_sweeps, p.precise_sweeps);
        total.converged += p.converged;
        total.columns += p.columns;
        total.kernel_launches += p.kernel_launches;
        total.gemm_ms += p.gemm_ms;
        total.residual_ms += p.residual_ms;
        total.other_ms += p.other_ms;
        total.gemm_launches += p.gemm_launches;
        total.gemm_columns += p.gemm_columns;
        if (cudaEventRecord(ev[2 * c + 1], s) != cudaSuccess || cudaStreamWaitEvent(sout, ev[2 * c + 1], 0) != cudaSuccess ||
            cudaMemcpyAsync(Vh + a * col_bytes, Vd + a * col_bytes, (b - a) * col_bytes, cudaMemcpyDeviceToHost, sout) !=
                cudaSuccess ||
            (iters_host && cudaMemcpyAsync(iters_host + a, w.it_dev + a, sizeof(int32_t) * (b - a),
                                           cudaMemcpyDeviceToHost, sout) != cudaSuccess) ||
            (mismatch_host && cudaMemcpyAsync(mismatch_host + a, w.mm_dev + a, sizeof(double) * (b - a),
                                              cudaMemcpyDeviceToHost, sout) != cudaSuccess)) {
            cleanup();
            return TPF_ECUDA;
        }
    }
    const bool ok = cudaStreamSynchronize(sout) == cudaSuccess;
    cleanup();
    h->stats = total;
    return ok ? result : TPF_ECUDA;
}

}  // namespace

extern "C" {

void tpf_default_opts(tpf_opts *o) {
    if (!o) return;
    o->tol = 1e-10;
    o->max_iter = 100;
    o->precision = TPF_PREC_MIXED;
    o->start = TPF_START_FLAT;
    o->switch_tol = 1e-4;
    o->profile = 0;
    o->method = TPF_METHOD_DENSE;
}

const char *tpf_strerror(tpf_status s) {
    switch (s) {
        case TPF_OK: return "TPF_OK";
        case TPF_EINVAL: return "TPF_EINVAL: invalid argument";
        case TPF_ESINGULAR: return "TPF_ESINGULAR: Y_dd is singular (a bus is not connected to the slack)";
        case TPF_ENOMEM: return "TPF_ENOMEM: allocation failed";
        case TPF_ECUDA: return "TPF_ECUDA: CUDA error";
        case TPF_ETIMEOUT: return "TPF_ETIMEOUT: a bounded device wait expired";
        case TPF_ENOCONV: return "TPF_ENOCONV: some columns did not converge";
        case TPF_EUNSUPPORTED: return "TPF_EUNSUPPORTED: not supported by this library or device";
    }
    return "TPF_UNKNOWN";
}

tpf_status tpf_precompute_host(int n_bus, int n_branch, const int32_t *from, const int32_t *to,
                               const double *z_pu, int slack, double v0_re, double v0_im, int n_pq,
                               const int32_t *pq_bus, double *K_out, double *W_out) {
    if (!K_out || !W_out) return TPF_EINVAL;
    tpf::Network net;
    tpf_status st;
    try {
        st = tpf::build_network(n_bus, n_branch, from, to, z_pu, slack, v0_re, v0_im, n_pq, pq_bus, net);
    } catch (const std::bad_alloc &) {
        return TPF_ENOMEM;
    }
    if (st != TPF_OK) return st;
    try {
        tpf::compute_dense(net);
    } catch (const std::bad_alloc &) {
        return TPF_ENOMEM;
    }
    std::memcpy(K_out, net.K.data(), net.K.size() * sizeof(double));
    std::memcpy(W_out, net.W.data(), net.W.size() * sizeof(double));
    return TPF_OK;
}

tpf_status tpf_create(int n_bus, int n_branch, const int32_t *from, const int32_t *to,
                      const double *z_pu, int slack, double v0_re, double v0_im, int n_pq,
                      const int32_t *pq_bus, tpf_handle **out) {
    if (!out) return TPF_EINVAL;
    *out = nullptr;
    tpf_handle *h = new (std::nothrow) tpf_handle();
    if (!h) return TPF_ENOMEM;
    tpf_status st;
    try {
        st = tpf::build_network(n_bus, n_branch, from, to, z_pu, slack, v0_re, v0_im, n_pq, pq_bus, h->net);
    } catch (const std::bad_alloc &) {
        st = TPF_ENOMEM;
    }
    if (st == TPF_OK) st = tpf::upload_network(h);
    if (st != TPF_OK) {
        tpf::free_device(h);
        delete h;
        return st;
    }
    *out = h;
    return TPF_OK;
}

tpf_status tpf_create_poly(int n_bus, int n_branch, int phases, const int32_t *from, const int32_t *to,
                           const double *z_pu, int slack, const double *v0, int n_pq, const int32_t *pq_bus,
                           tpf_handle **out) {
    if (!out) return TPF_EINVAL;
    *out = nullptr;
    if (phases == 1) {
        if (!v0) return TPF_EINVAL;
        return tpf_create(n_bus, n_branch, from, to, z_pu, slack, v0[0], v0[1], n_pq, pq_bus, out);
    }
    tpf_handle *h = new (std::nothrow) tpf_handle();
    if (!h) return TPF_ENOMEM;
    tpf_status st;
    try {
        st = tpf::build_network_poly(n_bus, n_branch, phases, from, to, z_pu, slack, v0, n_pq, pq_bus, h->net);
    } catch (const std::bad_alloc &) {
        st = TPF_ENOMEM;
    }
    if (st == TPF_OK) st = tpf::upload_network(h);
    if (st != TPF_OK) {
        tpf::free_device(h);
        delete h;
        return st;
    }
    *out = h;
    return TPF_OK;
}

void tpf_destroy(tpf_handle *h) {
    if (!h) return;
    tpf::DeviceScope dscope(h->device);
    tpf::free_device(h);
    delete h;
}

int tpf_n_pq(const tpf_handle *h) { return h ? h->net.n_pq : -1; }

tpf_status tpf_last_stats(const tpf_handle *h, tpf_stats *out) {
    if (!h || !out) return TPF_EINVAL;
    *out = h->stats;
    return TPF_OK;
}

static tpf_status check_opts(const tpf_opts *in, tpf_opts &o) {
    tpf_default_opts(&o);
    if (in) o = *in;
    if (!(o.tol >= 0.0) || o.max_iter < 1 || o.max_iter > 100000) return TPF_EINVAL;
    if (o.precision != TPF_PREC_FP64 && o.precision != TPF_PREC_MIXED) return TPF_EINVAL;
    if (o.start != TPF_START_FLAT && o.start != TPF_START_GIVEN && o.start != TPF_START_WARM) return TPF_EINVAL;
    if (!(o.switch_tol >= 0.0)) return TPF_EINVAL;
    if (o.method != TPF_METHOD_DENSE && o.method != TPF_METHOD_SPARSE) return TPF_EINVAL;
    return TPF_OK;
}

tpf_status tpf_solve(tpf_handle *h, int64_t T, const void *S_dev, void *V_dev, int32_t *iters_dev,
                     double *mismatch_dev, const tpf_opts *opts, void *stream) {
    if (!h || T < 0) return TPF_EINVAL;
    tpf_opts o;
    tpf_status st = check_opts(opts, o);
    if (st != TPF_OK) return st;
    h->stats = tpf_stats{};
    h->stats.columns = T;
    if (T == 0) return TPF_OK;
    if (!S_dev || !V_dev) return TPF_EINVAL;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (o.method == TPF_METHOD_SPARSE)
        return o.precision == TPF_PREC_FP64 ? tpf::solve_tree64(h, T, S_dev, V_dev, iters_dev, mismatch_dev, o, s)
                                            : tpf::solve_sparse(h, T, S_dev, V_dev, iters_dev, mismatch_dev, o, s);
    if (o.precision == TPF_PREC_FP64) return tpf::solve_fp64(h, T, S_dev, V_dev, iters_dev, mismatch_dev, o, s);
    return tpf::solve_mixed(h, T, S_dev, V_dev, iters_dev, mismatch_dev, o, s);
}

tpf_status tpf_batch_create(int F, tpf_handle *const *hs, const int64_t *T, const void *const *S_dev,
                            void *const *V_dev, int32_t *const *iters_dev, double *const *mismatch_dev,
                            const tpf_opts *opts, tpf_batch **out) {
    if (!out) return TPF_EINVAL;
    *out = nullptr;
    if (F < 1 || !hs || !T || !S_dev || !V_dev) return TPF_EINVAL;
    tpf_opts o;
    tpf_status st = check_opts(opts, o);
    if (st != TPF_OK) return st;
    for (int f = 0; f < F; ++f) {
        if (!hs[f] || T[f] < 0 || (T[f] > 0 && (!S_dev[f] || !V_dev[f]))) return TPF_EINVAL;
        if (hs[f]->device != hs[0]->device) return TPF_EINVAL;
        for (int g = 0; g < f; ++g)
            if (hs[g] == hs[f]) return TPF_EINVAL;
    }
    if (o.method != TPF_METHOD_SPARSE || o.precision != TPF_PREC_MIXED) return TPF_EUNSUPPORTED;
    for (int f = 0; f < F; ++f)  // (feeders past 4,096 buses take chunked launches with scratch)
        if (!hs[f]->dev.radial || hs[f]->dev.t_threads <= 0 || hs[f]->dev.t_bpt == tpf::kTreeBigBPT)
            return TPF_EUNSUPPORTED;
    tpf::DeviceScope dscope(hs[0]->device);
    if (!dscope.ok) return TPF_ECUDA;
    return tpf::batch_plan_create(F, hs, T, S_dev, V_dev, iters_dev, mismatch_dev, o, out);
}

tpf_status tpf_batch_launch(tpf_batch *b, void *stream) {
    if (!b) return TPF_EINVAL;
    tpf::DeviceScope dscope(tpf::batch_device(b));
    if (!dscope.ok) return TPF_ECUDA;
    return tpf::batch_plan_launch(b, reinterpret_cast<cudaStream_t>(stream));
}

tpf_status tpf_batch_wait(tpf_batch *b, int64_t *converged_out, tpf_stats *stats_out) {
    if (!b) return TPF_EINVAL;
    tpf::DeviceScope dscope(tpf::batch_device(b));
    if (!dscope.ok) return TPF_ECUDA;
    return tpf::batch_plan_wait(b, converged_out, stats_out);
}

void tpf_batch_destroy(tpf_batch *b) { tpf::batch_plan_destroy(b); }

tpf_status tpf_autotune(tpf_handle *h, int64_t T, const void *S_dev, const tpf_opts *opts, int *bpt_out,
                        void *stream) {
    if (!h || T <= 0 || !S_dev) return TPF_EINVAL;
    tpf_opts o;
    tpf_status st = check_opts(opts, o);
    if (st != TPF_OK) return st;
    if (o.precision != TPF_PREC_MIXED) return TPF_EUNSUPPORTED;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    st = tpf::autotune_sparse(h, T, S_dev, o, reinterpret_cast<cudaStream_t>(stream), bpt_out);
    h->stats = tpf_stats{};
    return st;
}

tpf_status tpf_set_zip(tpf_handle *h, const double *alpha) {
    if (!h) return TPF_EINVAL;
    if (alpha) {
        for (size_t k = 0; k < 3 * (size_t)h->net.n_pq; ++k)
            if (!std::isfinite(alpha[k])) return TPF_EINVAL;
    }
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    return tpf::set_zip(h, alpha);
}

tpf_status tpf_solve_ex(tpf_handle *h, int64_t T, const void *S_dev, void *V_dev, int32_t *iters_dev,
                        double *mismatch_dev, const tpf_outputs *out, const tpf_opts *opts, void *stream) {
    if (!out) return tpf_solve(h, T, S_dev, V_dev, iters_dev, mismatch_dev, opts, stream);
    if (!h || T < 0) return TPF_EINVAL;
    tpf_opts o;
    tpf_status st = check_opts(opts, o);
    if (st != TPF_OK) return st;
    if (o.method != TPF_METHOD_SPARSE) return TPF_EUNSUPPORTED;
    if (!(out->v_min <= out->v_max)) return TPF_EINVAL;
    h->stats = tpf_stats{};
    h->stats.columns = T;
    if (T == 0) return TPF_OK;
    if (!S_dev || (!V_dev && o.start != TPF_START_FLAT)) return TPF_EINVAL;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    return tpf::solve_sparse_ex(h, T, S_dev, V_dev, iters_dev, mismatch_dev, out, o,
                                reinterpret_cast<cudaStream_t>(stream));
}

tpf_status tpf_solve_batch(int F, tpf_handle *const *hs, const int64_t *T, const void *const *S_dev,
                           void *const *V_dev, int32_t *const *iters_dev, double *const *mismatch_dev,
                           const tpf_opts *opts, int64_t *converged_out, tpf_stats *stats_out, void *stream) {
    if (F < 0 || (F > 0 && (!hs || !T || !S_dev || !V_dev))) return TPF_EINVAL;
    tpf_opts o;
    tpf_status st = check_opts(opts, o);
    if (st != TPF_OK) return st;
    if (stats_out) *stats_out = tpf_stats{};
    if (F == 0) return TPF_OK;
    for (int f = 0; f < F; ++f) {
        if (!hs[f] || T[f] < 0 || (T[f] > 0 && (!S_dev[f] || !V_dev[f]))) return TPF_EINVAL;
        if (hs[f]->device != hs[0]->device) return TPF_EINVAL;
        for (int g = 0; g < f; ++g)
            if (hs[g] == hs[f]) return TPF_EINVAL;  // each handle's workspaces serve one feeder
    }
    tpf::DeviceScope dscope(hs[0]->device);
    if (!dscope.ok) return TPF_ECUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Radial feeders under the sparse method share launches; the rest are solved one by one.
    std::vector<int> grouped, single;
    for (int f = 0; f < F; ++f) {
        const bool fits = o.method == TPF_METHOD_SPARSE && o.precision == TPF_PREC_MIXED && hs[f]->dev.radial &&
                          hs[f]->dev.t_threads > 0 && hs[f]->dev.t_bpt != tpf::kTreeBigBPT;
        (fits ? grouped : single).push_back(f);
    }
    tpf_stats tot{};
    bool all = true;
    if (!grouped.empty()) {
        const int G = (int)grouped.size();
        std::vector<tpf_handle *> gh(G);
        std::vector<int64_t> gT(G), gconv(G);
        std::vector<const void *> gS(G);
        std::vector<void *> gV(G);
        std::vector<int32_t *> gi(G);
        std::vector<double *> gm(G);
        for (int k = 0; k < G; ++k) {
            const int f = grouped[k];
            gh[k] = hs[f];
            gT[k] = T[f];
            gS[k] = S_dev[f];
            gV[k] = V_dev[f];
            gi[k] = iters_dev ? iters_dev[f] : nullptr;
            gm[k] = mismatch_dev ? mismatch_dev[f] : nullptr;
        }
        st = tpf::solve_batch_sparse(G, gh.data(), gT.data(), gS.data(), gV.data(), gi.data(), gm.data(), o,
                                     gconv.data(), &tot, s);
        if (st != TPF_OK && st != TPF_ENOCONV) return st;
        all = st == TPF_OK;
        for (int k = 0; k < G; ++k)
            if (converged_out) converged_out[grouped[k]] = gconv[k];
    }
    for (int f : single) {
        // Large radial feeders keep the sparse method (its chunked large-feeder kernel), as do
        // FP64 solves of the radial single-phase feeders the FP64 sparse kernel takes; feeders the
        // sparse kernels cannot take use the dense form.
        tpf_opts of = o;
        const tpf::DeviceNet &df = hs[f]->dev;
        const bool sparse_ok = o.method == TPF_METHOD_SPARSE && df.radial && df.t_threads > 0 &&
                               (o.precision == TPF_PREC_MIXED ||
                                (df.phases == 1 && df.t_bpt != tpf::kTreeBigBPT &&
                                 tpf::tree64_smem(df.t_threads, df.t_bpt) <= 227 * 1024));
        if (!sparse_ok) of.method = TPF_METHOD_DENSE;
        st = tpf_solve(hs[f], T[f], S_dev[f], V_dev[f], iters_dev ? iters_dev[f] : nullptr,
                       mismatch_dev ? mismatch_dev[f] : nullptr, &of, stream);
        if (st != TPF_OK && st != TPF_ENOCONV) return st;
        all = all && st == TPF_OK;
        const tpf_stats &fs = hs[f]->stats;
        if (converged_out) converged_out[f] = fs.converged;
        tot.converged += fs.converged;
        tot.columns += fs.columns;
        tot.sweeps = std::max(tot.sweeps, fs.sweeps);
        tot.kernel_launches += fs.kernel_launches;
        tot.gemm_ms += fs.gemm_ms;
        tot.residual_ms += fs.residual_ms;
        tot.other_ms += fs.other_ms;
    }
    if (stats_out) *stats_out = tot;
    return all ? TPF_OK : TPF_ENOCONV;
}

tpf_status tpf_solve_host(tpf_handle *h, int64_t T, const void *S_host, void *V_host,
                          int32_t *iters_host, double *mismatch_host, const tpf_opts *opts,
                          void *stream) {
    if (!h || T < 0) return TPF_EINVAL;
    tpf_opts o;
    tpf_status st = check_opts(opts, o);
    if (st != TPF_OK) return st;
    if (T == 0) {
        h->stats = tpf_stats{};
        return TPF_OK;
    }
    if (!S_host || !V_host) return TPF_EINVAL;
    tpf::DeviceScope dscope(h->device);
    if (!dscope.ok) return TPF_ECUDA;
    return host_chunks(h, T, S_host, V_host, iters_host, mismatch_host, o, stream, o.start != TPF_START_FLAT,
                       [&](int64_t cols, void *Sd, void *Vd, int32_t *itd, double *mmd) {
                           return tpf_solve(h, cols, Sd, Vd, itd, mmd, &o, stream);
                       });
}

tpf_status tpf_solve_learned_host(tpf_handle *hd, tpf_mlp *net, int64_t T, const void *S_host, void *V_host,
                                  int32_t *iters_host, double *mismatch_host, const tpf_opts *opts,
                                  int64_t *fallback_out, void *stream) {
    if (fallback_out) *fallback_out = 0;
    if (!hd || !net || T < 0) return TPF_EINVAL;
    tpf_opts o;
    tpf_status st = check_opts(opts, o);
    if (st != TPF_OK) return st;
    if (o.method != TPF_METHOD_SPARSE || o.precision != TPF_PREC_MIXED) return TPF_EUNSUPPORTED;
    if (T == 0) {
        hd->stats = tpf_stats{};
        return TPF_OK;
    }
    if (!S_host || !V_host) return TPF_EINVAL;
    tpf::DeviceScope dscope(hd->device);
    if (!dscope.ok) return TPF_ECUDA;
    int64_t fallback = 0;
    st = host_chunks(hd, T, S_host, V_host, iters_host, mismatch_host, o, stream, false,
                     [&](int64_t cols, void *Sd, void *Vd, int32_t *itd, double *mmd) {
                         int64_t fb = 0;
                         const tpf_status r = tpf_solve_learned(hd, net, cols, Sd, Vd, itd, mmd, &o, &fb, stream);
                         fallback += fb;
                         return r;
                     });
    if (fallback_out) *fallback_out = fallback;
    return st;
}

tpf_status tpf_selftest_gemm(int M, int N, int K, const void *A_re, const void *A_im, const void *B_re,
                             const void *B_im, float *D_re, float *D_im, void *stream) {
    if (M <= 0 || N <= 0 || K <= 0 || M % tpf::kTileM || N % tpf::kTileN || K % tpf::kChunkK) return TPF_EINVAL;
    if (!A_re || !A_im || !B_re || !B_im || !D_re || !D_im) return TPF_EINVAL;
    return tpf::selftest_gemm(M, N, K, A_re, A_im, B_re, B_im, D_re, D_im, reinterpret_cast<cudaStream_t>(stream));
}

tpf_status tpf_selftest_gemm_wait(int M, int N, int K, const void *A_re, const void *A_im, const void *B_re,
                                  const void *B_im, float *D_re, float *D_im, double wait_s, int withhold_loads,
                                  void *stream) {
    if (M <= 0 || N <= 0 || K <= 0 || M % tpf::kTileM || N % tpf::kTileN || K % tpf::kChunkK) return TPF_EINVAL;
    if (!A_re || !A_im || !B_re || !B_im || !D_re || !D_im) return TPF_EINVAL;
    if (!(wait_s >= 1e-6 && wait_s <= 10.0)) return TPF_EINVAL;
    return tpf::selftest_gemm(M, N, K, A_re, A_im, B_re, B_im, D_re, D_im, reinterpret_cast<cudaStream_t>(stream),
                              (uint64_t)(wait_s * 1e9), withhold_loads ? 1 : 0);
}

}  // extern "C"
