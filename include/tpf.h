/*
 * tpf.h -- C ABI of the GB300 tensor power flow library (libtpf.so).
 *
 * The library solves many power flows of one distribution feeder at once with the fixed-point
 * iteration of the paper, in its dense form (Sec. II Eq. 2-3, Sec. IV-A Eq. 12, Algorithm 1) or,
 * on radial feeders, its sparse form (Sec. IV-B Eq. 13-14, Algorithm 2; TPF_METHOD_SPARSE):
 *
 *     V_{k+1} = K conj(S ./ V_k) + W,      K = -Y_dd^{-1},   W = K Y_ds v_s,
 *
 * applied to every column (time step x scenario) of the load tensor S.  S is the *load*
 * (consumption positive), so the current drawn at a demand bus is conj(S_i / V_i) (Eq. 1).
 *
 * Data layout.  A load tensor holds T power flows; column t is the contiguous row
 * S[t*n_pq .. (t+1)*n_pq) of complex128 values (real, imaginary interleaved), i.e. the reshaped
 * S-dot of Eq. 12 stored with the bus index fastest.  V, iteration counts and mismatches use the
 * same column order.  Bus order inside a column is the order of pq_bus given to tpf_create.
 *
 * Ownership.  A tpf_handle owns K, W, the network arrays and all device workspaces.  The caller
 * owns every tensor passed to a solve; the library never frees or keeps caller pointers after
 * the call returns.
 *
 * Errors.  Every entry point returns a tpf_status.  Argument errors are detected on the host
 * before any device work.  Device-side failures (a bounded wait that expired, a CUDA error) are
 * reported by the solve that met them.  tpf_strerror() names a status.
 *
 * Threads and streams.  A handle may be used by one host thread at a time.  All device work of a
 * solve is issued on the stream passed to it (a cudaStream_t, passed as void*; NULL = legacy
 * default stream), and the solve returns only after that work has finished.
 */
#ifndef TPF_H
#define TPF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tpf_handle tpf_handle;
typedef struct tpf_batch tpf_batch;   /* a prepared batch of feeders (tpf_batch_create) */

typedef enum {
    TPF_OK = 0,
    TPF_EINVAL = 1,       /* a bad argument (sizes, indices, NULL pointers, options)            */
    TPF_ESINGULAR = 2,    /* Y_dd is singular: a bus is not connected to the slack              */
    TPF_ENOMEM = 3,       /* a host or device allocation failed                                 */
    TPF_ECUDA = 4,        /* a CUDA runtime or driver call failed (including "no device")       */
    TPF_ETIMEOUT = 5,     /* a bounded device-side wait expired; outputs are not valid          */
    TPF_ENOCONV = 6,      /* at least one column did not converge; all outputs are valid       */
    TPF_EUNSUPPORTED = 7  /* the request is valid but this library or device cannot serve it   */
} tpf_status;

/* Arithmetic of a solve. */
enum {
    TPF_PREC_FP64 = 0,  /* the plain double-precision fixed-point iteration (direct form)          */
    TPF_PREC_MIXED = 1  /* fp16 tensor-core sweeps with FP32 accumulation in residual form         *
                         * V <- V + K rho(V); V is carried as two floats and rho is evaluated    *
                         * against a double-float anchor, so results reach FP64-level accuracy  */
};

/* Starting point of a solve. */
enum {
    TPF_START_FLAT = 0,  /* V_0 = 1 + j0 at every bus (Algorithm 1)                             */
    TPF_START_GIVEN = 1, /* V_0 is read from the V buffer passed to the solve.  Mixed precision:   *
                          * every column is anchored at V_0 at once, which suits a V_0 that is    *
                          * already close to the solution (a restart, a converged neighbour)     */
    TPF_START_WARM = 2   /* V_0 is read from the V buffer as an approximate start (a learned      *
                          * prediction, a neighbouring time step).  Mixed precision: the FP32     *
                          * sweeps start from fl32(V_0) and a column is anchored once its step is *
                          * small, as from the flat start.  FP64: the same as TPF_START_GIVEN     */
};

typedef struct {
    double tol;       /* per-column stop: max_i |V_{k+1,i} - V_{k,i}| <= tol (pu).  Default 1e-10 */
    int max_iter;     /* cap on sweeps per column (Algorithm 1's "iterations").  Default 100     */
    int precision;    /* TPF_PREC_*.  Default TPF_PREC_MIXED                                      */
    int start;        /* TPF_START_*.  Default TPF_START_FLAT                                     */
    double switch_tol;/* mixed only: once a column's step falls below this (pu), or is predicted  *
                       * to fall below 3e-6 pu in the next sweep, its V is frozen as the anchor   *
                       * V_ref, rho(V_ref) is evaluated once in double-float, and later sweeps    *
                       * add FP32 corrections in V - V_ref.  Default 1e-4                         */
    int profile;      /* nonzero: time every kernel of the solve with CUDA events on its stream  *
                       * and report the totals in tpf_stats.  Default 0                           */
    int method;       /* TPF_METHOD_*.  Default TPF_METHOD_DENSE                                   */
} tpf_opts;

/* Formulation of a solve (both give the same iterates in exact arithmetic). */
enum {
    TPF_METHOD_DENSE = 0,  /* Algorithm 1 / Eq. 12: the dense product with K = -Y_dd^{-1}.  Mixed  *
                            * precision up to 2,048 demand unknowns; FP64 any size                   */
    TPF_METHOD_SPARSE = 1  /* Algorithm 2 / Eq. 13-14: a sparse solve with Y_dd each sweep, here the  *
                            * fill-in-free tree substitution of a radial feeder, O(n) per column and  *
                            * sweep, the whole sweep loop of a column on chip.  TPF_PREC_MIXED: radial *
                            * networks of up to 6,144 demand unknowns (past 4,096 in chunks of 8,192  *
                            * columns with device scratch).  TPF_PREC_FP64: the same substitution in  *
                            * plain double precision, single-phase radial networks of up to 4,096    *
                            * demand buses (constant power or ZIP).  TPF_EUNSUPPORTED otherwise      */
};

/* Per-solve counters (filled by tpf_last_stats after a solve). */
typedef struct {
    int sweeps;           /* sweeps launched (the largest per-column count)                    */
    int precise_sweeps;   /* mixed: sweeps in which at least one column was anchored            */
    int64_t converged;    /* columns that met tol                                               */
    int64_t columns;      /* T of the last solve                                                */
    int64_t kernel_launches; /* kernels of this library launched by the last solve              */
    /* Filled only when opts.profile was set (milliseconds of device time, CUDA events):        */
    double gemm_ms;          /* the dense sweep kernel: tensor-core GEMM (mixed) or FP64 sweep   */
    double residual_ms;      /* mixed: the per-sweep residual / decision kernel; FP64: decision  */
    double other_ms;         /* packing, initialisation and the output / mismatch kernel         */
    int64_t gemm_launches;   /* launches of the dense sweep kernel                               */
    int64_t gemm_columns;    /* sum over those launches of the columns still iterating           */
} tpf_stats;

/* Fill *opts with the defaults listed in tpf_opts. */
void tpf_default_opts(tpf_opts *opts);

/* Name of a status (static string, never NULL). */
const char *tpf_strerror(tpf_status status);

/*
 * Build a feeder: Eq. 1's admittance matrix from the branch list, then K = -Y_dd^{-1} and
 * W = K Y_ds v_s (Eq. 3 with constant power, Algorithm 1's Z_B and W), on the host in double
 * precision, and upload them with the network arrays to the current CUDA device.
 *
 *   n_bus, n_branch    number of buses (>= 2) and of branches (>= n_bus - 1)
 *   from, to           [n_branch] bus indices in [0, n_bus) of each branch's ends
 *   z_pu               [2*n_branch] series impedance r + jx of each branch in pu, interleaved;
 *                      no shunts.  |z| must be > 0.
 *   slack              index of the slack bus;  v0_re + j v0_im its voltage (pu)
 *   n_pq, pq_bus       the demand buses, [n_pq] distinct indices, every bus but the slack
 *                      (n_pq = n_bus - 1); their order is the bus order of every tensor.
 *   out                receives the new handle (set to NULL on failure)
 *
 * A radial network (a tree rooted at the slack) gets K from the path sums of its branch
 * impedances; any other connected network from a dense LU inverse of Y_dd.  Returns TPF_EINVAL
 * for bad indices or sizes, TPF_ESINGULAR if some bus is not connected to the slack, TPF_ECUDA
 * if no device can be used.  All arrays are host memory, read during the call only.
 */
tpf_status tpf_create(int n_bus, int n_branch, const int32_t *from, const int32_t *to,
                      const double *z_pu, int slack, double v0_re, double v0_im, int n_pq,
                      const int32_t *pq_bus, tpf_handle **out);

/* Release a handle and every device buffer it owns (NULL is a no-op). */
/*
 * Build a polyphase feeder (Eq. 1 with phases > 1): every bus has `phases` nodes; branch e joins
 * from[e] and to[e] through the phases x phases series impedance block z_pu[e] (pu, row-major,
 * interleaved complex: z_pu[2*((e*phases + p)*phases + q)] + j z_pu[... + 1]; self impedances on
 * the diagonal, mutual impedances off it; each block must be invertible); the slack bus holds
 * v0[p] (interleaved complex, [phases]).  The unknowns are the phases x n_pq demand-node voltages,
 * ordered bus-major: unknown i*phases + p is phase p of demand bus pq_bus[i], so load and voltage
 * tensors are [T][n_pq][phases] (tpf_n_pq returns n_pq * phases).  Loads are wye-connected: the
 * current drawn at a node is conj(S / V) of that node.  Served by TPF_PREC_FP64 (any connected
 * network, K = -Y_dd^{-1} by LU) and, for radial networks with phases == 3, TPF_METHOD_SPARSE
 * (the tree substitution with phases x phases branch blocks); the dense mixed path and ZIP
 * coefficients return TPF_EUNSUPPORTED.  phases == 1 is tpf_create.  Errors as tpf_create, and
 * TPF_EINVAL for phases outside 1..3 or a singular branch block.
 */
tpf_status tpf_create_poly(int n_bus, int n_branch, int phases, const int32_t *from, const int32_t *to,
                           const double *z_pu, int slack, const double *v0, int n_pq, const int32_t *pq_bus,
                           tpf_handle **out);

void tpf_destroy(tpf_handle *h);

/* Number of demand buses of a handle (the column length of every tensor). */
int tpf_n_pq(const tpf_handle *h);

/*
 * Host-only precomputation (no device needed): the same K (= -Y_dd^{-1}) and W (= K Y_ds v_s) that
 * tpf_create uploads, written to caller host buffers K_out [2*n_pq*n_pq] (row-major complex,
 * interleaved) and W_out [2*n_pq].  Arguments and errors as tpf_create.
 */
tpf_status tpf_precompute_host(int n_bus, int n_branch, const int32_t *from, const int32_t *to,
                               const double *z_pu, int slack, double v0_re, double v0_im,
                               int n_pq, const int32_t *pq_bus, double *K_out, double *W_out);

/*
 * Solve T power flows (Algorithm 1, one column per power flow, each column stopping on its own):
 *
 *   S_dev        device, complex128 [T][n_pq], the loads (read only)
 *   V_dev        device, complex128 [T][n_pq], receives V.  Read first as V_0 when
 *                opts->start is TPF_START_GIVEN or TPF_START_WARM.
 *   iters_dev    device, int32 [T], receives the sweeps applied to each column, or -max_iter
 *                for a column that never met tol (NULL: not written)
 *   mismatch_dev device, float64 [T], receives max_i |V_i conj((Y v)_i) + S_i| in pu, the power
 *                balance of Eq. 1 at the returned V (NULL: not written)
 *   opts         NULL for defaults
 *   stream       cudaStream_t for all device work
 *
 * T = 0 is a valid empty solve.  Returns TPF_OK when every column met tol, TPF_ENOCONV when some
 * did not (outputs still valid), TPF_ETIMEOUT or TPF_ECUDA on device failures.  Device buffers
 * must not overlap.  The call blocks until the stream has finished the solve.
 */
tpf_status tpf_solve(tpf_handle *h, int64_t T, const void *S_dev, void *V_dev, int32_t *iters_dev,
                     double *mismatch_dev, const tpf_opts *opts, void *stream);

/*
 * tpf_solve with HOST buffers (same shapes and meaning): copies S (and V_0) to the device, solves,
 * and copies V, iteration counts and mismatches back, all on `stream`.  Device staging buffers
 * are owned by the handle and grow to the largest T seen.  Host buffers may be pageable or
 * pinned; pinned memory is faster.  iters_host and mismatch_host may be NULL.
 */
tpf_status tpf_solve_host(tpf_handle *h, int64_t T, const void *S_host, void *V_host,
                          int32_t *iters_host, double *mismatch_host, const tpf_opts *opts,
                          void *stream);

/* Counters of the last solve on this handle. */
tpf_status tpf_last_stats(const tpf_handle *h, tpf_stats *out);

/*
 * Autotune the sparse formulation's launch shape for this feeder: time the kernel with 2, 4 and 8
 * demand buses per thread (the block sizes that follow from them) on the T columns of S_dev
 * (device, complex128 [T][n_pq], a representative sample such as the first few thousand columns
 * of a workload), flat start and opts' tolerances, and keep the fastest for every later sparse
 * solve.  bpt_out (host, may be NULL) receives the choice.  Allocates a scratch V of T columns.
 * TPF_EUNSUPPORTED for networks the sparse formulation does not take or opts->precision FP64.
 */
tpf_status tpf_autotune(tpf_handle *h, int64_t T, const void *S_dev, const tpf_opts *opts, int *bpt_out,
                        void *stream);

/*
 * ZIP loads (Eq. 3).  alpha is host memory [3][n_pq]: alpha_P, alpha_I and alpha_Z of every demand
 * bus (bus order of tpf_create), applied to every later solve on this handle:
 *
 *     i_d = alpha_P conj(S ./ V) + alpha_I conj(S) + alpha_Z conj(S) .* V
 *
 * (constant power, constant current and constant impedance parts of each bus's load S).  The
 * solves keep the shared K = -Y_dd^{-1} and evaluate i_d from the current iterate,
 * V <- K i_d(V) + W; Eq. 3's per-operating-point F = -B^{-1} A and w = -B^{-1} c have the same
 * fixed point, but B depends on each column's S when alpha_Z != 0, so a tensor of columns cannot
 * share them.  alpha == NULL returns the handle to constant power.  Served by TPF_METHOD_SPARSE and
 * TPF_PREC_FP64; the dense mixed path returns TPF_EUNSUPPORTED while ZIP coefficients are set.
 * On the sparse path the coefficients take a fourth shared-memory region; a feeder with 3,073 to
 * 4,096 demand buses, which would need more than 227 KB per block at 8 buses per thread, is laid
 * out at 16 buses per thread while coefficients are set (its kernel keeps them in device scratch)
 * and goes back to the default layout when they are dropped; its FP64 sparse solves then return
 * TPF_EUNSUPPORTED (TPF_METHOD_DENSE serves them).  TPF_EINVAL for non-finite coefficients.
 */
tpf_status tpf_set_zip(tpf_handle *h, const double *alpha);

/*
 * Scenario / time tensors (Sec. IV: the load tensor may have any number of scenario and time
 * dimensions; its columns are flattened in C order, bus fastest) with per-column and per-bus
 * statistics of the kind probabilistic and time-series studies report, computed in the solve's
 * own final pass.  Every pointer is a device pointer and may be NULL (not written).
 */
typedef struct {
    int s_complex64;    /* S is complex64 [T][n_pq] (else complex128)                           */
    int v_complex64;    /* V is complex64 [T][n_pq] (else complex128); V_dev may be NULL when    *
                         * opts->start is TPF_START_FLAT (statistics only)                       */
    double v_min, v_max;          /* voltage band in pu for the counts below                     */
    float *col_vmin, *col_vmax;   /* [T]: min and max |V_i| of each column                       */
    int32_t *col_viol;            /* [T]: buses of each column with |V_i| outside [v_min, v_max] */
    int32_t *bus_under, *bus_over;/* [n_pq]: ADDED TO: columns with |V_i| < v_min (> v_max);     *
                                   * the caller zeroes them before the first call                */
} tpf_outputs;

/*
 * tpf_solve with the outputs above.  Sparse formulation only (opts->method TPF_METHOD_SPARSE,
 * TPF_PREC_MIXED, radial network; TPF_EUNSUPPORTED otherwise).  out == NULL is tpf_solve.
 */
tpf_status tpf_solve_ex(tpf_handle *h, int64_t T, const void *S_dev, void *V_dev, int32_t *iters_dev,
                        double *mismatch_dev, const tpf_outputs *out, const tpf_opts *opts,
                        void *stream);

/*
 * Solve F feeders at once (many networks of different sizes, Sec. V): feeder f has handle hs[f],
 * T[f] columns, device tensors S[f] and V[f] (complex128 [T[f]][n_pq of hs[f]], V read as V_0
 * when opts->start is TPF_START_GIVEN or TPF_START_WARM), and optional iters[f] / mismatch[f] (the arrays iters and
 * mismatch may be NULL, as may their entries).  Radial feeders under TPF_METHOD_SPARSE with
 * TPF_PREC_MIXED share one launch per launch shape (feeders grouped by the block size the sparse
 * kernel uses for them), each block finding its feeder in a device table; any other feeder is
 * solved on its own with tpf_solve: radial feeders past 4,096 demand buses with the sparse method
 * (chunked launches), the rest with TPF_METHOD_DENSE.  converged_out (host, F entries, may be NULL) receives each
 * feeder's converged-column count; stats_out (host, may be NULL) the totals.  Handles must be on
 * the current device and distinct.  Returns TPF_OK when every column of every feeder met tol,
 * TPF_ENOCONV when some did not.  Blocks until the stream has finished.
 */
tpf_status tpf_solve_batch(int F, tpf_handle *const *hs, const int64_t *T, const void *const *S_dev,
                           void *const *V_dev, int32_t *const *iters_dev, double *const *mismatch_dev,
                           const tpf_opts *opts, int64_t *converged_out, tpf_stats *stats_out,
                           void *stream);

/*
 * A prepared batch (Sec. V, one submission for many feeders): the arguments of tpf_solve_batch,
 * fixed once, with every feeder radial with at most 4,096 demand unknowns,
 * opts->method == TPF_METHOD_SPARSE and opts->precision == TPF_PREC_MIXED (else TPF_EUNSUPPORTED).  tpf_batch_create uploads the work
 * table and captures one solve of all feeders (counter reset, one kernel per launch shape, copy of
 * the counts to pinned host memory) as a CUDA graph; tpf_batch_launch replays it on `stream` with
 * one graph launch and returns at once; tpf_batch_wait blocks until that replay has finished and
 * fills converged_out (F entries, may be NULL) and stats_out (may be NULL), returning TPF_OK when
 * every column met tol, TPF_ENOCONV otherwise, TPF_EINVAL when nothing was launched.
 * Each replay reads the current contents of S (and V for a given or warm start) and writes V,
 * iters and mismatch, so new loads are solved by rewriting S in place and launching again.  The
 * handles and all tensors must outlive the batch.  A feeder whose layout changed since creation
 * (tpf_autotune, tpf_set_zip) makes tpf_batch_launch return TPF_EINVAL.  A second launch waits
 * for the first to finish.  tpf_batch_destroy(NULL) is a no-op.
 */
tpf_status tpf_batch_create(int F, tpf_handle *const *hs, const int64_t *T, const void *const *S_dev,
                            void *const *V_dev, int32_t *const *iters_dev, double *const *mismatch_dev,
                            const tpf_opts *opts, tpf_batch **out);
tpf_status tpf_batch_launch(tpf_batch *b, void *stream);
tpf_status tpf_batch_wait(tpf_batch *b, int64_t *converged_out, tpf_stats *stats_out);
void tpf_batch_destroy(tpf_batch *b);

/*
 * Learned warm start.  The paper starts Algorithm 1 from the flat profile V_0 = 1; these entry
 * points train and run a small multilayer perceptron that predicts V_0 from a column's loads, so
 * that a solve started from it (TPF_START_WARM) needs fewer sweeps.  The iteration still decides
 * the result: it converges to the same high-voltage solution from any start (Sec. III).
 *
 * Network: inputs P_1..P_n, Q_1..Q_n (real and imaginary parts of a column of S), z-scored per
 * feature; n_hidden_layers hidden layers of `hidden` units with the erf GELU; linear outputs
 * Re V_i - 1, Im V_i, z-scored.  Loss: mean squared error.  Optimiser: Adam (beta 0.9, 0.999,
 * eps 1e-8).  Every product runs on the tensor cores in BF16 with FP32 accumulation; weights are
 * kept in FP32 (Xavier-uniform initialisation from `seed`, zero biases).  Buffers are sized for
 * batches of up to max_batch columns (a positive multiple of 128).
 */
typedef struct tpf_mlp tpf_mlp;

tpf_status tpf_mlp_create(int n_pq, int hidden, int n_hidden_layers, int max_batch, uint64_t seed,
                          tpf_mlp **out);
void tpf_mlp_destroy(tpf_mlp *h);
/* Number of parameters: per layer W (out x in) then b (out). */
int64_t tpf_mlp_param_count(const tpf_mlp *h);
/* Parameters as one flat FP32 host array in the order above (get: copy out; set: copy in). */
tpf_status tpf_mlp_get_params(tpf_mlp *h, float *host);
tpf_status tpf_mlp_set_params(tpf_mlp *h, const float *host);
/* Per-feature and per-target mean and standard deviation over T training columns
 * (S_dev, V_dev: device complex128 [T][n_pq], V the solved voltages).  Must precede training. */
tpf_status tpf_mlp_fit_normalization(tpf_mlp *h, int64_t T, const void *S_dev, const void *V_dev,
                                     void *stream);
/* The fitted statistics, 2 n_pq floats each (host). */
tpf_status tpf_mlp_get_normalization(tpf_mlp *h, float *in_mean, float *in_std, float *out_mean,
                                     float *out_std);
/* One Adam step on a batch of B columns (B a multiple of 128, <= max_batch): S_dev and V_dev are
 * device complex128 [B][n_pq].  loss_out (host, may be NULL) receives the batch loss before the
 * step; with loss_out the call waits for the stream, otherwise it only enqueues work. */
tpf_status tpf_mlp_train_step(tpf_mlp *h, int B, const void *S_dev, const void *V_dev, double lr,
                              double *loss_out, void *stream);
/* Loss and gradients of the current parameters on a batch (no update); grads_host (may be NULL)
 * receives them in the parameter order.  Blocks. */
tpf_status tpf_mlp_gradients(tpf_mlp *h, int B, const void *S_dev, const void *V_dev,
                             double *loss_out, float *grads_host, void *stream);
/* Predicted V_0 for T columns (device complex128 [T][n_pq] in and out; S_dev 16-byte aligned).
 * A column whose predicted |V_i| leaves [0.7, 1.1] at any bus gets the flat start; fallback_out
 * (host, may be NULL) receives how many.  Blocks. */
tpf_status tpf_mlp_predict(tpf_mlp *h, int64_t T, const void *S_dev, void *V0_dev,
                           int64_t *fallback_out, void *stream);

/*
 * Learned-start solve: the network predicts V_0 for every column (the fused inference of all its
 * layers, one tcgen05 kernel per chunk of columns that reads S itself, V_0 kept as half-precision
 * deviations from the flat start, Re V - 1 and Im V), then the sparse mixed solve runs from it
 * (TPF_START_WARM: FP32 sweeps from the prediction, anchoring once the step is small).  A column
 * whose prediction leaves |V| in [0.7, 1.1] at any bus starts flat; fallback_out (host, may be
 * NULL) receives how many did.  The iteration decides the result, so the outputs are those of
 * tpf_solve (Sec. III: the fixed point is reached from any nearby start).
 *
 *   hd, net      a feeder and a network for it (same n_pq, same device); the network's hidden
 *                width must be 128 or 256 with at most 7 hidden layers (TPF_EUNSUPPORTED otherwise)
 *   S_dev ... stream   as tpf_solve; opts->method must be TPF_METHOD_SPARSE and opts->precision
 *                TPF_PREC_MIXED (TPF_EUNSUPPORTED otherwise); opts->start is ignored
 *
 * The columns go in equal chunks of at most 1,048,576; the network keeps a buffer for the
 * predictions of one chunk (4 bytes per bus and column: 2.1 GB for a one-minute year at 1,000
 * buses).  S_dev must be 16-byte aligned (TPF_EINVAL otherwise).  tpf_last_stats(hd) reports the
 * totals over the chunks.
 * Blocks until done.
 */
tpf_status tpf_solve_learned(tpf_handle *hd, tpf_mlp *net, int64_t T, const void *S_dev, void *V_dev,
                             int32_t *iters_dev, double *mismatch_dev, const tpf_opts *opts, int64_t *fallback_out,
                             void *stream);

/*
 * The learned-start solve from HOST buffers (the host-buffer counterpart of tpf_solve_learned, as
 * tpf_solve_host is of tpf_solve): S_host [T][n_pq] complex128 in, V_host [T][n_pq] complex128,
 * iters_host [T] and mismatch_host [T] (both may be NULL) out.  The columns go through the
 * handle's device workspace in up to 32 chunks: every host-to-device copy is queued at once, each
 * chunk's prediction and solve wait only for its own copy, and its results go back while the next
 * chunk is solved (pinned host memory overlaps copies and compute; pageable memory works, with the
 * copies serialised).  fallback_out (host, may be NULL) receives the columns that started flat.
 * opts as tpf_solve_learned; errors as tpf_solve_learned, plus TPF_ENOMEM when the workspace
 * (2 x 16 n_pq + 12 bytes per column) cannot be allocated.  Blocks until done.
 */
tpf_status tpf_solve_learned_host(tpf_handle *hd, tpf_mlp *net, int64_t T, const void *S_host, void *V_host,
                                  int32_t *iters_host, double *mismatch_host, const tpf_opts *opts,
                                  int64_t *fallback_out, void *stream);

/*
 * Allocation-free FP64 solve.  The paper has no counterpart to this entry point; it exists for
 * callers that must not allocate device memory themselves or have the library do it: runtimes
 * that hand out device memory only from their own pool (raw cudaMalloc/cudaFree would escape
 * their accounting), and latency-bound loops where cudaMalloc/cudaFree may synchronise the device
 * or block for an unbounded time.  It runs the same FP64 kernels as tpf_solve with
 * TPF_PREC_FP64 (Algorithm 1 in direct form, per-column stopping) but needs no handle: the
 * caller passes K and W on the device, and the solve's scratch (the second V buffer and the
 * per-column state) lives in a fixed array compiled into libtpf.so.
 *
 *   n          demand buses (the column length)
 *   K_dev      device, complex128 [n][n], K = -Y_dd^{-1} (e.g. from tpf_precompute_host)
 *   W_dev      device, complex128 [n], W = K Y_ds v_s
 *   T          columns; T = 0 is a valid empty solve
 *   S_dev      device, complex128 [T][n], the loads (read only)
 *   V_dev      device, complex128 [T][n], receives V; read first as V_0 if given_start != 0,
 *              otherwise the flat start 1 + j0 is used
 *   iters_dev  device, int32 [T], sweeps applied per column or -max_iter (NULL: not written)
 *   tol, max_iter  as in tpf_opts;   stream  a cudaStream_t
 *
 * Scratch limit: the solve needs 1024 + 16 * T_128 * (n + 1) bytes of the built-in array, where
 * T_128 is T rounded up to a multiple of 128; more than TPF_NOALLOC_SCRATCH_BYTES (64 MiB) is
 * rejected with TPF_EINVAL before any device work.  No power mismatch is computed (there is no
 * network on the device here).  The array occupies 64 MiB on every device that loads the library,
 * until the process exits.
 *
 * Set-up: the first call on each device looks the array's device address up (with that device
 * current) and keeps it; make that first call before any stream capture begins.  Every call uses
 * the same array and leaves its contents behind; each call re-initialises the state it reads, but
 * calls whose device work overlaps (different streams, or different host threads, on one device)
 * race on the array and must be serialised by the caller.  Blocks until the stream has finished.
 * This entry point calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define TPF_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
tpf_status tpf_solve_fp64_noalloc(int n, const void *K_dev, const void *W_dev, int64_t T,
                                  const void *S_dev, void *V_dev, int32_t *iters_dev, double tol,
                                  int max_iter, int given_start, void *stream);

/*
 * Self-test of the tensor-core complex GEMM used by the mixed solve (tcgen05, fp16 operands,
 * FP32 accumulation): D = A B^T over complex numbers, with
 *   A_re, A_im  device fp16 [M][K] (row-major, K fastest),  B_re, B_im device fp16 [N][K],
 *   D_re, D_im  device float32 [N][M] (D[n][m] = sum_k A[m][k] B[n][k]).
 * M, N, K must be positive multiples of 128, 128 and 64.  Blocks until done.
 */
tpf_status tpf_selftest_gemm(int M, int N, int K, const void *A_re, const void *A_im,
                             const void *B_re, const void *B_im, float *D_re, float *D_im,
                             void *stream);

/*
 * Self-test of the GEMM's bounded device waits (failure detection; the paper has no counterpart).
 * The same product as tpf_selftest_gemm, with every wait of the kernel for its work (a copy that
 * fills a ring slot, an MMA that frees one, an accumulator for the epilogue) limited to wait_s
 * seconds, 1e-6 <= wait_s <= 10 (the solves use 2 s).  withhold_loads != 0 makes the kernel's
 * copy producer issue nothing, so the MMA and epilogue waits run out: the kernel raises its error
 * flag, waits (2 s at most) for its own copies and MMAs, frees its tensor memory and returns, and
 * the call returns TPF_ETIMEOUT after about 2 wait_s with the CUDA context still usable.  D is
 * unspecified after TPF_ETIMEOUT.  withhold_loads == 0 with a generous wait_s computes D as
 * tpf_selftest_gemm does.  Arguments and errors otherwise as tpf_selftest_gemm.  Blocks.
 */
tpf_status tpf_selftest_gemm_wait(int M, int N, int K, const void *A_re, const void *A_im,
                                  const void *B_re, const void *B_im, float *D_re, float *D_im,
                                  double wait_s, int withhold_loads, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TPF_H */
