/*
 * Oracle for the tensor power flow -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, double-precision CPU restatement of the paper's dense fixed-point power flow
 * (Sec. II Eq. 1-3, Sec. IV-A Eq. 12 and Algorithm 1).  It exists to check the CUDA library; only
 * the tests, the smoke check and the benchmark's CPU legs (CPU baseline, reference arm, accuracy
 * checks after each timed region) may load it.  It shares no code with the library.
 *
 * Conventions (all complex numbers are C99 double complex, laid out like numpy complex128):
 *   - Y is the dense (n_bus x n_bus) nodal admittance matrix of Eq. 1, built branch by branch.
 *   - The PQ (demand) buses are listed in pq[0..n_pq); Y_dd = Y[pq][pq], Y_ds = Y[pq][slack].
 *   - S is the load (consumption positive), so the demand-node current of Eq. 1 is
 *     i_d = conj(S ./ v), and the constant-power case of Eq. 3 (alpha_P = 1, alpha_Z = alpha_I = 0)
 *     gives  v <- K conj(S ./ v) + W  with  K = -Y_dd^{-1},  W = K Y_ds v_s.
 *   - Load tensors are row-major [T][n_pq]: one power flow (one column of Eq. 12's reshaped
 *     S-dot) per row.
 *
 * Stopping rule: the paper's Algorithm 1 loops while a global tolerance is not met; here each
 * column stops on its own at the first iterate with max_i |v_{k+1,i} - v_{k,i}| <= tol, and its
 * iteration count is the number of updates applied (-max_iter if it never met tol).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Eq. 1: Y = sum over branches e=(a,b) of y_e (u_a - u_b)(u_a - u_b)^T, y_e = 1/z_e (no shunts). */
int orc_build_ybus(int n_bus, int n_branch, const int *from, const int *to, const cplx *z, cplx *Y)
{
    memset(Y, 0, sizeof(cplx) * (size_t)n_bus * n_bus);
    for (int e = 0; e < n_branch; ++e) {
        int a = from[e], b = to[e];
        if (a < 0 || b < 0 || a >= n_bus || b >= n_bus || a == b) return 1;
        if (z[e] == 0) return 2;
        cplx y = 1.0 / z[e];
        Y[(size_t)a * n_bus + a] += y;
        Y[(size_t)b * n_bus + b] += y;
        Y[(size_t)a * n_bus + b] -= y;
        Y[(size_t)b * n_bus + a] -= y;
    }
    return 0;
}

/* In-place inverse of a dense complex n x n matrix by Gauss-Jordan elimination with partial
 * pivoting.  Returns 0, or 1 if a pivot is (numerically) zero. */
int orc_invert(int n, cplx *A)
{
    size_t N = (size_t)n;
    cplx *aug = (cplx *)malloc(sizeof(cplx) * N * 2 * N);
    if (!aug) return 2;
    for (size_t i = 0; i < N; ++i) {
        for (size_t j = 0; j < N; ++j) {
            aug[i * 2 * N + j] = A[i * N + j];
            aug[i * 2 * N + N + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    double scale = 0.0;
    for (size_t i = 0; i < N * N; ++i) scale = fmax(scale, cabs(A[i]));
    for (size_t c = 0; c < N; ++c) {
        size_t piv = c;
        double best = cabs(aug[c * 2 * N + c]);
        for (size_t r = c + 1; r < N; ++r) {
            double v = cabs(aug[r * 2 * N + c]);
            if (v > best) { best = v; piv = r; }
        }
        if (!(best > 1e-300) || best < 1e-14 * scale) { free(aug); return 1; }
        if (piv != c) {
            for (size_t j = 0; j < 2 * N; ++j) {
                cplx t = aug[c * 2 * N + j];
                aug[c * 2 * N + j] = aug[piv * 2 * N + j];
                aug[piv * 2 * N + j] = t;
            }
        }
        cplx inv = 1.0 / aug[c * 2 * N + c];
        for (size_t j = 0; j < 2 * N; ++j) aug[c * 2 * N + j] *= inv;
        for (size_t r = 0; r < N; ++r) {
            if (r == c) continue;
            cplx f = aug[r * 2 * N + c];
            if (f == 0) continue;
            for (size_t j = 0; j < 2 * N; ++j) aug[r * 2 * N + j] -= f * aug[c * 2 * N + j];
        }
    }
    for (size_t i = 0; i < N; ++i)
        for (size_t j = 0; j < N; ++j) A[i * N + j] = aug[i * 2 * N + N + j];
    free(aug);
    return 0;
}

/* Eq. 3 for constant power: K = -Y_dd^{-1} (the paper's Z_B with the sign of F = -B^{-1}A folded
 * in) and W = K Y_ds v_s.  Returns 0, or 1 if Y_dd is singular. */
int orc_precompute(int n_bus, const cplx *Y, int slack, double vs_re, double vs_im, int n_pq, const int *pq,
                   cplx *K, cplx *W)
{
    cplx vs = vs_re + I * vs_im;
    size_t n = (size_t)n_pq;
    for (size_t i = 0; i < n; ++i)
        for (size_t j = 0; j < n; ++j) K[i * n + j] = Y[(size_t)pq[i] * n_bus + pq[j]];
    if (orc_invert(n_pq, K)) return 1;
    for (size_t i = 0; i < n * n; ++i) K[i] = -K[i];
    for (size_t i = 0; i < n; ++i) {
        cplx acc = 0;
        for (size_t j = 0; j < n; ++j) acc += K[i * n + j] * Y[(size_t)pq[j] * n_bus + slack];
        W[i] = acc * vs;
    }
    return 0;
}

/* Algorithm 1 with per-column stopping.  For each column t of S ([T][n] row-major):
 *   v_0 = V0[t] (or 1 + j0, the flat start, when V0 is NULL)
 *   v_{k+1} = K conj(S[t] ./ v_k) + W           (Eq. 2 / Eq. 12, one column of the tensor)
 *   stop at the first k with max_i |v_{k+1,i} - v_{k,i}| <= tol, or after max_iter updates.
 * Outputs V[t] = last iterate, iters[t] = updates applied (negated to -max_iter if tol was never
 * met), last_delta[t] = the last max-norm step.  n_threads <= 0 uses the OpenMP default. */
void orc_fpi(int n, const cplx *K, const cplx *W, long T, const cplx *S, const cplx *V0, double tol,
             int max_iter, cplx *V, int *iters, double *last_delta, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
#pragma omp parallel
    {
        cplx *v = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *cur = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *vn = (cplx *)malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(dynamic, 4)
        for (long t = 0; t < T; ++t) {
            const cplx *s = S + (size_t)t * n;
            for (int i = 0; i < n; ++i) v[i] = V0 ? V0[(size_t)t * n + i] : 1.0;
            int k = 0, done = 0;
            double delta = INFINITY;
            while (k < max_iter) {
                for (int j = 0; j < n; ++j) cur[j] = conj(s[j] / v[j]);
                delta = 0.0;
                for (int i = 0; i < n; ++i) {
                    const cplx *Ki = K + (size_t)i * n;
                    cplx acc = 0;
                    for (int j = 0; j < n; ++j) acc += Ki[j] * cur[j];
                    vn[i] = acc + W[i];
                    double d = cabs(vn[i] - v[i]);
                    if (!(d <= delta)) delta = d; /* NaN propagates */
                }
                memcpy(v, vn, sizeof(cplx) * (size_t)n);
                ++k;
                if (delta <= tol) { done = 1; break; }
            }
            memcpy(V + (size_t)t * n, v, sizeof(cplx) * (size_t)n);
            iters[t] = done ? k : -max_iter;
            last_delta[t] = delta;
        }
        free(v);
        free(cur);
        free(vn);
    }
}

/* Power mismatch of each column: max_i |V_i conj((Y v)_i) + S_i| over the PQ buses, with the
 * slack held at vs (Eq. 1 with the injection of a PQ bus equal to minus its load). */
void orc_mismatch(int n_bus, const cplx *Y, int slack, double vs_re, double vs_im, int n_pq, const int *pq,
                  long T, const cplx *S, const cplx *V, double *out)
{
    cplx vs = vs_re + I * vs_im;
    cplx *full = (cplx *)malloc(sizeof(cplx) * (size_t)n_bus);
    for (long t = 0; t < T; ++t) {
        full[slack] = vs;
        for (int i = 0; i < n_pq; ++i) full[pq[i]] = V[(size_t)t * n_pq + i];
        double worst = 0.0;
        for (int i = 0; i < n_pq; ++i) {
            const cplx *Yr = Y + (size_t)pq[i] * n_bus;
            cplx acc = 0;
            for (int j = 0; j < n_bus; ++j) acc += Yr[j] * full[j];
            double m = cabs(full[pq[i]] * conj(acc) + S[(size_t)t * n_pq + i]);
            if (!(m <= worst)) worst = m;
        }
        out[t] = worst;
    }
    free(full);
}

/* Eq. 3 with the ZIP load model of the paper, one column at a time.  alpha is [3][n_pq]: the
 * alpha_P, alpha_I and alpha_Z coefficients of every demand bus.  The demand current of Eq. 1 is
 * i_d = alpha_P .* conj(s) ./ conj(v) + alpha_I .* conj(s) + alpha_Z .* conj(s) .* v, and for
 * each column s (its own operating point):
 *   A = diag(alpha_P .* conj(s)),  B = diag(alpha_Z .* conj(s)) + Y_dd,
 *   c = Y_ds v_s + alpha_I .* conj(s),  F = -B^{-1} A,  w = -B^{-1} c,
 *   v_{k+1} = F conj(v_k)^{.-1} + w
 * with orc_fpi's start and stopping rule.  A column whose B is singular returns NaN and
 * -max_iter.  Dense, O(n^3) per column: for small test cases only. */
void orc_fpi_zip(int n_bus, const cplx *Y, int slack, double vs_re, double vs_im, int n_pq, const int *pq,
                 const double *alpha, long T, const cplx *S, const cplx *V0, double tol, int max_iter,
                 cplx *V, int *iters, double *last_delta, int n_threads)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const cplx vs = vs_re + I * vs_im;
    const int n = n_pq;
    const double *aP = alpha, *aI = alpha + n, *aZ = alpha + 2 * n;
#pragma omp parallel
    {
        cplx *B = (cplx *)malloc(sizeof(cplx) * (size_t)n * n);
        cplx *F = (cplx *)malloc(sizeof(cplx) * (size_t)n * n);
        cplx *w = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *c = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *v = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *cur = (cplx *)malloc(sizeof(cplx) * (size_t)n);
        cplx *vn = (cplx *)malloc(sizeof(cplx) * (size_t)n);
#pragma omp for schedule(dynamic, 1)
        for (long t = 0; t < T; ++t) {
            const cplx *s = S + (size_t)t * n;
            for (int i = 0; i < n; ++i) {
                for (int j = 0; j < n; ++j) B[(size_t)i * n + j] = Y[(size_t)pq[i] * n_bus + pq[j]];
                B[(size_t)i * n + i] += aZ[i] * conj(s[i]);
                c[i] = Y[(size_t)pq[i] * n_bus + slack] * vs + aI[i] * conj(s[i]);
            }
            if (orc_invert(n, B)) {
                for (int i = 0; i < n; ++i) V[(size_t)t * n + i] = NAN;
                iters[t] = -max_iter;
                last_delta[t] = INFINITY;
                continue;
            }
            for (int i = 0; i < n; ++i) {
                cplx acc = 0;
                for (int j = 0; j < n; ++j) {
                    F[(size_t)i * n + j] = -B[(size_t)i * n + j] * (aP[j] * conj(s[j]));
                    acc += B[(size_t)i * n + j] * c[j];
                }
                w[i] = -acc;
            }
            for (int i = 0; i < n; ++i) v[i] = V0 ? V0[(size_t)t * n + i] : 1.0;
            int k = 0, done = 0;
            double delta = INFINITY;
            while (k < max_iter) {
                for (int j = 0; j < n; ++j) cur[j] = 1.0 / conj(v[j]);
                delta = 0.0;
                for (int i = 0; i < n; ++i) {
                    cplx acc = 0;
                    for (int j = 0; j < n; ++j) acc += F[(size_t)i * n + j] * cur[j];
                    vn[i] = acc + w[i];
                    double d = cabs(vn[i] - v[i]);
                    if (!(d <= delta)) delta = d;
                }
                memcpy(v, vn, sizeof(cplx) * (size_t)n);
                ++k;
                if (delta <= tol) { done = 1; break; }
            }
            memcpy(V + (size_t)t * n, v, sizeof(cplx) * (size_t)n);
            iters[t] = done ? k : -max_iter;
            last_delta[t] = delta;
        }
        free(B); free(F); free(w); free(c); free(v); free(cur); free(vn);
    }
}

/* Power balance of Eq. 1 with ZIP loads: max_i |V_i| |(Y v)_i + i_d,i| over the demand buses, with
 * i_d as in orc_fpi_zip (for alpha_P = 1 this is orc_mismatch's |V_i conj((Y v)_i) + S_i|). */
void orc_mismatch_zip(int n_bus, const cplx *Y, int slack, double vs_re, double vs_im, int n_pq, const int *pq,
                      const double *alpha, long T, const cplx *S, const cplx *V, double *out)
{
    cplx vs = vs_re + I * vs_im;
    const double *aP = alpha, *aI = alpha + n_pq, *aZ = alpha + 2 * n_pq;
    cplx *full = (cplx *)malloc(sizeof(cplx) * (size_t)n_bus);
    for (long t = 0; t < T; ++t) {
        full[slack] = vs;
        for (int i = 0; i < n_pq; ++i) full[pq[i]] = V[(size_t)t * n_pq + i];
        double worst = 0.0;
        for (int i = 0; i < n_pq; ++i) {
            const cplx *Yr = Y + (size_t)pq[i] * n_bus;
            cplx acc = 0;
            for (int j = 0; j < n_bus; ++j) acc += Yr[j] * full[j];
            const cplx s = S[(size_t)t * n_pq + i], vi = full[pq[i]];
            const cplx id = aP[i] * conj(s / vi) + aI[i] * conj(s) + aZ[i] * conj(s) * vi;
            double m = cabs(vi) * cabs(acc + id);
            if (!(m <= worst)) worst = m;
        }
        out[t] = worst;
    }
    free(full);
}

/* Admittance matrix of Eq. 1 for a polyphase network, node index b*phases + p
 * for bus b and phase p.  Branch e joins from[e] and to[e] with the phases x phases series impedance
 * matrix Z_e (row-major, z + e*phases*phases); its admittance Y_e = Z_e^{-1} adds to the two
 * diagonal blocks and subtracts from the two off-diagonal blocks.  Returns 0, or 1 for a bus index
 * out of range, 2 for a singular branch matrix. */
int orc_build_ybus_poly(int n_bus, int n_branch, int phases, const int *from, const int *to, const cplx *z,
                        cplx *Y)
{
    const int ph = phases, N = n_bus * phases;
    memset(Y, 0, sizeof(cplx) * (size_t)N * N);
    cplx *Ye = (cplx *)malloc(sizeof(cplx) * (size_t)ph * ph);
    for (int e = 0; e < n_branch; ++e) {
        const int a = from[e], b = to[e];
        if (a < 0 || b < 0 || a >= n_bus || b >= n_bus || a == b) { free(Ye); return 1; }
        memcpy(Ye, z + (size_t)e * ph * ph, sizeof(cplx) * (size_t)ph * ph);
        if (orc_invert(ph, Ye)) { free(Ye); return 2; }
        for (int p = 0; p < ph; ++p)
            for (int q = 0; q < ph; ++q) {
                const cplx y = Ye[p * ph + q];
                Y[(size_t)(a * ph + p) * N + a * ph + q] += y;
                Y[(size_t)(b * ph + p) * N + b * ph + q] += y;
                Y[(size_t)(a * ph + p) * N + b * ph + q] -= y;
                Y[(size_t)(b * ph + p) * N + a * ph + q] -= y;
            }
    }
    free(Ye);
    return 0;
}
