/*
 * qpr_oracle.c -- plain FP64 CPU oracle for the quantum PageRank RK4 path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library. The GPU library
 * shares no code with it.
 *
 * What it computes, step by step, in the paper's order:
 *   - adjacency A from the edge list: A_ij = w for a link j -> i
 *     (Supplementary Note 1, first paragraph), outDeg(j) = sum_i A_ij;
 *   - Hamiltonian H_ij = -max(A_ij, A_ji) for i != j (Eq. S6); the diagonal
 *     is 0 (mode 0, the symmetrised-adjacency reading) or -outDeg(i)
 *     (mode 1, Eq. S6 taken literally);
 *   - Google matrix G = alpha*S + (1-alpha)*F (Eq. S4 with the
 *     column-normalised adjacency S in place of M) with F_ij = 1/(N-1) off
 *     the diagonal (Eq. S2); a dangling column j of S (outDeg(j) = 0) is
 *     replaced by F's column (mode 0) or by the uniform 1/N column (mode 1);
 *     c_j = sum_i G_ij;
 *   - Lindblad right-hand side (Eq. 1 / Eq. S7) with the N^2 jump operators
 *     L_ij = sqrt(G_ij)|i><j|:
 *        f(rho) = -(1-omega) i (H rho - rho H)
 *                 + omega ( diag(G p) - 1/2 (c_a + c_b) rho_ab ),
 *     p_a = rho_aa. The second line is sum_ij L rho L^dag - 1/2{L^dag L, rho}
 *     written out: L_ij rho L_ij^dag = G_ij rho_jj |i><i| and
 *     L_ij^dag L_ij = G_ij |j><j|;
 *   - classical RK4 (Supplementary Note 2, the fourth-order scheme):
 *        k1 = f(y), k2 = f(y + dt/2 k1), k3 = f(y + dt/2 k2),
 *        k4 = f(y + dt k3), y <- y + dt (k1 + 2 k2 + 2 k3 + k4) / 6,
 *     followed by division by Re tr y;
 *   - residual r = ||f(y)||_F over all N^2 complex entries; the steady-state
 *     loop stops at the first step index n whose r_n < tol.
 *   - the adaptive RKF45 scheme of Supplementary Note 2 (oracle_rkf45): the
 *     six stages of Eq. S10, the fourth-order solution y of Eq. S11 and the
 *     fifth-order solution z of Eq. S12 (the printed 845/4101 and 2197/4101
 *     read as 845/4104 and 2197/4104, the values that make the stage rows sum
 *     to their nodes and the weights of Eq. S11 sum to one), and the step
 *     factor s of Eq. S13. Readings where the note is silent are listed at
 *     oracle_rkf45.
 *
 * The initial state is first made exactly Hermitian, (rho + rho^dag)/2,
 * and divided by its real trace.
 *
 * Matrices are row-major. Complex matrices are interleaved (re, im) pairs,
 * i.e. C99 double complex arrays. H rho and rho H use a CSR copy of H (the
 * same numbers as the dense H; only zero entries are skipped).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { OR_OK = 0, OR_E_ARG = 1, OR_E_GRAPH = 2, OR_E_OOM = 4, OR_E_NOT_CONVERGED = 6, OR_E_NONFINITE = 8 };

typedef struct {
    int64_t n;
    double alpha, omega;
    int h_diag, dangling;
    double *A;      /* n*n adjacency, A[i*n+j] = weight of link j -> i */
    double *H;      /* n*n Hamiltonian */
    double *G;      /* n*n Google matrix */
    double *c;      /* n column sums of G */
    int64_t *h_ptr; /* CSR of H: row pointers (n+1) */
    int64_t *h_col; /* column indices */
    double *h_val;  /* values */
    int64_t self_loops, zero_weights;
    /* work buffers for RK4 (n*n complex each) */
    cplx *k, *acc, *tmp;
    /* work buffers for RKF45, allocated on first use: k1..k6, the stage
     * input, the fourth- and fifth-order solutions (n*n complex each) */
    cplx *rk[6], *rin, *ry, *rz;
} oracle_t;

void oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_free(oracle_t *o) {
    if (!o) return;
    free(o->A); free(o->H); free(o->G); free(o->c);
    free(o->h_ptr); free(o->h_col); free(o->h_val);
    free(o->k); free(o->acc); free(o->tmp);
    for (int i = 0; i < 6; ++i) free(o->rk[i]);
    free(o->rin); free(o->ry); free(o->rz);
    free(o);
}

/* Build every operator from the edge list. Returns NULL and sets *status on
 * invalid input: n < 2, alpha or omega outside [0, 1], an index outside
 * [0, n), or a weight that is negative or not finite. Self-loops and
 * zero-weight edges are dropped (and counted); duplicate links sum. */
oracle_t *oracle_create(int64_t n, int64_t m, const int64_t *src, const int64_t *dst,
                        const double *w, double alpha, double omega, int h_diag,
                        int dangling, int *status) {
    *status = OR_OK;
    if (n < 2 || m < 0 || !(alpha >= 0.0 && alpha <= 1.0) || !(omega >= 0.0 && omega <= 1.0) ||
        (h_diag != 0 && h_diag != 1) || (dangling != 0 && dangling != 1) ||
        (m > 0 && (!src || !dst))) {
        *status = OR_E_ARG;
        return NULL;
    }
    for (int64_t e = 0; e < m; ++e) {
        double we = w ? w[e] : 1.0;
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n || !isfinite(we) || we < 0.0) {
            *status = OR_E_GRAPH;
            return NULL;
        }
    }
    oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
    if (!o) { *status = OR_E_OOM; return NULL; }
    o->n = n; o->alpha = alpha; o->omega = omega; o->h_diag = h_diag; o->dangling = dangling;
    size_t nn = (size_t)n * (size_t)n;
    o->A = (double *)calloc(nn, sizeof(double));
    o->H = (double *)calloc(nn, sizeof(double));
    o->G = (double *)calloc(nn, sizeof(double));
    o->c = (double *)calloc((size_t)n, sizeof(double));
    o->k = (cplx *)malloc(nn * sizeof(cplx));
    o->acc = (cplx *)malloc(nn * sizeof(cplx));
    o->tmp = (cplx *)malloc(nn * sizeof(cplx));
    if (!o->A || !o->H || !o->G || !o->c || !o->k || !o->acc || !o->tmp) {
        oracle_free(o); *status = OR_E_OOM; return NULL;
    }
    /* adjacency: A_ij = w for the link j -> i (edge src=j, dst=i) */
    for (int64_t e = 0; e < m; ++e) {
        double we = w ? w[e] : 1.0;
        if (src[e] == dst[e]) { o->self_loops++; continue; }
        if (we == 0.0) { o->zero_weights++; continue; }
        o->A[dst[e] * n + src[e]] += we;
    }
    /* out-degree outDeg(j) = sum_i A_ij */
    double *outdeg = (double *)calloc((size_t)n, sizeof(double));
    if (!outdeg) { oracle_free(o); *status = OR_E_OOM; return NULL; }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) outdeg[j] += o->A[i * n + j];
    /* Hamiltonian, Eq. S6 */
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            if (i != j) {
                double aij = o->A[i * n + j], aji = o->A[j * n + i];
                o->H[i * n + j] = -(aij > aji ? aij : aji);
            } else {
                o->H[i * n + i] = (h_diag == 1) ? -outdeg[i] : 0.0;
            }
        }
    /* Google matrix G = alpha S + (1 - alpha) F */
    double fo = 1.0 / (double)(n - 1);
    for (int64_t j = 0; j < n; ++j) {
        for (int64_t i = 0; i < n; ++i) {
            double s;
            if (outdeg[j] > 0.0) s = o->A[i * n + j] / outdeg[j];
            else if (dangling == 0) s = (i != j) ? fo : 0.0;
            else s = 1.0 / (double)n;
            double f = (i != j) ? fo : 0.0;
            o->G[i * n + j] = alpha * s + (1.0 - alpha) * f;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) o->c[j] += o->G[i * n + j];
    free(outdeg);
    /* CSR copy of H */
    int64_t nnz = 0;
    for (size_t q = 0; q < nn; ++q) nnz += (o->H[q] != 0.0);
    o->h_ptr = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    o->h_col = (int64_t *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int64_t));
    o->h_val = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
    if (!o->h_ptr || !o->h_col || !o->h_val) { oracle_free(o); *status = OR_E_OOM; return NULL; }
    int64_t q = 0;
    for (int64_t i = 0; i < n; ++i) {
        o->h_ptr[i] = q;
        for (int64_t j = 0; j < n; ++j)
            if (o->H[i * n + j] != 0.0) { o->h_col[q] = j; o->h_val[q] = o->H[i * n + j]; ++q; }
    }
    o->h_ptr[n] = q;
    return o;
}

int64_t oracle_n(const oracle_t *o) { return o->n; }
int64_t oracle_h_nnz(const oracle_t *o) { return o->h_ptr[o->n]; }
int64_t oracle_dropped_self_loops(const oracle_t *o) { return o->self_loops; }

void oracle_get_operators(const oracle_t *o, double *A, double *H, double *G, double *c) {
    size_t nn = (size_t)o->n * (size_t)o->n;
    if (A) memcpy(A, o->A, nn * sizeof(double));
    if (H) memcpy(H, o->H, nn * sizeof(double));
    if (G) memcpy(G, o->G, nn * sizeof(double));
    if (c) memcpy(c, o->c, (size_t)o->n * sizeof(double));
}

/* out = f(rho), Eq. S7 with L_ij = sqrt(G_ij)|i><j| (see the file header). */
void oracle_rhs(const oracle_t *o, const cplx *rho, cplx *out) {
    const int64_t n = o->n;
    const double om = o->omega;
    /* gain g = G p, p_j = Re rho_jj */
    double *g = (double *)malloc((size_t)n * sizeof(double));
    #pragma omp parallel for schedule(static)
    for (int64_t a = 0; a < n; ++a) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += o->G[a * n + j] * creal(rho[j * n + j]);
        g[a] = s;
    }
    #pragma omp parallel
    {
        cplx *hr = (cplx *)malloc((size_t)n * sizeof(cplx));
        cplx *rh = (cplx *)malloc((size_t)n * sizeof(cplx));
        #pragma omp for schedule(dynamic, 4)
        for (int64_t a = 0; a < n; ++a) {
            for (int64_t b = 0; b < n; ++b) { hr[b] = 0.0; rh[b] = 0.0; }
            /* (H rho)_{a,:} = sum_k H_ak rho_{k,:} */
            for (int64_t q = o->h_ptr[a]; q < o->h_ptr[a + 1]; ++q) {
                const int64_t k = o->h_col[q];
                const double h = o->h_val[q];
                const cplx *rk = rho + k * n;
                for (int64_t b = 0; b < n; ++b) hr[b] += h * rk[b];
            }
            /* (rho H)_{a,:} = sum_k rho_ak H_{k,:} */
            for (int64_t k = 0; k < n; ++k) {
                const cplx r = rho[a * n + k];
                for (int64_t q = o->h_ptr[k]; q < o->h_ptr[k + 1]; ++q) rh[o->h_col[q]] += r * o->h_val[q];
            }
            for (int64_t b = 0; b < n; ++b) {
                cplx coh = -(1.0 - om) * I * (hr[b] - rh[b]);
                cplx dis = -0.5 * (o->c[a] + o->c[b]) * rho[a * n + b];
                if (a == b) dis += g[a];
                out[a * n + b] = coh + om * dis;
            }
        }
        free(hr);
        free(rh);
    }
    free(g);
}

double oracle_frobenius(int64_t n, const cplx *x) {
    double s = 0.0;
    size_t nn = (size_t)n * (size_t)n;
    for (size_t q = 0; q < nn; ++q) s += creal(x[q]) * creal(x[q]) + cimag(x[q]) * cimag(x[q]);
    return sqrt(s);
}

double oracle_residual(oracle_t *o, const cplx *rho) {
    oracle_rhs(o, rho, o->k);
    return oracle_frobenius(o->n, o->k);
}

/* rho <- (rho + rho^dag)/2, then rho <- rho / Re tr rho. Returns the trace
 * used, or a non-positive / non-finite value on failure. */
double oracle_prepare(int64_t n, cplx *rho) {
    for (int64_t a = 0; a < n; ++a)
        for (int64_t b = a; b < n; ++b) {
            cplx x = rho[a * n + b], y = rho[b * n + a];
            cplx h = 0.5 * (x + conj(y));
            rho[a * n + b] = h;
            rho[b * n + a] = conj(h);
        }
    double tr = 0.0;
    for (int64_t a = 0; a < n; ++a) tr += creal(rho[a * n + a]);
    if (!(tr > 0.0) || !isfinite(tr)) return tr;
    size_t nn = (size_t)n * (size_t)n;
    for (size_t q = 0; q < nn; ++q) rho[q] /= tr;
    return tr;
}

/* One classical RK4 step of length dt on y, given k1 = f(y) already in o->k.
 * Afterwards y is divided by Re tr y. */
static void rk4_finish(oracle_t *o, cplx *y, double dt) {
    const int64_t n = o->n;
    const size_t nn = (size_t)n * (size_t)n;
    cplx *k = o->k, *acc = o->acc, *tmp = o->tmp;
    /* acc = k1 ; tmp = y + dt/2 k1 */
    for (size_t q = 0; q < nn; ++q) { acc[q] = k[q]; tmp[q] = y[q] + 0.5 * dt * k[q]; }
    oracle_rhs(o, tmp, k); /* k2 */
    for (size_t q = 0; q < nn; ++q) { acc[q] += 2.0 * k[q]; tmp[q] = y[q] + 0.5 * dt * k[q]; }
    oracle_rhs(o, tmp, k); /* k3 */
    for (size_t q = 0; q < nn; ++q) { acc[q] += 2.0 * k[q]; tmp[q] = y[q] + dt * k[q]; }
    oracle_rhs(o, tmp, k); /* k4 */
    for (size_t q = 0; q < nn; ++q) { acc[q] += k[q]; y[q] += (dt / 6.0) * acc[q]; }
    double tr = 0.0;
    for (int64_t a = 0; a < n; ++a) tr += creal(y[a * n + a]);
    for (size_t q = 0; q < nn; ++q) y[q] /= tr;
}

/* Fixed-step RK4: prepare rho, then take `steps` steps in place. */
int oracle_evolve(oracle_t *o, cplx *rho, double dt, int64_t steps) {
    if (!(dt > 0.0) || steps < 0) return OR_E_ARG;
    double tr = oracle_prepare(o->n, rho);
    if (!(tr > 0.0) || !isfinite(tr)) return OR_E_ARG;
    for (int64_t s = 0; s < steps; ++s) {
        oracle_rhs(o, rho, o->k);
        rk4_finish(o, rho, dt);
    }
    return OR_OK;
}

/* RK4 until the first step index n with ||f(y_n)||_F < tol (y_n is left in
 * rho), or until max_steps steps were taken (status OR_E_NOT_CONVERGED).
 * The residual of every step index is written to resid_hist when given
 * (length max_steps + 1). */
int oracle_steady_state(oracle_t *o, cplx *rho, double dt, double tol, int64_t max_steps,
                        int64_t *steps_out, double *resid_out, double *resid_hist) {
    if (!(dt > 0.0) || !(tol > 0.0) || max_steps < 0) return OR_E_ARG;
    double tr = oracle_prepare(o->n, rho);
    if (!(tr > 0.0) || !isfinite(tr)) return OR_E_ARG;
    for (int64_t s = 0;; ++s) {
        oracle_rhs(o, rho, o->k);
        double r = oracle_frobenius(o->n, o->k);
        if (resid_hist) resid_hist[s] = r;
        if (steps_out) *steps_out = s;
        if (resid_out) *resid_out = r;
        if (!isfinite(r)) return OR_E_NONFINITE;
        if (r < tol) return OR_OK;
        if (s == max_steps) return OR_E_NOT_CONVERGED;
        rk4_finish(o, rho, dt);
    }
}

/* ---- RKF45, Supplementary Note 2 (Eq. S10 - S13) ----
 *
 * The coefficients of Eq. S10 (stage inputs), Eq. S11 (fourth order) and
 * Eq. S12 (fifth order), written as the note prints them, with the two
 * garbled 4101 denominators read as 4104. */
static const double RKF_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4.0, 0, 0, 0, 0},
    {3.0 / 32.0, 9.0 / 32.0, 0, 0, 0},
    {1932.0 / 2197.0, -7200.0 / 2197.0, 7296.0 / 2197.0, 0, 0},
    {439.0 / 216.0, -8.0, 3680.0 / 513.0, -845.0 / 4104.0, 0},
    {-8.0 / 27.0, 2.0, -3544.0 / 2565.0, 1859.0 / 4104.0, -11.0 / 40.0}};
static const double RKF_Y[6] = {25.0 / 216.0, 0.0, 1408.0 / 2565.0, 2197.0 / 4104.0, -1.0 / 5.0, 0.0};
static const double RKF_Z[6] = {16.0 / 135.0, 0.0, 6656.0 / 12825.0, 28561.0 / 56430.0, -9.0 / 50.0, 2.0 / 55.0};

static int rkf_alloc(oracle_t *o) {
    if (o->rin) return 1;
    const size_t nn = (size_t)o->n * (size_t)o->n;
    for (int i = 0; i < 6; ++i) o->rk[i] = (cplx *)malloc(nn * sizeof(cplx));
    o->rin = (cplx *)malloc(nn * sizeof(cplx));
    o->ry = (cplx *)malloc(nn * sizeof(cplx));
    o->rz = (cplx *)malloc(nn * sizeof(cplx));
    int ok = o->rin && o->ry && o->rz;
    for (int i = 0; i < 6; ++i) ok = ok && o->rk[i];
    if (!ok) {
        for (int i = 0; i < 6; ++i) { free(o->rk[i]); o->rk[i] = NULL; }
        free(o->rin); free(o->ry); free(o->rz);
        o->rin = o->ry = o->rz = NULL;
    }
    return ok;
}

/* One attempt of step h from y_k (Eq. S10 - S12), with f(y_k) already in
 * o->k: k1 = h f(y_k), k_s = h f(y_k + sum_j a_sj k_j), then y_{k+1} into
 * o->ry, z_{k+1} into o->rz. Returns the discrepancy |z_{k+1} - y_{k+1}|,
 * read as the largest modulus over the N^2 entries. */
static double rkf_attempt(oracle_t *o, const cplx *y, double h) {
    const size_t nn = (size_t)o->n * (size_t)o->n;
    for (size_t q = 0; q < nn; ++q) o->rk[0][q] = h * o->k[q];
    for (int s = 1; s < 6; ++s) {
        for (size_t q = 0; q < nn; ++q) {
            cplx v = y[q];
            for (int j = 0; j < s; ++j) v += RKF_A[s][j] * o->rk[j][q];
            o->rin[q] = v;
        }
        oracle_rhs(o, o->rin, o->rk[s]);
        for (size_t q = 0; q < nn; ++q) o->rk[s][q] *= h;
    }
    double err = 0.0;
    for (size_t q = 0; q < nn; ++q) {
        cplx yv = y[q], zv = y[q];
        for (int j = 0; j < 6; ++j) {
            yv += RKF_Y[j] * o->rk[j][q];
            zv += RKF_Z[j] * o->rk[j][q];
        }
        o->ry[q] = yv;
        o->rz[q] = zv;
        const double d = cabs(zv - yv);
        if (d > err || isnan(d)) err = d;
    }
    return err;
}

/* Adaptive RKF45 on rho in place (Supplementary Note 2, Eq. S10 - S13).
 *
 * Each attempt from the current state y_k with step h forms k1..k6, the
 * fourth-order y_{k+1} and the fifth-order z_{k+1}, and the factor
 * s = (step_tol h / (2 |z_{k+1} - y_{k+1}|))^(1/4) of Eq. S13; the next
 * attempt uses s h. Readings where the note is silent:
 *   - |.| is the largest modulus of the N^2 complex entries of z - y;
 *   - an attempt is accepted when |z_{k+1} - y_{k+1}| <= step_tol h (a
 *     discrepancy within the tolerance per unit time), and then y_{k+1}, the
 *     fourth-order solution that Eq. S11 defines as the approximation, is
 *     the new state (order = 4), or z_{k+1}, the fifth-order relationship the
 *     note offers as the alternative (order = 5); otherwise the state is kept
 *     and the attempt is repeated with s h;
 *   - s is clipped to [1/10, 4] and s h to h_max (a discrepancy of zero
 *     gives the largest factor), and in a trajectory the last step is
 *     shortened to end exactly at t_end;
 *   - after every accepted step the state is divided by its real trace, as
 *     in the fixed-step RK4 of this file.
 * Stops at the first accepted state y_k with ||f(y_k)||_F < resid_tol
 * (steady state; resid_tol = 0 never stops this way), when the integrated
 * time reaches t_end (trajectory; INFINITY for none), or after max_steps
 * accepted steps (OR_E_NOT_CONVERGED in steady-state mode). The initial
 * state is prepared as in oracle_evolve. Outputs (nullable): accepted and
 * rejected attempts, the time reached, the step size the next attempt would
 * use, the residual of the returned state; hist (nullable, 5 doubles per
 * attempt, at most hist_cap attempts): t, h, discrepancy, s, accepted. */
int oracle_rkf45(oracle_t *o, cplx *rho, double h0, double step_tol, double h_max, double resid_tol, double t_end,
                 int64_t max_steps, int order, int64_t *accepted_out, int64_t *rejected_out, double *t_out,
                 double *h_out, double *resid_out, double *hist, int64_t hist_cap) {
    if (!(h0 > 0.0) || !(step_tol > 0.0) || !(h_max > 0.0) || !(resid_tol >= 0.0) || max_steps < 0 ||
        !(t_end > 0.0) || (order != 4 && order != 5))
        return OR_E_ARG;
    double tr = oracle_prepare(o->n, rho);
    if (!(tr > 0.0) || !isfinite(tr)) return OR_E_ARG;
    if (!rkf_alloc(o)) return OR_E_OOM;
    const int64_t n = o->n;
    const size_t nn = (size_t)n * (size_t)n;
    double h = h0 < h_max ? h0 : h_max, t = 0.0, r = 0.0;
    int64_t acc = 0, rej = 0, na = 0;
    int status = OR_OK;
    oracle_rhs(o, rho, o->k);
    r = oracle_frobenius(n, o->k);
    for (;;) {
        if (!isfinite(r)) { status = OR_E_NONFINITE; break; }
        if (resid_tol > 0.0 && r < resid_tol) break;
        if (t >= t_end) break;
        if (acc >= max_steps) { status = (resid_tol > 0.0) ? OR_E_NOT_CONVERGED : OR_OK; break; }
        const double hs = (t + h > t_end) ? t_end - t : h;
        const double err = rkf_attempt(o, rho, hs);
        if (!isfinite(err)) { status = OR_E_NONFINITE; break; }
        double sfac = (err > 0.0) ? pow(step_tol * hs / (2.0 * err), 0.25) : 4.0;
        if (sfac < 0.1) sfac = 0.1;
        if (sfac > 4.0) sfac = 4.0;
        const int ok = err <= step_tol * hs;
        if (hist && na < hist_cap) {
            double *e = hist + 5 * na;
            e[0] = t; e[1] = hs; e[2] = err; e[3] = sfac; e[4] = ok ? 1.0 : 0.0;
        }
        ++na;
        if (ok) {
            memcpy(rho, order == 5 ? o->rz : o->ry, nn * sizeof(cplx));
            double trc = 0.0;
            for (int64_t a = 0; a < n; ++a) trc += creal(rho[a * n + a]);
            for (size_t q = 0; q < nn; ++q) rho[q] /= trc;
            t = (t + hs > t_end) ? t_end : t + hs;
            ++acc;
            oracle_rhs(o, rho, o->k);
            r = oracle_frobenius(n, o->k);
        } else {
            ++rej;
        }
        h = sfac * hs;
        if (h > h_max) h = h_max;
    }
    if (accepted_out) *accepted_out = acc;
    if (rejected_out) *rejected_out = rej;
    if (t_out) *t_out = t;
    if (h_out) *h_out = h;
    if (resid_out) *resid_out = r;
    return status;
}

/* One RKF45 attempt of step h from rho (prepared as in oracle_evolve) with
 * no step-size control: y_{k+1} (Eq. S11) into y4 and z_{k+1} (Eq. S12)
 * into z5 (each nullable); returns the discrepancy |z - y| (largest modulus). */
double oracle_rkf45_step(oracle_t *o, const cplx *rho, double h, cplx *y4, cplx *z5) {
    if (!rkf_alloc(o)) return NAN;
    const size_t nn = (size_t)o->n * (size_t)o->n;
    oracle_rhs(o, rho, o->k);
    const double err = rkf_attempt(o, rho, h);
    if (y4) memcpy(y4, o->ry, nn * sizeof(cplx));
    if (z5) memcpy(z5, o->rz, nn * sizeof(cplx));
    return err;
}
