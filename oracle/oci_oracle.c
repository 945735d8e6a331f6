/*
 * FP64 CPU oracle for MB-SCB transient slab S_N transport (arXiv 2305.13555).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file; only the tests, the package's smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code with the CUDA implementation.
 *
 * What it computes, in the paper's notation and order:
 *   - Gauss-Legendre S_N quadrature (Sec. 2: "Gauss Legendre quadrature was used
 *     in all presented explorations"), weights summing to 2 as implied by the
 *     1/2 factor of Eq. 1.
 *   - One OCI iteration (Sec. "One-Cell Inversion (OCI)"): for every cell j the
 *     dense 4N x 4N system (A - S) Psi = c is assembled literally from the
 *     printed A^+ / A^- matrices, the scattering matrix S_{l,n} = dx Sigma_s w_n/4
 *     (read as coupling the same corner / time moment across ordinates) and the
 *     printed c^+ / c^- vectors whose neighbour fluxes come from iterate l; the
 *     system is solved by LU with partial pivoting, factorised once per distinct
 *     material per call.
 *   - One SI iteration (Sec. "Source Iteration (SI)"): per ordinate a transport
 *     sweep in the direction of travel, solving the printed 4x4 A^+/A^- system
 *     with the printed b^+/b^- right-hand side (lagged scalar flux) by LU with
 *     partial pivoting, then the scalar-flux update sum_n w_n psi_n.
 *   - The time-step driver: iterate until ||phi^{l+1}-phi^l||_2/||phi^{l+1}||_2
 *     < tol (the paper says only "until ... ceases changing"; the relative L2
 *     norm over all 4 moments of all cells is this implementation's reading),
 *     then psi_{k-1/2} <- psi_{k+1/2} (multiple balance, Eqs. 2-3).
 *
 * Readings of points the paper leaves open (stated once here):
 *   - initial iterate of a step: Psi^(0) has both time moments equal to the
 *     previous time-edge flux psi_{k-1/2} (L and R corners), phi^(0) = sum w Psi^(0);
 *   - reflecting boundary: the incident flux equals the mirror ordinate's
 *     outgoing flux at that face; OCI takes it from iterate l, SI sweeps mu<0
 *     first so a reflecting left face sees the current sweep, while a reflecting
 *     right face uses iterate l;
 *   - prescribed incident boundary values are given per time moment (k, k+1/2).
 *
 * Backward-Euler variant (the paper's disabled section "Backward Euler transient
 * implementation"): one time level per step, the total cross section becomes
 * Sigma_hat = Sigma + 1/(v dt) and the previous step's angular flux enters as a
 * source psi^{n-1}/(v dt).  In space it is the same SCB cell: the per-ordinate
 * 2x2 block is the SCB part of the printed A^+/A^- (their k-rows with the time
 * terms removed) with Sigma_hat, and S couples the same corner across ordinates.
 * Reading: the source at the new time is Q_{k+1/2} (components 2, 3 of q).
 *   be_psi [J][N][2] (L,R) at the new time; be_phi [J][2].
 *
 * Layouts (row-major, doubles):
 *   ordinates m = 0..N-1 ascending in mu (mu_m < 0 for m < N/2); mirror(m) = N-1-m;
 *   psi      [J][N][4]  components (k,L) (k,R) (k+1/2,L) (k+1/2,R), Eq. for psi_n;
 *   psi_edge [J][N][2]  time-edge flux (L,R);
 *   phi      [J][4]     same component order as psi;
 *   q        [J][4]     Q_{k,L} Q_{k,R} Q_{k+1/2,L} Q_{k+1/2,R};
 *   bc       [N/2][2]   (k, k+1/2) for pair p: left face -> ordinate N/2+p (mu>0),
 *                       right face -> ordinate N/2-1-p (mu<0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_BC_VACUUM = 0, ORC_BC_REFLECT = 1, ORC_BC_INCIDENT = 2 };
enum { ORC_OCI = 0, ORC_SI = 1 };

typedef struct {
    int32_t n_cells;
    int32_t n_ord;
    const double *dx, *sigma_t, *sigma_s; /* [J] */
    const double *q;                      /* [J][4] */
    double v, dt;                         /* v may be +inf: steady state (1/(v dt) = 0) */
    int32_t bc_left, bc_right;
    const double *psi_bc_left, *psi_bc_right; /* [N/2][2] or NULL */
} oracle_problem;

/* ---------------------------------------------------------------- quadrature */

/* Gauss-Legendre nodes/weights on [-1,1] by Newton's method on P_N, using the
 * three-term recurrence (k+1)P_{k+1} = (2k+1) x P_k - k P_{k-1} and
 * w = 2 / ((1-x^2) P_N'(x)^2).  Nodes returned in ascending order. */
int oracle_gauss_legendre(int32_t n, double *mu, double *w)
{
    if (n < 1) return 1;
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double x = cos(pi * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 1; k < n; ++k) {
                double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = x; p0 = 1.0; }
            dp = n * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) {
                /* one more pass to settle dp at the converged node */
                p0 = 1.0; p1 = x;
                for (int k = 1; k < n; ++k) {
                    double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
                    p0 = p1;
                    p1 = p2;
                }
                if (n == 1) { p1 = x; p0 = 1.0; }
                dp = n * (x * p1 - p0) / (x * x - 1.0);
                break;
            }
        }
        double wi = 2.0 / ((1.0 - x * x) * dp * dp);
        /* x is the i-th largest node */
        mu[n - 1 - i] = x;
        mu[i] = -x;
        w[n - 1 - i] = wi;
        w[i] = wi;
    }
    if (n % 2 == 1) mu[n / 2] = 0.0;
    return 0;
}

/* ------------------------------------------------------------ dense LU helpers */

/* In-place LU with partial pivoting of an n x n row-major matrix (the operation
 * of LAPACK's _gesv factorisation step).  Returns 0, or 1 for a zero pivot. */
static int lu_factor(int n, double *a, int *piv)
{
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(a[(size_t)k * n + k]);
        for (int i = k + 1; i < n; ++i) {
            double v = fabs(a[(size_t)i * n + k]);
            if (v > best) { best = v; p = i; }
        }
        piv[k] = p;
        if (best == 0.0) return 1;
        if (p != k) {
            for (int c = 0; c < n; ++c) {
                double t = a[(size_t)k * n + c];
                a[(size_t)k * n + c] = a[(size_t)p * n + c];
                a[(size_t)p * n + c] = t;
            }
        }
        double inv = 1.0 / a[(size_t)k * n + k];
        for (int i = k + 1; i < n; ++i) {
            double f = a[(size_t)i * n + k] * inv;
            a[(size_t)i * n + k] = f;
            if (f != 0.0)
                for (int c = k + 1; c < n; ++c) a[(size_t)i * n + c] -= f * a[(size_t)k * n + c];
        }
    }
    return 0;
}

/* Solve with the factors of lu_factor; b is overwritten by the solution.
 * lu_factor interchanges whole rows (multipliers included), so P A = L U with
 * P the product of all interchanges: apply them all to b first, then the two
 * triangular solves. */
static void lu_solve(int n, const double *lu, const int *piv, double *b)
{
    for (int k = 0; k < n; ++k) {
        int p = piv[k];
        if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; }
    }
    for (int k = 0; k < n; ++k)
        for (int i = k + 1; i < n; ++i) b[i] -= lu[(size_t)i * n + k] * b[k];
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int c = i + 1; c < n; ++c) s -= lu[(size_t)i * n + c] * b[c];
        b[i] = s / lu[(size_t)i * n + i];
    }
}

/* ------------------------------------------------------- per-ordinate A^+/A^- */

/* The 4x4 matrix printed for A^+ (mu_m > 0) and A^- (mu_m < 0) in the SI section,
 * written element by element as printed.  Row-major into a[16]. */
static void assemble_A_m(double mu, double dx, double sig, double v, double dt, double *a)
{
    const double e = dx / (2.0 * v * dt); /* dx / (2 v dt) */
    const double E = dx / (v * dt);       /* dx / (v dt)   */
    double d;
    if (mu > 0.0) d = (mu + dx * sig) / 2.0;   /* A^+ diagonal */
    else          d = (-mu + dx * sig) / 2.0;  /* A^- diagonal */
    const double h = mu / 2.0;
    double A[16] = {
        d,   h,    e,     0.0,
        -h,  d,    0.0,   e,
        -E,  0.0,  E + d, h,
        0.0, -E,   -h,    E + d,
    };
    memcpy(a, A, sizeof(A));
}

/* ------------------------------------------------------------------ helpers */

static inline size_t ix_psi(int j, int m, int c, int N) { return ((size_t)j * N + m) * 4 + c; }

/* Incident flux on cell j for ordinate m at time moment tm (0 = k, 1 = k+1/2),
 * taken from the iterate `psi` (upwind closure, Eqs. for psi_{m,k,j+1/2}).
 * mu_m > 0: from cell j-1 corner R, or the left boundary at j = 0.
 * mu_m < 0: from cell j+1 corner L, or the right boundary at j = J-1.       */
static double incident(const oracle_problem *p, const double *mu, const double *psi, int j, int m, int tm)
{
    const int J = p->n_cells, N = p->n_ord, P = N / 2;
    const int cR = tm ? 3 : 1, cL = tm ? 2 : 0;
    if (mu[m] > 0.0) {
        if (j > 0) return psi[ix_psi(j - 1, m, cR, N)];
        if (p->bc_left == ORC_BC_REFLECT) return psi[ix_psi(0, N - 1 - m, cL, N)];
        if (p->bc_left == ORC_BC_INCIDENT && p->psi_bc_left) return p->psi_bc_left[(m - P) * 2 + tm];
        return 0.0;
    } else {
        if (j < J - 1) return psi[ix_psi(j + 1, m, cL, N)];
        if (p->bc_right == ORC_BC_REFLECT) return psi[ix_psi(J - 1, N - 1 - m, cR, N)];
        if (p->bc_right == ORC_BC_INCIDENT && p->psi_bc_right) return p->psi_bc_right[(P - 1 - m) * 2 + tm];
        return 0.0;
    }
}

/* -------------------------------------------------------------- OCI iteration */

typedef struct {
    double dx, st, ss;
    double *lu; /* (4N)^2 */
    int *piv;
    int singular;
} oci_material;

static int same_material(const oci_material *m, double dx, double st, double ss)
{
    return m->dx == dx && m->st == st && m->ss == ss;
}

/* Assemble A - S for one cell (block-diagonal A of the per-ordinate A_m, and
 * S_{(m,i),(n,i)} = dx Sigma_s w_n / 4 on the same component i). */
static void assemble_cell_matrix(int N, const double *mu, const double *w, double dx, double st, double ss,
                                 double v, double dt, double *M)
{
    const int n4 = 4 * N;
    memset(M, 0, sizeof(double) * (size_t)n4 * n4);
    double a[16];
    for (int m = 0; m < N; ++m) {
        assemble_A_m(mu[m], dx, st, v, dt, a);
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) M[(size_t)(4 * m + r) * n4 + 4 * m + c] += a[r * 4 + c];
    }
    const double s = dx * ss / 4.0;
    for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n)
            for (int i = 0; i < 4; ++i) M[(size_t)(4 * m + i) * n4 + 4 * n + i] -= s * w[n];
}

/* Find-or-add the material of cell j; returns its index.  The table holds at
 * most n_cells entries. */
static int material_index(oci_material *tab, int *ntab, double dx, double st, double ss)
{
    for (int i = *ntab - 1; i >= 0; --i)
        if (same_material(&tab[i], dx, st, ss)) return i;
    tab[*ntab].dx = dx;
    tab[*ntab].st = st;
    tab[*ntab].ss = ss;
    tab[*ntab].lu = NULL;
    tab[*ntab].piv = NULL;
    tab[*ntab].singular = 0;
    return (*ntab)++;
}

/* One OCI iteration.  psi_in: iterate l [J][N][4]; psi_edge: psi_{k-1/2} [J][N][2].
 * Writes psi_out (iterate l+1) and phi_out [J][4] = sum_n w_n psi_n.
 * Returns 0, 2 on allocation failure, 3 on a singular cell matrix. */
int oracle_oci_iteration(const oracle_problem *p, const double *psi_edge, const double *psi_in,
                         double *psi_out, double *phi_out)
{
    const int J = p->n_cells, N = p->n_ord, n4 = 4 * N;
    double *mu = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N);
    int *mat_of = malloc(sizeof(int) * (size_t)J);
    oci_material *tab = malloc(sizeof(oci_material) * (size_t)J);
    if (!mu || !w || !mat_of || !tab) { free(mu); free(w); free(mat_of); free(tab); return 2; }
    oracle_gauss_legendre(N, mu, w);
    int ntab = 0, last = -1;
    for (int j = 0; j < J; ++j) {
        if (last >= 0 && same_material(&tab[last], p->dx[j], p->sigma_t[j], p->sigma_s[j])) {
            mat_of[j] = last;
            continue;
        }
        last = material_index(tab, &ntab, p->dx[j], p->sigma_t[j], p->sigma_s[j]);
        mat_of[j] = last;
    }
    int err = 0;
    for (int i = 0; i < ntab; ++i) {
        tab[i].lu = malloc(sizeof(double) * (size_t)n4 * n4);
        tab[i].piv = malloc(sizeof(int) * (size_t)n4);
        if (!tab[i].lu || !tab[i].piv) { err = 2; continue; }
        assemble_cell_matrix(N, mu, w, tab[i].dx, tab[i].st, tab[i].ss, p->v, p->dt, tab[i].lu);
        tab[i].singular = lu_factor(n4, tab[i].lu, tab[i].piv);
        if (tab[i].singular) err = 3;
    }
    if (!err) {
#pragma omp parallel
        {
            double *c = malloc(sizeof(double) * (size_t)n4);
#pragma omp for schedule(static)
            for (int j = 0; j < J; ++j) {
                if (!c) continue;
                const double dx = p->dx[j];
                const double e = dx / (2.0 * p->v * p->dt);
                const double *Q = p->q + (size_t)j * 4;
                for (int m = 0; m < N; ++m) {
                    const double pL = psi_edge[((size_t)j * N + m) * 2 + 0];
                    const double pR = psi_edge[((size_t)j * N + m) * 2 + 1];
                    const double ink = incident(p, mu, psi_in, j, m, 0);
                    const double inh = incident(p, mu, psi_in, j, m, 1);
                    double *cm = c + 4 * m;
                    if (mu[m] > 0.0) { /* c^+ as printed */
                        cm[0] = dx / 4.0 * Q[0] + e * pL + mu[m] * ink;
                        cm[1] = dx / 4.0 * Q[1] + e * pR;
                        cm[2] = dx / 4.0 * Q[2] + mu[m] * inh;
                        cm[3] = dx / 4.0 * Q[3];
                    } else {           /* c^- as printed */
                        cm[0] = dx / 4.0 * Q[0] + e * pL;
                        cm[1] = dx / 4.0 * Q[1] + e * pR - mu[m] * ink;
                        cm[2] = dx / 4.0 * Q[2];
                        cm[3] = dx / 4.0 * Q[3] - mu[m] * inh;
                    }
                }
                const oci_material *mt = &tab[mat_of[j]];
                lu_solve(n4, mt->lu, mt->piv, c);
                memcpy(psi_out + ix_psi(j, 0, 0, N), c, sizeof(double) * (size_t)n4);
            }
            free(c);
        }
        for (int j = 0; j < J; ++j)
            for (int i = 0; i < 4; ++i) {
                double s = 0.0;
                for (int n = 0; n < N; ++n) s += w[n] * psi_out[ix_psi(j, n, i, N)];
                phi_out[(size_t)j * 4 + i] = s;
            }
    }
    for (int i = 0; i < ntab; ++i) { free(tab[i].lu); free(tab[i].piv); }
    free(tab); free(mat_of); free(mu); free(w);
    return err;
}

/* --------------------------------------------------------------- SI iteration */

/* Solve one cell of the SI sweep for ordinate m given the incident fluxes. */
static int si_cell(const oracle_problem *p, double mu, int j, const double *phi_lag, const double *pedge,
                   double ink, double inh, double *out4)
{
    const double dx = p->dx[j], st = p->sigma_t[j], ss = p->sigma_s[j];
    const double e = dx / (2.0 * p->v * p->dt);
    const double *Q = p->q + (size_t)j * 4;
    const double *ph = phi_lag + (size_t)j * 4;
    double a[16], b[4];
    int piv[4];
    assemble_A_m(mu, dx, st, p->v, p->dt, a);
    if (mu > 0.0) { /* b^+ as printed */
        b[0] = dx / 4.0 * (ss * ph[0] + Q[0]) + e * pedge[0] + mu * ink;
        b[1] = dx / 4.0 * (ss * ph[1] + Q[1]) + e * pedge[1];
        b[2] = dx / 4.0 * (ss * ph[2] + Q[2]) + mu * inh;
        b[3] = dx / 4.0 * (ss * ph[3] + Q[3]);
    } else {        /* b^- as printed */
        b[0] = dx / 4.0 * (ss * ph[0] + Q[0]) + e * pedge[0];
        b[1] = dx / 4.0 * (ss * ph[1] + Q[1]) + e * pedge[1] - mu * ink;
        b[2] = dx / 4.0 * (ss * ph[2] + Q[2]);
        b[3] = dx / 4.0 * (ss * ph[3] + Q[3]) - mu * inh;
    }
    if (lu_factor(4, a, piv)) return 3;
    lu_solve(4, a, piv, b);
    memcpy(out4, b, sizeof(b));
    return 0;
}

/* One SI iteration.  phi_in: phi^(l) [J][4] (lagged scattering source);
 * psi_in: iterate l [J][N][4] (only used for a reflecting right face, which is
 * lagged); writes psi_out (iterate l+1) and phi_out. */
int oracle_si_iteration(const oracle_problem *p, const double *psi_edge, const double *phi_in,
                        const double *psi_in, double *psi_out, double *phi_out)
{
    const int J = p->n_cells, N = p->n_ord, P = N / 2;
    double *mu = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N);
    if (!mu || !w) { free(mu); free(w); return 2; }
    oracle_gauss_legendre(N, mu, w);
    int err = 0;
    /* mu < 0 ordinates first, sweeping right to left */
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int m = 0; m < P; ++m) {
        double ink, inh;
        if (p->bc_right == ORC_BC_REFLECT) { /* lagged: mirror mu>0 outgoing R corner of the last cell, iterate l */
            ink = psi_in[ix_psi(J - 1, N - 1 - m, 1, N)];
            inh = psi_in[ix_psi(J - 1, N - 1 - m, 3, N)];
        } else if (p->bc_right == ORC_BC_INCIDENT && p->psi_bc_right) {
            ink = p->psi_bc_right[(P - 1 - m) * 2 + 0];
            inh = p->psi_bc_right[(P - 1 - m) * 2 + 1];
        } else { ink = 0.0; inh = 0.0; }
        for (int j = J - 1; j >= 0; --j) {
            double *o = psi_out + ix_psi(j, m, 0, N);
            err |= si_cell(p, mu[m], j, phi_in, psi_edge + ((size_t)j * N + m) * 2, ink, inh, o);
            ink = o[0]; /* outgoing through the left face: corner L */
            inh = o[2];
        }
    }
    /* then mu > 0 ordinates, sweeping left to right */
#pragma omp parallel for schedule(static) reduction(| : err)
    for (int m = P; m < N; ++m) {
        double ink, inh;
        if (p->bc_left == ORC_BC_REFLECT) { /* current sweep's mirror outgoing L corner of cell 0 */
            ink = psi_out[ix_psi(0, N - 1 - m, 0, N)];
            inh = psi_out[ix_psi(0, N - 1 - m, 2, N)];
        } else if (p->bc_left == ORC_BC_INCIDENT && p->psi_bc_left) {
            ink = p->psi_bc_left[(m - P) * 2 + 0];
            inh = p->psi_bc_left[(m - P) * 2 + 1];
        } else { ink = 0.0; inh = 0.0; }
        for (int j = 0; j < J; ++j) {
            double *o = psi_out + ix_psi(j, m, 0, N);
            err |= si_cell(p, mu[m], j, phi_in, psi_edge + ((size_t)j * N + m) * 2, ink, inh, o);
            ink = o[1]; /* outgoing through the right face: corner R */
            inh = o[3];
        }
    }
    for (int j = 0; j < J; ++j)
        for (int i = 0; i < 4; ++i) {
            double s = 0.0;
            for (int n = 0; n < N; ++n) s += w[n] * psi_out[ix_psi(j, n, i, N)];
            phi_out[(size_t)j * 4 + i] = s;
        }
    free(mu); free(w);
    return err;
}

/* ------------------------------------------------------------ time-step driver */

static double rel_change(int n, const double *a_new, const double *a_old)
{
    double d2 = 0.0, n2 = 0.0;
    for (int i = 0; i < n; ++i) {
        double d = a_new[i] - a_old[i];
        d2 += d * d;
        n2 += a_new[i] * a_new[i];
    }
    if (n2 == 0.0) return d2 == 0.0 ? 0.0 : INFINITY;
    return sqrt(d2 / n2);
}

/*
 * March n_steps time steps with OCI (method 0) or SI (method 1).
 * psi_edge [J][N][2]: on entry psi at the start (psi_{m,0}); on exit the last
 *   committed time-edge flux.
 * phi_steps [n_steps][J][4] (may be NULL): converged phi of each step.
 * iters/resid [n_steps] (may be NULL): iterations used and the last relative change.
 * A step that does not reach tol within max_iter is committed only when
 * commit_unconverged != 0; otherwise the run stops there and returns 4.
 * n_threads <= 0 keeps the OpenMP default.
 */
int oracle_run(const oracle_problem *p, int32_t method, int32_t n_steps, double tol, int32_t max_iter,
               int32_t commit_unconverged, double *psi_edge, double *phi_steps, int32_t *iters,
               double *resid, int32_t n_threads)
{
    const int J = p->n_cells, N = p->n_ord;
    if (J < 1 || N < 2 || (N & 1) || max_iter < 1) return 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const size_t npsi = (size_t)J * N * 4;
    double *psiA = malloc(sizeof(double) * npsi), *psiB = malloc(sizeof(double) * npsi);
    double *phiA = malloc(sizeof(double) * (size_t)J * 4), *phiB = malloc(sizeof(double) * (size_t)J * 4);
    double *mu = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N);
    if (!psiA || !psiB || !phiA || !phiB || !mu || !w) {
        free(psiA); free(psiB); free(phiA); free(phiB); free(mu); free(w);
        return 2;
    }
    oracle_gauss_legendre(N, mu, w);
    int status = 0;
    for (int step = 0; step < n_steps && status == 0; ++step) {
        /* Psi^(0): both time moments equal psi_{k-1/2}; phi^(0) = sum_n w_n Psi^(0) */
        for (int j = 0; j < J; ++j)
            for (int m = 0; m < N; ++m) {
                const double L = psi_edge[((size_t)j * N + m) * 2], R = psi_edge[((size_t)j * N + m) * 2 + 1];
                double *o = psiA + ix_psi(j, m, 0, N);
                o[0] = L; o[1] = R; o[2] = L; o[3] = R;
            }
        for (int j = 0; j < J; ++j)
            for (int i = 0; i < 4; ++i) {
                double s = 0.0;
                for (int n = 0; n < N; ++n) s += w[n] * psiA[ix_psi(j, n, i, N)];
                phiA[(size_t)j * 4 + i] = s;
            }
        double *pc = psiA, *pn = psiB, *fc = phiA, *fn = phiB;
        int it = 0, conv = 0;
        double d = INFINITY;
        while (it < max_iter) {
            int e = method == ORC_OCI ? oracle_oci_iteration(p, psi_edge, pc, pn, fn)
                                      : oracle_si_iteration(p, psi_edge, fc, pc, pn, fn);
            if (e) { status = e; break; }
            ++it;
            d = rel_change(J * 4, fn, fc);
            double *t = pc; pc = pn; pn = t;
            t = fc; fc = fn; fn = t;
            if (!(d == d)) { status = 5; break; } /* NaN */
            if (d < tol) { conv = 1; break; }
        }
        if (iters) iters[step] = it;
        if (resid) resid[step] = d;
        if (status) break;
        if (!conv && !commit_unconverged) { status = 4; break; }
        for (int j = 0; j < J; ++j)
            for (int m = 0; m < N; ++m) {
                psi_edge[((size_t)j * N + m) * 2 + 0] = pc[ix_psi(j, m, 2, N)];
                psi_edge[((size_t)j * N + m) * 2 + 1] = pc[ix_psi(j, m, 3, N)];
            }
        if (phi_steps) memcpy(phi_steps + (size_t)step * J * 4, fc, sizeof(double) * (size_t)J * 4);
    }
    free(psiA); free(psiB); free(phiA); free(phiB); free(mu); free(w);
    return status;
}

/* ------------------------------------------------------ backward Euler (BE) */

/* SCB block of ordinate mu with total cross section sig_hat: the k-rows of the
 * printed A^+/A^- with 1/(v dt) = 0 (steady state) and Sigma -> Sigma_hat. */
static void assemble_B_m(double mu, double dx, double sig_hat, double *b)
{
    double a[16];
    assemble_A_m(mu, dx, sig_hat, INFINITY, 1.0, a);
    b[0] = a[0]; b[1] = a[1];
    b[2] = a[4]; b[3] = a[5];
}

static inline size_t ix_be(int j, int m, int c, int N) { return ((size_t)j * N + m) * 2 + c; }

/* Incident flux of ordinate m on cell j from the BE iterate psi [J][N][2]. */
static double be_incident(const oracle_problem *p, const double *mu, const double *psi, int j, int m)
{
    const int J = p->n_cells, N = p->n_ord, P = N / 2;
    if (mu[m] > 0.0) {
        if (j > 0) return psi[ix_be(j - 1, m, 1, N)];
        if (p->bc_left == ORC_BC_REFLECT) return psi[ix_be(0, N - 1 - m, 0, N)];
        if (p->bc_left == ORC_BC_INCIDENT && p->psi_bc_left) return p->psi_bc_left[(m - P) * 2 + 1];
        return 0.0;
    } else {
        if (j < J - 1) return psi[ix_be(j + 1, m, 0, N)];
        if (p->bc_right == ORC_BC_REFLECT) return psi[ix_be(J - 1, N - 1 - m, 1, N)];
        if (p->bc_right == ORC_BC_INCIDENT && p->psi_bc_right) return p->psi_bc_right[(P - 1 - m) * 2 + 1];
        return 0.0;
    }
}

/* Fixed part of the BE right-hand side of ordinate m in cell j plus the
 * incident term: (dx/4) Q_{k+1/2} + e psi^{n-1} (e = dx/(2 v dt), the
 * half-cell integral of psi^{n-1}/(v dt)) + |mu| psi_in in the upstream corner. */
static void be_rhs(const oracle_problem *p, double mu, int j, const double *pprev, double in, double *c2)
{
    const double dx = p->dx[j];
    const double e = dx / (2.0 * p->v * p->dt);
    const double *Q = p->q + (size_t)j * 4;
    c2[0] = dx / 4.0 * Q[2] + e * pprev[0];
    c2[1] = dx / 4.0 * Q[3] + e * pprev[1];
    if (mu > 0.0) c2[0] += mu * in;
    else c2[1] -= mu * in;
}

/* One BE OCI iteration: per cell the dense 2N x 2N system (B - S) psi = c,
 * LU with partial pivoting per distinct material.  psi_prev [J][N][2] is
 * psi^{n-1}; psi_in the iterate l; writes psi_out and phi_out [J][2]. */
int oracle_be_oci_iteration(const oracle_problem *p, const double *psi_prev, const double *psi_in,
                            double *psi_out, double *phi_out)
{
    const int J = p->n_cells, N = p->n_ord, n2 = 2 * N;
    double *mu = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N);
    double *M = malloc(sizeof(double) * (size_t)n2 * n2);
    int *piv = malloc(sizeof(int) * (size_t)n2);
    double *c = malloc(sizeof(double) * (size_t)n2);
    if (!mu || !w || !M || !piv || !c) { free(mu); free(w); free(M); free(piv); free(c); return 2; }
    oracle_gauss_legendre(N, mu, w);
    int err = 0;
    double cdx = NAN, cst = NAN, css = NAN;
    for (int j = 0; j < J && !err; ++j) {
        const double dx = p->dx[j], st = p->sigma_t[j], ss = p->sigma_s[j];
        if (!(dx == cdx && st == cst && ss == css)) { /* factorise once per run of one material */
            const double sig_hat = st + 1.0 / (p->v * p->dt);
            memset(M, 0, sizeof(double) * (size_t)n2 * n2);
            double b[4];
            for (int m = 0; m < N; ++m) {
                assemble_B_m(mu[m], dx, sig_hat, b);
                for (int r = 0; r < 2; ++r)
                    for (int q = 0; q < 2; ++q) M[(size_t)(2 * m + r) * n2 + 2 * m + q] += b[r * 2 + q];
            }
            const double s = dx * ss / 4.0;
            for (int m = 0; m < N; ++m)
                for (int n = 0; n < N; ++n)
                    for (int i = 0; i < 2; ++i) M[(size_t)(2 * m + i) * n2 + 2 * n + i] -= s * w[n];
            if (lu_factor(n2, M, piv)) { err = 3; break; }
            cdx = dx; cst = st; css = ss;
        }
        for (int m = 0; m < N; ++m)
            be_rhs(p, mu[m], j, psi_prev + ix_be(j, m, 0, N), be_incident(p, mu, psi_in, j, m), c + 2 * m);
        lu_solve(n2, M, piv, c);
        memcpy(psi_out + ix_be(j, 0, 0, N), c, sizeof(double) * (size_t)n2);
    }
    if (!err)
        for (int j = 0; j < J; ++j)
            for (int i = 0; i < 2; ++i) {
                double sum = 0.0;
                for (int n = 0; n < N; ++n) sum += w[n] * psi_out[ix_be(j, n, i, N)];
                phi_out[(size_t)j * 2 + i] = sum;
            }
    free(mu); free(w); free(M); free(piv); free(c);
    return err;
}

/* One BE SI iteration: per ordinate a sweep in the direction of travel
 * (mu < 0 first), each cell's 2x2 SCB block solved with the lagged scalar
 * flux phi_in [J][2] in the source. */
int oracle_be_si_iteration(const oracle_problem *p, const double *psi_prev, const double *phi_in,
                           const double *psi_in, double *psi_out, double *phi_out)
{
    const int J = p->n_cells, N = p->n_ord, P = N / 2;
    double *mu = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N);
    if (!mu || !w) { free(mu); free(w); return 2; }
    oracle_gauss_legendre(N, mu, w);
    int err = 0;
    for (int pass = 0; pass < 2 && !err; ++pass) {
        const int m0 = pass == 0 ? 0 : P, m1 = pass == 0 ? P : N;
        for (int m = m0; m < m1; ++m) {
            double in;
            if (mu[m] < 0.0) {
                if (p->bc_right == ORC_BC_REFLECT) in = psi_in[ix_be(J - 1, N - 1 - m, 1, N)];  /* lagged */
                else if (p->bc_right == ORC_BC_INCIDENT && p->psi_bc_right) in = p->psi_bc_right[(P - 1 - m) * 2 + 1];
                else in = 0.0;
            } else {
                if (p->bc_left == ORC_BC_REFLECT) in = psi_out[ix_be(0, N - 1 - m, 0, N)];  /* this sweep */
                else if (p->bc_left == ORC_BC_INCIDENT && p->psi_bc_left) in = p->psi_bc_left[(m - P) * 2 + 1];
                else in = 0.0;
            }
            for (int t = 0; t < J; ++t) {
                const int j = mu[m] > 0.0 ? t : J - 1 - t;
                const double dx = p->dx[j], st = p->sigma_t[j], ss = p->sigma_s[j];
                double b[4], c2[2];
                int piv[2];
                assemble_B_m(mu[m], dx, st + 1.0 / (p->v * p->dt), b);
                be_rhs(p, mu[m], j, psi_prev + ix_be(j, m, 0, N), in, c2);
                c2[0] += dx * ss / 4.0 * phi_in[(size_t)j * 2 + 0];
                c2[1] += dx * ss / 4.0 * phi_in[(size_t)j * 2 + 1];
                if (lu_factor(2, b, piv)) { err = 3; break; }
                lu_solve(2, b, piv, c2);
                psi_out[ix_be(j, m, 0, N)] = c2[0];
                psi_out[ix_be(j, m, 1, N)] = c2[1];
                in = mu[m] > 0.0 ? c2[1] : c2[0];  /* outgoing corner */
            }
        }
    }
    if (!err)
        for (int j = 0; j < J; ++j)
            for (int i = 0; i < 2; ++i) {
                double sum = 0.0;
                for (int n = 0; n < N; ++n) sum += w[n] * psi_out[ix_be(j, n, i, N)];
                phi_out[(size_t)j * 2 + i] = sum;
            }
    free(mu); free(w);
    return err;
}

/* March n_steps BE steps (method 0 OCI, 1 SI).  psi [J][N][2]: on entry
 * psi^0, on exit the last committed step's flux; phi_steps [n_steps][J][2];
 * same controls and return codes as oracle_run.  The initial iterate of a
 * step is psi^{n-1}. */
int oracle_be_run(const oracle_problem *p, int32_t method, int32_t n_steps, double tol, int32_t max_iter,
                  int32_t commit_unconverged, double *psi, double *phi_steps, int32_t *iters, double *resid,
                  int32_t n_threads)
{
    const int J = p->n_cells, N = p->n_ord;
    if (J < 1 || N < 2 || (N & 1) || max_iter < 1) return 1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const size_t npsi = (size_t)J * N * 2;
    double *pa = malloc(sizeof(double) * npsi), *pb = malloc(sizeof(double) * npsi);
    double *fa = malloc(sizeof(double) * (size_t)J * 2), *fb = malloc(sizeof(double) * (size_t)J * 2);
    double *mu = malloc(sizeof(double) * N), *w = malloc(sizeof(double) * N);
    if (!pa || !pb || !fa || !fb || !mu || !w) {
        free(pa); free(pb); free(fa); free(fb); free(mu); free(w);
        return 2;
    }
    oracle_gauss_legendre(N, mu, w);
    int status = 0;
    for (int step = 0; step < n_steps && status == 0; ++step) {
        memcpy(pa, psi, sizeof(double) * npsi);
        for (int j = 0; j < J; ++j)
            for (int i = 0; i < 2; ++i) {
                double sum = 0.0;
                for (int n = 0; n < N; ++n) sum += w[n] * pa[ix_be(j, n, i, N)];
                fa[(size_t)j * 2 + i] = sum;
            }
        double *pc = pa, *pn = pb, *fc = fa, *fn = fb;
        int it = 0, conv = 0;
        double d = INFINITY;
        while (it < max_iter) {
            int e = method == ORC_OCI ? oracle_be_oci_iteration(p, psi, pc, pn, fn)
                                      : oracle_be_si_iteration(p, psi, fc, pc, pn, fn);
            if (e) { status = e; break; }
            ++it;
            d = rel_change(J * 2, fn, fc);
            double *t = pc; pc = pn; pn = t;
            t = fc; fc = fn; fn = t;
            if (!(d == d)) { status = 5; break; }
            if (d < tol) { conv = 1; break; }
        }
        if (iters) iters[step] = it;
        if (resid) resid[step] = d;
        if (status) break;
        if (!conv && !commit_unconverged) { status = 4; break; }
        memcpy(psi, pc, sizeof(double) * npsi);
        if (phi_steps) memcpy(phi_steps + (size_t)step * J * 2, fc, sizeof(double) * (size_t)J * 2);
    }
    free(pa); free(pb); free(fa); free(fb); free(mu); free(w);
    return status;
}

/* Threads the OpenMP runtime will use (1 without OpenMP). */
int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
