/*
 * chhs_oracle.c -- plain, slow, double-precision CPU oracle for one time step
 * of the second-order convex-splitting scheme for Cahn-Hilliard-Hele-Shaw
 * (Chen, Feng, Liu, Wang, Wise; arXiv:1611.02967).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library and never serves a product call.
 *
 * What it computes (Section 2, Eqs. 2.4-2.7): given phi^m and phi^{m-1} on a
 * cell-centred grid with homogeneous Neumann boundaries (Appendix A), find
 * (phi^{m+1}, mu^{m+1/2}, p^{m+1/2}) solving
 *
 *   N1(u) = phi - s div_h(M(A_h phi*) grad_h mu) - s div_h(A_h phi* grad_h p) = phi^m
 *   N2(u) = mu - chi(phi, phi^m) + (3/4) eps^2 Lap_h phi
 *                                     = -phi* - (1/4) eps^2 Lap_h phi^{m-1}
 *   N3(u) = -Lap_h p - gamma div_h(A_h phi* grad_h mu)                = 0
 *
 * with phi* = 3/2 phi^m - 1/2 phi^{m-1}, chi(a,b) = (a^2+b^2)(a+b)/4 and
 * M(x) = 1 + gamma x^2 (Eq. 2.4 and the definition before Eq. 2.5).  This is
 * Eq. 2.5-2.7 with every term moved to the left except the known data.
 *
 * How it solves it: the paper names FAS nonlinear multigrid with V-cycles,
 * nu1 = nu2 = 2 smoothing sweeps, tolerance 1e-10 and a 2x2 coarsest grid
 * (Section 5 preamble) and omits the rest.  The readings taken here:
 *   - smoother: lexicographic (x fastest) nonlinear Gauss-Seidel; at each cell
 *     one Newton step on the cell's own (phi_c, mu_c, p_c) with the
 *     neighbours frozen, done as a 2x2 Newton step on (phi_c, mu_c) after
 *     eliminating the cell's own pressure equation, then p_c from N3;
 *   - restriction: mean of the 2^d children; prolongation: piecewise constant;
 *   - coarse operators: the same equations rediscretised at 2h, with phi* and
 *     phi^m restricted by the same mean;
 *   - FAS coarse right-hand side f_c = R(f - N(u)) + N_c(R u);
 *   - coarsest grid: the smoother repeated until its residual stops falling;
 *   - pressure gauge: mean(p) = 0 after every V-cycle (p is unique only up to
 *     a constant under pure Neumann conditions);
 *   - stopping norm: ||r|| = sqrt( (1/N) sum_c r_phi^2 + r_mu^2 + (s r_p)^2 ),
 *     the cell-average of the three residuals (r_p scaled by s because the
 *     pressure enters N1 multiplied by s).
 * Any convergent smoother reaches the same answer: the step's solution is
 * unique (Theorem 2.1), so these choices move iterates, not the result.
 *
 * Grid functions are stored x fastest, then y, then z, interior cells only;
 * the Neumann ghost values of Eq. A.1-A.3 (ghost = mirror of its neighbour)
 * make every boundary-face difference zero, so boundary faces carry no flux
 * and are simply skipped in the sums below.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_NOT_CONVERGED 1
#define ORACLE_DIVERGED 2
#define ORACLE_BAD_ARG 3
#define ORACLE_OOM 4

typedef struct {
    int dim;
    int n[3];
    int ncell;
    double h;
    /* unknowns */
    double *phi, *mu, *p;
    /* FAS right-hand sides */
    double *fphi, *fmu, *fp;
    /* frozen coefficients: phi^m and phi* on this level */
    double *phim, *phis;
    /* residual and the restricted iterate kept for the FAS correction */
    double *rphi, *rmu, *rp;
    double *phi0, *mu0, *p0;
} level_t;

typedef struct {
    double eps, gamma, s;
    int nu1, nu2;
} params_t;

/* ---------------------------------------------------------------- helpers */

/* Neumaier-compensated running sum, so that sums over 10^6 cells keep full
 * double precision independent of the cell count. */
typedef struct { double sum, comp; } ksum_t;
static void kadd(ksum_t* k, double v) {
    double t = k->sum + v;
    if (fabs(k->sum) >= fabs(v)) k->comp += (k->sum - t) + v;
    else k->comp += (v - t) + k->sum;
    k->sum = t;
}
static double kval(const ksum_t* k) { return k->sum + k->comp; }

/* chi(a, b) = (a^2 + b^2)(a + b)/4  (Eq. 2.4) and its derivative in a. */
static double chi(double a, double b) { return 0.25 * (a * a + b * b) * (a + b); }
static double dchi_da(double a, double b) { return 0.25 * (3.0 * a * a + 2.0 * a * b + b * b); }

/* Collect the interior neighbours of cell c.  A neighbour across a boundary
 * face is a Neumann ghost equal to c itself, whose differences vanish, so it
 * is left out.  Returns the count (n_c). */
static int neighbours(const level_t* L, int c, int nb[6]) {
    int nx = L->n[0], ny = L->n[1], nz = L->n[2];
    int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    int m = 0;
    if (i > 0) nb[m++] = c - 1;
    if (i < nx - 1) nb[m++] = c + 1;
    if (j > 0) nb[m++] = c - nx;
    if (j < ny - 1) nb[m++] = c + nx;
    if (L->dim == 3) {
        if (k > 0) nb[m++] = c - nx * ny;
        if (k < nz - 1) nb[m++] = c + nx * ny;
    }
    return m;
}

/* The three equations at cell c, written with face sums:
 *   div_h(kappa grad_h v)_c = (1/h^2) sum_{faces f of c} kappa_f (v_nb - v_c)
 * which is d_x(kappa D_x v) + d_y(...) (+ d_z(...)) from Appendix A.2 with
 * zero flux on boundary faces. */
static void apply_N(const level_t* L, const params_t* P, int c, double* n1, double* n2, double* n3) {
    int nb[6];
    int m = neighbours(L, c, nb);
    double ih2 = 1.0 / (L->h * L->h);
    double div_Mgmu = 0.0, div_agp = 0.0, div_agmu = 0.0, lap_phi = 0.0, lap_p = 0.0;
    for (int q = 0; q < m; ++q) {
        int e = nb[q];
        double af = 0.5 * (L->phis[c] + L->phis[e]);  /* A_h phi* on the face */
        double Mf = 1.0 + P->gamma * af * af;           /* M(A_h phi*) */
        double dmu = L->mu[e] - L->mu[c];
        double dp = L->p[e] - L->p[c];
        div_Mgmu += Mf * dmu;
        div_agp += af * dp;
        div_agmu += af * dmu;
        lap_phi += L->phi[e] - L->phi[c];
        lap_p += dp;
    }
    div_Mgmu *= ih2; div_agp *= ih2; div_agmu *= ih2; lap_phi *= ih2; lap_p *= ih2;
    *n1 = L->phi[c] - P->s * div_Mgmu - P->s * div_agp;
    *n2 = L->mu[c] - chi(L->phi[c], L->phim[c]) + 0.75 * P->eps * P->eps * lap_phi;
    *n3 = -lap_p - P->gamma * div_agmu;
}

/* r = f - N(u) on every cell; returns the stopping norm. */
static double residual(level_t* L, const params_t* P) {
    ksum_t acc = {0, 0};
    for (int c = 0; c < L->ncell; ++c) {
        double n1, n2, n3;
        apply_N(L, P, c, &n1, &n2, &n3);
        L->rphi[c] = L->fphi[c] - n1;
        L->rmu[c] = L->fmu[c] - n2;
        L->rp[c] = L->fp[c] - n3;
        double sp = P->s * L->rp[c];
        kadd(&acc, L->rphi[c] * L->rphi[c] + L->rmu[c] * L->rmu[c] + sp * sp);
    }
    return sqrt(kval(&acc) / L->ncell);
}

/* One smoothing sweep: lexicographic nonlinear Gauss-Seidel.  At each cell,
 * with every neighbour frozen, one Newton step on the cell's three equations
 * in its own unknowns (phi_c, mu_c, p_c).  The local Jacobian is
 *
 *        phi_c   mu_c   p_c
 *   N1 [   1      A      C  ]   A = s sum_f M_f / h^2,  C = s sum_f a_f / h^2
 *   N2 [  -B      1      0  ]   B = chi_a(phi_c, phi^m_c) + (3/4) eps^2 n_c / h^2
 *   N3 [   0      G      Dn ]   G = gamma sum_f a_f / h^2,  Dn = n_c / h^2
 *
 * (a_f = A_h phi* on face f, M_f = 1 + gamma a_f^2, n_c = interior faces).
 * Eliminating the cell's own pressure equation leaves a 2x2 Newton system in
 * (phi_c, mu_c) with A replaced by Ae = A - C G / Dn, and
 * Ae >= s n_c / h^2 > 0 because (sum a_f)^2 <= n_c sum a_f^2, so
 * det = 1 + Ae B >= 1 always.  The pressure then follows from N3. */
static void smooth(level_t* L, const params_t* P) {
    double h2 = L->h * L->h;
    double ee = 0.75 * P->eps * P->eps;
    for (int c = 0; c < L->ncell; ++c) {
        int nb[6];
        int m = neighbours(L, c, nb);
        double n1, n2, n3;
        apply_N(L, P, c, &n1, &n2, &n3);
        double R1 = L->fphi[c] - n1, R2 = L->fmu[c] - n2, R3 = L->fp[c] - n3;
        double sumM = 0.0, suma = 0.0;
        for (int q = 0; q < m; ++q) {
            double af = 0.5 * (L->phis[c] + L->phis[nb[q]]);
            sumM += 1.0 + P->gamma * af * af;
            suma += af;
        }
        double A = P->s * sumM / h2, C = P->s * suma / h2;
        double G = P->gamma * suma / h2, Dn = m / h2;
        double B = dchi_da(L->phi[c], L->phim[c]) + ee * m / h2;
        double Ae = A - C * G / Dn;
        double dphi = (R1 - Ae * R2 - (C / Dn) * R3) / (1.0 + Ae * B);
        double dmu = R2 + B * dphi;
        double dp = (R3 - G * dmu) / Dn;
        L->phi[c] += dphi;
        L->mu[c] += dmu;
        L->p[c] += dp;
    }
}

static void remove_mean(double* v, int n) {
    ksum_t acc = {0, 0};
    for (int c = 0; c < n; ++c) kadd(&acc, v[c]);
    double mean = kval(&acc) / n;
    for (int c = 0; c < n; ++c) v[c] -= mean;
}

/* Coarse cell of fine cell (i,j,k) is (i/2, j/2, k/2). */
static int parent(const level_t* F, const level_t* C, int c) {
    int nx = F->n[0], ny = F->n[1];
    int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    return (i / 2) + C->n[0] * ((j / 2) + C->n[1] * (k / 2));
}

/* R: coarse value = mean of its 2^d children. */
static void restrict_mean(const level_t* F, const level_t* C, const double* fine, double* coarse) {
    double w = F->dim == 2 ? 0.25 : 0.125;
    for (int c = 0; c < C->ncell; ++c) coarse[c] = 0.0;
    for (int c = 0; c < F->ncell; ++c) coarse[parent(F, C, c)] += w * fine[c];
}

/* ---------------------------------------------------------------- FAS */

/* The coarsest grid (the Section 5 preamble's "2x2", read as the coarsest
 * level): the smoother repeated until the residual has fallen by 1e-13 or
 * stops falling, then the pressure gauge. */
static void coarse_solve(level_t* L, const params_t* P) {
    double r0 = residual(L, P), prev = r0;
    for (int it = 0; it < 2000; ++it) {
        smooth(L, P);
        double r = residual(L, P);
        if (!(r > 1e-13 * r0) || r < 1e-300) break;
        if (it > 50 && r > 0.999 * prev) break; /* at the roundoff floor */
        prev = r;
    }
    remove_mean(L->p, L->ncell);
}

/* One FAS V(nu1, nu2)-cycle from level l (Section 5 preamble): pre-smooth,
 * restrict the iterate and the residual, coarse right-hand side
 * R r + N_c(R u), recurse, add the prolonged coarse correction, post-smooth. */
static void vcycle(level_t* lev, int l, int nlev, const params_t* P) {
    level_t* L = &lev[l];
    if (l == nlev - 1) {
        coarse_solve(L, P);
        return;
    }
    level_t* C = &lev[l + 1];
    for (int k = 0; k < P->nu1; ++k) smooth(L, P);
    residual(L, P);
    /* u_c = R u, kept as u_c^0 for the correction */
    restrict_mean(L, C, L->phi, C->phi);
    restrict_mean(L, C, L->mu, C->mu);
    restrict_mean(L, C, L->p, C->p);
    memcpy(C->phi0, C->phi, sizeof(double) * C->ncell);
    memcpy(C->mu0, C->mu, sizeof(double) * C->ncell);
    memcpy(C->p0, C->p, sizeof(double) * C->ncell);
    /* f_c = R r + N_c(R u) */
    restrict_mean(L, C, L->rphi, C->fphi);
    restrict_mean(L, C, L->rmu, C->fmu);
    restrict_mean(L, C, L->rp, C->fp);
    for (int c = 0; c < C->ncell; ++c) {
        double n1, n2, n3;
        apply_N(C, P, c, &n1, &n2, &n3);
        C->fphi[c] += n1;
        C->fmu[c] += n2;
        C->fp[c] += n3;
    }
    vcycle(lev, l + 1, nlev, P);
    /* u += P(u_c - u_c^0), P piecewise constant */
    for (int c = 0; c < L->ncell; ++c) {
        int q = parent(L, C, c);
        L->phi[c] += C->phi[q] - C->phi0[q];
        L->mu[c] += C->mu[q] - C->mu0[q];
        L->p[c] += C->p[q] - C->p0[q];
    }
    for (int k = 0; k < P->nu2; ++k) smooth(L, P);
}

/* ---------------------------------------------------------------- hierarchy */

static int count_levels(int dim, const int n[3], int coarsest) {
    int nl = 1;
    int m[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    for (;;) {
        int ok = 1;
        for (int a = 0; a < dim; ++a)
            if (m[a] % 2 != 0 || m[a] / 2 < coarsest) ok = 0;
        if (!ok) break;
        for (int a = 0; a < dim; ++a) m[a] /= 2;
        ++nl;
    }
    return nl;
}

static void free_levels(level_t* lev, int nlev) {
    if (!lev) return;
    for (int l = 0; l < nlev; ++l) {
        double** f[] = {&lev[l].phi, &lev[l].mu, &lev[l].p, &lev[l].fphi, &lev[l].fmu, &lev[l].fp,
                        &lev[l].phim, &lev[l].phis, &lev[l].rphi, &lev[l].rmu, &lev[l].rp,
                        &lev[l].phi0, &lev[l].mu0, &lev[l].p0};
        for (unsigned q = 0; q < sizeof(f) / sizeof(f[0]); ++q) free(*f[q]);
    }
    free(lev);
}

static level_t* make_levels(int dim, const int n[3], double h, int nlev) {
    level_t* lev = (level_t*)calloc(nlev, sizeof(level_t));
    if (!lev) return NULL;
    int m[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    double hl = h;
    for (int l = 0; l < nlev; ++l) {
        level_t* L = &lev[l];
        L->dim = dim;
        L->n[0] = m[0]; L->n[1] = m[1]; L->n[2] = m[2];
        L->ncell = m[0] * m[1] * m[2];
        L->h = hl;
        double** f[] = {&L->phi, &L->mu, &L->p, &L->fphi, &L->fmu, &L->fp, &L->phim, &L->phis,
                        &L->rphi, &L->rmu, &L->rp, &L->phi0, &L->mu0, &L->p0};
        for (unsigned q = 0; q < sizeof(f) / sizeof(f[0]); ++q) {
            *f[q] = (double*)calloc(L->ncell, sizeof(double));
            if (!*f[q]) { free_levels(lev, nlev); return NULL; }
        }
        for (int a = 0; a < dim; ++a) m[a] /= 2;
        hl *= 2.0;
    }
    return lev;
}

static int check_args(int dim, const int* n, double h, double eps, double gamma, double s) {
    if (dim != 2 && dim != 3) return 0;
    for (int a = 0; a < dim; ++a)
        if (n[a] < 2) return 0;
    if (!(h > 0) || !(eps > 0) || !(s > 0) || !(gamma >= 0)) return 0;
    return 1;
}

static void load_fine(level_t* L, const double* phim, const double* phimm1, double eps) {
    /* phi* = 3/2 phi^m - 1/2 phi^{m-1}  (Eq. 2.4) */
    for (int c = 0; c < L->ncell; ++c) {
        L->phim[c] = phim[c];
        L->phis[c] = 1.5 * phim[c] - 0.5 * phimm1[c];
    }
    /* f_phi = phi^m, f_mu = -phi* - (1/4) eps^2 Lap_h phi^{m-1}, f_p = 0 */
    double ih2 = 1.0 / (L->h * L->h);
    for (int c = 0; c < L->ncell; ++c) {
        int nb[6];
        int m = neighbours(L, c, nb);
        double lap = 0.0;
        for (int q = 0; q < m; ++q) lap += phimm1[nb[q]] - phimm1[c];
        lap *= ih2;
        L->fphi[c] = phim[c];
        L->fmu[c] = -L->phis[c] - 0.25 * eps * eps * lap;
        L->fp[c] = 0.0;
    }
}

/* ---------------------------------------------------------------- public */

int oracle_num_levels(int dim, const int* n, int coarsest) {
    int m[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    return count_levels(dim, m, coarsest);
}

/*
 * One time step.  phi, mu, p are in/out: on entry the initial guess, on exit
 * the solution (p with zero mean).  Returns ORACLE_OK when the stopping norm
 * reached tol, or when it stopped falling below 1e-12 (the double-precision
 * floor, used when tol is set below what the arithmetic can reach);
 * ORACLE_NOT_CONVERGED after max_v cycles; ORACLE_DIVERGED on a non-finite
 * or exploding residual.
 */
int oracle_step(int dim, const int* n, double h, double eps, double gamma, double s,
                const double* phim, const double* phimm1,
                double* phi, double* mu, double* p,
                int nu1, int nu2, int max_v, double tol, int coarsest,
                int* vcycles_out, double* resid_out) {
    if (!check_args(dim, n, h, eps, gamma, s)) return ORACLE_BAD_ARG;
    int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    int nlev = count_levels(dim, nn, coarsest < 1 ? 1 : coarsest);
    level_t* lev = make_levels(dim, nn, h, nlev);
    if (!lev) return ORACLE_OOM;
    params_t P = {eps, gamma, s, nu1, nu2};
    level_t* L = &lev[0];
    load_fine(L, phim, phimm1, eps);
    for (int l = 1; l < nlev; ++l) {
        restrict_mean(&lev[l - 1], &lev[l], lev[l - 1].phim, lev[l].phim);
        restrict_mean(&lev[l - 1], &lev[l], lev[l - 1].phis, lev[l].phis);
    }
    memcpy(L->phi, phi, sizeof(double) * L->ncell);
    memcpy(L->mu, mu, sizeof(double) * L->ncell);
    memcpy(L->p, p, sizeof(double) * L->ncell);

    double r = residual(L, &P), r0 = r;
    int v = 0, status = ORACLE_NOT_CONVERGED;
    if (r <= tol) status = ORACLE_OK;
    while (status == ORACLE_NOT_CONVERGED && v < max_v) {
        vcycle(lev, 0, nlev, &P);
        remove_mean(L->p, L->ncell);
        ++v;
        double rn = residual(L, &P);
        if (!isfinite(rn) || rn > 1e8 * (r0 + 1.0)) { r = rn; status = ORACLE_DIVERGED; break; }
        if (rn <= tol) status = ORACLE_OK;
        else if (rn < 1e-12 && rn > 0.5 * r) status = ORACLE_OK; /* roundoff floor */
        r = rn;
    }
    memcpy(phi, L->phi, sizeof(double) * L->ncell);
    memcpy(mu, L->mu, sizeof(double) * L->ncell);
    memcpy(p, L->p, sizeof(double) * L->ncell);
    if (vcycles_out) *vcycles_out = v;
    if (resid_out) *resid_out = r;
    free_levels(lev, nlev);
    return status;
}

/* r = f - N(u) on the fine grid for given (phi, mu, p); returns the norm. */
double oracle_residual(int dim, const int* n, double h, double eps, double gamma, double s,
                       const double* phim, const double* phimm1,
                       const double* phi, const double* mu, const double* p,
                       double* rphi, double* rmu, double* rp) {
    if (!check_args(dim, n, h, eps, gamma, s)) return -1.0;
    int nn[3] = {n[0], n[1], dim == 3 ? n[2] : 1};
    level_t* lev = make_levels(dim, nn, h, 1);
    if (!lev) return -1.0;
    params_t P = {eps, gamma, s, 0, 0};
    level_t* L = &lev[0];
    load_fine(L, phim, phimm1, eps);
    memcpy(L->phi, phi, sizeof(double) * L->ncell);
    memcpy(L->mu, mu, sizeof(double) * L->ncell);
    memcpy(L->p, p, sizeof(double) * L->ncell);
    double r = residual(L, &P);
    if (rphi) memcpy(rphi, L->rphi, sizeof(double) * L->ncell);
    if (rmu) memcpy(rmu, L->rmu, sizeof(double) * L->ncell);
    if (rp) memcpy(rp, L->rp, sizeof(double) * L->ncell);
    free_levels(lev, 1);
    return r;
}

/* Lap_h v = div_h grad_h v with Neumann ghosts (Appendix A.2). */
void oracle_laplacian(int dim, const int* n, double h, const double* v, double* out) {
    level_t L;
    memset(&L, 0, sizeof(L));
    L.dim = dim; L.n[0] = n[0]; L.n[1] = n[1]; L.n[2] = dim == 3 ? n[2] : 1;
    L.ncell = L.n[0] * L.n[1] * L.n[2];
    L.h = h;
    double ih2 = 1.0 / (h * h);
    for (int c = 0; c < L.ncell; ++c) {
        int nb[6];
        int m = neighbours(&L, c, nb);
        double acc = 0.0;
        for (int q = 0; q < m; ++q) acc += v[nb[q]] - v[c];
        out[c] = acc * ih2;
    }
}

/* (f, g) = h^d sum_c f_c g_c  (Appendix A.2, cell inner product) */
double oracle_inner(int dim, const int* n, double h, const double* f, const double* g) {
    int nc = n[0] * n[1] * (dim == 3 ? n[2] : 1);
    ksum_t acc = {0, 0};
    for (int c = 0; c < nc; ++c) kadd(&acc, f[c] * g[c]);
    return (dim == 2 ? h * h : h * h * h) * kval(&acc);
}

/* (grad_h f, grad_h g) = sum over axes of [D f, D g]: each interior face is
 * shared by two cells with weight 1/2 each, boundary faces carry D = 0, so it
 * is h^d times the sum over interior faces (Eq. A "inner product-def 2"). */
double oracle_grad_inner(int dim, const int* n, double h, const double* f, const double* g) {
    int nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
    ksum_t acc = {0, 0};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int c = i + nx * (j + ny * k);
                if (i + 1 < nx) kadd(&acc, ((f[c + 1] - f[c]) / h) * ((g[c + 1] - g[c]) / h));
                if (j + 1 < ny) kadd(&acc, ((f[c + nx] - f[c]) / h) * ((g[c + nx] - g[c]) / h));
                if (dim == 3 && k + 1 < nz)
                    kadd(&acc, ((f[c + nx * ny] - f[c]) / h) * ((g[c + nx * ny] - g[c]) / h));
            }
    return (dim == 2 ? h * h : h * h * h) * kval(&acc);
}

/* mass (phi, 1) = h^d sum phi  (Section 4, discrete mass conservation) */
double oracle_mass(int dim, const int* n, double h, const double* phi) {
    int nc = n[0] * n[1] * (dim == 3 ? n[2] : 1);
    ksum_t acc = {0, 0};
    for (int c = 0; c < nc; ++c) kadd(&acc, phi[c]);
    return (dim == 2 ? h * h : h * h * h) * kval(&acc);
}

/* E_h(phi) (Eq. 2.8) and F_h(phi, psi) (Eq. 2.9). */
void oracle_energy(int dim, const int* n, double h, double eps, const double* phi, const double* psi,
                   double* E_out, double* F_out) {
    int nc = n[0] * n[1] * (dim == 3 ? n[2] : 1);
    double hd = dim == 2 ? h * h : h * h * h;
    ksum_t q4 = {0, 0}, q2 = {0, 0}, dd = {0, 0};
    for (int c = 0; c < nc; ++c) {
        double v = phi[c];
        kadd(&q4, v * v * v * v);
        kadd(&q2, v * v);
        if (psi) kadd(&dd, (v - psi[c]) * (v - psi[c]));
    }
    double g2 = oracle_grad_inner(dim, n, h, phi, phi);
    double E = 0.25 * hd * kval(&q4) - 0.5 * hd * kval(&q2) + 0.5 * eps * eps * g2;
    if (E_out) *E_out = E;
    if (F_out && psi) {
        double* d = (double*)malloc(sizeof(double) * nc);
        if (!d) { *F_out = NAN; return; }
        for (int c = 0; c < nc; ++c) d[c] = phi[c] - psi[c];
        double gd = oracle_grad_inner(dim, n, h, d, d);
        free(d);
        *F_out = E + 0.25 * hd * kval(&dd) + 0.125 * eps * eps * gd;
    }
}

/*
 * Velocity of Eq. 2.3, u = -grad_h p - gamma A_h phi* grad_h mu, on interior
 * faces (boundary faces carry u.n = 0).  Writes ||u||_2^2 with the face inner
 * product of Appendix A.2, if div_out is given div_h u per cell, and if
 * faces_out is given the face values themselves: faces_out[a * N + c] is the
 * a-component on the face between cell c and its +a neighbour (0 where that
 * face is a boundary face).
 */
double oracle_velocity(int dim, const int* n, double h, double gamma,
                       const double* phis, const double* mu, const double* p, double* div_out,
                       double* faces_out) {
    int nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
    int nc = nx * ny * nz;
    if (div_out) for (int c = 0; c < nc; ++c) div_out[c] = 0.0;
    if (faces_out) for (int c = 0; c < dim * nc; ++c) faces_out[c] = 0.0;
    ksum_t acc = {0, 0};
    int stride[3] = {1, nx, nx * ny};
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int c = i + nx * (j + ny * k);
                int idx[3] = {i, j, k};
                for (int a = 0; a < dim; ++a) {
                    if (idx[a] + 1 >= n[a]) continue;
                    int e = c + stride[a];
                    double af = 0.5 * (phis[c] + phis[e]);
                    double u = -(p[e] - p[c]) / h - gamma * af * (mu[e] - mu[c]) / h;
                    kadd(&acc, u * u);
                    if (div_out) { div_out[c] += u / h; div_out[e] -= u / h; }
                    if (faces_out) faces_out[a * nc + c] = u;
                }
            }
    return (dim == 2 ? h * h : h * h * h) * kval(&acc);
}
