/*
 * fcd_oracle.c -- plain, slow, FP64 CPU oracle of the coupled time step of
 * arXiv 2410.11129 (phase-field MRT lattice Boltzmann + finite-difference
 * magnetic potential for a ferrofluid compound droplet).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the
 * benchmark's CPU-baseline leg. The CUDA library never links or calls it and
 * the two share no source, header or table.
 *
 * Every routine follows one equation of the paper, written as directly as
 * possible (dense 9x9 moment matrices, literal stencil sums, conjugate
 * gradients for the potential). Readings of passages the paper leaves open are
 * marked "reading:" where they are used.
 *
 * Threads: when built with OpenMP, the loops over nodes whose iterations write
 * disjoint outputs run row-parallel (orc_set_threads); sums stay serial, so the
 * results are bitwise the same for any thread count. The default is 1 thread.
 */
#include "fcd_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int n_threads = 1;

void orc_set_threads(int n) { n_threads = n > 0 ? n : 1; }

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

#define Q 9
#define PI 3.14159265358979323846

/* Eq. 20: D2Q9 velocities, rest, E, N, W, S, NE, NW, SW, SE. */
static const int EX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* Eq. 17: weights. */
static const double W[Q] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0; /* c_s^2 below Eq. 14 */

static double Mmat[Q * Q], Minv[Q * Q];
static int tables_ready = 0;

/* Orthogonal D2Q9 moment matrix of Lallemand & Luo (ref. [48] of the paper):
 * rows rho, e, eps, jx, qx, jy, qy, pxx, pxy as polynomials of e_alpha. */
static void build_tables(void) {
    if (tables_ready) return;
    for (int a = 0; a < Q; a++) {
        double ex = EX[a], ey = EY[a], e2 = ex * ex + ey * ey;
        double row[Q] = {1.0,
                         3.0 * e2 - 4.0,
                         (9.0 * e2 * e2 - 21.0 * e2 + 8.0) / 2.0,
                         ex,
                         (3.0 * e2 - 5.0) * ex,
                         ey,
                         (3.0 * e2 - 5.0) * ey,
                         ex * ex - ey * ey,
                         ex * ey};
        for (int k = 0; k < Q; k++) Mmat[k * Q + a] = row[k];
    }
    /* Gauss-Jordan inverse with partial pivoting. */
    double A[Q][2 * Q];
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < 2 * Q; j++)
            A[i][j] = j < Q ? Mmat[i * Q + j] : (j - Q == i ? 1.0 : 0.0);
    for (int c = 0; c < Q; c++) {
        int piv = c;
        for (int r = c + 1; r < Q; r++)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        for (int j = 0; j < 2 * Q; j++) {
            double t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t;
        }
        double d = A[c][c];
        for (int j = 0; j < 2 * Q; j++) A[c][j] /= d;
        for (int r = 0; r < Q; r++) {
            if (r == c) continue;
            double m = A[r][c];
            for (int j = 0; j < 2 * Q; j++) A[r][j] -= m * A[c][j];
        }
    }
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < Q; j++) Minv[i * Q + j] = A[i][Q + j];
    tables_ready = 1;
}

void orc_tables(double *w, int *ex, int *ey, double *M, double *Mi) {
    build_tables();
    for (int a = 0; a < Q; a++) { w[a] = W[a]; ex[a] = EX[a]; ey[a] = EY[a]; }
    memcpy(M, Mmat, sizeof Mmat);
    memcpy(Mi, Minv, sizeof Minv);
}

/* Dimensionless groups (Eqs. 14, 26, 27, 30, 40, 41) mapped to lattice units. */
void orc_derive(const orc_params *p, orc_derived *d) {
    memset(d, 0, sizeof *d);
    d->u_avg = 2.0 * p->u_max / 3.0; /* mean of the Poiseuille profile */
    double s23 = p->sigma23 > 0.0 ? p->sigma23 : p->rho[2] * p->nu[2] * d->u_avg / p->Ca;
    double s12 = s23 / p->s23_over_s12;
    double s13 = p->s13_over_s12 * s12;
    d->sigma[0][1] = d->sigma[1][0] = s12;
    d->sigma[0][2] = d->sigma[2][0] = s13;
    d->sigma[1][2] = d->sigma[2][1] = s23;
    d->gamma[0] = s12 + s13 - s23; /* Eq. 27 */
    d->gamma[1] = s12 + s23 - s13;
    d->gamma[2] = s13 + s23 - s12;
    d->gammaT = 3.0 / (1.0 / d->gamma[0] + 1.0 / d->gamma[1] + 1.0 / d->gamma[2]); /* Eq. 26 */
    for (int i = 0; i < 3; i++) d->tau[i] = p->nu[i] / CS2; /* Eq. 14, dt = 1 */
    d->tau_phi = p->mobility / CS2;                         /* Eq. 30 */
    d->mu0H0sq = 0.0;
    if (p->ferro_phase == 1 && p->chi[0] > 0.0)
        d->mu0H0sq = p->Bo_m * 2.0 * s12 / (p->chi[0] * p->r1); /* Eq. 41, core */
    else if (p->ferro_phase == 2 && p->chi[1] > 0.0)
        d->mu0H0sq = p->Bo_m * 2.0 * (s12 * p->r1 + s23 * p->r2) /
                     (p->chi[1] * (p->r2 * p->r2 - p->r1 * p->r1)); /* Eq. 41, shell */
    d->H0 = sqrt(d->mu0H0sq); /* mu0 = 1 in lattice units */
    /* reading: body force giving the Poiseuille centre-line speed u_max
     * between half-way walls a distance ny apart */
    d->G = 8.0 * p->rho[2] * p->nu[2] * p->u_max / ((double)p->ny * p->ny);
    if (p->open_x) d->G = 0.0; /* the open channel is driven by its inlet */
}

/* Eq. 18, with the quadratic u.u term over 2 c_s^2 (reading: the printed
 * equation drops the 2, which would break sum_a Gamma_a = 1). */
void orc_gamma(double ux, double uy, double *G9) {
    double uu = ux * ux + uy * uy;
    for (int a = 0; a < Q; a++) {
        double eu = EX[a] * ux + EY[a] * uy;
        G9[a] = W[a] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. 16. */
void orc_feq(double pstar, double ux, double uy, double *feq9) {
    double G9[Q];
    orc_gamma(ux, uy, G9);
    for (int a = 0; a < Q; a++) feq9[a] = pstar * W[a] + (G9[a] - W[a]);
}

/* M^-1 Lambda M h with Lambda of Eq. 13. reading: nine entries, all 1 but the
 * two stress moments pxx, pxy which relax with 1/(1/2 + tau). */
void orc_mrt_apply(const double *h9, double s_nu, double *out9) {
    build_tables();
    double lam[Q] = {1, 1, 1, 1, 1, 1, 1, s_nu, s_nu};
    double m[Q];
    for (int k = 0; k < Q; k++) {
        m[k] = 0.0;
        for (int a = 0; a < Q; a++) m[k] += Mmat[k * Q + a] * h9[a];
        m[k] *= lam[k];
    }
    for (int a = 0; a < Q; a++) {
        out9[a] = 0.0;
        for (int k = 0; k < Q; k++) out9[a] += Minv[a * Q + k] * m[k];
    }
}

/* Eq. 28. */
double orc_H(const orc_derived *d, double eta, const double *ph) {
    double p1 = ph[0], p2 = ph[1], p3 = ph[2];
    return d->sigma[0][1] * p1 * p1 * p2 * p2 + d->sigma[0][2] * p1 * p1 * p3 * p3 +
           d->sigma[1][2] * p2 * p2 * p3 * p3 +
           p1 * p2 * p3 * (d->gamma[0] * p1 + d->gamma[1] * p2 + d->gamma[2] * p3) +
           eta * p1 * p1 * p2 * p2 * p3 * p3;
}

/* Partial derivatives of Eq. 28, the three phi_i taken as independent. */
void orc_dH(const orc_derived *d, double eta, const double *ph, double *dH) {
    double p1 = ph[0], p2 = ph[1], p3 = ph[2];
    double s12 = d->sigma[0][1], s13 = d->sigma[0][2], s23 = d->sigma[1][2];
    double gp = d->gamma[0] * p1 + d->gamma[1] * p2 + d->gamma[2] * p3;
    double ppp = p1 * p2 * p3;
    dH[0] = 2.0 * s12 * p1 * p2 * p2 + 2.0 * s13 * p1 * p3 * p3 + p2 * p3 * gp +
            ppp * d->gamma[0] + 2.0 * eta * p1 * p2 * p2 * p3 * p3;
    dH[1] = 2.0 * s12 * p1 * p1 * p2 + 2.0 * s23 * p2 * p3 * p3 + p1 * p3 * gp +
            ppp * d->gamma[1] + 2.0 * eta * p1 * p1 * p2 * p3 * p3;
    dH[2] = 2.0 * s13 * p1 * p1 * p3 + 2.0 * s23 * p2 * p2 * p3 + p1 * p2 * gp +
            ppp * d->gamma[2] + 2.0 * eta * p1 * p1 * p2 * p2 * p3;
}

/* Eq. 25. reading: the Laplacian coefficient printed "gamma_t" is gamma_i. */
void orc_chem(const orc_derived *d, double eta, double xi, const double *ph,
              const double *lap, double *mu) {
    double dH[3];
    orc_dH(d, eta, ph, dH);
    for (int i = 0; i < 3; i++) {
        double s = 0.0;
        for (int j = 0; j < 3; j++)
            if (j != i) s += (dH[i] - dH[j]) / d->gamma[j];
        mu[i] = 4.0 * d->gammaT / xi * s - 0.75 * xi * d->gamma[i] * lap[i];
    }
}

/* Field access: x periodic, or mirrored at the inlet and outlet columns of an
 * open channel (reading: zero normal gradient there); y mirrored about the
 * half-way walls (reading: zero normal gradient of phi at the walls, i.e. a
 * 90 degree contact angle). */
static double at_mirror_x(const double *a, int nx, int ny, int x, int y, int open) {
    if (open) x = x < 0 ? 0 : (x >= nx ? nx - 1 : x);
    else x = ((x % nx) + nx) % nx;
    if (y < 0) y = 0;
    if (y >= ny) y = ny - 1;
    return a[(long)y * nx + x];
}

static double at_mirror(const double *a, int nx, int ny, int x, int y) {
    return at_mirror_x(a, nx, ny, x, y, 0);
}

/* psi' vanishes on the half-way walls (reading): odd reflection. */
static double at_odd(const double *a, int nx, int ny, int x, int y) {
    x = ((x % nx) + nx) % nx;
    if (y < 0) return -a[x];
    if (y >= ny) return -a[(long)(ny - 1) * nx + x];
    return a[(long)y * nx + x];
}

/* Eq. 34 (c = dx = 1). odd: psi' (periodic in x in both channel kinds,
 * reading); else phi-like fields (mirrored at open ends). */
static void grad_node_x(const double *a, int nx, int ny, int x, int y, int odd, int open,
                        double *gx, double *gy) {
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < Q; k++) {
        double v = odd ? at_odd(a, nx, ny, x + EX[k], y + EY[k])
                       : at_mirror_x(a, nx, ny, x + EX[k], y + EY[k], open);
        sx += W[k] * EX[k] * v;
        sy += W[k] * EY[k] * v;
    }
    *gx = sx / CS2;
    *gy = sy / CS2;
}

static void grad_node(const double *a, int nx, int ny, int x, int y, int odd, double *gx,
                      double *gy) {
    grad_node_x(a, nx, ny, x, y, odd, 0, gx, gy);
}

/* Eq. 35. */
static double lap_node_x(const double *a, int nx, int ny, int x, int y, int open) {
    double c = a[(long)y * nx + x], s = 0.0;
    for (int k = 0; k < Q; k++)
        s += W[k] * (at_mirror_x(a, nx, ny, x + EX[k], y + EY[k], open) - c);
    return 2.0 * s / CS2;
}

static double lap_node(const double *a, int nx, int ny, int x, int y) {
    return lap_node_x(a, nx, ny, x, y, 0);
}

void orc_grad(int nx, int ny, const double *a, double *gx, double *gy) {
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++)
            grad_node(a, nx, ny, x, y, 0, &gx[(long)y * nx + x], &gy[(long)y * nx + x]);
}

void orc_lap(int nx, int ny, const double *a, double *out) {
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) out[(long)y * nx + x] = lap_node(a, nx, ny, x, y);
}

static double clamp01(double v) { return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v); }

/* Eqs. 32, 24 and 8: phi_i = sum_a g^i_a, phi_3 = 1 - phi_1 - phi_2,
 * 1/(1+chi) = sum_i phi_i/(1+chi_i) (reading: the subscript i restored). */
void orc_phase(const orc_params *p, const double *g, double *phi, double *k) {
    long N = (long)p->nx * p->ny;
#pragma omp parallel for schedule(static) num_threads(n_threads)
    for (long n = 0; n < N; n++) {
        double s1 = 0.0, s2 = 0.0;
        for (int a = 0; a < Q; a++) {
            s1 += g[(0 * Q + a) * N + n];
            s2 += g[(1 * Q + a) * N + n];
        }
        phi[n] = s1;
        phi[N + n] = s2;
        phi[2 * N + n] = 1.0 - s1 - s2;
        if (k) {
            double inv = 0.0;
            for (int i = 0; i < 3; i++) inv += clamp01(phi[i * N + n]) / (1.0 + p->chi[i]);
            k[n] = 1.0 / inv;
        }
    }
}

/* Eq. 6 on the lattice: (L psi)_0 = (2/c_s^2) sum_a w_a k_0a (psi_a - psi_0),
 * k_0a = (k_0 + k_a)/2. For uniform k this is k times the Eq. 35 Laplacian
 * (reading of the paper's "isotropic central FDM"). psi = psi0 + psi' with
 * psi0 = -H0 (x cos(alpha) + y sin(alpha)), whose differences are exact. */
void orc_mag_apply(int nx, int ny, const double *k, const double *psi, double H0,
                   double alpha, double *out) {
    double ca = cos(alpha), sa = sin(alpha);
#pragma omp parallel for schedule(static) num_threads(n_threads)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            long n = (long)y * nx + x;
            double s = 0.0;
            for (int a = 1; a < Q; a++) {
                double kn = at_mirror(k, nx, ny, x + EX[a], y + EY[a]);
                double pn = at_odd(psi, nx, ny, x + EX[a], y + EY[a]);
                double d0 = -H0 * (EX[a] * ca + EY[a] * sa);
                s += W[a] * 0.5 * (k[n] + kn) * ((pn - psi[n]) + d0);
            }
            out[n] = 2.0 * s / CS2;
        }
}

/* b = -L psi0 so that L psi' = b. */
void orc_mag_rhs(int nx, int ny, const double *k, double H0, double alpha, double *b) {
    long N = (long)nx * ny;
    double *z = calloc(N, sizeof(double));
    orc_mag_apply(nx, ny, k, z, H0, alpha, b);
    for (long n = 0; n < N; n++) b[n] = -b[n];
    free(z);
}

static double dot(const double *a, const double *b, long N) {
    double s = 0.0;
    for (long n = 0; n < N; n++) s += a[n] * b[n];
    return s;
}

static double maxabs(const double *a, long N) {
    double m = 0.0;
#pragma omp parallel for schedule(static) num_threads(n_threads) reduction(max : m)
    for (long n = 0; n < N; n++) if (fabs(a[n]) > m) m = fabs(a[n]);
    return m;
}

/* Conjugate gradients on A = -L (symmetric positive definite) for psi',
 * warm-started from psi. Stops when ||L(psi0 + psi')||_inf <= tol * H0,
 * checked on the true residual. Returns 0 when converged, 1 otherwise. */
int orc_mag_solve(int nx, int ny, const double *k, double H0, double alpha, double *psi,
                  double tol, int max_iter, int *iters, double *resid) {
    long N = (long)nx * ny;
    if (H0 == 0.0) {
        memset(psi, 0, N * sizeof(double));
        if (iters) *iters = 0;
        if (resid) *resid = 0.0;
        return 0;
    }
    double *r = malloc(N * sizeof(double)), *pd = malloc(N * sizeof(double));
    double *Ap = malloc(N * sizeof(double));
    double target = tol * H0;
    int it = 0, status = 1;
    orc_mag_apply(nx, ny, k, psi, H0, alpha, r); /* r = b_cg - A psi = L(psi0+psi') */
    double rn = maxabs(r, N);
    if (rn <= target) status = 0;
    while (status && it < max_iter) {
        memcpy(pd, r, N * sizeof(double));
        double rr = dot(r, r, N);
        int restart = 0;
        while (it < max_iter) {
            orc_mag_apply(nx, ny, k, pd, 0.0, alpha, Ap);
#pragma omp parallel for schedule(static) num_threads(n_threads)
            for (long n = 0; n < N; n++) Ap[n] = -Ap[n];
            double pAp = dot(pd, Ap, N);
            if (!(pAp > 0.0)) { restart = 1; break; }
            double al = rr / pAp;
#pragma omp parallel for schedule(static) num_threads(n_threads)
            for (long n = 0; n < N; n++) { psi[n] += al * pd[n]; r[n] -= al * Ap[n]; }
            it++;
            if (maxabs(r, N) <= target) {
                orc_mag_apply(nx, ny, k, psi, H0, alpha, r);
                rn = maxabs(r, N);
                if (rn <= target) status = 0;
                restart = 1;
                break;
            }
            double rr2 = dot(r, r, N);
            const double beta = rr2 / rr;
#pragma omp parallel for schedule(static) num_threads(n_threads)
            for (long n = 0; n < N; n++) pd[n] = r[n] + beta * pd[n];
            rr = rr2;
        }
        if (!restart) break;
    }
    orc_mag_apply(nx, ny, k, psi, H0, alpha, r);
    rn = maxabs(r, N);
    if (iters) *iters = it;
    if (resid) *resid = rn / H0;
    free(r); free(pd); free(Ap);
    return rn <= target ? 0 : status;
}

/* Everything one node needs from one step. */
typedef struct {
    double Fs[2], Fm[2], Fp[2], Fmu[2], u[2], rho, pstar, H[2];
    double fpost[Q], gpost[2][Q];
} node_out;

typedef struct {
    const orc_params *p;
    orc_derived d;
    long N;
    const double *phi;  /* 3 planes, raw */
    const double *rhof; /* density field from clamped phases (Eq. 33) */
    const double *psi;
} step_ctx;

static void node_update(const step_ctx *c, const double *f, const double *g, int x, int y,
                        node_out *o) {
    const orc_params *p = c->p;
    const orc_derived *d = &c->d;
    int nx = p->nx, ny = p->ny;
    long N = c->N, n = (long)y * nx + x;
    double ph[3], phc[3], gph[3][2], lph[3];
    for (int i = 0; i < 2; i++) {
        grad_node_x(c->phi + i * N, nx, ny, x, y, 0, p->open_x, &gph[i][0], &gph[i][1]);
        lph[i] = lap_node_x(c->phi + i * N, nx, ny, x, y, p->open_x);
    }
    /* phi_3 = 1 - phi_1 - phi_2 (Eq. 24), so its derivatives follow. */
    gph[2][0] = -(gph[0][0] + gph[1][0]);
    gph[2][1] = -(gph[0][1] + gph[1][1]);
    lph[2] = -(lph[0] + lph[1]);
    for (int i = 0; i < 3; i++) { ph[i] = c->phi[i * N + n]; phc[i] = clamp01(ph[i]); }

    /* Surface tension, Eqs. 25 and 36. */
    double mu[3];
    orc_chem(d, p->eta, p->xi, ph, lph, mu);
    o->Fs[0] = o->Fs[1] = 0.0;
    for (int i = 0; i < 3; i++) { o->Fs[0] += mu[i] * gph[i][0]; o->Fs[1] += mu[i] * gph[i][1]; }

    /* Kelvin force, Eqs. 5, 7, 9. */
    double inv = 0.0, sgx = 0.0, sgy = 0.0;
    for (int i = 0; i < 3; i++) {
        inv += phc[i] / (1.0 + p->chi[i]);
        sgx += gph[i][0] / (1.0 + p->chi[i]);
        sgy += gph[i][1] / (1.0 + p->chi[i]);
    }
    double gchi_x = -sgx / (inv * inv), gchi_y = -sgy / (inv * inv);
    double dpx, dpy;
    grad_node(c->psi, nx, ny, x, y, 1, &dpx, &dpy);
    o->H[0] = d->H0 * cos(p->alpha) - dpx;
    o->H[1] = d->H0 * sin(p->alpha) - dpy;
    double H2 = o->H[0] * o->H[0] + o->H[1] * o->H[1];
    o->Fm[0] = -0.5 * H2 * gchi_x;
    o->Fm[1] = -0.5 * H2 * gchi_y;

    /* Pressure, density gradient, Eqs. 19, 21, 33. */
    double fl[Q];
    for (int a = 0; a < Q; a++) fl[a] = f[a * N + n];
    double ps = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < Q; a++) { ps += fl[a]; jx += fl[a] * EX[a]; jy += fl[a] * EY[a]; }
    double rho = c->rhof[n], grx, gry;
    grad_node_x(c->rhof, nx, ny, x, y, 0, p->open_x, &grx, &gry);
    o->Fp[0] = -ps * CS2 * grx;
    o->Fp[1] = -ps * CS2 * gry;
    double Fb[2] = {d->G, 0.0};

    /* Velocity without the viscous force, then F_mu = nu [grad u + grad u^T].grad rho
     * in the local non-equilibrium form (reading), then Eq. 22. */
    double F0x = o->Fs[0] + o->Fm[0] + o->Fp[0] + Fb[0];
    double F0y = o->Fs[1] + o->Fm[1] + o->Fp[1] + Fb[1];
    double upx = jx + F0x / (2.0 * rho), upy = jy + F0y / (2.0 * rho);
    double tau = 0.0;
    for (int i = 0; i < 3; i++) tau += phc[i] * d->tau[i]; /* reading: linear in nu */
    double s_nu = 1.0 / (0.5 + tau);
    double feq[Q], h[Q], mh[Q];
    orc_feq(ps, upx, upy, feq);
    for (int a = 0; a < Q; a++) h[a] = fl[a] - feq[a];
    orc_mrt_apply(h, s_nu, mh);
    double Pxx = 0.0, Pxy = 0.0, Pyy = 0.0;
    for (int a = 0; a < Q; a++) {
        Pxx += EX[a] * EX[a] * mh[a];
        Pxy += EX[a] * EY[a] * mh[a];
        Pyy += EY[a] * EY[a] * mh[a];
    }
    double nu_over_cs2 = tau; /* nu = c_s^2 tau (Eq. 14) */
    o->Fmu[0] = -nu_over_cs2 * (Pxx * grx + Pxy * gry);
    o->Fmu[1] = -nu_over_cs2 * (Pxy * grx + Pyy * gry);
    double Ftx = F0x + o->Fmu[0], Fty = F0y + o->Fmu[1];
    double ux = upx + o->Fmu[0] / (2.0 * rho), uy = upy + o->Fmu[1] / (2.0 * rho);
    o->u[0] = ux; o->u[1] = uy; o->rho = rho; o->pstar = ps;

    /* MRT collision, Eqs. 12, 15, 16, 19. */
    double Fa[Q], hb[Q], ch[Q];
    orc_feq(ps, ux, uy, feq);
    for (int a = 0; a < Q; a++) {
        Fa[a] = W[a] * (EX[a] * Ftx + EY[a] * Fty) / (rho * CS2);
        hb[a] = fl[a] - (feq[a] - 0.5 * Fa[a]);
    }
    orc_mrt_apply(hb, s_nu, ch);
    for (int a = 0; a < Q; a++) o->fpost[a] = fl[a] - ch[a] + Fa[a];

    /* Phase-field collision, Eqs. 29-31. reading of the source term of ref. [39]:
     * F_a = w_a e_a . q_i with q_i = theta_i n_i - (1/3) sum_j theta_j n_j,
     * theta_j = (4/xi) phi_j (1 - phi_j), which recovers the flux of Eq. 23. */
    double th[3], nn[3][2], G9[Q];
    for (int j = 0; j < 3; j++) {
        th[j] = 4.0 / p->xi * phc[j] * (1.0 - phc[j]);
        double mag = sqrt(gph[j][0] * gph[j][0] + gph[j][1] * gph[j][1]) + p->eps_n;
        nn[j][0] = gph[j][0] / mag;
        nn[j][1] = gph[j][1] / mag;
    }
    double mx = 0.0, my = 0.0;
    for (int j = 0; j < 3; j++) { mx += th[j] * nn[j][0]; my += th[j] * nn[j][1]; }
    orc_gamma(ux, uy, G9);
    double taup = 0.5 + d->tau_phi;
    for (int i = 0; i < 2; i++) {
        double qx = th[i] * nn[i][0] - mx / 3.0, qy = th[i] * nn[i][1] - my / 3.0;
        for (int a = 0; a < Q; a++) {
            double Fp = W[a] * (EX[a] * qx + EY[a] * qy);
            double geq = ph[i] * G9[a] - 0.5 * Fp;
            double gv = g[(i * Q + a) * N + n];
            o->gpost[i][a] = gv - (gv - geq) / taup + Fp;
        }
    }
}

static void prepare(const orc_params *p, const double *g, step_ctx *c, double *phi,
                    double *rhof, double *k) {
    long N = (long)p->nx * p->ny;
    c->p = p;
    orc_derive(p, &c->d);
    c->N = N;
    orc_phase(p, g, phi, k);
#pragma omp parallel for schedule(static) num_threads(n_threads)
    for (long n = 0; n < N; n++) {
        double r = 0.0;
        for (int i = 0; i < 3; i++) r += p->rho[i] * clamp01(phi[i * N + n]); /* Eq. 33 */
        rhof[n] = r;
    }
    c->phi = phi;
    c->rhof = rhof;
}

void orc_forces(const orc_params *p, const double *f, const double *g, const double *psi,
                double *out) {
    long N = (long)p->nx * p->ny;
    double *phi = malloc(3 * N * sizeof(double)), *rhof = malloc(N * sizeof(double));
    step_ctx c;
    prepare(p, g, &c, phi, rhof, NULL);
    c.psi = psi;
    for (int y = 0; y < p->ny; y++)
        for (int x = 0; x < p->nx; x++) {
            node_out o;
            long n = (long)y * p->nx + x;
            node_update(&c, f, g, x, y, &o);
            double v[14] = {o.Fs[0], o.Fs[1], o.Fm[0], o.Fm[1], o.Fp[0], o.Fp[1], o.Fmu[0],
                            o.Fmu[1], o.u[0], o.u[1], o.rho, o.pstar, o.H[0], o.H[1]};
            for (int j = 0; j < 14; j++) out[j * N + n] = v[j];
        }
    free(phi); free(rhof);
}

/* reading of "the inner droplet touches the interface of the shell": some node
 * with clamped phi_1 >= 1/2 has a D2Q9 neighbour inside the channel with clamped
 * phi_3 >= 1/2; the reported node is the smallest (y, x). */
static int find_touch(int nx, int ny, int open, const double *phi, int *bx, int *by) {
    long N = (long)nx * ny;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            if (clamp01(phi[(long)y * nx + x]) < 0.5) continue;
            for (int a = 1; a < Q; a++) {
                int yy = y + EY[a];
                if (yy < 0 || yy >= ny) continue;
                int xx = x + EX[a];
                if (xx < 0 || xx >= nx) {
                    if (open) continue;
                    xx = (xx + nx) % nx;
                }
                if (clamp01(phi[2 * N + (long)yy * nx + xx]) >= 0.5) {
                    *bx = x; *by = y;
                    return 1;
                }
            }
        }
    return 0;
}

static void init_fields(const orc_params *p, double *f, double *g, double *macro) {
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    for (int y = 0; y < ny; y++) {
        /* Poiseuille profile between half-way walls at -1/2 and ny - 1/2 */
        double u0 = p->u_max * 4.0 * (y + 0.5) * (ny - 0.5 - y) / ((double)ny * ny);
        double feq[Q], G9[Q];
        orc_feq(0.0, u0, 0.0, feq);
        orc_gamma(u0, 0.0, G9);
        for (int x = 0; x < nx; x++) {
            long n = (long)y * nx + x;
            double dx = x - p->xc;
            dx -= nx * floor(dx / nx + 0.5); /* nearest periodic image in x */
            double r = sqrt(dx * dx + (y - p->yc) * (y - p->yc));
            /* reading: tanh profiles of width xi for the shell and core */
            double pout = 0.5 * (1.0 - tanh(2.0 * (r - p->r2) / p->xi));
            double p1 = 0.5 * (1.0 - tanh(2.0 * (r - p->r1) / p->xi));
            double p2 = pout - p1;
            for (int a = 0; a < Q; a++) {
                f[a * N + n] = feq[a];
                g[(0 * Q + a) * N + n] = p1 * G9[a];
                g[(1 * Q + a) * N + n] = p2 * G9[a];
            }
            if (macro) { macro[n] = u0; macro[N + n] = 0.0; macro[2 * N + n] = 0.0; }
        }
    }
}

int orc_init(const orc_params *p, double *f, double *g, double *psi, double *macro,
             int *mag_iters, double *mag_resid) {
    long N = (long)p->nx * p->ny;
    init_fields(p, f, g, macro);
    memset(psi, 0, N * sizeof(double));
    orc_derived d;
    orc_derive(p, &d);
    double *phi = malloc(3 * N * sizeof(double)), *k = malloc(N * sizeof(double));
    orc_phase(p, g, phi, k);
    int st = orc_mag_solve(p->nx, p->ny, k, d.H0, p->alpha, psi, p->mag_tol,
                           p->mag_max_iter, mag_iters, mag_resid);
    free(phi); free(k);
    return st;
}

/* One coupled step per iteration, in the order: phases (Eq. 32), permeability
 * (Eq. 8), potential (Eq. 6), forces (Eqs. 5-9, 19, 25, 33-36), velocity
 * (Eq. 22), collisions (Eqs. 12, 29), streaming with half-way bounce-back. */
/* Open channel: the populations that would enter from outside the channel.
 * fn, gn: this step's post-streaming values (complete except these); f, g:
 * the previous step's (before collision). */
static void open_boundaries(const orc_params *p, const orc_derived *d, const double *f,
                            const double *g, double *fn, double *gn) {
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    for (int y = 0; y < ny; y++) {
        /* Inlet, Eq. 37 (reading: the Poiseuille parabola with centre-line speed u_max
         * between the half-way walls, mean u_avg). Zou-He in the velocity-based form:
         * the unknown populations 1, 5, 8 reflect the non-equilibrium part of their
         * opposites, f_a = f_opp(a) + f^eq_a - f^eq_opp(a) = f_opp(a) + 6 w_a e_a.u,
         * with the transverse correction -/+ (f2 - f4)/2 on 5 and 8 that zeroes the
         * wall-normal momentum. At the two corner nodes the wall supplies one of 5, 8
         * (bounce-back) and the two unknowns follow from both momentum components. */
        double u = p->u_max * 4.0 * (y + 0.5) * (ny - 0.5 - y) / ((double)ny * ny);
        long n = (long)y * nx;
        double fl[Q];
        for (int a = 0; a < Q; a++) fl[a] = fn[a * N + n];
        if (y == 0) {            /* f5 from the wall; solve f8 (j_y = 0), then f1 (j_x = u) */
            fl[8] = fl[2] - fl[4] + fl[5] + fl[6] - fl[7];
        } else if (y == ny - 1) { /* f8 from the wall; solve f5, then f1 */
            fl[5] = fl[4] - fl[2] - fl[6] + fl[7] + fl[8];
        } else {
            fl[5] = fl[7] + 6.0 * W[5] * u - 0.5 * (fl[2] - fl[4]);
            fl[8] = fl[6] + 6.0 * W[8] * u + 0.5 * (fl[2] - fl[4]);
        }
        if (y == 0 || y == ny - 1) fl[1] = u + fl[3] - fl[5] + fl[6] + fl[7] - fl[8];
        else fl[1] = fl[3] + 6.0 * W[1] * u;
        fn[1 * N + n] = fl[1];
        fn[5 * N + n] = fl[5];
        fn[8 * N + n] = fl[8];
        /* reading: the inflow is pure carrier (phi_1 = phi_2 = 0): zero populations */
        for (int i = 0; i < 2; i++) {
            gn[(i * Q + 1) * N + n] = 0.0;
            if (y != 0) gn[(i * Q + 5) * N + n] = 0.0;
            if (y != ny - 1) gn[(i * Q + 8) * N + n] = 0.0;
        }
        /* Outlet: convective condition d chi/dt + U d chi/dx = 0 (refs. [61, 62]) for
         * the populations entering from x = nx, upwind in x and implicit in time,
         * chi(t+1, nx-1) = (chi(t, nx-1) + U chi(t+1, nx-2)) / (1 + U), with U the mean
         * inflow speed u_avg. reading: for f it acts on f_a - w_a p*, the part
         * carried by the flow, while the pressure part takes the reference p* = 0
         * at the outlet (the pressure of this incompressible form is defined up
         * to a constant). A convective condition on all of f holds p* constant
         * across the outlet, starves the outflow of developed channel flow and lets
         * the pressure level drift; linear extrapolation of p* leaves the level
         * free. g is advected as it is. */
        long o = n + nx - 1, b = o - 1;
        double pb = 0.0, po = 0.0;
        for (int a = 0; a < Q; a++) {
            pb += fn[a * N + b];
            po += f[a * N + o];
        }
        const double pout = 0.0;
        double U = d->u_avg;
        const int in3[3] = {3, 6, 7};
        for (int k = 0; k < 3; k++) {
            int a = in3[k];
            if ((a == 6 && y == 0) || (a == 7 && y == ny - 1)) continue; /* from the wall */
            double chi = ((f[a * N + o] - W[a] * po) + U * (fn[a * N + b] - W[a] * pb)) / (1.0 + U);
            fn[a * N + o] = chi + W[a] * pout;
            for (int i = 0; i < 2; i++)
                gn[(i * Q + a) * N + o] = (g[(i * Q + a) * N + o] + U * gn[(i * Q + a) * N + b]) / (1.0 + U);
        }
    }
}

int orc_step(const orc_params *p, double *f, double *g, double *psi, double *macro,
             long step0, long nsteps, orc_track *trk, int *mag_iters, double *mag_resid) {
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    double *phi = malloc(3 * N * sizeof(double)), *rhof = malloc(N * sizeof(double));
    double *k = malloc(N * sizeof(double));
    double *fn = malloc(Q * N * sizeof(double)), *gn = malloc(2 * Q * N * sizeof(double));
    int status = 0;
    build_tables(); /* before the parallel loop: node_update reads them */
    for (long s = 0; s < nsteps; s++) {
        step_ctx c;
        prepare(p, g, &c, phi, rhof, k);
        if (trk && trk->b_step < 0) {
            int bx, by;
            if (find_touch(nx, ny, p->open_x, phi, &bx, &by)) {
                trk->b_step = step0 + s; trk->bx = bx; trk->by = by;
            }
        }
        int it = 0;
        double res = 0.0;
        if (orc_mag_solve(nx, ny, k, c.d.H0, p->alpha, psi, p->mag_tol, p->mag_max_iter, &it,
                          &res))
            status = 1;
        if (mag_iters) *mag_iters = it;
        if (mag_resid) *mag_resid = res;
        c.psi = psi;
        /* each node writes its own post-collision values to distinct slots */
#pragma omp parallel for schedule(static) num_threads(n_threads)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                node_out o;
                long n = (long)y * nx + x;
                node_update(&c, f, g, x, y, &o);
                if (macro) { macro[n] = o.u[0]; macro[N + n] = o.u[1]; macro[2 * N + n] = o.pstar; }
                for (int a = 0; a < Q; a++) {
                    int yy = y + EY[a];
                    if (yy >= 0 && yy < ny) {
                        int xx = x + EX[a];
                        if (p->open_x && (xx < 0 || xx >= nx)) continue; /* leaves the channel */
                        xx = (xx % nx + nx) % nx;
                        long m = (long)yy * nx + xx;
                        fn[a * N + m] = o.fpost[a];
                        gn[(0 * Q + a) * N + m] = o.gpost[0][a];
                        gn[(1 * Q + a) * N + m] = o.gpost[1][a];
                    } else { /* half-way bounce-back at the wall */
                        fn[OPP[a] * N + n] = o.fpost[a];
                        gn[(0 * Q + OPP[a]) * N + n] = o.gpost[0][a];
                        gn[(1 * Q + OPP[a]) * N + n] = o.gpost[1][a];
                    }
                }
            }
        if (p->open_x) open_boundaries(p, &c.d, f, g, fn, gn);
        memcpy(f, fn, Q * N * sizeof(double));
        memcpy(g, gn, 2 * Q * N * sizeof(double));
    }
    free(phi); free(rhof); free(k); free(fn); free(gn);
    return status;
}

/* Crossings of the level 1/2 along a line of samples v[0..n-1] padded with
 * zeros outside: first upward crossing and last downward crossing, linearly
 * interpolated. Returns 0 when the line never reaches 1/2. */
static int crossings(const double *v, int n, double *lo, double *hi) {
    int first = -2, last = -2;
    for (int i = -1; i < n; i++) {
        double a = i < 0 ? 0.0 : v[i], b = i + 1 < n ? v[i + 1] : 0.0;
        if (a < 0.5 && b >= 0.5 && first == -2) { first = i; *lo = i + (0.5 - a) / (b - a); }
        if (a >= 0.5 && b < 0.5) { last = i; *hi = i + (a - 0.5) / (a - b); }
    }
    return first != -2 && last != -2;
}

/* Eq. 42 and the breakup metrics (Fig. 3 is missing; readings):
 *  outer indicator phi1+phi2, inner indicator phi1 (clamped);
 *  l_x: extent of the 1/2-level along the centre line (mean of the two middle
 *       rows when ny is even), scanned from the emptiest column so that a
 *       droplet across the periodic seam stays contiguous;
 *  l_y: largest vertical extent of the 1/2-level over the columns;
 *  centroids: indicator-weighted means in the same unwrapped frame. */
void orc_observe(const orc_params *p, const double *g, const orc_track *trk, long step,
                 orc_obs *o) {
    int nx = p->nx, ny = p->ny;
    long N = (long)nx * ny;
    orc_derived d;
    orc_derive(p, &d);
    double *phi = malloc(3 * N * sizeof(double));
    orc_phase(p, g, phi, NULL);
    memset(o, 0, sizeof *o);
    o->step = step;
    o->t_star = step * d.u_avg / (2.0 * p->r2); /* Eq. 38 */
    for (int i = 0; i < 3; i++) {
        double m = 0.0;
        for (long n = 0; n < N; n++) m += phi[i * N + n];
        o->mass[i] = m;
    }
    double *so = malloc(N * sizeof(double)), *si = malloc(N * sizeof(double));
    for (long n = 0; n < N; n++) {
        si[n] = clamp01(phi[n]);
        so[n] = si[n] + clamp01(phi[N + n]);
    }
    int xcut = 0;
    double best = 0.0;
    for (int x = 0; x < nx && !p->open_x; x++) { /* open channel: the frame starts at the inlet */
        double s = 0.0;
        for (int y = 0; y < ny; y++) s += so[(long)y * nx + x];
        if (x == 0 || s < best) { best = s; xcut = x; }
    }
    double *line = malloc((nx > ny ? nx : ny) * sizeof(double));
    for (int which = 0; which < 2; which++) {
        const double *s = which == 0 ? so : si;
        double m = 0.0, mxs = 0.0, mys = 0.0;
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                double v = s[(long)y * nx + x];
                int xu = x >= xcut ? x : x + nx;
                m += v; mxs += v * xu; mys += v * y;
            }
        double cx = m > 0.0 ? fmod(mxs / m, (double)nx) : 0.0, cy = m > 0.0 ? mys / m : 0.0;
        for (int j = 0; j < nx; j++) {
            int x = (xcut + j) % nx;
            line[j] = ny % 2 ? s[(long)(ny / 2) * nx + x]
                             : 0.5 * (s[(long)(ny / 2 - 1) * nx + x] + s[(long)(ny / 2) * nx + x]);
        }
        double lo, hi, lx = 0.0, ly = 0.0;
        if (crossings(line, nx, &lo, &hi)) lx = hi - lo;
        for (int x = 0; x < nx; x++) {
            for (int y = 0; y < ny; y++) line[y] = s[(long)y * nx + x];
            if (crossings(line, ny, &lo, &hi) && hi - lo > ly) ly = hi - lo;
        }
        double T = (lx + ly) > 0.0 ? (ly - lx) / (ly + lx) : 0.0;
        if (which == 0) {
            o->xc_shell = cx; o->yc_shell = cy; o->lx_o = lx; o->ly_o = ly; o->T_o = T;
        } else {
            o->xc_core = cx; o->yc_core = cy; o->lx_i = lx; o->ly_i = ly; o->T_i = T;
        }
    }
    long bs = trk ? trk->b_step : -1;
    int bx = trk ? trk->bx : 0, by = trk ? trk->by : 0;
    if (bs < 0 && find_touch(nx, ny, p->open_x, phi, &bx, &by)) bs = step;
    o->b_step = bs;
    if (bs >= 0) {
        o->breakup = 1;
        o->xb = bx; o->yb = by;
        o->tb_star = bs * d.u_avg / (2.0 * p->r2);
        o->Lb_star = (double)bx / ny;
        o->yb_star = fabs(by - 0.5 * (ny - 1)) / ny;
    }
    free(phi); free(so); free(si); free(line);
}
