/*
 * fcd_oracle.h -- plain FP64 CPU oracle of the coupled ferrofluid-compound-
 * droplet time step (arXiv 2410.11129, Sections 2.1-2.5).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library links, includes
 * or calls this code; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark do. It shares no source with the CUDA path.
 *
 * Every array is row-major, unpadded, FP64:
 *   scalar field   a[y*nx + x]                  (ny*nx)
 *   f              f[a*ny*nx + y*nx + x]         (9*ny*nx)
 *   g              g[(i*9 + a)*ny*nx + y*nx + x] (2*9*ny*nx), i = 0 core, 1 shell
 *   psi            perturbation potential psi' (total psi = psi0 + psi')
 *   macro          [ux | uy | p*] of the last step (3*ny*nx)
 * x is periodic, or (open_x) an inlet at x = 0 and an outlet at x = nx - 1;
 * half-way walls sit at y = -1/2 and y = ny - 1/2.
 */
#ifndef FCD_ORACLE_H
#define FCD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int nx, ny;
    double rho[3], nu[3], chi[3]; /* per phase: 1 core, 2 shell, 3 carrier */
    double mobility, xi, eta;     /* M (Eq. 30), interface width, Eq. 28 eta */
    double Ca, Bo_m, alpha;       /* Eq. 40, Eq. 41, field angle [rad] */
    double r1, r2, xc, yc;        /* core/shell radii and centre */
    double s13_over_s12, s23_over_s12; /* Table 2 ratios */
    double sigma23;               /* > 0: use this sigma23 instead of Eq. 40 */
    double u_max;                 /* centre-line velocity of the driving flow */
    int ferro_phase;              /* 1 core, 2 shell, 0 none (Eq. 41 branch) */
    double mag_tol;               /* ||L psi||_inf / H0 target per solve */
    int mag_max_iter;             /* CG iteration cap per solve */
    double eps_n;                 /* regulariser of n = grad phi / |grad phi| */
    int open_x;                   /* 1: velocity inlet (Eq. 37) + convective outlet */
} orc_params;

typedef struct {
    double u_avg, sigma[3][3], gamma[3], gammaT;
    double tau[3], tau_phi, mu0H0sq, H0, G;
} orc_derived;

typedef struct { long b_step; int bx, by; } orc_track; /* b_step < 0: none */

typedef struct {
    long step; double t_star;
    double T_o, T_i, lx_o, ly_o, lx_i, ly_i;
    double xc_core, yc_core, xc_shell, yc_shell;
    double mass[3];
    int breakup; long b_step; double xb, yb, tb_star, Lb_star, yb_star;
} orc_obs;

/* lattice and moment tables: w[9], ex[9], ey[9], M[81], Minv[81] */
void orc_tables(double *w, int *ex, int *ey, double *M, double *Minv);
void orc_derive(const orc_params *p, orc_derived *d);

/* node-level pieces (used by the pins) */
void orc_gamma(double ux, double uy, double *G9);
void orc_feq(double pstar, double ux, double uy, double *feq9);
void orc_mrt_apply(const double *h9, double s_nu, double *out9); /* M^-1 Lambda M h */
void orc_dH(const orc_derived *d, double eta, const double *phi3, double *dH3);
double orc_H(const orc_derived *d, double eta, const double *phi3);
void orc_chem(const orc_derived *d, double eta, double xi, const double *phi3,
              const double *lap3, double *mu3);

/* field-level pieces */
void orc_grad(int nx, int ny, const double *a, double *gx, double *gy);
void orc_lap(int nx, int ny, const double *a, double *out);
void orc_phase(const orc_params *p, const double *g, double *phi3n, double *k);
void orc_mag_apply(int nx, int ny, const double *k, const double *psi, double H0,
                   double alpha, double *out);
void orc_mag_rhs(int nx, int ny, const double *k, double H0, double alpha, double *b);
int orc_mag_solve(int nx, int ny, const double *k, double H0, double alpha,
                  double *psi, double tol, int max_iter, int *iters, double *resid);
/* per-node diagnostics of one step's force evaluation: 14 planes
 * [Fs_x Fs_y Fm_x Fm_y Fp_x Fp_y Fmu_x Fmu_y ux uy rho pstar Hx Hy] */
void orc_forces(const orc_params *p, const double *f, const double *g,
                const double *psi, double *out);

/* whole-path entry points */
int orc_init(const orc_params *p, double *f, double *g, double *psi, double *macro,
             int *mag_iters, double *mag_resid);
int orc_step(const orc_params *p, double *f, double *g, double *psi, double *macro,
             long step0, long nsteps, orc_track *trk, int *mag_iters, double *mag_resid);
void orc_observe(const orc_params *p, const double *g, const orc_track *trk,
                 long step, orc_obs *o);
/* Threads of the row-parallel node loops (1 by default; results are bitwise
 * the same for any count) and the host's processor count (1 without OpenMP). */
void orc_set_threads(int n);
int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
