/*
 * FP64 CPU oracle of the polar-coordinate discrete-Boltzmann (lattice Boltzmann
 * kinetic) detonation model of Lin, Xu, Zhang and Li, "Polar coordinate lattice
 * Boltzmann kinetic modeling of detonation phenomena" (arXiv:1308.0653).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library
 * against the paper.  Only the test suite, the smoke check of the package entry
 * point and the CPU-baseline leg of the benchmark may load it.  The product
 * path never calls it and shares no code, header or table with it.
 *
 * Conventions (they are the documented interface of the library as well, so
 * arrays can be compared element by element; the code is independent):
 *   - grid: cell-centred r_j = r_in + (j + 1/2) dr, dr = (r_out - r_in)/nr,
 *           theta_m = m dtheta, dtheta = span / ntheta (span 2 pi, or pi/4 for a
 *           sector), j in [0,nr), m in [0,ntheta)
 *   - macroscopic fields: row-major [ntheta][nr]
 *   - distribution: f[v][ntheta][nr], v = 0 for the rest particle (k = 0),
 *           v = 1 + 8 (k - 1) + i for ring k = 1..4 and direction i = 0..7.
 */
#ifndef DBM_ORACLE_H
#define DBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_NV 33

typedef struct oracle_params {
    int nr, ntheta;          /* grid size                                      */
    double r_in, r_out;      /* annulus radii                                  */
    double dt, tau;          /* time step and BGK relaxation time              */
    double Q;                /* heat release per unit mass                     */
    double omega1, omega2;   /* Cochran rate constants                         */
    double m, n;             /* Cochran pressure exponents                     */
    double T_th;             /* ignition temperature                           */
    double v[4];             /* ring speeds v_1..v_4                           */
    int reaction_energy;     /* 0: R(lambda^t) in M (paper); 1: R = dlambda/dt */
    int sector;              /* 0: full 2 pi grid; 1: pi/4 sector (Sec. II.D)   */
    int r_bc_inner;          /* 0: zero-gradient outflow; 1: disc centre (r_in = 0) */
} oracle_params;

/* Sec. II.B: F_k(T), k = 0..4 (the quartic weights of the D2V33 equilibrium). */
void oracle_weights(const double v[4], double T, double F[5]);

/* Sec. II.B: polar components (v_kir, v_kith) of all 33 velocities at angle theta. */
void oracle_velocities(const double v[4], double theta, double vr[33], double vth[33]);

/* Sec. II.B, Eq. (feq): discrete equilibrium at one site (polar components). */
void oracle_feq(const double v[4], double theta, double rho, double ur, double uth,
                double T, double feq[33]);

/* Sec. II.B: rho, u = (u_r, u_theta) and T of one site's 33 f values. */
void oracle_site_moments(const double v[4], double theta, const double f[33],
                         double *rho, double *ur, double *uth, double *T);

/* Sec. II.B (discrete M_ki): the chemical term for all 33 velocities, given R. */
void oracle_chem(const double v[4], double theta, double rho, double ur, double uth,
                 double T, double Q, double R, double M[33]);

/* Sec. III.A, Eq. (Cochran): rate constants a, b (0 below ignition) and R. */
double oracle_rate(const oracle_params *p, double rho, double T, double lam,
                   double *a, double *b);

/* Sec. III.A, Eq. (Eqlambda), reaction part: exact one-step solution of
 * d lambda/dt = (1 - lambda)(a + b lambda) with a, b frozen. */
double oracle_lambda_react(double lam, double a, double b, double dt);

/* Initial state: f = f^eq(rho, u, T) at every site; lambda copied. */
void oracle_init(const oracle_params *p, const double *rho, const double *ur,
                 const double *uth, const double *T, const double *lam,
                 double *f, double *lam_f);

/* One time step, Sec. II.C Eq. (LB_evolution_equation) and Sec. III.A
 * Eq. (Eqlambda): (f, lam) at t -> (f_new, lam_new) at t + dt.
 * Returns the number of sites whose lambda was clamped to [0, 1]. */
long oracle_step(const oracle_params *p, const double *f, const double *lam,
                 double *f_new, double *lam_new);

/* Macroscopic fields of a state (any output pointer may be NULL). */
void oracle_macro(const oracle_params *p, const double *f, const double *lam,
                  double *rho, double *ur, double *uth, double *T, double *lam_out);

/* Area-weighted FP64 totals: mass, Cartesian momentum x and y, and total
 * energy (rho T + rho u^2 / 2 for D = 2), each summed with weight r dr dtheta. */
void oracle_totals(const oracle_params *p, const double *f, double totals[4]);

/* Sec. II.E, Eq. (M_absolute): central moments of one site's 33 values g
 * (f or f^eq) about the velocity u = (ur, uth), polar components:
 * out[0..2]  M*_2      rr, rth, thth      = sum g v*_a v*_b
 * out[3..6]  M*_3      rrr, rrth, rthth, ththth = sum g v*_a v*_b v*_c
 * out[7..8]  M*_{3,1}  r, th              = sum (1/2) g |v*|^2 v*_a
 * out[9..11] M*_{4,2}  rr, rth, thth      = sum (1/2) g |v*|^2 v*_a v*_b
 * with v* = v_ki - u. */
void oracle_central_moments(const double v[4], double theta, const double g[33], double ur,
                            double uth, double out[12]);

/* Sec. II.E, Eq. (D_absolute): Delta*_m = M*_m(f) - M*_m(f^eq) at every site,
 * written as out[c * N + s] for the 12 components c of oracle_central_moments
 * (N = nr * ntheta, s = m * nr + j), u and f^eq taken from f's own moments. */
void oracle_noneq(const oracle_params *p, const double *f, double *out);

/* init + nsteps steps + macro.  Returns 0, or -1 on allocation failure. */
int oracle_run(const oracle_params *p, const double *rho0, const double *ur0,
               const double *uth0, const double *T0, const double *lam0, long nsteps,
               double *rho, double *ur, double *uth, double *T, double *lam);

/* OpenMP thread count used by oracle_step (1 = serial); returns the count in use. */
int oracle_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
