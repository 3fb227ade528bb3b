/*
 * FP64 CPU oracle of the polar-coordinate discrete-Boltzmann detonation model
 * (Lin, Xu, Zhang, Li, arXiv:1308.0653).
 *
 * TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it; the product path never does.  It is written from
 * the paper, in the paper's order and notation (polar velocity components
 * v_kir, v_kith), one site at a time, with no blocking, fusion or reordering
 * beyond what the equations state.  Readings taken where the printed formulas
 * are garbled or silent are marked "READING" below.
 *
 * Pins (tests/test_oracle_*.py): Maxwellian moment identities of F_k and
 * f^eq, the moment identities of M, an exact ODE solution for the lambda
 * update, a homogeneous-reactor closed form, uniform-state invariance, 8-fold
 * rotation and mirror equivariance, the direction of pure advection, and the
 * Chapman-Jouguet state of the planar detonation of Sec. III.B.
 */
#include "dbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NV ORACLE_NV
#define DIM 2.0 /* D, the number of spatial dimensions (Sec. II.A) */

static const double PI = 3.14159265358979323846;

static int g_threads = 1;

int oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n < 1) n = omp_get_num_procs();
    g_threads = n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}

/* Velocity index of (k, i): the rest particle is 0, ring k >= 1 direction i is
 * 1 + 8 (k - 1) + i. */
static int vindex(int k, int i) { return k == 0 ? 0 : 1 + 8 * (k - 1) + i; }

/* ------------------------------------------------------------------------- */
/* Sec. II.B: weighting coefficients F_k(T).                                 */
/* ------------------------------------------------------------------------- */
/* F_k = [48 T^4 - 6 (x_{k+1}+x_{k+2}+x_{k+3}) T^3
 *        + (x_{k+1}x_{k+2} + x_{k+2}x_{k+3} + x_{k+3}x_{k+1}) T^2
 *        - (1/4) x_{k+1}x_{k+2}x_{k+3} T]
 *       / [x_k (x_k - x_{k+1})(x_k - x_{k+2})(x_k - x_{k+3})],  x = v^2,
 * with the subscript k+l read as k+l-4 when k+l > 4, and F_0 = 1 - 8 sum F_k.
 * READING: the printed sign of the last (linear-in-T) term is "+"; only "-"
 * makes sum_{k,i} F_k v_k^{2n} equal the Maxwellian value (2T)^n n! for
 * n = 1..4, which the weights exist to satisfy. */
void oracle_weights(const double v[4], double T, double F[5])
{
    double x[5];
    double sum = 0.0;
    for (int k = 1; k <= 4; ++k) x[k] = v[k - 1] * v[k - 1];
    for (int k = 1; k <= 4; ++k) {
        int k1 = k + 1 > 4 ? k + 1 - 4 : k + 1;
        int k2 = k + 2 > 4 ? k + 2 - 4 : k + 2;
        int k3 = k + 3 > 4 ? k + 3 - 4 : k + 3;
        double a = x[k1], b = x[k2], c = x[k3];
        double den = x[k] * (x[k] - a) * (x[k] - b) * (x[k] - c);
        double num = 48.0 * T * T * T * T
                   - 6.0 * (a + b + c) * T * T * T
                   + (a * b + b * c + c * a) * T * T
                   - 0.25 * a * b * c * T;
        F[k] = num / den;
        sum += F[k];
    }
    F[0] = 1.0 - 8.0 * sum;
}

/* Sec. II.B: v_ki = v_kir e_r + v_kith e_theta with
 * v_kir = v_k cos(i pi/4 - theta), v_kith = v_k sin(i pi/4 - theta)
 * (the printed "v_kir e_theta" is read as v_kith e_theta). */
void oracle_velocities(const double v[4], double theta, double vr[33], double vth[33])
{
    vr[0] = 0.0;
    vth[0] = 0.0;
    for (int k = 1; k <= 4; ++k) {
        for (int i = 0; i < 8; ++i) {
            double ang = i * PI / 4.0 - theta;
            vr[vindex(k, i)] = v[k - 1] * cos(ang);
            vth[vindex(k, i)] = v[k - 1] * sin(ang);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Sec. II.B, Eq. (feq): the 4th-order discrete equilibrium.                  */
/* ------------------------------------------------------------------------- */
static void feq_with_velocities(const double v[4], const double *vr, const double *vth,
                                double rho, double ur, double uth, double T,
                                double feq[33])
{
    double F[5];
    oracle_weights(v, T, F);
    double u2 = ur * ur + uth * uth;
    for (int k = 0; k <= 4; ++k) {
        int ni = k == 0 ? 1 : 8;
        for (int i = 0; i < ni; ++i) {
            int q = vindex(k, i);
            double vu = vr[q] * ur + vth[q] * uth; /* v_{ki,eps} u_eps */
            double term0 = 1.0 - u2 / (2.0 * T) + u2 * u2 / (8.0 * T * T);
            double term1 = vu / T * (1.0 - u2 / (2.0 * T));
            double term2 = vu * vu / (2.0 * T * T) * (1.0 - u2 / (2.0 * T));
            double term3 = vu * vu * vu / (6.0 * T * T * T);
            double term4 = vu * vu * vu * vu / (24.0 * T * T * T * T);
            feq[q] = rho * F[k] * (term0 + term1 + term2 + term3 + term4);
        }
    }
}

void oracle_feq(const double v[4], double theta, double rho, double ur, double uth,
                double T, double feq[33])
{
    double vr[NV], vth[NV];
    oracle_velocities(v, theta, vr, vth);
    feq_with_velocities(v, vr, vth, rho, ur, uth, T, feq);
}

/* Sec. II.B: rho = sum f, u = sum f v / rho, T = sum (1/2) f (v-u).(v-u) / rho. */
static void moments_with_velocities(const double *vr, const double *vth, const double *f,
                                    long stride, double *rho, double *ur, double *uth,
                                    double *T)
{
    double r = 0.0, jr = 0.0, jt = 0.0;
    for (int q = 0; q < NV; ++q) {
        double fq = f[q * stride];
        r += fq;
        jr += fq * vr[q];
        jt += fq * vth[q];
    }
    double u_r = jr / r, u_t = jt / r;
    double e = 0.0;
    for (int q = 0; q < NV; ++q) {
        double dr_ = vr[q] - u_r, dt_ = vth[q] - u_t;
        e += 0.5 * f[q * stride] * (dr_ * dr_ + dt_ * dt_);
    }
    *rho = r;
    *ur = u_r;
    *uth = u_t;
    *T = e / r;
}

void oracle_site_moments(const double v[4], double theta, const double f[33],
                         double *rho, double *ur, double *uth, double *T)
{
    double vr[NV], vth[NV];
    oracle_velocities(v, theta, vr, vth);
    moments_with_velocities(vr, vth, f, 1, rho, ur, uth, T);
}

/* ------------------------------------------------------------------------- */
/* Sec. II.B: M_ki = f^eq_ki (-D T + (v_ki - u)^2) / (2 T^2) (2Q/D) R.        */
/* ------------------------------------------------------------------------- */
static void chem_with_velocities(const double *vr, const double *vth, const double *feq,
                                 double ur, double uth, double T, double Q, double R,
                                 double M[33])
{
    for (int q = 0; q < NV; ++q) {
        double dr_ = vr[q] - ur, dt_ = vth[q] - uth;
        double c2 = dr_ * dr_ + dt_ * dt_;
        M[q] = feq[q] * (-DIM * T + c2) / (2.0 * T * T) * (2.0 * Q / DIM) * R;
    }
}

void oracle_chem(const double v[4], double theta, double rho, double ur, double uth,
                 double T, double Q, double R, double M[33])
{
    double vr[NV], vth[NV], feq[NV];
    oracle_velocities(v, theta, vr, vth);
    feq_with_velocities(v, vr, vth, rho, ur, uth, T, feq);
    chem_with_velocities(vr, vth, feq, ur, uth, T, Q, R, M);
}

/* ------------------------------------------------------------------------- */
/* Sec. III.A, Eq. (Cochran): R = w1 P^m (1 - lam) + w2 P^n lam (1 - lam),   */
/* with a = w1 P^m, b = w2 P^n and the ignition condition T > T_th.          */
/* P = rho T: ideal gas with particle mass 1 and k = 1 (Sec. II.A).          */
/* ------------------------------------------------------------------------- */
double oracle_rate(const oracle_params *p, double rho, double T, double lam,
                   double *a, double *b)
{
    double P = rho * T;
    double aa = 0.0, bb = 0.0;
    if (T > p->T_th) {
        aa = p->omega1 * pow(P, p->m);
        bb = p->omega2 * pow(P, p->n);
    }
    *a = aa;
    *b = bb;
    return aa * (1.0 - lam) + bb * lam * (1.0 - lam);
}

/* Sec. III.A, Eq. (Eqlambda), reaction part, E = exp((a + b) dt):
 *   lam+ = [(a + b lam) E - a (1 - lam)] / [(a + b lam) E + b (1 - lam)].
 * READING: the printed denominator has a(1 - lam); the exact solution of
 * d lam/dt = (1 - lam)(a + b lam) with a, b frozen has b(1 - lam) there (the
 * conclusions state the reaction is integrated analytically; the printed form
 * starts at half the rate).  With a = b = 0 (no reaction) lam is unchanged. */
double oracle_lambda_react(double lam, double a, double b, double dt)
{
    if (a + b == 0.0) return lam;
    double E = exp((a + b) * dt);
    return ((a + b * lam) * E - a * (1.0 - lam)) / ((a + b * lam) * E + b * (1.0 - lam));
}

/* ------------------------------------------------------------------------- */
/* Initial state.  READING: f starts at f^eq of the given fields (the paper  */
/* gives macroscopic initial data only).                                     */
/* ------------------------------------------------------------------------- */
/* Sec. II.D: the domain is a full annulus/disc (theta span 2 pi) or, as in the
 * paper's runs, a sector of 1/8 of it (span pi/4). */
static double dtheta_of(const oracle_params *p) { return (p->sector ? PI / 4.0 : 2.0 * PI) / p->ntheta; }
static double theta_of(const oracle_params *p, int m) { return m * dtheta_of(p); }
static double r_of(const oracle_params *p, int j)
{
    double dr = (p->r_out - p->r_in) / p->nr;
    return p->r_in + (j + 0.5) * dr;
}

void oracle_init(const oracle_params *p, const double *rho, const double *ur,
                 const double *uth, const double *T, const double *lam,
                 double *f, double *lam_f)
{
    long N = (long)p->nr * p->ntheta;
    for (int m = 0; m < p->ntheta; ++m) {
        double vr[NV], vth[NV], feq[NV];
        oracle_velocities(p->v, theta_of(p, m), vr, vth);
        for (int j = 0; j < p->nr; ++j) {
            long s = (long)m * p->nr + j;
            feq_with_velocities(p->v, vr, vth, rho[s], ur[s], uth[s], T[s], feq);
            for (int q = 0; q < NV; ++q) f[q * N + s] = feq[q];
            lam_f[s] = lam[s];
        }
    }
}

/* ------------------------------------------------------------------------- */
/* One time step.                                                            */
/* ------------------------------------------------------------------------- */
/* Neighbour values (Sec. II.D).
 * theta: periodic.  On a full 2 pi grid row -1 is row ntheta-1.  READING for a
 * pi/4 sector: with the velocity set fixed in the Cartesian frame, the periodic
 * image of the point below row 0 is the point at row ntheta-1 rotated by
 * +pi/4, where direction i has become i+1 (Fig. 1 shows the same rotation
 * between sectors); above the last row it is row 0 with i-1.
 * r, outer boundary and inner boundary of an annulus: READING (the paper defers
 * them to its Ref. XuLin2014): zero-gradient outflow, the ghost at j = -1
 * (j = nr) equals j = 0 (j = nr - 1), same theta and velocity.
 * r, disc centre (r_in = 0): the ghost at j = -1 (r = -dr/2) is the point at
 * r = +dr/2 on the opposite side of the centre.  In a sector that is the
 * paper's rule f(i_r) = f(1 - i_r) with i -> i+4 (same theta index); on a full
 * grid it is row m + ntheta/2 with the same velocity. */
static int vrot(int q, int s)
{
    if (q == 0) return 0;
    int k = (q - 1) / 8, i = (q - 1) % 8;
    return 1 + 8 * k + (((i + s) % 8) + 8) % 8;
}

static long at(const oracle_params *p, long N, int q, int m, int j)
{
    return q * N + (long)m * p->nr + j;
}

static double f_inner(const oracle_params *p, const double *f, long N, int q, int m, int j)
{
    if (j > 0) return f[at(p, N, q, m, j - 1)];
    if (p->r_bc_inner == 1) {
        if (p->sector) return f[at(p, N, vrot(q, 4), m, 0)];
        return f[at(p, N, q, (m + p->ntheta / 2) % p->ntheta, 0)];
    }
    return f[at(p, N, q, m, 0)];
}

static double f_outer(const oracle_params *p, const double *f, long N, int q, int m, int j)
{
    return f[at(p, N, q, m, j < p->nr - 1 ? j + 1 : p->nr - 1)];
}

static double f_below(const oracle_params *p, const double *f, long N, int q, int m, int j)
{
    if (m > 0) return f[at(p, N, q, m - 1, j)];
    return f[at(p, N, p->sector ? vrot(q, 1) : q, p->ntheta - 1, j)];
}

static double f_above(const oracle_params *p, const double *f, long N, int q, int m, int j)
{
    if (m < p->ntheta - 1) return f[at(p, N, q, m + 1, j)];
    return f[at(p, N, p->sector ? vrot(q, -1) : q, 0, j)];
}

/* lambda is a scalar: the same neighbours without the velocity rotation. */
static double l_inner(const oracle_params *p, const double *lam, int m, int j)
{
    if (j > 0) return lam[(long)m * p->nr + j - 1];
    if (p->r_bc_inner == 1 && !p->sector) return lam[(long)((m + p->ntheta / 2) % p->ntheta) * p->nr];
    return lam[(long)m * p->nr];
}
static double l_outer(const oracle_params *p, const double *lam, int m, int j)
{
    return lam[(long)m * p->nr + (j < p->nr - 1 ? j + 1 : p->nr - 1)];
}
static double l_below(const oracle_params *p, const double *lam, int m, int j)
{
    return lam[(long)(m > 0 ? m - 1 : p->ntheta - 1) * p->nr + j];
}
static double l_above(const oracle_params *p, const double *lam, int m, int j)
{
    return lam[(long)(m < p->ntheta - 1 ? m + 1 : 0) * p->nr + j];
}

long oracle_step(const oracle_params *p, const double *f, const double *lam,
                 double *f_new, double *lam_new)
{
    const long N = (long)p->nr * p->ntheta;
    const double dr = (p->r_out - p->r_in) / p->nr;
    const double dth = dtheta_of(p);
    const double dt = p->dt;
    long clamped = 0;

#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(+ : clamped)
#endif
    for (int m = 0; m < p->ntheta; ++m) {
        double vr[NV], vth[NV], fs[NV], feq[NV], M[NV];
        oracle_velocities(p->v, theta_of(p, m), vr, vth);
        for (int j = 0; j < p->nr; ++j) {
            const long s = (long)m * p->nr + j;
            const double r = r_of(p, j);

            /* Moments of f^t at the site (Sec. II.B). */
            for (int q = 0; q < NV; ++q) fs[q] = f[q * N + s];
            double rho, ur, uth, T;
            moments_with_velocities(vr, vth, fs, 1, &rho, &ur, &uth, &T);

            /* Equilibrium (Eq. feq) and Cochran rate (Eq. Cochran). */
            feq_with_velocities(p->v, vr, vth, rho, ur, uth, T, feq);
            double a, b;
            double R = oracle_rate(p, rho, T, lam[s], &a, &b);

            /* Reaction part of the lambda update (Eq. Eqlambda). */
            double lam_react = oracle_lambda_react(lam[s], a, b, dt);
            /* READING (option): R taken as the step's own lambda increment
             * over dt, so that the heat put into f equals rho Q d(lambda). */
            if (p->reaction_energy == 1) R = (lam_react - lam[s]) / dt;

            /* Chemical term M_ki (Sec. II.B). */
            chem_with_velocities(vr, vth, feq, ur, uth, T, p->Q, R, M);

            /* Eq. (LB_evolution_equation) with first-order upwind streaming.
             * C_r = v_kir dt/dr, C_theta = v_kith dt/(r dtheta);
             * f*_r = C_r [f(i_r) - f(i_r - 1)] for C_r >= 0,
             *        C_r [f(i_r + 1) - f(i_r)] for C_r < 0 (same for theta).
             * READING: the printed equation adds +f*_r + f*_theta, which is
             * the downwind (unstable) sign for the transport term
             * -v.grad f; the update subtracts them, as the lambda analogue of
             * Eq. (Eqlambda) does with its explicit minus sign. */
            const double decay = exp(-dt / p->tau);
            for (int q = 0; q < NV; ++q) {
                double Cr = vr[q] * dt / dr;
                double Ct = vth[q] * dt / (r * dth);
                double fr_star, ft_star;
                if (Cr >= 0.0)
                    fr_star = Cr * (fs[q] - f_inner(p, f, N, q, m, j));
                else
                    fr_star = Cr * (f_outer(p, f, N, q, m, j) - fs[q]);
                if (Ct >= 0.0)
                    ft_star = Ct * (fs[q] - f_below(p, f, N, q, m, j));
                else
                    ft_star = Ct * (f_above(p, f, N, q, m, j) - fs[q]);
                f_new[q * N + s] = feq[q] + (fs[q] - feq[q]) * decay - fr_star - ft_star
                                 + M[q] * dt;
            }

            /* Upwind lambda advection with u_r, u_theta from f (Eq. Eqlambda). */
            double lr_star, lt_star;
            if (ur >= 0.0)
                lr_star = -ur * (lam[s] - l_inner(p, lam, m, j)) / dr * dt;
            else
                lr_star = -ur * (l_outer(p, lam, m, j) - lam[s]) / dr * dt;
            if (uth >= 0.0)
                lt_star = -uth * (lam[s] - l_below(p, lam, m, j)) / (r * dth) * dt;
            else
                lt_star = -uth * (l_above(p, lam, m, j) - lam[s]) / (r * dth) * dt;
            double ln = lam_react + lr_star + lt_star;
            /* READING: lambda is a mass fraction (Sec. III.A), kept in [0, 1]. */
            if (ln < 0.0) { ln = 0.0; ++clamped; }
            if (ln > 1.0) { ln = 1.0; ++clamped; }
            lam_new[s] = ln;
        }
    }
    return clamped;
}

void oracle_macro(const oracle_params *p, const double *f, const double *lam,
                  double *rho, double *ur, double *uth, double *T, double *lam_out)
{
    long N = (long)p->nr * p->ntheta;
    for (int m = 0; m < p->ntheta; ++m) {
        double vr[NV], vth[NV];
        oracle_velocities(p->v, theta_of(p, m), vr, vth);
        for (int j = 0; j < p->nr; ++j) {
            long s = (long)m * p->nr + j;
            double a, b, c, d;
            moments_with_velocities(vr, vth, f + s, N, &a, &b, &c, &d);
            if (rho) rho[s] = a;
            if (ur) ur[s] = b;
            if (uth) uth[s] = c;
            if (T) T[s] = d;
            if (lam_out) lam_out[s] = lam[s];
        }
    }
}

void oracle_totals(const oracle_params *p, const double *f, double totals[4])
{
    long N = (long)p->nr * p->ntheta;
    double dr = (p->r_out - p->r_in) / p->nr;
    double dth = dtheta_of(p);
    double mass = 0.0, px = 0.0, py = 0.0, en = 0.0;
    for (int m = 0; m < p->ntheta; ++m) {
        double th = theta_of(p, m);
        double vr[NV], vth[NV];
        oracle_velocities(p->v, th, vr, vth);
        for (int j = 0; j < p->nr; ++j) {
            long s = (long)m * p->nr + j;
            double w = r_of(p, j) * dr * dth;
            double rho, ur, uth, T;
            moments_with_velocities(vr, vth, f + s, N, &rho, &ur, &uth, &T);
            mass += rho * w;
            px += rho * (ur * cos(th) - uth * sin(th)) * w;
            py += rho * (ur * sin(th) + uth * cos(th)) * w;
            en += (rho * T + 0.5 * rho * (ur * ur + uth * uth)) * w;
        }
    }
    totals[0] = mass;
    totals[1] = px;
    totals[2] = py;
    totals[3] = en;
}

/* ------------------------------------------------------------------------- */
/* Sec. II.E: non-equilibrium manifestations.                                */
/* ------------------------------------------------------------------------- */
static void central_with_velocities(const double *vr, const double *vth, const double *g,
                                    long stride, double ur, double uth, double out[12])
{
    for (int c = 0; c < 12; ++c) out[c] = 0.0;
    for (int q = 0; q < NV; ++q) {
        double gq = g[q * stride];
        double a = vr[q] - ur, b = vth[q] - uth;  /* v* in polar components */
        double s2 = a * a + b * b;
        out[0] += gq * a * a;
        out[1] += gq * a * b;
        out[2] += gq * b * b;
        out[3] += gq * a * a * a;
        out[4] += gq * a * a * b;
        out[5] += gq * a * b * b;
        out[6] += gq * b * b * b;
        out[7] += 0.5 * gq * s2 * a;
        out[8] += 0.5 * gq * s2 * b;
        out[9] += 0.5 * gq * s2 * a * a;
        out[10] += 0.5 * gq * s2 * a * b;
        out[11] += 0.5 * gq * s2 * b * b;
    }
}

void oracle_central_moments(const double v[4], double theta, const double g[33], double ur,
                            double uth, double out[12])
{
    double vr[NV], vth[NV];
    oracle_velocities(v, theta, vr, vth);
    central_with_velocities(vr, vth, g, 1, ur, uth, out);
}

void oracle_noneq(const oracle_params *p, const double *f, double *out)
{
    long N = (long)p->nr * p->ntheta;
    for (int m = 0; m < p->ntheta; ++m) {
        double vr[NV], vth[NV], feq[NV];
        oracle_velocities(p->v, theta_of(p, m), vr, vth);
        for (int j = 0; j < p->nr; ++j) {
            long s = (long)m * p->nr + j;
            double rho, ur, uth, T, mf[12], me[12];
            moments_with_velocities(vr, vth, f + s, N, &rho, &ur, &uth, &T);
            feq_with_velocities(p->v, vr, vth, rho, ur, uth, T, feq);
            central_with_velocities(vr, vth, f + s, N, ur, uth, mf);
            central_with_velocities(vr, vth, feq, 1, ur, uth, me);
            for (int c = 0; c < 12; ++c) out[c * N + s] = mf[c] - me[c];
        }
    }
}

int oracle_run(const oracle_params *p, const double *rho0, const double *ur0,
               const double *uth0, const double *T0, const double *lam0, long nsteps,
               double *rho, double *ur, double *uth, double *T, double *lam)
{
    long N = (long)p->nr * p->ntheta;
    double *fa = (double *)malloc(sizeof(double) * NV * N);
    double *fb = (double *)malloc(sizeof(double) * NV * N);
    double *la = (double *)malloc(sizeof(double) * N);
    double *lb = (double *)malloc(sizeof(double) * N);
    if (!fa || !fb || !la || !lb) {
        free(fa); free(fb); free(la); free(lb);
        return -1;
    }
    oracle_init(p, rho0, ur0, uth0, T0, lam0, fa, la);
    for (long t = 0; t < nsteps; ++t) {
        oracle_step(p, fa, la, fb, lb);
        double *tf = fa; fa = fb; fb = tf;
        double *tl = la; la = lb; lb = tl;
    }
    oracle_macro(p, fa, la, rho, ur, uth, T, lam);
    free(fa); free(fb); free(la); free(lb);
    return 0;
}
