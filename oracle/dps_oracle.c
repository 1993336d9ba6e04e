/*
 * dps_oracle.c -- FP64 CPU oracle of the coupled LBM-DEM discrete particle step
 * (Rettinger & Ruede, arXiv:1711.00336).
 *
 * TEST INFRASTRUCTURE ONLY: the plain, slow restatement of the method that the
 * CUDA library is checked against.  Only tests, the smoke check and the CPU
 * baseline leg of the benchmark use it.  No code, header, table or constant is
 * shared with the CUDA library.
 *
 * Plain loops in the order of the paper's Algorithm 1, FP64 throughout,
 * compiled without floating-point contraction.  Readings of passages that the
 * paper leaves open are marked "reading:" where they are taken.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "dps_oracle.h"

#define NQ 19
static const double PI = 3.14159265358979323846;

/* ---------------------------------------------------------------------------
 * D3Q19 lattice (Sec. 3.2.2; weights of Qian et al.: 1/3, 1/18, 1/36).
 * Order: rest, the six axis directions (+x,-x,+y,-y,+z,-z), then the twelve
 * face diagonals in opposite pairs.
 * ------------------------------------------------------------------------- */
static const int CQ[NQ][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double CS2 = 1.0 / 3.0; /* lattice speed of sound squared */

static const double WQ[NQ] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* opposite direction: the list above stores each direction next to its opposite */
static const int OPPQ[NQ] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};

static double wq(int q) { return WQ[q]; }
static int opposite(int q) { return OPPQ[q]; }

void orc_lattice(int c[19][3], double w[19], int opp[19]) {
    for (int q = 0; q < NQ; ++q) {
        for (int a = 0; a < 3; ++a) c[q][a] = CQ[q][a];
        w[q] = wq(q);
        opp[q] = opposite(q);
    }
}

static void cross(const double a[3], const double b[3], double out[3]);
static long ncell_of(const orc_params *P) { return (long)P->n[0] * P->n[1] * P->n[2]; }
static long cidx(const orc_params *P, int ix, int iy, int iz) {
    return ix + (long)P->n[0] * (iy + (long)P->n[1] * iz);
}

/* neighbour index along one axis; -1 if it lies beyond a wall */
static int nb_index(int i, int L, int periodic) {
    if (i >= 0 && i < L) return i;
    if (!periodic) return -1;
    return ((i % L) + L) % L;
}

/* ---------------------------------------------------------------------------
 * Eq. filter_def: three-point discrete delta function of Roma et al.
 * reading: applied per axis, D(x,xp) = phi(|dx|) phi(|dy|) phi(|dz|), which
 * keeps the partition of unity that exact volume and momentum transfer need.
 * ------------------------------------------------------------------------- */
double orc_phi(double r) {
    r = fabs(r);
    if (r < 0.5) return (1.0 + sqrt(1.0 - 3.0 * r * r)) / 3.0;
    if (r < 1.5) return (5.0 - 3.0 * r - sqrt(1.0 - 3.0 * (1.0 - r) * (1.0 - r))) / 6.0;
    return 0.0;
}

/* cell containing the particle along one axis */
static int base_cell(double xp, int L) {
    int i = (int)floor(xp);
    if (i < 0) i = 0;
    if (i > L - 1) i = L - 1;
    return i;
}

/* the cells i-1, i, i+1 around the containing cell i (the kernel support of
 * radius 1.5 cells) and their weights.  reading: across a wall the missing
 * cells are dropped and the remaining weights renormalised to sum to one. */
void orc_weights_1d(double xp, int L, int periodic, int idx[3], double wt[3]) {
    int i = base_cell(xp, L);
    double sum = 0.0;
    for (int o = -1; o <= 1; ++o) {
        int c = i + o;
        double r = (c + 0.5) - xp;
        int k = nb_index(c, L, periodic);
        idx[o + 1] = k;
        wt[o + 1] = (k < 0) ? 0.0 : orc_phi(r);
        sum += wt[o + 1];
    }
    if (!periodic) {
        if (sum > 0.0) {
            for (int o = 0; o < 3; ++o) wt[o] /= sum;
        } else { /* particle far outside the box: put it on the nearest cell */
            wt[0] = wt[2] = 0.0;
            wt[1] = 1.0;
            idx[1] = i;
        }
    }
}

typedef struct {
    int idx[3][3];
    double wt[3][3];
} stencil27;

static void particle_stencil(const orc_params *P, const double xp[3], stencil27 *s) {
    for (int a = 0; a < 3; ++a) orc_weights_1d(xp[a], P->n[a], P->periodic[a], s->idx[a], s->wt[a]);
}

/* Eq. fluid_volume_fraction, solid part: eps_p(x) = dx^-3 sum_i D(x,x_i) V_i */
void orc_solid_fraction(const orc_params *P, long np, const double *x, const double *d,
                        double *eps_p) {
    long nc = ncell_of(P);
    for (long c = 0; c < nc; ++c) eps_p[c] = 0.0;
    for (long i = 0; i < np; ++i) {
        double V = PI / 6.0 * d[i] * d[i] * d[i];
        stencil27 s;
        particle_stencil(P, &x[3 * i], &s);
        for (int oz = 0; oz < 3; ++oz)
            for (int oy = 0; oy < 3; ++oy)
                for (int ox = 0; ox < 3; ++ox) {
                    if (s.idx[0][ox] < 0 || s.idx[1][oy] < 0 || s.idx[2][oz] < 0) continue;
                    double D = s.wt[0][ox] * s.wt[1][oy] * s.wt[2][oz];
                    eps_p[cidx(P, s.idx[0][ox], s.idx[1][oy], s.idx[2][oz])] += D * V;
                }
    }
}

/* eps_f = 1 - eps_p.  reading: floored at eps_min; returns how many cells hit the floor */
long orc_fluid_fraction(const orc_params *P, long np, const double *x, const double *d,
                        double *eps_f) {
    long nc = ncell_of(P), nclamp = 0;
    orc_solid_fraction(P, np, x, d, eps_f);
    for (long c = 0; c < nc; ++c) {
        double e = 1.0 - eps_f[c];
        if (e < P->eps_min) {
            e = P->eps_min;
            ++nclamp;
        }
        eps_f[c] = e;
    }
    return nclamp;
}

/* Eq. distribution_filter applied to a particle vector */
void orc_distribute(const orc_params *P, long np, const double *x, const double *F,
                    double scale, double *out) {
    long nc = ncell_of(P);
    for (long i = 0; i < np; ++i) {
        stencil27 s;
        particle_stencil(P, &x[3 * i], &s);
        for (int oz = 0; oz < 3; ++oz)
            for (int oy = 0; oy < 3; ++oy)
                for (int ox = 0; ox < 3; ++ox) {
                    if (s.idx[0][ox] < 0 || s.idx[1][oy] < 0 || s.idx[2][oz] < 0) continue;
                    double D = s.wt[0][ox] * s.wt[1][oy] * s.wt[2][oz];
                    long c = cidx(P, s.idx[0][ox], s.idx[1][oy], s.idx[2][oz]);
                    for (int a = 0; a < 3; ++a) out[a * nc + c] += scale * D * F[3 * i + a];
                }
    }
}

/* Eq. interpolation */
void orc_interpolate(const orc_params *P, const double *field, int ncomp, const double xp[3],
                     double *out) {
    long nc = ncell_of(P);
    stencil27 s;
    particle_stencil(P, xp, &s);
    for (int k = 0; k < ncomp; ++k) out[k] = 0.0;
    for (int oz = 0; oz < 3; ++oz)
        for (int oy = 0; oy < 3; ++oy)
            for (int ox = 0; ox < 3; ++ox) {
                if (s.idx[0][ox] < 0 || s.idx[1][oy] < 0 || s.idx[2][oz] < 0) continue;
                double D = s.wt[0][ox] * s.wt[1][oy] * s.wt[2][oz];
                long c = cidx(P, s.idx[0][ox], s.idx[1][oy], s.idx[2][oz]);
                for (int k = 0; k < ncomp; ++k) out[k] += D * field[k * nc + c];
            }
}

/* ---------------------------------------------------------------------------
 * Eq. LBM_EQ: porous equilibrium of Guo & Zhao
 * ------------------------------------------------------------------------- */
void orc_equilibrium(double rho, const double u[3], double eps, double feq[19]) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int q = 0; q < NQ; ++q) {
        double cu = CQ[q][0] * u[0] + CQ[q][1] * u[1] + CQ[q][2] * u[2];
        feq[q] = wq(q) * rho *
                 (1.0 + cu / CS2 + (cu * cu) / (2.0 * eps * CS2 * CS2) - uu / (2.0 * eps * CS2));
    }
}

/* Eq. Forcing */
void orc_forcing(double tau, const double u[3], double eps, const double F[3], double Fq[19]) {
    for (int q = 0; q < NQ; ++q) {
        double cu = CQ[q][0] * u[0] + CQ[q][1] * u[1] + CQ[q][2] * u[2];
        double s = 0.0;
        for (int a = 0; a < 3; ++a) {
            double term = CQ[q][a] / CS2 - u[a] / (eps * CS2) + cu / (eps * CS2 * CS2) * CQ[q][a];
            s += term * F[a];
        }
        Fq[q] = wq(q) * (1.0 - 1.0 / (2.0 * tau)) * s;
    }
}

/* Eq. MacVel: rho = sum f_q, j = sum f_q c_q */
void orc_moments(const orc_params *P, const double *f, double *rho, double *j) {
    long nc = ncell_of(P);
    for (long c = 0; c < nc; ++c) {
        double r = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < NQ; ++q) {
            double v = f[q * nc + c];
            r += v;
            for (int a = 0; a < 3; ++a) m[a] += v * CQ[q][a];
        }
        rho[c] = r;
        for (int a = 0; a < 3; ++a) j[a * nc + c] = m[a];
    }
}

/* Eq. LBM_Equation: f_q(x+c_q, t+1) = f_q + (f_q^eq - f_q)/tau + F_q.
 * Walls (non-periodic faces) use halfway bounce-back: a population that would
 * leave the box through a wall returns to its cell with the opposite velocity. */
void orc_collide_stream(const orc_params *P, const double *f, const double *eps,
                        const double *fext, double *fnew) {
    long nc = ncell_of(P);
    for (int iz = 0; iz < P->n[2]; ++iz)
        for (int iy = 0; iy < P->n[1]; ++iy)
            for (int ix = 0; ix < P->n[0]; ++ix) {
                long c = cidx(P, ix, iy, iz);
                double fl[NQ], feq[NQ], Fq[NQ], rho = 0.0, j[3] = {0, 0, 0}, F[3], u[3];
                for (int q = 0; q < NQ; ++q) {
                    fl[q] = f[q * nc + c];
                    rho += fl[q];
                    for (int a = 0; a < 3; ++a) j[a] += fl[q] * CQ[q][a];
                }
                for (int a = 0; a < 3; ++a) {
                    F[a] = fext[a * nc + c];
                    u[a] = j[a] / rho + F[a] / (2.0 * rho);
                }
                /* Eq. tau_e: constant tau, or the Eilers / Smagorinsky value */
                double tau = (P->eilers || P->smagorinsky) ? orc_tau_e(P, fl, rho, u, eps[c]) : P->tau;
                orc_equilibrium(rho, u, eps[c], feq);
                orc_forcing(tau, u, eps[c], F, Fq);
                for (int q = 0; q < NQ; ++q) {
                    double post = fl[q] + (feq[q] - fl[q]) / tau + Fq[q];
                    int tx = nb_index(ix + CQ[q][0], P->n[0], P->periodic[0]);
                    int ty = nb_index(iy + CQ[q][1], P->n[1], P->periodic[1]);
                    int tz = nb_index(iz + CQ[q][2], P->n[2], P->periodic[2]);
                    if (tx < 0 || ty < 0 || tz < 0)
                        fnew[opposite(q) * nc + c] = post;
                    else
                        fnew[q * nc + cidx(P, tx, ty, tz)] = post;
                }
            }
}

/* Sec. 3.2.3: grad phi ~ c_s^-2 sum_q w_q c_q phi(x + c_q).
 * reading: a neighbour beyond a wall is mirrored back across the wall face
 * (its coordinate along the wall normal is clamped into the box), which keeps
 * tangential derivatives exact and gives the one-sided normal derivative. */
static int clamp_index(int i, int L, int periodic) {
    if (i >= 0 && i < L) return i;
    if (periodic) return ((i % L) + L) % L;
    return i < 0 ? 0 : (i > L - 1 ? L - 1 : i);
}

void orc_lattice_gradient(const orc_params *P, const double *phi, double *grad) {
    long nc = ncell_of(P);
    for (int iz = 0; iz < P->n[2]; ++iz)
        for (int iy = 0; iy < P->n[1]; ++iy)
            for (int ix = 0; ix < P->n[0]; ++ix) {
                long c = cidx(P, ix, iy, iz);
                double g[3] = {0, 0, 0};
                for (int q = 0; q < NQ; ++q) {
                    int tx = clamp_index(ix + CQ[q][0], P->n[0], P->periodic[0]);
                    int ty = clamp_index(iy + CQ[q][1], P->n[1], P->periodic[1]);
                    int tz = clamp_index(iz + CQ[q][2], P->n[2], P->periodic[2]);
                    double v = phi[cidx(P, tx, ty, tz)];
                    for (int a = 0; a < 3; ++a) g[a] += wq(q) * CQ[q][a] * v;
                }
                for (int a = 0; a < 3; ++a) grad[a * nc + c] = g[a] / CS2;
            }
}

/* Sec. 3.2.3: curl psi ~ c_s^-2 sum_q w_q c_q x psi(x + c_q), same neighbour
 * rule as the gradient */
void orc_lattice_curl(const orc_params *P, const double *psi, double *curl) {
    long nc = ncell_of(P);
    for (int iz = 0; iz < P->n[2]; ++iz)
        for (int iy = 0; iy < P->n[1]; ++iy)
            for (int ix = 0; ix < P->n[0]; ++ix) {
                long c = cidx(P, ix, iy, iz);
                double r[3] = {0, 0, 0};
                for (int q = 0; q < NQ; ++q) {
                    int tx = clamp_index(ix + CQ[q][0], P->n[0], P->periodic[0]);
                    int ty = clamp_index(iy + CQ[q][1], P->n[1], P->periodic[1]);
                    int tz = clamp_index(iz + CQ[q][2], P->n[2], P->periodic[2]);
                    long n = cidx(P, tx, ty, tz);
                    double v[3] = {psi[n], psi[nc + n], psi[2 * nc + n]};
                    double cq[3] = {CQ[q][0], CQ[q][1], CQ[q][2]};
                    r[0] += wq(q) * (cq[1] * v[2] - cq[2] * v[1]);
                    r[1] += wq(q) * (cq[2] * v[0] - cq[0] * v[2]);
                    r[2] += wq(q) * (cq[0] * v[1] - cq[1] * v[0]);
                }
                for (int a = 0; a < 3; ++a) curl[a * nc + c] = r[a] / CS2;
            }
}

/* ---------------------------------------------------------------------------
 * Eq. visc_eilers: mu_* / mu_0 = (1 + 0.5 [mu] eps_p / (1 - eps_p/eps_cp))^2,
 * [mu] = 2.5, eps_cp = 0.64.  reading: the printed "(1 - eps_p)/eps_cp" is
 * taken as Eilers' (1 - eps_p/eps_cp) (the printed form contradicts the
 * Einstein limit 1 + 2.5 eps_p); eps_p/eps_cp is capped at 0.9 where the
 * closure diverges.
 * ------------------------------------------------------------------------- */
double orc_eilers_factor(double eps_p) {
    const double intrinsic = 2.5, eps_cp = 0.64;
    double ratio = eps_p / eps_cp;
    if (ratio > 0.9) ratio = 0.9;
    if (ratio < 0.0) ratio = 0.0;
    double a = 1.0 + 0.5 * intrinsic * (ratio * eps_cp) / (1.0 - ratio);
    return a * a;
}

/* Eq. tau_t (Smagorinsky, C_S = 0.1, dx_LES = dx = 1).
 * reading: Qbar is the one Eq. visc_turb defines, sqrt(2 sum Q_ab Q_ab).
 * Eq. visc_turb with tau_e = tau_* + tau_t gives the quadratic
 * tau_t (tau_* + tau_t) = C_S^2 Qbar / (2 rho c_s^4); its positive root is the
 * printed Eq. tau_t once the printed 2 sqrt(2) factor is taken with the
 * momentum-flux norm sqrt(sum Q_ab Q_ab) of the cited LES scheme, i.e. with
 * Qbar / sqrt(2). */
double orc_tau_turb(double tau_star, double Qbar, double rho) {
    const double Cs = 0.1;
    double arg = tau_star * tau_star + 2.0 * Cs * Cs / (rho * CS2 * CS2) * Qbar;
    return 0.5 * (sqrt(arg) - tau_star);
}

/* Eqs. visc_tau_*, visc_turb, tau_e for one cell: tau_* from mu_* (Eilers,
 * with eps_p = 1 - eps_f of the cell) and tau_t from the non-equilibrium
 * momentum flux Q_ab = sum_q c_a c_b (f_q - f_q^eq) */
double orc_tau_e(const orc_params *P, const double f[19], double rho, const double u[3], double eps) {
    double nu0 = (P->tau - 0.5) * CS2;
    double tau_star = P->tau;
    if (P->eilers) tau_star = 0.5 + nu0 * orc_eilers_factor(1.0 - eps) / CS2;
    if (!P->smagorinsky) return tau_star;
    double feq[NQ];
    orc_equilibrium(rho, u, eps, feq);
    double Q2 = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double Qab = 0.0;
            for (int q = 0; q < NQ; ++q) Qab += CQ[q][a] * CQ[q][b] * (f[q] - feq[q]);
            Q2 += Qab * Qab;
        }
    double Qbar = sqrt(2.0 * Q2);
    return tau_star + orc_tau_turb(tau_star, Qbar, rho);
}

/* Table 1: F_l = 1.61 d^2 sqrt(mu rho_f / |w|) ((u_f - u_p) x w), w = curl u_f
 * at the particle; zero where the vorticity vanishes */
void orc_lift(double d, double mu, double rho_f, const double du[3], const double w[3], double F[3]) {
    double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (!(wn > 0.0)) {
        F[0] = F[1] = F[2] = 0.0;
        return;
    }
    double k = 1.61 * d * d * sqrt(mu * rho_f / wn);
    double c[3];
    cross(du, w, c);
    for (int a = 0; a < 3; ++a) F[a] = k * c[a];
}

/* ---------------------------------------------------------------------------
 * Table 1: drag correlation of Tenneti et al. and the particle Reynolds number
 * ------------------------------------------------------------------------- */
double orc_cd(double Re, double eps_p) {
    double e1 = 1.0 - eps_p;
    double cd0 = 1.0 + 0.15 * pow(Re, 0.687);
    double A = 5.81 * eps_p / (e1 * e1 * e1) + 0.48 * cbrt(eps_p) / (e1 * e1 * e1 * e1);
    double B = eps_p * eps_p * eps_p * Re * (0.95 + 0.61 * eps_p * eps_p * eps_p / (e1 * e1));
    return e1 * (cd0 / (e1 * e1 * e1) + A + B);
}

double orc_reynolds(double eps_f, double rho_f, double d, double du, double mu) {
    return eps_f * rho_f * d * du / mu;
}

/* ---------------------------------------------------------------------------
 * Sec. 3.1.1: contact constants from e_n and T_c.  Eq. damping_to_stiffness
 * and Eq. collision_time solved for k_n and xi_n.
 * ------------------------------------------------------------------------- */
void orc_contact_constants(double m_ij, double e_n, double T_c, double *k_n, double *xi_n) {
    double le = log(e_n);
    /* T_c = 2 pi m / sqrt(4 m k - xi^2) with xi^2 = 4 ln^2(e) m k / (pi^2 + ln^2 e) */
    *k_n = m_ij * (PI * PI + le * le) / (T_c * T_c);
    *xi_n = -2.0 * le * sqrt(m_ij * (*k_n)) / sqrt(PI * PI + le * le);
}

/* Sec. 3.1.3, coefficients of Eq. lubrication_force (Ball & Melrose) */
void orc_lub_coefficients(double dmean, double h, double mu, double *a_sq, double *a_sh_eff) {
    double L = log(dmean / (2.0 * h));
    *a_sq = 1.5 * PI * mu * dmean *
            (dmean / (4.0 * h) + 18.0 / 40.0 * L + 9.0 / 84.0 * (h / dmean) * L);
    double a_sh = 0.5 * PI * mu * dmean * L * (dmean + h) * (dmean + h) / 4.0;
    double s = 2.0 / (h + dmean);
    *a_sh_eff = a_sh * s * s;
}

static void cross(const double a[3], const double b[3], double out[3]) {
    out[0] = a[1] * b[2] - a[2] * b[1];
    out[1] = a[2] * b[0] - a[0] * b[2];
    out[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static double particle_mass(double d, double rho_p) { return rho_p * PI / 6.0 * d * d * d; }

/* force (and torque) on particle i from one partner: another sphere, or a wall
 * (partner at rest, infinite mass, d_j -> infinity).
 *   n      unit normal from i towards the partner
 *   dist   centre distance (for a wall: centre-to-wall distance)
 *   sumr   (d_i+d_j)/2 (for a wall: d_i/2)
 *   uj, wj_term   partner velocity and (d_j/2) omega_j (zero for a wall)
 *   m_ij   reduced mass (m_i for a wall), dmean = <d> (2 d_i for a wall) */
static void partner_force(const orc_params *P, orc_state *S, double dt_dem, const double n[3],
                          double dist, double sumr, const double ui[3], const double wi[3],
                          double di, const double uj[3], const double wj_half[3], double m_ij,
                          double dmean, double Fc[3], double Tc[3], double Fl[3]) {
    /* Sec. 3.1.1: overlap, contact-point relative velocity, spring-dashpot */
    double delta = sumr - dist;
    if (P->contact && delta > 0.0) {
        double k_n, xi_n;
        orc_contact_constants(m_ij, P->e_n, P->T_c, &k_n, &xi_n);
        double xi_t = xi_n; /* the paper always takes xi_n = xi_t */
        double wsum[3], wx[3], ur[3];
        for (int a = 0; a < 3; ++a) wsum[a] = 0.5 * di * wi[a] + wj_half[a];
        cross(wsum, n, wx);
        for (int a = 0; a < 3; ++a) ur[a] = ui[a] - uj[a] + wx[a];
        double urn = dot(ur, n);
        double un[3], ut[3], Fn[3];
        for (int a = 0; a < 3; ++a) {
            un[a] = urn * n[a];
            ut[a] = ur[a] - un[a];
            Fn[a] = -k_n * delta * n[a] - xi_n * un[a];
        }
        double Fn_abs = sqrt(dot(Fn, Fn));
        double ut_abs = sqrt(dot(ut, ut));
        double Ft[3] = {0, 0, 0};
        if (ut_abs > 0.0) {
            double mag = fmin(P->mu_c * Fn_abs, xi_t * ut_abs);
            for (int a = 0; a < 3; ++a) Ft[a] = -mag * ut[a] / ut_abs;
        }
        /* Eq. torques_collision.  reading: torque = r x F with the contact point
         * at r = (d_i/2) n, i.e. (d_i/2) n x F_t; the printed operand order
         * F_t x n has the opposite sign and would feed, not damp, slip. */
        double nxF[3];
        cross(n, Ft, nxF);
        for (int a = 0; a < 3; ++a) {
            Fc[a] += Fn[a] + Ft[a];
            Tc[a] += 0.5 * di * nxF[a];
        }
    }
    /* Sec. 3.1.3: lubrication for gaps below h_c, gap floored at h_min.
     * reading: only for pairs that do not overlap (0 <= h < h_c); the floor
     * bounds the force of nearly touching pairs.  Applied at the floored gap
     * during contact as well, it would damp a sphere hitting a wall by a
     * factor ~1e-4 over one collision time, while Sec. 5 (Table 3) reports
     * rebounds with lubrication on.  Coefficients clamped at >= 0 (the printed
     * series turns negative at large gaps); with the limiter on each
     * coefficient is capped at lub_cap*m_ij/dt_DEM so the explicit update
     * stays stable. */
    double h = dist - sumr;
    if (P->lubrication && h >= 0.0 && h < P->h_c) {
        double hh = fmax(h, P->h_min);
        double mu = P->rho_f * (P->tau - 0.5) * CS2;
        double a_sq, a_sh;
        orc_lub_coefficients(dmean, hh, mu, &a_sq, &a_sh);
        a_sq = fmax(a_sq, 0.0);
        a_sh = fmax(a_sh, 0.0);
        if (P->lub_limiter) {
            double cap = P->lub_cap * m_ij / dt_dem;
            if (a_sq > cap) { a_sq = cap; S->n_lub_limited++; }
            if (a_sh > cap) { a_sh = cap; S->n_lub_limited++; }
        }
        double upr[3];
        for (int a = 0; a < 3; ++a) upr[a] = ui[a] - uj[a];
        double upn = dot(upr, n);
        for (int a = 0; a < 3; ++a)
            Fl[a] += -a_sq * upn * n[a] - a_sh * (upr[a] - upn * n[a]);
    }
}

/* minimum-image separation along one axis */
static double min_image(double dx, int L, int periodic) {
    if (!periodic) return dx;
    return dx - L * nearbyint(dx / L);
}

static double pair_range(const orc_params *P, double di, double dj) {
    return 0.5 * (di + dj) + (P->lubrication ? fmax(P->h_c, 0.0) : 0.0);
}

static void pair_contribution(const orc_params *P, orc_state *S, double dt_dem, long i, long j) {
    double dx[3];
    for (int a = 0; a < 3; ++a)
        dx[a] = min_image(S->x[3 * j + a] - S->x[3 * i + a], P->n[a], P->periodic[a]);
    double dist = sqrt(dot(dx, dx));
    double di = S->d[i], dj = S->d[j];
    if (!(dist < pair_range(P, di, dj))) return;
    if (dist == 0.0) { S->n_coincident++; return; }
    double n[3] = {dx[0] / dist, dx[1] / dist, dx[2] / dist};
    double mi = particle_mass(di, S->rho_p[i]), mj = particle_mass(dj, S->rho_p[j]);
    double m_ij = mi * mj / (mi + mj);
    double dmean = 2.0 * di * dj / (di + dj);
    double wj_half[3];
    for (int a = 0; a < 3; ++a) wj_half[a] = 0.5 * dj * S->w[3 * j + a];
    partner_force(P, S, dt_dem, n, dist, 0.5 * (di + dj), &S->u[3 * i], &S->w[3 * i], di,
                  &S->u[3 * j], wj_half, m_ij, dmean, &S->F_c[3 * i], &S->T_c[3 * i],
                  &S->F_lub[3 * i]);
}

/* ---------------------------------------------------------------------------
 * Linked-cell list.  Cells of the lattice are grouped into bins of B cells
 * per axis (the last bin of an axis takes the remainder); the key of a
 * lattice cell orders cells bin-major (bz,by,bx), then (z,y,x) inside the bin.
 * Particles are sorted stably by the key of the cell that contains them.
 * ------------------------------------------------------------------------- */
static int n_bins(int L, int B) { int nb = L / B; return nb < 1 ? 1 : nb; }
static int bin_of(int i, int B, int nb) { int b = i / B; return b > nb - 1 ? nb - 1 : b; }
static int bin_start(int b, int B) { return b * B; }
static int bin_width(int b, int B, int nb, int L) { return b == nb - 1 ? L - b * B : B; }

static long cell_key(const orc_params *P, int B, const int ic[3]) {
    int nb[3], b[3], s[3], W[3];
    for (int a = 0; a < 3; ++a) {
        nb[a] = n_bins(P->n[a], B);
        b[a] = bin_of(ic[a], B, nb[a]);
        s[a] = bin_start(b[a], B);
        W[a] = bin_width(b[a], B, nb[a], P->n[a]);
    }
    long Lx = P->n[0], Ly = P->n[1];
    long before = (long)s[2] * Ly * Lx + (long)W[2] * s[1] * Lx + (long)W[2] * W[1] * s[0];
    long local = ((long)(ic[2] - s[2]) * W[1] + (ic[1] - s[1])) * W[0] + (ic[0] - s[0]);
    return before + local;
}

static void particle_cell(const orc_params *P, const double *xp, int ic[3]) {
    for (int a = 0; a < 3; ++a) ic[a] = base_cell(xp[a], P->n[a]);
}

void orc_cell_list(const orc_params *P, long np, const double *x, int B, int *cell_start,
                   int *order, int *key) {
    long nc = ncell_of(P);
    for (long c = 0; c <= nc; ++c) cell_start[c] = 0;
    for (long i = 0; i < np; ++i) {
        int ic[3];
        particle_cell(P, &x[3 * i], ic);
        key[i] = (int)cell_key(P, B, ic);
        cell_start[key[i] + 1]++;
    }
    for (long c = 0; c < nc; ++c) cell_start[c + 1] += cell_start[c];
    int *fill = (int *)calloc((size_t)(nc > 0 ? nc : 1), sizeof(int));
    for (long i = 0; i < np; ++i) { /* ascending id: stable */
        order[cell_start[key[i]] + fill[key[i]]] = (int)i;
        fill[key[i]]++;
    }
    free(fill);
}

/* pair loop with a plain linked-cell structure (head/next chains) */
static void pairs_linked_cells(const orc_params *P, orc_state *S, double dt_dem) {
    double dmax = 0.0;
    for (long i = 0; i < S->np; ++i) dmax = fmax(dmax, S->d[i]);
    double rc = pair_range(P, dmax, dmax);
    int nb[3];
    double bw[3];
    for (int a = 0; a < 3; ++a) {
        nb[a] = (int)floor(P->n[a] / rc);
        if (nb[a] < 1) nb[a] = 1;
        bw[a] = (double)P->n[a] / nb[a];
    }
    long nbin = (long)nb[0] * nb[1] * nb[2];
    long *head = (long *)malloc(sizeof(long) * nbin);
    long *next = (long *)malloc(sizeof(long) * (S->np > 0 ? S->np : 1));
    int *bi = (int *)malloc(sizeof(int) * 3 * (S->np > 0 ? S->np : 1));
    for (long b = 0; b < nbin; ++b) head[b] = -1;
    for (long i = S->np - 1; i >= 0; --i) {
        int b3[3];
        for (int a = 0; a < 3; ++a) {
            int k = (int)floor(S->x[3 * i + a] / bw[a]);
            if (k < 0) k = 0;
            if (k > nb[a] - 1) k = nb[a] - 1;
            b3[a] = k;
            bi[3 * i + a] = k;
        }
        long b = b3[0] + (long)nb[0] * (b3[1] + (long)nb[1] * b3[2]);
        next[i] = head[b];
        head[b] = i;
    }
    for (long i = 0; i < S->np; ++i) {
        /* distinct neighbour bins per axis */
        int list[3][3], cnt[3];
        for (int a = 0; a < 3; ++a) {
            cnt[a] = 0;
            for (int o = -1; o <= 1; ++o) {
                int k = bi[3 * i + a] + o;
                if (P->periodic[a]) k = ((k % nb[a]) + nb[a]) % nb[a];
                else if (k < 0 || k >= nb[a]) continue;
                int dup = 0;
                for (int m = 0; m < cnt[a]; ++m) dup |= (list[a][m] == k);
                if (!dup) list[a][cnt[a]++] = k;
            }
        }
        for (int cz = 0; cz < cnt[2]; ++cz)
            for (int cy = 0; cy < cnt[1]; ++cy)
                for (int cx = 0; cx < cnt[0]; ++cx) {
                    long b = list[0][cx] + (long)nb[0] * (list[1][cy] + (long)nb[1] * list[2][cz]);
                    for (long j = head[b]; j >= 0; j = next[j])
                        if (j != i) pair_contribution(P, S, dt_dem, i, j);
                }
    }
    free(head);
    free(next);
    free(bi);
}

/* walls: the faces x_a = 0 and x_a = n[a] of every non-periodic axis */
static void wall_contributions(const orc_params *P, orc_state *S, double dt_dem, long i) {
    static const double zero[3] = {0, 0, 0};
    double di = S->d[i];
    double mi = particle_mass(di, S->rho_p[i]);
    for (int a = 0; a < 3; ++a) {
        if (P->periodic[a]) continue;
        for (int side = 0; side < 2; ++side) {
            double dist = side == 0 ? S->x[3 * i + a] : P->n[a] - S->x[3 * i + a];
            double range = 0.5 * di + (P->lubrication ? fmax(P->h_c, 0.0) : 0.0);
            if (!(dist < range)) continue;
            double n[3] = {0, 0, 0};
            n[a] = side == 0 ? -1.0 : 1.0;
            /* Sec. 3.1.1: m_ij = m_i for a wall; Sec. 3.1.3: <d> = 2 d_i */
            partner_force(P, S, dt_dem, n, dist, 0.5 * di, &S->u[3 * i], &S->w[3 * i], di, zero,
                          zero, mi, 2.0 * di, &S->F_c[3 * i], &S->T_c[3 * i], &S->F_lub[3 * i]);
        }
    }
}

void orc_dem_forces(const orc_params *P, orc_state *S, double dt_dem) {
    long np = S->np;
    for (long k = 0; k < 3 * np; ++k) S->F_c[k] = S->T_c[k] = S->F_lub[k] = 0.0;
    if (P->pair_search == 0) {
        for (long i = 0; i < np; ++i)
            for (long j = 0; j < np; ++j)
                if (j != i) pair_contribution(P, S, dt_dem, i, j);
    } else {
        pairs_linked_cells(P, S, dt_dem);
    }
    for (long i = 0; i < np; ++i) wall_contributions(P, S, dt_dem, i);
}

/* Eq. particle_motion integrated over one DEM substep.  reading: semi-implicit
 * Euler, velocities first, positions with the new velocity; I_p = m d^2 / 10. */
static void integrate(const orc_params *P, orc_state *S, double dt) {
    for (long i = 0; i < S->np; ++i) {
        double m = particle_mass(S->d[i], S->rho_p[i]);
        double I = m * S->d[i] * S->d[i] / 10.0;
        for (int a = 0; a < 3; ++a) {
            double F = S->F_hyd[3 * i + a] + S->F_c[3 * i + a] + S->F_lub[3 * i + a];
            S->u[3 * i + a] += dt * F / m;
            S->w[3 * i + a] += dt * S->T_c[3 * i + a] / I;
            double xn = S->x[3 * i + a] + dt * S->u[3 * i + a];
            if (P->periodic[a]) {
                int L = P->n[a];
                xn -= L * floor(xn / L);
                if (xn >= L) xn -= L;
            }
            S->x[3 * i + a] = xn;
        }
    }
}

/* ---------------------------------------------------------------------------
 * Algorithm 1
 * ------------------------------------------------------------------------- */
void orc_init(const orc_params *P, orc_state *S) {
    long nc = ncell_of(P);
    /* Algorithm 1: initial fluid volume fraction */
    S->n_eps_clamp += orc_fluid_fraction(P, S->np, S->x, S->d, S->eps_f);
    /* reading: fluid at rest with unit density, f = f^eq(1, 0, eps_f) = w_q */
    for (int q = 0; q < NQ; ++q)
        for (long c = 0; c < nc; ++c) S->f[q * nc + c] = wq(q);
    for (long k = 0; k < 3 * nc; ++k) S->fpf[k] = 0.0;
    S->have_u_prev = 0;
    S->have_u_sub = 0;
    S->step = 0;
}

/* fluid-phase velocity u_f = ubar/eps_f, ubar from Eq. MacVel with force F */
static void fluid_velocity(long nc, const double *rho, const double *j, const double *eps,
                           const double *F, double *uf) {
    for (int a = 0; a < 3; ++a)
        for (long c = 0; c < nc; ++c)
            uf[a * nc + c] = (j[a * nc + c] + 0.5 * F[a * nc + c]) / rho[c] / eps[c];
}

int orc_step(const orc_params *P, orc_state *S, long nsteps) {
    long nc = ncell_of(P), np = S->np;
    double mu = P->rho_f * (P->tau - 0.5) * CS2;          /* Eq. visc_tau */
    double dt_sub = 1.0 / P->n_int;                        /* one interaction subcycle */
    double dt_dem = 1.0 / ((double)P->n_int * P->n_dem);  /* dt / (n_int n_DEM) */
    double *rho = (double *)malloc(sizeof(double) * nc);
    double *j = (double *)malloc(sizeof(double) * 3 * nc);
    double *P_tot = (double *)malloc(sizeof(double) * nc);
    double *gradP = (double *)malloc(sizeof(double) * 3 * nc);
    double *uD = (double *)malloc(sizeof(double) * 3 * nc);
    double *DuDt = (double *)malloc(sizeof(double) * 3 * nc);
    double *grad = (double *)malloc(sizeof(double) * 3 * nc);
    double *F = (double *)malloc(sizeof(double) * 3 * nc);
    double *fpf_k = (double *)malloc(sizeof(double) * 3 * nc);
    double *fpf_sum = (double *)malloc(sizeof(double) * 3 * nc);
    double *uf = (double *)malloc(sizeof(double) * 3 * nc);
    double *curl = (double *)malloc(sizeof(double) * 3 * nc);
    double *fnew = (double *)malloc(sizeof(double) * NQ * nc);
    double *F_am = (double *)malloc(sizeof(double) * 3 * (np > 0 ? np : 1));
    double *F_d = (double *)malloc(sizeof(double) * 3 * (np > 0 ? np : 1));
    if (!rho || !j || !P_tot || !gradP || !uD || !DuDt || !grad || !F || !fpf_k || !fpf_sum ||
        !uf || !curl || !fnew || !F_am || !F_d)
        return -1;

    for (long s = 0; s < nsteps; ++s) {
        orc_moments(P, S->f, rho, j);

        /* Algorithm 1: Du_f/Dt, once per time step.  reading: backward
         * difference of u_f between steps (zero on the first step) plus the
         * convective part (u_f . grad) u_f with the lattice gradient; u_f is
         * taken with the force density of the last LBM step. */
        for (int a = 0; a < 3; ++a)
            for (long c = 0; c < nc; ++c)
                F[a * nc + c] = S->eps_f[c] * P->f_b[a] + S->fpf[a * nc + c];
        fluid_velocity(nc, rho, j, S->eps_f, F, uD);
        if (!S->have_u_prev) memcpy(S->u_prev, uD, sizeof(double) * 3 * nc);
        for (long k = 0; k < 3 * nc; ++k) DuDt[k] = uD[k] - S->u_prev[k];
        for (int b = 0; b < 3; ++b) { /* DuDt_b += sum_a u_a d_a u_b */
            orc_lattice_gradient(P, &uD[b * nc], grad);
            for (int a = 0; a < 3; ++a)
                for (long c = 0; c < nc; ++c) DuDt[b * nc + c] += uD[a * nc + c] * grad[a * nc + c];
        }
        memcpy(S->u_prev, uD, sizeof(double) * 3 * nc);
        S->have_u_prev = 1;

        /* Table 1 / Sec. 3.2.3: total pressure P = eps_f p = c_s^2 rho */
        for (long c = 0; c < nc; ++c) P_tot[c] = CS2 * rho[c];
        orc_lattice_gradient(P, P_tot, gradP);

        for (long k = 0; k < 3 * nc; ++k) fpf_sum[k] = 0.0;

        for (int sub = 0; sub < P->n_int; ++sub) {
            /* reading: each subcycle starts from f_ext = eps_f f_b and adds only
             * its own particle reactions; the LBM step uses their average. */
            for (long k = 0; k < 3 * nc; ++k) fpf_k[k] = 0.0;

            /* Algorithm 1: u_f and its curl at the subcycle start (f_ext =
             * eps_f f_b), for the lift force */
            if (P->lift) {
                for (int a = 0; a < 3; ++a)
                    for (long c = 0; c < nc; ++c) F[a * nc + c] = S->eps_f[c] * P->f_b[a];
                fluid_velocity(nc, rho, j, S->eps_f, F, uf);
                orc_lattice_curl(P, uf, curl);
            }
            /* added mass: F_am = C_am rho_f V (Du_f/Dt|p - du_p/dt).
             * reading: du_p/dt is the change of u_p over the last subcycle.
             * The lift force (Table 1) is distributed together with it. */
            for (long i = 0; i < np; ++i) {
                double V = PI / 6.0 * S->d[i] * S->d[i] * S->d[i];
                double Dup[3], dudt[3];
                orc_interpolate(P, DuDt, 3, &S->x[3 * i], Dup);
                for (int a = 0; a < 3; ++a) {
                    dudt[a] = S->have_u_sub ? (S->u[3 * i + a] - S->u_sub[3 * i + a]) / dt_sub : 0.0;
                    S->u_sub[3 * i + a] = S->u[3 * i + a];
                    F_am[3 * i + a] = P->added_mass ? P->C_am * P->rho_f * V * (Dup[a] - dudt[a]) : 0.0;
                }
                if (P->lift) {
                    double ufp[3], wp[3], du[3], Fl[3];
                    orc_interpolate(P, uf, 3, &S->x[3 * i], ufp);
                    orc_interpolate(P, curl, 3, &S->x[3 * i], wp);
                    for (int a = 0; a < 3; ++a) du[a] = ufp[a] - S->u[3 * i + a];
                    orc_lift(S->d[i], mu, P->rho_f, du, wp, Fl);
                    for (int a = 0; a < 3; ++a) F_am[3 * i + a] += Fl[a];
                }
            }
            S->have_u_sub = 1;
            /* Eq. forces_pf (added-mass part) */
            orc_distribute(P, np, S->x, F_am, -1.0, fpf_k);

            /* re-evaluate u_f with the updated force density (Sec. 3.2.3) */
            for (int a = 0; a < 3; ++a)
                for (long c = 0; c < nc; ++c)
                    F[a * nc + c] = S->eps_f[c] * P->f_b[a] + fpf_k[a * nc + c];
            fluid_velocity(nc, rho, j, S->eps_f, F, uf);

            /* pressure-gradient, drag and gravity forces (Table 1) */
            for (long i = 0; i < np; ++i) {
                double di = S->d[i];
                double V = PI / 6.0 * di * di * di;
                double ufp[3], gPp[3], efp;
                orc_interpolate(P, uf, 3, &S->x[3 * i], ufp);
                orc_interpolate(P, gradP, 3, &S->x[3 * i], gPp);
                orc_interpolate(P, S->eps_f, 1, &S->x[3 * i], &efp);
                double epp = 1.0 - efp;
                double du[3], dun = 0.0;
                for (int a = 0; a < 3; ++a) {
                    du[a] = ufp[a] - S->u[3 * i + a];
                    dun += du[a] * du[a];
                }
                dun = sqrt(dun);
                double Re = orc_reynolds(efp, P->rho_f, di, dun, mu);
                double coef = P->drag ? 3.0 * PI * di * mu * (1.0 - epp) * orc_cd(Re, epp) : 0.0;
                for (int a = 0; a < 3; ++a) {
                    F_d[3 * i + a] = coef * du[a];
                    double Fpr = P->pressure ? -V * gPp[a] : 0.0;
                    /* Sec. 3.1.2: gravity on the particle plus buoyancy, as
                     * gravity does not act on the fluid */
                    double Fg = (S->rho_p[i] - P->rho_f) * V * P->g[a];
                    S->F_hyd[3 * i + a] = F_d[3 * i + a] + Fpr + F_am[3 * i + a] + Fg;
                }
            }
            /* Eq. forces_pf (drag part) */
            orc_distribute(P, np, S->x, F_d, -1.0, fpf_k);
            for (long k = 0; k < 3 * nc; ++k) fpf_sum[k] += fpf_k[k];

            /* DEM substeps with F_fp and F_g frozen (Sec. 3.3) */
            for (int sd = 0; sd < P->n_dem; ++sd) {
                orc_dem_forces(P, S, dt_dem);
                integrate(P, S, dt_dem);
            }

            /* re-evaluate the fluid volume fraction */
            S->n_eps_clamp += orc_fluid_fraction(P, np, S->x, S->d, S->eps_f);
        }
        for (long k = 0; k < 3 * nc; ++k) S->fpf[k] = fpf_sum[k] / P->n_int;

        /* GNS-LBM step with f_ext = f_pf + eps_f f_b */
        for (int a = 0; a < 3; ++a)
            for (long c = 0; c < nc; ++c)
                F[a * nc + c] = S->fpf[a * nc + c] + S->eps_f[c] * P->f_b[a];
        orc_collide_stream(P, S->f, S->eps_f, F, fnew);
        memcpy(S->f, fnew, sizeof(double) * NQ * nc);
        S->step++;
    }
    free(rho); free(j); free(P_tot); free(gradP); free(uD); free(DuDt); free(grad);
    free(F); free(fpf_k); free(fpf_sum); free(uf); free(curl); free(fnew); free(F_am); free(F_d);
    return 0;
}

/* Eq. hinderedCoefficientRZ */
double orc_rz_kappa(double Re_T) {
    if (Re_T < 0.2) return 4.65;
    if (Re_T < 1.0) return 4.35 * pow(Re_T, -0.03);
    if (Re_T < 500.0) return 4.45 * pow(Re_T, -0.1);
    return 2.39;
}
