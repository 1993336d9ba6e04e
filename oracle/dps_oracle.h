/*
 * dps_oracle.h -- FP64 CPU oracle for the coupled lattice Boltzmann / discrete
 * element step of Rettinger & Ruede, "A Coupled Lattice Boltzmann Method and
 * Discrete Element Method for Discrete Particle Simulations of Particulate
 * Flows" (arXiv:1711.00336).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, plain reference against which
 * the CUDA path is checked.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant with the CUDA library: every formula here is written out
 * again from the paper.
 *
 * Conventions (lattice units, Sec. 3.2.2: dx = dt = 1, c_s^2 = 1/3):
 *   - cell (ix,iy,iz) has its centre at (ix+0.5, iy+0.5, iz+0.5); the linear
 *     cell index is ix + nx*(iy + ny*iz) (x fastest);
 *   - PDFs are stored q-major: f[q*ncell + cell];
 *   - vector fields are component-major: v[a*ncell + cell];
 *   - particle vectors are interleaved: x[3*i + a].
 *
 * Function names follow the paper's notation; each definition cites the
 * section / equation it restates.
 */
#ifndef DPS_ORACLE_H
#define DPS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int n[3];            /* lattice cells per axis */
    int periodic[3];     /* 1: periodic axis, 0: no-slip walls at the faces 0 and n[a] */
    double tau;          /* relaxation time tau_e (Eq. LBM_Equation), constant */
    double rho_f;        /* fluid reference density used by the particle closures */
    double g[3];         /* gravitational acceleration, acts on the particles only */
    double f_b[3];       /* body force density on the fluid, applied as eps_f*f_b */
    double e_n;          /* dry coefficient of restitution (Eq. damping_to_stiffness) */
    double mu_c;         /* Coulomb friction coefficient */
    double T_c;          /* collision duration (Eq. collision_time) */
    double h_c;          /* lubrication cut-off gap */
    double h_min;        /* lower gap limit (Sec. 3.1.3) */
    double C_am;         /* added-mass coefficient (Table 1) */
    int n_int;           /* interaction subcycles per LBM step (Algorithm 1) */
    int n_dem;           /* DEM substeps per interaction subcycle */
    int drag, pressure, added_mass, lubrication, contact;  /* 0/1 toggles */
    int lub_limiter;     /* 1: cap lubrication coefficients at lub_cap*m_ij/dt_DEM */
    double lub_cap;
    double eps_min;      /* floor of eps_f */
    int pair_search;     /* 0: brute force O(N^2), 1: linked cells */
    int lift;            /* Table 1 shear lift (Saffman) with the lattice curl */
    int eilers;          /* Eq. visc_eilers: modified viscosity mu_* from eps_p */
    int smagorinsky;     /* Eqs. visc_turb, tau_t: Smagorinsky LES relaxation time */
} orc_params;

typedef struct {
    /* fluid */
    double *f;           /* [19*ncell] PDFs f_q(x,t) before the collision of step t */
    double *eps_f;       /* [ncell] fluid volume fraction */
    double *fpf;         /* [3*ncell] particle->fluid force density of the last LBM step
                            (average over its interaction subcycles) */
    double *u_prev;      /* [3*ncell] fluid velocity of the previous step (for Du/Dt) */
    int have_u_prev;
    /* particles */
    long np;
    double *x, *u, *w;   /* [3*np] position, velocity, angular velocity */
    double *d, *rho_p;   /* [np] diameter, density */
    double *u_sub;       /* [3*np] particle velocity at the start of the previous subcycle */
    int have_u_sub;
    double *F_hyd;       /* [3*np] frozen fluid-particle force + gravity of the last subcycle */
    double *F_c, *T_c, *F_lub;  /* [3*np] of the last DEM substep */
    /* counters */
    long n_eps_clamp;
    long n_lub_limited;
    long n_coincident;
    long step;
} orc_state;

/* lattice model (Sec. 3.2.2, D3Q19) */
void orc_lattice(int c[19][3], double w[19], int opp[19]);

/* Eq. filter_def: one-dimensional three-point discrete delta function */
double orc_phi(double r);
/* the 3 cells along one axis that a particle at xp touches, with their weights */
void orc_weights_1d(double xp, int L, int periodic, int idx[3], double wt[3]);
/* Eq. fluid_volume_fraction */
void orc_solid_fraction(const orc_params *P, long np, const double *x, const double *d,
                        double *eps_p);
long orc_fluid_fraction(const orc_params *P, long np, const double *x, const double *d,
                        double *eps_f);
/* Eq. distribution_filter: out[a*ncell+c] += scale * sum_i D(x_c, x_i) F[3*i+a] */
void orc_distribute(const orc_params *P, long np, const double *x, const double *F,
                    double scale, double *out);
/* Eq. interpolation: out[k] = sum_x I(x, xp) field[k*ncell + x], k < ncomp */
void orc_interpolate(const orc_params *P, const double *field, int ncomp,
                     const double xp[3], double *out);

/* Eq. LBM_EQ */
void orc_equilibrium(double rho, const double u[3], double eps, double feq[19]);
/* Eq. Forcing */
void orc_forcing(double tau, const double u[3], double eps, const double F[3], double Fq[19]);
/* Eq. MacVel (first two moments, without the force correction) */
void orc_moments(const orc_params *P, const double *f, double *rho, double *j);
/* Eq. LBM_Equation with halfway bounce-back walls: fnew from f */
void orc_collide_stream(const orc_params *P, const double *f, const double *eps,
                        const double *fext, double *fnew);
/* Sec. 3.2.3: lattice gradient of a scalar field */
void orc_lattice_gradient(const orc_params *P, const double *phi, double *grad);

/* Sec. 3.2.3: lattice curl of a vector field (3 planes) */
void orc_lattice_curl(const orc_params *P, const double *psi, double *curl);
/* Eq. visc_eilers (reading: (1 - eps_p/eps_cp) in the denominator) */
double orc_eilers_factor(double eps_p);
/* Eq. tau_t: Smagorinsky relaxation time from Qbar, tau_* and rho */
double orc_tau_turb(double tau_star, double Qbar, double rho);
/* per-cell relaxation time tau_e = tau_* + tau_t (Eq. tau_e) for the
 * pre-collision populations f of one cell */
double orc_tau_e(const orc_params *P, const double f[19], double rho, const double u[3], double eps);
/* Table 1: shear lift force on a particle */
void orc_lift(double d, double mu, double rho_f, const double du[3], const double w[3], double F[3]);

/* Table 1: drag coefficient and Reynolds number */
double orc_cd(double Re, double eps_p);
double orc_reynolds(double eps_f, double rho_f, double d, double du, double mu);

/* Sec. 3.1.1, Eqs. damping_to_stiffness / collision_time */
void orc_contact_constants(double m_ij, double e_n, double T_c, double *k_n, double *xi_n);
/* Sec. 3.1.3: raw lubrication coefficients a_sq and a_sh*(2/(h+<d>))^2 */
void orc_lub_coefficients(double dmean, double h, double mu, double *a_sq, double *a_sh_eff);

/* Sec. 3.1.1 + 3.1.3: contact, torque and lubrication on all particles */
void orc_dem_forces(const orc_params *P, orc_state *S, double dt_dem);
/* linked-cell list (neighbour search), for the bit-exact comparison of the sort */
void orc_cell_list(const orc_params *P, long np, const double *x, int B,
                   int *cell_start, int *order, int *key);

/* Algorithm 1 */
void orc_init(const orc_params *P, orc_state *S);
int  orc_step(const orc_params *P, orc_state *S, long nsteps);

/* Sec. 4: hindered settling correlation of Richardson and Zaki */
double orc_rz_kappa(double Re_T);

#ifdef __cplusplus
}
#endif
#endif
