/*
 * dps.h -- C ABI of the GB300 (sm_103a) discrete particle simulation library:
 * the coupled lattice Boltzmann / discrete element time step of Rettinger &
 * Ruede, "A Coupled Lattice Boltzmann Method and Discrete Element Method for
 * Discrete Particle Simulations of Particulate Flows", arXiv:1711.00336.
 *
 * Units are lattice units (Sec. 3.2.2): dx = dt = 1, c_s^2 = 1/3, rho_0 = 1.
 * A lattice cell (ix,iy,iz) has its centre at (ix+0.5, iy+0.5, iz+0.5) and the
 * linear index ix + nx*(iy + ny*iz) ("cell order", x fastest).  Positions of
 * periodic axes live in [0, n); non-periodic axes have no-slip walls at the
 * faces 0 and n (halfway bounce-back for the fluid, planar walls for the DEM).
 *
 * Conventions of every call:
 *   - every function returns an int status: DPS_OK (0) or a negative DPS_ERR_*;
 *     dps_last_error() gives a message for the last failure on a handle;
 *   - no C++ exception crosses this boundary;
 *   - the library owns every device buffer of a domain; the caller owns every
 *     host buffer it passes; each transfer is a copy (host pointers are read or
 *     written before the call returns);
 *   - calls on one handle are not thread-safe; distinct handles are independent;
 *   - a box holds at most 2^27 lattice cells;
 *   - the "op" entry points at the end work on caller-owned DEVICE buffers and
 *     are stream-ordered on the stream they are given.
 */
#ifndef DPS_H
#define DPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define DPS_OK            0
#define DPS_ERR_ARG      -1  /* invalid argument (size, pointer, parameter) */
#define DPS_ERR_OOM      -2  /* device allocation failed */
#define DPS_ERR_STATE    -3  /* call not valid in the current state */
#define DPS_ERR_UNSTABLE -4  /* NaN, non-positive density, or particles moved beyond the skin */
#define DPS_ERR_TIMEOUT  -5  /* a bounded device wait gave up */
#define DPS_ERR_CUDA     -6  /* a CUDA runtime call failed */

/* ---- precision forms --------------------------------------------------- */
#define DPS_F64  0  /* PDFs and fields FP64, FP64 arithmetic (the plain method) */
#define DPS_F32  1  /* PDFs stored FP32 as f_q - w_q*rho_0, fields and arithmetic FP32 */
#define DPS_F16S 2  /* PDFs stored FP16 as f_q - w_q*rho_0, fields and arithmetic FP32 */

/* ---- field masks for dps_read_fields / dps_write_fields ---------------- */
#define DPS_FIELD_RHO    0x001u  /* density rho_f = sum_q f_q (Eq. MacVel), 1 plane */
#define DPS_FIELD_UBAR   0x002u  /* volume-averaged velocity ubar (Eq. MacVel), 3 planes */
#define DPS_FIELD_UF     0x004u  /* fluid-phase velocity u_f = ubar/eps_f (Sec. 3.2.3), 3 planes */
#define DPS_FIELD_EPS    0x008u  /* fluid volume fraction eps_f (Eq. fluid_volume_fraction), 1 plane */
#define DPS_FIELD_FEXT   0x010u  /* f_ext = f_pf + eps_f f_b applied in the last LBM step, 3 planes */
#define DPS_FIELD_P      0x020u  /* pressure p = c_s^2 rho / eps_f (Sec. 3.2.2), 1 plane */
#define DPS_FIELD_FPF    0x040u  /* f_pf of the last LBM step (Eq. forces_pf, subcycle average), 3 planes */
#define DPS_FIELD_GRADP  0x080u  /* grad(eps_f p) of the current step (Sec. 3.2.3), 3 planes */
#define DPS_FIELD_DUDT   0x100u  /* Du_f/Dt of the current step (Table 1, added mass), 3 planes */

typedef struct dps_domain *dps_handle;

/* Device allocator hooks.  alloc returns a device pointer (NULL on failure,
 * which the library reports as DPS_ERR_OOM); free releases it.  Both NULL:
 * the library uses cudaMalloc / cudaFree. */
typedef void *(*dps_alloc_fn)(size_t bytes, void *ctx);
typedef void (*dps_free_fn)(void *ptr, void *ctx);

/* Domain description: the box and the fluid of Sec. 3.2 (Eq. GNS). */
typedef struct {
    int n[3];                 /* lattice cells per axis, each >= 1 */
    int periodic[3];          /* 1 periodic, 0 no-slip walls at both faces */
    double tau;               /* relaxation time tau_e (Eq. visc_tau), > 0.5 */
    double rho_f;             /* fluid density in the particle closures (rho_0 = 1) */
    int precision;            /* DPS_F64 / DPS_F32 / DPS_F16S */
    int64_t max_particles;    /* capacity of the particle arrays, >= 0 */
    void *stream;             /* cudaStream_t for all work; NULL: the library creates one */
    dps_alloc_fn alloc;       /* optional allocator hooks (see above) */
    dps_free_fn free;
    void *alloc_ctx;
} dps_domain_desc;

/* Closure: the models and constants of Sec. 3.1 and Algorithm 1. */
typedef struct {
    int drag;                 /* Table 1 drag (Tenneti et al.) */
    int pressure;             /* Table 1 pressure-gradient force */
    int added_mass;           /* Table 1 added-mass force */
    int lubrication;          /* Sec. 3.1.3 (Ball & Melrose), on pairs and walls that do not
                                 overlap and whose gap is below h_c (floored at h_min) */
    int contact;              /* Sec. 3.1.1 spring-dashpot contact */
    double g[3];              /* gravity, acting on the particles only (Sec. 3.1.2) */
    int fb_mode;              /* body force on the fluid, applied as eps_f*f_b:
                                 0 f_b = fb[3] as given,
                                 1 f_b balances the buoyant weight of all particles
                                   (f_b = -sum_i (rho_p,i - rho_f) V_i g / (cells - sum_i V_i)),
                                 2 the literal Sec. 4.1 form f_b = -<eps_p> (rho_p - rho_f) g */
    double fb[3];
    double e_n;               /* dry restitution (Eq. damping_to_stiffness), (0, 1] */
    double mu_c;              /* Coulomb friction coefficient */
    double T_c;               /* collision duration (Eq. collision_time), > 0 */
    double h_c;               /* lubrication cut-off gap, >= 0 */
    double h_min;             /* gap floor (Sec. 3.1.3: 1e-5 dx) */
    double C_am;              /* added-mass coefficient (Table 1: 0.5) */
    int n_int;                /* interaction subcycles per LBM step (Algorithm 1), >= 1 */
    int n_dem;                /* DEM substeps per subcycle, >= 1 */
    int lub_limiter;          /* 1: cap each lubrication coefficient at lub_cap*m_ij/dt_DEM */
    double lub_cap;
    double eps_min;           /* floor of eps_f, in (0, 1) */
    double skin;              /* neighbour-list skin in dx (>= 0): particles may move skin/2
                                 within one subcycle before DPS_ERR_UNSTABLE is raised */
    int lift;                 /* Table 1 shear lift 1.61 d^2 sqrt(mu rho_f/|w|) (u_f - u_p) x w, with
                                 w the lattice curl (Sec. 3.2.3) of u_f at the subcycle start; it is
                                 applied and distributed together with the added-mass force */
    int eilers;               /* Eq. visc_eilers: tau_* of each cell from the Eilers viscosity of its
                                 eps_p = 1 - eps_f (eps_p/eps_cp capped at 0.9); the particle closures
                                 keep the base viscosity of tau */
    int smagorinsky;          /* Eqs. visc_turb, tau_t, tau_e: Smagorinsky LES (C_S = 0.1) added to
                                 tau_* per cell from the non-equilibrium momentum flux */
} dps_closure;

/* Global sums (FP64, deterministic order). */
typedef struct {
    double mass;              /* sum_x rho */
    double fluid_j[3];        /* sum_x sum_q f_q c_q */
    double fluid_ubar[3];     /* sum_x ubar (with the applied f_ext) */
    double uf_mean[3];        /* mean over cells of u_f */
    double particle_momentum[3]; /* sum_i m_i u_i */
    double up_mean[3];        /* mean over particles of u_p */
    double u_pS[3];           /* <u_pS> of Sec. 4.1: up_mean - uf_mean */
    double eps_min_seen;      /* smallest eps_f before the floor */
    int64_t step;             /* LBM steps done */
    int64_t n_particles;
    int64_t n_eps_clamp;      /* cells floored at eps_min (cumulative) */
    int64_t n_lub_limited;    /* lubrication coefficients capped (cumulative) */
    int status;               /* sticky status bits, 0 when healthy */
} dps_stats;

/* ---- library ----------------------------------------------------------- */
const char *dps_version(void);
/* message of the last failing call on h (h may be NULL for create failures) */
const char *dps_last_error(dps_handle h);

/* ---- domain API -------------------------------------------------------- */

/* Create a domain: the lattice of Sec. 3.2.2 with the fluid at rest,
 * f_q = f_q^eq(rho_0 = 1, ubar = 0) = w_q, and no particles.
 * Errors: DPS_ERR_ARG (bad sizes, tau <= 0.5, unknown precision),
 * DPS_ERR_OOM, DPS_ERR_CUDA.  On failure *out is NULL. */
int dps_create_domain(const dps_domain_desc *desc, dps_handle *out);
int dps_destroy(dps_handle h);

/* Append n particles (Eq. particle_motion: position x, velocity u, angular
 * velocity w, diameter d, density rho_p).  x3/u3/w3 hold 3 doubles per
 * particle (x0,y0,z0,x1,...); u3 and w3 may be NULL (zero).  Positions on
 * periodic axes are wrapped into [0, n); on wall axes they must lie in
 * (0, n).  Errors: DPS_ERR_ARG (d <= 0, rho_p <= 0, position outside,
 * capacity exceeded, a particle-carrying axis shorter than 3 cells). */
int dps_add_particles(dps_handle h, int64_t n, const double *x3, const double *u3,
                      const double *w3, const double *d, const double *rho_p);

/* Overwrite the state (x, u, w) of all particles, in insertion order.  Used to
 * couple an external particle code; NULL arrays are left unchanged. */
int dps_write_particles(dps_handle h, int64_t n, const double *x3, const double *u3,
                        const double *w3);

/* Set the closure (all models and constants).  Must precede dps_step. */
int dps_set_closure(dps_handle h, const dps_closure *c);
/* The closure defaults of the paper's hindered-settling setup (Sec. 4.1):
 * all forces on, mu_c 0.25, e_n 0.88, h_c 1, h_min 1e-5, C_am 0.5, n_int 10,
 * n_dem 50, T_c 0.5, limiter on (cap 0.25), eps_min 0.05, skin 0.5, fb_mode 1. */
void dps_closure_defaults(dps_closure *c);

/* Algorithm 1 initialisation: sort the particles, evaluate eps_f and the
 * body force eps_f f_b.  dps_step calls it when particles changed. */
int dps_prepare(dps_handle h);

/* Run n coupled time steps of Algorithm 1 on the domain's stream, then wait
 * for them and check the device status word once.
 * Errors: DPS_ERR_STATE (no closure), DPS_ERR_UNSTABLE, DPS_ERR_CUDA. */
int dps_step(dps_handle h, int64_t n);
/* As dps_step but returns right after enqueueing (no wait, no status check);
 * dps_check() waits and reports the status accumulated since the last check. */
int dps_step_async(dps_handle h, int64_t n);
int dps_check(dps_handle h);
/* Run n steps of the GNS-LBM collide-stream only (Eq. LBM_Equation) with the
 * current eps_f and f_ext, without particles (fluid-only use). */
int dps_collide_stream(dps_handle h, int64_t n);
int dps_sync(dps_handle h);

/* Copy fields to the host.  out receives the planes of the requested fields in
 * mask-bit order, each plane ncell doubles in cell order (vectors as 3 planes
 * x,y,z).  cap = capacity of out in doubles.  Values are at the current time
 * (before the next step's collision), converted to FP64. */
int dps_read_fields(dps_handle h, uint32_t mask, double *out, int64_t cap);
/* Overwrite eps_f (DPS_FIELD_EPS) and/or f_pf (DPS_FIELD_FPF) from the host,
 * in the same layout.  Other mask bits are DPS_ERR_ARG. */
int dps_write_fields(dps_handle h, uint32_t mask, const double *in, int64_t count);
/* Read / write the PDFs f_q(x,t) at the current time: 19 planes of ncell
 * doubles in the lattice order of dps_lattice(). */
int dps_read_pdfs(dps_handle h, double *out, int64_t cap);
int dps_write_pdfs(dps_handle h, const double *in, int64_t count);
/* The D3Q19 velocities (19x3 ints) and weights of the PDF planes. */
void dps_lattice(int c[19][3], double w[19]);

/* Particles in insertion order: x, u, w and the frozen fluid-particle force
 * plus gravity F (Eq. particle_motion, F_fp + F_g) of the last subcycle.
 * Any pointer may be NULL.  cap = capacity in particles. */
int dps_read_particles(dps_handle h, double *x3, double *u3, double *w3, double *F3,
                       int64_t cap);
int dps_stats_get(dps_handle h, dps_stats *s);

/* ---- checkpoint / resume ------------------------------------------------- */
/* The state one coupled step of Algorithm 1 (Sec. 3.3) carries into the next,
 * copied into a caller-owned host buffer between steps: the PDFs f_q(x,t) as
 * stored (in the canonical layout, whatever the AA parity), eps_f (Eq.
 * fluid_volume_fraction), the f_pf applied in the last step (Eq. forces_pf),
 * the fluid velocity of the last step (for Du_f/Dt, Table 1), the particle
 * state of Eq. particle_motion (x, u, w, d, rho_p and the per-particle history:
 * u at the last subcycle start, the frozen forces), the step count, closure,
 * counters and status.  Linked cells, neighbour lists and the other derived
 * arrays are rebuilt on load by the initialisation sort, bit for bit as the
 * uninterrupted run holds them, so N steps + save + load (into a new domain)
 * + N steps gives the same bits as 2N steps.  The buffer format is private to
 * this library version (a header checks it).
 * dps_state_size: bytes of the checkpoint of h with its current particle count.
 * dps_save_state: waits for h's stream, writes the checkpoint into buf
 *   (cap bytes).  Errors: DPS_ERR_ARG (buf NULL or too small), DPS_ERR_CUDA.
 * dps_load_state: restores a checkpoint into h, which must have been created
 *   with the same n, periodic, tau, rho_f and precision and with
 *   max_particles >= the saved particle count; h's own particles and fluid are
 *   replaced.  Errors: DPS_ERR_ARG (not a checkpoint, truncated, or of another
 *   geometry / form), DPS_ERR_OOM, DPS_ERR_CUDA. */
int dps_state_size(dps_handle h, size_t *bytes);
int dps_save_state(dps_handle h, void *buf, size_t cap);
int dps_load_state(dps_handle h, const void *buf, size_t size);

/* The current linked-cell sort (the neighbour search of the DEM and the
 * gather of the coupling): cell_start[ncell+1] over cell keys, order[np] the
 * insertion indices in sorted order.  See dps_op_cell_sort for the key. */
int dps_read_cell_list(dps_handle h, int32_t *cell_start, int32_t *order, int64_t cap_cells,
                       int64_t cap_particles);
/* The neighbour (Verlet) list of the DEM substeps (Sec. 3.1, pairs that
 * the contact and lubrication laws may reach) as built at the last linked-
 * cell sort: for particle i (insertion order) every partner j != i whose
 * centre lay within (d_i + d_j)/2 + h_c + skin of x_i at that sort (minimum
 * image on periodic axes; the search compares in FP32 with a margin of 1e-3
 * dx, so pairs within that margin of the range may be listed), as CSR:
 * offsets[np + 1] (int64) and partners[offsets[np]] (insertion indices, each
 * row ascending).  partners may be NULL to learn offsets only; cap = capacity
 * of partners.  Errors: DPS_ERR_ARG (capacity), DPS_ERR_CUDA. */
int dps_read_neighbor_list(dps_handle h, int64_t *offsets, int32_t *partners, int64_t cap);
/* bin edge B (cells) chosen for the current closure */
int dps_bin_edge(dps_handle h, int *B);

/* ---- tracing: per-phase CUDA-event timing of the coupled step ---------- */
/* Phases, in the order of Algorithm 1:
 *   0 moments + fields (rho, j, u_f, grad P, Du_f/Dt)   1 added-mass force
 *   2 added-mass reaction gather                          3 drag/pressure/gravity force
 *   4 drag reaction gather                                5 DEM substeps
 *   6 linked-cell sort                                    7 eps_f gather
 *   8 collide-stream                                                                  */
#define DPS_NPHASE 9
/* enable / disable event pairs around every phase (captured into the step graph) */
int dps_set_timing(dps_handle h, int enable);
/* wait for the stream, then add the phase times of the last step to the totals */
int dps_collect_timing(dps_handle h);
/* totals since the last reset: milliseconds and kernel launches per phase */
int dps_get_timing(dps_handle h, double ms[DPS_NPHASE], int64_t launches[DPS_NPHASE], int reset);
/* number of kernels one coupled step launches with the current closure */
int dps_launches_per_step(dps_handle h, int64_t *n);

/* ---- batch API: many independent boxes advanced by one launch per phase --- */
/* A batch holds boxes of different sizes (each its own lattice, particles and
 * closure; n_int and n_dem must agree across the batch).  Every phase kernel
 * of the coupled step runs once for all boxes over a list of tiles (cells or
 * particles of one box), and the whole step is one CUDA graph replay.  Box ids
 * stay valid until the box is removed.  Results of a box do not depend on the
 * other boxes in the batch.  Errors as for the domain API. */
typedef struct dps_batch_s *dps_batch;
typedef struct {
    int precision;            /* DPS_F64 / DPS_F32 / DPS_F16S for every box */
    void *stream;             /* cudaStream_t; NULL: the library creates one */
    dps_alloc_fn alloc;       /* optional allocator hooks */
    dps_free_fn free;
    void *alloc_ctx;
} dps_batch_desc;

int dps_batch_create(const dps_batch_desc *desc, dps_batch *out);
/* message of the last failing call on b */
const char *dps_batch_last_error(dps_batch b);
int dps_batch_destroy(dps_batch b);
/* add a box (fluid at rest, no particles); *box receives its id */
int dps_batch_add_box(dps_batch b, const int n[3], const int periodic[3], double tau, double rho_f,
                      int64_t max_particles, int *box);
int dps_batch_remove_box(dps_batch b, int box);
int dps_batch_add_particles(dps_batch b, int box, int64_t n, const double *x3, const double *u3,
                            const double *w3, const double *d, const double *rho_p);
int dps_batch_set_closure(dps_batch b, int box, const dps_closure *c);
int dps_batch_step(dps_batch b, int64_t n);
int dps_batch_step_async(dps_batch b, int64_t n);
int dps_batch_check(dps_batch b);
int dps_batch_read_particles(dps_batch b, int box, double *x3, double *u3, double *w3, double *F3, int64_t cap);
int dps_batch_read_fields(dps_batch b, int box, uint32_t mask, double *out, int64_t cap);
int dps_batch_stats(dps_batch b, int box, dps_stats *s);
/* mean particle velocity of a box (FP64, fixed summation order) */
int dps_batch_particle_mean(dps_batch b, int box, double u[3]);
int dps_batch_num_boxes(dps_batch b, int *n);
/* checkpoint / resume of one box of a batch: the format and rules of
 * dps_save_state / dps_load_state.  A box restored into a batch at the other
 * AA parity has its PDFs moved to that parity's layout (a permutation of the
 * stored values, no arithmetic). */
int dps_batch_state_size(dps_batch b, int box, size_t *bytes);
int dps_batch_save_box(dps_batch b, int box, void *buf, size_t cap);
int dps_batch_load_box(dps_batch b, int box, const void *buf, size_t size);
/* launch shape: cfg = {cell threads/block, cells/tile, particle threads/block,
 * particles/tile, collide-stream variant 0 ... 7 (register budget and cells
 * per thread of the low-precision forms; ignored in FP64)} */
int dps_batch_set_tuning(dps_batch b, const int cfg[5]);
int dps_batch_get_tuning(dps_batch b, int cfg[5]);
/* autotuner: time every candidate launch shape for `steps` steps on the
 * current boxes (their state advances) and keep the fastest; ms[0] receives
 * the best time per step */
int dps_batch_autotune(dps_batch b, int steps, double *best_ms);
int dps_batch_set_timing(dps_batch b, int enable);
int dps_batch_collect_timing(dps_batch b);
int dps_batch_get_timing(dps_batch b, double ms[DPS_NPHASE], int64_t launches[DPS_NPHASE], int reset);
int dps_batch_launches_per_step(dps_batch b, int64_t *n);
/* device bytes one box needs (for admission by free HBM) */
int dps_box_bytes(int precision, const int n[3], int64_t max_particles, size_t *bytes);

/* ---- serving: continuous batching of settling-suspension runs ----------- */
/* A server owns a worker thread and one batch per subcycle class (n_int,
 * n_dem).  Requests (one periodic or walled box with its particles and
 * closure) queue on submit; the worker admits queued requests first come
 * first served, each into the batch of its class, while a slot (max_boxes
 * over all classes) is free and cudaMemGetInfo shows room for the box
 * (dps_box_bytes) plus the reserve, steps all running boxes in chunks (the
 * class batches concurrently, each on its own stream), samples each box's mean particle velocity every chunk and
 * retires a box once the mean over its last `window` steps changed by less
 * than rel_tol (relative, along g) from the window before, or after max_steps.
 * A box's result does not depend on which other requests shared the GPU. */
typedef struct dps_server_s *dps_server;
typedef struct {
    int precision;            /* form of every box */
    int device;               /* CUDA device of the worker thread */
    int max_boxes;            /* batch slots */
    size_t hbm_reserve_bytes; /* free HBM kept aside when admitting */
    int64_t chunk_steps;      /* steps between scheduling rounds (also the sampling period) */
} dps_serve_desc;
typedef struct {
    int n[3];
    int periodic[3];
    double tau, rho_f;
    int64_t np;                     /* particles; x3/d/rho_p are copied at submit */
    const double *x3, *d, *rho_p;
    dps_closure closure;
    int64_t max_steps;              /* cap (e.g. 20000) */
    int64_t window;                 /* steps per averaging window (a multiple of chunk_steps) */
    double rel_tol;                 /* convergence threshold on the windowed mean (e.g. 1e-3) */
} dps_request;
#define DPS_REQ_QUEUED 0
#define DPS_REQ_RUNNING 1
#define DPS_REQ_DONE 2
#define DPS_REQ_FAILED 3
#define DPS_REQ_CANCELLED 4
typedef struct {
    int state;                /* DPS_REQ_* */
    int capped;               /* 1 if stopped by max_steps */
    int status;               /* DPS_OK or the error of a failed run */
    int64_t steps;
    double up_mean[3];        /* windowed mean particle velocity at the end */
    double u_pS[3];           /* <u_pS> (Sec. 4.1) at the end */
    double t_submit, t_start, t_end;  /* seconds since the server started */
} dps_result;
typedef struct {
    int64_t submitted, admitted, completed, failed, running, queued;
    int peak_boxes;
    double cell_updates;      /* sum over boxes of cells x steps */
    double busy_s;            /* time with at least one running box */
    double wall_s;            /* since the server started */
} dps_serve_stats;

int dps_serve_create(const dps_serve_desc *desc, dps_server *out);
int dps_serve_submit(dps_server s, const dps_request *r, int64_t *id);
int dps_serve_poll(dps_server s, int64_t id, dps_result *res);
int dps_serve_cancel(dps_server s, int64_t id);
/* wait until nothing is queued or running (timeout in seconds, <0: forever);
 * DPS_ERR_TIMEOUT when the time runs out */
int dps_serve_wait_idle(dps_server s, double timeout_s);
int dps_serve_stats_get(dps_server s, dps_serve_stats *st);
int dps_serve_destroy(dps_server s);

/* ---- op API (caller-owned device buffers) ------------------------------- */

/* Linked-cell sort of np particles (device x3, 3 doubles each, interleaved;
 * device ids[np], the tie-break).  Lattice cells are grouped in bins of B
 * cells per axis (the last bin of an axis takes the remainder); the key of a
 * cell orders cells bin-major (bz,by,bx), then (z,y,x) inside the bin, so
 * that every bin and every cell is one contiguous key range.  Particles are
 * sorted by (key of the cell containing them, ids, input index): ids are the
 * tie-break of the method (the particle numbering) and should be distinct;
 * equal ids keep their input order.  Outputs (device): cell_start[ncell+1]
 * (exclusive prefix of the counts per key) and order[np] (input index of
 * each sorted slot).  Every coordinate must lie in [0, n) on its axis
 * (periodic axes already wrapped); the call waits for its stream to read a
 * status word back and returns DPS_ERR_ARG if some coordinate lies outside or
 * is not finite (the outputs then count such a particle in the clamped edge
 * cell).  Scratch is allocated on the stream (stream-ordered).
 * Errors: DPS_ERR_ARG, DPS_ERR_OOM, DPS_ERR_CUDA. */
int dps_op_cell_sort(const int n[3], const int periodic[3], int B, int64_t np,
                     const double *x3, const int32_t *ids, int32_t *cell_start, int32_t *order,
                     void *stream);

/* ---- measurement ----------------------------------------------------------- */
/* The paper has no counterpart: a property of the GPU, not of the method.
 * Measured FP64 throughput of the current device in GFLOP/s (independent
 * fused multiply-add chains on every SM, best of 5 timed launches, 2 flops
 * per FMA), the peak against which the FP64-bound kernels of this library
 * are reported.  Allocates 8 bytes of device memory for its run.
 * Errors: DPS_ERR_ARG (NULL), DPS_ERR_OOM, DPS_ERR_CUDA. */
int dps_probe_fp64_peak(double *gflops);

/* The natural logarithm of the FP64 lubrication term (Sec. 3.1.3, ln(<d>/2h))
 * evaluated for checking: a table-driven method (Tang, ACM TOMS 16(4),
 * 1990) whose error stays below one unit in the last place plus 2^-60.
 * y[i] = that logarithm of x[i], y_lib[i] = the C / CUDA library log of x[i],
 * for i < n (caller-owned host arrays).  device = 0: both computed on the
 * host (the same source as the device path, with every operation rounded to
 * nearest, so the two agree bit for bit); device != 0: on the current GPU
 * (allocates 24 n bytes of device memory for the call, synchronous).
 * Errors: DPS_ERR_ARG (n < 0 or a NULL array), DPS_ERR_OOM, DPS_ERR_CUDA. */
int dps_check_tlog(const double *x, double *y, double *y_lib, int64_t n, int device);

/* ---- allocation-free variant of the cell sort ---------------------------- */
/* The paper has no counterpart: this entry point is a property of the
 * library, not of the method.  dps_op_cell_sort takes its scratch memory
 * (per-cell counts, per-particle keys and permutation, scan partials) from the
 * stream-ordered allocator.  Callers that cannot allocate device memory while
 * they run -- a program that handed the whole device to its own pool
 * allocator, or a time-stepping loop that must not allocate (nor wait on an
 * allocation) once it is running -- call dps_op_cell_sort_noalloc instead: the
 * same sort, with its scratch in a fixed array compiled into the library
 * (about 5 MB held on every GPU that loads the library, until the process
 * exits).  Inputs, outputs and results are those of dps_op_cell_sort, for at
 * most DPS_NOALLOC_MAX_CELLS cells and DPS_NOALLOC_MAX_PARTICLES particles;
 * larger sizes return DPS_ERR_ARG.  It calls no cudaMalloc/cudaFree or other
 * allocating routine.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  The address is kept for the life of
 * the process: the library must not be used on a device after a
 * cudaDeviceReset of it.  Every call uses the one array and leaves its
 * contents behind: calls that overlap on the GPU (other streams or threads)
 * race, so the caller must serialise them.  Like dps_op_cell_sort it waits
 * for its stream to read the status word back. */
#define DPS_NOALLOC_MAX_CELLS 262144
#define DPS_NOALLOC_MAX_PARTICLES 262144
int dps_op_cell_sort_noalloc(const int n[3], const int periodic[3], int B, int64_t np, const double *x3,
                             const int32_t *ids, int32_t *cell_start, int32_t *order, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DPS_H */
