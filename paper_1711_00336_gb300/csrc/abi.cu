// abi.cu -- the C ABI of include/dps.h: domain lifetime, Algorithm 1 driver
// (one coupled step = a fixed sequence of kernel launches on the domain's
// stream, replayed as a CUDA graph once the history flags are set), status
// handling and host<->device copies.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dps_internal.cuh"

namespace dps {
// launchers (lbm.cu, coupling.cu, dem.cu, scan.cu, io.cu)
template <typename ST, typename FT, typename CT>
void launch_collide_stream(void *, const void *, const void *, const Geom &, const double *, double, int, int, int *,
                           cudaStream_t);
template <typename ST, typename FT, typename CT>
void launch_moments(const void *, const void *, const void *, const Geom &, const double *, int, void *, void *, void *,
                    cudaStream_t);
template <typename FT, typename CT>
void launch_fields(const void *, const void *, void *, const Geom &, int, void *, void *, cudaStream_t);
template <typename ST>
void launch_pdf_export(const void *, const Geom &, int, double *, cudaStream_t);
template <typename ST>
void launch_pdf_import(void *, long long, const double *, cudaStream_t);
void launch_sort_count(const double *, const double *, const double *, long long, long long, const Geom &, int *, int *,
                       int *, cudaStream_t);
void launch_sort_scatter(const int *, long long, const int *, int *, int *, cudaStream_t);
void launch_sort_rank(const int *, const int *, long long, const int *, const int *, int *, cudaStream_t);
void launch_sort_gather(const double *, const double *, const int *, long long, long long, const int *, const int *,
                        const Geom &, double *, int *, cudaStream_t);
template <typename FT>
void launch_eps(const Geom &, const int *, const double *, long long, double, void *, unsigned long long *, int *,
                cudaStream_t);
template <typename FT>
void launch_force_am(const Geom &, double *, const double *, long long, long long, const void *, const Phys &, int,
                     cudaStream_t);
template <typename FT>
void launch_force_drag(const Geom &, double *, const double *, long long, long long, const void *, const void *,
                       const void *, const void *, const void *, const Phys &, cudaStream_t);
template <typename FT>
void launch_reaction_am(const Geom &, const int *, const double *, long long, void *, cudaStream_t);
template <typename FT>
void launch_reaction_drag(const Geom &, const int *, const double *, long long, const void *, void *, void *, int, int,
                          double, cudaStream_t);
void launch_dem_substep(const double *, double *, const double *, const int *, long long, long long, int, const Geom &,
                        const Phys &, int *, unsigned long long *, cudaStream_t);
long long scan_scratch_words(long long);
void exclusive_scan(const int *, long long, int *, int *, cudaStream_t);
template <typename ST>
void launch_pdf_rest(void *, long long, cudaStream_t);
template <typename FT>
void launch_fill(void *, long long, double, cudaStream_t);
template <typename FT>
void launch_to_double(const void *, long long, double *, cudaStream_t);
template <typename FT>
void launch_from_double(const double *, long long, void *, cudaStream_t);
template <typename ST, typename FT>
void launch_fluid_export(const void *, const void *, const void *, const Geom &, const double *, int, int, double *,
                         cudaStream_t);
template <typename ST, typename FT>
void launch_fluid_sums(const void *, const void *, const void *, const Geom &, const double *, int, double *, double *,
                       cudaStream_t);
void launch_particle_sums(const double *, const double *, long long, long long, double *, double *, cudaStream_t);
void launch_particles_export(const double *, int, long long, long long, const int *, double *, cudaStream_t);
void launch_particles_import(double *, int, long long, long long, const int *, const double *, cudaStream_t);
long long reduce_partials_doubles();
}  // namespace dps

using namespace dps;

static const double PI_H = 3.14159265358979323846;

struct dps_domain {
    dps_domain_desc desc{};
    Geom g{};
    int prec = DPS_F64;
    size_t pdf_elem = 8, fel = 8;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    std::vector<void *> allocs;

    // fluid
    void *pdf = nullptr;
    void *eps = nullptr, *fpf = nullptr, *fam = nullptr, *acc = nullptr, *rho = nullptr, *j = nullptr,
         *uD = nullptr, *uprev = nullptr, *gradP = nullptr, *DuDt = nullptr;
    int parity = 0;
    int have_uprev = 0;

    // particles
    long long cap = 0, np = 0;
    double *pf[2] = {nullptr, nullptr};
    int *pi[2] = {nullptr, nullptr};
    double *xtmp = nullptr;
    int cur = 0;
    int have_usub = 0;
    double sumV = 0.0, sumWb = 0.0, dmax = 0.0;  // sum V, sum (rho_p - rho_f) V, max d

    // sort
    int *cell_start = nullptr, *count = nullptr, *fill = nullptr, *key = nullptr, *tmp = nullptr, *perm = nullptr,
        *scan_scratch = nullptr;

    // status
    int *d_status = nullptr;
    unsigned long long *d_counters = nullptr;
    double *d_red = nullptr, *d_redout = nullptr;
    int sticky = 0;

    // closure
    dps_closure cl{};
    bool have_closure = false;
    Phys ph{};
    int R = 1;
    bool prepared = false;
    long long step = 0;

    // graphs keyed by (parity, cur)
    cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};
    bool use_graphs = true;

    // tracing: event pairs around each phase of a step, in launch order
    bool timing = false;
    std::vector<cudaEvent_t> ev;     // 2 per phase instance
    std::vector<int> ev_phase, ev_nl;  // phase and kernel launches of each instance
    size_t ev_used = 0;
    double ph_ms[DPS_NPHASE] = {0};
    long long ph_nl[DPS_NPHASE] = {0};
    long long launches_step = 0;     // kernels per step (counted while enqueueing)
    long long launch_count = 0;
};

enum { PH_MOM = 0, PH_FAM, PH_RAM, PH_FDRAG, PH_RDRAG, PH_DEM, PH_SORT, PH_EPS, PH_COLLIDE };

static void tbegin(dps_domain *h) {
    if (!h->timing) return;
    if (h->ev_used * 2 + 2 > h->ev.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        h->ev.push_back(a);
        h->ev.push_back(b);
        h->ev_phase.push_back(0);
        h->ev_nl.push_back(0);
    }
    cudaEventRecord(h->ev[2 * h->ev_used], h->stream);
}
static void tend(dps_domain *h, int phase, int nlaunch) {
    h->launch_count += nlaunch;
    if (!h->timing) return;
    cudaEventRecord(h->ev[2 * h->ev_used + 1], h->stream);
    h->ev_phase[h->ev_used] = phase;
    h->ev_nl[h->ev_used] = nlaunch;
    h->ev_used++;
}

static thread_local std::string g_create_err;

#define FAIL(h, code, ...)                                   \
    do {                                                     \
        char _b[512];                                        \
        snprintf(_b, sizeof(_b), __VA_ARGS__);               \
        (h)->err = _b;                                       \
        return code;                                         \
    } while (0)

#define CK(h, call)                                                                         \
    do {                                                                                    \
        cudaError_t _e = (call);                                                            \
        if (_e != cudaSuccess) FAIL(h, DPS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
    } while (0)

static void *dalloc(dps_domain *h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (h->desc.alloc) {
        p = h->desc.alloc(bytes, h->desc.alloc_ctx);
    } else {
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    if (p) h->allocs.push_back(p);
    return p;
}

static void free_all(dps_domain *h) {
    for (int k = 0; k < 4; ++k)
        if (h->gexec[k]) cudaGraphExecDestroy(h->gexec[k]);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    h->ev.clear();
    for (void *p : h->allocs) {
        if (h->desc.free)
            h->desc.free(p, h->desc.alloc_ctx);
        else
            cudaFree(p);
    }
    h->allocs.clear();
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

static void invalidate_graphs(dps_domain *h) {
    for (int k = 0; k < 4; ++k)
        if (h->gexec[k]) {
            cudaGraphExecDestroy(h->gexec[k]);
            h->gexec[k] = nullptr;
        }
}

// ---- precision dispatch ------------------------------------------------------------------
#define DISPATCH_PREC(h, F64CALL, F32CALL, F16CALL) \
    do {                                            \
        if ((h)->prec == DPS_F64) {                 \
            F64CALL;                                \
        } else if ((h)->prec == DPS_F32) {          \
            F32CALL;                                \
        } else {                                    \
            F16CALL;                                \
        }                                           \
    } while (0)

static void k1(dps_domain *h, const double fb[3], int n_avg) {
    DISPATCH_PREC(h,
                  (launch_collide_stream<double, double, double>(h->pdf, h->eps, h->fpf, h->g, fb, h->desc.tau, n_avg,
                                                                 h->parity, h->d_status, h->stream)),
                  (launch_collide_stream<float, float, float>(h->pdf, h->eps, h->fpf, h->g, fb, h->desc.tau, n_avg,
                                                              h->parity, h->d_status, h->stream)),
                  (launch_collide_stream<__half, float, float>(h->pdf, h->eps, h->fpf, h->g, fb, h->desc.tau, n_avg,
                                                               h->parity, h->d_status, h->stream)));
}

static void k2(dps_domain *h) {
    const double *fb = h->ph.fb;
    DISPATCH_PREC(h,
                  (launch_moments<double, double, double>(h->pdf, h->eps, h->fpf, h->g, fb, h->parity, h->rho, h->j,
                                                          h->uD, h->stream)),
                  (launch_moments<float, float, float>(h->pdf, h->eps, h->fpf, h->g, fb, h->parity, h->rho, h->j, h->uD,
                                                       h->stream)),
                  (launch_moments<__half, float, float>(h->pdf, h->eps, h->fpf, h->g, fb, h->parity, h->rho, h->j,
                                                        h->uD, h->stream)));
    if (h->prec == DPS_F64)
        launch_fields<double, double>(h->rho, h->uD, h->uprev, h->g, h->have_uprev, h->gradP, h->DuDt, h->stream);
    else
        launch_fields<float, float>(h->rho, h->uD, h->uprev, h->g, h->have_uprev, h->gradP, h->DuDt, h->stream);
}

static int scan_launches(long long n) {
    const long long tile = 8192;
    if (n <= tile) return 1;
    return 2 + scan_launches((n + tile - 1) / tile);
}

static double *main_f(dps_domain *h) { return h->pf[h->cur]; }
static int *main_i(dps_domain *h) { return h->pi[h->cur]; }

// S1: sort by (containing cell, id), reorder into the other set, swap
static void do_sort(dps_domain *h, const double *xuw) {
    const long long N = h->g.ncell, cap = h->cap, np = h->np;
    cudaMemsetAsync(h->count, 0, sizeof(int) * N, h->stream);
    launch_sort_count(xuw, xuw + cap, xuw + 2 * cap, 1, np, h->g, h->count, h->key, h->d_status, h->stream);
    exclusive_scan(h->count, N, h->cell_start, h->scan_scratch, h->stream);
    cudaMemsetAsync(h->fill, 0, sizeof(int) * N, h->stream);
    launch_sort_scatter(h->key, np, h->cell_start, h->fill, h->tmp, h->stream);
    launch_sort_rank(h->key, main_i(h) + IID * cap, np, h->cell_start, h->tmp, h->perm, h->stream);
    int other = 1 - h->cur;
    launch_sort_gather(main_f(h), xuw, main_i(h), cap, np, h->perm, h->key, h->g, h->pf[other], h->pi[other],
                       h->stream);
    h->cur = other;
}

static void eps_eval(dps_domain *h) {
    if (h->prec == DPS_F64)
        launch_eps<double>(h->g, h->cell_start, main_f(h), h->cap, h->ph.eps_min, h->eps, h->d_counters, h->d_status,
                           h->stream);
    else
        launch_eps<float>(h->g, h->cell_start, main_f(h), h->cap, h->ph.eps_min, h->eps, h->d_counters, h->d_status,
                          h->stream);
}

// one coupled LBM step (Algorithm 1), enqueued on h->stream
static void enqueue_step(dps_domain *h) {
    const long long cap = h->cap, np = h->np;
    const Phys &ph = h->ph;
    const int pl = np > 0 ? 1 : 0;  // particle kernels are skipped without particles
    h->ev_used = 0;
    h->launch_count = 0;
    // Du_f/Dt and grad P once per step
    tbegin(h);
    k2(h);
    tend(h, PH_MOM, 2);
    h->have_uprev = 1;
    for (int k = 0; k < ph.n_int; ++k) {
        double *pf = main_f(h);
        const double *xuw = pf;  // x,u,w are in planes 0..8 of the main set after every sort
        const bool f64 = h->prec == DPS_F64;
        tbegin(h);
        if (f64) launch_force_am<double>(h->g, pf, xuw, cap, np, h->DuDt, ph, h->have_usub, h->stream);
        else launch_force_am<float>(h->g, pf, xuw, cap, np, h->DuDt, ph, h->have_usub, h->stream);
        tend(h, PH_FAM, pl);
        tbegin(h);
        if (f64) launch_reaction_am<double>(h->g, h->cell_start, pf, cap, h->fam, h->stream);
        else launch_reaction_am<float>(h->g, h->cell_start, pf, cap, h->fam, h->stream);
        tend(h, PH_RAM, 1);
        tbegin(h);
        if (f64) launch_force_drag<double>(h->g, pf, xuw, cap, np, h->rho, h->j, h->eps, h->fam, h->gradP, ph, h->stream);
        else launch_force_drag<float>(h->g, pf, xuw, cap, np, h->rho, h->j, h->eps, h->fam, h->gradP, ph, h->stream);
        tend(h, PH_FDRAG, pl);
        tbegin(h);
        if (f64)
            launch_reaction_drag<double>(h->g, h->cell_start, pf, cap, h->fam, h->acc, h->fpf, k == 0,
                                         k == ph.n_int - 1, 1.0 / ph.n_int, h->stream);
        else
            launch_reaction_drag<float>(h->g, h->cell_start, pf, cap, h->fam, h->acc, h->fpf, k == 0,
                                        k == ph.n_int - 1, 1.0 / ph.n_int, h->stream);
        tend(h, PH_RDRAG, 1);
        h->have_usub = 1;
        // DEM substeps: ping-pong between the main set's planes 0..8 and xtmp
        const double *xin = pf;
        double *xout = h->xtmp;
        tbegin(h);
        for (int s = 0; s < ph.n_dem; ++s) {
            launch_dem_substep(xin, xout, pf, h->cell_start, cap, np, h->R, h->g, ph, h->d_status, h->d_counters,
                               h->stream);
            const double *t = xin;
            xin = xout;
            xout = (double *)t;
        }
        tend(h, PH_DEM, pl * ph.n_dem);
        // re-sort with the new positions, then re-evaluate eps_f
        tbegin(h);
        do_sort(h, xin);
        tend(h, PH_SORT, scan_launches(h->g.ncell) + 4 * pl);
        tbegin(h);
        eps_eval(h);
        tend(h, PH_EPS, 1);
    }
    tbegin(h);
    k1(h, ph.fb, 1);
    tend(h, PH_COLLIDE, 1);
    h->launches_step = h->launch_count;
    h->parity ^= 1;
    h->step++;
}

static int check_status(dps_domain *h) {
    int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (st) {
        CK(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        h->sticky |= st;
        std::string m;
        if (st & ST_NAN) m += "non-finite or non-positive state; ";
        if (st & ST_SKIN) m += "a particle moved more than skin/2 within one subcycle (increase skin or n_int); ";
        if (st & ST_EPS_NEG) m += "eps_f < 0 before the floor; ";
        if (st & ST_BAD_CELL) m += "a particle left the box through a wall; ";
        FAIL(h, DPS_ERR_UNSTABLE, "unstable: %s", m.c_str());
    }
    return DPS_OK;
}

static void compute_phys(dps_domain *h) {
    const dps_closure &c = h->cl;
    Phys &p = h->ph;
    p.tau = h->desc.tau;
    p.omega = 1.0 / h->desc.tau;
    p.rho_f = h->desc.rho_f;
    p.mu = h->desc.rho_f * (h->desc.tau - 0.5) / 3.0;  // Eq. visc_tau
    for (int a = 0; a < 3; ++a) p.g[a] = c.g[a];
    const double cells = (double)h->g.ncell;
    for (int a = 0; a < 3; ++a) {
        if (c.fb_mode == 1)
            p.fb[a] = (cells - h->sumV) > 0 ? -h->sumWb * c.g[a] / (cells - h->sumV) : 0.0;
        else if (c.fb_mode == 2)
            p.fb[a] = h->np > 0 ? -(h->sumV / cells) * (h->sumWb / h->sumV) * c.g[a] : 0.0;
        else
            p.fb[a] = c.fb[a];
    }
    p.e_n = c.e_n;
    p.mu_c = c.mu_c;
    p.T_c = c.T_c;
    p.h_c = c.h_c;
    p.h_min = c.h_min;
    p.C_am = c.C_am;
    p.lub_cap = c.lub_cap;
    p.eps_min = c.eps_min;
    p.n_int = c.n_int;
    p.n_dem = c.n_dem;
    p.dt_sub = 1.0 / c.n_int;
    p.dt_dem = 1.0 / ((double)c.n_int * c.n_dem);
    p.drag = c.drag;
    p.pressure = c.pressure;
    p.added_mass = c.added_mass;
    p.lubrication = c.lubrication;
    p.contact = c.contact;
    p.lub_limiter = c.lub_limiter;
    const double cutoff = h->dmax + (c.lubrication ? std::fmax(c.h_c, 0.0) : 0.0);
    h->R = (int)std::floor(cutoff + c.skin) + 1;
    const double slack = h->R - cutoff;
    p.skin_half2 = 0.25 * slack * slack;
}

static int prepare(dps_domain *h) {
    if (!h->have_closure) FAIL(h, DPS_ERR_STATE, "dps_set_closure must be called first");
    compute_phys(h);
    do_sort(h, main_f(h));
    eps_eval(h);
    invalidate_graphs(h);
    h->prepared = true;
    return check_status(h);
}

// ===============================================================================================
extern "C" {

const char *dps_version(void) { return "dps-gb300 0.1 (sm_103a)"; }

const char *dps_last_error(dps_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

void dps_lattice(int c[19][3], double w[19]) {
    for (int q = 0; q < Q; ++q) {
        c[q][0] = CX(q);
        c[q][1] = CY(q);
        c[q][2] = CZ(q);
        w[q] = WQ(q);
    }
}

void dps_closure_defaults(dps_closure *c) {
    std::memset(c, 0, sizeof(*c));
    c->drag = c->pressure = c->added_mass = c->lubrication = c->contact = 1;
    c->fb_mode = 1;
    c->e_n = 0.88;
    c->mu_c = 0.25;
    c->T_c = 0.5;
    c->h_c = 1.0;
    c->h_min = 1e-5;
    c->C_am = 0.5;
    c->n_int = 10;
    c->n_dem = 50;
    c->lub_limiter = 1;
    c->lub_cap = 0.25;
    c->eps_min = 0.05;
    c->skin = 0.5;
}

int dps_create_domain(const dps_domain_desc *desc, dps_handle *out) {
    if (out) *out = nullptr;
    if (!desc || !out) {
        g_create_err = "null argument";
        return DPS_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if (desc->n[a] < 1) {
            g_create_err = "lattice size must be >= 1 per axis";
            return DPS_ERR_ARG;
        }
    long long ncell = (long long)desc->n[0] * desc->n[1] * desc->n[2];
    if (ncell >= (1LL << 31) - 1) {
        g_create_err = "lattice too large for 32-bit cell indices";
        return DPS_ERR_ARG;
    }
    if (!(desc->tau > 0.5) || !(desc->rho_f > 0.0) || desc->max_particles < 0 || desc->max_particles >= (1LL << 31) ||
        desc->precision < DPS_F64 || desc->precision > DPS_F16S || ((desc->alloc == nullptr) != (desc->free == nullptr))) {
        g_create_err = "invalid domain description (tau > 0.5, rho_f > 0, precision, particles, allocator pair)";
        return DPS_ERR_ARG;
    }
    dps_domain *h = new dps_domain();
    h->desc = *desc;
    h->prec = desc->precision;
    h->pdf_elem = desc->precision == DPS_F64 ? 8 : (desc->precision == DPS_F32 ? 4 : 2);
    h->fel = desc->precision == DPS_F64 ? 8 : 4;
    for (int a = 0; a < 3; ++a) {
        h->g.n[a] = desc->n[a];
        h->g.per[a] = desc->periodic[a] ? 1 : 0;
    }
    h->g.ncell = ncell;
    h->g.B = 1;
    for (int a = 0; a < 3; ++a) h->g.nb[a] = desc->n[a];
    h->cap = desc->max_particles > 0 ? desc->max_particles : 1;
    const char *env = getenv("DPS_NO_GRAPH");
    h->use_graphs = !(env && env[0] == '1');

    auto bail = [&](int code, const char *msg) {
        g_create_err = msg;
        free_all(h);
        delete h;
        return code;
    };
    const size_t N = (size_t)ncell, cap = (size_t)h->cap;
    // allocations (fluid, particles, sort, status)
    h->pdf = dalloc(h, (size_t)Q * N * h->pdf_elem);
    void **fields[] = {&h->eps, &h->rho};
    for (void **f : fields) *f = dalloc(h, N * h->fel);
    void **vec[] = {&h->fpf, &h->fam, &h->acc, &h->j, &h->uD, &h->uprev, &h->gradP, &h->DuDt};
    for (void **f : vec) *f = dalloc(h, 3 * N * h->fel);
    for (int s = 0; s < 2; ++s) {
        h->pf[s] = (double *)dalloc(h, (size_t)NPF * cap * sizeof(double));
        h->pi[s] = (int *)dalloc(h, (size_t)NPI * cap * sizeof(int));
    }
    h->xtmp = (double *)dalloc(h, 9 * cap * sizeof(double));
    h->cell_start = (int *)dalloc(h, (N + 1) * sizeof(int));
    h->count = (int *)dalloc(h, N * sizeof(int));
    h->fill = (int *)dalloc(h, N * sizeof(int));
    h->key = (int *)dalloc(h, cap * sizeof(int));
    h->tmp = (int *)dalloc(h, cap * sizeof(int));
    h->perm = (int *)dalloc(h, cap * sizeof(int));
    h->scan_scratch = (int *)dalloc(h, (size_t)scan_scratch_words((long long)N) * sizeof(int));
    h->d_status = (int *)dalloc(h, sizeof(int) * 4);
    h->d_counters = (unsigned long long *)dalloc(h, sizeof(unsigned long long) * CNT_N);
    h->d_red = (double *)dalloc(h, (size_t)reduce_partials_doubles() * sizeof(double));
    h->d_redout = (double *)dalloc(h, 32 * sizeof(double));
    for (void *p : {(void *)h->pdf, h->eps, h->rho, h->fpf, h->fam, h->acc, h->j, h->uD, h->uprev, h->gradP, h->DuDt,
                    (void *)h->pf[0], (void *)h->pf[1], (void *)h->pi[0], (void *)h->pi[1], (void *)h->xtmp,
                    (void *)h->cell_start, (void *)h->count, (void *)h->fill, (void *)h->key, (void *)h->tmp,
                    (void *)h->perm, (void *)h->scan_scratch, (void *)h->d_status, (void *)h->d_counters,
                    (void *)h->d_red, (void *)h->d_redout})
        if (!p) return bail(DPS_ERR_OOM, "device allocation failed");

    if (desc->stream) {
        h->stream = (cudaStream_t)desc->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return bail(DPS_ERR_CUDA, "cudaStreamCreate failed");
        }
        h->own_stream = true;
    }
    // fluid at rest: f = w_q, eps_f = 1, all force fields zero
    cudaStream_t s = h->stream;
    DISPATCH_PREC(h, launch_pdf_rest<double>(h->pdf, ncell, s), launch_pdf_rest<float>(h->pdf, ncell, s),
                  launch_pdf_rest<__half>(h->pdf, ncell, s));
    if (h->prec == DPS_F64)
        launch_fill<double>(h->eps, ncell, 1.0, s);
    else
        launch_fill<float>(h->eps, ncell, 1.0, s);
    for (void *p : {h->fpf, h->fam, h->acc, h->j, h->uD, h->uprev, h->gradP, h->DuDt})
        cudaMemsetAsync(p, 0, 3 * N * h->fel, s);
    cudaMemsetAsync(h->rho, 0, N * h->fel, s);
    for (int k = 0; k < 2; ++k) {
        cudaMemsetAsync(h->pf[k], 0, (size_t)NPF * cap * sizeof(double), s);
        cudaMemsetAsync(h->pi[k], 0, (size_t)NPI * cap * sizeof(int), s);
    }
    cudaMemsetAsync(h->cell_start, 0, (N + 1) * sizeof(int), s);
    cudaMemsetAsync(h->d_status, 0, sizeof(int) * 4, s);
    cudaMemsetAsync(h->d_counters, 0, sizeof(unsigned long long) * CNT_N, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return bail(DPS_ERR_CUDA, "initialisation kernels failed");
    *out = h;
    return DPS_OK;
}

int dps_destroy(dps_handle h) {
    if (!h) return DPS_ERR_ARG;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
    return DPS_OK;
}

int dps_add_particles(dps_handle h, int64_t n, const double *x3, const double *u3, const double *w3, const double *d,
                      const double *rho_p) {
    if (!h) return DPS_ERR_ARG;
    if (n < 0 || (n > 0 && (!x3 || !d || !rho_p))) FAIL(h, DPS_ERR_ARG, "bad particle arrays");
    if (n == 0) return DPS_OK;
    if (h->np + n > h->desc.max_particles) FAIL(h, DPS_ERR_ARG, "capacity exceeded (%lld + %lld > %lld)",
                                                (long long)h->np, (long long)n, (long long)h->desc.max_particles);
    for (int a = 0; a < 3; ++a)
        if (h->g.n[a] < 3) FAIL(h, DPS_ERR_ARG, "particles need at least 3 cells per axis");
    const long long cap = h->cap;
    std::vector<double> st((size_t)11 * n);  // planes x,y,z,u,v,w,ox,oy,oz,d,rho
    std::vector<int> ids((size_t)n);
    double sV = 0, sW = 0, dm = h->dmax;
    for (long long i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            double x = x3[3 * i + a];
            if (!std::isfinite(x)) FAIL(h, DPS_ERR_ARG, "non-finite position");
            const int L = h->g.n[a];
            if (h->g.per[a]) {
                x -= L * std::floor(x / L);
                if (x >= L) x -= L;
            } else if (!(x > 0.0 && x < L)) {
                FAIL(h, DPS_ERR_ARG, "particle %lld outside the walls on axis %d", i, a);
            }
            st[(size_t)a * n + i] = x;
            st[(size_t)(3 + a) * n + i] = u3 ? u3[3 * i + a] : 0.0;
            st[(size_t)(6 + a) * n + i] = w3 ? w3[3 * i + a] : 0.0;
        }
        if (!(d[i] > 0.0) || !(rho_p[i] > 0.0)) FAIL(h, DPS_ERR_ARG, "d and rho_p must be > 0");
        st[(size_t)9 * n + i] = d[i];
        st[(size_t)10 * n + i] = rho_p[i];
        ids[i] = (int)(h->np + i);
        double V = PI_H / 6.0 * d[i] * d[i] * d[i];
        sV += V;
        sW += (rho_p[i] - h->desc.rho_f) * V;
        dm = std::fmax(dm, d[i]);
    }
    double *pf = main_f(h);
    const long long off = h->np;
    for (int f = 0; f < 11; ++f)
        CK(h, cudaMemcpyAsync(pf + (size_t)f * cap + off, st.data() + (size_t)f * n, sizeof(double) * n,
                              cudaMemcpyHostToDevice, h->stream));
    // u at the start of the previous subcycle := u (no acceleration history yet)
    for (int a = 0; a < 3; ++a)
        CK(h, cudaMemcpyAsync(pf + (size_t)(PUS0 + a) * cap + off, st.data() + (size_t)(3 + a) * n, sizeof(double) * n,
                              cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(main_i(h) + IID * cap + off, ids.data(), sizeof(int) * n, cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->np += n;
    h->sumV += sV;
    h->sumWb += sW;
    h->dmax = dm;
    h->prepared = false;
    return DPS_OK;
}

int dps_write_particles(dps_handle h, int64_t n, const double *x3, const double *u3, const double *w3) {
    if (!h) return DPS_ERR_ARG;
    if (n != h->np) FAIL(h, DPS_ERR_ARG, "n must equal the number of particles (%lld)", (long long)h->np);
    if (n == 0) return DPS_OK;
    double *buf = nullptr;
    CK(h, cudaMallocAsync((void **)&buf, sizeof(double) * 3 * n, h->stream));
    const double *src[3] = {x3, u3, w3};
    for (int k = 0; k < 3; ++k) {
        if (!src[k]) continue;
        if (k == 0)
            for (long long i = 0; i < 3 * n; ++i)
                if (!std::isfinite(x3[i])) {
                    cudaFreeAsync(buf, h->stream);
                    FAIL(h, DPS_ERR_ARG, "non-finite position");
                }
        CK(h, cudaMemcpyAsync(buf, src[k], sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream));
        launch_particles_import(main_f(h), 3 * k, h->cap, n, main_i(h) + IID * h->cap, buf, h->stream);
    }
    CK(h, cudaFreeAsync(buf, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (x3) h->prepared = false;
    return DPS_OK;
}

int dps_set_closure(dps_handle h, const dps_closure *c) {
    if (!h || !c) return DPS_ERR_ARG;
    if (c->n_int < 1 || c->n_dem < 1 || !(c->e_n > 0.0 && c->e_n <= 1.0) || !(c->T_c > 0.0) || !(c->h_c >= 0.0) ||
        !(c->h_min > 0.0) || !(c->mu_c >= 0.0) || !(c->eps_min > 0.0 && c->eps_min < 1.0) || !(c->skin >= 0.0) ||
        !(c->lub_cap > 0.0) || c->fb_mode < 0 || c->fb_mode > 2)
        FAIL(h, DPS_ERR_ARG, "invalid closure parameter");
    h->cl = *c;
    h->have_closure = true;
    h->prepared = false;
    return DPS_OK;
}

int dps_prepare(dps_handle h) {
    if (!h) return DPS_ERR_ARG;
    return prepare(h);
}

static int run_steps(dps_handle h, int64_t n) {
    if (!h->have_closure) FAIL(h, DPS_ERR_STATE, "dps_set_closure must be called first");
    if (!h->prepared) {
        int rc = prepare(h);
        if (rc) return rc;
    }
    for (int64_t s = 0; s < n; ++s) {
        if (!h->use_graphs || !h->have_uprev || !h->have_usub) {
            enqueue_step(h);
            continue;
        }
        const int key = h->parity * 2 + h->cur;
        if (!h->gexec[key]) {
            const int p0 = h->parity, c0 = h->cur;
            const long long st0 = h->step;
            cudaGraph_t graph;
            CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
            enqueue_step(h);
            CK(h, cudaStreamEndCapture(h->stream, &graph));
            cudaError_t e = cudaGraphInstantiate(&h->gexec[key], graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) FAIL(h, DPS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
            // the capture only recorded the step: restore the host state
            h->parity = p0;
            h->cur = c0;
            h->step = st0;
        }
        CK(h, cudaGraphLaunch(h->gexec[key], h->stream));
        // advance the host-side state exactly as the step would
        h->parity ^= 1;
        if (h->ph.n_int & 1) h->cur ^= 1;
        h->step++;
    }
    return DPS_OK;
}

int dps_step_async(dps_handle h, int64_t n) {
    if (!h || n < 0) return DPS_ERR_ARG;
    int rc = run_steps(h, n);
    if (rc) return rc;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) FAIL(h, DPS_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    return DPS_OK;
}

int dps_check(dps_handle h) {
    if (!h) return DPS_ERR_ARG;
    return check_status(h);
}

int dps_step(dps_handle h, int64_t n) {
    int rc = dps_step_async(h, n);
    if (rc) return rc;
    return check_status(h);
}

int dps_collide_stream(dps_handle h, int64_t n) {
    if (!h || n < 0) return DPS_ERR_ARG;
    double fb[3] = {0, 0, 0};
    if (h->have_closure) {
        compute_phys(h);
        for (int a = 0; a < 3; ++a) fb[a] = h->ph.fb[a];
    }
    for (int64_t s = 0; s < n; ++s) {
        k1(h, fb, 1);
        h->parity ^= 1;
    }
    return check_status(h);
}

int dps_sync(dps_handle h) {
    if (!h) return DPS_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    return DPS_OK;
}

static const double *current_fb(dps_handle h) {
    static thread_local double zero[3] = {0, 0, 0};
    if (!h->have_closure) return zero;
    compute_phys(h);
    return h->ph.fb;
}

int dps_read_fields(dps_handle h, uint32_t mask, double *out, int64_t cap) {
    if (!h || (!out && mask)) return DPS_ERR_ARG;
    if (mask & ~0x1FFu) FAIL(h, DPS_ERR_ARG, "unknown field bits");
    const long long N = h->g.ncell;
    static const int planes[9] = {1, 3, 3, 1, 3, 1, 3, 3, 3};
    long long need = 0;
    for (int b = 0; b < 9; ++b)
        if (mask & (1u << b)) need += planes[b] * N;
    if (cap < need) FAIL(h, DPS_ERR_ARG, "output capacity %lld < %lld", (long long)cap, need);
    if (h->have_closure && !h->prepared) {
        int rc = prepare(h);
        if (rc) return rc;
    }
    const double *fb = current_fb(h);
    double *buf = nullptr;
    CK(h, cudaMallocAsync((void **)&buf, sizeof(double) * 3 * N, h->stream));
    long long off = 0;
    for (int b = 0; b < 9; ++b) {
        if (!(mask & (1u << b))) continue;
        const uint32_t bit = 1u << b;
        if (bit == DPS_FIELD_RHO || bit == DPS_FIELD_UBAR || bit == DPS_FIELD_UF || bit == DPS_FIELD_P ||
            bit == DPS_FIELD_FEXT) {
            int what = bit == DPS_FIELD_RHO ? 0 : bit == DPS_FIELD_UBAR ? 1 : bit == DPS_FIELD_UF ? 2 : bit == DPS_FIELD_P ? 3 : 4;
            DISPATCH_PREC(h, (launch_fluid_export<double, double>(h->pdf, h->eps, h->fpf, h->g, fb, h->parity, what, buf, h->stream)),
                          (launch_fluid_export<float, float>(h->pdf, h->eps, h->fpf, h->g, fb, h->parity, what, buf, h->stream)),
                          (launch_fluid_export<__half, float>(h->pdf, h->eps, h->fpf, h->g, fb, h->parity, what, buf, h->stream)));
        } else {
            const void *src = bit == DPS_FIELD_EPS ? h->eps : bit == DPS_FIELD_FPF ? h->fpf : bit == DPS_FIELD_GRADP ? h->gradP : h->DuDt;
            if (h->fel == 8)
                launch_to_double<double>(src, planes[b] * N, buf, h->stream);
            else
                launch_to_double<float>(src, planes[b] * N, buf, h->stream);
        }
        CK(h, cudaMemcpyAsync(out + off, buf, sizeof(double) * planes[b] * N, cudaMemcpyDeviceToHost, h->stream));
        off += planes[b] * N;
    }
    CK(h, cudaFreeAsync(buf, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return DPS_OK;
}

int dps_write_fields(dps_handle h, uint32_t mask, const double *in, int64_t count) {
    if (!h || !in) return DPS_ERR_ARG;
    if (mask & ~(DPS_FIELD_EPS | DPS_FIELD_FPF)) FAIL(h, DPS_ERR_ARG, "only eps_f and f_pf can be written");
    const long long N = h->g.ncell;
    long long need = ((mask & DPS_FIELD_EPS) ? N : 0) + ((mask & DPS_FIELD_FPF) ? 3 * N : 0);
    if (count < need) FAIL(h, DPS_ERR_ARG, "input has %lld values, %lld needed", (long long)count, need);
    double *buf = nullptr;
    CK(h, cudaMallocAsync((void **)&buf, sizeof(double) * 3 * N, h->stream));
    long long off = 0;
    if (mask & DPS_FIELD_EPS) {
        for (long long c = 0; c < N; ++c)
            if (!(in[c] > 0.0 && in[c] <= 1.0)) {
                cudaFreeAsync(buf, h->stream);
                FAIL(h, DPS_ERR_ARG, "eps_f must lie in (0, 1]");
            }
        CK(h, cudaMemcpyAsync(buf, in, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
        if (h->fel == 8) launch_from_double<double>(buf, N, h->eps, h->stream);
        else launch_from_double<float>(buf, N, h->eps, h->stream);
        off += N;
    }
    if (mask & DPS_FIELD_FPF) {
        CK(h, cudaMemcpyAsync(buf, in + off, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, h->stream));
        if (h->fel == 8) launch_from_double<double>(buf, 3 * N, h->fpf, h->stream);
        else launch_from_double<float>(buf, 3 * N, h->fpf, h->stream);
    }
    CK(h, cudaFreeAsync(buf, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return DPS_OK;
}

int dps_read_pdfs(dps_handle h, double *out, int64_t cap) {
    if (!h || !out) return DPS_ERR_ARG;
    const long long N = h->g.ncell;
    if (cap < (long long)Q * N) FAIL(h, DPS_ERR_ARG, "output capacity too small");
    double *buf = nullptr;
    CK(h, cudaMallocAsync((void **)&buf, sizeof(double) * Q * N, h->stream));
    DISPATCH_PREC(h, launch_pdf_export<double>(h->pdf, h->g, h->parity, buf, h->stream),
                  launch_pdf_export<float>(h->pdf, h->g, h->parity, buf, h->stream),
                  launch_pdf_export<__half>(h->pdf, h->g, h->parity, buf, h->stream));
    CK(h, cudaMemcpyAsync(out, buf, sizeof(double) * Q * N, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaFreeAsync(buf, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return DPS_OK;
}

int dps_write_pdfs(dps_handle h, const double *in, int64_t count) {
    if (!h || !in) return DPS_ERR_ARG;
    const long long N = h->g.ncell;
    if (count < (long long)Q * N) FAIL(h, DPS_ERR_ARG, "input too small");
    double *buf = nullptr;
    CK(h, cudaMallocAsync((void **)&buf, sizeof(double) * Q * N, h->stream));
    CK(h, cudaMemcpyAsync(buf, in, sizeof(double) * Q * N, cudaMemcpyHostToDevice, h->stream));
    DISPATCH_PREC(h, launch_pdf_import<double>(h->pdf, N, buf, h->stream), launch_pdf_import<float>(h->pdf, N, buf, h->stream),
                  launch_pdf_import<__half>(h->pdf, N, buf, h->stream));
    CK(h, cudaFreeAsync(buf, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->parity = 0;
    invalidate_graphs(h);
    return DPS_OK;
}

int dps_read_particles(dps_handle h, double *x3, double *u3, double *w3, double *F3, int64_t cap) {
    if (!h) return DPS_ERR_ARG;
    const long long np = h->np;
    if (cap < np) FAIL(h, DPS_ERR_ARG, "capacity %lld < %lld particles", (long long)cap, np);
    if (np == 0) return DPS_OK;
    double *buf = nullptr;
    CK(h, cudaMallocAsync((void **)&buf, sizeof(double) * 3 * np, h->stream));
    double *dst[4] = {x3, u3, w3, F3};
    const int plane[4] = {PX, PU, POX, PFH0};
    for (int k = 0; k < 4; ++k) {
        if (!dst[k]) continue;
        launch_particles_export(main_f(h), plane[k], h->cap, np, main_i(h) + IID * h->cap, buf, h->stream);
        CK(h, cudaMemcpyAsync(dst[k], buf, sizeof(double) * 3 * np, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaFreeAsync(buf, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return DPS_OK;
}

int dps_stats_get(dps_handle h, dps_stats *s) {
    if (!h || !s) return DPS_ERR_ARG;
    std::memset(s, 0, sizeof(*s));
    const double *fb = current_fb(h);
    double fl[12], pt[6];
    DISPATCH_PREC(h, (launch_fluid_sums<double, double>(h->pdf, h->eps, h->fpf, h->g, fb, h->parity, h->d_red, h->d_redout, h->stream)),
                  (launch_fluid_sums<float, float>(h->pdf, h->eps, h->fpf, h->g, fb, h->parity, h->d_red, h->d_redout, h->stream)),
                  (launch_fluid_sums<__half, float>(h->pdf, h->eps, h->fpf, h->g, fb, h->parity, h->d_red, h->d_redout, h->stream)));
    CK(h, cudaMemcpyAsync(fl, h->d_redout, sizeof(fl), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    launch_particle_sums(main_f(h), main_f(h), h->cap, h->np, h->d_red, h->d_redout, h->stream);
    CK(h, cudaMemcpyAsync(pt, h->d_redout, sizeof(pt), cudaMemcpyDeviceToHost, h->stream));
    unsigned long long cnt[CNT_N];
    CK(h, cudaMemcpyAsync(cnt, h->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
    int st = 0;
    CK(h, cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    const double N = (double)h->g.ncell;
    s->mass = fl[0];
    for (int a = 0; a < 3; ++a) {
        s->fluid_j[a] = fl[1 + a];
        s->fluid_ubar[a] = fl[4 + a];
        s->uf_mean[a] = fl[7 + a] / N;
        s->particle_momentum[a] = pt[a];
        s->up_mean[a] = h->np ? pt[3 + a] / h->np : 0.0;
        s->u_pS[a] = s->up_mean[a] - s->uf_mean[a];
    }
    s->eps_min_seen = fl[10];
    s->step = h->step;
    s->n_particles = h->np;
    s->n_eps_clamp = (int64_t)cnt[CNT_EPS_CLAMP];
    s->n_lub_limited = (int64_t)cnt[CNT_LUB_LIMITED];
    s->status = h->sticky | st;
    return DPS_OK;
}

int dps_read_cell_list(dps_handle h, int32_t *cell_start, int32_t *order, int64_t cap_cells, int64_t cap_particles) {
    if (!h || !cell_start || !order) return DPS_ERR_ARG;
    if (cap_cells < h->g.ncell + 1 || cap_particles < h->np) FAIL(h, DPS_ERR_ARG, "capacity too small");
    if (h->have_closure && !h->prepared) {
        int rc = prepare(h);
        if (rc) return rc;
    }
    CK(h, cudaMemcpyAsync(cell_start, h->cell_start, sizeof(int) * (h->g.ncell + 1), cudaMemcpyDeviceToHost, h->stream));
    if (h->np)
        CK(h, cudaMemcpyAsync(order, main_i(h) + IID * h->cap, sizeof(int) * h->np, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return DPS_OK;
}

int dps_bin_edge(dps_handle h, int *B) {
    if (!h || !B) return DPS_ERR_ARG;
    if (!h->have_closure) FAIL(h, DPS_ERR_STATE, "no closure");
    compute_phys(h);
    *B = h->R;
    return DPS_OK;
}

int dps_set_timing(dps_handle h, int enable) {
    if (!h) return DPS_ERR_ARG;
    if ((enable != 0) != h->timing) {
        CK(h, cudaStreamSynchronize(h->stream));
        h->timing = enable != 0;
        invalidate_graphs(h);
    }
    return DPS_OK;
}

int dps_collect_timing(dps_handle h) {
    if (!h) return DPS_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    if (!h->timing) return DPS_OK;
    for (size_t k = 0; k < h->ev_used; ++k) {
        float ms = 0.f;
        CK(h, cudaEventElapsedTime(&ms, h->ev[2 * k], h->ev[2 * k + 1]));
        h->ph_ms[h->ev_phase[k]] += ms;
        h->ph_nl[h->ev_phase[k]] += h->ev_nl[k];
    }
    return DPS_OK;
}

int dps_get_timing(dps_handle h, double ms[DPS_NPHASE], int64_t launches[DPS_NPHASE], int reset) {
    if (!h) return DPS_ERR_ARG;
    for (int k = 0; k < DPS_NPHASE; ++k) {
        if (ms) ms[k] = h->ph_ms[k];
        if (launches) launches[k] = h->ph_nl[k];
        if (reset) {
            h->ph_ms[k] = 0;
            h->ph_nl[k] = 0;
        }
    }
    return DPS_OK;
}

int dps_launches_per_step(dps_handle h, int64_t *n) {
    if (!h || !n) return DPS_ERR_ARG;
    if (!h->have_closure) FAIL(h, DPS_ERR_STATE, "no closure");
    compute_phys(h);
    const int pl = h->np > 0 ? 1 : 0;
    *n = 2 + 1 + (long long)h->ph.n_int * (pl * 2 + 2 + pl * h->ph.n_dem + scan_launches(h->g.ncell) + 4 * pl + 1);
    return DPS_OK;
}

int dps_op_cell_sort(const int n[3], const int periodic[3], int B, int64_t np, const double *x3, const int32_t *ids,
                     int32_t *cell_start, int32_t *order, void *stream) {
    if (!n || !periodic || np < 0 || (np > 0 && (!x3 || !ids || !order)) || !cell_start) return DPS_ERR_ARG;
    if (B != 1) return DPS_ERR_ARG;  // cells of one lattice spacing
    Geom g{};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1) return DPS_ERR_ARG;
        g.n[a] = n[a];
        g.per[a] = periodic[a] ? 1 : 0;
        g.nb[a] = n[a];
    }
    g.B = 1;
    g.ncell = (long long)n[0] * n[1] * n[2];
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = g.ncell;
    int *scr = nullptr;
    const long long words = 2 * N + 3 * (np > 0 ? np : 1) + scan_scratch_words(N) + 4;
    if (cudaMallocAsync((void **)&scr, sizeof(int) * words, s) != cudaSuccess) {
        cudaGetLastError();
        return DPS_ERR_OOM;
    }
    int *count = scr, *fill = scr + N, *key = fill + N, *tmp = key + np, *perm = tmp + np, *scan = perm + np,
        *status = scan + scan_scratch_words(N);
    cudaMemsetAsync(count, 0, sizeof(int) * N, s);
    cudaMemsetAsync(status, 0, sizeof(int), s);
    launch_sort_count(x3, x3 + 1, x3 + 2, 3, np, g, count, key, status, s);
    exclusive_scan(count, N, cell_start, scan, s);
    cudaMemsetAsync(fill, 0, sizeof(int) * N, s);
    launch_sort_scatter(key, np, cell_start, fill, tmp, s);
    launch_sort_rank(key, ids, np, cell_start, tmp, np > 0 ? order : perm, s);
    cudaFreeAsync(scr, s);
    return cudaGetLastError() == cudaSuccess ? DPS_OK : DPS_ERR_CUDA;
}

}  // extern "C"
