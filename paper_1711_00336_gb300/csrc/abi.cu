// abi.cu -- the C ABI of include/dps.h.
//
// Everything runs through one host object, the Batch: a device table of boxes
// (BoxDev) and tile lists over their cells and particles.  A coupled step of
// Algorithm 1 is a fixed sequence of launches, each covering every box of the
// batch; the per-box step state (AA parity, current particle set, history
// flags) is advanced on the device, so the sequence is captured once as a CUDA
// graph and replayed for every step until the set of boxes changes.  A domain
// (dps_handle) is a batch of one box.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "box.cuh"

namespace dps {
// launchers (lbm.cu, coupling.cu, dem.cu, scan.cu, io.cu)
template <typename ST, typename FT, typename CT>
void launch_collide_stream(const BoxDev *, const Tile *, int, int, int, bool, bool, int, int, cudaStream_t);
template <typename ST, typename FT, typename CT>
void launch_moments(const BoxDev *, const Tile *, int, int, int, int, cudaStream_t);
template <typename FT, typename CT>
void launch_fields(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
template <typename FT, typename CT>
void launch_curl(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
template <typename ST>
void launch_pdf_export(const void *, const Geom &, int, double *, cudaStream_t);
template <typename ST>
void launch_pdf_import(void *, long long, const double *, cudaStream_t);
void launch_sort_count(const double *, const double *, const double *, long long, long long, const Geom &, int *, int *,
                       int *, cudaStream_t);
void launch_sort_scatter(const int *, long long, const int *, int *, int *, cudaStream_t);
void launch_sort_rank(const int *, const int *, long long, const int *, const int *, int *, cudaStream_t);
void launch_bsort_count(const BoxDev *, const Tile *, int, int, int, int, cudaStream_t);
void launch_bsort_scatter(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
void launch_bsort_rank(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
void launch_bsort_gather(const BoxDev *, const Tile *, int, int, int, int, cudaStream_t);
void launch_bsort_flip(BoxDev *, int, int, cudaStream_t);
void launch_end_step(BoxDev *, int, cudaStream_t);
void launch_bscan(const BoxDev *, int, const Tile *, int, cudaStream_t);
int scan_tile_cells();
void brick_tiles(int, const int *, std::vector<Tile> &);
template <typename FT>
void launch_eps(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
template <typename FT>
void launch_force_am(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
template <typename FT>
void launch_force_drag(const BoxDev *, const Tile *, int, int, int, int, cudaStream_t);
template <typename FT>
void launch_reaction_am(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
template <typename FT>
void launch_reaction_drag(const BoxDev *, const Tile *, int, int, int, int, int, cudaStream_t);
void launch_dem_substep(const BoxDev *, const Tile *, int, int, int, int, int, int, int, int, cudaStream_t);
void launch_build_nlist(const BoxDev *, const Tile *, int, int, int, int, cudaStream_t);
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
void launch_particles_import(double *, int, long long, long long, const int *, const double *, cudaStream_t);
void launch_particles_export4(const BoxDev *, int, const double *, const int *, long long, long long, double *,
                              cudaStream_t);
long long reduce_partials_doubles();
void launch_pdf_relayout(const void *, const Geom &, int, int, void *, cudaStream_t);
}  // namespace dps

using namespace dps;

static const double PI_H = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// host objects
// ---------------------------------------------------------------------------
struct BoxHost {
    BoxDev d{};                   // table entry (state fields authoritative on the device)
    std::vector<void *> allocs;
    dps_closure cl{};
    bool have_closure = false;
    double sumV = 0, sumWb = 0, dmax = 0, dmin = 1e300;
    long long max_particles = 0;
    double tau = 0.65, rho_f = 1.0;
    bool prepared = false;
    long long steps = 0;
    int sticky = 0;
    double *d_red = nullptr, *d_redout = nullptr;
    int64_t user_id = -1;
};

enum { PH_MOM = 0, PH_FAM, PH_RAM, PH_FDRAG, PH_RDRAG, PH_DEM, PH_SORT, PH_EPS, PH_COLLIDE, NPH };

struct Tuning {
    int cell_block = 128, cell_tile = 1024;   // threads per block, cells per tile
    int part_block = 128, part_tile = 256;    // threads per block, particles per tile
    int k1v = 6;                              // collide-stream variant (FP32/FP16: vector cell pairs)
};

struct Batch {
    int prec = DPS_F64;
    size_t pdf_elem = 8, fel = 8;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // second stream of the step: the drag reaction runs beside the DEM
    // substeps (fork and join by events, captured into the step graph)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // read-back staging: device buffer and pinned host buffer for particle
    // exports, pinned status words (one copy and one synchronisation per call)
    double *d_pstage = nullptr, *h_pstage = nullptr;
    size_t cap_dpstage = 0, cap_hpstage = 0;
    int *h_status = nullptr;
    size_t cap_status = 0;
    dps_alloc_fn alloc = nullptr;
    dps_free_fn free = nullptr;
    void *ctx = nullptr;
    std::string err;
    std::vector<BoxHost *> boxes;
    std::vector<BoxHost *> dev_order;  // box of each device-table entry (null: removed since)
    int table_cap = 0;
    BoxDev *d_table = nullptr;
    std::vector<void *> allocs;  // batch-level buffers (table, tiles)
    Tile *d_cell = nullptr, *d_part = nullptr, *d_scan = nullptr, *d_brick = nullptr;
    int n_cell = 0, n_part = 0, n_scan = 0, n_brick = 0;
    size_t cap_cell = 0, cap_part = 0, cap_scan = 0, cap_brick = 0;
    Tuning tune;
    bool tuned = false;
    bool shape_fixed = false;     // launch shapes set by the caller or the autotuner
    int n_int = 0, n_dem = 0;
    bool any_lift = false;        // some box applies the lift force (curl launch per subcycle)
    bool any_walls = true;        // some box with particles has a wall axis (DEM wall code)
    int part_off[5] = {0, 0, 0, 0, 0};  // particle tiles grouped by DEM lanes class (1, 2, 4, 8)
    int cpl_lanes = 1;            // most lanes per particle of the force kernels over the batch
    int n_cell_plain = 0;         // cell tiles of boxes with a constant tau (listed first);
                                  // the rest relax with a per-cell tau_e (K1 variant)
    bool layout_dirty = true;     // table/tiles must be rebuilt and uploaded
    int parity = 0;               // AA parity of every box of the batch
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // step graphs by parity
    bool use_graphs = true;
    long long launches_step = 0, launch_count = 0;
    // tracing
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_phase, ev_nl;
    size_t ev_used = 0;
    double ph_ms[NPH] = {0};
    long long ph_nl[NPH] = {0};
};

static thread_local std::string g_create_err;

#define FAILB(b, code, ...)                      \
    do {                                         \
        char _m[512];                            \
        snprintf(_m, sizeof(_m), __VA_ARGS__);   \
        (b)->err = _m;                           \
        return code;                             \
    } while (0)

#define CKB(b, call)                                                                           \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess) FAILB(b, DPS_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
    } while (0)

static void *dalloc_raw(Batch *B, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (B->alloc) {
        p = B->alloc(bytes, B->ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    return p;
}
static void dfree_raw(Batch *B, void *p) {
    if (!p) return;
    if (B->free)
        B->free(p, B->ctx);
    else
        cudaFree(p);
}
static void *box_alloc(Batch *B, BoxHost *h, size_t bytes) {
    void *p = dalloc_raw(B, bytes);
    if (p) h->allocs.push_back(p);
    return p;
}
static void box_free(Batch *B, BoxHost *h) {
    for (void *p : h->allocs) dfree_raw(B, p);
    h->allocs.clear();
}

static void invalidate_graph(Batch *B) {
    for (int k = 0; k < 2; ++k)
        if (B->gexec[k]) {
            cudaGraphExecDestroy(B->gexec[k]);
            B->gexec[k] = nullptr;
        }
}

// ---- phase timing -----------------------------------------------------------
static void tbegin(Batch *B, cudaStream_t on = nullptr) {
    if (!B->timing) return;
    if (B->ev_used * 2 + 2 > B->ev.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        B->ev.push_back(a);
        B->ev.push_back(b);
        B->ev_phase.push_back(0);
        B->ev_nl.push_back(0);
    }
    // external record nodes: the events stay readable after graph replays
    cudaEventRecordWithFlags(B->ev[2 * B->ev_used], on ? on : B->stream, cudaEventRecordExternal);
}
static void tend(Batch *B, int phase, int nl, cudaStream_t on = nullptr) {
    B->launch_count += nl;
    if (!B->timing) return;
    cudaEventRecordWithFlags(B->ev[2 * B->ev_used + 1], on ? on : B->stream, cudaEventRecordExternal);
    B->ev_phase[B->ev_used] = phase;
    B->ev_nl[B->ev_used] = nl;
    B->ev_used++;
}

// ---- physics constants of a box ---------------------------------------------
static void compute_phys(BoxHost *h) {
    const dps_closure &c = h->cl;
    Phys &p = h->d.ph;
    p.tau = h->tau;
    p.omega = 1.0 / h->tau;
    p.kf = 1.0 - 0.5 / h->tau;
    p.omega_f = (float)p.omega;
    p.kf_f = (float)p.kf;
    p.rho_f = h->rho_f;
    p.mu = h->rho_f * (h->tau - 0.5) / 3.0;  // Eq. visc_tau
    const double cells = (double)h->d.g.ncell;
    for (int a = 0; a < 3; ++a) {
        p.g[a] = h->have_closure ? c.g[a] : 0.0;
        if (!h->have_closure)
            p.fb[a] = 0.0;
        else if (c.fb_mode == 1)
            p.fb[a] = (cells - h->sumV) > 0 ? -h->sumWb * c.g[a] / (cells - h->sumV) : 0.0;
        else if (c.fb_mode == 2)
            p.fb[a] = h->sumV > 0 ? -(h->sumV / cells) * (h->sumWb / h->sumV) * c.g[a] : 0.0;
        else
            p.fb[a] = c.fb[a];
    }
    for (int a = 0; a < 3; ++a) p.fb_f[a] = (float)p.fb[a];
    p.lift = h->have_closure ? c.lift : 0;
    p.eilers = h->have_closure ? c.eilers : 0;
    p.smag = h->have_closure ? c.smagorinsky : 0;
    if (!h->have_closure) {
        p.eps_min = 0.05;
        p.n_int = p.n_dem = 1;
        p.dt_sub = p.dt_dem = 1.0;
        h->d.R = 1;
        p.skin = 0.0;
        p.skin_half2 = 0.25;
        return;
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
    {
        const double le = std::log(c.e_n);
        p.kfac = (PI_H * PI_H + le * le) / (c.T_c * c.T_c);  // k_n / m_ij
        p.xfac = -2.0 * le / c.T_c;                          // xi_n / m_ij
        p.capfac = c.lub_cap / p.dt_dem;                     // lubrication cap / m_ij
    }
    // Verlet list: partners within (d_i+d_j)/2 + h_c + skin; linked cells of
    // +-R cells cover that range; particles may move skin/2 between sorts
    const double cutoff = h->dmax + (c.lubrication ? std::fmax(c.h_c, 0.0) : 0.0);
    p.skin = c.skin;
    h->d.R = (int)std::floor(cutoff + c.skin + 1e-3) + 1;
    p.skin_half2 = 0.25 * c.skin * c.skin;
}

// ---- table and tiles ------------------------------------------------------------
// copy the device-side step state of every box into the host entries
static int pull_state(Batch *B) {
    if (B->dev_order.empty() || !B->d_table) return DPS_OK;
    CKB(B, cudaStreamSynchronize(B->stream));
    std::vector<BoxDev> t(B->dev_order.size());
    CKB(B, cudaMemcpy(t.data(), B->d_table, sizeof(BoxDev) * t.size(), cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < B->dev_order.size(); ++k) {
        BoxHost *h = B->dev_order[k];
        if (!h) continue;
        BoxDev &d = h->d;
        d.parity = t[k].parity;
        d.cur = t[k].cur;
        d.have_uprev = t[k].have_uprev;
        d.have_usub = t[k].have_usub;
    }
    return DPS_OK;
}

// a box leaves the batch: its device-table entry no longer maps to it
static void forget_box(Batch *B, BoxHost *h) {
    for (auto &p : B->dev_order)
        if (p == h) p = nullptr;
    B->boxes.erase(std::remove(B->boxes.begin(), B->boxes.end(), h), B->boxes.end());
    B->layout_dirty = true;
}

static int ensure_buf(Batch *B, Tile **p, size_t *cap, size_t need) {
    if (need <= *cap && *p) return DPS_OK;
    size_t n = std::max<size_t>(need, 64);
    Tile *q = (Tile *)dalloc_raw(B, n * sizeof(Tile));
    if (!q) FAILB(B, DPS_ERR_OOM, "tile list allocation failed");
    if (*p) {
        dfree_raw(B, *p);
        B->allocs.erase(std::remove(B->allocs.begin(), B->allocs.end(), (void *)*p), B->allocs.end());
    }
    B->allocs.push_back(q);
    *p = q;
    *cap = n;
    return DPS_OK;
}

// lanes per particle in the DEM substep of a box (class 0..3 = 1, 2, 4, 8
// lanes): about one neighbour-list entry per lane or more, from the expected
// list length (number density times the list sphere).  A property of the box
// alone, so a box gets the same arithmetic alone and in any batch.
static int dem_lanes_class(const BoxHost *h) {
    if (!h->have_closure || h->d.np == 0) return 0;
    const dps_closure &c = h->cl;
    const double rl = h->dmax + (c.lubrication ? std::fmax(c.h_c, 0.0) : 0.0) + c.skin;
    const double est = (double)h->d.np / (double)h->d.g.ncell * 4.18879 * rl * rl * rl;
    int cls = est >= 24.0 ? 3 : est >= 8.0 ? 2 : est >= 3.0 ? 1 : 0;
    // few particles: a warp costs the longest list among its particles and
    // there are few warps per SM, so spread every particle over more lanes
    // (about one warp per SM scheduler at np x lanes / 32)
    for (long long lanes = 1LL << cls; cls < 3 && h->d.np * lanes < 19456; lanes <<= 1) ++cls;
    return cls;
}

// lanes per particle of the force kernels (Tile::first of the particle
// tiles): the few-particles rule of the DEM substep alone (the 27-cell
// support gathers do not grow with the neighbour count)
static int force_lanes(const BoxHost *h) {
    int lanes = 1;
    while (lanes < 8 && h->d.np * lanes < 19456) lanes <<= 1;
    return lanes;
}

// rebuild the device table and the tile lists from the host boxes (the
// device step state must have been pulled first)
static int push_layout(Batch *B) {
    const int nb = (int)B->boxes.size();
    if (nb > B->table_cap) {
        int cap = std::max(nb, std::max(2 * B->table_cap, 4));
        BoxDev *t = (BoxDev *)dalloc_raw(B, sizeof(BoxDev) * cap);
        if (!t) FAILB(B, DPS_ERR_OOM, "box table allocation failed");
        if (B->d_table) {
            dfree_raw(B, B->d_table);
            B->allocs.erase(std::remove(B->allocs.begin(), B->allocs.end(), (void *)B->d_table), B->allocs.end());
        }
        B->allocs.push_back(t);
        B->d_table = t;
        B->table_cap = cap;
    }
    std::vector<BoxDev> tab(nb);
    std::vector<Tile> cell, part, scan, brick;
    const long long ST = scan_tile_cells();
    std::vector<Tile> cellv;  // cell tiles of the boxes with a per-cell tau_e
    if (!B->shape_fixed) {
        // default particle tiles: small enough that every SM gets a block when
        // the batch holds few particles (a particle thread is latency- or
        // FP64-bound, so spreading them over all SMs is what counts)
        long long npt = 0;
        for (BoxHost *h : B->boxes) npt += h->d.np;
        int pt = 256;
        while (pt > 32 && npt < 2LL * 152 * pt) pt /= 2;
        B->tune.part_tile = pt;
        B->tune.part_block = std::min(128, pt);
    }
    std::vector<Tile> partc[4];  // particle tiles by DEM lanes class
    B->any_lift = false;
    B->any_walls = false;
    B->cpl_lanes = 1;
    for (int k = 0; k < nb; ++k) {
        BoxHost *h = B->boxes[k];
        compute_phys(h);
        B->any_lift |= h->d.ph.lift && h->d.np > 0;
        B->any_walls |= h->d.np > 0 && !(h->d.g.per[0] && h->d.g.per[1] && h->d.g.per[2]);
        std::vector<Tile> &ct = (h->d.ph.eilers || h->d.ph.smag) ? cellv : cell;
        tab[k] = h->d;
        const long long N = h->d.g.ncell, np = h->d.np;
        for (long long c = 0; c < N; c += B->tune.cell_tile)
            ct.push_back(Tile{k, 0, c, std::min(N, c + B->tune.cell_tile)});
        const int lc = dem_lanes_class(h), fl = force_lanes(h);
        B->cpl_lanes = std::max(B->cpl_lanes, fl);
        for (long long p = 0; p < np; p += B->tune.part_tile)
            partc[lc].push_back(Tile{k, fl, p, std::min(np, p + B->tune.part_tile)});
        int idx = 0;
        for (long long c = 0; c < N; c += ST) scan.push_back(Tile{k, idx++, c, std::min(N, c + ST)});
        brick_tiles(k, h->d.g.n, brick);
    }
    B->n_cell_plain = (int)cell.size();
    cell.insert(cell.end(), cellv.begin(), cellv.end());
    for (int c = 0; c < 4; ++c) {
        B->part_off[c] = (int)part.size();
        part.insert(part.end(), partc[c].begin(), partc[c].end());
    }
    B->part_off[4] = (int)part.size();
    int rc;
    if ((rc = ensure_buf(B, &B->d_cell, &B->cap_cell, cell.size()))) return rc;
    if ((rc = ensure_buf(B, &B->d_part, &B->cap_part, part.size()))) return rc;
    if ((rc = ensure_buf(B, &B->d_scan, &B->cap_scan, scan.size()))) return rc;
    if ((rc = ensure_buf(B, &B->d_brick, &B->cap_brick, brick.size()))) return rc;
    if (nb) CKB(B, cudaMemcpyAsync(B->d_table, tab.data(), sizeof(BoxDev) * nb, cudaMemcpyHostToDevice, B->stream));
    if (!cell.empty())
        CKB(B, cudaMemcpyAsync(B->d_cell, cell.data(), sizeof(Tile) * cell.size(), cudaMemcpyHostToDevice, B->stream));
    if (!part.empty())
        CKB(B, cudaMemcpyAsync(B->d_part, part.data(), sizeof(Tile) * part.size(), cudaMemcpyHostToDevice, B->stream));
    if (!scan.empty())
        CKB(B, cudaMemcpyAsync(B->d_scan, scan.data(), sizeof(Tile) * scan.size(), cudaMemcpyHostToDevice, B->stream));
    if (!brick.empty())
        CKB(B, cudaMemcpyAsync(B->d_brick, brick.data(), sizeof(Tile) * brick.size(), cudaMemcpyHostToDevice, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    B->n_cell = (int)cell.size();
    B->n_part = (int)part.size();
    B->n_scan = (int)scan.size();
    B->n_brick = (int)brick.size();
    B->dev_order = B->boxes;
    B->layout_dirty = false;
    invalidate_graph(B);
    return DPS_OK;
}

static int grid_of(int ntiles) { return std::max(1, std::min(ntiles, 152 * 8)); }

// threads per block of a particle kernel with `lanes` lanes per particle:
// the tuned block, or all lane groups of a tile when they fit in 256 threads
// (the small tiles of boxes with few particles); a multiple of 32, since the
// lane-group shuffles take all 32 lanes of a warp.  Large tiles keep the tuned
// block: these kernels hold 100-200 registers a thread, and 256-thread blocks
// would leave one block per SM.
static int part_threads(const Tuning &u, int lanes) {
    const long long want = (long long)u.part_tile * lanes;
    const long long b = lanes > 1 && want > u.part_block && want <= 256 ? want : u.part_block;
    return (int)((b + 31) / 32 * 32);
}

// ---- the coupled step --------------------------------------------------------------
#define PREC_CALL(B, F64CALL, F32CALL, F16CALL) \
    do {                                        \
        if ((B)->prec == DPS_F64) {             \
            F64CALL;                            \
        } else if ((B)->prec == DPS_F32) {      \
            F32CALL;                            \
        } else {                                \
            F16CALL;                            \
        }                                       \
    } while (0)

// K1 over the cell tiles of the boxes with a constant tau, then the per-cell
// tau_e variant over those of the boxes with the Eilers / Smagorinsky
// closures (one launch when the batch holds one kind); returns the launches.
// mom_in: K2a ran on these populations in this step (the coupled step), so
// the FP64 form takes rho and j from it.
static int enqueue_collide(Batch *B, int par, bool mom_in) {
    const BoxDev *T = B->d_table;
    const Tuning &u = B->tune;
    cudaStream_t s = B->stream;
    int nl = 0;
    for (int v = 0; v < 2; ++v) {
        const int nt = v ? B->n_cell - B->n_cell_plain : B->n_cell_plain;
        if (nt <= 0) continue;
        const Tile *tl = B->d_cell + (v ? B->n_cell_plain : 0);
        const bool vi = v == 1;
        PREC_CALL(B, (launch_collide_stream<double, double, double>(T, tl, nt, par, u.k1v, vi, mom_in, grid_of(nt), u.cell_block, s)),
                  (launch_collide_stream<float, float, float>(T, tl, nt, par, u.k1v, vi, mom_in, grid_of(nt), u.cell_block, s)),
                  (launch_collide_stream<__half, float, float>(T, tl, nt, par, u.k1v, vi, mom_in, grid_of(nt), u.cell_block, s)));
        ++nl;
    }
    return nl;
}

// have_keys: the last DEM substep already wrote the linked cells and counts
static void enqueue_sort_eps(Batch *B, int xsel, int mark_usub, bool have_keys) {
    const BoxDev *T = B->d_table;
    const int nb = (int)B->boxes.size();
    const Tuning &u = B->tune;
    const int pl = B->n_part > 0;
    const int cnt = pl && !have_keys;
    tbegin(B);
    if (cnt) launch_bsort_count(T, B->d_part, B->n_part, xsel, grid_of(B->n_part), u.part_block, B->stream);
    launch_bscan(T, nb, B->d_scan, B->n_scan, B->stream);
    if (pl) {
        launch_bsort_scatter(T, B->d_part, B->n_part, grid_of(B->n_part), u.part_block, B->stream);
        launch_bsort_rank(T, B->d_part, B->n_part, grid_of(B->n_part), u.part_block, B->stream);
        launch_bsort_gather(T, B->d_part, B->n_part, xsel, grid_of(B->n_part), part_threads(u, B->cpl_lanes),
                            B->stream);
    }
    launch_bsort_flip(B->d_table, nb, mark_usub, B->stream);
    const int pairs = B->prec == DPS_F64;  // the FP64 form evaluates each pair once
    if (pl)
        launch_build_nlist(T, B->d_part, B->n_part, grid_of(B->n_part), part_threads(u, B->cpl_lanes), pairs,
                           B->stream);
    tend(B, PH_SORT, cnt + 3 + 3 * pl + 1 + pl * (1 + 2 * pairs));
    tbegin(B);
    if (B->fel == 8)
        launch_eps<double>(T, B->d_brick, B->n_brick, grid_of(B->n_brick), 256, B->stream);
    else
        launch_eps<float>(T, B->d_brick, B->n_brick, grid_of(B->n_brick), 256, B->stream);
    tend(B, PH_EPS, 1);
}

static void enqueue_step(Batch *B) {
    const BoxDev *T = B->d_table;
    const Tuning &u = B->tune;
    const int gc = grid_of(B->n_cell), gp = grid_of(B->n_part), gb = grid_of(B->n_brick);
    const int pl = B->n_part > 0;
    const bool f64 = B->fel == 8;
    cudaStream_t s = B->stream;
    B->ev_used = 0;
    B->launch_count = 0;
    // Du_f/Dt and grad P, once per step
    tbegin(B);
    const int par = B->parity;
    PREC_CALL(B, (launch_moments<double, double, double>(T, B->d_cell, B->n_cell, par, gc, u.cell_block, s)),
              (launch_moments<float, float, float>(T, B->d_cell, B->n_cell, par, gc, u.cell_block, s)),
              (launch_moments<__half, float, float>(T, B->d_cell, B->n_cell, par, gc, u.cell_block, s)));
    if (f64)
        launch_fields<double, double>(T, B->d_cell, B->n_cell, gc, u.cell_block, s);
    else
        launch_fields<float, float>(T, B->d_cell, B->n_cell, gc, u.cell_block, s);
    tend(B, PH_MOM, 2);
    const int nl = pl && B->any_lift;
    for (int k = 0; k < B->n_int; ++k) {
        tbegin(B);
        if (nl) {
            if (f64) launch_curl<double, double>(T, B->d_cell, B->n_cell, gc, u.cell_block, s);
            else launch_curl<float, float>(T, B->d_cell, B->n_cell, gc, u.cell_block, s);
        }
        if (pl) {
            if (f64) launch_force_am<double>(T, B->d_part, B->n_part, gp, part_threads(u, B->cpl_lanes), s);
            else launch_force_am<float>(T, B->d_part, B->n_part, gp, part_threads(u, B->cpl_lanes), s);
        }
        tend(B, PH_FAM, pl + nl);
        tbegin(B);
        if (f64) launch_reaction_am<double>(T, B->d_brick, B->n_brick, gb, 256, s);
        else launch_reaction_am<float>(T, B->d_brick, B->n_brick, gb, 256, s);
        tend(B, PH_RAM, 1);
        tbegin(B);
        if (pl) {
            if (f64) launch_force_drag<double>(T, B->d_part, B->n_part, k == 0, gp, part_threads(u, B->cpl_lanes), s);
            else launch_force_drag<float>(T, B->d_part, B->n_part, k == 0, gp, part_threads(u, B->cpl_lanes), s);
        }
        tend(B, PH_FDRAG, pl);
        // the drag reaction (cell fields from the frozen particle forces and
        // weights) and the DEM substeps (particle kinematics) touch disjoint
        // data: the reaction runs on the side stream (its phase timed there)
        // and joins before the sort, which reorders the particles it reads
        const bool fork = B->side != nullptr;
        cudaStream_t rs = s;
        if (fork) {
            cudaEventRecord(B->ev_fork, s);
            cudaStreamWaitEvent(B->side, B->ev_fork, 0);
            rs = B->side;
        }
        tbegin(B, rs);
        if (f64)
            launch_reaction_drag<double>(T, B->d_brick, B->n_brick, k == 0, k == B->n_int - 1, gb, 256, rs);
        else
            launch_reaction_drag<float>(T, B->d_brick, B->n_brick, k == 0, k == B->n_int - 1, gb, 256, rs);
        tend(B, PH_RDRAG, 1, rs);
        if (fork) cudaEventRecord(B->ev_join, B->side);
        tbegin(B);
        int ndl = 0;
        if (pl)
            for (int sd = 0; sd < B->n_dem; ++sd)
                for (int c = 0; c < 4; ++c) {
                    const int nt = B->part_off[c + 1] - B->part_off[c];
                    if (nt <= 0) continue;
                    // mixed forms: a block holds all lane groups of a particle tile,
                    // at most 256 threads (two such blocks fit an SM); FP64 form:
                    // the particle-kernel rule (its 200 registers a thread allow
                    // one 256-thread block per SM)
                    const int blk = B->prec != DPS_F64
                                        ? (int)std::min<long long>(256, (std::max<long long>(u.part_block,
                                                                                             (long long)u.part_tile << c) +
                                                                         31) / 32 * 32)
                                        : part_threads(u, 1 << c);
                    launch_dem_substep(T, B->d_part + B->part_off[c], nt, sd & 1, sd == B->n_dem - 1,
                                       B->prec != DPS_F64, 1 << c, B->any_walls, grid_of(nt), blk, s);
                    ndl += 2;  // pair kernel + gather / integration kernel
                }
        tend(B, PH_DEM, ndl);
        if (fork) cudaStreamWaitEvent(s, B->ev_join, 0);
        enqueue_sort_eps(B, B->n_dem & 1, 1, B->n_dem > 0);
    }
    tbegin(B);
    const int nk1 = enqueue_collide(B, par, true);
    launch_end_step(B->d_table, (int)B->boxes.size(), s);
    tend(B, PH_COLLIDE, nk1 + 1);
    B->launches_step = B->launch_count;
}

static int check_boxes(Batch *B) {
    std::string m;
    int bad = 0;
    const size_t nb = B->boxes.size();
    if (nb > B->cap_status) {
        if (B->h_status) cudaFreeHost(B->h_status);
        B->h_status = nullptr;
        B->cap_status = 0;
        CKB(B, cudaMallocHost((void **)&B->h_status, sizeof(int) * std::max<size_t>(nb, 16)));
        B->cap_status = std::max<size_t>(nb, 16);
    }
    for (size_t k = 0; k < nb; ++k)
        CKB(B, cudaMemcpyAsync(B->h_status + k, B->boxes[k]->d.status, sizeof(int), cudaMemcpyDeviceToHost,
                               B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    for (size_t k = 0; k < nb; ++k) {
        BoxHost *h = B->boxes[k];
        const int st = B->h_status[k];
        if (st) {
            CKB(B, cudaMemset(h->d.status, 0, sizeof(int)));
            h->sticky |= st;
            bad |= st;
        }
    }
    if (bad) {
        if (bad & ST_NAN) m += "non-finite or non-positive state; ";
        if (bad & ST_SKIN) m += "a particle moved more than skin/2 within one subcycle (increase skin or n_int); ";
        if (bad & ST_EPS_NEG) m += "eps_f < 0 before the floor; ";
        if (bad & ST_BAD_CELL) m += "a particle left the box through a wall; ";
        if (bad & ST_NLIST) m += "a neighbour list overflowed; ";
        FAILB(B, DPS_ERR_UNSTABLE, "unstable: %s", m.c_str());
    }
    return DPS_OK;
}

// Verlet-list capacity: at most as many spheres of the smallest diameter as
// fit (at the densest packing, 0.7405) in the list radius around a centre
static int list_capacity(const BoxHost *h) {
    if (h->d.np == 0 || !h->have_closure) return 1;
    const dps_closure &c = h->cl;
    const double rl = h->dmax + (c.lubrication ? std::fmax(c.h_c, 0.0) : 0.0) + c.skin + 1e-3;
    const double r0 = 0.5 * h->dmin;
    double n = 0.7405 * std::pow((rl + r0) / r0, 3.0) + 1.0;
    n = std::fmin(n, (double)h->d.np);
    return (int)std::fmax(1.0, std::fmin(n, 1024.0));
}

static void box_release(Batch *B, BoxHost *h, void *p) {
    if (!p) return;
    dfree_raw(B, p);
    h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), p), h->allocs.end());
}

// the pair slots of the FP64 form: every unordered pair of the list once;
// the list holds at most maxn partners per particle, so at most cap*maxn/2
// pairs
static long long pair_capacity(const BoxHost *h, int maxn) { return (long long)h->d.cap * maxn / 2 + 1; }

static int ensure_lists(Batch *B) {
    for (BoxHost *h : B->boxes) {
        const int need = list_capacity(h);
        if (need <= h->d.maxn && h->d.nlist) continue;
        const size_t C = (size_t)h->d.cap;
        void *p = box_alloc(B, h, (size_t)need * C * 4);
        if (!p) FAILB(B, DPS_ERR_OOM, "neighbour list allocation failed");
        box_release(B, h, h->d.nlist);
        h->d.nlist = (int *)p;
        if (B->prec == DPS_F64) {
            const long long pc = pair_capacity(h, need);
            if (pc >= (1LL << 31)) FAILB(B, DPS_ERR_ARG, "too many neighbour pairs for one box (%lld)", pc);
            void *hj = box_alloc(B, h, (size_t)pc * 4), *rr = box_alloc(B, h, (size_t)need * C * 4);
            void *pr = box_alloc(B, h, (size_t)pc * 48), *pg = box_alloc(B, h, (size_t)pc);
            if (!hj || !rr || !pr || !pg) FAILB(B, DPS_ERR_OOM, "pair list allocation failed");
            box_release(B, h, h->d.hj);
            box_release(B, h, h->d.rrow);
            box_release(B, h, h->d.pres);
            box_release(B, h, h->d.pflag);
            h->d.hj = (int *)hj;
            h->d.rrow = (int *)rr;
            h->d.pres = (double *)pr;
            h->d.pflag = (unsigned char *)pg;
            h->d.pcap = pc;
        }
        h->d.maxn = need;
        B->layout_dirty = true;
    }
    return DPS_OK;
}

// uniform subcycle counts over the batch; layout upload; prepare new boxes
static int ready(Batch *B) {
    for (BoxHost *h : B->boxes)
        if (!h->have_closure) FAILB(B, DPS_ERR_STATE, "dps_set_closure must be called for every box first");
    if (B->boxes.empty()) return DPS_OK;
    B->n_int = B->boxes[0]->cl.n_int;
    B->n_dem = B->boxes[0]->cl.n_dem;
    for (BoxHost *h : B->boxes)
        if (h->cl.n_int != B->n_int || h->cl.n_dem != B->n_dem)
            FAILB(B, DPS_ERR_ARG, "all boxes of a batch need the same n_int and n_dem");
    bool need_prep = false;
    for (BoxHost *h : B->boxes) need_prep |= !h->prepared;
    if (need_prep) {
        int rc = ensure_lists(B);
        if (rc) return rc;
    }
    if (B->layout_dirty || need_prep) {
        int rc = pull_state(B);
        if (rc) return rc;
        if ((rc = push_layout(B))) return rc;
    }
    if (need_prep) {
        // Algorithm 1 initialisation: sort and eps_f for every box (idempotent
        // for boxes already prepared: their particles did not move)
        B->ev_used = 0;
        bool t = B->timing;
        B->timing = false;
        enqueue_sort_eps(B, 0, 0, false);
        B->timing = t;
        for (BoxHost *h : B->boxes) h->prepared = true;
        int rc = check_boxes(B);
        if (rc) return rc;
    }
    return DPS_OK;
}

static int run_steps(Batch *B, long long n) {
    int rc = ready(B);
    if (rc) return rc;
    if (B->boxes.empty()) return DPS_OK;
    for (long long s = 0; s < n; ++s) {
        if (!B->use_graphs) {
            enqueue_step(B);
        } else {
            cudaGraphExec_t &ge = B->gexec[B->parity];
            if (!ge) {
                cudaGraph_t g;
                CKB(B, cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
                enqueue_step(B);
                CKB(B, cudaStreamEndCapture(B->stream, &g));
                cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) FAILB(B, DPS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
            }
            CKB(B, cudaGraphLaunch(ge, B->stream));
        }
        B->parity ^= 1;
        for (BoxHost *h : B->boxes) h->steps++;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) FAILB(B, DPS_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
    return DPS_OK;
}

// ---- boxes ------------------------------------------------------------------------------
static int batch_init(Batch *B, int precision, void *stream, dps_alloc_fn a, dps_free_fn f, void *ctx) {
    B->prec = precision;
    // collide-stream default: adjacent cell pairs moved as two-element
    // vectors, 4 blocks per SM (measured at 256^3: FP32 6.2 TB/s, FP16s
    // 4.7 TB/s; two scalar cells per thread: 5.4 and 3.0 TB/s)
    B->tune.k1v = 6;
    B->pdf_elem = precision == DPS_F64 ? 8 : (precision == DPS_F32 ? 4 : 2);
    B->fel = precision == DPS_F64 ? 8 : 4;
    B->alloc = a;
    B->free = f;
    B->ctx = ctx;
    const char *env = getenv("DPS_NO_GRAPH");
    B->use_graphs = !(env && env[0] == '1');
    B->stream = (cudaStream_t)stream;  // NULL: created with the first box
    return DPS_OK;
}

static int ensure_stream(Batch *B) {
    if (!B->side) {
        if (cudaStreamCreateWithFlags(&B->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            FAILB(B, DPS_ERR_CUDA, "stream or event creation failed");
        }
    }
    if (B->stream) return DPS_OK;
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        FAILB(B, DPS_ERR_CUDA, "cudaStreamCreate failed");
    }
    B->own_stream = true;
    return DPS_OK;
}

static void batch_release(Batch *B) {
    if (B->stream) cudaStreamSynchronize(B->stream);
    invalidate_graph(B);
    for (BoxHost *h : B->boxes) {
        box_free(B, h);
        delete h;
    }
    B->boxes.clear();
    for (void *p : B->allocs) dfree_raw(B, p);
    B->allocs.clear();
    for (cudaEvent_t e : B->ev) cudaEventDestroy(e);
    B->ev.clear();
    if (B->h_pstage) cudaFreeHost(B->h_pstage);
    if (B->h_status) cudaFreeHost(B->h_status);
    B->h_pstage = nullptr;
    B->h_status = nullptr;
    B->cap_hpstage = B->cap_status = 0;
    B->d_pstage = nullptr;  // in B->allocs, freed above
    B->cap_dpstage = 0;
    if (B->side) {
        cudaStreamSynchronize(B->side);
        cudaStreamDestroy(B->side);
        cudaEventDestroy(B->ev_fork);
        cudaEventDestroy(B->ev_join);
        B->side = nullptr;
        B->ev_fork = B->ev_join = nullptr;
    }
    if (B->own_stream && B->stream) cudaStreamDestroy(B->stream);
    B->stream = nullptr;
}

// bytes of device memory a box of n cells and cap particles needs
static size_t box_bytes(int prec, long long ncell, long long cap) {
    size_t pe = prec == DPS_F64 ? 8 : (prec == DPS_F32 ? 4 : 2), fe = prec == DPS_F64 ? 8 : 4;
    size_t N = (size_t)ncell, C = (size_t)(cap > 0 ? cap : 1);
    size_t b = 19 * N * pe + 27 * N * fe;
    b += 2 * (size_t)NPF * C * 8 + 2 * (size_t)NPI * C * 4 + 9 * C * 8 + 6 * C * 16 + C * 4 + 64 * C * 4 + 18 * C * 4;
    if (prec != DPS_F64) b += 6 * C * 8;  // mixed-form pair sums
    if (prec == DPS_F64) b += 64 * C * 4 + 32 * C * (4 + 48 + 1);  // pair lists and results (64 partners)
    b += (3 * N + 1) * 4 + 3 * C * 4 + ((N + 8191) / 8192 + 1) * 4;
    b += 4096 + (size_t)reduce_partials_doubles() * 8;
    return b;
}

// allocate and initialise one box (fluid at rest, eps_f = 1, no particles)
static int box_create(Batch *B, const int n[3], const int per[3], double tau, double rho_f, long long max_particles,
                      BoxHost **out) {
    *out = nullptr;
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1) FAILB(B, DPS_ERR_ARG, "lattice size must be >= 1 per axis");
    long long ncell = (long long)n[0] * n[1] * n[2];
    if (ncell > (1LL << 27)) FAILB(B, DPS_ERR_ARG, "lattice too large: at most 2^27 cells per box");
    if (!(tau > 0.5) || !(rho_f > 0.0) || max_particles < 0 || max_particles >= (1LL << 31))
        FAILB(B, DPS_ERR_ARG, "invalid box (tau > 0.5, rho_f > 0, particle capacity)");
    BoxHost *h = new BoxHost();
    h->tau = tau;
    h->rho_f = rho_f;
    h->max_particles = max_particles;
    BoxDev &d = h->d;
    for (int a = 0; a < 3; ++a) {
        d.g.n[a] = n[a];
        d.g.per[a] = per[a] ? 1 : 0;
        d.g.nb[a] = n[a];
    }
    d.g.B = 1;
    d.g.ncell = ncell;
    d.cap = max_particles > 0 ? max_particles : 1;
    d.np = 0;
    const size_t N = (size_t)ncell, cap = (size_t)d.cap;
    bool ok = true;
    auto A = [&](size_t bytes) {
        void *p = box_alloc(B, h, bytes);
        ok = ok && p;
        return p;
    };
    d.pdf = A(19 * N * B->pdf_elem);
    d.eps = A(N * B->fel);
    d.rho = A(N * B->fel);
    d.ire = A(N * B->fel);
    void **vec[] = {&d.fpf, &d.fam, &d.acc, &d.j, &d.uD, &d.uprev, &d.gradP, &d.DuDt};
    for (void **v : vec) *v = A(3 * N * B->fel);
    d.curl = d.uD;
    for (int s = 0; s < 2; ++s) {
        d.pf[s] = (double *)A((size_t)NPF * cap * 8);
        d.pi[s] = (int *)A((size_t)NPI * cap * 4);
    }
    d.xtmp = (double *)A(9 * cap * 8);
    for (int k = 0; k < 2; ++k) {
        d.xf[k] = (float4 *)A(cap * 16);
        d.vf[k] = (float4 *)A(cap * 16);
        d.of[k] = (float4 *)A(cap * 16);
    }
    d.nlist_n = (int *)A(cap * 4);
    d.lowp = B->prec != DPS_F64;
    d.pwf = d.lowp ? (float *)A(9 * cap * 4) : nullptr;
    d.f32p = d.lowp ? (float *)A(6 * cap * 4) : nullptr;
    d.psum = d.lowp ? (double *)A(6 * cap * 8) : nullptr;
    d.nlist = nullptr;  // sized at preparation (depends on the closure)
    d.maxn = 0;
    d.hj = d.rrow = nullptr;
    d.pres = nullptr;
    d.pflag = nullptr;
    d.pcap = 0;
    d.hoff = (int *)A(cap * 4);
    d.hn = (int *)A(cap * 4);
    d.rn = (int *)A(cap * 4);
    d.ptop = (unsigned long long *)A(16);
    d.cell_start = (int *)A((N + 1) * 4);
    d.count = (int *)A(N * 4);
    d.fill = (int *)A(N * 4);
    d.key = (int *)A(cap * 4);
    d.tmp = (int *)A(cap * 4);
    d.perm = (int *)A(cap * 4);
    d.scan_part = (int *)A(((N + 8191) / 8192 + 1) * 4);
    d.status = (int *)A(64);
    d.counters = (unsigned long long *)A(8 * CNT_N);
    h->d_red = (double *)A((size_t)reduce_partials_doubles() * 8);
    h->d_redout = (double *)A(32 * 8);
    if (!ok) {
        box_free(B, h);
        delete h;
        FAILB(B, DPS_ERR_OOM, "device allocation failed");
    }
    if (ensure_stream(B)) {
        box_free(B, h);
        delete h;
        return DPS_ERR_CUDA;
    }
    cudaStream_t s = B->stream;
    PREC_CALL(B, launch_pdf_rest<double>(d.pdf, ncell, s), launch_pdf_rest<float>(d.pdf, ncell, s),
              launch_pdf_rest<__half>(d.pdf, ncell, s));
    if (B->fel == 8)
        launch_fill<double>(d.eps, ncell, 1.0, s);
    else
        launch_fill<float>(d.eps, ncell, 1.0, s);
    for (void *p : {d.fpf, d.fam, d.acc, d.j, d.uD, d.uprev, d.gradP, d.DuDt}) cudaMemsetAsync(p, 0, 3 * N * B->fel, s);
    cudaMemsetAsync(d.rho, 0, N * B->fel, s);
    cudaMemsetAsync(d.ire, 0, N * B->fel, s);
    cudaMemsetAsync(d.nlist_n, 0, cap * 4, s);
    for (int *z : {d.hoff, d.hn, d.rn}) cudaMemsetAsync(z, 0, cap * 4, s);
    cudaMemsetAsync(d.ptop, 0, 16, s);
    for (int k = 0; k < 2; ++k) {
        cudaMemsetAsync(d.xf[k], 0, cap * 16, s);
        cudaMemsetAsync(d.vf[k], 0, cap * 16, s);
        cudaMemsetAsync(d.of[k], 0, cap * 16, s);
        cudaMemsetAsync(d.pf[k], 0, (size_t)NPF * cap * 8, s);
        cudaMemsetAsync(d.pi[k], 0, (size_t)NPI * cap * 4, s);
    }
    cudaMemsetAsync(d.cell_start, 0, (N + 1) * 4, s);
    cudaMemsetAsync(d.count, 0, N * 4, s);
    cudaMemsetAsync(d.fill, 0, N * 4, s);
    cudaMemsetAsync(d.status, 0, 64, s);
    cudaMemsetAsync(d.counters, 0, 8 * CNT_N, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        box_free(B, h);
        delete h;
        FAILB(B, DPS_ERR_CUDA, "initialisation kernels failed");
    }
    d.parity = d.cur = d.have_uprev = d.have_usub = 0;
    compute_phys(h);
    *out = h;
    return DPS_OK;
}

static int box_add_particles(Batch *B, BoxHost *h, long long n, const double *x3, const double *u3, const double *w3,
                             const double *dd, const double *rp) {
    if (n < 0 || (n > 0 && (!x3 || !dd || !rp))) FAILB(B, DPS_ERR_ARG, "bad particle arrays");
    if (n == 0) return DPS_OK;
    if (h->d.np + n > h->max_particles)
        FAILB(B, DPS_ERR_ARG, "capacity exceeded (%lld + %lld > %lld)", h->d.np, n, h->max_particles);
    for (int a = 0; a < 3; ++a)
        if (h->d.g.n[a] < 3) FAILB(B, DPS_ERR_ARG, "particles need at least 3 cells per axis");
    int rc = pull_state(B);
    if (rc) return rc;
    const long long cap = h->d.cap;
    std::vector<double> st((size_t)11 * n);
    std::vector<int> ids((size_t)n);
    double sV = 0, sW = 0, dm = h->dmax, dn = h->dmin;
    for (long long i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            double x = x3[3 * i + a];
            if (!std::isfinite(x)) FAILB(B, DPS_ERR_ARG, "non-finite position");
            const int L = h->d.g.n[a];
            if (h->d.g.per[a]) {
                x -= L * std::floor(x / L);
                if (x >= L) x -= L;
            } else if (!(x > 0.0 && x < L)) {
                FAILB(B, DPS_ERR_ARG, "particle %lld outside the walls on axis %d", i, a);
            }
            st[(size_t)a * n + i] = x;
            st[(size_t)(3 + a) * n + i] = u3 ? u3[3 * i + a] : 0.0;
            st[(size_t)(6 + a) * n + i] = w3 ? w3[3 * i + a] : 0.0;
        }
        if (!(dd[i] > 0.0) || !(rp[i] > 0.0)) FAILB(B, DPS_ERR_ARG, "d and rho_p must be > 0");
        st[(size_t)9 * n + i] = dd[i];
        st[(size_t)10 * n + i] = rp[i];
        ids[i] = (int)(h->d.np + i);
        double V = PI_H / 6.0 * dd[i] * dd[i] * dd[i];
        sV += V;
        sW += (rp[i] - h->rho_f) * V;
        dm = std::fmax(dm, dd[i]);
        dn = std::fmin(dn, dd[i]);
    }
    double *pf = h->d.pf[h->d.cur];
    const long long off = h->d.np;
    for (int f = 0; f < 11; ++f)
        CKB(B, cudaMemcpyAsync(pf + (size_t)f * cap + off, st.data() + (size_t)f * n, 8 * n, cudaMemcpyHostToDevice,
                               B->stream));
    for (int a = 0; a < 3; ++a)
        CKB(B, cudaMemcpyAsync(pf + (size_t)(PUS0 + a) * cap + off, st.data() + (size_t)(3 + a) * n, 8 * n,
                               cudaMemcpyHostToDevice, B->stream));
    CKB(B, cudaMemcpyAsync(h->d.pi[h->d.cur] + IID * cap + off, ids.data(), 4 * n, cudaMemcpyHostToDevice, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    h->d.np += n;
    h->sumV += sV;
    h->sumWb += sW;
    h->dmax = dm;
    h->dmin = dn;
    h->prepared = false;
    B->layout_dirty = true;
    return DPS_OK;
}

static int check_closure(Batch *B, const dps_closure *c) {
    if (!c) FAILB(B, DPS_ERR_ARG, "null closure");
    if (c->n_int < 1 || c->n_dem < 1 || !(c->e_n > 0.0 && c->e_n <= 1.0) || !(c->T_c > 0.0) || !(c->h_c >= 0.0) ||
        !(c->h_min > 0.0) || !(c->mu_c >= 0.0) || !(c->eps_min > 0.0 && c->eps_min < 1.0) || !(c->skin >= 0.0) ||
        !(c->lub_cap > 0.0) || c->fb_mode < 0 || c->fb_mode > 2)
        FAILB(B, DPS_ERR_ARG, "invalid closure parameter");
    return DPS_OK;
}

// ---- per-box host views -------------------------------------------------------------------
static int box_read_fields(Batch *B, BoxHost *h, uint32_t mask, double *out, long long cap) {
    if (mask & ~0x1FFu) FAILB(B, DPS_ERR_ARG, "unknown field bits");
    const long long N = h->d.g.ncell;
    static const int planes[9] = {1, 3, 3, 1, 3, 1, 3, 3, 3};
    long long need = 0;
    for (int b = 0; b < 9; ++b)
        if (mask & (1u << b)) need += planes[b] * N;
    if (!out && need) FAILB(B, DPS_ERR_ARG, "null output");
    if (cap < need) FAILB(B, DPS_ERR_ARG, "output capacity %lld < %lld", cap, need);
    int rc = h->have_closure && !h->prepared ? ready(B) : pull_state(B);
    if (rc) return rc;
    compute_phys(h);
    const double *fb = h->d.ph.fb;
    const BoxDev &d = h->d;
    double *buf = nullptr;
    CKB(B, cudaMallocAsync((void **)&buf, 8 * 3 * N, B->stream));
    long long off = 0;
    for (int b = 0; b < 9; ++b) {
        if (!(mask & (1u << b))) continue;
        const uint32_t bit = 1u << b;
        if (bit == DPS_FIELD_RHO || bit == DPS_FIELD_UBAR || bit == DPS_FIELD_UF || bit == DPS_FIELD_P ||
            bit == DPS_FIELD_FEXT) {
            int what = bit == DPS_FIELD_RHO ? 0 : bit == DPS_FIELD_UBAR ? 1 : bit == DPS_FIELD_UF ? 2 : bit == DPS_FIELD_P ? 3 : 4;
            PREC_CALL(B, (launch_fluid_export<double, double>(d.pdf, d.eps, d.fpf, d.g, fb, B->parity, what, buf, B->stream)),
                      (launch_fluid_export<float, float>(d.pdf, d.eps, d.fpf, d.g, fb, B->parity, what, buf, B->stream)),
                      (launch_fluid_export<__half, float>(d.pdf, d.eps, d.fpf, d.g, fb, B->parity, what, buf, B->stream)));
        } else {
            const void *src = bit == DPS_FIELD_EPS ? d.eps : bit == DPS_FIELD_FPF ? d.fpf : bit == DPS_FIELD_GRADP ? d.gradP : d.DuDt;
            if (B->fel == 8)
                launch_to_double<double>(src, planes[b] * N, buf, B->stream);
            else
                launch_to_double<float>(src, planes[b] * N, buf, B->stream);
        }
        CKB(B, cudaMemcpyAsync(out + off, buf, 8 * planes[b] * N, cudaMemcpyDeviceToHost, B->stream));
        off += planes[b] * N;
    }
    CKB(B, cudaFreeAsync(buf, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    return DPS_OK;
}

static int box_read_particles(Batch *B, BoxHost *h, double *x3, double *u3, double *w3, double *F3, long long cap) {
    const long long np = h->d.np;
    if (cap < np) FAILB(B, DPS_ERR_ARG, "capacity %lld < %lld particles", cap, np);
    if (np == 0) return DPS_OK;
    // the box's device-table entry holds its current particle set; for a box
    // not (yet) in the table the host copy is current once pulled
    int k = -1;
    for (size_t q = 0; q < B->dev_order.size(); ++q)
        if (B->dev_order[q] == h) k = (int)q;
    if (k < 0) {
        int rc = pull_state(B);
        if (rc) return rc;
    }
    const size_t n = 12 * (size_t)np;
    if (n > B->cap_dpstage) {
        void *p = dalloc_raw(B, n * 8);
        if (!p) FAILB(B, DPS_ERR_OOM, "read-back buffer allocation failed");
        if (B->d_pstage) {
            CKB(B, cudaStreamSynchronize(B->stream));
            dfree_raw(B, B->d_pstage);
            B->allocs.erase(std::remove(B->allocs.begin(), B->allocs.end(), (void *)B->d_pstage), B->allocs.end());
        }
        B->allocs.push_back(p);
        B->d_pstage = (double *)p;
        B->cap_dpstage = n;
    }
    if (n > B->cap_hpstage) {
        if (B->h_pstage) cudaFreeHost(B->h_pstage);
        B->h_pstage = nullptr;
        B->cap_hpstage = 0;
        CKB(B, cudaMallocHost((void **)&B->h_pstage, n * 8));
        B->cap_hpstage = n;
    }
    launch_particles_export4(k >= 0 ? B->d_table : nullptr, k, h->d.pf[h->d.cur], h->d.pi[h->d.cur] + IID * h->d.cap,
                             h->d.cap, np, B->d_pstage, B->stream);
    CKB(B, cudaMemcpyAsync(B->h_pstage, B->d_pstage, n * 8, cudaMemcpyDeviceToHost, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    double *dst[4] = {x3, u3, w3, F3};
    for (int q = 0; q < 4; ++q)
        if (dst[q]) std::memcpy(dst[q], B->h_pstage + (size_t)q * 3 * np, 8 * 3 * (size_t)np);
    return DPS_OK;
}

static int box_write_particles(Batch *B, BoxHost *h, long long n, const double *x3, const double *u3, const double *w3) {
    if (n != h->d.np) FAILB(B, DPS_ERR_ARG, "n must equal the number of particles (%lld)", h->d.np);
    if (n == 0) return DPS_OK;
    if (x3)
        for (long long i = 0; i < 3 * n; ++i)
            if (!std::isfinite(x3[i])) FAILB(B, DPS_ERR_ARG, "non-finite position");
    int rc = pull_state(B);
    if (rc) return rc;
    double *buf = nullptr;
    CKB(B, cudaMallocAsync((void **)&buf, 8 * 3 * n, B->stream));
    const double *src[3] = {x3, u3, w3};
    double *pf = h->d.pf[h->d.cur];
    const int *ids = h->d.pi[h->d.cur] + IID * h->d.cap;
    for (int k = 0; k < 3; ++k) {
        if (!src[k]) continue;
        CKB(B, cudaMemcpyAsync(buf, src[k], 8 * 3 * n, cudaMemcpyHostToDevice, B->stream));
        launch_particles_import(pf, 3 * k, h->d.cap, n, ids, buf, B->stream);
    }
    CKB(B, cudaFreeAsync(buf, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    if (x3) h->prepared = false;
    return DPS_OK;
}

static int box_stats(Batch *B, BoxHost *h, dps_stats *s) {
    std::memset(s, 0, sizeof(*s));
    int rc = pull_state(B);
    if (rc) return rc;
    compute_phys(h);
    const BoxDev &d = h->d;
    double fl[12], pt[6];
    PREC_CALL(B, (launch_fluid_sums<double, double>(d.pdf, d.eps, d.fpf, d.g, d.ph.fb, B->parity, h->d_red, h->d_redout, B->stream)),
              (launch_fluid_sums<float, float>(d.pdf, d.eps, d.fpf, d.g, d.ph.fb, B->parity, h->d_red, h->d_redout, B->stream)),
              (launch_fluid_sums<__half, float>(d.pdf, d.eps, d.fpf, d.g, d.ph.fb, B->parity, h->d_red, h->d_redout, B->stream)));
    CKB(B, cudaMemcpyAsync(fl, h->d_redout, sizeof(fl), cudaMemcpyDeviceToHost, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    launch_particle_sums(d.pf[d.cur], d.pf[d.cur], d.cap, d.np, h->d_red, h->d_redout, B->stream);
    CKB(B, cudaMemcpyAsync(pt, h->d_redout, sizeof(pt), cudaMemcpyDeviceToHost, B->stream));
    unsigned long long cnt[CNT_N];
    CKB(B, cudaMemcpyAsync(cnt, d.counters, sizeof(cnt), cudaMemcpyDeviceToHost, B->stream));
    int st = 0;
    CKB(B, cudaMemcpyAsync(&st, d.status, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    const double N = (double)d.g.ncell;
    s->mass = fl[0];
    for (int a = 0; a < 3; ++a) {
        s->fluid_j[a] = fl[1 + a];
        s->fluid_ubar[a] = fl[4 + a];
        s->uf_mean[a] = fl[7 + a] / N;
        s->particle_momentum[a] = pt[a];
        s->up_mean[a] = d.np ? pt[3 + a] / d.np : 0.0;
        s->u_pS[a] = s->up_mean[a] - s->uf_mean[a];
    }
    s->eps_min_seen = fl[10];
    s->step = h->steps;
    s->n_particles = d.np;
    s->n_eps_clamp = (int64_t)cnt[CNT_EPS_CLAMP];
    s->n_lub_limited = (int64_t)cnt[CNT_LUB_LIMITED];
    s->status = h->sticky | st;
    return DPS_OK;
}

// ---- checkpoint / resume ------------------------------------------------------------------
// A checkpoint holds the state that one coupled step carries into the next:
// the PDFs as stored (canonical layout, plane q of cell x holding f_q(x),
// whatever the AA parity), eps_f, the f_pf applied in the last step, the
// fluid velocity of the last step (Du_f/Dt), the current particle set (all
// planes in cell-sorted order, u at the last subcycle start included), the
// counters and status, and the host-side box state (step count, closure,
// subcycle history flags, parity).  Everything else is re-derived on load by
// the linked-cell sort of Algorithm 1's initialisation, which on an already
// sorted set reproduces the neighbour lists, float copies and kernel
// weights bit for bit.
struct CkptHeader {
    char magic[8];
    int version, precision;
    int n[3], per[3];
    double tau, rho_f;
    long long np, steps;
    int parity, have_uprev, have_usub, sticky;
    int have_closure, prepared;
    double sumV, sumWb, dmax, dmin;
    dps_closure cl;
};
static const char CKPT_MAGIC[8] = {'D', 'P', 'S', 'C', 'K', 'P', 'T', '1'};

static size_t box_state_bytes(const Batch *B, const BoxHost *h) {
    const size_t N = (size_t)h->d.g.ncell, np = (size_t)h->d.np;
    return sizeof(CkptHeader) + 19 * N * B->pdf_elem + 7 * N * B->fel + np * ((size_t)NPF * 8 + (size_t)NPI * 4) +
           8 * CNT_N + 8;
}

static int box_save_state(Batch *B, BoxHost *h, void *buf, size_t cap) {
    if (!buf) FAILB(B, DPS_ERR_ARG, "null buffer");
    const size_t need = box_state_bytes(B, h);
    if (cap < need) FAILB(B, DPS_ERR_ARG, "buffer of %zu bytes, the state needs %zu", cap, need);
    int rc = pull_state(B);
    if (rc) return rc;
    const BoxDev &d = h->d;
    const size_t N = (size_t)d.g.ncell, np = (size_t)d.np, cp = (size_t)d.cap;
    CkptHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, CKPT_MAGIC, 8);
    hd.version = 1;
    hd.precision = B->prec;
    for (int a = 0; a < 3; ++a) {
        hd.n[a] = d.g.n[a];
        hd.per[a] = d.g.per[a];
    }
    hd.tau = h->tau;
    hd.rho_f = h->rho_f;
    hd.np = d.np;
    hd.steps = h->steps;
    hd.parity = B->parity;
    hd.have_uprev = d.have_uprev;
    hd.have_usub = d.have_usub;
    hd.sticky = h->sticky;
    hd.have_closure = h->have_closure;
    hd.prepared = h->prepared;
    hd.sumV = h->sumV;
    hd.sumWb = h->sumWb;
    hd.dmax = h->dmax;
    hd.dmin = h->dmin;
    hd.cl = h->cl;
    char *o = (char *)buf;
    std::memcpy(o, &hd, sizeof(hd));
    o += sizeof(hd);
    const size_t pdf_bytes = 19 * N * B->pdf_elem;
    cudaStream_t s = B->stream;
    if (B->parity) {
        void *tmp = nullptr;
        CKB(B, cudaMallocAsync(&tmp, pdf_bytes, s));
        launch_pdf_relayout(d.pdf, d.g, (int)B->pdf_elem, 1, tmp, s);
        CKB(B, cudaMemcpyAsync(o, tmp, pdf_bytes, cudaMemcpyDeviceToHost, s));
        CKB(B, cudaFreeAsync(tmp, s));
    } else {
        CKB(B, cudaMemcpyAsync(o, d.pdf, pdf_bytes, cudaMemcpyDeviceToHost, s));
    }
    o += pdf_bytes;
    CKB(B, cudaMemcpyAsync(o, d.eps, N * B->fel, cudaMemcpyDeviceToHost, s));
    o += N * B->fel;
    CKB(B, cudaMemcpyAsync(o, d.fpf, 3 * N * B->fel, cudaMemcpyDeviceToHost, s));
    o += 3 * N * B->fel;
    CKB(B, cudaMemcpyAsync(o, d.uprev, 3 * N * B->fel, cudaMemcpyDeviceToHost, s));
    o += 3 * N * B->fel;
    if (np) {
        CKB(B, cudaMemcpy2DAsync(o, np * 8, d.pf[d.cur], cp * 8, np * 8, NPF, cudaMemcpyDeviceToHost, s));
        o += (size_t)NPF * np * 8;
        CKB(B, cudaMemcpy2DAsync(o, np * 4, d.pi[d.cur], cp * 4, np * 4, NPI, cudaMemcpyDeviceToHost, s));
        o += (size_t)NPI * np * 4;
    }
    CKB(B, cudaMemcpyAsync(o, d.counters, 8 * CNT_N, cudaMemcpyDeviceToHost, s));
    o += 8 * CNT_N;
    std::memset(o, 0, 8);
    CKB(B, cudaMemcpyAsync(o, d.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CKB(B, cudaStreamSynchronize(s));
    return DPS_OK;
}

// restore a checkpoint into box h, which has the geometry, fluid and form of
// the saved box and room for its particles
static int box_load_state(Batch *B, BoxHost *h, const void *buf, size_t size) {
    if (!buf || size < sizeof(CkptHeader)) FAILB(B, DPS_ERR_ARG, "not a checkpoint (too short)");
    CkptHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, CKPT_MAGIC, 8) != 0 || hd.version != 1) FAILB(B, DPS_ERR_ARG, "not a checkpoint");
    BoxDev &d = h->d;
    if (hd.precision != B->prec) FAILB(B, DPS_ERR_ARG, "checkpoint precision form %d, box %d", hd.precision, B->prec);
    for (int a = 0; a < 3; ++a)
        if (hd.n[a] != d.g.n[a] || (hd.per[a] != 0) != (d.g.per[a] != 0))
            FAILB(B, DPS_ERR_ARG, "checkpoint lattice or boundaries differ from the box");
    if (hd.tau != h->tau || hd.rho_f != h->rho_f) FAILB(B, DPS_ERR_ARG, "checkpoint tau or rho_f differ from the box");
    if (hd.np < 0 || hd.np > h->max_particles)
        FAILB(B, DPS_ERR_ARG, "checkpoint holds %lld particles, the box has room for %lld", hd.np, h->max_particles);
    if (hd.have_closure) {
        int rc = check_closure(B, &hd.cl);
        if (rc) return rc;
    }
    int rc = pull_state(B);
    if (rc) return rc;
    const size_t N = (size_t)d.g.ncell, np = (size_t)hd.np, cp = (size_t)d.cap;
    h->d.np = hd.np;
    if (box_state_bytes(B, h) > size) {
        h->d.np = 0;
        FAILB(B, DPS_ERR_ARG, "checkpoint truncated (%zu bytes)", size);
    }
    h->sumV = hd.sumV;
    h->sumWb = hd.sumWb;
    h->dmax = hd.dmax;
    h->dmin = hd.dmin;
    h->cl = hd.cl;
    h->have_closure = hd.have_closure != 0;
    h->steps = hd.steps;
    h->sticky = hd.sticky;
    const char *in = (const char *)buf + sizeof(hd);
    const size_t pdf_bytes = 19 * N * B->pdf_elem;
    const char *in_pdf = in;
    const char *in_fields = in + pdf_bytes;
    const char *in_part = in_fields + 7 * N * B->fel;
    const char *in_tail = in_part + np * ((size_t)NPF * 8 + (size_t)NPI * 4);
    cudaStream_t s = B->stream;
    // the particle set first: the initialisation sort below re-derives the
    // linked cells, lists, float copies and weights from it
    if (np) {
        CKB(B, cudaMemcpy2DAsync(d.pf[d.cur], cp * 8, in_part, np * 8, np * 8, NPF, cudaMemcpyHostToDevice, s));
        CKB(B, cudaMemcpy2DAsync(d.pi[d.cur], cp * 4, in_part + (size_t)NPF * np * 8, np * 4, np * 4, NPI,
                                 cudaMemcpyHostToDevice, s));
    }
    CKB(B, cudaStreamSynchronize(s));
    h->prepared = false;
    B->layout_dirty = true;
    if (h->have_closure && hd.prepared) {
        if ((rc = ready(B))) return rc;
    }
    // subcycle history flags and the AA parity of the saved step
    if ((rc = pull_state(B))) return rc;
    d.have_uprev = hd.have_uprev;
    d.have_usub = hd.have_usub;
    if (B->boxes.size() == 1) B->parity = hd.parity;
    if ((rc = push_layout(B))) return rc;
    if (B->parity) {
        void *tmp = nullptr;
        CKB(B, cudaMallocAsync(&tmp, pdf_bytes, s));
        CKB(B, cudaMemcpyAsync(tmp, in_pdf, pdf_bytes, cudaMemcpyHostToDevice, s));
        launch_pdf_relayout(tmp, d.g, (int)B->pdf_elem, 0, d.pdf, s);
        CKB(B, cudaFreeAsync(tmp, s));
    } else {
        CKB(B, cudaMemcpyAsync(d.pdf, in_pdf, pdf_bytes, cudaMemcpyHostToDevice, s));
    }
    CKB(B, cudaMemcpyAsync(d.eps, in_fields, N * B->fel, cudaMemcpyHostToDevice, s));
    CKB(B, cudaMemcpyAsync(d.fpf, in_fields + N * B->fel, 3 * N * B->fel, cudaMemcpyHostToDevice, s));
    CKB(B, cudaMemcpyAsync(d.uprev, in_fields + 4 * N * B->fel, 3 * N * B->fel, cudaMemcpyHostToDevice, s));
    CKB(B, cudaMemcpyAsync(d.counters, in_tail, 8 * CNT_N, cudaMemcpyHostToDevice, s));
    CKB(B, cudaMemcpyAsync(d.status, in_tail + 8 * CNT_N, sizeof(int), cudaMemcpyHostToDevice, s));
    CKB(B, cudaStreamSynchronize(s));
    h->prepared = hd.prepared != 0 && h->have_closure;
    invalidate_graph(B);
    return DPS_OK;
}

// ===============================================================================================
// domain = batch of one box
// ===============================================================================================
struct dps_domain {
    Batch B;
    BoxHost *box = nullptr;
};

#define DOM_ERR(h) (h)->B.err

extern "C" {

const char *dps_version(void) { return "dps-gb300 0.2 (sm_103a)"; }

const char *dps_last_error(dps_handle h) { return h ? h->B.err.c_str() : g_create_err.c_str(); }

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
    if (desc->precision < DPS_F64 || desc->precision > DPS_F16S || ((desc->alloc == nullptr) != (desc->free == nullptr))) {
        g_create_err = "invalid domain description (precision, allocator pair)";
        return DPS_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if (desc->n[a] < 1) {
            g_create_err = "lattice size must be >= 1 per axis";
            return DPS_ERR_ARG;
        }
    if (!(desc->tau > 0.5) || !(desc->rho_f > 0.0) || desc->max_particles < 0 || desc->max_particles >= (1LL << 31)) {
        g_create_err = "invalid domain description (tau > 0.5, rho_f > 0, particle capacity)";
        return DPS_ERR_ARG;
    }
    dps_domain *h = new dps_domain();
    if (batch_init(&h->B, desc->precision, desc->stream, desc->alloc, desc->free, desc->alloc_ctx)) {
        g_create_err = "cudaStreamCreate failed";
        delete h;
        return DPS_ERR_CUDA;
    }
    BoxHost *bx = nullptr;
    int rc = box_create(&h->B, desc->n, desc->periodic, desc->tau, desc->rho_f, desc->max_particles, &bx);
    if (rc) {
        g_create_err = h->B.err;
        batch_release(&h->B);
        delete h;
        return rc;
    }
    h->box = bx;
    h->B.boxes.push_back(bx);
    h->B.layout_dirty = true;
    *out = h;
    return DPS_OK;
}

int dps_destroy(dps_handle h) {
    if (!h) return DPS_ERR_ARG;
    batch_release(&h->B);
    delete h;
    return DPS_OK;
}

int dps_add_particles(dps_handle h, int64_t n, const double *x3, const double *u3, const double *w3, const double *d,
                      const double *rho_p) {
    if (!h) return DPS_ERR_ARG;
    return box_add_particles(&h->B, h->box, n, x3, u3, w3, d, rho_p);
}

int dps_write_particles(dps_handle h, int64_t n, const double *x3, const double *u3, const double *w3) {
    if (!h) return DPS_ERR_ARG;
    return box_write_particles(&h->B, h->box, n, x3, u3, w3);
}

int dps_set_closure(dps_handle h, const dps_closure *c) {
    if (!h) return DPS_ERR_ARG;
    int rc = check_closure(&h->B, c);
    if (rc) return rc;
    h->box->cl = *c;
    h->box->have_closure = true;
    h->box->prepared = false;
    h->B.layout_dirty = true;
    return DPS_OK;
}

int dps_prepare(dps_handle h) {
    if (!h) return DPS_ERR_ARG;
    h->box->prepared = false;
    return ready(&h->B);
}

int dps_step_async(dps_handle h, int64_t n) {
    if (!h || n < 0) return DPS_ERR_ARG;
    return run_steps(&h->B, n);
}

int dps_check(dps_handle h) {
    if (!h) return DPS_ERR_ARG;
    return check_boxes(&h->B);
}

int dps_step(dps_handle h, int64_t n) {
    int rc = dps_step_async(h, n);
    if (rc) return rc;
    return check_boxes(&h->B);
}

int dps_collide_stream(dps_handle h, int64_t n) {
    if (!h || n < 0) return DPS_ERR_ARG;
    Batch *B = &h->B;
    int rc = pull_state(B);
    if (rc) return rc;
    if ((rc = push_layout(B))) return rc;
    for (int64_t s = 0; s < n; ++s) {
        enqueue_collide(B, B->parity, false);
        B->parity ^= 1;
    }
    return check_boxes(B);
}

int dps_sync(dps_handle h) {
    if (!h) return DPS_ERR_ARG;
    CKB(&h->B, cudaStreamSynchronize(h->B.stream));
    return DPS_OK;
}

int dps_read_fields(dps_handle h, uint32_t mask, double *out, int64_t cap) {
    if (!h) return DPS_ERR_ARG;
    return box_read_fields(&h->B, h->box, mask, out, cap);
}

int dps_write_fields(dps_handle h, uint32_t mask, const double *in, int64_t count) {
    if (!h || !in) return DPS_ERR_ARG;
    Batch *B = &h->B;
    BoxDev &d = h->box->d;
    if (mask & ~(DPS_FIELD_EPS | DPS_FIELD_FPF)) FAILB(B, DPS_ERR_ARG, "only eps_f and f_pf can be written");
    const long long N = d.g.ncell;
    long long need = ((mask & DPS_FIELD_EPS) ? N : 0) + ((mask & DPS_FIELD_FPF) ? 3 * N : 0);
    if (count < need) FAILB(B, DPS_ERR_ARG, "input has %lld values, %lld needed", (long long)count, need);
    if (mask & DPS_FIELD_EPS)
        for (long long c = 0; c < N; ++c)
            if (!(in[c] > 0.0 && in[c] <= 1.0)) FAILB(B, DPS_ERR_ARG, "eps_f must lie in (0, 1]");
    double *buf = nullptr;
    CKB(B, cudaMallocAsync((void **)&buf, 8 * 3 * N, B->stream));
    long long off = 0;
    if (mask & DPS_FIELD_EPS) {
        CKB(B, cudaMemcpyAsync(buf, in, 8 * N, cudaMemcpyHostToDevice, B->stream));
        if (B->fel == 8) launch_from_double<double>(buf, N, d.eps, B->stream);
        else launch_from_double<float>(buf, N, d.eps, B->stream);
        off += N;
    }
    if (mask & DPS_FIELD_FPF) {
        CKB(B, cudaMemcpyAsync(buf, in + off, 8 * 3 * N, cudaMemcpyHostToDevice, B->stream));
        if (B->fel == 8) launch_from_double<double>(buf, 3 * N, d.fpf, B->stream);
        else launch_from_double<float>(buf, 3 * N, d.fpf, B->stream);
    }
    CKB(B, cudaFreeAsync(buf, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    return DPS_OK;
}

int dps_read_pdfs(dps_handle h, double *out, int64_t cap) {
    if (!h || !out) return DPS_ERR_ARG;
    Batch *B = &h->B;
    int rc = pull_state(B);
    if (rc) return rc;
    const BoxDev &d = h->box->d;
    const long long N = d.g.ncell;
    if (cap < (long long)Q * N) FAILB(B, DPS_ERR_ARG, "output capacity too small");
    double *buf = nullptr;
    CKB(B, cudaMallocAsync((void **)&buf, 8 * Q * N, B->stream));
    PREC_CALL(B, launch_pdf_export<double>(d.pdf, d.g, B->parity, buf, B->stream),
              launch_pdf_export<float>(d.pdf, d.g, B->parity, buf, B->stream),
              launch_pdf_export<__half>(d.pdf, d.g, B->parity, buf, B->stream));
    CKB(B, cudaMemcpyAsync(out, buf, 8 * Q * N, cudaMemcpyDeviceToHost, B->stream));
    CKB(B, cudaFreeAsync(buf, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    return DPS_OK;
}

int dps_write_pdfs(dps_handle h, const double *in, int64_t count) {
    if (!h || !in) return DPS_ERR_ARG;
    Batch *B = &h->B;
    int rc = pull_state(B);
    if (rc) return rc;
    BoxDev &d = h->box->d;
    const long long N = d.g.ncell;
    if (count < (long long)Q * N) FAILB(B, DPS_ERR_ARG, "input too small");
    double *buf = nullptr;
    CKB(B, cudaMallocAsync((void **)&buf, 8 * Q * N, B->stream));
    CKB(B, cudaMemcpyAsync(buf, in, 8 * Q * N, cudaMemcpyHostToDevice, B->stream));
    PREC_CALL(B, launch_pdf_import<double>(d.pdf, N, buf, B->stream), launch_pdf_import<float>(d.pdf, N, buf, B->stream),
              launch_pdf_import<__half>(d.pdf, N, buf, B->stream));
    CKB(B, cudaFreeAsync(buf, B->stream));
    CKB(B, cudaStreamSynchronize(B->stream));
    B->parity = 0;  // imported in the canonical layout
    invalidate_graph(B);
    return DPS_OK;
}

int dps_read_particles(dps_handle h, double *x3, double *u3, double *w3, double *F3, int64_t cap) {
    if (!h) return DPS_ERR_ARG;
    return box_read_particles(&h->B, h->box, x3, u3, w3, F3, cap);
}

int dps_stats_get(dps_handle h, dps_stats *s) {
    if (!h || !s) return DPS_ERR_ARG;
    return box_stats(&h->B, h->box, s);
}

int dps_state_size(dps_handle h, size_t *bytes) {
    if (!h || !bytes) return DPS_ERR_ARG;
    *bytes = box_state_bytes(&h->B, h->box);
    return DPS_OK;
}

int dps_save_state(dps_handle h, void *buf, size_t cap) {
    if (!h) return DPS_ERR_ARG;
    return box_save_state(&h->B, h->box, buf, cap);
}

int dps_load_state(dps_handle h, const void *buf, size_t size) {
    if (!h) return DPS_ERR_ARG;
    return box_load_state(&h->B, h->box, buf, size);
}

int dps_read_cell_list(dps_handle h, int32_t *cell_start, int32_t *order, int64_t cap_cells, int64_t cap_particles) {
    if (!h || !cell_start || !order) return DPS_ERR_ARG;
    Batch *B = &h->B;
    const BoxDev &d0 = h->box->d;
    if (cap_cells < d0.g.ncell + 1 || cap_particles < d0.np) FAILB(B, DPS_ERR_ARG, "capacity too small");
    int rc = h->box->have_closure && !h->box->prepared ? ready(B) : pull_state(B);
    if (rc) return rc;
    const BoxDev &d = h->box->d;
    CKB(B, cudaMemcpy(cell_start, d.cell_start, 4 * (d.g.ncell + 1), cudaMemcpyDeviceToHost));
    if (d.np) CKB(B, cudaMemcpy(order, d.pi[d.cur] + IID * d.cap, 4 * d.np, cudaMemcpyDeviceToHost));
    return DPS_OK;
}

int dps_read_neighbor_list(dps_handle h, int64_t *offsets, int32_t *partners, int64_t cap) {
    if (!h || !offsets) return DPS_ERR_ARG;
    Batch *B = &h->B;
    int rc = h->box->have_closure && !h->box->prepared ? ready(B) : pull_state(B);
    if (rc) return rc;
    const BoxDev &d = h->box->d;
    const long long np = d.np;
    if (np == 0 || !d.nlist) {
        for (long long i = 0; i <= np; ++i) offsets[i] = 0;
        return DPS_OK;
    }
    std::vector<int> cnt((size_t)np), ids((size_t)np), rows((size_t)np * d.maxn);
    CKB(B, cudaMemcpy(cnt.data(), d.nlist_n, 4 * np, cudaMemcpyDeviceToHost));
    CKB(B, cudaMemcpy(ids.data(), d.pi[d.cur] + IID * d.cap, 4 * np, cudaMemcpyDeviceToHost));
    CKB(B, cudaMemcpy(rows.data(), d.nlist, 4 * (size_t)np * d.maxn, cudaMemcpyDeviceToHost));
    // rows by insertion id, partners as insertion ids in ascending order
    std::vector<long long> len((size_t)np, 0);
    for (long long s = 0; s < np; ++s) len[ids[s]] = cnt[s];
    offsets[0] = 0;
    for (long long i = 0; i < np; ++i) offsets[i + 1] = offsets[i] + len[i];
    if (!partners) return DPS_OK;
    if (cap < offsets[np]) FAILB(B, DPS_ERR_ARG, "capacity %lld < %lld list entries", (long long)cap, (long long)offsets[np]);
    for (long long s = 0; s < np; ++s) {
        int32_t *o = partners + offsets[ids[s]];
        for (int k = 0; k < cnt[s]; ++k) o[k] = ids[rows[(size_t)s * d.maxn + k]];
        std::sort(o, o + cnt[s]);
    }
    return DPS_OK;
}

int dps_bin_edge(dps_handle h, int *R) {
    if (!h || !R) return DPS_ERR_ARG;
    if (!h->box->have_closure) FAILB(&h->B, DPS_ERR_STATE, "no closure");
    compute_phys(h->box);
    *R = h->box->d.R;
    return DPS_OK;
}

// ---- tracing -------------------------------------------------------------------------------
static int b_set_timing(Batch *B, int enable) {
    if ((enable != 0) != B->timing) {
        CKB(B, cudaStreamSynchronize(B->stream));
        B->timing = enable != 0;
        invalidate_graph(B);
    }
    return DPS_OK;
}
static int b_collect_timing(Batch *B) {
    CKB(B, cudaStreamSynchronize(B->stream));
    if (!B->timing) return DPS_OK;
    for (size_t k = 0; k < B->ev_used; ++k) {
        float ms = 0.f;
        CKB(B, cudaEventElapsedTime(&ms, B->ev[2 * k], B->ev[2 * k + 1]));
        B->ph_ms[B->ev_phase[k]] += ms;
        B->ph_nl[B->ev_phase[k]] += B->ev_nl[k];
    }
    return DPS_OK;
}
static void b_get_timing(Batch *B, double *ms, int64_t *nl, int reset) {
    for (int k = 0; k < NPH; ++k) {
        if (ms) ms[k] = B->ph_ms[k];
        if (nl) nl[k] = B->ph_nl[k];
        if (reset) {
            B->ph_ms[k] = 0;
            B->ph_nl[k] = 0;
        }
    }
}
static long long b_launches_per_step(Batch *B) {
    long long np = 0;
    for (BoxHost *h : B->boxes) np += h->d.np;
    const int pl = np > 0;
    const int n_int = B->boxes.empty() ? 1 : B->boxes[0]->cl.n_int;
    const int n_dem = B->boxes.empty() ? 1 : B->boxes[0]->cl.n_dem;
    const int f64 = B->prec == DPS_F64;
    return 2 + 2 + (long long)n_int * (2 * pl + 2 + pl * n_dem * 2 + 3 + (5 + 2 * f64) * pl + 1 + 1);
}

int dps_set_timing(dps_handle h, int enable) { return h ? b_set_timing(&h->B, enable) : DPS_ERR_ARG; }
int dps_collect_timing(dps_handle h) { return h ? b_collect_timing(&h->B) : DPS_ERR_ARG; }
int dps_get_timing(dps_handle h, double ms[DPS_NPHASE], int64_t launches[DPS_NPHASE], int reset) {
    if (!h) return DPS_ERR_ARG;
    b_get_timing(&h->B, ms, launches, reset);
    return DPS_OK;
}
int dps_launches_per_step(dps_handle h, int64_t *n) {
    if (!h || !n) return DPS_ERR_ARG;
    if (!h->box->have_closure) FAILB(&h->B, DPS_ERR_STATE, "no closure");
    *n = b_launches_per_step(&h->B);
    return DPS_OK;
}

// ===============================================================================================
// batch API
// ===============================================================================================
struct dps_batch_s {
    Batch B;
    std::vector<std::pair<int, BoxHost *>> ids;  // id -> box
    int next_id = 0;
};

static BoxHost *find_box(dps_batch b, int id) {
    for (auto &p : b->ids)
        if (p.first == id) return p.second;
    return nullptr;
}

#define BOX_OR_FAIL(b, id, h)                                              \
    BoxHost *h = find_box(b, id);                                          \
    if (!h) FAILB(&(b)->B, DPS_ERR_ARG, "unknown box id %d", (int)(id));

int dps_batch_create(const dps_batch_desc *desc, dps_batch *out) {
    if (out) *out = nullptr;
    if (!desc || !out || desc->precision < DPS_F64 || desc->precision > DPS_F16S ||
        ((desc->alloc == nullptr) != (desc->free == nullptr))) {
        g_create_err = "invalid batch description";
        return DPS_ERR_ARG;
    }
    dps_batch b = new dps_batch_s();
    batch_init(&b->B, desc->precision, desc->stream, desc->alloc, desc->free, desc->alloc_ctx);
    *out = b;
    return DPS_OK;
}

const char *dps_batch_last_error(dps_batch b) { return b ? b->B.err.c_str() : g_create_err.c_str(); }

int dps_batch_destroy(dps_batch b) {
    if (!b) return DPS_ERR_ARG;
    batch_release(&b->B);
    delete b;
    return DPS_OK;
}

int dps_batch_add_box(dps_batch b, const int n[3], const int periodic[3], double tau, double rho_f,
                      int64_t max_particles, int *box) {
    if (!b || !n || !periodic || !box) return DPS_ERR_ARG;
    int rc = pull_state(&b->B);
    if (rc) return rc;
    BoxHost *h = nullptr;
    rc = box_create(&b->B, n, periodic, tau, rho_f, max_particles, &h);
    if (rc) return rc;
    h->user_id = b->next_id;
    b->B.boxes.push_back(h);
    b->ids.push_back({b->next_id, h});
    *box = b->next_id++;
    b->B.layout_dirty = true;
    return DPS_OK;
}

int dps_batch_remove_box(dps_batch b, int id) {
    if (!b) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    int rc = pull_state(&b->B);
    if (rc) return rc;
    forget_box(&b->B, h);
    b->ids.erase(std::remove_if(b->ids.begin(), b->ids.end(), [&](const std::pair<int, BoxHost *> &p) { return p.first == id; }),
                 b->ids.end());
    box_free(&b->B, h);
    delete h;
    b->B.layout_dirty = true;
    invalidate_graph(&b->B);
    return DPS_OK;
}

int dps_batch_add_particles(dps_batch b, int id, int64_t n, const double *x3, const double *u3, const double *w3,
                            const double *d, const double *rho_p) {
    if (!b) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    return box_add_particles(&b->B, h, n, x3, u3, w3, d, rho_p);
}

int dps_batch_set_closure(dps_batch b, int id, const dps_closure *c) {
    if (!b) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    int rc = check_closure(&b->B, c);
    if (rc) return rc;
    h->cl = *c;
    h->have_closure = true;
    h->prepared = false;
    b->B.layout_dirty = true;
    return DPS_OK;
}

int dps_batch_step_async(dps_batch b, int64_t n) {
    if (!b || n < 0) return DPS_ERR_ARG;
    return run_steps(&b->B, n);
}
int dps_batch_check(dps_batch b) { return b ? check_boxes(&b->B) : DPS_ERR_ARG; }
int dps_batch_step(dps_batch b, int64_t n) {
    int rc = dps_batch_step_async(b, n);
    return rc ? rc : check_boxes(&b->B);
}

int dps_batch_read_particles(dps_batch b, int id, double *x3, double *u3, double *w3, double *F3, int64_t cap) {
    if (!b) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    return box_read_particles(&b->B, h, x3, u3, w3, F3, cap);
}
int dps_batch_read_fields(dps_batch b, int id, uint32_t mask, double *out, int64_t cap) {
    if (!b) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    return box_read_fields(&b->B, h, mask, out, cap);
}
int dps_batch_stats(dps_batch b, int id, dps_stats *s) {
    if (!b || !s) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    return box_stats(&b->B, h, s);
}
int dps_batch_particle_mean(dps_batch b, int id, double u[3]) {
    if (!b || !u) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    Batch *B = &b->B;
    int rc = pull_state(B);
    if (rc) return rc;
    const BoxDev &d = h->d;
    double pt[6] = {0, 0, 0, 0, 0, 0};
    if (d.np) {
        launch_particle_sums(d.pf[d.cur], d.pf[d.cur], d.cap, d.np, h->d_red, h->d_redout, B->stream);
        CKB(B, cudaMemcpyAsync(pt, h->d_redout, sizeof(pt), cudaMemcpyDeviceToHost, B->stream));
        CKB(B, cudaStreamSynchronize(B->stream));
    }
    for (int a = 0; a < 3; ++a) u[a] = d.np ? pt[3 + a] / d.np : 0.0;
    return DPS_OK;
}
int dps_batch_state_size(dps_batch b, int id, size_t *bytes) {
    if (!b || !bytes) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    *bytes = box_state_bytes(&b->B, h);
    return DPS_OK;
}
int dps_batch_save_box(dps_batch b, int id, void *buf, size_t cap) {
    if (!b) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    return box_save_state(&b->B, h, buf, cap);
}
int dps_batch_load_box(dps_batch b, int id, const void *buf, size_t size) {
    if (!b) return DPS_ERR_ARG;
    BOX_OR_FAIL(b, id, h);
    return box_load_state(&b->B, h, buf, size);
}
int dps_batch_num_boxes(dps_batch b, int *n) {
    if (!b || !n) return DPS_ERR_ARG;
    *n = (int)b->B.boxes.size();
    return DPS_OK;
}
int dps_batch_set_tuning(dps_batch b, const int cfg[5]) {
    if (!b || !cfg) return DPS_ERR_ARG;
    for (int k = 0; k < 4; ++k)
        if (cfg[k] < 32 || cfg[k] > (1 << 20)) FAILB(&b->B, DPS_ERR_ARG, "invalid launch shape");
    if (cfg[0] > 256 || cfg[2] > 256 || (cfg[0] & 31) || (cfg[2] & 31))
        FAILB(&b->B, DPS_ERR_ARG, "threads per block must be a multiple of 32, at most 256");
    if (cfg[4] < 0 || cfg[4] > 7) FAILB(&b->B, DPS_ERR_ARG, "collide-stream variant must be 0 ... 7");
    int rc = pull_state(&b->B);
    if (rc) return rc;
    b->B.tune = Tuning{cfg[0], cfg[1], cfg[2], cfg[3], cfg[4]};
    b->B.shape_fixed = true;
    b->B.layout_dirty = true;
    return DPS_OK;
}
int dps_batch_get_tuning(dps_batch b, int cfg[5]) {
    if (!b || !cfg) return DPS_ERR_ARG;
    cfg[0] = b->B.tune.cell_block;
    cfg[1] = b->B.tune.cell_tile;
    cfg[2] = b->B.tune.part_block;
    cfg[3] = b->B.tune.part_tile;
    cfg[4] = b->B.tune.k1v;
    return DPS_OK;
}

// autotuner: candidate launch shapes for the cell kernels and the particle
// kernels, each timed over `steps` replays of the step graph
static int autotune(Batch *B, int steps, double *best_ms) {
    static const int cell_c[][2] = {{128, 512}, {128, 2048}, {256, 1024}, {256, 4096}, {64, 256}, {128, 8192}};
    static const int part_c[][2] = {{128, 128}, {128, 512}, {256, 256}, {64, 64}, {32, 32}};
    if (steps < 1) steps = 1;
    int rc = ready(B);
    if (rc) return rc;
    B->shape_fixed = true;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_cfg = [&](const Tuning &t, double *ms) -> int {
        int r = pull_state(B);
        if (r) return r;
        B->tune = t;
        if ((r = push_layout(B))) return r;
        if ((r = run_steps(B, 1))) return r;  // capture
        cudaEventRecord(e0, B->stream);
        if ((r = run_steps(B, steps))) return r;
        cudaEventRecord(e1, B->stream);
        CKB(B, cudaEventSynchronize(e1));
        float f = 0;
        cudaEventElapsedTime(&f, e0, e1);
        *ms = f / steps;
        return check_boxes(B);
    };
    Tuning best = B->tune;
    double bms = 1e30;
    for (auto &c : cell_c) {
        Tuning t = best;
        t.cell_block = c[0];
        t.cell_tile = c[1];
        double ms;
        if ((rc = time_cfg(t, &ms))) break;
        if (ms < bms) { bms = ms; best = t; }
    }
    if (!rc && B->prec != DPS_F64) {
        const int v0 = best.k1v;  // timed with the launch shapes above
        for (int v = 0; v < 8; ++v) {
            if (v == v0) continue;
            Tuning t = best;
            t.k1v = v;
            double ms;
            if ((rc = time_cfg(t, &ms))) break;
            if (ms < bms) { bms = ms; best = t; }
        }
    }
    if (!rc)
        for (auto &c : part_c) {
            Tuning t = best;
            t.part_block = c[0];
            t.part_tile = c[1];
            double ms;
            if ((rc = time_cfg(t, &ms))) break;
            if (ms < bms) { bms = ms; best = t; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = pull_state(B))) return rc;
    B->tune = best;
    B->tuned = true;
    if ((rc = push_layout(B))) return rc;
    if (best_ms) *best_ms = bms;
    return DPS_OK;
}

int dps_batch_autotune(dps_batch b, int steps, double *best_ms) { return b ? autotune(&b->B, steps, best_ms) : DPS_ERR_ARG; }
int dps_batch_set_timing(dps_batch b, int enable) { return b ? b_set_timing(&b->B, enable) : DPS_ERR_ARG; }
int dps_batch_collect_timing(dps_batch b) { return b ? b_collect_timing(&b->B) : DPS_ERR_ARG; }
int dps_batch_get_timing(dps_batch b, double ms[DPS_NPHASE], int64_t launches[DPS_NPHASE], int reset) {
    if (!b) return DPS_ERR_ARG;
    b_get_timing(&b->B, ms, launches, reset);
    return DPS_OK;
}
int dps_batch_launches_per_step(dps_batch b, int64_t *n) {
    if (!b || !n) return DPS_ERR_ARG;
    *n = b_launches_per_step(&b->B);
    return DPS_OK;
}
int dps_box_bytes(int precision, const int n[3], int64_t max_particles, size_t *bytes) {
    if (!n || !bytes || precision < DPS_F64 || precision > DPS_F16S) return DPS_ERR_ARG;
    *bytes = box_bytes(precision, (long long)n[0] * n[1] * n[2], max_particles);
    return DPS_OK;
}

// ---- stateless op -------------------------------------------------------------------------
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
    int st = 0;
    const cudaError_t ec = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(scr, s);
    if (ec != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        cudaGetLastError();
        return DPS_ERR_CUDA;
    }
    return (st & ST_BAD_CELL) ? DPS_ERR_ARG : DPS_OK;
}

}  // extern "C"
