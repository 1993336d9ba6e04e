// coupling.cu -- Euler<->Lagrange coupling of the discrete particle method.
//
//  S1 linked-cell sort: particles ordered by (containing lattice cell, id).
//     Counting sort (atomic counts, exact integer scan), scatter, then a
//     per-cell rank by id that makes the order independent of atomics.  The
//     gather that reorders the particle SoA also evaluates each particle's
//     1D kernel weights (Eq. filter_def) for the three cells per axis.
//  S2 eps_f (Eq. fluid_volume_fraction) as a gather over the 27 cells around
//     each lattice cell: no atomics, a fixed summation order.
//  S4 particle forces (Table 1): added mass; pressure gradient, drag, gravity.
//  S5 reaction force density (Eq. forces_pf) as the same 27-cell gather.
#include <vector>

#include "box.cuh"

namespace dps {

static constexpr double PI_D = 3.14159265358979323846;

// ---- Eq. filter_def, one axis ---------------------------------------------
// both branches take sqrt(1 - 3 s^2), s = r or 1 - r: one square root per
// call whichever branch a lane is in (no divergent FP64 chains in a warp)
__device__ __forceinline__ double roma_phi(double r) {
    r = fabs(r);
    const bool inner = r < 0.5;
    const double s = inner ? r : 1.0 - r;
    const double q = sqrt(1.0 - 3.0 * s * s);
    if (inner) return (1.0 + q) * (1.0 / 3.0);
    if (r < 1.5) return (5.0 - 3.0 * r - q) * (1.0 / 6.0);
    return 0.0;
}

// weights of cells i-1, i, i+1 around the containing cell i; across a wall the
// missing cell gets weight 0 and the rest is renormalised to sum 1.
__device__ __forceinline__ void axis_weights(double x, int L, int periodic, double w[3]) {
    int i = containing_cell(x, L);
    double sum = 0.0;
#pragma unroll
    for (int o = -1; o <= 1; ++o) {
        int c = i + o;
        bool ok = periodic || (c >= 0 && c < L);
        w[o + 1] = ok ? roma_phi((c + 0.5) - x) : 0.0;
        sum += w[o + 1];
    }
    if (!periodic) {
        if (sum > 0.0) {
            double inv = 1.0 / sum;
            w[0] *= inv;
            w[1] *= inv;
            w[2] *= inv;
        } else {
            w[0] = w[2] = 0.0;
            w[1] = 1.0;
        }
    }
}

// FP32 variant for the low-precision forms: the distances to the cell
// centres are taken in FP64 (positions are FP64), the kernel in FP32
__device__ __forceinline__ float roma_phi_f(float r) {
    r = fabsf(r);
    if (r < 0.5f) return (1.0f + sqrtf(1.0f - 3.0f * r * r)) * (1.0f / 3.0f);
    if (r < 1.5f) {
        const float s = 1.0f - r;
        return (5.0f - 3.0f * r - sqrtf(1.0f - 3.0f * s * s)) * (1.0f / 6.0f);
    }
    return 0.0f;
}
__device__ __forceinline__ void axis_weights_f(double x, int L, int periodic, float w[3]) {
    int i = containing_cell(x, L);
    float sum = 0.0f;
#pragma unroll
    for (int o = -1; o <= 1; ++o) {
        int c = i + o;
        bool ok = periodic || (c >= 0 && c < L);
        w[o + 1] = ok ? roma_phi_f((float)((c + 0.5) - x)) : 0.0f;
        sum += w[o + 1];
    }
    if (!periodic) {
        if (sum > 0.0f) {
            const float inv = 1.0f / sum;
            w[0] *= inv;
            w[1] *= inv;
            w[2] *= inv;
        } else {
            w[0] = w[2] = 0.0f;
            w[1] = 1.0f;
        }
    }
}

// ---- S1: sort ----------------------------------------------------------------
// key = containing cell of x (current position arrays given separately).  The
// op entry points take positions from the caller: any coordinate outside
// [0, n) (or not finite) on any axis is flagged ST_BAD_CELL; it is counted in
// the clamped edge cell, and the op reports the flag as an argument error.
__global__ void k_sort_count(const double *__restrict__ px, const double *__restrict__ py,
                             const double *__restrict__ pz, long long stride, long long np, Geom g,
                             int *__restrict__ count, int *__restrict__ key, int *status) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = px[i * stride], y = py[i * stride], z = pz[i * stride];
        if (!(x >= 0.0 && x < g.n[0] && y >= 0.0 && y < g.n[1] && z >= 0.0 && z < g.n[2])) atomicOr(status, ST_BAD_CELL);
        long long c = particle_cell(g, x, y, z, nullptr);
        key[i] = (int)c;
        atomicAdd(&count[c], 1);
    }
}

__global__ void k_sort_scatter(const int *__restrict__ key, long long np, const int *__restrict__ cell_start,
                               int *__restrict__ fill, int *__restrict__ tmp) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        int k = key[i];
        int pos = cell_start[k] + atomicAdd(&fill[k], 1);
        tmp[pos] = (int)i;
    }
}

// rank each particle inside its cell by (id, input index): final slot =
// segment start + rank; equal ids keep their input order, so every slot of
// the segment is written exactly once
__global__ void k_sort_rank(const int *__restrict__ key, const int *__restrict__ ids, long long np,
                            const int *__restrict__ cell_start, const int *__restrict__ tmp,
                            int *__restrict__ perm) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        int k = key[i];
        int s = cell_start[k], e = cell_start[k + 1];
        int my = ids[i], r = 0;
        for (int t = s; t < e; ++t) {
            const int o = tmp[t], io = ids[o];
            r += io < my || (io == my && o < i);
        }
        perm[s + r] = (int)i;
    }
}

// Particle tiles carry the lanes per particle of the particle-side coupling
// kernels in Tile::first (1, 2, 4 or 8): a box with few particles spreads
// each over several lanes, so its latency-bound work runs on more warps.  The block size is a multiple of 32 and of the
// lanes; the loop over a tile's particles has a trip count uniform over the block.
#define DPS_PARTICLE_GROUPS(tl, lanes, lane, base, p, act)                                  \
    const int lanes = (tl).first > 1 ? (tl).first : 1;                                     \
    const int lane = (int)threadIdx.x % lanes, ngrp_ = (int)blockDim.x / lanes;            \
    for (long long base = (tl).begin, p = (tl).begin + (int)threadIdx.x / lanes; base < (tl).end; \
         base += ngrp_, p += ngrp_)                                                          \
        if (const bool act = p < (tl).end; true)

// ---- S1 on the box table ----------------------------------------------------
// x/u/w of box B: planes 0..8 of the current set, or the DEM ping-pong planes
__device__ __forceinline__ const double *xuw_of(const BoxDev &B, int xsel) {
    return xsel ? B.xtmp : B.pf[B.cur];
}

__global__ void k_bsort_count(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles,
                              int xsel) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        const double *x = xuw_of(B, xsel);
        const long long cap = B.cap;
        for (long long i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            long long c = particle_cell(g, x[i], x[cap + i], x[2 * cap + i], B.status);
            B.key[i] = (int)c;
            atomicAdd(&B.count[c], 1);
        }
    }
}

__global__ void k_bsort_scatter(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        for (long long i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            int k = B.key[i];
            B.tmp[B.cell_start[k] + atomicAdd(&B.fill[k], 1)] = (int)i;
        }
    }
}

__global__ void k_bsort_rank(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const int *ids = B.pi[B.cur] + IID * B.cap;
        for (long long i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            int k = B.key[i];
            int s = B.cell_start[k], e = B.cell_start[k + 1];
            int my = ids[i], r = 0;
            for (int q = s; q < e; ++q) r += ids[B.tmp[q]] < my;
            B.perm[s + r] = (int)i;
        }
    }
}

// reorder every particle field into the other set in the sorted order;
// record the sort position and the kernel weights (Eq. filter_def) per axis
__global__ void k_bsort_gather(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles,
                               int xsel) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        const long long cap = B.cap;
        const double *srcf = B.pf[B.cur], *xuw = xuw_of(B, xsel);
        const int *srci = B.pi[B.cur];
        double *dstf = B.pf[1 - B.cur];
        int *dsti = B.pi[1 - B.cur];
        // the lanes of a particle share the plane copies and the three axes
        // of kernel weights (lane a takes axis a: one instruction stream for
        // the warp, no divergent per-axis branches); the last share (mass,
        // ints, float copies) goes to lane 3 mod lanes
        DPS_PARTICLE_GROUPS(tl, lanes, lane, base, k, act) {
            if (!act) continue;
            const int lm = lanes - 1;
            const long long i = B.perm[k];
            // all plane copies issued back to back (predicated per lane)
#pragma unroll
            for (int f = 0; f < PXS0; ++f)
                if ((f & lm) == lane) dstf[f * cap + k] = f < 9 ? xuw[f * cap + i] : srcf[f * cap + i];
            for (int a = lane; a < 3; a += lanes) {
                const double xa = xuw[a * cap + i];
                const int La = a == 0 ? g.n[0] : (a == 1 ? g.n[1] : g.n[2]);
                const int pa = a == 0 ? g.per[0] : (a == 1 ? g.per[1] : g.per[2]);
                dstf[(PXS0 + a) * cap + k] = xa;
                if (B.lowp) {
                    float w[3];
                    axis_weights_f(xa, La, pa, w);
                    B.pwf[(3 * a + 0) * cap + k] = w[0];
                    B.pwf[(3 * a + 1) * cap + k] = w[1];
                    B.pwf[(3 * a + 2) * cap + k] = w[2];
                } else {
                    double w[3];
                    axis_weights(xa, La, pa, w);
                    dstf[(PW0 + 3 * a + 0) * cap + k] = w[0];
                    dstf[(PW0 + 3 * a + 1) * cap + k] = w[1];
                    dstf[(PW0 + 3 * a + 2) * cap + k] = w[2];
                }
            }
            if ((3 & lm) != lane) continue;
            // mass and the inverse factors of Eq. particle_motion (I = m d^2 / 10)
            const double dd = srcf[PD * cap + i];
            const double m = srcf[PRHO * cap + i] * PI_D / 6.0 * dd * dd * dd;
            dstf[PM * cap + k] = m;
            dstf[PIM * cap + k] = 1.0 / m;
            dstf[PII * cap + k] = 10.0 / (m * dd * dd);
            dstf[PVOL * cap + k] = double(PI_D / 6.0) * dd * dd * dd;
            dsti[IID * cap + k] = srci[IID * cap + i];
            dsti[ICELL * cap + k] = B.key[i];
            dsti[IKEY * cap + k] = B.key[i];
            B.xf[0][k] = make_float4((float)xuw[i], (float)xuw[cap + i], (float)xuw[2 * cap + i], (float)dd);
            B.vf[0][k] = make_float4((float)xuw[3 * cap + i], (float)xuw[4 * cap + i], (float)xuw[5 * cap + i], (float)m);
            B.of[0][k] = make_float4((float)xuw[6 * cap + i], (float)xuw[7 * cap + i], (float)xuw[8 * cap + i], 0.f);
        }
    }
}

// after the gather: the other set becomes current; after a subcycle (not the
// initial sort) the particles' u at the subcycle start exists
__global__ void k_bsort_flip(BoxDev *boxes, int nboxes, int mark_usub) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nboxes) {
        boxes[b].cur ^= 1;
        if (mark_usub) boxes[b].have_usub = 1;
        *boxes[b].ptop = 0;  // pair slots of the list built next
    }
}

// end of an LBM step: the previous-step fluid velocity now exists
__global__ void k_end_step(BoxDev *boxes, int nboxes) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nboxes) boxes[b].have_uprev = 1;
}

// ---- 27-cell gather helpers ---------------------------------------------------
// cell coordinate i on an axis of L cells: wrapped on a periodic axis, -1
// beyond a wall
__device__ __forceinline__ int wrap_axis(int i, int L, int per) {
    if (i >= 0 && i < L) return i;
    if (!per) return -1;
    return i < 0 ? i + L : i - L;
}

// the kernel weights of a box in the compute type FT of its form
template <typename FT> __device__ __forceinline__ const FT *weights_of(const BoxDev &B, const double *pf);
template <> __device__ __forceinline__ const double *weights_of<double>(const BoxDev &B, const double *pf) {
    return pf + PW0 * B.cap;
}
template <> __device__ __forceinline__ const float *weights_of<float>(const BoxDev &B, const double *) { return B.pwf; }

// ---- brick-tiled gathers ---------------------------------------------------------
// A brick is a block of up to 8x8x8 cells of one box (Tile::begin and
// Tile::end pack its origin and extent, 21 bits per axis).  The block first
// stages the particle ranges of the brick's cells and their one-cell halo in
// shared memory (one cell_start pair per halo cell instead of 27 per cell),
// then every thread gathers over the 27 neighbours of its cells in a fixed
// order: o_z, o_y, o_x ascending, then the sorted order inside a cell.
constexpr int BRICK = 8;
constexpr int HALO = BRICK + 2;
constexpr int HALO3 = HALO * HALO * HALO;

__host__ __device__ inline long long brick_pack(int x, int y, int z) {
    return (long long)x | ((long long)y << 21) | ((long long)z << 42);
}
__device__ __forceinline__ void brick_unpack(long long v, int &x, int &y, int &z) {
    x = (int)(v & 0x1FFFFF);
    y = (int)((v >> 21) & 0x1FFFFF);
    z = (int)((v >> 42) & 0x1FFFFF);
}

struct BrickRanges {
    int s[HALO3], e[HALO3];
};

// gather over the 27 halo neighbours of brick cell (lx,ly,lz) with weights w
template <typename WT, typename Fn>
__device__ __forceinline__ void gather27_staged(const BrickRanges &R, int lx, int ly, int lz, const WT *__restrict__ w,
                                                long long cap, Fn &&fn) {
#pragma unroll 1
    for (int oz = -1; oz <= 1; ++oz) {
        const WT *wz = w + (6 + 1 - oz) * cap;
#pragma unroll 1
        for (int oy = -1; oy <= 1; ++oy) {
            const WT *wy = w + (3 + 1 - oy) * cap;
            const int hrow = (lz + 1 + oz) * HALO * HALO + (ly + 1 + oy) * HALO + (lx + 1);
#pragma unroll
            for (int ox = -1; ox <= 1; ++ox) {
                const int h = hrow + ox;
                const int s = R.s[h], e = R.e[h];
                const WT *wx = w + (1 - ox) * cap;
                for (int p = s; p < e; ++p) fn(p, wx[p] * wy[p] * wz[p]);
            }
        }
    }
}

// iterate the cells of the current brick tile: fn(cell index, lx, ly, lz)
template <typename Fn>
__device__ __forceinline__ void for_brick_cells(const Geom &g, int ox, int oy, int oz, int ex, int ey, int ez, Fn &&fn) {
    const int nb = ex * ey * ez;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const int lx = k % ex, ly = (k / ex) % ey, lz = k / (ex * ey);
        fn(cell_index(g, ox + lx, oy + ly, oz + lz), lx, ly, lz);
    }
}

// Compacted particle list of a brick and its halo: entry m is particle P[m]
// of halo cell with x coordinate hx[m]; the entries of halo cell h are
// [off[h], off[h+1]) in ascending h, then sorted order.  A warp gathers over
// the rows (hz, hy) of the bounding box of its cells' supports only, so with
// sparse particles it visits the few particles near it once, instead of each
// lane testing all 27 neighbour cells (a warp pays for the busiest lane of
// every neighbour cell).  The per-cell visit order is the one of
// gather27_staged: ascending h is ascending (o_z, o_y, o_x) for a fixed cell.
constexpr int BRICK_THREADS = 256;  // block size of every brick kernel
// entries; above it (about 0.13 particles per halo cell) the block takes the
// per-cell walk of gather27_staged, faster once most probes find particles
// (measured: the list wins at 0.02 particles per cell, the walk at 0.2)
constexpr int BL_MAX = 128;
constexpr int BL_PER_THREAD = (HALO3 + BRICK_THREADS - 1) / BRICK_THREADS;

struct BrickList {
    BrickRanges R;
    int off[HALO3 + 1];
    int P[BL_MAX];
    unsigned char hx[BL_MAX];
    int wsum[BRICK_THREADS / 32];
    int n;  // entries, or -1 when over BL_MAX
};

// stage the ranges and the compacted list of brick (ox,oy,oz); ends with a barrier
__device__ __forceinline__ void stage_list(const BoxDev &B, int ox, int oy, int oz, BrickList &L) {
    const Geom &g = B.g;
    int s0[BL_PER_THREAD], cnt[BL_PER_THREAD], tot = 0;
#pragma unroll
    for (int u = 0; u < BL_PER_THREAD; ++u) {
        const int h = BL_PER_THREAD * threadIdx.x + u;
        int a = 0, e = 0;
        if (h < HALO3) {
            const int hx = h % HALO, hy = (h / HALO) % HALO, hz = h / (HALO * HALO);
            const int x = wrap_axis(ox + hx - 1, g.n[0], g.per[0]);
            const int y = wrap_axis(oy + hy - 1, g.n[1], g.per[1]);
            const int z = wrap_axis(oz + hz - 1, g.n[2], g.per[2]);
            if (x >= 0 && y >= 0 && z >= 0) {
                const long long n = cell_index(g, x, y, z);
                a = B.cell_start[n];
                e = B.cell_start[n + 1];
            }
            L.R.s[h] = a;
            L.R.e[h] = e;
        }
        s0[u] = a;
        cnt[u] = e - a;
        tot += e - a;
    }
    // block-wide exclusive prefix of the per-thread totals
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) L.wsum[wid] = incl;
    __syncthreads();
    int base = 0, total = 0;
#pragma unroll
    for (int q = 0; q < BRICK_THREADS / 32; ++q) {
        base += q < wid ? L.wsum[q] : 0;
        total += L.wsum[q];
    }
    int run = base + incl - tot;
    const bool fits = total <= BL_MAX;
#pragma unroll
    for (int u = 0; u < BL_PER_THREAD; ++u) {
        const int h = BL_PER_THREAD * threadIdx.x + u;
        if (h < HALO3) {
            L.off[h] = run;
            if (fits)
                for (int m = 0; m < cnt[u]; ++m) {
                    L.P[run + m] = s0[u] + m;
                    L.hx[run + m] = (unsigned char)(h % HALO);
                }
        }
        run += cnt[u];
    }
    if (threadIdx.x == 0) {
        L.off[HALO3] = total;
        L.n = fits ? total : -1;
    }
    __syncthreads();
}

// for every cell c of the brick: St st{}; acc(st, p, W_p(c)) over the
// particles of its support in the order of gather27_staged; fin(st, c)
template <typename St, typename WT, typename Acc, typename Fin>
__device__ __forceinline__ void brick_gather(const Geom &g, const BrickList &L, int ox, int oy, int oz, int ex, int ey,
                                             int ez, const WT *__restrict__ w, long long cap, Acc &&acc, Fin &&fin) {
    if (L.n < 0) {
        for_brick_cells(g, ox, oy, oz, ex, ey, ez, [&](long long c, int lx, int ly, int lz) {
            St st{};
            gather27_staged(L.R, lx, ly, lz, w, cap, [&](int p, WT W) { acc(st, p, W); });
            fin(st, c);
        });
        return;
    }
    const int nb = ex * ey * ez;
    for (int k0 = 0; k0 < nb; k0 += blockDim.x) {  // trip count uniform over the block
        const int k = k0 + threadIdx.x;
        const bool act = k < nb;
        int lx = 0, ly = 0, lz = 0;
        if (act) {
            lx = k % ex;
            ly = (k / ex) % ey;
            lz = k / (ex * ey);
        }
        if (!__any_sync(0xffffffffu, act)) continue;
        // halo bounding box of the warp's supports: [min l, max l + 2] per axis
        const int BIG = 1 << 20;
        const int bx0 = __reduce_min_sync(0xffffffffu, act ? lx : BIG);
        const int by0 = __reduce_min_sync(0xffffffffu, act ? ly : BIG);
        const int bz0 = __reduce_min_sync(0xffffffffu, act ? lz : BIG);
        const int bx1 = __reduce_max_sync(0xffffffffu, act ? lx : -BIG) + 2;
        const int by1 = __reduce_max_sync(0xffffffffu, act ? ly : -BIG) + 2;
        const int bz1 = __reduce_max_sync(0xffffffffu, act ? lz : -BIG) + 2;
        St st{};
        for (int hz = bz0; hz <= bz1; ++hz) {
            const int dz = hz - (lz + 1);
            for (int hy = by0; hy <= by1; ++hy) {
                const int dy = hy - (ly + 1);
                const int hrow = (hz * HALO + hy) * HALO;
                const int m0 = L.off[hrow + bx0], m1 = L.off[hrow + bx1 + 1];
                if (!act || dz < -1 || dz > 1 || dy < -1 || dy > 1) continue;
                const WT *wz = w + (6 + 1 - dz) * cap, *wy = w + (3 + 1 - dy) * cap;
                for (int m = m0; m < m1; ++m) {
                    const int dx = (int)L.hx[m] - (lx + 1);
                    if (dx < -1 || dx > 1) continue;
                    const int p = L.P[m];
                    const WT *wx = w + (1 - dx) * cap;
                    acc(st, p, wx[p] * wy[p] * wz[p]);
                }
            }
        }
        if (act) fin(st, cell_index(g, ox + lx, oy + ly, oz + lz));
    }
}

// ---- S2: eps_f ------------------------------------------------------------------
// FT is the compute type of the form: FP64 for the plain method, FP32 (with
// FP32 kernel weights) for the low-precision forms.  Also clears the sort
// counts for the next sort (every cell is visited once).
template <typename FT>
__global__ void __launch_bounds__(BRICK_THREADS) k_eps_gather(const BoxDev *__restrict__ boxes,
                                                              const Tile *__restrict__ tiles, int ntiles) {
    __shared__ BrickList L;
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        int ox, oy, oz, ex, ey, ez;
        brick_unpack(tl.begin, ox, oy, oz);
        brick_unpack(tl.end, ex, ey, ez);
        __syncthreads();  // the previous brick is done with L
        stage_list(B, ox, oy, oz, L);
        const double *pf = B.pf[B.cur];
        const long long cap = B.cap;
        const FT *w = weights_of<FT>(B, pf);
        const float4 *xf = B.xf[0];
        FT *eps = (FT *)B.eps;
        const FT eps_min = (FT)B.ph.eps_min;
        unsigned nclamp = 0;
        struct St {
            FT ep;
        };
        brick_gather<St>(
            g, L, ox, oy, oz, ex, ey, ez, w, cap,
            [&](St &st, int p, FT W) {
                if (sizeof(FT) == 8) {
                    st.ep += W * (FT)pf[PVOL * cap + p];  // the volume stored at the sort
                } else {
                    const FT d = (FT)xf[p].w;
                    st.ep += W * (FT(PI_D / 6.0) * d * d * d);
                }
            },
            [&](St &st, long long c) {
                FT e = FT(1) - st.ep;
                if (e < eps_min) {
                    if (e < FT(0)) atomicOr(B.status, ST_EPS_NEG);
                    ++nclamp;
                    e = eps_min;
                }
                eps[c] = e;
                B.count[c] = 0;
            });
        if (nclamp) atomicAdd(&B.counters[CNT_EPS_CLAMP], (unsigned long long)nclamp);
    }
}

// ---- S4: particle forces --------------------------------------------------------
// the 27-cell support of particle p: weights and the base cell of the sort
template <typename FT>
struct Support {
    FT wx[3], wy[3], wz[3];
    int b[3];
};

template <typename FT>
__device__ __forceinline__ Support<FT> support_of(const BoxDev &B, const double *pf, long long p) {
    const long long cap = B.cap;
    const FT *w = weights_of<FT>(B, pf);
    Support<FT> S;
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        S.wx[o] = w[o * cap + p];
        S.wy[o] = w[(3 + o) * cap + p];
        S.wz[o] = w[(6 + o) * cap + p];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) S.b[a] = containing_cell(pf[(PXS0 + a) * cap + p], B.g.n[a]);
    return S;
}

// the cells s = lane, lane + lanes, ... (s < 27, s = 9 o_z + 3 o_y + o_x) of
// the support (Eq. interpolation); with one lane in (o_z, o_y, o_x) order
template <typename FT, typename Fn>
__device__ __forceinline__ void for_support_lanes(const Geom &g, const Support<FT> &S, int lane, int lanes, Fn &&fn) {
#pragma unroll 1
    for (int s = lane; s < 27; s += lanes) {
        const int oz = s / 9, oy = (s / 3) % 3, ox = s % 3;
        const int z = wrap_axis(S.b[2] + oz - 1, g.n[2], g.per[2]);
        const int y = wrap_axis(S.b[1] + oy - 1, g.n[1], g.per[1]);
        const int x = wrap_axis(S.b[0] + ox - 1, g.n[0], g.per[0]);
        if (x < 0 || y < 0 || z < 0) continue;
        // selects keep the weights in registers (no indexed local array)
        const FT wx = ox == 0 ? S.wx[0] : (ox == 1 ? S.wx[1] : S.wx[2]);
        const FT wy = oy == 0 ? S.wy[0] : (oy == 1 ? S.wy[1] : S.wy[2]);
        const FT wz = oz == 0 ? S.wz[0] : (oz == 1 ? S.wz[1] : S.wz[2]);
        fn(cell_index(g, x, y, z), wx * wy * wz);
    }
}

// sum over the lanes of a particle's lane group (xor tree: every lane of the
// group ends with the same bits); all 32 lanes of the warp take part
template <typename FT, int NV>
__device__ __forceinline__ void lanes_sum(FT (&v)[NV], int lanes) {
    for (int o = lanes >> 1; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}


// K5a: added mass, F_am = C_am rho_f V (Du_f/Dt|p - du_p/dt) (Table 1);
// du_p/dt is the change of u_p over the previous subcycle (taken in FP64).
// With lift, the shear lift F_l = 1.61 d^2 sqrt(mu rho_f / |w|) (u_f - u_p) x w
// (Table 1; zero where w vanishes) is added to F_am and distributed with it:
// u_f = (j + eps_f f_b/2)/(rho eps_f) at the subcycle start and its curl w
// (written by k_curl) are interpolated at the particle.
template <typename FT>
__global__ void k_force_am(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        const long long N = g.ncell;
        const Phys &ph = B.ph;
        double *pf = B.pf[B.cur];
        const long long cap = B.cap;
        const FT *DuDt = (const FT *)B.DuDt;
        const int have_usub = B.have_usub;
        const int lift = ph.lift;
        const FT *rho = (const FT *)B.rho, *j = (const FT *)B.j, *eps = (const FT *)B.eps;
        const FT *curl = (const FT *)B.curl;
        const FT hb[3] = {FT(0.5) * (FT)ph.fb[0], FT(0.5) * (FT)ph.fb[1], FT(0.5) * (FT)ph.fb[2]};
        DPS_PARTICLE_GROUPS(tl, lanes, lane, base, p, act) {
            // v: Du_f/Dt at the particle, then (lift) u_f and the vorticity w
            FT v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            Support<FT> S;
            if (act) {
                S = support_of<FT>(B, pf, p);
                if (lift)
                    for_support_lanes(g, S, lane, lanes, [&](long long c, FT W) {
                        v[0] += W * DuDt[c];
                        v[1] += W * DuDt[N + c];
                        v[2] += W * DuDt[2 * N + c];
                        const FT e = eps[c];
                        const FT sc = W / (rho[c] * e);
                        v[3] += (j[c] + e * hb[0]) * sc;
                        v[4] += (j[N + c] + e * hb[1]) * sc;
                        v[5] += (j[2 * N + c] + e * hb[2]) * sc;
                        v[6] += W * curl[c];
                        v[7] += W * curl[N + c];
                        v[8] += W * curl[2 * N + c];
                    });
                else
                    for_support_lanes(g, S, lane, lanes, [&](long long c, FT W) {
                        v[0] += W * DuDt[c];
                        v[1] += W * DuDt[N + c];
                        v[2] += W * DuDt[2 * N + c];
                    });
            }
            if (lanes > 1) {
                if (lift)
                    lanes_sum(v, lanes);
                else {
                    FT u3[3] = {v[0], v[1], v[2]};
                    lanes_sum(u3, lanes);
                    v[0] = u3[0];
                    v[1] = u3[1];
                    v[2] = u3[2];
                }
            }
            if (!act || lane != 0) continue;
            const FT Du[3] = {v[0], v[1], v[2]};
            FT Fl[3] = {0, 0, 0};
            if (lift) {
                const FT uf[3] = {v[3], v[4], v[5]}, w[3] = {v[6], v[7], v[8]};
                const FT wn = m_sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                if (wn > FT(0)) {
                    const double dp = pf[PD * cap + p];
                    const FT du[3] = {uf[0] - (FT)pf[PU * cap + p], uf[1] - (FT)pf[PV * cap + p],
                                      uf[2] - (FT)pf[PW * cap + p]};
                    const FT k = FT(1.61 * dp * dp) * m_sqrt((FT)(ph.mu * ph.rho_f) / wn);
                    Fl[0] = k * (du[1] * w[2] - du[2] * w[1]);
                    Fl[1] = k * (du[2] * w[0] - du[0] * w[2]);
                    Fl[2] = k * (du[0] * w[1] - du[1] * w[0]);
                }
            }
            const double d = pf[PD * cap + p];
            const FT cV = (FT)(ph.C_am * ph.rho_f * PI_D / 6.0 * d * d * d);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double u = pf[(PU + a) * cap + p];
                const double dudt = have_usub ? (u - pf[(PUS0 + a) * cap + p]) / ph.dt_sub : 0.0;
                pf[(PUS0 + a) * cap + p] = u;
                const FT Fa = (ph.added_mass ? cV * (Du[a] - (FT)dudt) : FT(0)) + Fl[a];
                pf[(PFA0 + a) * cap + p] = (double)Fa;
                if (sizeof(FT) == 4) B.f32p[a * cap + p] = (float)Fa;
            }
        }
    }
}

// Table 1 drag correlation (Tenneti et al.).  In FP64 each dependent
// instruction costs GB300 tens of cycles, so the chain is kept short:
// Re^0.687 as exp(0.687 ln Re) (Re > 0; relative error a few 1e-16, far below
// the FP64 parity tolerance), and one division, 1/(1 - eps_p), for the four
// quotients.
__device__ __forceinline__ double drag_cd(double Re, double e) {
    const double e1 = 1.0 - e;
    const double i1 = 1.0 / e1;
    const double i3 = i1 * i1 * i1;
    const double cd0 = 1.0 + 0.15 * (Re > 0.0 ? exp(0.687 * log(Re)) : 0.0);
    const double A = 5.81 * e * i3 + 0.48 * cbrt(e) * (i3 * i1);
    const double e3 = e * e * e;
    const double B = e3 * Re * (0.95 + 0.61 * e3 * (i1 * i1));
    return e1 * (cd0 * i3 + A + B);
}
__device__ __forceinline__ float drag_cd(float Re, float e) {
    float e1 = 1.0f - e;
    float e13 = e1 * e1 * e1;
    float cd0 = 1.0f + 0.15f * powf(Re, 0.687f);
    float A = 5.81f * e / e13 + 0.48f * cbrtf(e) / (e13 * e1);
    float e3 = e * e * e;
    float B = e3 * Re * (0.95f + 0.61f * e3 / (e1 * e1));
    return e1 * (cd0 / e13 + A + B);
}

// K5b: pressure gradient, drag and gravity (Table 1, Sec. 3.1.2).  u_f at the
// 27 cells is evaluated on the fly from rho, j and the force density of this
// subcycle: u_f = (j + (eps f_b + f_pf,am)/2)/(rho eps).
// first: the first subcycle of the step, whose eps_f is the one the moments
// pass divided by: 1/(rho eps_f) is read from it instead of divided again
// (the same rounded value)
template <typename FT>
__global__ void k_force_drag(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles,
                             int first) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &Bx = boxes[tl.box];
        const Geom g = Bx.g;
        const Phys &ph = Bx.ph;
        const long long N = g.ncell, cap = Bx.cap;
        double *pf = Bx.pf[Bx.cur];
        const FT *rho = (const FT *)Bx.rho, *j = (const FT *)Bx.j, *eps = (const FT *)Bx.eps;
        const FT *fam = (const FT *)Bx.fam, *gradP = (const FT *)Bx.gradP, *ire = (const FT *)Bx.ire;
        const FT fb[3] = {(FT)ph.fb[0], (FT)ph.fb[1], (FT)ph.fb[2]};
        DPS_PARTICLE_GROUPS(tl, lanes, lane, base, p, act) {
            // v: u_f (3), grad P (3), eps_f at the particle
            FT v[7] = {0, 0, 0, 0, 0, 0, 0};
            if (act) {
                const Support<FT> S = support_of<FT>(Bx, pf, p);
                for_support_lanes(g, S, lane, lanes, [&](long long c, FT W) {
                    const FT e = eps[c];
                    const FT s = first ? ire[c] : FT(1) / (rho[c] * e);
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const FT F = e * fb[a] + fam[a * N + c];
                        v[a] += W * (j[a * N + c] + FT(0.5) * F) * s;
                        v[3 + a] += W * gradP[a * N + c];
                    }
                    v[6] += W * e;
                });
            }
            if (lanes > 1) lanes_sum(v, lanes);
            if (!act || lane != 0) continue;
            const FT ef = v[6];
            const double d = pf[PD * cap + p], rp = pf[PRHO * cap + p];
            const double V = PI_D / 6.0 * d * d * d;
            const FT ep = FT(1) - ef;
            FT du[3], dun = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                du[a] = v[a] - (FT)pf[(PU + a) * cap + p];
                dun += du[a] * du[a];
            }
            dun = m_sqrt(dun);
            const FT mu = (FT)ph.mu, dd = (FT)d;
            const FT Re = ef * (FT)ph.rho_f * dd * dun / mu;
            const FT coef = ph.drag ? FT(3.0 * PI_D) * dd * mu * (FT(1) - ep) * drag_cd(Re, ep) : FT(0);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const FT Fd = coef * du[a];
                const FT Fpr = ph.pressure ? -(FT)V * v[3 + a] : FT(0);
                const double Fg = (rp - ph.rho_f) * V * ph.g[a];  // gravity + buoyancy
                pf[(PFD0 + a) * cap + p] = (double)Fd;
                if (sizeof(FT) == 4) Bx.f32p[(3 + a) * cap + p] = (float)Fd;
                pf[(PFH0 + a) * cap + p] = (double)Fd + (double)Fpr + pf[(PFA0 + a) * cap + p] + Fg;
            }
        }
    }
}

// ---- S5: reaction force density (Eq. forces_pf) -----------------------------------
// particle force planes in the compute type: FP64 planes of the particle SoA,
// or their FP32 copies in the low-precision forms
template <typename FT> __device__ __forceinline__ const FT *force_planes(const BoxDev &B, const double *pf, int which);
template <> __device__ __forceinline__ const double *force_planes<double>(const BoxDev &B, const double *pf, int which) {
    return pf + (which ? PFD0 : PFA0) * B.cap;
}
template <> __device__ __forceinline__ const float *force_planes<float>(const BoxDev &B, const double *, int which) {
    return B.f32p + (which ? 3 : 0) * B.cap;
}

// K6a: f_pf,am(c) = -sum_p W F_am
template <typename FT>
__global__ void __launch_bounds__(BRICK_THREADS) k_reaction_am(const BoxDev *__restrict__ boxes,
                                                               const Tile *__restrict__ tiles, int ntiles) {
    __shared__ BrickList L;
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        int ox, oy, oz, ex, ey, ez;
        brick_unpack(tl.begin, ox, oy, oz);
        brick_unpack(tl.end, ex, ey, ez);
        __syncthreads();
        stage_list(B, ox, oy, oz, L);
        const long long N = g.ncell, cap = B.cap;
        const double *pf = B.pf[B.cur];
        const FT *w = weights_of<FT>(B, pf), *Fa = force_planes<FT>(B, pf, 0);
        FT *fam = (FT *)B.fam;
        struct St {
            FT s0, s1, s2;
        };
        brick_gather<St>(
            g, L, ox, oy, oz, ex, ey, ez, w, cap,
            [&](St &st, int p, FT W) {
                st.s0 += W * Fa[p];
                st.s1 += W * Fa[cap + p];
                st.s2 += W * Fa[2 * cap + p];
            },
            [&](St &st, long long c) {
                fam[c] = -st.s0;
                fam[N + c] = -st.s1;
                fam[2 * N + c] = -st.s2;
            });
    }
}

// K6b: acc = (first ? 0 : acc) + f_pf,am - sum_p W F_d; after the last subcycle
// the applied f_pf is the subcycle average.
template <typename FT>
__global__ void __launch_bounds__(BRICK_THREADS) k_reaction_drag(const BoxDev *__restrict__ boxes,
                                                                 const Tile *__restrict__ tiles, int ntiles, int first,
                                                                 int last) {
    __shared__ BrickList L;
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        int ox, oy, oz, ex, ey, ez;
        brick_unpack(tl.begin, ox, oy, oz);
        brick_unpack(tl.end, ex, ey, ez);
        __syncthreads();
        stage_list(B, ox, oy, oz, L);
        const long long N = g.ncell, cap = B.cap;
        const double *pf = B.pf[B.cur];
        const FT *w = weights_of<FT>(B, pf), *Fd = force_planes<FT>(B, pf, 1);
        const FT *fam = (const FT *)B.fam;
        FT *acc = (FT *)B.acc, *fpf = (FT *)B.fpf;
        const FT inv_nint = (FT)B.ph.dt_sub;
        struct St {
            FT s[3];
        };
        brick_gather<St>(
            g, L, ox, oy, oz, ex, ey, ez, w, cap,
            [&](St &st, int p, FT W) {
                st.s[0] += W * Fd[p];
                st.s[1] += W * Fd[cap + p];
                st.s[2] += W * Fd[2 * cap + p];
            },
            [&](St &st, long long c) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const FT k = fam[a * N + c] - st.s[a];
                    const FT v = first ? k : acc[a * N + c] + k;
                    if (last)
                        fpf[a * N + c] = v * inv_nint;
                    else
                        acc[a * N + c] = v;
                }
            });
    }
}

// ---- host launchers ------------------------------------------------------------------
// brick tiles of one box (appended to `out`)
void brick_tiles(int box, const int n[3], std::vector<Tile> &out) {
    for (int z = 0; z < n[2]; z += BRICK)
        for (int y = 0; y < n[1]; y += BRICK)
            for (int x = 0; x < n[0]; x += BRICK) {
                const int ex = n[0] - x < BRICK ? n[0] - x : BRICK;
                const int ey = n[1] - y < BRICK ? n[1] - y : BRICK;
                const int ez = n[2] - z < BRICK ? n[2] - z : BRICK;
                out.push_back(Tile{box, 0, brick_pack(x, y, z), brick_pack(ex, ey, ez)});
            }
}

static int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

// stateless sort op (device buffers): x of particle i at px[i*stride]...
void launch_sort_count(const double *px, const double *py, const double *pz, long long stride, long long np,
                       const Geom &g, int *count, int *key, int *status, cudaStream_t s) {
    if (np <= 0) return;
    k_sort_count<<<grid_for(np, 256), 256, 0, s>>>(px, py, pz, stride, np, g, count, key, status);
}
void launch_sort_scatter(const int *key, long long np, const int *cell_start, int *fill, int *tmp,
                         cudaStream_t s) {
    if (np <= 0) return;
    k_sort_scatter<<<grid_for(np, 256), 256, 0, s>>>(key, np, cell_start, fill, tmp);
}
void launch_sort_rank(const int *key, const int *ids, long long np, const int *cell_start, const int *tmp,
                      int *perm, cudaStream_t s) {
    if (np <= 0) return;
    k_sort_rank<<<grid_for(np, 256), 256, 0, s>>>(key, ids, np, cell_start, tmp, perm);
}

// box-table launchers: (grid, block) chosen by the caller
void launch_bsort_count(const BoxDev *b, const Tile *t, int nt, int xsel, int grid, int block, cudaStream_t s) {
    k_bsort_count<<<grid, block, 0, s>>>(b, t, nt, xsel);
}
void launch_bsort_scatter(const BoxDev *b, const Tile *t, int nt, int grid, int block, cudaStream_t s) {
    k_bsort_scatter<<<grid, block, 0, s>>>(b, t, nt);
}
void launch_bsort_rank(const BoxDev *b, const Tile *t, int nt, int grid, int block, cudaStream_t s) {
    k_bsort_rank<<<grid, block, 0, s>>>(b, t, nt);
}
void launch_bsort_gather(const BoxDev *b, const Tile *t, int nt, int xsel, int grid, int block, cudaStream_t s) {
    k_bsort_gather<<<grid, block, 0, s>>>(b, t, nt, xsel);
}
void launch_bsort_flip(BoxDev *b, int nb, int mark_usub, cudaStream_t s) {
    k_bsort_flip<<<(nb + 127) / 128, 128, 0, s>>>(b, nb, mark_usub);
}
void launch_end_step(BoxDev *b, int nb, cudaStream_t s) { k_end_step<<<(nb + 127) / 128, 128, 0, s>>>(b, nb); }

template <typename FT>
void launch_eps(const BoxDev *b, const Tile *t, int nt, int grid, int block, cudaStream_t s) {
    k_eps_gather<FT><<<grid, BRICK_THREADS, 0, s>>>(b, t, nt);
}
template <typename FT>
void launch_force_am(const BoxDev *b, const Tile *t, int nt, int grid, int block, cudaStream_t s) {
    k_force_am<FT><<<grid, block, 0, s>>>(b, t, nt);
}
template <typename FT>
void launch_force_drag(const BoxDev *b, const Tile *t, int nt, int first, int grid, int block, cudaStream_t s) {
    k_force_drag<FT><<<grid, block, 0, s>>>(b, t, nt, first);
}
template <typename FT>
void launch_reaction_am(const BoxDev *b, const Tile *t, int nt, int grid, int block, cudaStream_t s) {
    k_reaction_am<FT><<<grid, BRICK_THREADS, 0, s>>>(b, t, nt);
}
template <typename FT>
void launch_reaction_drag(const BoxDev *b, const Tile *t, int nt, int first, int last, int grid, int block,
                          cudaStream_t s) {
    k_reaction_drag<FT><<<grid, BRICK_THREADS, 0, s>>>(b, t, nt, first, last);
}

#define DPS_CPL_INST(FT)                                                                                  \
    template void launch_eps<FT>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);              \
    template void launch_force_am<FT>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);         \
    template void launch_force_drag<FT>(const BoxDev *, const Tile *, int, int, int, int, cudaStream_t);  \
    template void launch_reaction_am<FT>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);      \
    template void launch_reaction_drag<FT>(const BoxDev *, const Tile *, int, int, int, int, int, cudaStream_t);
DPS_CPL_INST(double)
DPS_CPL_INST(float)

}  // namespace dps
