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
#include "box.cuh"

namespace dps {

static constexpr double PI_D = 3.14159265358979323846;

// ---- Eq. filter_def, one axis ---------------------------------------------
__device__ __forceinline__ double roma_phi(double r) {
    r = fabs(r);
    if (r < 0.5) return (1.0 + sqrt(1.0 - 3.0 * r * r)) * (1.0 / 3.0);
    if (r < 1.5) {
        double s = 1.0 - r;
        return (5.0 - 3.0 * r - sqrt(1.0 - 3.0 * s * s)) * (1.0 / 6.0);
    }
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

__device__ __forceinline__ long long particle_cell(const Geom &g, double x, double y, double z, int *st) {
    int ix = containing_cell(x, g.n[0]), iy = containing_cell(y, g.n[1]), iz = containing_cell(z, g.n[2]);
    if (st && ((!g.per[0] && (x < 0.0 || x >= g.n[0])) || (!g.per[1] && (y < 0.0 || y >= g.n[1])) ||
               (!g.per[2] && (z < 0.0 || z >= g.n[2]))))
        atomicOr(st, ST_BAD_CELL);
    return cell_index(g, ix, iy, iz);
}

// ---- S1: sort ----------------------------------------------------------------
// key = containing cell of x (current position arrays given separately)
__global__ void k_sort_count(const double *__restrict__ px, const double *__restrict__ py,
                             const double *__restrict__ pz, long long stride, long long np, Geom g,
                             int *__restrict__ count, int *__restrict__ key, int *status) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        long long c = particle_cell(g, px[i * stride], py[i * stride], pz[i * stride], status);
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

// rank each particle inside its cell by id: final slot = segment start + rank
__global__ void k_sort_rank(const int *__restrict__ key, const int *__restrict__ ids, long long np,
                            const int *__restrict__ cell_start, const int *__restrict__ tmp,
                            int *__restrict__ perm) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        int k = key[i];
        int s = cell_start[k], e = cell_start[k + 1];
        int my = ids[i], r = 0;
        for (int t = s; t < e; ++t) r += ids[tmp[t]] < my;
        perm[s + r] = (int)i;
    }
}

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
        for (long long k = tl.begin + threadIdx.x; k < tl.end; k += blockDim.x) {
            const long long i = B.perm[k];
            double x[3];
#pragma unroll
            for (int f = 0; f < 9; ++f) {
                double v = xuw[f * cap + i];
                dstf[f * cap + k] = v;
                if (f < 3) x[f] = v;
            }
#pragma unroll
            for (int f = 9; f < PXS0; ++f) dstf[f * cap + k] = srcf[f * cap + i];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                dstf[(PXS0 + a) * cap + k] = x[a];
                double w[3];
                axis_weights(x[a], g.n[a], g.per[a], w);
                dstf[(PW0 + 3 * a + 0) * cap + k] = w[0];
                dstf[(PW0 + 3 * a + 1) * cap + k] = w[1];
                dstf[(PW0 + 3 * a + 2) * cap + k] = w[2];
            }
            dsti[IID * cap + k] = srci[IID * cap + i];
            dsti[ICELL * cap + k] = B.key[i];
            dsti[IKEY * cap + k] = B.key[i];
            B.xf[0][k] = make_float4((float)x[0], (float)x[1], (float)x[2], (float)srcf[PD * cap + i]);
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
    }
}

// end of an LBM step: the previous-step fluid velocity now exists
__global__ void k_end_step(BoxDev *boxes, int nboxes) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nboxes) boxes[b].have_uprev = 1;
}

// ---- 27-cell gather helpers ---------------------------------------------------
struct CellNb {
    long long c[3][3];   // neighbour linear index per axis offset (partial sums), -1 if beyond a wall
};

__device__ __forceinline__ void cell_coords_c(const Geom &g, long long c, int &ix, int &iy, int &iz) {
    long long nxy = (long long)g.n[0] * g.n[1];
    iz = (int)(c / nxy);
    long long r = c - (long long)iz * nxy;
    iy = (int)(r / g.n[0]);
    ix = (int)(r - (long long)iy * g.n[0]);
}

__device__ __forceinline__ int wrap_axis(int i, int L, int per) {
    if (i >= 0 && i < L) return i;
    if (!per) return -1;
    return i < 0 ? i + L : i - L;
}

// Gather over the particles whose kernel support covers cell c: the particles
// of the 27 cells c+o, o in {-1,0,1}^3, with weight W_p(c) =
// w_x[1-o_x] w_y[1-o_y] w_z[1-o_z].  Visit order: o_z, o_y, o_x ascending,
// then the sorted order inside a cell.
template <typename Fn>
__device__ __forceinline__ void gather27(const Geom &g, long long c, const int *__restrict__ cell_start,
                                         const double *__restrict__ pf, long long cap, Fn &&fn) {
    int ix, iy, iz;
    cell_coords_c(g, c, ix, iy, iz);
#pragma unroll 1
    for (int oz = -1; oz <= 1; ++oz) {
        int z = wrap_axis(iz + oz, g.n[2], g.per[2]);
        if (z < 0) continue;
#pragma unroll 1
        for (int oy = -1; oy <= 1; ++oy) {
            int y = wrap_axis(iy + oy, g.n[1], g.per[1]);
            if (y < 0) continue;
#pragma unroll 1
            for (int ox = -1; ox <= 1; ++ox) {
                int x = wrap_axis(ix + ox, g.n[0], g.per[0]);
                if (x < 0) continue;
                long long n = cell_index(g, x, y, z);
                int s = cell_start[n], e = cell_start[n + 1];
                for (int p = s; p < e; ++p) {
                    double W = pf[(PW0 + 0 + 1 - ox) * cap + p] * pf[(PW0 + 3 + 1 - oy) * cap + p] *
                               pf[(PW0 + 6 + 1 - oz) * cap + p];
                    fn(p, W);
                }
            }
        }
    }
}

// ---- S2: eps_f ------------------------------------------------------------------
// also clears the sort counts for the next sort (every cell visited once)
template <typename FT>
__global__ void k_eps_gather(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        const double *pf = B.pf[B.cur];
        const long long cap = B.cap;
        FT *eps = (FT *)B.eps;
        const double eps_min = B.ph.eps_min;
        unsigned nclamp = 0;
        for (long long c = tl.begin + threadIdx.x; c < tl.end; c += blockDim.x) {
            double ep = 0.0;
            gather27(g, c, B.cell_start, pf, cap, [&](int p, double W) {
                double d = pf[PD * cap + p];
                ep += W * (PI_D / 6.0 * d * d * d);
            });
            double e = 1.0 - ep;
            if (e < eps_min) {
                if (e < 0.0) atomicOr(B.status, ST_EPS_NEG);
                ++nclamp;
                e = eps_min;
            }
            eps[c] = (FT)e;
            B.count[c] = 0;
        }
        if (nclamp) atomicAdd(&B.counters[CNT_EPS_CLAMP], (unsigned long long)nclamp);
    }
}

// ---- S4: particle forces --------------------------------------------------------
// interpolation (Eq. interpolation) of ncomp planes of a field at particle p
template <typename FT, int NC>
__device__ __forceinline__ void interp(const Geom &g, const double *__restrict__ pf, long long cap, long long p,
                                       const FT *__restrict__ field, double out[NC]) {
    const long long N = g.ncell;
    double wx[3], wy[3], wz[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
        wx[o] = pf[(PW0 + o) * cap + p];
        wy[o] = pf[(PW0 + 3 + o) * cap + p];
        wz[o] = pf[(PW0 + 6 + o) * cap + p];
    }
    int bx = containing_cell(pf[PXS0 * cap + p], g.n[0]);
    int by = containing_cell(pf[(PXS0 + 1) * cap + p], g.n[1]);
    int bz = containing_cell(pf[(PXS0 + 2) * cap + p], g.n[2]);
#pragma unroll
    for (int k = 0; k < NC; ++k) out[k] = 0.0;
#pragma unroll 1
    for (int oz = 0; oz < 3; ++oz) {
        int z = wrap_axis(bz + oz - 1, g.n[2], g.per[2]);
        if (z < 0) continue;
        for (int oy = 0; oy < 3; ++oy) {
            int y = wrap_axis(by + oy - 1, g.n[1], g.per[1]);
            if (y < 0) continue;
            for (int ox = 0; ox < 3; ++ox) {
                int x = wrap_axis(bx + ox - 1, g.n[0], g.per[0]);
                if (x < 0) continue;
                long long c = cell_index(g, x, y, z);
                double W = wx[ox] * wy[oy] * wz[oz];
#pragma unroll
                for (int k = 0; k < NC; ++k) out[k] += W * (double)field[k * N + c];
            }
        }
    }
}

// K5a: added mass, F_am = C_am rho_f V (Du_f/Dt|p - du_p/dt) (Table 1);
// du_p/dt is the change of u_p over the previous subcycle.
template <typename FT>
__global__ void k_force_am(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        const Phys &ph = B.ph;
        double *pf = B.pf[B.cur];
        const long long cap = B.cap;
        const FT *DuDt = (const FT *)B.DuDt;
        const int have_usub = B.have_usub;
        for (long long p = tl.begin + threadIdx.x; p < tl.end; p += blockDim.x) {
            double Du[3];
            interp<FT, 3>(g, pf, cap, p, DuDt, Du);
            double d = pf[PD * cap + p];
            double V = PI_D / 6.0 * d * d * d;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double u = pf[(PU + a) * cap + p];
                double dudt = have_usub ? (u - pf[(PUS0 + a) * cap + p]) / ph.dt_sub : 0.0;
                pf[(PUS0 + a) * cap + p] = u;
                pf[(PFA0 + a) * cap + p] = ph.added_mass ? ph.C_am * ph.rho_f * V * (Du[a] - dudt) : 0.0;
            }
        }
    }
}

// Table 1 drag correlation (Tenneti et al.)
__device__ __forceinline__ double drag_cd(double Re, double e) {
    double e1 = 1.0 - e;
    double e13 = e1 * e1 * e1;
    double cd0 = 1.0 + 0.15 * pow(Re, 0.687);
    double A = 5.81 * e / e13 + 0.48 * cbrt(e) / (e13 * e1);
    double e3 = e * e * e;
    double B = e3 * Re * (0.95 + 0.61 * e3 / (e1 * e1));
    return e1 * (cd0 / e13 + A + B);
}

// K5b: pressure gradient, drag and gravity (Table 1, Sec. 3.1.2).  u_f at the
// 27 cells is evaluated on the fly from rho, j and the force density of this
// subcycle: u_f = (j + (eps f_b + f_pf,am)/2)/(rho eps).
template <typename FT>
__global__ void k_force_drag(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &Bx = boxes[tl.box];
        const Geom g = Bx.g;
        const Phys &ph = Bx.ph;
        const long long N = g.ncell, cap = Bx.cap;
        double *pf = Bx.pf[Bx.cur];
        const FT *rho = (const FT *)Bx.rho, *j = (const FT *)Bx.j, *eps = (const FT *)Bx.eps;
        const FT *fam = (const FT *)Bx.fam, *gradP = (const FT *)Bx.gradP;
        for (long long p = tl.begin + threadIdx.x; p < tl.end; p += blockDim.x) {
            double wx[3], wy[3], wz[3];
#pragma unroll
            for (int o = 0; o < 3; ++o) {
                wx[o] = pf[(PW0 + o) * cap + p];
                wy[o] = pf[(PW0 + 3 + o) * cap + p];
                wz[o] = pf[(PW0 + 6 + o) * cap + p];
            }
            int bx = containing_cell(pf[PXS0 * cap + p], g.n[0]);
            int by = containing_cell(pf[(PXS0 + 1) * cap + p], g.n[1]);
            int bz = containing_cell(pf[(PXS0 + 2) * cap + p], g.n[2]);
            double uf[3] = {0, 0, 0}, gp[3] = {0, 0, 0}, ef = 0.0;
#pragma unroll 1
            for (int oz = 0; oz < 3; ++oz) {
                int z = wrap_axis(bz + oz - 1, g.n[2], g.per[2]);
                if (z < 0) continue;
                for (int oy = 0; oy < 3; ++oy) {
                    int y = wrap_axis(by + oy - 1, g.n[1], g.per[1]);
                    if (y < 0) continue;
                    for (int ox = 0; ox < 3; ++ox) {
                        int x = wrap_axis(bx + ox - 1, g.n[0], g.per[0]);
                        if (x < 0) continue;
                        long long c = cell_index(g, x, y, z);
                        double W = wx[ox] * wy[oy] * wz[oz];
                        double e = (double)eps[c], r = (double)rho[c];
                        double s = 1.0 / (r * e);
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            double F = e * ph.fb[a] + (double)fam[a * N + c];
                            uf[a] += W * ((double)j[a * N + c] + 0.5 * F) * s;
                            gp[a] += W * (double)gradP[a * N + c];
                        }
                        ef += W * e;
                    }
                }
            }
            double d = pf[PD * cap + p], rp = pf[PRHO * cap + p];
            double V = PI_D / 6.0 * d * d * d;
            double ep = 1.0 - ef;
            double du[3], dun = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                du[a] = uf[a] - pf[(PU + a) * cap + p];
                dun += du[a] * du[a];
            }
            dun = sqrt(dun);
            double Re = ef * ph.rho_f * d * dun / ph.mu;
            double coef = ph.drag ? 3.0 * PI_D * d * ph.mu * (1.0 - ep) * drag_cd(Re, ep) : 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double Fd = coef * du[a];
                double Fpr = ph.pressure ? -V * gp[a] : 0.0;
                double Fg = (rp - ph.rho_f) * V * ph.g[a];  // gravity + buoyancy
                pf[(PFD0 + a) * cap + p] = Fd;
                pf[(PFH0 + a) * cap + p] = Fd + Fpr + pf[(PFA0 + a) * cap + p] + Fg;
            }
        }
    }
}

// ---- S5: reaction force density (Eq. forces_pf) -----------------------------------
// K6a: f_pf,am(c) = -sum_p W F_am
template <typename FT>
__global__ void k_reaction_am(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        const long long N = g.ncell, cap = B.cap;
        const double *pf = B.pf[B.cur];
        FT *fam = (FT *)B.fam;
        for (long long c = tl.begin + threadIdx.x; c < tl.end; c += blockDim.x) {
            double s[3] = {0, 0, 0};
            gather27(g, c, B.cell_start, pf, cap, [&](int p, double W) {
                s[0] += W * pf[PFA0 * cap + p];
                s[1] += W * pf[(PFA0 + 1) * cap + p];
                s[2] += W * pf[(PFA0 + 2) * cap + p];
            });
            fam[c] = (FT)(-s[0]);
            fam[N + c] = (FT)(-s[1]);
            fam[2 * N + c] = (FT)(-s[2]);
        }
    }
}

// K6b: acc = (first ? 0 : acc) + f_pf,am - sum_p W F_d; after the last subcycle
// the applied f_pf is the subcycle average.
template <typename FT>
__global__ void k_reaction_drag(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles, int ntiles,
                                int first, int last) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        const long long N = g.ncell, cap = B.cap;
        const double *pf = B.pf[B.cur];
        const FT *fam = (const FT *)B.fam;
        FT *acc = (FT *)B.acc, *fpf = (FT *)B.fpf;
        const double inv_nint = B.ph.dt_sub;
        for (long long c = tl.begin + threadIdx.x; c < tl.end; c += blockDim.x) {
            double s[3] = {0, 0, 0};
            gather27(g, c, B.cell_start, pf, cap, [&](int p, double W) {
                s[0] += W * pf[PFD0 * cap + p];
                s[1] += W * pf[(PFD0 + 1) * cap + p];
                s[2] += W * pf[(PFD0 + 2) * cap + p];
            });
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double k = (double)fam[a * N + c] - s[a];
                double v = first ? k : (double)acc[a * N + c] + k;
                if (last)
                    fpf[a * N + c] = (FT)(v * inv_nint);
                else
                    acc[a * N + c] = (FT)v;
            }
        }
    }
}

// ---- host launchers ------------------------------------------------------------------
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
    k_eps_gather<FT><<<grid, block, 0, s>>>(b, t, nt);
}
template <typename FT>
void launch_force_am(const BoxDev *b, const Tile *t, int nt, int grid, int block, cudaStream_t s) {
    k_force_am<FT><<<grid, block, 0, s>>>(b, t, nt);
}
template <typename FT>
void launch_force_drag(const BoxDev *b, const Tile *t, int nt, int grid, int block, cudaStream_t s) {
    k_force_drag<FT><<<grid, block, 0, s>>>(b, t, nt);
}
template <typename FT>
void launch_reaction_am(const BoxDev *b, const Tile *t, int nt, int grid, int block, cudaStream_t s) {
    k_reaction_am<FT><<<grid, block, 0, s>>>(b, t, nt);
}
template <typename FT>
void launch_reaction_drag(const BoxDev *b, const Tile *t, int nt, int first, int last, int grid, int block,
                          cudaStream_t s) {
    k_reaction_drag<FT><<<grid, block, 0, s>>>(b, t, nt, first, last);
}

#define DPS_CPL_INST(FT)                                                                                  \
    template void launch_eps<FT>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);              \
    template void launch_force_am<FT>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);         \
    template void launch_force_drag<FT>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);       \
    template void launch_reaction_am<FT>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);      \
    template void launch_reaction_drag<FT>(const BoxDev *, const Tile *, int, int, int, int, int, cudaStream_t);
DPS_CPL_INST(double)
DPS_CPL_INST(float)

}  // namespace dps
