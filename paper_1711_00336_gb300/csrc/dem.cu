// dem.cu -- S6: one DEM substep of Algorithm 1 for all particles.
//
// Per particle (cell-sorted order): contact (Sec. 3.1.1, linear spring-dashpot
// with Coulomb-capped viscous friction), lubrication (Sec. 3.1.3, Ball &
// Melrose) against neighbours and walls, then the explicit update of Eq.
// particle_motion with the frozen F_fp + F_g.  Neighbours are found through the
// linked cells of the last sort: every particle whose containing cell (at sort
// time) lies within +-R cells per axis, one contiguous slice of the sorted
// arrays per lattice row.  R exceeds the interaction range by the skin, and the
// kernel flags a particle that moved more than skin/2 since the sort.
// Positions/velocities are read from one buffer and written to the other
// (ping-pong), so all pair forces see the state at the start of the substep.
#include "box.cuh"

namespace dps {

static constexpr double PI_D = 3.14159265358979323846;

__device__ __forceinline__ double min_image(double dx, int L, int per) {
    return per ? dx - L * rint(dx / L) : dx;
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// force and torque on i from one partner (sphere or wall), as in Sec. 3.1.1 /
// 3.1.3; the torque uses (d_i/2) n x F_t (r x F at the contact point r = d_i/2 n).
__device__ __forceinline__ void partner(const Phys &ph, const double n[3], double dist, double sumr,
                                        const double ui[3], const double wi[3], double di, const double uj[3],
                                        const double wjh[3], double m_ij, double dmean, double F[3], double T[3],
                                        unsigned &nlim) {
    const double delta = sumr - dist;
    if (ph.contact && delta > 0.0) {
        const double le = log(ph.e_n);
        const double k_n = m_ij * (PI_D * PI_D + le * le) / (ph.T_c * ph.T_c);
        const double xi = -2.0 * le * sqrt(m_ij * k_n) / sqrt(PI_D * PI_D + le * le);
        double ws[3], wx[3], ur[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) ws[a] = 0.5 * di * wi[a] + wjh[a];
        cross3(ws, n, wx);
#pragma unroll
        for (int a = 0; a < 3; ++a) ur[a] = ui[a] - uj[a] + wx[a];
        const double urn = ur[0] * n[0] + ur[1] * n[1] + ur[2] * n[2];
        double ut[3], Fn[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ut[a] = ur[a] - urn * n[a];
            Fn[a] = -k_n * delta * n[a] - xi * (urn * n[a]);
        }
        const double Fn_abs = sqrt(Fn[0] * Fn[0] + Fn[1] * Fn[1] + Fn[2] * Fn[2]);
        const double ut_abs = sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
        double Ft[3] = {0.0, 0.0, 0.0};
        if (ut_abs > 0.0) {
            const double mag = fmin(ph.mu_c * Fn_abs, xi * ut_abs);
#pragma unroll
            for (int a = 0; a < 3; ++a) Ft[a] = -mag * ut[a] / ut_abs;
        }
        double nF[3];
        cross3(n, Ft, nF);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            F[a] += Fn[a] + Ft[a];
            T[a] += 0.5 * di * nF[a];
        }
    }
    const double h = dist - sumr;
    if (ph.lubrication && h < ph.h_c) {
        const double hh = fmax(h, ph.h_min);
        const double L = log(dmean / (2.0 * hh));
        double a_sq = 1.5 * PI_D * ph.mu * dmean * (dmean / (4.0 * hh) + 18.0 / 40.0 * L + 9.0 / 84.0 * (hh / dmean) * L);
        const double a_sh0 = 0.5 * PI_D * ph.mu * dmean * L * (dmean + hh) * (dmean + hh) / 4.0;
        const double s = 2.0 / (hh + dmean);
        double a_sh = a_sh0 * s * s;
        a_sq = fmax(a_sq, 0.0);
        a_sh = fmax(a_sh, 0.0);
        if (ph.lub_limiter) {
            const double cap = ph.lub_cap * m_ij / ph.dt_dem;
            if (a_sq > cap) { a_sq = cap; ++nlim; }
            if (a_sh > cap) { a_sh = cap; ++nlim; }
        }
        double upr[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) upr[a] = ui[a] - uj[a];
        const double upn = upr[0] * n[0] + upr[1] * n[1] + upr[2] * n[2];
#pragma unroll
        for (int a = 0; a < 3; ++a) F[a] += -a_sq * upn * n[a] - a_sh * (upr[a] - upn * n[a]);
    }
}

// src_tmp = 0: read x/u/w from the current set, write the ping-pong planes;
// src_tmp = 1: the other way round
__global__ void __launch_bounds__(256) k_dem_substep(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles,
                                                     int ntiles, int src_tmp) {
  DPS_FOR_TILES(tiles, ntiles, t) {
    const Tile tl = tiles[t];
    const BoxDev &Bx = boxes[tl.box];
    struct {
        const double *xin;
        double *xout;
        const double *pf;
        const int *cell_start;
        int R;
        int *status;
        unsigned long long *counters;
    } A{src_tmp ? Bx.xtmp : Bx.pf[Bx.cur], src_tmp ? Bx.pf[Bx.cur] : Bx.xtmp, Bx.pf[Bx.cur], Bx.cell_start,
        Bx.R, Bx.status, Bx.counters};
    const long long cap = Bx.cap;
    const Geom g = Bx.g;
    const Phys &ph = Bx.ph;
    const double rng_extra = ph.lubrication ? fmax(ph.h_c, 0.0) : 0.0;
    for (long long i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
        double xi[3], ui[3], wi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xi[a] = A.xin[a * cap + i];
            ui[a] = A.xin[(3 + a) * cap + i];
            wi[a] = A.xin[(6 + a) * cap + i];
        }
        const double di = A.pf[PD * cap + i];
        const double mi = A.pf[PRHO * cap + i] * PI_D / 6.0 * di * di * di;
        double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
        unsigned nlim = 0;
        // containing cell at sort time
        int b[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) b[a] = containing_cell(A.pf[(PXS0 + a) * cap + i], g.n[a]);
        // z and y ranges: each row visited once
        int lo[3], hi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (g.per[a] && 2 * A.R + 1 >= g.n[a]) {
                lo[a] = 0;
                hi[a] = g.n[a] - 1;
            } else if (g.per[a]) {
                lo[a] = b[a] - A.R;
                hi[a] = b[a] + A.R;
            } else {
                lo[a] = max(b[a] - A.R, 0);
                hi[a] = min(b[a] + A.R, g.n[a] - 1);
            }
        }
        for (int zz = lo[2]; zz <= hi[2]; ++zz) {
            const int z = zz < 0 ? zz + g.n[2] : (zz >= g.n[2] ? zz - g.n[2] : zz);
            for (int yy = lo[1]; yy <= hi[1]; ++yy) {
                const int y = yy < 0 ? yy + g.n[1] : (yy >= g.n[1] ? yy - g.n[1] : yy);
                const long long row = cell_index(g, 0, y, z);
                // x slice(s) of this row
                int xs0[2], xs1[2], nseg = 0;
                if (lo[0] >= 0 && hi[0] <= g.n[0] - 1) {
                    xs0[0] = lo[0]; xs1[0] = hi[0]; nseg = 1;
                } else if (lo[0] < 0) {
                    xs0[0] = 0; xs1[0] = hi[0];
                    xs0[1] = lo[0] + g.n[0]; xs1[1] = g.n[0] - 1; nseg = 2;
                } else {
                    xs0[0] = lo[0]; xs1[0] = g.n[0] - 1;
                    xs0[1] = 0; xs1[1] = hi[0] - g.n[0]; nseg = 2;
                }
                for (int sgi = 0; sgi < nseg; ++sgi) {
                    const int s = A.cell_start[row + xs0[sgi]], e = A.cell_start[row + xs1[sgi] + 1];
                    for (int j = s; j < e; ++j) {
                        if (j == i) continue;
                        double dx[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) dx[a] = min_image(A.xin[a * cap + j] - xi[a], g.n[a], g.per[a]);
                        const double dist2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
                        const double dj = A.pf[PD * cap + j];
                        const double range = 0.5 * (di + dj) + rng_extra;
                        // loose pre-filter; the exact test is on the distance itself
                        if (!(dist2 < range * range * (1.0 + 1e-12))) continue;
                        const double dist = sqrt(dist2);
                        if (!(dist < range) || dist == 0.0) continue;
                        const double n[3] = {dx[0] / dist, dx[1] / dist, dx[2] / dist};
                        const double mj = A.pf[PRHO * cap + j] * PI_D / 6.0 * dj * dj * dj;
                        const double m_ij = mi * mj / (mi + mj);
                        const double dmean = 2.0 * di * dj / (di + dj);
                        double uj[3], wjh[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            uj[a] = A.xin[(3 + a) * cap + j];
                            wjh[a] = 0.5 * dj * A.xin[(6 + a) * cap + j];
                        }
                        partner(ph, n, dist, 0.5 * (di + dj), ui, wi, di, uj, wjh, m_ij, dmean, F, T, nlim);
                    }
                }
            }
        }
        // walls: the faces of every non-periodic axis (m_ij = m_i, <d> = 2 d_i)
        const double zero[3] = {0, 0, 0};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (g.per[a]) continue;
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const double dist = side == 0 ? xi[a] : g.n[a] - xi[a];
                const double range = 0.5 * di + rng_extra;
                if (!(dist < range)) continue;
                double n[3] = {0, 0, 0};
                n[a] = side == 0 ? -1.0 : 1.0;
                partner(ph, n, dist, 0.5 * di, ui, wi, di, zero, zero, mi, 2.0 * di, F, T, nlim);
            }
        }
        // Eq. particle_motion, semi-implicit Euler with I = m d^2 / 10
        const double I = mi * di * di / 10.0;
        double d2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double Ft = A.pf[(PFH0 + a) * cap + i] + F[a];
            const double un = ui[a] + ph.dt_dem * Ft / mi;
            const double wn = wi[a] + ph.dt_dem * T[a] / I;
            double xn = xi[a] + ph.dt_dem * un;
            if (g.per[a]) {
                const int L = g.n[a];
                xn -= L * floor(xn / L);
                if (xn >= L) xn -= L;
            }
            A.xout[a * cap + i] = xn;
            A.xout[(3 + a) * cap + i] = un;
            A.xout[(6 + a) * cap + i] = wn;
            const double dd = min_image(xn - A.pf[(PXS0 + a) * cap + i], g.n[a], g.per[a]);
            d2 += dd * dd;
        }
        if (d2 > ph.skin_half2) atomicOr(A.status, ST_SKIN);
        if (!(d2 < 1e30)) atomicOr(A.status, ST_NAN);
        if (nlim) atomicAdd(&A.counters[CNT_LUB_LIMITED], (unsigned long long)nlim);
    }
  }
}

void launch_dem_substep(const BoxDev *boxes, const Tile *tiles, int ntiles, int src_tmp, int grid, int block,
                        cudaStream_t s) {
    k_dem_substep<<<grid, block, 0, s>>>(boxes, tiles, ntiles, src_tmp);
}

}  // namespace dps
