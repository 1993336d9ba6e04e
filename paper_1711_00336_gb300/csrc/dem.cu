// dem.cu -- S6: the DEM substeps of Algorithm 1.
//
// Per particle (cell-sorted order): contact (Sec. 3.1.1, linear spring-dashpot
// with Coulomb-capped viscous friction), lubrication (Sec. 3.1.3, Ball &
// Melrose) against neighbours and walls, then the explicit update of Eq.
// particle_motion with the frozen F_fp + F_g.
//
// Neighbour list: after every sort a Verlet list is built per particle from
// the linked cells of the +-R cells around it, keeping every partner within
// the interaction range plus the skin; the n_DEM substeps then loop over the
// list only.  FP64 form: each pair of the list is evaluated once per substep
// (k_dem_pairs64) and a gather kernel adds it to both partners in an order
// fixed by the list (k_dem_gather64).  Mixed forms: a substep gives each
// particle a group of LANES consecutive lanes of a warp: lane l takes the list
// entries l, l + LANES, ... and the group's force and torque sums are combined
// by warp shuffles (a fixed xor tree, so the result does not depend on the
// launch shape); one thread per particle then adds the walls and integrates.
// A particle that moves more than skin/2 before the next sort raises
// DPS_ERR_UNSTABLE.  Candidate distances are screened in FP32 (a float
// copy of the positions, refreshed every substep, with a margin far above its
// rounding) and every pair that passes is evaluated: in FP64 for the FP64
// form, and in FP32 for the low-precision forms, where a pair close to
// contact (gap below 1e-3 dx or overlap) takes its separation from the FP64
// positions.  Positions, velocities and the integration are FP64 in every
// form.  State is read from one buffer and
// written to the other (ping-pong), so every pair sees the substep start.
#include "box.cuh"

namespace dps {

static constexpr double PI_D = 3.14159265358979323846;
static constexpr float SCREEN_MARGIN = 1e-3f;  // >> FP32 rounding of positions < 2^16 cells
static constexpr double H_NEAR = 1e-3;         // gaps below this: separation from the FP64 positions (mixed forms)

// minimum image for |dx| < L (positions live in [0, L))
__device__ __forceinline__ double min_image(double dx, int L, int per) {
    if (!per) return dx;
    const double h = 0.5 * L;
    return dx > h ? dx - L : (dx < -h ? dx + L : dx);
}
__device__ __forceinline__ float min_image_f(float dx, float L, int per) {
    if (!per) return dx;
    const float h = 0.5f * L;
    return dx > h ? dx - L : (dx < -h ? dx + L : dx);
}

template <typename T>
__device__ __forceinline__ void cross3(const T a[3], const T b[3], T o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// closure constants of the pair forces in arithmetic T, converted once per
// tile (no FP64 conversions inside the FP32 pair loop)
template <typename T>
struct PairPar {
    T kfac, xfac, mu_c, h_c, h_min, mu, capfac;
    int contact, lubrication, lub_limiter;
};
template <typename T>
__device__ __forceinline__ PairPar<T> pair_par(const Phys &ph) {
    PairPar<T> q;
    q.kfac = (T)ph.kfac;
    q.xfac = (T)ph.xfac;
    q.mu_c = (T)ph.mu_c;
    q.h_c = (T)ph.h_c;
    q.h_min = (T)ph.h_min;
    q.mu = (T)ph.mu;
    q.capfac = (T)ph.capfac;
    q.contact = ph.contact;
    q.lubrication = ph.lubrication;
    q.lub_limiter = ph.lub_limiter;
    return q;
}

// spring-dashpot contact with Coulomb friction (Sec. 3.1.1) for overlap
// delta > 0, in arithmetic T, accumulated in T; the torque is
// (d_i/2) n x F_t (r x F at the contact point r = d_i/2 n).
// lev: the lever of the torque, d_i/2 (or 1, which leaves n x F_t in Tq for
// the pair kernel of the FP64 form: both partners take it times their d/2)
template <typename T>
__device__ __forceinline__ void contact_force(const PairPar<T> &ph, const T n[3], T delta, const T ui[3],
                                              const T wi[3], T di, const T uj[3], const T wjh[3], T m_ij, T lev,
                                              T F[3], T Tq[3]) {
    // k_n and xi_n of Eqs. damping_to_stiffness / collision_time, solved
    // for the given e_n and T_c: both proportional to m_ij
    const T k_n = m_ij * ph.kfac;
    const T xi = m_ij * ph.xfac;
    T ws[3], wx[3], ur[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) ws[a] = T(0.5) * di * wi[a] + wjh[a];
    cross3(ws, n, wx);
#pragma unroll
    for (int a = 0; a < 3; ++a) ur[a] = ui[a] - uj[a] + wx[a];
    const T urn = ur[0] * n[0] + ur[1] * n[1] + ur[2] * n[2];
    T ut[3], Fn[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        ut[a] = ur[a] - urn * n[a];
        Fn[a] = -k_n * delta * n[a] - xi * (urn * n[a]);
    }
    const T Fn_abs = m_sqrt(Fn[0] * Fn[0] + Fn[1] * Fn[1] + Fn[2] * Fn[2]);
    const T ut_abs = m_sqrt(ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2]);
    T Ft[3] = {0, 0, 0};
    if (ut_abs > T(0)) {
        const T mag = m_min(ph.mu_c * Fn_abs, xi * ut_abs) / ut_abs;
#pragma unroll
        for (int a = 0; a < 3; ++a) Ft[a] = -mag * ut[a];
    }
    T nF[3];
    cross3(n, Ft, nF);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        F[a] += Fn[a] + Ft[a];
        Tq[a] += lev * nF[a];
    }
}

// lubrication correction (Sec. 3.1.3) at the floored gap hh, given <d>,
// r = <d>/hh, ir = 1/r and the limiter cap m_ij capfac
template <typename T>
__device__ __forceinline__ void lub_force(const PairPar<T> &ph, const T n[3], T dmean, T r, T ir, T cap,
                                          const T ui[3], const T uj[3], T F[3], unsigned &nlim) {
    const T L = m_log(T(0.5) * r);  // ln(<d>/(2h))
    T a_sq = T(1.5 * PI_D) * ph.mu * dmean * (T(0.25) * r + T(18.0 / 40.0) * L + T(9.0 / 84.0) * L * ir);
    // a_sh (2/(h+<d>))^2 = (pi/2) mu <d> ln(<d>/(2h))
    T a_sh = T(0.5 * PI_D) * ph.mu * dmean * L;
    a_sq = m_max(a_sq, T(0));
    a_sh = m_max(a_sh, T(0));
    if (ph.lub_limiter) {
        if (a_sq > cap) { a_sq = cap; ++nlim; }
        if (a_sh > cap) { a_sh = cap; ++nlim; }
    }
    T upr[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) upr[a] = ui[a] - uj[a];
    const T upn = upr[0] * n[0] + upr[1] * n[1] + upr[2] * n[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) F[a] += -a_sq * upn * n[a] - a_sh * (upr[a] - upn * n[a]);
}

// force and torque on i from one partner (sphere or wall), Sec. 3.1.1 / 3.1.3,
// given m_ij and <d>: contact while overlapping, lubrication on pairs that do
// not overlap, 0 <= h < h_c (in contact the spring-dashpot acts alone, which
// keeps the wet rebound of Sec. 5)
// gap = |x_j - x_i| - (d_i + d_j)/2 (negative: the overlap).
template <typename T>
__device__ __forceinline__ void partner(const PairPar<T> &ph, const T n[3], T gap, const T ui[3], const T wi[3],
                                        T di, const T uj[3], const T wjh[3], T m_ij, T dmean, T F[3], T Tq[3],
                                        unsigned &nlim) {
    const T delta = -gap;
    if (ph.contact && delta > T(0)) contact_force(ph, n, delta, ui, wi, di, uj, wjh, m_ij, T(0.5) * di, F, Tq);
    const T h = gap;
    if (ph.lubrication && h >= T(0) && h < ph.h_c) {
        const T hh = m_max(h, ph.h_min);
        const T q = T(1) / (dmean * hh);  // r and 1/r from one division
        lub_force(ph, n, dmean, dmean * dmean * q, hh * hh * q, m_ij * ph.capfac, ui, uj, F, nlim);
    }
}

// list of particle i: partners j != i with |x_j - x_i| < (d_i+d_j)/2 + extra + skin
// (screened in FP32 with a margin), stored row by row: nlist[i*maxn + k].
// LANES lanes share a particle (the tile's lanes of the particle-side
// kernels): lane l scans the cell rows l, l + LANES, ...
// of the (2R+1)^2 rows around it, counts its partners, takes its offset from
// an exclusive sum over the lanes, then scans again and writes them, so the
// list is in lane-major row order whatever the launch shape.
constexpr int NL_CACHE = 8;  // partners per lane kept between the two passes

#ifndef DPS_NLIST_MINB
#define DPS_NLIST_MINB 4  // 256-thread blocks per SM the register budget is sized for (a latency-bound search)
#endif
__global__ void __launch_bounds__(256, DPS_NLIST_MINB) k_build_nlist(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles,
                                                     int ntiles) {
    __shared__ int nl_cache[256][NL_CACHE];
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &Bx = boxes[tl.box];
        // lanes per particle of the tile (1 for large boxes, whose lists then
        // run in plain row order; more for boxes with few particles)
        const int LANES = tl.first > 1 ? tl.first : 1;
        const int lane = threadIdx.x % LANES, grp = threadIdx.x / LANES, ngrp = blockDim.x / LANES;
        const Geom g = Bx.g;
        const Phys &ph = Bx.ph;
        const float4 *xf = Bx.xf[0];
        const float extra = (float)((ph.lubrication ? fmax(ph.h_c, 0.0) : 0.0) + ph.skin) + SCREEN_MARGIN;
        const float Lf[3] = {(float)g.n[0], (float)g.n[1], (float)g.n[2]};
        const int R = Bx.R, maxn = Bx.maxn;
        // the trip count is uniform over the block: every lane reaches the shuffles
        for (long long base = tl.begin; base < tl.end; base += ngrp) {
            const long long i = base + grp;
            const bool act = i < tl.end;
            float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
            int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
            if (act) {
                pi = xf[i];
                const int b[3] = {containing_cell((double)pi.x, g.n[0]), containing_cell((double)pi.y, g.n[1]),
                                  containing_cell((double)pi.z, g.n[2])};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (g.per[a] && 2 * R + 1 >= g.n[a]) {
                        lo[a] = 0;
                        hi[a] = g.n[a] - 1;
                    } else if (g.per[a]) {
                        lo[a] = b[a] - R;
                        hi[a] = b[a] + R;
                    } else {
                        lo[a] = max(b[a] - R, 0);
                        hi[a] = min(b[a] + R, g.n[a] - 1);
                    }
                }
            }
            const int ny = hi[1] - lo[1] + 1, nz = hi[2] - lo[2] + 1, nrows = act ? ny * nz : 0;
            // the x segments of a cell row (two where the row wraps
            // periodically), and the rows, are visited in ascending cell index
            // of the wrapped cells, so that one lane's partners come out in
            // ascending sorted index (the cells are the sort's keys)
            int xs0[2] = {lo[0], 0}, xs1[2] = {hi[0], -1};
            if (lo[0] < 0) {
                xs0[0] = 0;
                xs1[0] = hi[0];
                xs0[1] = lo[0] + g.n[0];
                xs1[1] = g.n[0] - 1;
            } else if (hi[0] > g.n[0] - 1) {
                xs0[0] = 0;
                xs1[0] = hi[0] - g.n[0];
                xs0[1] = lo[0];
                xs1[1] = g.n[0] - 1;
            }
            const int roty = lo[1] < 0 ? -lo[1] : (hi[1] > g.n[1] - 1 ? g.n[1] - lo[1] : 0);
            const int rotz = lo[2] < 0 ? -lo[2] : (hi[2] > g.n[2] - 1 ? g.n[2] - lo[2] : 0);
            // partners of particle i in this lane's rows r = lane, lane +
            // LANES, ..., in row order, then the sorted order inside a row; the
            // particle ranges of RB rows are loaded together before any is
            // scanned, so their loads are in flight at once
            constexpr int RB = 8;
            auto scan_rows = [&](auto &&fn) {
                for (int r0 = lane; r0 < nrows; r0 += RB * LANES) {
                    int s[2 * RB], e[2 * RB];
#pragma unroll
                    for (int u = 0; u < RB; ++u) {
                        const int r = r0 + u * LANES;
                        s[2 * u] = e[2 * u] = s[2 * u + 1] = e[2 * u + 1] = 0;
                        if (r >= nrows) continue;
                        const int yy = lo[1] + (r % ny + roty) % ny, zz = lo[2] + (r / ny + rotz) % nz;
                        const int z = zz < 0 ? zz + g.n[2] : (zz >= g.n[2] ? zz - g.n[2] : zz);
                        const int y = yy < 0 ? yy + g.n[1] : (yy >= g.n[1] ? yy - g.n[1] : yy);
                        const long long row = cell_index(g, 0, y, z);
#pragma unroll
                        for (int sg = 0; sg < 2; ++sg)
                            if (xs1[sg] >= xs0[sg]) {
                                s[2 * u + sg] = Bx.cell_start[row + xs0[sg]];
                                e[2 * u + sg] = Bx.cell_start[row + xs1[sg] + 1];
                            }
                    }
#pragma unroll
                    for (int v = 0; v < 2 * RB; ++v)
                        for (int j = s[v]; j < e[v]; ++j) {
                            if (j == i) continue;
                            const float4 pj = xf[j];
                            const float dx = min_image_f(pj.x - pi.x, Lf[0], g.per[0]);
                            const float dy = min_image_f(pj.y - pi.y, Lf[1], g.per[1]);
                            const float dz = min_image_f(pj.z - pi.z, Lf[2], g.per[2]);
                            const float rr = 0.5f * (pi.w + pj.w) + extra;
                            if (dx * dx + dy * dy + dz * dz < rr * rr) fn(j);
                        }
                }
            };
            // one lane: a single pass writes the list.  Several lanes: pass 1
            // counts and keeps the first NL_CACHE partners of the lane in
            // shared memory; pass 2 writes them (scanning again only past that)
            int cnt = 0;
            int *cache = nl_cache[threadIdx.x];
            int *lst = Bx.nlist + i * (long long)maxn;
            if (LANES == 1) {
                scan_rows([&](int j) {
                    if (cnt < maxn) lst[cnt] = j;
                    ++cnt;
                });
                if (act) {
                    Bx.nlist_n[i] = min(cnt, maxn);
                    if (cnt > maxn) atomicOr(Bx.status, ST_NLIST);
                }
                continue;
            }
            scan_rows([&](int j) {
                if (cnt < NL_CACHE) cache[cnt] = j;
                ++cnt;
            });
            // exclusive sum of the counts over the lanes of the group
            int off = cnt;
            for (int o = 1; o < LANES; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, off, o);
                if (lane >= o) off += v;
            }
            const int total = __shfl_sync(0xffffffffu, off, (threadIdx.x & 31) - lane + LANES - 1);
            off -= cnt;
            if (!act) continue;
            if (cnt <= NL_CACHE) {
                for (int c = 0; c < cnt; ++c)
                    if (off + c < maxn) lst[off + c] = cache[c];
            } else {
                int w = off;
                scan_rows([&](int j) {
                    if (w < maxn && w < off + cnt) lst[w] = j;  // within the lane's counted slots
                    ++w;
                });
            }
            if (lane == 0) {
                Bx.nlist_n[i] = min(total, maxn);
                if (total > maxn) atomicOr(Bx.status, ST_NLIST);
            }
        }
    }
}

// the exact FP64 interaction with entry j (Sec. 3.1.1 / 3.1.3): a sphere
// (j >= 0; separation from the FP64 positions) or a wall face
// (j = -1 - (2 axis + side), side 1 the face at n[axis]; m_ij = m_i,
// <d> = 2 d_i, partner at rest).  Both kinds run one contact / lubrication
// body.  Out of line in the mixed forms, where it runs for the rare pairs
// near contact only, so that its registers do not limit the occupancy of the
// FP32 pair loop.
__device__ __forceinline__ void pair64_body(const PairPar<double> &pd, const double *__restrict__ xin,
                                            const double *__restrict__ pf, long long cap, const Geom &g, long long j,
                                            const double xi[3], const double ui[3], const double wi[3], double di,
                                            double mi, double rng_extra, double lev, double F[3], double T[3],
                                            unsigned &nlim) {
    double n[3] = {0, 0, 0}, uj[3] = {0, 0, 0}, wjh[3] = {0, 0, 0};
    double dist, sumr, dj = 0.0, mj = 1.0;
    const bool wall = j < 0;
    if (!wall) {
        double dx[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) dx[a] = min_image(xin[a * cap + j] - xi[a], g.n[a], g.per[a]);
        const double dist2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
        dj = pf[PD * cap + j];
        sumr = 0.5 * (di + dj);
        if (!(dist2 > 0.0)) return;
        const double inv = rsqrt(dist2);  // 1/|dx| and |dx| from one reciprocal square root
        dist = dist2 * inv;
        if (!(dist < sumr + rng_extra)) return;
        mj = pf[PM * cap + j];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            n[a] = dx[a] * inv;
            uj[a] = xin[(3 + a) * cap + j];
        }
    } else {
        const int face = -1 - (int)j, ax = face >> 1, side = face & 1;
        const double xa = ax == 0 ? xi[0] : (ax == 1 ? xi[1] : xi[2]);
        const int L = ax == 0 ? g.n[0] : (ax == 1 ? g.n[1] : g.n[2]);
        dist = side == 0 ? xa : L - xa;
        sumr = 0.5 * di;
        if (!(dist < sumr + rng_extra)) return;
        const double sg = side == 0 ? -1.0 : 1.0;
        n[0] = ax == 0 ? sg : 0.0;
        n[1] = ax == 1 ? sg : 0.0;
        n[2] = ax == 2 ? sg : 0.0;
    }
    // m_ij = A / Bm and <d> = C / D: spheres m_i m_j / (m_i + m_j) and
    // 2 d_i d_j / (d_i + d_j), walls m_i and 2 d_i; one division per pair
    // (FP64 instructions bound this path on GB300)
    const double A = wall ? mi : mi * mj, Bm = wall ? 1.0 : mi + mj;
    const double C = wall ? 2.0 * di : 2.0 * di * dj, D = wall ? 1.0 : di + dj;
    const double delta = sumr - dist;
    if (pd.contact && delta > 0.0) {
        // the partner's spin only matters in contact (the friction)
        if (!wall) {
#pragma unroll
            for (int a = 0; a < 3; ++a) wjh[a] = 0.5 * dj * xin[(6 + a) * cap + j];
        }
        contact_force(pd, n, delta, ui, wi, di, uj, wjh, A / Bm, lev, F, T);
    }
    const double h = dist - sumr;
    if (pd.lubrication && h >= 0.0 && h < pd.h_c) {
        const double hh = fmax(h, pd.h_min);
        const double q = 1.0 / (Bm * D * hh * C);
        const double dmean = wall ? C : C * C * Bm * hh * q;  // C / D
        const double r = C * C * Bm * q;                      // <d> / hh
        const double ir = Bm * D * D * hh * hh * q;           // hh / <d>
        const double cap = (wall ? A : A * D * hh * C * q) * pd.capfac;  // m_ij capfac
        lub_force(pd, n, dmean, r, ir, cap, ui, uj, F, nlim);
    }
}
// the mixed forms' pair within H_NEAR of contact.  The float copies of the
// positions carry absolute errors of up to ~3e-5 at x ~ 256, too coarse for
// such gaps, so the separation comes from the FP64 positions: |dx|^2 - s^2
// in FP64, divided by |dx| + s in FP32, a gap (or overlap) with FP32's
// relative precision however small it is; the forces then run in FP32 like
// every other pair.  Out of line, and returning its terms, so that the rare
// call costs the FP32 pair loop no registers.
struct NearTerms {
    float F[3], T[3];
    unsigned nlim;
};
__device__ __noinline__ NearTerms near_pair32(const BoxDev &Bx, const double *__restrict__ xin,
                                              const float4 *__restrict__ vin, const float4 *__restrict__ oin,
                                              const PairPar<float> &pfl, long long i, int j, float4 pi, float4 pj,
                                              float4 vi, float4 oi, float rng_extra_f) {
    NearTerms o = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, 0u};
    const double *pf = Bx.pf[Bx.cur];
    const long long cap = Bx.cap;
    const Geom g = Bx.g;
    double dx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) dx[a] = min_image(xin[a * cap + j] - xin[a * cap + i], g.n[a], g.per[a]);
    const double d2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2];
    const double s = 0.5 * (pf[PD * cap + i] + pf[PD * cap + j]);
    const float distf = sqrtf((float)d2);
    if (!(distf > 0.f)) return o;
    const float gap = (float)fma(-s, s, d2) / (distf + (float)s);
    if (!(gap < rng_extra_f)) return o;
    const float4 vj = vin[j], oj = oin[j];
    const float inv = 1.0f / distf;
    const float n[3] = {(float)dx[0] * inv, (float)dx[1] * inv, (float)dx[2] * inv};
    const float uif[3] = {vi.x, vi.y, vi.z}, wif[3] = {oi.x, oi.y, oi.z};
    const float uj[3] = {vj.x, vj.y, vj.z};
    const float wjh[3] = {0.5f * pj.w * oj.x, 0.5f * pj.w * oj.y, 0.5f * pj.w * oj.z};
    const float m_ij = vi.w * vj.w / (vi.w + vj.w);
    const float dmean = 2.0f * pi.w * pj.w / (pi.w + pj.w);
    partner<float>(pfl, n, gap, uif, wif, pi.w, uj, wjh, m_ij, dmean, o.F, o.T, o.nlim);
    return o;
}

// one thread per particle: wall partners (WALLS; the FP64 form evaluates
// them with the sphere pairs), then Eq. particle_motion (semi-implicit Euler)
// and the outputs of the substep
template <bool WALLS>
__device__ __forceinline__ void finish_particle(const BoxDev &Bx, const PairPar<double> &pd, long long i,
                                               int src_tmp, double F[3], double T[3], unsigned nlim, int key_out) {
    const double *xin = src_tmp ? Bx.xtmp : Bx.pf[Bx.cur];
    double *xout = src_tmp ? Bx.pf[Bx.cur] : Bx.xtmp;
    const float4 *fin = Bx.xf[src_tmp], *vin = Bx.vf[src_tmp];
    float4 *fout = Bx.xf[1 - src_tmp], *vout = Bx.vf[1 - src_tmp], *oout = Bx.of[1 - src_tmp];
    const double *pf = Bx.pf[Bx.cur];
    const long long cap = Bx.cap;
    const Geom g = Bx.g;
    const Phys &ph = Bx.ph;
    const double rng_extra = ph.lubrication ? fmax(ph.h_c, 0.0) : 0.0;
    double xi[3], ui[3], wi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        xi[a] = xin[a * cap + i];
        ui[a] = xin[(3 + a) * cap + i];
        wi[a] = xin[(6 + a) * cap + i];
    }
    const float4 pi = fin[i], vi = vin[i];
    const double di = pf[PD * cap + i];
    const double mi = pf[PM * cap + i];
    // walls: the faces of every non-periodic axis (m_ij = m_i, <d> = 2 d_i)
    const double zero[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!WALLS || g.per[a]) continue;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const double dist = side == 0 ? xi[a] : g.n[a] - xi[a];
            const double range = 0.5 * di + rng_extra;
            if (!(dist < range)) continue;
            double n[3] = {0, 0, 0};
            n[a] = side == 0 ? -1.0 : 1.0;
            partner<double>(pd, n, dist - 0.5 * di, ui, wi, di, zero, zero, mi, 2.0 * di, F, T, nlim);
        }
    }
    // Eq. particle_motion, semi-implicit Euler with I = m d^2 / 10
    const double dt_m = ph.dt_dem * pf[PIM * cap + i], dt_I = ph.dt_dem * pf[PII * cap + i];
    double d2 = 0.0, xn3[3], un3[3], wn3[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double Ft = pf[(PFH0 + a) * cap + i] + F[a];
        const double un = ui[a] + dt_m * Ft;
        const double wn = wi[a] + dt_I * T[a];
        double xn = xi[a] + ph.dt_dem * un;
        if (g.per[a]) {
            const double L = g.n[a];
            // a particle that left the box folds back in (two comparisons
            // for the rest, which stay put)
            if (!(xn >= 0.0 && xn < L)) {
                if (xn >= L) xn -= L;
                else if (xn < 0.0) xn += L;
                if (xn >= L || xn < 0.0) xn -= L * floor(xn / L);
                if (xn >= L) xn -= L;
            }
        }
        xn3[a] = xn;
        un3[a] = un;
        wn3[a] = wn;
        xout[a * cap + i] = xn;
        xout[(3 + a) * cap + i] = un;
        xout[(6 + a) * cap + i] = wn;
        const double dd = min_image(xn - pf[(PXS0 + a) * cap + i], g.n[a], g.per[a]);
        d2 += dd * dd;
    }
    fout[i] = make_float4((float)xn3[0], (float)xn3[1], (float)xn3[2], pi.w);
    vout[i] = make_float4((float)un3[0], (float)un3[1], (float)un3[2], vi.w);
    oout[i] = make_float4((float)wn3[0], (float)wn3[1], (float)wn3[2], 0.f);
    if (key_out) {
        // last substep of the subcycle: the linked cell of the new position,
        // counted for the sort that follows (its counting pass)
        const long long c = particle_cell(g, xn3[0], xn3[1], xn3[2], Bx.status);
        Bx.key[i] = (int)c;
        atomicAdd(&Bx.count[c], 1);
    }
    if (d2 > ph.skin_half2) atomicOr(Bx.status, ST_SKIN);
    if (!(d2 < 1e30)) atomicOr(Bx.status, ST_NAN);
    if (nlim) atomicAdd(&Bx.counters[CNT_LUB_LIMITED], (unsigned long long)nlim);
}

// ---- the substep of the mixed forms ----------------------------------------------------
// src_tmp = 0: read x/u/w (and the float positions) from the current set,
// write the ping-pong buffers; src_tmp = 1: the other way round.
// k_dem_pairsum_mixed: lane groups of LANES lanes per particle walk its list;
// pairs away from contact run in FP32 from the float copies, pairs near
// contact in FP32 from an FP64 separation (out of line); the group's sums (a
// fixed xor tree) go
// to psum[6][cap] (force, torque) and the lubrication-cap count to the
// counters.  k_dem_integrate then adds the walls and integrates, one thread
// per particle.  Two kernels so that each has its own register budget: the
// pair loop waits on the partners' loads and needs every warp slot of the SM,
// the FP64 update needs registers.
#ifndef DPS_MIXED_MINB
#define DPS_MIXED_MINB 8  // 256-thread blocks per SM the register budget of the pair loop is sized for
#endif
template <int LANES>
__global__ void __launch_bounds__(256, DPS_MIXED_MINB) k_dem_pairsum_mixed(const BoxDev *__restrict__ boxes,
                                                                       const Tile *__restrict__ tiles, int ntiles,
                                                                       int src_tmp) {
    const int lane = threadIdx.x % LANES, grp = threadIdx.x / LANES, ngrp = blockDim.x / LANES;
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &Bx = boxes[tl.box];
        const double *xin = src_tmp ? Bx.xtmp : Bx.pf[Bx.cur];
        const float4 *fin = Bx.xf[src_tmp], *vin = Bx.vf[src_tmp], *oin = Bx.of[src_tmp];
        const Geom g = Bx.g;
        const Phys &ph = Bx.ph;
        const float rng_extra_f = (float)(ph.lubrication ? fmax(ph.h_c, 0.0) : 0.0);
        const float Lf[3] = {(float)g.n[0], (float)g.n[1], (float)g.n[2]};
        const PairPar<float> pfl = pair_par<float>(ph);
        const long long cap = Bx.cap;
        // the trip count is uniform over the block, so every lane reaches the shuffles
        for (long long base = tl.begin; base < tl.end; base += ngrp) {
            const long long i = base + grp;
            const bool act = i < tl.end;
            float Ff[3] = {0, 0, 0}, Tf[3] = {0, 0, 0};
            unsigned nlim = 0;
            if (act) {
                const float4 pi = fin[i], vi = vin[i], oi = oin[i];
                const int nn = Bx.nlist_n[i];
                const int *row = Bx.nlist + i * (long long)Bx.maxn;
                for (int k = lane; k < nn; k += LANES) {
                    const int j = row[k];
                    const float4 pj = fin[j];
                    const float fx = min_image_f(pj.x - pi.x, Lf[0], g.per[0]);
                    const float fy = min_image_f(pj.y - pi.y, Lf[1], g.per[1]);
                    const float fz = min_image_f(pj.z - pi.z, Lf[2], g.per[2]);
                    const float sumr_f = 0.5f * (pi.w + pj.w);
                    const float fr = sumr_f + rng_extra_f + SCREEN_MARGIN;
                    const float d2f = fx * fx + fy * fy + fz * fz;
                    if (!(d2f < fr * fr)) continue;
                    const float distf = sqrtf(d2f);
                    if (distf - sumr_f > (float)H_NEAR + SCREEN_MARGIN) {
                        // away from contact: the separation from the float copies
                        if (!(distf < sumr_f + rng_extra_f)) continue;
                        const float4 vj = vin[j], oj = oin[j];
                        const float inv = 1.0f / distf;
                        const float n[3] = {fx * inv, fy * inv, fz * inv};
                        const float uif[3] = {vi.x, vi.y, vi.z}, wif[3] = {oi.x, oi.y, oi.z};
                        const float uj[3] = {vj.x, vj.y, vj.z};
                        const float wjh[3] = {0.5f * pj.w * oj.x, 0.5f * pj.w * oj.y, 0.5f * pj.w * oj.z};
                        const float m_ij = vi.w * vj.w / (vi.w + vj.w);
                        const float dmean = 2.0f * pi.w * pj.w / (pi.w + pj.w);
                        partner<float>(pfl, n, distf - sumr_f, uif, wif, pi.w, uj, wjh, m_ij, dmean, Ff, Tf, nlim);
                        continue;
                    }
                    // near contact: the separation from the FP64 positions
                    const NearTerms o = near_pair32(Bx, xin, vin, oin, pfl, i, j, pi, pj, vi, oi, rng_extra_f);
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        Ff[a] += o.F[a];
                        Tf[a] += o.T[a];
                    }
                    nlim += o.nlim;
                }
            }
            if (LANES > 1) {
#pragma unroll
                for (int o = LANES / 2; o > 0; o >>= 1) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        Ff[a] += __shfl_xor_sync(0xffffffffu, Ff[a], o);
                        Tf[a] += __shfl_xor_sync(0xffffffffu, Tf[a], o);
                    }
                    nlim += __shfl_xor_sync(0xffffffffu, nlim, o);
                }
            }
            if (act && lane == 0) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Bx.psum[a * cap + i] = (double)Ff[a];
                    Bx.psum[(3 + a) * cap + i] = (double)Tf[a];
                }
                if (nlim) atomicAdd(&Bx.counters[CNT_LUB_LIMITED], (unsigned long long)nlim);
            }
        }
    }
}

// walls and Eq. particle_motion of the mixed forms, one thread per particle
template <bool WALLS>
__global__ void __launch_bounds__(128) k_dem_integrate(const BoxDev *__restrict__ boxes,
                                                                     const Tile *__restrict__ tiles, int ntiles,
                                                                     int src_tmp, int key_out) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &Bx = boxes[tl.box];
        const long long cap = Bx.cap;
        const PairPar<double> pd = pair_par<double>(Bx.ph);
        for (long long i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            double F[3], T[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                F[a] = Bx.psum[a * cap + i];
                T[a] = Bx.psum[(3 + a) * cap + i];
            }
            finish_particle<WALLS>(Bx, pd, i, src_tmp, F, T, 0u, key_out);
        }
    }
}

// block-wide exclusive sum of one int per thread (blockDim a multiple of 32,
// at most 256); total over the block; ws: 9 ints of shared memory
__device__ __forceinline__ int block_excl_sum(int v, int *ws, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += u;
    }
    if (lane == 31) ws[wid] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int w = lane < nw ? ws[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += u;
        }
        if (lane < nw) ws[lane] = wi - w;
        if (lane == nw - 1) ws[8] = wi;
    }
    __syncthreads();
    const int r = ws[wid] + inc - v;
    total = ws[8];
    __syncthreads();  // ws may be reused
    return r;
}

// ---- FP64 form: every pair once (Newton's third law) ------------------------------
// The FP64 pair chain is what bounds this form on GB300 (a dense settling box
// keeps the FP64 pipe ~70 % busy), and the contact and lubrication laws of
// Sec. 3.1.1 / 3.1.3 are antisymmetric: F_ji = -F_ij, and with n_ji = -n_ij,
// F_t,ji = -F_t,ij the torques (d/2) n x F_t of both partners share n x F_t.
// So each substep evaluates each pair of the neighbour list once and a second
// kernel gathers, per particle and in a fixed order (its own pairs by
// ascending partner, then the pairs owned by its lower partners by ascending
// owner, then the walls), before the explicit update of Eq. particle_motion.

// After the list build: the pairs particle i owns (partners j > i, ascending
// j) get consecutive slots from a per-block allocation; its partners k < i
// go to rrow (ascending k) until k_reverse_slots replaces them by the slots
// of the pairs (k, i).  Ranks by counting keep the rows free of any sort.
__global__ void __launch_bounds__(256) k_half_rows(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles,
                                                   int ntiles) {
    __shared__ int ws[9];
    __shared__ unsigned long long sbase;
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &Bx = boxes[tl.box];
        const int maxn = Bx.maxn;
        for (long long base = tl.begin; base < tl.end; base += blockDim.x) {  // uniform trip count
            const long long i = base + threadIdx.x;
            const bool act = i < tl.end;
            int nn = 0, nh = 0;
            const int *row = Bx.nlist;
            if (act) {
                nn = min(Bx.nlist_n[i], maxn);
                row = Bx.nlist + i * (long long)maxn;
                for (int k = 0; k < nn; ++k) nh += row[k] > i;
            }
            int total;
            const int off = block_excl_sum(nh, ws, total);
            if (threadIdx.x == 0) sbase = atomicAdd(Bx.ptop, (unsigned long long)total);
            __syncthreads();
            const long long h0 = (long long)sbase + off;
            __syncthreads();  // sbase is written again in the next round
            if (!act) continue;
            if (h0 + nh > Bx.pcap) {  // not reached: pcap bounds the pairs of any list
                atomicOr(Bx.status, ST_NLIST);
                Bx.hn[i] = Bx.rn[i] = 0;
                continue;
            }
            Bx.hoff[i] = (int)h0;
            Bx.hn[i] = nh;
            Bx.rn[i] = nn - nh;
            int *rr = Bx.rrow + i * (long long)maxn;
            bool asc = true;  // rows of one lane come out ascending
            for (int k = 1; k < nn; ++k) asc = asc && row[k] > row[k - 1];
            if (asc) {
                const int lo = nn - nh;
                for (int k = 0; k < lo; ++k) rr[k] = row[k];
                for (int k = lo; k < nn; ++k) Bx.hj[h0 + k - lo] = row[k];
                continue;
            }
            for (int k = 0; k < nn; ++k) {
                const int j = row[k];
                const bool up = j > i;
                int r = 0;  // rank of j among the partners on its side of i
                for (int m = 0; m < nn; ++m) {
                    const int o = row[m];
                    r += o < j && (up ? o > i : o < i);
                }
                if (up)
                    Bx.hj[h0 + r] = j;
                else
                    rr[r] = j;
            }
        }
    }
}

// rrow: lower partner k -> the slot of the pair (k, i) (binary search of i in
// the ascending row of k)
__global__ void __launch_bounds__(256) k_reverse_slots(const BoxDev *__restrict__ boxes,
                                                       const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &Bx = boxes[tl.box];
        for (long long i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            const int nr = Bx.rn[i];
            int *rr = Bx.rrow + i * (long long)Bx.maxn;
            for (int r = 0; r < nr; ++r) {
                const int k = rr[r];
                const int hk = Bx.hn[k], ok = Bx.hoff[k];
                const int *h = Bx.hj + ok;
                int lo = 0, hi = hk;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (h[mid] < i)
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                if (lo < hk && h[lo] == i) {
                    rr[r] = ok + lo;
                } else {  // not reached: the list search is symmetric
                    rr[r] = -1;
                    atomicOr(Bx.status, ST_NLIST);
                }
            }
        }
    }
}

// The pairs of a substep.  Lane groups of LANES lanes screen the owned pairs
// of a particle in FP32 (with a margin); a block-wide exclusive sum places the
// entries that pass in a queue, evaluated one per thread by the exact FP64
// contact / lubrication body (an FP64 instruction costs a warp the same
// whatever number of its lanes are active), which writes the force on the
// owner and n x F_t to the pair's slot.  Every owned slot gets its flag.
constexpr int DQ_CAP = 512;

#ifndef DPS_PAIRS_MINB
#define DPS_PAIRS_MINB 2  // 256-thread blocks per SM the register budget is sized for
#endif
template <int LANES>
__global__ void __launch_bounds__(256, DPS_PAIRS_MINB) k_dem_pairs64(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles,
                                                     int ntiles, int src_tmp) {
    __shared__ int qS[DQ_CAP], qJ[DQ_CAP], qP[DQ_CAP];
    __shared__ int ws[9];
    const int lane = threadIdx.x % LANES, grp = threadIdx.x / LANES, ngrp = blockDim.x / LANES;
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &Bx = boxes[tl.box];
        const double *xin = src_tmp ? Bx.xtmp : Bx.pf[Bx.cur];
        const float4 *fin = Bx.xf[src_tmp];
        const double *pf = Bx.pf[Bx.cur];
        const long long cap = Bx.cap;
        const Geom g = Bx.g;
        const Phys &ph = Bx.ph;
        const double rng_extra = ph.lubrication ? fmax(ph.h_c, 0.0) : 0.0;
        const float rng_extra_f = (float)rng_extra;
        const float Lf[3] = {(float)g.n[0], (float)g.n[1], (float)g.n[2]};
        const PairPar<double> pd = pair_par<double>(ph);
        unsigned nlim = 0;
        for (long long base = tl.begin; base < tl.end; base += ngrp) {  // uniform trip count
            const long long i = base + grp;
            const bool act = i < tl.end;
            float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
            int nh = 0, h0 = 0;
            if (act) {
                pi = fin[i];
                nh = Bx.hn[i];
                h0 = Bx.hoff[i];
            }
            // the owned pairs of this lane (c = lane, lane + LANES, ...) that
            // pass the FP32 screen, in order: fn(slot, j)
            auto entries = [&](bool flag, auto &&fn) {
                for (int c = lane; c < nh; c += LANES) {
                    const int sl = h0 + c, j = Bx.hj[sl];
                    const float4 pj = fin[j];
                    const float fx = min_image_f(pj.x - pi.x, Lf[0], g.per[0]);
                    const float fy = min_image_f(pj.y - pi.y, Lf[1], g.per[1]);
                    const float fz = min_image_f(pj.z - pi.z, Lf[2], g.per[2]);
                    const float fr = 0.5f * (pi.w + pj.w) + rng_extra_f + SCREEN_MARGIN;
                    const bool pass = fx * fx + fy * fy + fz * fz < fr * fr;
                    if (flag) Bx.pflag[sl] = pass;
                    if (pass) fn(sl, j);
                }
            };
            int cnt = 0;
            if (act) entries(true, [&](int, int) { ++cnt; });
            int M;
            const int off = block_excl_sum(cnt, ws, M);
            for (int w0 = 0; w0 < M; w0 += DQ_CAP) {
                const int mw = M - w0 < DQ_CAP ? M - w0 : DQ_CAP;
                if (act && off < w0 + mw && off + cnt > w0) {
                    int c = off;
                    entries(false, [&](int sl, int j) {
                        // (c < off + cnt: both passes screen alike; the bound only
                        // keeps a lane inside its own slots)
                        if (c >= w0 && c < w0 + mw && c < off + cnt) {
                            qS[c - w0] = sl;
                            qJ[c - w0] = j;
                            qP[c - w0] = (int)(i - tl.begin);
                        }
                        ++c;
                    });
                }
                __syncthreads();
                for (int q = threadIdx.x; q < mw; q += blockDim.x) {
                    const long long ii = tl.begin + qP[q];
                    double xi[3], ui[3], wi[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        xi[a] = xin[a * cap + ii];
                        ui[a] = xin[(3 + a) * cap + ii];
                        wi[a] = xin[(6 + a) * cap + ii];
                    }
                    double Fq[3] = {0, 0, 0}, Cq[3] = {0, 0, 0};
                    pair64_body(pd, xin, pf, cap, g, qJ[q], xi, ui, wi, pf[PD * cap + ii], pf[PM * cap + ii],
                                rng_extra, 1.0, Fq, Cq, nlim);
                    // the force in the first plane; n x F_t, nonzero only for
                    // pairs in contact with friction, in the second, flagged 2
                    const long long sq = qS[q];
#pragma unroll
                    for (int a = 0; a < 3; ++a) Bx.pres[3 * sq + a] = Fq[a];
                    if (Cq[0] != 0.0 || Cq[1] != 0.0 || Cq[2] != 0.0) {
#pragma unroll
                        for (int a = 0; a < 3; ++a) Bx.pres[3 * (Bx.pcap + sq) + a] = Cq[a];
                        Bx.pflag[sq] = 2;
                    }
                }
                __syncthreads();  // the next window overwrites the queue
            }
        }
        // each capped coefficient acts on both partners (the count of the
        // per-particle evaluation of Sec. 3.1.3)
        if (nlim) atomicAdd(&Bx.counters[CNT_LUB_LIMITED], 2ull * nlim);
    }
}

// The sums of a substep and the update: one thread per particle adds the
// forces of its owned pairs (ascending partner), minus those of the pairs its
// lower partners own (ascending owner), each pair's n x F_t times d_i/2, then
// the walls and Eq. particle_motion.  The order depends on the list alone.
// WALLS: some box of the batch has a wall axis (else the wall code is left
// out: 128 registers instead of 168, more warps for a kernel that waits on
// the scattered loads of the pair results)
#ifndef DPS_GATHER_GC
#define DPS_GATHER_GC 4  // entries whose loads are issued before any is added
#endif
#ifndef DPS_GATHER_MINB
#define DPS_GATHER_MINB 4  // 128-thread blocks per SM the register budget is sized for
#endif
template <bool WALLS>
__global__ void __launch_bounds__(128, WALLS ? 1 : DPS_GATHER_MINB) k_dem_gather64(const BoxDev *__restrict__ boxes,
                                                        const Tile *__restrict__ tiles, int ntiles, int src_tmp,
                                                        int key_out) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &Bx = boxes[tl.box];
        const double *pf = Bx.pf[Bx.cur];
        const long long cap = Bx.cap;
        const PairPar<double> pd = pair_par<double>(Bx.ph);
        for (long long i = tl.begin + threadIdx.x; i < tl.end; i += blockDim.x) {
            const double lev = 0.5 * pf[PD * cap + i];
            double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
            const int h0 = Bx.hoff[i], nh = Bx.hn[i];
            const int nr = Bx.rn[i];
            const int *rr = Bx.rrow + i * (long long)Bx.maxn;
            // the entries in chunks of GC: the slot indices, flags and results
            // of a chunk are loaded before any is added (the loads, not the
            // additions, bound this kernel), a screened-out pair adding zero;
            // the additions keep the list order
            constexpr int GC = DPS_GATHER_GC;
            for (int c0 = 0; c0 < nh + nr; c0 += GC) {
                long long sl[GC];
                bool on[GC];
                double sg[GC];
#pragma unroll
                for (int u = 0; u < GC; ++u) {
                    const int c = c0 + u;
                    const int s = c < nh ? h0 + c : (c < nh + nr ? rr[c - nh] : -1);
                    sl[u] = s < 0 ? 0 : s;
                    on[u] = s >= 0;
                    sg[u] = c < nh ? 1.0 : -1.0;  // the owner's force, or its opposite on the partner
                }
                int fl[GC];
#pragma unroll
                for (int u = 0; u < GC; ++u) {
                    fl[u] = on[u] ? Bx.pflag[sl[u]] : 0;
                    on[u] = fl[u] != 0;
                }
                // the force of every pair that passed; n x F_t only where the
                // pair kernel flagged it (2): zero for all others
                double v[GC][6];
#pragma unroll
                for (int u = 0; u < GC; ++u)
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        v[u][a] = on[u] ? Bx.pres[3 * sl[u] + a] : 0.0;
                        v[u][3 + a] = fl[u] == 2 ? Bx.pres[3 * (Bx.pcap + sl[u]) + a] : 0.0;
                    }
#pragma unroll
                for (int u = 0; u < GC; ++u) {
                    if (!on[u]) continue;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        F[a] += sg[u] * v[u][a];
                        T[a] += lev * v[u][3 + a];
                    }
                }
            }
            finish_particle<WALLS>(Bx, pd, i, src_tmp, F, T, 0u, key_out);
        }
    }
}

// block: a multiple of 32 and of every tile's lanes (Tile::first).
// pairs: also the pair rows of the FP64 form (two more launches)
void launch_build_nlist(const BoxDev *boxes, const Tile *tiles, int ntiles, int grid, int block, int pairs,
                        cudaStream_t s) {
    k_build_nlist<<<grid, block, 0, s>>>(boxes, tiles, ntiles);
    if (pairs) {
        k_half_rows<<<grid, 128, 0, s>>>(boxes, tiles, ntiles);
        k_reverse_slots<<<grid, 128, 0, s>>>(boxes, tiles, ntiles);
    }
}

// lanes: 1, 2, 4 or 8 lanes per particle (block a multiple of 32); the FP64
// form launches its pair kernel and then its gather kernel; walls: some box
// has a wall axis
// key_out: the last substep of a subcycle also writes the particles' linked
// cells and their counts for the sort that follows
void launch_dem_substep(const BoxDev *boxes, const Tile *tiles, int ntiles, int src_tmp, int key_out, int mixed,
                        int lanes, int walls, int grid, int block, cudaStream_t s) {
#define DPS_DEM(K, L) K<L><<<grid, block, 0, s>>>(boxes, tiles, ntiles, src_tmp)
    if (mixed) {
        if (lanes >= 8) DPS_DEM(k_dem_pairsum_mixed, 8);
        else if (lanes == 4) DPS_DEM(k_dem_pairsum_mixed, 4);
        else if (lanes == 2) DPS_DEM(k_dem_pairsum_mixed, 2);
        else DPS_DEM(k_dem_pairsum_mixed, 1);
        if (walls)
            k_dem_integrate<true><<<grid, 128, 0, s>>>(boxes, tiles, ntiles, src_tmp, key_out);
        else
            k_dem_integrate<false><<<grid, 128, 0, s>>>(boxes, tiles, ntiles, src_tmp, key_out);
    } else {
#define DPS_PAIRS(L) k_dem_pairs64<L><<<grid, block, 0, s>>>(boxes, tiles, ntiles, src_tmp)
        if (lanes >= 8) DPS_PAIRS(8);
        else if (lanes == 4) DPS_PAIRS(4);
        else if (lanes == 2) DPS_PAIRS(2);
        else DPS_PAIRS(1);
#undef DPS_PAIRS
        if (walls)
            k_dem_gather64<true><<<grid, 128, 0, s>>>(boxes, tiles, ntiles, src_tmp, key_out);
        else
            k_dem_gather64<false><<<grid, 128, 0, s>>>(boxes, tiles, ntiles, src_tmp, key_out);
    }
#undef DPS_DEM
}

}  // namespace dps
