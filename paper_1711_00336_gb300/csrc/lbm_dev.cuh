// lbm_dev.cuh -- device helpers of the AA-pattern PDF storage: neighbour
// index deltas with periodic wrap / wall detection, parity-aware loads and
// stores of the 19 populations, and their first two moments (Eq. MacVel).
#pragma once
#include "dps_internal.cuh"

namespace dps {

// linear-index deltas to the -1/+1 neighbour along each axis; INV marks a
// neighbour beyond a wall.
// (ncell <= 2^27: 19 planes of offsets fit in 32 bits and no real delta equals INV)
constexpr int INV = (1 << 30);

struct NbDelta {
    int d[3][3];  // [axis][offset+1]
};

__device__ __forceinline__ void cell_coords(const Geom &g, long long c, int &ix, int &iy, int &iz) {
    const unsigned cc = (unsigned)c, nx = (unsigned)g.n[0], nxy = nx * (unsigned)g.n[1];
    const unsigned z = cc / nxy, r = cc - z * nxy, y = r / nx;
    iz = (int)z;
    iy = (int)y;
    ix = (int)(r - y * nx);
}

__device__ __forceinline__ NbDelta neighbour_deltas(const Geom &g, int ix, int iy, int iz) {
    NbDelta D;
    const int ii[3] = {ix, iy, iz};
    const int stride[3] = {1, g.n[0], g.n[0] * g.n[1]};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int L = g.n[a];
        D.d[a][1] = 0;
        D.d[a][0] = ii[a] > 0 ? -stride[a] : (g.per[a] ? (L - 1) * stride[a] : INV);
        D.d[a][2] = ii[a] < L - 1 ? stride[a] : (g.per[a] ? -(L - 1) * stride[a] : INV);
    }
    return D;
}

__device__ __forceinline__ int nb_delta(const NbDelta &D, int q) {
    const int dx = D.d[0][CX(q) + 1], dy = D.d[1][CY(q) + 1], dz = D.d[2][CZ(q) + 1];
    if (dx == INV || dy == INV || dz == INV) return INV;
    return dx + dy + dz;
}

// Load f_q(x,t) for all q at cell c under the AA parity.
template <typename ST, typename CT, int PAR>
__device__ __forceinline__ void load_pdfs(const ST *__restrict__ pdf, long long N, long long c,
                                          const NbDelta &D, CT f[Q]) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        if (PAR == 0 || q == 0) {
            f[q] = Store<ST>::load(pdf + (unsigned)(q * (unsigned)N + (unsigned)c));
        } else {
            // f_q(x) was written by the upstream cell x - c_q into plane opp(q);
            // across a wall it is the own cell's bounced value in plane q.
            int dm;
            {
                const int dx = D.d[0][-CX(q) + 1], dy = D.d[1][-CY(q) + 1], dz = D.d[2][-CZ(q) + 1];
                dm = (dx == INV || dy == INV || dz == INV) ? INV : dx + dy + dz;
            }
            if (dm != INV)
                f[q] = Store<ST>::load(pdf + (unsigned)(OPP(q) * (unsigned)N + (unsigned)c + (unsigned)dm));
            else
                f[q] = Store<ST>::load(pdf + (unsigned)(q * (unsigned)N + (unsigned)c));
        }
    }
}

// store the post-collision pair (k, k+9) under the AA parity
template <typename ST, typename CT, int PAR>
__device__ __forceinline__ void store_pair(ST *__restrict__ pdf, long long N, long long c, const NbDelta &D, int k,
                                           CT vk, CT vo) {
    const int o = k + 9;
    if (PAR == 0) {
        Store<ST>::store(pdf + (unsigned)(o * (unsigned)N + (unsigned)c), vk);
        Store<ST>::store(pdf + (unsigned)(k * (unsigned)N + (unsigned)c), vo);
    } else {
        const int dk = nb_delta(D, k), d_o = nb_delta(D, o);
        if (dk != INV) Store<ST>::store(pdf + (unsigned)(k * (unsigned)N + (unsigned)c + (unsigned)dk), vk);
        else Store<ST>::store(pdf + (unsigned)(o * (unsigned)N + (unsigned)c), vk);
        if (d_o != INV) Store<ST>::store(pdf + (unsigned)(o * (unsigned)N + (unsigned)c + (unsigned)d_o), vo);
        else Store<ST>::store(pdf + (unsigned)(k * (unsigned)N + (unsigned)c), vo);
    }
}

// cells with no wall neighbour (interior, or next to periodic faces only):
// the odd-parity neighbours are at the deltas of D with no bounce-back to
// resolve, so the loads and stores take no per-direction wall test
__device__ __forceinline__ bool no_wall_neighbour(const NbDelta &D) {
    return D.d[0][0] != INV && D.d[0][2] != INV && D.d[1][0] != INV && D.d[1][2] != INV && D.d[2][0] != INV &&
           D.d[2][2] != INV;
}

__device__ __forceinline__ unsigned wall_free_delta(const NbDelta &D, int cx, int cy, int cz) {
    return (unsigned)(D.d[0][cx + 1] + D.d[1][cy + 1] + D.d[2][cz + 1]);
}

// odd parity, no wall neighbour: f_q(x) sits in plane opp(q) of x - c_q
template <typename ST, typename CT>
__device__ __forceinline__ void load_pdfs_wall_free(const ST *__restrict__ pdf, unsigned N, unsigned c,
                                                    const NbDelta &D, CT f[Q]) {
    f[0] = Store<ST>::load(pdf + c);
#pragma unroll
    for (int q = 1; q < Q; ++q)
        f[q] = Store<ST>::load(pdf + ((unsigned)OPP(q) * N + c + wall_free_delta(D, -CX(q), -CY(q), -CZ(q))));
}

// odd parity, no wall neighbour: the post-collision pair (k, k+9) goes to the
// downstream cells x + c_k (plane k) and x - c_k (plane k+9)
template <typename ST, typename CT>
__device__ __forceinline__ void store_pair_wall_free(ST *__restrict__ pdf, unsigned N, unsigned c, const NbDelta &D,
                                                     int k, CT vk, CT vo) {
    Store<ST>::store(pdf + ((unsigned)k * N + c + wall_free_delta(D, CX(k), CY(k), CZ(k))), vk);
    Store<ST>::store(pdf + ((unsigned)(k + 9) * N + c + wall_free_delta(D, -CX(k), -CY(k), -CZ(k))), vo);
}

template <typename CT>
__device__ __forceinline__ void moments(const CT f[Q], CT &rho, CT &jx, CT &jy, CT &jz) {
    // pair sums: direction q and its opposite q+9
    CT r = f[0];
    CT x = 0, y = 0, z = 0;
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
        r += f[k] + f[k + 9];
        CT d = f[k] - f[k + 9];
        if (CX(k) != 0) x += CX(k) * d;
        if (CY(k) != 0) y += CY(k) * d;
        if (CZ(k) != 0) z += CZ(k) * d;
    }
    rho = r;
    jx = x;
    jy = y;
    jz = z;
}

}  // namespace dps
