// dps_internal.cuh -- shared definitions of the CUDA implementation of the
// coupled LBM-DEM step (Rettinger & Ruede, arXiv:1711.00336) for sm_103a.
//
// Data layout in HBM (one domain):
//   PDFs      19 planes of ncell values, SoA, plane q at pdf + q*ncell; the
//             storage type is double (DPS_F64), float or half (shifted by
//             w_q rho_0 in the two low-precision forms).  In-place AA pattern:
//             at even parity plane q holds f_q(x); at odd parity f_q(x) sits in
//             plane opp(q) of the upstream cell x - c_q.
//   fields    planes of ncell values of the field type FT (double for DPS_F64,
//             float otherwise): eps_f, rho, j(3), u_D(3), u_prev(3), DuDt(3),
//             gradP(3), f_pf applied (3), f_pf of the subcycle (3), f_pf sum (3);
//             with the lift force the u_D planes hold, during the subcycles,
//             the curl of the subcycle-start fluid velocity
//   particles SoA of doubles [field][cap] in cell-sorted order, two sets
//             (main / alternate) for the sort gather and the DEM ping-pong.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "dps.h"
#include "tlog.cuh"

namespace dps {

constexpr int Q = 19;

// ---------------------------------------------------------------------------
// D3Q19 (Sec. 3.2.2).  Direction 0 is the rest population; 1..9 are the
// "positive" velocities and q+9 is the opposite of q, which pairs every
// population with its bounce-back partner.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pos_cx(int k) {  // k = 1..9
    return k == 1 ? 1 : k == 2 ? 0 : k == 3 ? 0 : k == 4 ? 1 : k == 5 ? 1 : k == 6 ? 1 : k == 7 ? 1 : 0;
}
__host__ __device__ constexpr int pos_cy(int k) {
    return k == 1 ? 0 : k == 2 ? 1 : k == 3 ? 0 : k == 4 ? 1 : k == 5 ? -1 : k == 6 ? 0 : k == 7 ? 0 : k == 8 ? 1 : 1;
}
__host__ __device__ constexpr int pos_cz(int k) {
    return k == 1 ? 0 : k == 2 ? 0 : k == 3 ? 1 : k == 4 ? 0 : k == 5 ? 0 : k == 6 ? 1 : k == 7 ? -1 : k == 8 ? 1 : -1;
}
__host__ __device__ constexpr int CX(int q) { return q == 0 ? 0 : (q <= 9 ? pos_cx(q) : -pos_cx(q - 9)); }
__host__ __device__ constexpr int CY(int q) { return q == 0 ? 0 : (q <= 9 ? pos_cy(q) : -pos_cy(q - 9)); }
__host__ __device__ constexpr int CZ(int q) { return q == 0 ? 0 : (q <= 9 ? pos_cz(q) : -pos_cz(q - 9)); }
__host__ __device__ constexpr int OPP(int q) { return q == 0 ? 0 : (q <= 9 ? q + 9 : q - 9); }
__host__ __device__ constexpr double WQ(int q) {
    return q == 0 ? 1.0 / 3.0 : ((CX(q) * CX(q) + CY(q) * CY(q) + CZ(q) * CZ(q)) == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// status bits of the device status word
enum : int {
    ST_NAN = 1,        // non-finite or non-positive density
    ST_SKIN = 2,       // a particle moved more than skin/2 since the last sort
    ST_EPS_NEG = 4,    // eps_f below zero before the floor
    ST_BAD_CELL = 8,   // particle outside the box on a wall axis
    ST_TIMEOUT = 16,
    ST_NLIST = 32,     // a neighbour list overflowed its capacity
};

// counters (unsigned long long) in device memory
enum : int { CNT_EPS_CLAMP = 0, CNT_LUB_LIMITED = 1, CNT_N = 4 };

// ---- particle SoA fields (doubles) ----------------------------------------
enum : int {
    PX = 0, PY, PZ,          // position
    PU, PV, PW,              // velocity
    POX, POY, POZ,           // angular velocity
    PD, PRHO,                // diameter, density
    PM, PIM, PII,            // mass m, 1/m and 10/(m d^2) (set at every sort)
    PVOL,                    // volume pi d^3 / 6 (set at every sort)
    PUS0, PUS1, PUS2,        // u at the start of the previous subcycle
    PFH0, PFH1, PFH2,        // frozen F_fp + F_g of the subcycle
    PFA0, PFA1, PFA2,        // added-mass force of the subcycle
    PFD0, PFD1, PFD2,        // drag force of the subcycle
    PXS0, PXS1, PXS2,        // position at the last sort (skin check)
    PW0,                     // 9 weights: axis a, offset o -> PW0 + 3a + o
    NPF = PW0 + 9
};
// ints
enum : int { IID = 0, ICELL, IKEY, NPI };

struct PSet {
    double *f;   // [NPF][cap]
    int32_t *i;  // [NPI][cap]
};

// geometry of a box, passed by value to kernels
struct Geom {
    int n[3];
    int per[3];
    long long ncell;
    int B;          // bin edge (cells)
    int nb[3];      // bins per axis
};

__host__ __device__ inline long long cell_index(const Geom &g, int ix, int iy, int iz) {
    return ix + (long long)g.n[0] * (iy + (long long)g.n[1] * iz);
}

// bin helpers (bins of B cells, last bin of an axis takes the remainder)
__host__ __device__ inline int bin_of(int i, int B, int nb) {
    int b = i / B;
    return b > nb - 1 ? nb - 1 : b;
}
__host__ __device__ inline int bin_width(int b, int B, int nb, int L) { return b == nb - 1 ? L - b * B : B; }

// key of cell (ix,iy,iz): bin-major (bz,by,bx), then (z,y,x) inside the bin
__host__ __device__ inline long long cell_key(const Geom &g, int ix, int iy, int iz) {
    int bx = bin_of(ix, g.B, g.nb[0]), by = bin_of(iy, g.B, g.nb[1]), bz = bin_of(iz, g.B, g.nb[2]);
    int sx = bx * g.B, sy = by * g.B, sz = bz * g.B;
    int Wx = bin_width(bx, g.B, g.nb[0], g.n[0]);
    int Wy = bin_width(by, g.B, g.nb[1], g.n[1]);
    int Wz = bin_width(bz, g.B, g.nb[2], g.n[2]);
    long long Lx = g.n[0], Ly = g.n[1];
    long long first = (long long)sz * Ly * Lx + (long long)Wz * sy * Lx + (long long)Wz * Wy * sx;
    return first + ((long long)(iz - sz) * Wy + (iy - sy)) * Wx + (ix - sx);
}
// first key and number of cells of bin (bx,by,bz)
__host__ __device__ inline void bin_range(const Geom &g, int bx, int by, int bz, long long *first,
                                          long long *count) {
    int sx = bx * g.B, sy = by * g.B, sz = bz * g.B;
    int Wx = bin_width(bx, g.B, g.nb[0], g.n[0]);
    int Wy = bin_width(by, g.B, g.nb[1], g.n[1]);
    int Wz = bin_width(bz, g.B, g.nb[2], g.n[2]);
    long long Lx = g.n[0], Ly = g.n[1];
    *first = (long long)sz * Ly * Lx + (long long)Wz * sy * Lx + (long long)Wz * Wy * sx;
    *count = (long long)Wx * Wy * Wz;
}

// cell containing coordinate x along an axis of L cells (clamped into the box)
__host__ __device__ inline int containing_cell(double x, int L) {
    int i = (int)floor(x);
    return i < 0 ? 0 : (i > L - 1 ? L - 1 : i);
}

// linked cell of a particle (flags a position outside the box on a wall axis)
__device__ __forceinline__ long long particle_cell(const Geom &g, double x, double y, double z, int *st) {
    int ix = containing_cell(x, g.n[0]), iy = containing_cell(y, g.n[1]), iz = containing_cell(z, g.n[2]);
    if (st && ((!g.per[0] && (x < 0.0 || x >= g.n[0])) || (!g.per[1] && (y < 0.0 || y >= g.n[1])) ||
               (!g.per[2] && (z < 0.0 || z >= g.n[2]))))
        atomicOr(st, ST_BAD_CELL);
    return cell_index(g, ix, iy, iz);
}

// closure constants, derived once on the host
struct Phys {
    double tau, omega, kf, rho_f, mu;   // kf = 1 - 1/(2 tau) (Eq. Forcing)
    float omega_f, kf_f, fb_f[3];       // the same in FP32 for the low-precision forms
    double g[3], fb[3];
    double e_n, mu_c, T_c, h_c, h_min, C_am;
    double lub_cap;
    double eps_min;
    double dt_sub, dt_dem;
    double skin;         // Verlet skin (dx)
    double kfac, xfac;   // k_n = m_ij kfac, xi_n = m_ij xfac (Eqs. damping_to_stiffness, collision_time)
    double capfac;       // lubrication cap = m_ij capfac
    double skin_half2;   // (skin / 2)^2: largest displacement between two sorts
    int n_int, n_dem;
    int drag, pressure, added_mass, lubrication, contact, lub_limiter;
    int lift;            // Table 1 shear lift (curl of u_f at the subcycle start)
    int eilers, smag;    // per-cell tau_e (Eqs. visc_eilers, tau_t, tau_e)
};

// ---- precision-preserving math -----------------------------------------------
// The kernels are templated on their arithmetic type; these overloads call the
// single-precision functions for float, so FP32 arithmetic never widens to
// FP64 (whose pipe is a small fraction of the FP32 rate on GB300).
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return tlog(x); }  // tlog.cuh
__device__ __forceinline__ float m_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double m_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float m_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double m_max(double a, double b) { return fmax(a, b); }

// ---- PDF storage traits ---------------------------------------------------
// FP64 stores f_q itself; the low-precision forms store the deviation
// f_q - w_q rho_0 (shifted populations) and do all arithmetic on deviations,
// so that FP32 / FP16 precision applies to the small non-equilibrium parts.
template <typename ST> struct Store;
template <> struct Store<double> {
    static constexpr bool shifted = false;
    __device__ static inline double load(const double *p) { return *p; }
    __device__ static inline void store(double *p, double v) { *p = v; }
};
template <> struct Store<float> {
    static constexpr bool shifted = true;
    __device__ static inline float load(const float *p) { return *p; }
    __device__ static inline void store(float *p, float v) { *p = v; }
};
template <> struct Store<__half> {
    static constexpr bool shifted = true;
    __device__ static inline float load(const __half *p) { return __half2float(*p); }
    __device__ static inline void store(__half *p, float v) { *p = __float2half_rn(v); }
};

}  // namespace dps
