// lbm.cu -- GNS lattice Boltzmann kernels (Sec. 3.2.2, Eqs. LBM_Equation,
// LBM_EQ, Forcing, MacVel) and the per-step fluid fields of Sec. 3.2.3.
//
// K1 collide-stream: one fused pass, in place with the AA pattern.  Even
//    parity reads and writes only the own cell (the post-collision value of
//    direction q goes to plane opp(q)); odd parity reads the upstream values
//    and writes the downstream cells.  Halfway bounce-back at wall faces is
//    folded into the odd-parity index map.  HBM traffic per cell: 19 loads and
//    19 stores of the PDF type plus eps_f and f_pf (4 loads of the field type);
//    in the FP64 coupled step also rho and j from K2a (4 more).
// K2a moments: rho, j of f(x,t), u_D = (j + f_ext/2)/(rho eps_f) and
//    1/(rho eps_f); one PDF read.
// K2b fields: stencil over rho and u_D giving grad(eps_f p) and Du_f/Dt.
#include "box.cuh"
#include "lbm_dev.cuh"

namespace dps {

// Eq. tau_e for one cell: tau_* from the Eilers viscosity of eps_p = 1 - eps_f
// (Eq. visc_eilers; eps_p/eps_cp capped at 0.9 where it diverges) plus the
// Smagorinsky tau_t (Eqs. visc_turb, tau_t) from the non-equilibrium momentum
// flux Q_ab = sum_q c_a c_b (f_q - f_q^eq) = Pi_ab - c_s^2 rho delta_ab -
// rho u_a u_b / eps.  Qbar = sqrt(2 sum Q_ab Q_ab); tau_t solves
// tau_t (tau_* + tau_t) = C_S^2 Qbar / (2 rho c_s^4) and is taken in the
// cancellation-free form x / (2 (sqrt(tau_*^2 + x) + tau_*)).  With DEV the
// second moments are of the deviations: Pi~_ab = Pi_ab - c_s^2 delta_ab, and
// s = rho - 1.
template <typename CT, bool DEV>
__device__ __forceinline__ CT tau_cell(const CT f[Q], CT s, CT rho, CT ux, CT uy, CT uz, CT e, CT ie, CT tau,
                                       int eilers, int smag) {
    CT ts = tau;
    if (eilers) {
        CT r = (CT(1) - e) * CT(1.0 / 0.64);
        r = r < CT(0) ? CT(0) : (r > CT(0.9) ? CT(0.9) : r);
        const CT a = CT(1) + CT(1.25 * 0.64) * r / (CT(1) - r);
        ts = CT(0.5) + (tau - CT(0.5)) * (a * a);
    }
    if (!smag) return ts;
    CT P[6] = {0, 0, 0, 0, 0, 0};  // xx yy zz xy xz yz
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
        const CT p = f[k] + f[k + 9];
        if (CX(k) != 0) P[0] += p;
        if (CY(k) != 0) P[1] += p;
        if (CZ(k) != 0) P[2] += p;
        if (CX(k) * CY(k) != 0) P[3] += CT(CX(k) * CY(k)) * p;
        if (CX(k) * CZ(k) != 0) P[4] += CT(CX(k) * CZ(k)) * p;
        if (CY(k) * CZ(k) != 0) P[5] += CT(CY(k) * CZ(k)) * p;
    }
    const CT iso = CT(1.0 / 3.0) * (DEV ? s : rho);
    const CT ri = rho * ie;
    const CT qxx = P[0] - iso - ri * ux * ux, qyy = P[1] - iso - ri * uy * uy, qzz = P[2] - iso - ri * uz * uz;
    const CT qxy = P[3] - ri * ux * uy, qxz = P[4] - ri * ux * uz, qyz = P[5] - ri * uy * uz;
    const CT q2 = qxx * qxx + qyy * qyy + qzz * qzz + CT(2) * (qxy * qxy + qxz * qxz + qyz * qyz);
    const CT x = CT(2 * 0.01 * 9) * m_sqrt(CT(2) * q2) / rho;  // 2 C_S^2 Qbar / (rho c_s^4)
    return ts + x / (CT(2) * (m_sqrt(ts * ts + x) + ts));
}

// K1 body for one cell: load the 19 populations (AA parity PAR), relax them
// (Eq. LBM_Equation, relax_cell) and store each opposite pair as soon as it
// is computed, which keeps few values live.  VISC: the box may
// relax with a per-cell tau_e (vmode bit 0 Eilers, bit 1 Smagorinsky).
template <typename ST, typename FT, typename CT, int PAR, bool VISC, bool MOMIN>
__device__ __forceinline__ void relax_store_cell(ST *__restrict__ pdf, CT f[Q], const NbDelta &D, bool in,
                                                 const Geom &g, CT e, CT fpx, CT fpy, CT fpz, long long N, long long c,
                                                 CT fbx, CT fby, CT fbz, CT omega_box, CT kf_box, CT tau, int vmode,
                                                 int *status, const CT *mom);

// the moments of cell c from K2a (MOMIN), else nothing
template <typename FT, typename CT, bool MOMIN>
__device__ __forceinline__ void load_moments(const FT *__restrict__ rho, const FT *__restrict__ j, long long N,
                                             long long c, CT mom[4]) {
    if (MOMIN) {
        mom[0] = (CT)rho[c];
        mom[1] = (CT)j[c];
        mom[2] = (CT)j[N + c];
        mom[3] = (CT)j[2 * N + c];
    }
}

template <typename ST, typename FT, typename CT, int PAR, bool VISC, bool MOMIN>
__device__ __forceinline__ void collide_stream_cell(ST *__restrict__ pdf, const FT *__restrict__ eps,
                                                    const FT *__restrict__ fpf, const FT *__restrict__ rho_m,
                                                    const FT *__restrict__ j_m, const Geom &g, long long c, CT fbx,
                                                    CT fby, CT fbz, CT omega_box, CT kf_box, CT tau, int vmode,
                                                    int *status) {
    const long long N = g.ncell;
    NbDelta D;
    bool in = false;
    CT f[Q];
    if (PAR) {
        int ix, iy, iz;
        cell_coords(g, c, ix, iy, iz);
        D = neighbour_deltas(g, ix, iy, iz);
        in = no_wall_neighbour(D);
        if (in)
            load_pdfs_wall_free<ST, CT>(pdf, (unsigned)N, (unsigned)c, D, f);
        else
            load_pdfs<ST, CT, PAR>(pdf, N, c, D, f);
    } else {
        load_pdfs<ST, CT, PAR>(pdf, N, c, D, f);
    }
    CT mom[4];
    load_moments<FT, CT, MOMIN>(rho_m, j_m, N, c, mom);
    relax_store_cell<ST, FT, CT, PAR, VISC, MOMIN>(pdf, f, D, in, g, (CT)eps[c], (CT)fpf[c], (CT)fpf[N + c],
                                                   (CT)fpf[2 * N + c], N, c, fbx, fby, fbz, omega_box, kf_box, tau,
                                                   vmode, status, mom);
}

// two cells per thread (c and c + stride): the loads of both are issued before
// either is relaxed, which doubles the bytes in flight per warp
template <typename ST, typename FT, typename CT, int PAR, bool VISC, bool MOMIN>
__device__ __forceinline__ void collide_stream_cell2(ST *__restrict__ pdf, const FT *__restrict__ eps,
                                                     const FT *__restrict__ fpf, const FT *__restrict__ rho_m,
                                                     const FT *__restrict__ j_m, const Geom &g, long long c,
                                                     long long c2, bool two, CT fbx, CT fby, CT fbz, CT omega_box,
                                                     CT kf_box, CT tau, int vmode, int *status) {
    const long long N = g.ncell;
    NbDelta D, D2;
    bool in = false, in2 = false;
    CT f[Q], f2[Q];
    if (PAR) {
        int ix, iy, iz;
        cell_coords(g, c, ix, iy, iz);
        D = neighbour_deltas(g, ix, iy, iz);
        in = no_wall_neighbour(D);
        if (in)
            load_pdfs_wall_free<ST, CT>(pdf, (unsigned)N, (unsigned)c, D, f);
        else
            load_pdfs<ST, CT, PAR>(pdf, N, c, D, f);
        if (two) {
            cell_coords(g, c2, ix, iy, iz);
            D2 = neighbour_deltas(g, ix, iy, iz);
            in2 = no_wall_neighbour(D2);
            if (in2)
                load_pdfs_wall_free<ST, CT>(pdf, (unsigned)N, (unsigned)c2, D2, f2);
            else
                load_pdfs<ST, CT, PAR>(pdf, N, c2, D2, f2);
        }
    } else {
        load_pdfs<ST, CT, PAR>(pdf, N, c, D, f);
        if (two) load_pdfs<ST, CT, PAR>(pdf, N, c2, D2, f2);
    }
    const CT e = (CT)eps[c], e2 = two ? (CT)eps[c2] : CT(1);
    const CT a0 = (CT)fpf[c], a1 = (CT)fpf[N + c], a2 = (CT)fpf[2 * N + c];
    CT b0 = 0, b1 = 0, b2 = 0;
    if (two) {
        b0 = (CT)fpf[c2];
        b1 = (CT)fpf[N + c2];
        b2 = (CT)fpf[2 * N + c2];
    }
    CT mom[4], mom2[4];
    load_moments<FT, CT, MOMIN>(rho_m, j_m, N, c, mom);
    if (two) load_moments<FT, CT, MOMIN>(rho_m, j_m, N, c2, mom2);
    relax_store_cell<ST, FT, CT, PAR, VISC, MOMIN>(pdf, f, D, in, g, e, a0, a1, a2, N, c, fbx, fby, fbz, omega_box,
                                                   kf_box, tau, vmode, status, mom);
    if (two)
        relax_store_cell<ST, FT, CT, PAR, VISC, MOMIN>(pdf, f2, D2, in2, g, e2, b0, b1, b2, N, c2, fbx, fby, fbz,
                                                       omega_box, kf_box, tau, vmode, status, mom2);
}

// two-element vectors of the stored type (low-precision forms): float2 or
// half2, converted exactly to and from the FP32 arithmetic (the FP16 stores
// round each element to nearest even, as the scalar stores do)
template <typename ST> struct Vec2;
template <> struct Vec2<float> {
    __device__ static inline void load(const float *p, float &a, float &b) {
        const float2 v = *reinterpret_cast<const float2 *>(p);
        a = v.x;
        b = v.y;
    }
    __device__ static inline void store(float *p, float a, float b) { *reinterpret_cast<float2 *>(p) = make_float2(a, b); }
};
template <> struct Vec2<double> {  // for completeness: the FP64 form keeps the scalar variant
    __device__ static inline void load(const double *p, double &a, double &b) {
        const double2 v = *reinterpret_cast<const double2 *>(p);
        a = v.x;
        b = v.y;
    }
    __device__ static inline void store(double *p, double a, double b) {
        *reinterpret_cast<double2 *>(p) = make_double2(a, b);
    }
};
template <> struct Vec2<__half> {
    __device__ static inline void load(const __half *p, float &a, float &b) {
        const float2 v = __half22float2(*reinterpret_cast<const __half2 *>(p));
        a = v.x;
        b = v.y;
    }
    __device__ static inline void store(__half *p, float a, float b) {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(a, b);
    }
};

template <typename ST, typename CT, bool VISC, bool MOMIN>
__device__ __forceinline__ void relax_cell(CT f[Q], CT e, CT fpx, CT fpy, CT fpz, CT fbx, CT fby, CT fbz,
                                           CT omega_box, CT kf_box, CT tau, int vmode, bool flag, int *status,
                                           const CT *mom);

// two cells c, c+1 of one x row (c even, nx even: the plane offsets, the
// pair and every y / z neighbour offset are even), both without a wall
// neighbour: a population whose memory offset keeps the pair aligned (even
// parity: every one; odd parity: those with c_x = 0) moves as one
// two-element vector, half the load and store instructions of the scalar
// path; the x-moving populations of the odd parity stay scalar.  A pair next
// to a wall takes the scalar path cell by cell.  The relaxation is that of
// the scalar path, so the results are the same bits.
template <typename ST, typename FT, typename CT, int PAR, bool VISC>
__device__ __forceinline__ void collide_stream_vec2(ST *__restrict__ pdf, const FT *__restrict__ eps,
                                                    const FT *__restrict__ fpf, const Geom &g, long long c, CT fbx,
                                                    CT fby, CT fbz, CT omega_box, CT kf_box, CT tau, int vmode,
                                                    int *status) {
    const long long N = g.ncell;
    int ix, iy, iz;
    cell_coords(g, c, ix, iy, iz);
    const NbDelta D = neighbour_deltas(g, ix, iy, iz), D1 = neighbour_deltas(g, ix + 1, iy, iz);
    if (!no_wall_neighbour(D) || !no_wall_neighbour(D1)) {
        collide_stream_cell<ST, FT, CT, PAR, VISC, false>(pdf, eps, fpf, nullptr, nullptr, g, c, fbx, fby, fbz,
                                                          omega_box, kf_box, tau, vmode, status);
        collide_stream_cell<ST, FT, CT, PAR, VISC, false>(pdf, eps, fpf, nullptr, nullptr, g, c + 1, fbx, fby, fbz,
                                                          omega_box, kf_box, tau, vmode, status);
        return;
    }
    const unsigned Nu = (unsigned)N, cu = (unsigned)c;
    CT f[Q], f1[Q];
    Vec2<ST>::load(pdf + cu, f[0], f1[0]);
#pragma unroll
    for (int q = 1; q < Q; ++q) {
        if (PAR == 0) {
            Vec2<ST>::load(pdf + ((unsigned)q * Nu + cu), f[q], f1[q]);
        } else if (CX(q) == 0) {
            Vec2<ST>::load(pdf + ((unsigned)OPP(q) * Nu + cu + wall_free_delta(D, 0, -CY(q), -CZ(q))), f[q], f1[q]);
        } else {
            f[q] = Store<ST>::load(pdf + ((unsigned)OPP(q) * Nu + cu + wall_free_delta(D, -CX(q), -CY(q), -CZ(q))));
            f1[q] = Store<ST>::load(pdf + ((unsigned)OPP(q) * Nu + cu + 1u +
                                           wall_free_delta(D1, -CX(q), -CY(q), -CZ(q))));
        }
    }
    // eps_f and f_pf of the pair as two-element vectors too (FT is float
    // in the forms that take this path; c and N are even)
    CT e0, e1, a[3], b[3];
    Vec2<FT>::load(eps + cu, e0, e1);
#pragma unroll
    for (int k = 0; k < 3; ++k) Vec2<FT>::load(fpf + ((unsigned)k * Nu + cu), a[k], b[k]);
    relax_cell<ST, CT, VISC, false>(f, e0, a[0], a[1], a[2], fbx, fby, fbz, omega_box, kf_box, tau, vmode, true,
                                    status, nullptr);
    relax_cell<ST, CT, VISC, false>(f1, e1, b[0], b[1], b[2], fbx, fby, fbz, omega_box, kf_box, tau, vmode, true,
                                    status, nullptr);
    Vec2<ST>::store(pdf + cu, f[0], f1[0]);
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
        if (PAR == 0) {
            Vec2<ST>::store(pdf + ((unsigned)(k + 9) * Nu + cu), f[k], f1[k]);
            Vec2<ST>::store(pdf + ((unsigned)k * Nu + cu), f[k + 9], f1[k + 9]);
        } else if (CX(k) == 0) {
            // (the offsets are summed in 32-bit unsigned arithmetic, where a
            // negative neighbour delta wraps, before they move the pointer)
            Vec2<ST>::store(pdf + ((unsigned)k * Nu + cu + wall_free_delta(D, 0, CY(k), CZ(k))), f[k], f1[k]);
            Vec2<ST>::store(pdf + ((unsigned)(k + 9) * Nu + cu + wall_free_delta(D, 0, -CY(k), -CZ(k))), f[k + 9],
                            f1[k + 9]);
        } else {
            store_pair_wall_free<ST, CT>(pdf, Nu, cu, D, k, f[k], f[k + 9]);
            store_pair_wall_free<ST, CT>(pdf, Nu, cu + 1u, D1, k, f1[k], f1[k + 9]);
        }
    }
}

// Correctly rounded single operations: the relaxation below spells out every
// multiply, add and fused multiply-add, so each K1 variant (register budget,
// cells per thread) rounds exactly alike and a box's result does not depend on
// the launch shape the autotuner picks.
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }

// relaxation (Eq. LBM_Equation) of one cell whose populations f, eps_f and
// f_pf are loaded: BGK relaxation towards the porous equilibrium (Eq.
// LBM_EQ) plus the Guo forcing term (Eq. Forcing); f is overwritten with the
// post-collision populations.  With deviation storage (shifted forms) the
// populations are f_q - w_q (rho_0 = 1): rho = 1 + sum, and the update of a
// deviation is f' - w = (1-omega)(f - w) + omega(f^eq - w) + F.  The update
// is written per opposite pair (q, q+9): the even part in c of
// omega f^eq + F is E = K0 + cu (K1 cu + K2 cF), the odd part
// O = K3 cu + K4 cF, with K0..K4 fixed per weight class.
// `flag`: report a non-finite or non-positive density.
// MOMIN: the moments s, j of these populations were computed by K2a in this
// step with the same sums (the FP64 form): they are passed in, not re-summed.
template <typename ST, typename CT, bool VISC, bool MOMIN = false>
__device__ __forceinline__ void relax_cell(CT f[Q], CT e, CT fpx, CT fpy, CT fpz, CT fbx, CT fby, CT fbz,
                                           CT omega_box, CT kf_box, CT tau, int vmode, bool flag, int *status,
                                           const CT *mom = nullptr) {
    constexpr bool DEV = Store<ST>::shifted;
    // f_ext = f_pf + eps_f f_b (Eq. Forcing)
    const CT Fx = r_fma(e, fbx, fpx);
    const CT Fy = r_fma(e, fby, fpy);
    const CT Fz = r_fma(e, fbz, fpz);
    CT s = f[0], jx = 0, jy = 0, jz = 0;
    if (MOMIN) {
        s = mom[0];
        jx = mom[1];
        jy = mom[2];
        jz = mom[3];
    } else {
#pragma unroll
        for (int k = 1; k <= 9; ++k) {
            s = r_add(s, r_add(f[k], f[k + 9]));
            const CT d = r_sub(f[k], f[k + 9]);
            if (CX(k) != 0) jx = CX(k) > 0 ? r_add(jx, d) : r_sub(jx, d);
            if (CY(k) != 0) jy = CY(k) > 0 ? r_add(jy, d) : r_sub(jy, d);
            if (CZ(k) != 0) jz = CZ(k) > 0 ? r_add(jz, d) : r_sub(jz, d);
        }
    }
    const CT rho = DEV ? r_add(CT(1), s) : s;
    if (flag && (!(rho > CT(0)) || !(rho < CT(1e30)))) atomicOr(status, ST_NAN);
    // 1/rho and 1/eps_f from one division (the FP64 form is bound by its
    // FP64 instruction count)
    const CT t = CT(1) / r_mul(rho, e);
    const CT ir = r_mul(e, t), ie = r_mul(rho, t);
    const CT ux = r_mul(r_fma(CT(0.5), Fx, jx), ir);  // Eq. MacVel
    const CT uy = r_mul(r_fma(CT(0.5), Fy, jy), ir);
    const CT uz = r_mul(r_fma(CT(0.5), Fz, jz), ir);
    CT omega = omega_box, kf = kf_box;
    if (VISC && vmode) {
        omega = CT(1) / tau_cell<CT, DEV>(f, s, rho, ux, uy, uz, e, ie, tau, vmode & 1, vmode & 2);
        kf = r_fma(CT(-0.5), omega, CT(1));
    }
    const CT uu = r_fma(ux, ux, r_fma(uy, uy, r_mul(uz, uz)));
    const CT uF = r_fma(ux, Fx, r_fma(uy, Fy, r_mul(uz, Fz)));
    const CT om1 = r_sub(CT(1), omega);
    const CT b2 = r_mul(r_mul(CT(-1.5), uu), ie);
    const CT e0 = DEV ? r_mul(omega, r_fma(rho, b2, s)) : r_mul(r_mul(omega, rho), r_add(CT(1), b2));
    const CT f0 = r_mul(r_mul(r_mul(CT(-3), kf), uF), ie);
    const CT ef = r_add(e0, f0);
    const CT k1 = r_mul(r_mul(r_mul(omega, rho), CT(4.5)), ie), k2 = r_mul(r_mul(CT(9), kf), ie);
    const CT k3 = r_mul(r_mul(CT(3), omega), rho), k4 = r_mul(CT(3), kf);
    f[0] = r_fma(om1, f[0], r_mul((CT)WQ(0), ef));
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
        const CT w = (CT)WQ(k);
        CT cu = 0, cF = 0;
        if (CX(k) != 0) { cu = CX(k) > 0 ? r_add(cu, ux) : r_sub(cu, ux); cF = CX(k) > 0 ? r_add(cF, Fx) : r_sub(cF, Fx); }
        if (CY(k) != 0) { cu = CY(k) > 0 ? r_add(cu, uy) : r_sub(cu, uy); cF = CY(k) > 0 ? r_add(cF, Fy) : r_sub(cF, Fy); }
        if (CZ(k) != 0) { cu = CZ(k) > 0 ? r_add(cu, uz) : r_sub(cu, uz); cF = CZ(k) > 0 ? r_add(cF, Fz) : r_sub(cF, Fz); }
        const CT E = r_mul(w, r_fma(cu, r_fma(k1, cu, r_mul(k2, cF)), ef));
        const CT O = r_mul(w, r_fma(k3, cu, r_mul(k4, cF)));
        const CT vk = r_fma(om1, f[k], r_add(E, O)), vo = r_fma(om1, f[k + 9], r_sub(E, O));
        f[k] = vk;
        f[k + 9] = vo;
    }
}

// relaxation and parity-aware stores of one cell
template <typename ST, typename FT, typename CT, int PAR, bool VISC, bool MOMIN>
__device__ __forceinline__ void relax_store_cell(ST *__restrict__ pdf, CT f[Q], const NbDelta &D, bool in,
                                                 const Geom &g, CT e, CT fpx, CT fpy, CT fpz, long long N, long long c,
                                                 CT fbx, CT fby, CT fbz, CT omega_box, CT kf_box, CT tau, int vmode,
                                                 int *status, const CT *mom) {
    relax_cell<ST, CT, VISC, MOMIN>(f, e, fpx, fpy, fpz, fbx, fby, fbz, omega_box, kf_box, tau, vmode, true, status,
                                    mom);
    Store<ST>::store(pdf + (unsigned)c, f[0]);
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
        if (PAR && in)
            store_pair_wall_free<ST, CT>(pdf, (unsigned)N, (unsigned)c, D, k, f[k], f[k + 9]);
        else
            store_pair<ST, CT, PAR>(pdf, N, c, D, k, f[k], f[k + 9]);
    }
}

template <typename CT> __device__ __forceinline__ CT pick(double d, float f);
template <> __device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float pick<float>(double, float f) { return f; }

// K1: every cell tile of every box, AA parity PAR (common to the batch).
// MOMIN: rho and j come from K2a of the same step (FP64 coupled step)
template <typename ST, typename FT, typename CT, int PAR, int MINB, bool VISC, int CPT, bool MOMIN = false>
__global__ void __launch_bounds__(128, MINB) k_collide_stream(const BoxDev *__restrict__ boxes,
                                                           const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        ST *pdf = (ST *)B.pdf;
        const FT *eps = (const FT *)B.eps, *fpf = (const FT *)B.fpf;
        const FT *rho_m = (const FT *)B.rho, *j_m = (const FT *)B.j;
        const CT fbx = pick<CT>(B.ph.fb[0], B.ph.fb_f[0]), fby = pick<CT>(B.ph.fb[1], B.ph.fb_f[1]),
                 fbz = pick<CT>(B.ph.fb[2], B.ph.fb_f[2]);
        const CT omega = pick<CT>(B.ph.omega, B.ph.omega_f), kf = pick<CT>(B.ph.kf, B.ph.kf_f);
        const CT tau = (CT)B.ph.tau;
        const int vmode = VISC ? (B.ph.eilers ? 1 : 0) | (B.ph.smag ? 2 : 0) : 0;
        int *st = B.status;
        if (CPT == 3 && sizeof(ST) < 8 && !MOMIN && !(g.n[0] & 1) && !(tl.begin & 1)) {
            // vector pairs (c even; nx even, so the tile ends are even too)
            for (long long c = tl.begin + 2 * threadIdx.x; c < tl.end; c += 2 * blockDim.x)
                collide_stream_vec2<ST, FT, CT, PAR, VISC>(pdf, eps, fpf, g, c, fbx, fby, fbz, omega, kf, tau, vmode,
                                                           st);
        } else if (CPT == 1 || CPT == 3) {
            for (long long c = tl.begin + threadIdx.x; c < tl.end; c += blockDim.x)
                collide_stream_cell<ST, FT, CT, PAR, VISC, MOMIN>(pdf, eps, fpf, rho_m, j_m, g, c, fbx, fby, fbz,
                                                                  omega, kf, tau, vmode, st);
        } else {
            for (long long c = tl.begin + threadIdx.x; c < tl.end; c += 2 * blockDim.x) {
                const long long c2 = c + blockDim.x;
                collide_stream_cell2<ST, FT, CT, PAR, VISC, MOMIN>(pdf, eps, fpf, rho_m, j_m, g, c, c2, c2 < tl.end,
                                                                   fbx, fby, fbz, omega, kf, tau, vmode, st);
            }
        }
    }
}

// K2a body: rho, j and u_D = (j + f_ext/2)/(rho eps) with the applied f_ext
template <typename ST, typename FT, typename CT, int PAR>
__device__ __forceinline__ void moments_cell(const ST *__restrict__ pdf, const FT *__restrict__ eps,
                                             const FT *__restrict__ fpf, const Geom &g, long long c, CT fbx, CT fby,
                                             CT fbz, FT *__restrict__ rho_o, FT *__restrict__ j_o,
                                             FT *__restrict__ uD, FT *__restrict__ ire) {
    const long long N = g.ncell;
    int ix, iy, iz;
    cell_coords(g, c, ix, iy, iz);
    NbDelta D = neighbour_deltas(g, ix, iy, iz);
    CT f[Q];
    load_pdfs<ST, CT, PAR>(pdf, N, c, D, f);
    CT rho, jx, jy, jz;
    moments(f, rho, jx, jy, jz);
    if (Store<ST>::shifted) rho += CT(1);  // deviations: sum of the shifts w_q is 1
    const CT e = (CT)eps[c];
    const CT Fx = (CT)fpf[c] + e * fbx, Fy = (CT)fpf[N + c] + e * fby, Fz = (CT)fpf[2 * N + c] + e * fbz;
    rho_o[c] = (FT)rho;
    j_o[c] = (FT)jx;
    j_o[N + c] = (FT)jy;
    j_o[2 * N + c] = (FT)jz;
    const CT s = CT(1) / (rho * e);
    ire[c] = (FT)s;  // the first subcycle's drag interpolation reuses it
    uD[c] = (FT)((jx + CT(0.5) * Fx) * s);
    uD[N + c] = (FT)((jy + CT(0.5) * Fy) * s);
    uD[2 * N + c] = (FT)((jz + CT(0.5) * Fz) * s);
}

template <typename ST, typename FT, typename CT, int PAR>
__global__ void __launch_bounds__(128, sizeof(CT) == 8 ? 2 : 4) k_moments(const BoxDev *__restrict__ boxes,
                                                    const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        const ST *pdf = (const ST *)B.pdf;
        const FT *eps = (const FT *)B.eps, *fpf = (const FT *)B.fpf;
        FT *rho = (FT *)B.rho, *j = (FT *)B.j, *uD = (FT *)B.uD, *ire = (FT *)B.ire;
        const CT fbx = pick<CT>(B.ph.fb[0], B.ph.fb_f[0]), fby = pick<CT>(B.ph.fb[1], B.ph.fb_f[1]),
                 fbz = pick<CT>(B.ph.fb[2], B.ph.fb_f[2]);
        for (long long c = tl.begin + threadIdx.x; c < tl.end; c += blockDim.x)
            moments_cell<ST, FT, CT, PAR>(pdf, eps, fpf, g, c, fbx, fby, fbz, rho, j, uD, ire);
    }
}

// K2b: grad P with P = eps_f p = c_s^2 rho, and Du_f/Dt = (u_D - u_prev) +
// (u_D . grad) u_D, with the lattice gradient of Sec. 3.2.3.  Neighbours
// beyond a wall are mirrored into the box (coordinate clamped).
template <typename FT, typename CT>
__global__ void __launch_bounds__(256) k_fields(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles,
                                                int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const Geom g = B.g;
        const long long N = g.ncell;
        const FT *rho = (const FT *)B.rho, *uD = (const FT *)B.uD;
        FT *uprev = (FT *)B.uprev, *gradP = (FT *)B.gradP, *DuDt = (FT *)B.DuDt;
        const int have_prev = B.have_uprev;
        for (long long c = tl.begin + threadIdx.x; c < tl.end; c += blockDim.x) {
            int ix, iy, iz;
            cell_coords(g, c, ix, iy, iz);
            long long stride[3] = {1, g.n[0], (long long)g.n[0] * g.n[1]};
            const int ii[3] = {ix, iy, iz};
            long long dd[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int L = g.n[a];
                dd[a][1] = 0;
                dd[a][0] = ii[a] > 0 ? -stride[a] : (g.per[a] ? (long long)(L - 1) * stride[a] : 0);
                dd[a][2] = ii[a] < L - 1 ? stride[a] : (g.per[a] ? -(long long)(L - 1) * stride[a] : 0);
            }
            CT gp[3] = {0, 0, 0};
            CT gu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // gu[a][b] = sum w c_a u_b
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const long long n = c + dd[0][CX(q) + 1] + dd[1][CY(q) + 1] + dd[2][CZ(q) + 1];
                const CT w = (CT)WQ(q);
                const CT r = (CT)rho[n];
                const CT u0 = (CT)uD[n], u1 = (CT)uD[N + n], u2 = (CT)uD[2 * N + n];
                const int cc[3] = {CX(q), CY(q), CZ(q)};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (cc[a] == 0) continue;
                    const CT wc = w * (CT)cc[a];
                    gp[a] += wc * r;
                    gu[a][0] += wc * u0;
                    gu[a][1] += wc * u1;
                    gu[a][2] += wc * u2;
                }
            }
            // c_s^-2 sum w c phi; for P = c_s^2 rho the c_s^2 cancels
            const CT u[3] = {(CT)uD[c], (CT)uD[N + c], (CT)uD[2 * N + c]};
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                gradP[b * N + c] = (FT)gp[b];
                const CT conv = CT(3) * (u[0] * gu[0][b] + u[1] * gu[1][b] + u[2] * gu[2][b]);
                const CT up = have_prev ? (CT)uprev[b * N + c] : u[b];
                DuDt[b * N + c] = (FT)((u[b] - up) + conv);
                uprev[b * N + c] = (FT)u[b];
            }
        }
    }
}

// Lift support (Table 1, Sec. 3.2.3): curl of the fluid velocity at the
// subcycle start, u_f = (j + eps_f f_b / 2)/(rho eps_f) with the current eps_f,
// by the lattice rule curl psi = c_s^-2 sum_q w_q c_q x psi(x + c_q) (walls:
// neighbour coordinate clamped, as for the gradient).  u_f of a neighbour is
// evaluated on the fly from rho, j and eps_f; boxes without lift are skipped.
template <typename FT, typename CT>
__global__ void __launch_bounds__(256) k_curl(const BoxDev *__restrict__ boxes, const Tile *__restrict__ tiles,
                                              int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        if (!B.ph.lift || B.np == 0) continue;
        const Geom g = B.g;
        const long long N = g.ncell;
        const FT *rho = (const FT *)B.rho, *j = (const FT *)B.j, *eps = (const FT *)B.eps;
        FT *curl = (FT *)B.curl;
        const CT hb[3] = {CT(0.5) * (CT)B.ph.fb[0], CT(0.5) * (CT)B.ph.fb[1], CT(0.5) * (CT)B.ph.fb[2]};
        for (long long c = tl.begin + threadIdx.x; c < tl.end; c += blockDim.x) {
            int ix, iy, iz;
            cell_coords(g, c, ix, iy, iz);
            long long stride[3] = {1, g.n[0], (long long)g.n[0] * g.n[1]};
            const int ii[3] = {ix, iy, iz};
            long long dd[3][3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                int L = g.n[a];
                dd[a][1] = 0;
                dd[a][0] = ii[a] > 0 ? -stride[a] : (g.per[a] ? (long long)(L - 1) * stride[a] : 0);
                dd[a][2] = ii[a] < L - 1 ? stride[a] : (g.per[a] ? -(long long)(L - 1) * stride[a] : 0);
            }
            CT r[3] = {0, 0, 0};
#pragma unroll
            for (int q = 1; q < Q; ++q) {
                const long long n = c + dd[0][CX(q) + 1] + dd[1][CY(q) + 1] + dd[2][CZ(q) + 1];
                const CT e = (CT)eps[n];
                const CT sc = CT(1) / ((CT)rho[n] * e);
                const CT v0 = ((CT)j[n] + e * hb[0]) * sc;
                const CT v1 = ((CT)j[N + n] + e * hb[1]) * sc;
                const CT v2 = ((CT)j[2 * N + n] + e * hb[2]) * sc;
                const CT w = CT(3) * (CT)WQ(q);
                if (CY(q) != 0 || CZ(q) != 0) r[0] += w * (CT(CY(q)) * v2 - CT(CZ(q)) * v1);
                if (CZ(q) != 0 || CX(q) != 0) r[1] += w * (CT(CZ(q)) * v0 - CT(CX(q)) * v2);
                if (CX(q) != 0 || CY(q) != 0) r[2] += w * (CT(CX(q)) * v1 - CT(CY(q)) * v0);
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) curl[a * N + c] = (FT)r[a];
        }
    }
}

// ---- canonical PDF export / import (FP64 host view) -------------------------
template <typename ST, int PAR>
__global__ void k_pdf_export(const ST *__restrict__ pdf, Geom g, double *__restrict__ out) {
    const long long N = g.ncell;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        cell_coords(g, c, ix, iy, iz);
        NbDelta D = neighbour_deltas(g, ix, iy, iz);
        if constexpr (sizeof(ST) == 8) {
            double f[Q];
            load_pdfs<ST, double, PAR>(pdf, N, c, D, f);
#pragma unroll
            for (int q = 0; q < Q; ++q) out[(long long)q * N + c] = f[q];
        } else {
            float f[Q];
            load_pdfs<ST, float, PAR>(pdf, N, c, D, f);
#pragma unroll
            for (int q = 0; q < Q; ++q) out[(long long)q * N + c] = (double)f[q] + WQ(q);
        }
    }
}

// import always writes the even (canonical) layout
template <typename ST>
__global__ void k_pdf_import(ST *__restrict__ pdf, long long N, const double *__restrict__ in) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if constexpr (sizeof(ST) == 8)
                Store<ST>::store(pdf + (long long)q * N + c, in[(long long)q * N + c]);
            else  // shifted storage: the deviation is taken in FP64, then rounded
                Store<ST>::store(pdf + (long long)q * N + c, (float)(in[(long long)q * N + c] - WQ(q)));
        }
    }
}

// ---- host launchers ----------------------------------------------------------
static int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    long long cap = 152LL * 16;  // grid-stride beyond this
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

// variant: register budget of K1 (blocks of 128 threads per SM the compiler
// must fit) and cells per thread (variants 3, 4, 5: two; 6, 7: two adjacent
// cells moved as two-element vectors); chosen by the batch
// autotuner.  visc: some box of the batch
// relaxes with a per-cell tau_e (one register budget for that variant).
template <typename ST, typename FT, typename CT>
void launch_collide_stream(const BoxDev *boxes, const Tile *tiles, int ntiles, int parity, int variant, bool visc,
                           bool mom_in, int grid, int block, cudaStream_t s) {
    block = 128;
    if (sizeof(CT) == 8) variant = 0;  // FP64: one register-heavy variant
#define DPS_K1VM(MB, V, CPT, M)                                                                           \
    do {                                                                                                  \
        if (parity)                                                                                       \
            k_collide_stream<ST, FT, CT, 1, MB, V, CPT, M><<<grid, block, 0, s>>>(boxes, tiles, ntiles);  \
        else                                                                                              \
            k_collide_stream<ST, FT, CT, 0, MB, V, CPT, M><<<grid, block, 0, s>>>(boxes, tiles, ntiles);  \
    } while (0)
#define DPS_K1V(MB, V, CPT) DPS_K1VM(MB, V, CPT, false)
#define DPS_K1(MB, CPT) DPS_K1V(MB, false, CPT)
    if constexpr (sizeof(CT) == 8) {
        // the FP64 coupled step takes rho and j from K2a (same sums, one
        // fifth fewer FP64 instructions)
        if (visc) {
            if (mom_in) DPS_K1VM(2, true, 1, true);
            else DPS_K1V(2, true, 1);
        } else {
            if (mom_in) DPS_K1VM(2, false, 1, true);
            else DPS_K1(2, 1);
        }
    } else if (visc)
        DPS_K1V(3, true, 1);
    else if (variant == 1)
        DPS_K1(3, 1);
    else if (variant == 2)
        DPS_K1(5, 1);
    else if (variant == 3)
        DPS_K1(3, 2);
    else if (variant == 4)
        DPS_K1(4, 2);
    else if (variant == 5)
        DPS_K1(2, 2);
    else if (variant == 6)
        DPS_K1(4, 3);
    else if (variant == 7)
        DPS_K1(3, 3);
    else
        DPS_K1(4, 1);
#undef DPS_K1
#undef DPS_K1V
#undef DPS_K1VM
}

template <typename ST, typename FT, typename CT>
void launch_moments(const BoxDev *boxes, const Tile *tiles, int ntiles, int parity, int grid, int block,
                    cudaStream_t s) {
    if (block > 128) block = 128;
    if (parity)
        k_moments<ST, FT, CT, 1><<<grid, block, 0, s>>>(boxes, tiles, ntiles);
    else
        k_moments<ST, FT, CT, 0><<<grid, block, 0, s>>>(boxes, tiles, ntiles);
}

template <typename FT, typename CT>
void launch_fields(const BoxDev *boxes, const Tile *tiles, int ntiles, int grid, int block, cudaStream_t s) {
    k_fields<FT, CT><<<grid, block, 0, s>>>(boxes, tiles, ntiles);
}

template <typename FT, typename CT>
void launch_curl(const BoxDev *boxes, const Tile *tiles, int ntiles, int grid, int block, cudaStream_t s) {
    k_curl<FT, CT><<<grid, block, 0, s>>>(boxes, tiles, ntiles);
}

template <typename ST>
void launch_pdf_export(const void *pdf, const Geom &g, int parity, double *out, cudaStream_t s) {
    const int B = 128;
    if (parity == 0)
        k_pdf_export<ST, 0><<<grid_for(g.ncell, B), B, 0, s>>>((const ST *)pdf, g, out);
    else
        k_pdf_export<ST, 1><<<grid_for(g.ncell, B), B, 0, s>>>((const ST *)pdf, g, out);
}

template <typename ST>
void launch_pdf_import(void *pdf, long long N, const double *in, cudaStream_t s) {
    const int B = 128;
    k_pdf_import<ST><<<grid_for(N, B), B, 0, s>>>((ST *)pdf, N, in);
}

// explicit instantiations for the three precision forms
#define DPS_LBM_INST(ST, FT, CT)                                                                             \
    template void launch_collide_stream<ST, FT, CT>(const BoxDev *, const Tile *, int, int, int, bool, bool, int, int, cudaStream_t); \
    template void launch_moments<ST, FT, CT>(const BoxDev *, const Tile *, int, int, int, int, cudaStream_t);
DPS_LBM_INST(double, double, double)
DPS_LBM_INST(float, float, float)
DPS_LBM_INST(__half, float, float)
template void launch_fields<double, double>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
template void launch_fields<float, float>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
template void launch_curl<double, double>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
template void launch_curl<float, float>(const BoxDev *, const Tile *, int, int, int, cudaStream_t);
template void launch_pdf_export<double>(const void *, const Geom &, int, double *, cudaStream_t);
template void launch_pdf_export<float>(const void *, const Geom &, int, double *, cudaStream_t);
template void launch_pdf_export<__half>(const void *, const Geom &, int, double *, cudaStream_t);
template void launch_pdf_import<double>(void *, long long, const double *, cudaStream_t);
template void launch_pdf_import<float>(void *, long long, const double *, cudaStream_t);
template void launch_pdf_import<__half>(void *, long long, const double *, cudaStream_t);

}  // namespace dps
