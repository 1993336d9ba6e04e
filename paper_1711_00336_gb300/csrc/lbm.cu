// lbm.cu -- GNS lattice Boltzmann kernels (Sec. 3.2.2, Eqs. LBM_Equation,
// LBM_EQ, Forcing, MacVel) and the per-step fluid fields of Sec. 3.2.3.
//
// K1 collide-stream: one fused pass, in place with the AA pattern.  Even
//    parity reads and writes only the own cell (the post-collision value of
//    direction q goes to plane opp(q)); odd parity reads the upstream values
//    and writes the downstream cells.  Halfway bounce-back at wall faces is
//    folded into the odd-parity index map.  HBM traffic per cell: 19 loads and
//    19 stores of the PDF type plus eps_f and f_pf (4 loads of the field type).
// K2a moments: rho, j of f(x,t) and u_D = (j + f_ext/2)/(rho eps_f); one PDF read.
// K2b fields: stencil over rho and u_D giving grad(eps_f p) and Du_f/Dt.
#include "lbm_dev.cuh"

namespace dps {

// Eq. LBM_Equation for one cell: BGK relaxation towards the porous
// equilibrium (Eq. LBM_EQ) plus the Guo forcing term (Eq. Forcing), written
// per opposite pair (q, q+9): their equilibria share the even part in c.u and
// their forcing terms share the part even in c.
template <typename CT>
__device__ __forceinline__ void collide(CT f[Q], CT eps, CT Fx, CT Fy, CT Fz, CT omega, CT kf,
                                        CT &rho_out) {
    CT rho, jx, jy, jz;
    moments(f, rho, jx, jy, jz);
    const CT ir = CT(1) / rho;
    const CT ux = (jx + CT(0.5) * Fx) * ir;  // Eq. MacVel
    const CT uy = (jy + CT(0.5) * Fy) * ir;
    const CT uz = (jz + CT(0.5) * Fz) * ir;
    const CT ie = CT(1) / eps;
    const CT uu = ux * ux + uy * uy + uz * uz;
    const CT uF = ux * Fx + uy * Fy + uz * Fz;
    // rest population: c = 0
    {
        const CT w0 = (CT)WQ(0);
        const CT feq = w0 * rho * (CT(1) - CT(1.5) * uu * ie);
        const CT Fq = w0 * kf * (CT(-3) * uF * ie);
        f[0] = f[0] + omega * (feq - f[0]) + Fq;
    }
    const CT base = CT(1) - CT(1.5) * uu * ie;  // 1 - u.u/(2 eps c_s^2)
#pragma unroll
    for (int k = 1; k <= 9; ++k) {
        const CT w = (CT)WQ(k);
        CT cu = 0, cF = 0;
        if (CX(k) != 0) { cu += CX(k) * ux; cF += CX(k) * Fx; }
        if (CY(k) != 0) { cu += CY(k) * uy; cF += CY(k) * Fy; }
        if (CZ(k) != 0) { cu += CZ(k) * uz; cF += CZ(k) * Fz; }
        const CT wr = w * rho;
        const CT even = wr * (base + CT(4.5) * cu * cu * ie);      // even part of f^eq
        const CT odd = wr * CT(3) * cu;                             // odd part of f^eq
        const CT Feven = w * kf * (CT(9) * cu * cF - CT(3) * uF) * ie;
        const CT Fodd = w * kf * CT(3) * cF;
        const CT fp = f[k], fm = f[k + 9];
        f[k] = fp + omega * (even + odd - fp) + Feven + Fodd;
        f[k + 9] = fm + omega * (even - odd - fm) + Feven - Fodd;
    }
    rho_out = rho;
}

// K1
template <typename ST, typename FT, typename CT, int PAR>
__global__ void __launch_bounds__(128) k_collide_stream(ST *__restrict__ pdf, const FT *__restrict__ eps,
                                                        const FT *__restrict__ fpf, Geom g, CT fbx, CT fby,
                                                        CT fbz, CT omega, CT kf, CT inv_navg,
                                                        int *__restrict__ status) {
    const long long N = g.ncell;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        cell_coords(g, c, ix, iy, iz);
        NbDelta D = neighbour_deltas(g, ix, iy, iz);
        CT f[Q];
        load_pdfs<ST, CT, PAR>(pdf, N, c, D, f);
        const CT e = (CT)eps[c];
        // f_ext = f_pf + eps_f f_b (Eq. Forcing)
        const CT Fx = (CT)fpf[c] * inv_navg + e * fbx;
        const CT Fy = (CT)fpf[N + c] * inv_navg + e * fby;
        const CT Fz = (CT)fpf[2 * N + c] * inv_navg + e * fbz;
        CT rho;
        collide<CT>(f, e, Fx, Fy, Fz, omega, kf, rho);
        if (!(rho > CT(0)) || !(rho < CT(1e30))) atomicOr(status, ST_NAN);
        store_pdfs<ST, CT, PAR>(pdf, N, c, D, f);
    }
}

// K2a: rho, j and u_D = (j + f_ext/2)/(rho eps) with the applied f_ext.
template <typename ST, typename FT, typename CT, int PAR>
__global__ void __launch_bounds__(128) k_moments(const ST *__restrict__ pdf, const FT *__restrict__ eps,
                                                 const FT *__restrict__ fpf, Geom g, CT fbx, CT fby,
                                                 CT fbz, FT *__restrict__ rho_o, FT *__restrict__ j_o,
                                                 FT *__restrict__ uD) {
    const long long N = g.ncell;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        cell_coords(g, c, ix, iy, iz);
        NbDelta D = neighbour_deltas(g, ix, iy, iz);
        CT f[Q];
        load_pdfs<ST, CT, PAR>(pdf, N, c, D, f);
        CT rho, jx, jy, jz;
        moments(f, rho, jx, jy, jz);
        const CT e = (CT)eps[c];
        const CT Fx = (CT)fpf[c] + e * fbx, Fy = (CT)fpf[N + c] + e * fby, Fz = (CT)fpf[2 * N + c] + e * fbz;
        rho_o[c] = (FT)rho;
        j_o[c] = (FT)jx;
        j_o[N + c] = (FT)jy;
        j_o[2 * N + c] = (FT)jz;
        const CT s = CT(1) / (rho * e);
        uD[c] = (FT)((jx + CT(0.5) * Fx) * s);
        uD[N + c] = (FT)((jy + CT(0.5) * Fy) * s);
        uD[2 * N + c] = (FT)((jz + CT(0.5) * Fz) * s);
    }
}

// K2b: grad P with P = eps_f p = c_s^2 rho, and Du_f/Dt = (u_D - u_prev) +
// (u_D . grad) u_D, with the lattice gradient of Sec. 3.2.3.  Neighbours
// beyond a wall are mirrored into the box (coordinate clamped).
template <typename FT, typename CT>
__global__ void __launch_bounds__(128) k_fields(const FT *__restrict__ rho, const FT *__restrict__ uD,
                                                FT *__restrict__ uprev, Geom g, int have_prev,
                                                FT *__restrict__ gradP, FT *__restrict__ DuDt) {
    const long long N = g.ncell;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
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
        CT gu[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};  // gu[a][b] = d_a u_b
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
            for (int q = 0; q < Q; ++q) out[(long long)q * N + c] = (double)f[q];
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
                Store<ST>::store(pdf + (long long)q * N + c, in[(long long)q * N + c], 0.0);
            else
                Store<ST>::store(pdf + (long long)q * N + c, (float)in[(long long)q * N + c], (float)WQ(q));
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

template <typename ST, typename FT, typename CT>
void launch_collide_stream(void *pdf, const void *eps, const void *fpf, const Geom &g, const double fb[3],
                           double tau, int n_avg, int parity, int *status, cudaStream_t s) {
    const int B = 128;
    CT omega = (CT)(1.0 / tau), kf = (CT)(1.0 - 0.5 / tau), inv = (CT)(1.0 / n_avg);
    int grid = grid_for(g.ncell, B);
    if (parity == 0)
        k_collide_stream<ST, FT, CT, 0><<<grid, B, 0, s>>>((ST *)pdf, (const FT *)eps, (const FT *)fpf, g,
                                                           (CT)fb[0], (CT)fb[1], (CT)fb[2], omega, kf, inv, status);
    else
        k_collide_stream<ST, FT, CT, 1><<<grid, B, 0, s>>>((ST *)pdf, (const FT *)eps, (const FT *)fpf, g,
                                                           (CT)fb[0], (CT)fb[1], (CT)fb[2], omega, kf, inv, status);
}

template <typename ST, typename FT, typename CT>
void launch_moments(const void *pdf, const void *eps, const void *fpf, const Geom &g, const double fb[3],
                    int parity, void *rho, void *j, void *uD, cudaStream_t s) {
    const int B = 128;
    int grid = grid_for(g.ncell, B);
    if (parity == 0)
        k_moments<ST, FT, CT, 0><<<grid, B, 0, s>>>((const ST *)pdf, (const FT *)eps, (const FT *)fpf, g,
                                                    (CT)fb[0], (CT)fb[1], (CT)fb[2], (FT *)rho, (FT *)j, (FT *)uD);
    else
        k_moments<ST, FT, CT, 1><<<grid, B, 0, s>>>((const ST *)pdf, (const FT *)eps, (const FT *)fpf, g,
                                                    (CT)fb[0], (CT)fb[1], (CT)fb[2], (FT *)rho, (FT *)j, (FT *)uD);
}

template <typename FT, typename CT>
void launch_fields(const void *rho, const void *uD, void *uprev, const Geom &g, int have_prev, void *gradP,
                   void *DuDt, cudaStream_t s) {
    const int B = 128;
    k_fields<FT, CT><<<grid_for(g.ncell, B), B, 0, s>>>((const FT *)rho, (const FT *)uD, (FT *)uprev, g,
                                                        have_prev, (FT *)gradP, (FT *)DuDt);
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
#define DPS_LBM_INST(ST, FT, CT)                                                                          \
    template void launch_collide_stream<ST, FT, CT>(void *, const void *, const void *, const Geom &,      \
                                                    const double *, double, int, int, int *, cudaStream_t); \
    template void launch_moments<ST, FT, CT>(const void *, const void *, const void *, const Geom &,       \
                                             const double *, int, void *, void *, void *, cudaStream_t);
DPS_LBM_INST(double, double, double)
DPS_LBM_INST(float, float, float)
DPS_LBM_INST(__half, float, float)
template void launch_fields<double, double>(const void *, const void *, void *, const Geom &, int, void *,
                                            void *, cudaStream_t);
template void launch_fields<float, float>(const void *, const void *, void *, const Geom &, int, void *,
                                          void *, cudaStream_t);
template void launch_pdf_export<double>(const void *, const Geom &, int, double *, cudaStream_t);
template void launch_pdf_export<float>(const void *, const Geom &, int, double *, cudaStream_t);
template void launch_pdf_export<__half>(const void *, const Geom &, int, double *, cudaStream_t);
template void launch_pdf_import<double>(void *, long long, const double *, cudaStream_t);
template void launch_pdf_import<float>(void *, long long, const double *, cudaStream_t);
template void launch_pdf_import<__half>(void *, long long, const double *, cudaStream_t);

}  // namespace dps
