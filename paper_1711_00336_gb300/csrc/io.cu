// io.cu -- host views of the device state and the global sums (S8).
//
//  - rest-state fill of the PDFs and constant fills of fields;
//  - export of fluid fields (rho, ubar, u_f, p, ...) as FP64 planes;
//  - particle export / import in insertion order (scatter / gather by id);
//  - deterministic FP64 sums: a fixed grid of blocks, each summing a fixed
//    strided subset and reducing it in a fixed tree, then one block summing
//    the partials in index order.
#include "box.cuh"
#include "lbm_dev.cuh"

namespace dps {

static int grid_for(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

template <typename ST>
__global__ void k_pdf_rest(ST *pdf, long long N) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if constexpr (sizeof(ST) == 8)
                Store<ST>::store(pdf + (long long)q * N + c, WQ(q));
            else  // deviation from the rest state is zero
                Store<ST>::store(pdf + (long long)q * N + c, 0.0f);
        }
    }
}

template <typename FT>
__global__ void k_fill(FT *p, long long n, double v) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = (FT)v;
}

template <typename FT>
__global__ void k_to_double(const FT *in, long long n, double *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

template <typename FT>
__global__ void k_from_double(const double *in, long long n, FT *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (FT)in[i];
}

// what = 0 rho, 1 ubar (3 planes), 2 u_f (3), 3 p, 4 f_ext (3)
template <typename ST, typename FT, int PAR>
__global__ void k_fluid_export(const ST *__restrict__ pdf, const FT *__restrict__ eps, const FT *__restrict__ fpf,
                               Geom g, double fbx, double fby, double fbz, int what, double *__restrict__ out) {
    const long long N = g.ncell;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        cell_coords(g, c, ix, iy, iz);
        NbDelta D = neighbour_deltas(g, ix, iy, iz);
        double f[Q];
        if constexpr (sizeof(ST) == 8) {
            load_pdfs<ST, double, PAR>(pdf, N, c, D, f);
        } else {
            float ff[Q];
            load_pdfs<ST, float, PAR>(pdf, N, c, D, ff);
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = (double)ff[q] + WQ(q);  // undo the shift in FP64
        }
        double rho, jx, jy, jz;
        moments(f, rho, jx, jy, jz);
        const double e = (double)eps[c];
        const double F[3] = {(double)fpf[c] + e * fbx, (double)fpf[N + c] + e * fby, (double)fpf[2 * N + c] + e * fbz};
        const double j[3] = {jx, jy, jz};
        if (what == 0) {
            out[c] = rho;
        } else if (what == 3) {
            out[c] = rho / 3.0 / e;
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                double ub = (j[a] + 0.5 * F[a]) / rho;
                out[a * N + c] = what == 1 ? ub : (what == 2 ? ub / e : F[a]);
            }
        }
    }
}

// ---- global sums ---------------------------------------------------------------
constexpr int RED_BLOCKS = 304;
constexpr int RED_THREADS = 256;
constexpr int FLUID_Q = 12;   // rho, j(3), ubar(3), u_f(3), min eps (as -max(-eps)), spare
constexpr int PART_Q = 6;     // m u (3), u (3)

template <int NQ>
__device__ __forceinline__ void block_sum_write(double v[NQ], double *partials, int mincomp) {
    __shared__ double sh[RED_THREADS / 32][NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = (k == mincomp) ? fmin(x, y) : x + y;
        }
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < NQ) {
        int k = threadIdx.x;
        double x = sh[0][k];
        for (int w = 1; w < RED_THREADS / 32; ++w) x = (k == mincomp) ? fmin(x, sh[w][k]) : x + sh[w][k];
        partials[blockIdx.x * NQ + k] = x;
    }
}

template <typename ST, typename FT, int PAR>
__global__ void __launch_bounds__(RED_THREADS) k_fluid_sums(const ST *__restrict__ pdf, const FT *__restrict__ eps,
                                                            const FT *__restrict__ fpf, Geom g, double fbx,
                                                            double fby, double fbz, double *partials) {
    const long long N = g.ncell;
    double v[FLUID_Q];
#pragma unroll
    for (int k = 0; k < FLUID_Q; ++k) v[k] = 0.0;
    v[10] = 1e300;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        cell_coords(g, c, ix, iy, iz);
        NbDelta D = neighbour_deltas(g, ix, iy, iz);
        double f[Q];
        if constexpr (sizeof(ST) == 8) {
            load_pdfs<ST, double, PAR>(pdf, N, c, D, f);
        } else {
            float ff[Q];
            load_pdfs<ST, float, PAR>(pdf, N, c, D, ff);
#pragma unroll
            for (int q = 0; q < Q; ++q) f[q] = (double)ff[q] + WQ(q);  // undo the shift in FP64
        }
        double rho, j[3];
        moments(f, rho, j[0], j[1], j[2]);
        const double e = (double)eps[c];
        const double fb[3] = {fbx, fby, fbz};
        v[0] += rho;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double F = (double)fpf[a * N + c] + e * fb[a];
            double ub = (j[a] + 0.5 * F) / rho;
            v[1 + a] += j[a];
            v[4 + a] += ub;
            v[7 + a] += ub / e;
        }
        v[10] = fmin(v[10], e);
    }
    block_sum_write<FLUID_Q>(v, partials, 10);
}

__global__ void __launch_bounds__(RED_THREADS) k_particle_sums(const double *__restrict__ xuw,
                                                               const double *__restrict__ pf, long long cap,
                                                               long long np, double *partials) {
    double v[PART_Q];
#pragma unroll
    for (int k = 0; k < PART_Q; ++k) v[k] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        double d = pf[PD * cap + i];
        double m = pf[PRHO * cap + i] * 3.14159265358979323846 / 6.0 * d * d * d;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double u = xuw[(3 + a) * cap + i];
            v[a] += m * u;
            v[3 + a] += u;
        }
    }
    block_sum_write<PART_Q>(v, partials, -1);
}

// sums the partials of each quantity in block order
__global__ void k_final_sums(const double *partials, int nblocks, int nq, int mincomp, double *out) {
    int k = threadIdx.x;
    if (k >= nq) return;
    double x = partials[k];
    for (int b = 1; b < nblocks; ++b) x = (k == mincomp) ? fmin(x, partials[b * nq + k]) : x + partials[b * nq + k];
    out[k] = x;
}

// ---- particles in insertion order -------------------------------------------------------
// out[3*id + a] = planes[(a)*cap + k] for the 3 planes starting at `plane`
// x, u, omega and the frozen force of a box in insertion order, one pass:
// out = [x(np,3) | u(np,3) | omega(np,3) | F(np,3)].  With a device table
// the current particle set is read from its entry k (no host round trip to
// learn it); else from pf / ids.
__global__ void k_particles_export4(const BoxDev *__restrict__ tab, int k, const double *__restrict__ pf0,
                                    const int *__restrict__ ids0, long long cap, long long np,
                                    double *__restrict__ out) {
    const double *pf = tab ? tab[k].pf[tab[k].cur] : pf0;
    const int *ids = tab ? tab[k].pi[tab[k].cur] + IID * cap : ids0;
    const int plane[4] = {PX, PU, POX, PFH0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        const long long id = ids[i];
#pragma unroll
        for (int gq = 0; gq < 4; ++gq)
#pragma unroll
            for (int a = 0; a < 3; ++a) out[gq * 3 * np + 3 * id + a] = pf[(plane[gq] + a) * cap + i];
    }
}

__global__ void k_particles_import(double *__restrict__ base, int plane, long long cap, long long np,
                                   const int *__restrict__ ids, const double *__restrict__ in) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < np; k += (long long)gridDim.x * blockDim.x) {
        long long id = ids[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) base[(plane + a) * cap + k] = in[3 * id + a];
    }
}

// ---- checkpoint layout of the PDFs -------------------------------------------------------
// Raw re-layout between the odd AA parity and the canonical layout (plane q
// of cell x holds f_q(x)), copying the stored bits (E: an unsigned type of
// the storage size, so no value is converted).  At odd parity f_q(x) sits in
// plane opp(q) of x - c_q, or in plane q of x itself when x - c_q lies beyond
// a wall (its bounced value).  TO_CANON = 1: odd -> canonical, 0: back.
template <typename E, int TO_CANON>
__global__ void k_pdf_relayout(const E *__restrict__ in, Geom g, E *__restrict__ out) {
    const long long N = g.ncell;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
         c += (long long)gridDim.x * blockDim.x) {
        int ix, iy, iz;
        cell_coords(g, c, ix, iy, iz);
        const NbDelta D = neighbour_deltas(g, ix, iy, iz);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            long long odd = (long long)q * N + c;
            if (q != 0) {
                const int dx = D.d[0][-CX(q) + 1], dy = D.d[1][-CY(q) + 1], dz = D.d[2][-CZ(q) + 1];
                if (dx != INV && dy != INV && dz != INV) odd = (long long)OPP(q) * N + c + dx + dy + dz;
            }
            const long long canon = (long long)q * N + c;
            if (TO_CANON)
                out[canon] = in[odd];
            else
                out[odd] = in[canon];
        }
    }
}

// ---- launchers ---------------------------------------------------------------------------
// elem: bytes per stored PDF value (8, 4 or 2); out of place
void launch_pdf_relayout(const void *in, const Geom &g, int elem, int to_canon, void *out, cudaStream_t s) {
    const int grid = grid_for(g.ncell, 256);
#define DPS_RELAYOUT(E)                                                                              \
    if (to_canon) k_pdf_relayout<E, 1><<<grid, 256, 0, s>>>((const E *)in, g, (E *)out);           \
    else k_pdf_relayout<E, 0><<<grid, 256, 0, s>>>((const E *)in, g, (E *)out);
    if (elem == 8) {
        DPS_RELAYOUT(unsigned long long)
    } else if (elem == 4) {
        DPS_RELAYOUT(unsigned int)
    } else {
        DPS_RELAYOUT(unsigned short)
    }
#undef DPS_RELAYOUT
}

template <typename ST>
void launch_pdf_rest(void *pdf, long long N, cudaStream_t s) {
    k_pdf_rest<ST><<<grid_for(N, 256), 256, 0, s>>>((ST *)pdf, N);
}
template <typename FT>
void launch_fill(void *p, long long n, double v, cudaStream_t s) {
    k_fill<FT><<<grid_for(n, 256), 256, 0, s>>>((FT *)p, n, v);
}
template <typename FT>
void launch_to_double(const void *in, long long n, double *out, cudaStream_t s) {
    k_to_double<FT><<<grid_for(n, 256), 256, 0, s>>>((const FT *)in, n, out);
}
template <typename FT>
void launch_from_double(const double *in, long long n, void *out, cudaStream_t s) {
    k_from_double<FT><<<grid_for(n, 256), 256, 0, s>>>(in, n, (FT *)out);
}
template <typename ST, typename FT>
void launch_fluid_export(const void *pdf, const void *eps, const void *fpf, const Geom &g, const double fb[3],
                         int parity, int what, double *out, cudaStream_t s) {
    if (parity == 0)
        k_fluid_export<ST, FT, 0><<<grid_for(g.ncell, 128), 128, 0, s>>>((const ST *)pdf, (const FT *)eps,
                                                                         (const FT *)fpf, g, fb[0], fb[1], fb[2],
                                                                         what, out);
    else
        k_fluid_export<ST, FT, 1><<<grid_for(g.ncell, 128), 128, 0, s>>>((const ST *)pdf, (const FT *)eps,
                                                                         (const FT *)fpf, g, fb[0], fb[1], fb[2],
                                                                         what, out);
}
// out[0..11]: fluid sums; partials needs RED_BLOCKS*FLUID_Q doubles
template <typename ST, typename FT>
void launch_fluid_sums(const void *pdf, const void *eps, const void *fpf, const Geom &g, const double fb[3],
                       int parity, double *partials, double *out, cudaStream_t s) {
    if (parity == 0)
        k_fluid_sums<ST, FT, 0><<<RED_BLOCKS, RED_THREADS, 0, s>>>((const ST *)pdf, (const FT *)eps, (const FT *)fpf, g,
                                                                  fb[0], fb[1], fb[2], partials);
    else
        k_fluid_sums<ST, FT, 1><<<RED_BLOCKS, RED_THREADS, 0, s>>>((const ST *)pdf, (const FT *)eps, (const FT *)fpf, g,
                                                                  fb[0], fb[1], fb[2], partials);
    k_final_sums<<<1, 32, 0, s>>>(partials, RED_BLOCKS, FLUID_Q, 10, out);
}
void launch_particle_sums(const double *xuw, const double *pf, long long cap, long long np, double *partials,
                          double *out, cudaStream_t s) {
    k_particle_sums<<<RED_BLOCKS, RED_THREADS, 0, s>>>(xuw, pf, cap, np, partials);
    k_final_sums<<<1, 32, 0, s>>>(partials, RED_BLOCKS, PART_Q, -1, out);
}
void launch_particles_export4(const BoxDev *tab, int k, const double *pf, const int *ids, long long cap, long long np,
                              double *out, cudaStream_t s) {
    if (np <= 0) return;
    k_particles_export4<<<grid_for(np, 256), 256, 0, s>>>(tab, k, pf, ids, cap, np, out);
}
void launch_particles_import(double *base, int plane, long long cap, long long np, const int *ids, const double *in,
                             cudaStream_t s) {
    if (np <= 0) return;
    k_particles_import<<<grid_for(np, 256), 256, 0, s>>>(base, plane, cap, np, ids, in);
}
long long reduce_partials_doubles() { return (long long)RED_BLOCKS * FLUID_Q; }

#define DPS_IO_INST_ST(ST, FT)                                                                                 \
    template void launch_pdf_rest<ST>(void *, long long, cudaStream_t);                                         \
    template void launch_fluid_export<ST, FT>(const void *, const void *, const void *, const Geom &,            \
                                              const double *, int, int, double *, cudaStream_t);                \
    template void launch_fluid_sums<ST, FT>(const void *, const void *, const void *, const Geom &,              \
                                            const double *, int, double *, double *, cudaStream_t);
DPS_IO_INST_ST(double, double)
DPS_IO_INST_ST(float, float)
DPS_IO_INST_ST(__half, float)
template void launch_fill<double>(void *, long long, double, cudaStream_t);
template void launch_fill<float>(void *, long long, double, cudaStream_t);
template void launch_to_double<double>(const void *, long long, double *, cudaStream_t);
template void launch_to_double<float>(const void *, long long, double *, cudaStream_t);
template void launch_from_double<double>(const double *, long long, void *, cudaStream_t);
template void launch_from_double<float>(const double *, long long, void *, cudaStream_t);

}  // namespace dps
