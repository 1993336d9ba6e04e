// noalloc.cu -- a variant of the linked-cell sort op that allocates nothing.
//
// dps_op_cell_sort takes its scratch (per-cell counts and fill counters,
// per-particle keys and permutation, scan partials) from the stream-ordered
// allocator.  Some callers cannot allow that: a host program that has handed
// the whole device to its own pool allocator, or a time-stepping loop that
// must not allocate (and possibly synchronise) once it is running.  For them
// dps_op_cell_sort_noalloc runs the same kernels on a fixed scratch array
// compiled into this library, of a stated maximum size.
#include <cuda_runtime.h>

#include <mutex>

#include "dps_internal.cuh"

namespace dps {
void launch_sort_count(const double *, const double *, const double *, long long, long long, const Geom &, int *, int *,
                       int *, cudaStream_t);
void launch_sort_scatter(const int *, long long, const int *, int *, int *, cudaStream_t);
void launch_sort_rank(const int *, const int *, long long, const int *, const int *, int *, cudaStream_t);
long long scan_scratch_words(long long);
void exclusive_scan(const int *, long long, int *, int *, cudaStream_t);
}  // namespace dps

using namespace dps;

namespace {
constexpr long long MAX_CELLS = DPS_NOALLOC_MAX_CELLS;
constexpr long long MAX_PARTICLES = DPS_NOALLOC_MAX_PARTICLES;
// counts + fill (cells), keys + tmp + perm (particles), scan partials, status
constexpr long long SCAN_WORDS = 2 * ((MAX_CELLS + 8191) / 8192) + 4;
constexpr long long WORDS = 2 * MAX_CELLS + 3 * MAX_PARTICLES + SCAN_WORDS + 8;
}  // namespace

// The scratch lives in every GPU that loads the library, for the life of the
// process.  In host code this name is only a host-side stand-in; the device
// address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) int g_sort_scratch[WORDS];

namespace {
std::mutex g_mu;
int *g_addr[128] = {nullptr};  // device address of the scratch, per device

// once per device, with that device current: look up the array's address
int scratch_for_current_device(int **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        cudaGetLastError();
        return DPS_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DPS_ERR_CUDA;
        }
        g_addr[dev] = (int *)p;
    }
    *out = g_addr[dev];
    return DPS_OK;
}
}  // namespace

extern "C" int dps_op_cell_sort_noalloc(const int n[3], const int periodic[3], int B, int64_t np, const double *x3,
                                        const int32_t *ids, int32_t *cell_start, int32_t *order, void *stream) {
    if (!n || !periodic || np < 0 || (np > 0 && (!x3 || !ids || !order)) || !cell_start) return DPS_ERR_ARG;
    if (B != 1) return DPS_ERR_ARG;
    Geom g{};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1) return DPS_ERR_ARG;
        g.n[a] = n[a];
        g.per[a] = periodic[a] ? 1 : 0;
        g.nb[a] = n[a];
    }
    g.B = 1;
    g.ncell = (long long)n[0] * n[1] * n[2];
    const long long N = g.ncell;
    if (N > MAX_CELLS || np > MAX_PARTICLES) return DPS_ERR_ARG;  // beyond the fixed scratch
    if (scan_scratch_words(N) > SCAN_WORDS) return DPS_ERR_ARG;
    int *scr = nullptr;
    int rc = scratch_for_current_device(&scr);
    if (rc != DPS_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int *count = scr, *fill = scr + MAX_CELLS, *key = fill + MAX_CELLS, *tmp = key + MAX_PARTICLES,
        *perm = tmp + MAX_PARTICLES, *scan = perm + MAX_PARTICLES, *status = scan + SCAN_WORDS;
    // the array keeps the previous call's contents: clear what must start at zero
    cudaMemsetAsync(count, 0, sizeof(int) * N, s);
    cudaMemsetAsync(status, 0, sizeof(int), s);
    launch_sort_count(x3, x3 + 1, x3 + 2, 3, np, g, count, key, status, s);
    exclusive_scan(count, N, cell_start, scan, s);
    cudaMemsetAsync(fill, 0, sizeof(int) * N, s);
    launch_sort_scatter(key, np, cell_start, fill, tmp, s);
    launch_sort_rank(key, ids, np, cell_start, tmp, np > 0 ? order : perm, s);
    // a host int is pageable memory: the copy allocates nothing and the
    // synchronisation that follows makes the status readable
    int st = 0;
    if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        cudaGetLastError();
        return DPS_ERR_CUDA;
    }
    return (st & ST_BAD_CELL) ? DPS_ERR_ARG : DPS_OK;
}
