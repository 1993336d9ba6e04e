// scan.cu -- exclusive prefix sum of int32 counts (the cell_start array of the
// linked-cell sort).  Reduce-then-scan over tiles of 8192 values: one pass
// writes tile totals, the totals are scanned (recursively), a second pass
// scans each tile and adds its offset.  Integer sums are exact, so the result
// does not depend on the launch shape.
#include "box.cuh"

namespace dps {

constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int warp_incl_scan(int v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= o) v += t;
    }
    return v;
}

// block-wide exclusive scan of one value per thread; total = block sum
__device__ __forceinline__ int block_excl_scan(int v, int &total) {
    constexpr int NW = SCAN_THREADS / 32;
    __shared__ int wsum[NW];
    __shared__ int s_total;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int t = lane < NW ? wsum[lane] : 0;
        int ti = warp_incl_scan(t);
        if (lane < NW) wsum[lane] = ti - t;  // exclusive prefix of the warp totals
        if (lane == NW - 1) s_total = ti;
    }
    __syncthreads();
    int res = wsum[wid] + inc - v;
    total = s_total;
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_tile_sums(const int *__restrict__ in, long long n,
                                                             int *__restrict__ sums) {
    long long base = (long long)blockIdx.x * SCAN_TILE;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long i = base + (long long)k * SCAN_THREADS + threadIdx.x;
        if (i < n) s += in[i];
    }
    // block reduction
    __shared__ int red[SCAN_THREADS / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = red[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) sums[blockIdx.x] = t;
    }
}

// exclusive scan of a tile with each thread owning SCAN_ITEMS consecutive values
__global__ void __launch_bounds__(SCAN_THREADS) k_tile_scan(const int *__restrict__ in, long long n,
                                                             const int *__restrict__ offsets,
                                                             int *__restrict__ out, int write_total) {
    long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int total;
    int ex = block_excl_scan(s, total);
    int off = (offsets ? offsets[blockIdx.x] : 0) + ex;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long i = base + k;
        if (i < n) out[i] = off;
        off += v[k];
    }
    // out[n] = grand total, written by the thread that owns the last value
    if (write_total && base <= n - 1 && n - 1 < base + SCAN_ITEMS) out[n] = off;
}

// number of int32 scratch words the scan of n values needs
long long scan_scratch_words(long long n) {
    long long words = 0;
    while (n > SCAN_TILE) {  // per level: tile sums (t) and their scan (t+1)
        long long t = (n + SCAN_TILE - 1) / SCAN_TILE;
        words += 2 * t + 2;
        n = t;
    }
    return words + 1;
}

// out[0..n] = exclusive prefix of in[0..n), out[n] = total.  in and out may
// not alias.  scratch holds scan_scratch_words(n) ints.
void exclusive_scan(const int *in, long long n, int *out, int *scratch, cudaStream_t s) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(int), s);
        return;
    }
    long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        k_tile_scan<<<1, SCAN_THREADS, 0, s>>>(in, n, nullptr, out, 1);
        return;
    }
    int *sums = scratch;                      // tiles values
    int *sums_scanned = scratch + tiles + 1;  // tiles+1 values, then deeper levels
    k_tile_sums<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums);
    exclusive_scan(sums, tiles, sums_scanned, sums_scanned + tiles + 1, s);
    k_tile_scan<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums_scanned, out, 1);
}

// ---- batched scan over the box table ----------------------------------------------
// Scan tiles are SCAN_TILE cells of one box; Tile::first is the tile's index
// inside its box.  Pass 1 writes each tile's count total, pass 2 scans the
// totals of every box (one block per box), pass 3 scans inside the tiles,
// writes cell_start (and its final entry, the particle count) and clears the
// fill counters used by the scatter.
__global__ void __launch_bounds__(SCAN_THREADS) k_bscan_sums(const BoxDev *__restrict__ boxes,
                                                              const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        int s = 0;
        for (long long i = tl.begin + threadIdx.x; i < tl.end; i += SCAN_THREADS) s += B.count[i];
        __shared__ int red[SCAN_THREADS / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            int v = red[threadIdx.x];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) B.scan_part[tl.first] = v;
        }
        __syncthreads();
    }
}

// one block per box: exclusive scan of its tile totals, in place
__global__ void __launch_bounds__(SCAN_THREADS) k_bscan_parts(const BoxDev *__restrict__ boxes, int nboxes) {
    for (int b = blockIdx.x; b < nboxes; b += gridDim.x) {
        const BoxDev &B = boxes[b];
        const long long nt = (B.g.ncell + SCAN_TILE - 1) / SCAN_TILE;
        int carry = 0;
        for (long long base = 0; base < nt; base += SCAN_THREADS) {
            long long i = base + threadIdx.x;
            int v = i < nt ? B.scan_part[i] : 0;
            int total;
            int ex = block_excl_scan(v, total);
            if (i < nt) B.scan_part[i] = carry + ex;
            carry += total;
        }
    }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_bscan_tiles(const BoxDev *__restrict__ boxes,
                                                               const Tile *__restrict__ tiles, int ntiles) {
    DPS_FOR_TILES(tiles, ntiles, t) {
        const Tile tl = tiles[t];
        const BoxDev &B = boxes[tl.box];
        const long long n = B.g.ncell;
        const long long base = tl.begin + (long long)threadIdx.x * SCAN_ITEMS;
        int v[SCAN_ITEMS];
        int s = 0;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            long long i = base + k;
            v[k] = i < tl.end ? B.count[i] : 0;
            s += v[k];
        }
        int total;
        int ex = block_excl_scan(s, total);
        int off = B.scan_part[tl.first] + ex;
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS; ++k) {
            long long i = base + k;
            if (i < tl.end) {
                B.cell_start[i] = off;
                B.fill[i] = 0;
            }
            off += v[k];
        }
        if (base <= n - 1 && n - 1 < base + SCAN_ITEMS && n - 1 < tl.end) B.cell_start[n] = off;
    }
}

void launch_bscan(const BoxDev *boxes, int nboxes, const Tile *scan_tiles, int ntiles, cudaStream_t s) {
    int grid = ntiles < 152 * 2 ? ntiles : 152 * 2;
    k_bscan_sums<<<grid, SCAN_THREADS, 0, s>>>(boxes, scan_tiles, ntiles);
    k_bscan_parts<<<nboxes, SCAN_THREADS, 0, s>>>(boxes, nboxes);
    k_bscan_tiles<<<grid, SCAN_THREADS, 0, s>>>(boxes, scan_tiles, ntiles);
}
int scan_tile_cells() { return SCAN_TILE; }

}  // namespace dps
