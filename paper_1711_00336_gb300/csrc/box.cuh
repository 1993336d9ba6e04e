// box.cuh -- the device box table.  Every kernel of the coupled step works on
// a list of tiles, each a contiguous range of cells or particles of one box;
// one launch therefore advances any number of boxes of different sizes (the
// single domain is a batch of one box).  Kernels read the box's geometry,
// physics and buffer pointers from the table; per-launch state common to all
// boxes (AA parity, which particle set is current) is passed by value.
#pragma once
#include "dps_internal.cuh"

namespace dps {

struct BoxDev {
    Geom g;
    Phys ph;
    int R;             // neighbour search radius (cells)
    // step state advanced on the device (current particle set, history
    // flags); the AA parity is common to the batch and passed per launch
    int parity, cur, have_uprev, have_usub;
    long long np, cap;
    // fluid
    void *pdf;
    void *eps, *fpf, *fam, *acc, *rho, *j, *uD, *uprev, *gradP, *DuDt;
    void *ire;         // 1/(rho eps_f) of the moments pass (eps_f of the step start)
    void *curl;        // curl of u_f for the lift force: the u_D planes, free after K2b
    // particles: two SoA sets and the DEM ping-pong planes
    double *pf[2];
    int *pi[2];
    double *xtmp;
    float4 *xf[2];     // float (x, y, z, d) of the current set / of the ping-pong planes
    float4 *vf[2];     // float (u, m) likewise
    float4 *of[2];     // float (omega, 0) likewise
    int *nlist;        // Verlet list, row by row: nlist[i*maxn + k]
    int *nlist_n;      // list length per particle
    int maxn;          // list capacity per particle
    // FP64 form: the list as unordered pairs, each evaluated once per
    // substep (Newton's third law).  Particle i owns the pairs with its
    // partners j > i: hn[i] of them, in ascending j, at slots hoff[i] ...
    // (hj: the partner of a slot; slots are allocated per block from *ptop).
    // rn[i] / rrow[i*maxn + r]: the slots of the pairs (k, i), k < i, in
    // ascending k.  pres[3 s ...]: force on the owner of slot s,
    // pres[3 (pcap + s) ...]: its n x F_t; pflag[s]: 1 the pair passed the
    // screen of this substep, 2 also n x F_t is nonzero (written).
    int *hj, *hoff, *hn, *rrow, *rn;
    double *pres;
    unsigned char *pflag;
    unsigned long long *ptop;
    long long pcap;    // slots
    int lowp;          // 1: low-precision form (FP32 coupling arithmetic)
    float *pwf;        // FP32 kernel weights [9][cap] (low-precision forms)
    float *f32p;       // FP32 copies of F_am (3 planes) and F_d (3 planes) [6][cap]
    double *psum;      // mixed-form DEM: pair sums of a substep, force and torque [6][cap]
    // linked cells
    int *cell_start, *count, *fill, *key, *tmp, *perm;
    int *scan_part;    // per scan tile partial sums of this box
    // status
    int *status;
    unsigned long long *counters;
};

struct Tile {
    int box;
    int first;         // index of this tile within its box (scan tiles)
    long long begin, end;
};

// iterate the tiles of a launch: one block per tile, blocks stride over tiles
#define DPS_FOR_TILES(tiles, ntiles, t) for (int t = blockIdx.x; t < (ntiles); t += gridDim.x)

}  // namespace dps
