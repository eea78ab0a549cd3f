// Device-side descriptors and kernel launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cas {

constexpr int TILE_X = 32;
constexpr int TILE_Y = 32;

// One simulation of a TM-form 2D kernel (TM, or TE on the dual lattice).
// Fields: two buffers (ping-pong by step parity) of three arrays u, vx, vy,
// each nx*ny elements, x fastest.
struct DevSim2D {
    void *fields;          // 6 * nx * ny elements of the run's precision
    const uint8_t *mat;    // per-cell material id
    const void *coef;      // [id][3]: 1/eps or 1/mu for u, vx, vy (0 masks PEC/PMC)
    const double *gw;      // g weights w_n, n = 1..T
    double *acc;           // FP64 accumulator of sum_n w_n s(n)
    double *tail;          // same, restricted to n > tail_from
    int64_t s0;            // launch index of step 0: step n runs at launch s0 + n
    int nx, ny;
    int T;
    int tail_from;
    int second_u;          // 1: the sigma / measured group is u; 0: it is (vx, vy)
    int pad;
    double a;              // (1 - sigma dt/2)/(1 + sigma dt/2)
    double bf;             // dt/(1 + sigma dt/2)/Delta
    double hf;             // dt/Delta (first group, halved on step 1)
};

struct DevEnt {
    int loc;               // (ly * TILE_X + lx) within the tile, array in bits 16..
    int pad;
    double w;              // measurement weight
};

struct DevTile {
    int sim;
    int i0, j0;
    int ne;                // entries of the surface functional in this tile
    const DevEnt *ents;
};

struct DevSrc {
    int64_t idx;           // element index inside the sim's buffer 0 (array * N + site)
    double v;
};

void launch_step2d(int fp64, const DevSim2D *sims, const DevTile *tiles, int ntiles,
                   const int64_t *launch_base, int64_t launch_add, cudaStream_t st);
void launch_inject(int fp64, void *fields, const DevSrc *src, int nsrc, cudaStream_t st);
void launch_bump(int64_t *launch_base, int64_t by, cudaStream_t st);

}  // namespace cas
