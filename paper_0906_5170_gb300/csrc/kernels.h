// Device-side descriptors and kernel launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cas {

constexpr int TILE_X = 120;   // four warp strips of 30 interior columns
#ifndef CAS_TILE_Y
#define CAS_TILE_Y 32
#endif
constexpr int TILE_Y = CAS_TILE_Y;   // rows of a 2D TM/TE tile

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
    int nmat;              // rows of the coefficient table
    double a;              // (1 - sigma dt/2)/(1 + sigma dt/2)
    double bf;             // dt/(1 + sigma dt/2)/Delta
    double hf;             // dt/Delta (first group, halved on step 1)
};

struct DevEnt {
    int loc;               // (ly * TILE_X + lx) within the tile in bits 0..15, array in bits 16..
    int pad;
    double w;              // measurement weight
};

struct DevTile {
    int sim;
    int i0, j0;
    int ne;                // entries of the surface functional in this tile
    const DevEnt *ents;
    int z0, z1;            // column-march tiles of 3D runs: the planes [z0, z1) of the tile
};

struct DevSrc {
    int64_t idx;           // element index inside the sim's buffer 0 (array * N + site)
    double v;
};

// One simulation of the six-component kernel (k_z, Bloch, 3D; CPML; Lorentz).
struct DevSim6 {
    void *fields;          // E_x..E_z, H_x..H_z planes of N elements (re, im pairs when complex)
    void *psi;             // CPML auxiliary fields, 4 planes per PML axis over its two slabs
    void *lor;             // Lorentz planes, per pole q: P_q of E_x..E_z then P_q-prev (6 planes; NULL: non-dispersive)
    const uint8_t *mat;    // per-cell material id
    const void *coef;      // [id][6]: 1/eps at E_x..E_z sites, 1/mu at H_x..H_z sites (0 masks)
    const double *lorentz; // [id][pole][3][2]: (delta_eps, omega0) per E component
    const void *lorc;      // [id][pole][3][4] in the run's precision: cp = 2 - w0^2 dt^2, cpm = 1 - sigma dt/2,
                           // ce = delta_eps w0^2 dt^2 (0: no such pole), cd = 1/(1 + sigma dt/2)
    const void *pml;       // CPML profiles: axis a at pml_off[a]: [half][b, c, 1/kappa][n_a]
    const double *gw;
    double *acc;
    double *tail;
    int64_t s0;
    int64_t psi_off[3];    // element offset of axis a's psi planes
    int64_t slab[3];       // cells of one psi plane of axis a
    int64_t pml_off[3];
    int n[3];
    int pml_d[3];          // CPML thickness per axis (0: none)
    int dims, magnetic, T, tail_from;
    double a, bs;          // sigma group: decay and dt/(1 + sigma dt/2)
    double dt, dt_full, sigma, inv_dx;
    double kz;             // complex fields: d/dz = i kz (two-dimensional runs)
    double kzA, kzB;       // real fields: d/dz = kzA on {Ex, Ey, Hz}, kzB on {Ez, Hx, Hy}
    double bre[3], bim[3]; // Bloch factors exp(i k_a L_a)
    // march kernel (two-dimensional runs): elements from buffer 0 to buffer 1 of the
    // ping-pong fields, psi and Lorentz planes (step n reads buffer (n-1)&1, writes n&1)
    int64_t fhalf, psi_half, lor_half;
    int tile_rows;         // march kernel: rows per strip tile (<= MARCH_H_MAX)
    int npoles;            // Lorentz poles in use (present poles first at every site; 0: none)
};

struct DevEnt6 {
    int off;               // cell offset from the tile's first cell
    int arr;               // field component 0..5
    double wre, wim;
};

constexpr int TILE6 = 2048;   // cells per CTA of the six-component kernel (8 per thread)

struct DevTile6 {
    int sim;
    int count;             // cells in this tile (<= TILE6)
    int64_t cell0;
    int ne;
    int pad;
    const DevEnt6 *ents;
};

struct DevSrc6 {
    int64_t idx_re, idx_im;   // element indices in the sim's field block (idx_im < 0: real fields)
    double re, im;
};

void launch_full(int fp64, int cplx, int dims, const DevSim6 *sims, const DevTile6 *tiles, int ntiles,
                 const int64_t *launch_base, int64_t launch_add, int phase, cudaStream_t st);

// Six-component march of two-dimensional runs: one warp per strip tile of MARCH_W columns and
// MARCH_H rows, one full step per launch (both half steps), ping-pong buffers.  Tile entries:
// DevEnt with loc = ly * MARCH_W + lx in bits 0..15, the field component in bits 16..18 and
// bit 19 set for the weight of the imaginary part (complex fields).  variant: 1 = CPML planes
// present, + 2 = cells with one Lorentz pole at most, + 4 = cells with up to three poles.
constexpr int MARCH_VARIANTS = 6;
constexpr int MARCH_W = 30;
constexpr int MARCH_H = 32;       // default rows per strip tile
constexpr int MARCH_H_MAX = 64;   // largest tile height the planner builds (loc stays below 2^16)
void launch_march6(int fp64, int cplx, int variant, const DevSim6 *sims, const DevTile *tiles, int ntiles,
                   const int64_t *launch_base, int64_t launch_add, cudaStream_t st);
// Shared-memory limits of the staged march variants; once per device before the first launch
// (outside any stream capture).
cudaError_t march6_prepare();
// The same march on a cylindrical (r, z) lattice (x = r from the axis, y = z), fields ~ exp(i m phi)
// in the real-phase form (kzA, kzB = +-m), no CPML, no Lorentz media.
void launch_march6_cyl(int fp64, const DevSim6 *sims, const DevTile *tiles, int ntiles,
                       const int64_t *launch_base, int64_t launch_add, cudaStream_t st);
void launch_inject6(int fp64, void *fields, const DevSrc6 *src, int nsrc, cudaStream_t st);

// Six-component half step of three-dimensional runs by x lines: a tile is 32 x cells (i0) of
// LINES3 consecutive (y, z) lines from line j0 (line = z * ny + y), one warp per line at a time,
// in place (one buffer).  Tile entries: DevEnt with loc = (line - j0) * 32 + (x - i0) in bits
// 0..15, the component in bits 16..18, bit 19 for the weight of the imaginary part.
constexpr int LINES3 = 64;
void launch_line3(int fp64, int cplx, const DevSim6 *sims, const DevTile *tiles, int ntiles,
                  const int64_t *launch_base, int64_t launch_add, int phase, cudaStream_t st);

// Six-component leapfrog of three-dimensional runs by column tiles: one warp per tile of
// COL3_W x COL3_H cells in (x, y) over the planes [z0, z1), both half steps in one launch;
// fields, CPML psi and Lorentz P ping-pong between two buffers (step n reads buffer (n-1)&1,
// writes n&1) with the march's fhalf / psi_half / lor_half.  Tile entries: DevEnt with
// loc = (y - j0) * 32 + (x - i0) in bits 0..15, the component in bits 16..18, bit 19 for the
// weight of the imaginary part, and pad = z.  variant: as for the march (1 = CPML planes in the
// tile's halo-extended box, + 2 = cells with one Lorentz pole at most, + 4 = up to three poles),
// + MARCH_VARIANTS for magnetic (K) sources.  A run's planes are cut into chunks of at most
// COL3_ZMAX.
constexpr int COL3_W = 30;
constexpr int COL3_H = 8;
constexpr int COL3_ZMAX = 40;
constexpr int COL3_VARIANTS = 12;
void launch_col3(int fp64, int cplx, int variant, const DevSim6 *sims, const DevTile *tiles, int ntiles,
                 const int64_t *launch_base, int64_t launch_add, cudaStream_t st);

// Multi-step tiles of the 2D kernels: four warp strips of 32 - 2K interior columns (K time
// steps per launch, K halo lanes per side); the tile's pixel entries sorted by row, with
// rowptr[ly] .. rowptr[ly+1] per row.
constexpr int WARPS_K = 4;
constexpr int tile_xk(int k) { return WARPS_K * (32 - 2 * k); }
constexpr int TILE_X2 = tile_xk(2);   // 112
struct DevTile2 {
    int sim;
    int i0, j0;
    int ne;
    const DevEnt *ents;    // loc = ly * tile_xk(K) + lx
    const int *rowptr;     // TILE_Y + 1 offsets into ents
};

// Two leapfrog steps per launch: launch number L (from the simulation's start) advances
// steps 2L-1 and 2L (only 2L-1 when 2L > T), reading buffer (L-1)&1 and writing L&1.
void launch_step2d_t2(int fp64, const DevSim2D *sims, const DevTile2 *tiles, int ntiles,
                      const int64_t *launch_base, int64_t launch_add, cudaStream_t st);
// K = 3 leapfrog steps per launch: launch L advances steps 3L-2 .. 3L (those up to T), reading
// buffer (L-1)&1 and writing L&1; tiles tile_xk(3) = 104 columns wide.
void launch_step2d_t3(int fp64, const DevSim2D *sims, const DevTile2 *tiles, int ntiles,
                      const int64_t *launch_base, int64_t launch_add, cudaStream_t st);
// Two steps per launch on the cylindrical lattice (fields ~ exp(i m phi), real): launch L
// advances steps 2L-1 and 2L (2L-1 alone when 2L > T), reading buffer (L-1)&1, writing L&1;
// strips of MARCH_W2 columns, tiles of S.tile_rows rows with row-sorted entries (loc =
// ly * MARCH_W2 + lx, the component in bits 16..18) and tile_rows + 1 row offsets.
constexpr int MARCH_W2 = 28;
void launch_march6_cyl2(int fp64, const DevSim6 *sims, const DevTile2 *tiles, int ntiles,
                        const int64_t *launch_base, int64_t launch_add, cudaStream_t st);
// Two steps per launch of the Cartesian six-component march (k_z, Bloch, CPML, one Lorentz pole
// at most per cell), FP32: the tiles of launch_march6_cyl2, with bit 19 of an entry's loc set for
// the weight of the imaginary part (complex fields).  variant: 1 = CPML planes in the tile's
// two-step halo box, + 2 = dispersive cells there.
constexpr int MAR2_VARIANTS = 4;
void launch_march6_2(int cplx, int variant, const DevSim6 *sims, const DevTile2 *tiles, int ntiles,
                     const int64_t *launch_base, int64_t launch_add, cudaStream_t st);

void launch_step2d(int fp64, const DevSim2D *sims, const DevTile *tiles, int ntiles,
                   const int64_t *launch_base, int64_t launch_add, cudaStream_t st);
void launch_inject(int fp64, void *fields, const DevSrc *src, int nsrc, cudaStream_t st);
void launch_bump(int64_t *launch_base, int64_t by, cudaStream_t st);

}  // namespace cas
