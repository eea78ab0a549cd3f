// Batched Yee leapfrog for two-dimensional (k_z = 0) simulations, fused with
// the surface projection and the g-weighted FP64 time integral.
//
// Method (arXiv:0906.5170): every simulation is the response to one harmonic
// source J = delta(t) f_n (or K) on the stress surface (Sec. II), evolved by the
// Yee scheme in a medium of uniform conductivity sigma (Sec. II); every step the
// surface functional s(n) (Sec. II, definition of Gamma) is weighted by
// w_n = 2 dt Im g(-n dt) (Eq. (1), Appendix A) and accumulated.
//
// Layout (TM form): u at (i, j), vx at (i, j+1/2), vy at (i+1/2, j) in the
// kernel's own lattice; TE runs the same update on the lattice shifted by half a
// cell (u = H_z, v = -E).  One step of one simulation:
//   sigma on u:  v  <- v -/+ hf c_v d(u)              then  u <- a u + bf c_u curl(v')
//   sigma on v:  u  <- u  +  hf c_u curl(v)           then  v <- a v -/+ bf c_v d(u')
// (hf is halved on step 1: the leapfrog starts with a half step.)
//
// Execution: a CTA owns a TILE_X x TILE_Y tile of one simulation.  Each warp
// owns a strip of STRIP columns plus one halo column on each side (lane 0 and
// lane STRIP+1) and marches down the tile's rows, keeping the stencil in
// registers: x neighbours come from warp shuffles, y neighbours from the row
// carried over from the previous iteration.  Rows are prefetched in batches of
// ROWS so that each lane has several independent loads in flight.  Both half
// steps therefore need one read and one write of every field: the fields
// ping-pong between two buffers (step parity).  After the march the tile's
// pixels are read back (the block's own writes) for the projection.
#include <cuda_runtime.h>

#include "kernels.h"

namespace cas {

namespace {

constexpr int STRIP = 30;                 // interior columns per warp
constexpr int WARPS = TILE_X / STRIP;     // warps per CTA
static_assert(WARPS * STRIP == TILE_X, "tile width must be a multiple of the strip");

// i in [-2n, 3n): rows up to two before and after the range, for any n >= 1
__device__ __forceinline__ int wrap(int i, int n)
{
    i += i < 0 ? n : 0;
    i += i < 0 ? n : 0;
    i -= i >= n ? n : 0;
    return i >= n ? i - n : i;
}

template <typename R>
__device__ __forceinline__ R shfl_dn(R v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename R>
__device__ __forceinline__ R shfl_up(R v) { return __shfl_up_sync(0xffffffffu, v, 1); }

// ROWS: rows prefetched per batch; MINB: resident CTAs per SM requested from the register allocator
template <typename R, int ROWS, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB)
k_step2d(const DevSim2D *__restrict__ sims, const DevTile *__restrict__ tiles,
         const int64_t *__restrict__ launch_base, int64_t launch_add)
{
    __shared__ double red[WARPS];
    const DevTile t = tiles[blockIdx.x];
    const DevSim2D &S = sims[t.sim];
    const int64_t n = *launch_base + launch_add - S.s0;
    if (n < 1 || n > S.T) return;

    const int nx = S.nx, ny = S.ny;
    const size_t N = (size_t)nx * ny;
    const R *__restrict__ su = reinterpret_cast<const R *>(S.fields) + ((n - 1) & 1) * 3 * N;
    const R *__restrict__ svx = su + N;
    const R *__restrict__ svy = su + 2 * N;
    R *__restrict__ du = reinterpret_cast<R *>(S.fields) + (n & 1) * 3 * N;
    R *__restrict__ dvx = du + N;
    R *__restrict__ dvy = du + 2 * N;
    const R *__restrict__ coef = reinterpret_cast<const R *>(S.coef);
    const uint8_t *__restrict__ mat = S.mat;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = t.i0 + warp * STRIP;               // first interior column of this strip
    const int w = min(STRIP, nx - i0);                // interior columns (may be <= 0)
    const int h = min(TILE_Y, ny - t.j0);
    const int col = ((i0 - 1 + lane) % nx + nx) % nx;  // this lane's column (lane 0: left halo), any nx >= 1
    const bool store = w > 0 && lane >= 1 && lane <= w;

    const R hf = (R)(n == 1 ? 0.5 * S.hf : S.hf);
    const R a = (R)S.a, bf = (R)S.bf;

    if (w > 0) {
        if (S.second_u) {
            // carried state: u of the current row, new vx of the previous row
            int jm = wrap(t.j0 - 1, ny);
            size_t gm = (size_t)jm * nx + col, g0 = (size_t)t.j0 * nx + col;
            R u_prev = su[gm];
            R u_cur = su[g0];
            int mm = mat[gm];
            R vxp = svx[gm] - hf * coef[3 * mm + 1] * (u_cur - u_prev);
            for (int jb = 0; jb < h; jb += ROWS) {
                R un[ROWS], vx[ROWS], vy[ROWS];
                int mt[ROWS];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    int j = t.j0 + jb + r;
                    if (jb + r < h) {
                        size_t g = (size_t)j * nx + col;
                        un[r] = su[(size_t)wrap(j + 1, ny) * nx + col];
                        vx[r] = svx[g];
                        vy[r] = svy[g];
                        mt[r] = mat[g];
                    }
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    if (jb + r >= h) break;
                    int m = mt[r];
                    R cu = coef[3 * m], cvx = coef[3 * m + 1], cvy = coef[3 * m + 2];
                    R vxn = vx[r] - hf * cvx * (un[r] - u_cur);
                    R u_right = shfl_dn(u_cur);
                    R vyn = vy[r] + hf * cvy * (u_right - u_cur);
                    R vy_left = shfl_up(vyn);
                    R unew = a * u_cur + bf * cu * ((vyn - vy_left) - (vxn - vxp));
                    if (store) {
                        size_t g = (size_t)(t.j0 + jb + r) * nx + col;
                        du[g] = unew;
                        dvx[g] = vxn;
                        dvy[g] = vyn;
                    }
                    vxp = vxn;
                    u_cur = un[r];
                }
            }
        } else {
            // carried state: old fields and new u of the current row
            int jm = wrap(t.j0 - 1, ny);
            size_t gm = (size_t)jm * nx + col, g0 = (size_t)t.j0 * nx + col;
            R vx_prev = svx[gm];
            R u_c = su[g0], vx_c = svx[g0], vy_c = svy[g0];
            int m_c = mat[g0];
            R vyl = shfl_up(vy_c);
            R up_c = u_c + hf * coef[3 * m_c] * ((vy_c - vyl) - (vx_c - vx_prev));
            for (int jb = 0; jb < h; jb += ROWS) {
                R un[ROWS], vx[ROWS], vy[ROWS];
                int mt[ROWS];
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    if (jb + r < h) {
                        size_t g = (size_t)wrap(t.j0 + jb + r + 1, ny) * nx + col;
                        un[r] = su[g];
                        vx[r] = svx[g];
                        vy[r] = svy[g];
                        mt[r] = mat[g];
                    }
                }
#pragma unroll
                for (int r = 0; r < ROWS; ++r) {
                    if (jb + r >= h) break;
                    // new u of the next row
                    R vyl_n = shfl_up(vy[r]);
                    R up_n = un[r] + hf * coef[3 * mt[r]] * ((vy[r] - vyl_n) - (vx[r] - vx_c));
                    // sigma half step of v on the current row
                    R cvx = coef[3 * m_c + 1], cvy = coef[3 * m_c + 2];
                    R up_right = shfl_dn(up_c);
                    R vxn = a * vx_c - bf * cvx * (up_n - up_c);
                    R vyn = a * vy_c + bf * cvy * (up_right - up_c);
                    if (store) {
                        size_t g = (size_t)(t.j0 + jb + r) * nx + col;
                        du[g] = up_c;
                        dvx[g] = vxn;
                        dvy[g] = vyn;
                    }
                    up_c = up_n;
                    vx_c = vx[r];
                    vy_c = vy[r];
                    m_c = mt[r];
                }
            }
        }
    }

    if (t.ne > 0) {
        // surface functional of this tile's pixels, accumulated as w_n * s(n)
        __syncthreads();                              // the block's field writes are visible
        double part = 0.0;
        for (int e = threadIdx.x; e < t.ne; e += blockDim.x) {
            DevEnt en = t.ents[e];
            int loc = en.loc & 0xffff, arr = en.loc >> 16;
            int ly = loc / TILE_X, lx = loc - ly * TILE_X;
            size_t g = (size_t)(t.j0 + ly) * nx + t.i0 + lx;
            R v = arr == 0 ? du[g] : (arr == 1 ? dvx[g] : dvy[g]);
            part += en.w * (double)v;
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < WARPS; ++q) s += red[q];
            double c = S.gw[n - 1] * s;
            atomicAdd(S.acc, c);
            if (n > S.tail_from) atomicAdd(S.tail, c);
        }
    }
}

template <typename R>
__global__ void k_inject(R *fields, const DevSrc *src, int nsrc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nsrc) fields[src[i].idx] = (R)src[i].v;
}

__global__ void k_bump(int64_t *base, int64_t by)
{
    *base += by;
}

}  // namespace

void launch_step2d(int fp64, const DevSim2D *sims, const DevTile *tiles, int ntiles,
                   const int64_t *launch_base, int64_t launch_add, cudaStream_t st)
{
    if (ntiles <= 0) return;
    // four rows in flight per lane; registers capped so that seven CTAs (28 warps) fit an SM
    // (measured best among prefetch depths 2-8 and caps of 40-106 registers)
    if (fp64)
        k_step2d<double, 4, 4><<<ntiles, WARPS * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
    else
        k_step2d<float, 4, 7><<<ntiles, WARPS * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
}

void launch_inject(int fp64, void *fields, const DevSrc *src, int nsrc, cudaStream_t st)
{
    if (nsrc <= 0) return;
    int b = (nsrc + 255) / 256;
    if (fp64)
        k_inject<double><<<b, 256, 0, st>>>(reinterpret_cast<double *>(fields), src, nsrc);
    else
        k_inject<float><<<b, 256, 0, st>>>(reinterpret_cast<float *>(fields), src, nsrc);
}

void launch_bump(int64_t *launch_base, int64_t by, cudaStream_t st)
{
    k_bump<<<1, 1, 0, st>>>(launch_base, by);
}

}  // namespace cas
