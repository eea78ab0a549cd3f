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
// cell (u = H_z, v = -E).  One CTA updates one TILE_X x TILE_Y tile of one
// simulation for one full step:
//   first group (no sigma):  v <- v -/+ hf c_v d(u)          (sims with sigma on u)
//                            u <- u  +  hf c_u curl(v)       (sims with sigma on v)
//   second group (sigma):    u <- a u + bf c_u curl(v')      /  v <- a v -/+ bf c_v d(u')
// The first group is recomputed on a one-cell halo so that both half steps
// need a single pass over HBM: the fields ping-pong between two buffers.
#include <cuda_runtime.h>

#include "kernels.h"

namespace cas {

namespace {

template <typename R>
__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

template <typename R>
__global__ void __launch_bounds__(256)
k_step2d(const DevSim2D *__restrict__ sims, const DevTile *__restrict__ tiles,
         const int64_t *__restrict__ launch_base, int64_t launch_add)
{
    constexpr int SX = TILE_X + 2, SY = TILE_Y + 2;
    __shared__ R su[SY][SX], svx[SY][SX], svy[SY][SX];
    __shared__ uint8_t sm[SY][SX];
    __shared__ double red[8];

    const DevTile t = tiles[blockIdx.x];
    const DevSim2D &S = sims[t.sim];
    const int64_t n = *launch_base + launch_add - S.s0;
    if (n < 1 || n > S.T) return;

    const int nx = S.nx, ny = S.ny;
    const int w = min(TILE_X, nx - t.i0), h = min(TILE_Y, ny - t.j0);
    const size_t N = (size_t)nx * ny;
    const R *src = reinterpret_cast<const R *>(S.fields) + ((n - 1) & 1) * 3 * N;
    R *dst = reinterpret_cast<R *>(S.fields) + (n & 1) * 3 * N;
    const R *coef = reinterpret_cast<const R *>(S.coef);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;

    // tile plus a one-cell halo, periodic wrap (walls are masked sites)
    for (int ly = ty; ly < h + 2; ly += 8) {
        int gj = t.j0 + ly - 1;
        gj += gj < 0 ? ny : 0;
        gj -= gj >= ny ? ny : 0;
        for (int lx = tx; lx < w + 2; lx += 32) {
            int gi = t.i0 + lx - 1;
            gi += gi < 0 ? nx : 0;
            gi -= gi >= nx ? nx : 0;
            size_t g = (size_t)gj * nx + gi;
            su[ly][lx] = src[g];
            svx[ly][lx] = src[N + g];
            svy[ly][lx] = src[2 * N + g];
            sm[ly][lx] = S.mat[g];
        }
    }
    __syncthreads();

    const R hf = (R)(n == 1 ? 0.5 * S.hf : S.hf);
    const R a = (R)S.a, bf = (R)S.bf;
    if (S.second_u) {
        // first group v on [0, w] x [0, h] (vx needs lx >= 1, vy needs ly >= 1)
        for (int ly = ty; ly <= h; ly += 8)
            for (int lx = tx; lx <= w; lx += 32) {
                int m = sm[ly][lx];
                R uc = su[ly][lx];
                if (lx >= 1) svx[ly][lx] = svx[ly][lx] - hf * coef[3 * m + 1] * (su[ly + 1][lx] - uc);
                if (ly >= 1) svy[ly][lx] = svy[ly][lx] + hf * coef[3 * m + 2] * (su[ly][lx + 1] - uc);
            }
        __syncthreads();
        for (int ly = 1 + ty; ly <= h; ly += 8)
            for (int lx = 1 + tx; lx <= w; lx += 32) {
                int m = sm[ly][lx];
                R c = (svy[ly][lx] - svy[ly][lx - 1]) - (svx[ly][lx] - svx[ly - 1][lx]);
                su[ly][lx] = a * su[ly][lx] + bf * coef[3 * m] * c;
            }
    } else {
        // first group u on [1, w+1] x [1, h+1]
        for (int ly = 1 + ty; ly <= h + 1; ly += 8)
            for (int lx = 1 + tx; lx <= w + 1; lx += 32) {
                int m = sm[ly][lx];
                R c = (svy[ly][lx] - svy[ly][lx - 1]) - (svx[ly][lx] - svx[ly - 1][lx]);
                su[ly][lx] = su[ly][lx] + hf * coef[3 * m] * c;
            }
        __syncthreads();
        for (int ly = 1 + ty; ly <= h; ly += 8)
            for (int lx = 1 + tx; lx <= w; lx += 32) {
                int m = sm[ly][lx];
                R uc = su[ly][lx];
                svx[ly][lx] = a * svx[ly][lx] - bf * coef[3 * m + 1] * (su[ly + 1][lx] - uc);
                svy[ly][lx] = a * svy[ly][lx] + bf * coef[3 * m + 2] * (su[ly][lx + 1] - uc);
            }
    }
    __syncthreads();

    for (int ly = 1 + ty; ly <= h; ly += 8) {
        size_t g = (size_t)(t.j0 + ly - 1) * nx + t.i0;
        for (int lx = 1 + tx; lx <= w; lx += 32) {
            dst[g + lx - 1] = su[ly][lx];
            dst[N + g + lx - 1] = svx[ly][lx];
            dst[2 * N + g + lx - 1] = svy[ly][lx];
        }
    }

    if (t.ne > 0) {
        // surface functional of this tile's pixels, accumulated as w_n * s(n)
        double part = 0.0;
        for (int e = threadIdx.x; e < t.ne; e += blockDim.x) {
            DevEnt en = t.ents[e];
            int loc = en.loc & 0xffff, arr = en.loc >> 16;
            int ly = loc / TILE_X + 1, lx = loc % TILE_X + 1;
            R v = arr == 0 ? su[ly][lx] : (arr == 1 ? svx[ly][lx] : svy[ly][lx]);
            part += en.w * (double)v;
        }
        double s = block_sum<R>(part, red);
        if (threadIdx.x == 0) {
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
    if (fp64)
        k_step2d<double><<<ntiles, 256, 0, st>>>(sims, tiles, launch_base, launch_add);
    else
        k_step2d<float><<<ntiles, 256, 0, st>>>(sims, tiles, launch_base, launch_add);
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
