// Two leapfrog steps per launch for the two-dimensional (TM-form) simulations.
//
// The same update as step2d.cu (McCauley et al., arXiv:0906.5170: harmonic
// source J = delta(t) f_n on S, Yee leapfrog in a medium of conductivity sigma,
// surface functional weighted by w_n = 2 dt Im g(-n dt), Eq. (1)), fused over
// two consecutive steps A = 2L-1 and B = 2L so that every field is read and
// written once per two steps.
//
// A warp owns a strip of STRIP2 = 28 interior columns plus two halo lanes on
// each side: after step A the outermost lane's values are stale, after step B
// the next one's, leaving lanes 2..29 exact.  It marches down the tile's rows;
// step B runs one row behind step A, which itself starts one row above the
// tile and ends one row below it.  Shuffles give the x neighbours, carried
// registers the y neighbours.  The measured (sigma) group of both steps is
// projected on the fly: the tile's pixel entries are sorted by row, and the
// lane holding an entry's column hands its value over by a shuffle.  Fields
// read buffer (L-1)&1 and write buffer L&1.
#include <cuda_runtime.h>

#include "kernels.h"

namespace cas {

namespace {

constexpr int STRIP2 = 28;
constexpr int WARPS2 = TILE_X2 / STRIP2;
static_assert(WARPS2 * STRIP2 == TILE_X2, "tile width must be a multiple of the strip");

// i in [-2n, 3n): rows up to two before and after the range, for any n >= 1
__device__ __forceinline__ int wrap2(int i, int n)
{
    i += i < 0 ? n : 0;
    i += i < 0 ? n : 0;
    i -= i >= n ? n : 0;
    return i >= n ? i - n : i;
}

template <typename R>
__device__ __forceinline__ R sdn(R v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename R>
__device__ __forceinline__ R sup(R v) { return __shfl_up_sync(0xffffffffu, v, 1); }

// Projection of one tile row: entries rowptr[ly] .. rowptr[ly+1]; a0/a1/a2 are this lane's
// values of u, vx, vy at the row; only entries in this warp's strip are taken.
template <typename R>
__device__ __forceinline__ double project_row(const DevTile2 &t, int ly, int strip_lo, int w, R a0, R a1, R a2)
{
    double part = 0.0;
    int e0 = t.rowptr[ly], e1 = t.rowptr[ly + 1];
    for (int base = e0; base < e1; base += 32) {
        int e = base + (int)(threadIdx.x & 31);
        int arr = 0, lx = -1;
        double wgt = 0.0;
        if (e < e1) {
            DevEnt en = t.ents[e];
            int loc = en.loc & 0xffff;
            arr = en.loc >> 16;
            lx = loc - ly * TILE_X2;
            wgt = en.w;
        }
        int off = lx - strip_lo;                   // interior column index within the strip
        bool mine = lx >= 0 && off >= 0 && off < w;
        int src = mine ? off + 2 : 0;
        R v0 = __shfl_sync(0xffffffffu, a0, src);
        R v1 = __shfl_sync(0xffffffffu, a1, src);
        R v2 = __shfl_sync(0xffffffffu, a2, src);
        if (mine) part += wgt * (double)(arr == 0 ? v0 : (arr == 1 ? v1 : v2));
    }
    return part;
}

template <typename R, int ROWS2, int MINB>
__global__ void __launch_bounds__(WARPS2 * 32, MINB)
k_step2d_t2(const DevSim2D *__restrict__ sims, const DevTile2 *__restrict__ tiles,
            const int64_t *__restrict__ launch_base, int64_t launch_add)
{
    __shared__ double redA[WARPS2], redB[WARPS2];
    const DevTile2 t = tiles[blockIdx.x];
    const DevSim2D &S = sims[t.sim];
    const int64_t L = *launch_base + launch_add - S.s0;
    const int64_t nA = 2 * L - 1;
    if (L < 1 || nA > S.T) return;
    const bool two = nA + 1 <= S.T;

    const int nx = S.nx, ny = S.ny;
    const unsigned N = (unsigned)nx * (unsigned)ny;   // 32-bit offsets: 3 N < 2^32 (checked by the planner)
    const R *__restrict__ su = reinterpret_cast<const R *>(S.fields) + ((L - 1) & 1) * 3 * N;
    const R *__restrict__ svx = su + N;
    const R *__restrict__ svy = su + 2 * N;
    R *__restrict__ du = reinterpret_cast<R *>(S.fields) + (L & 1) * 3 * N;
    R *__restrict__ dvx = du + N;
    R *__restrict__ dvy = du + 2 * N;
    const R *__restrict__ coef = reinterpret_cast<const R *>(S.coef);
    const uint8_t *__restrict__ mat = S.mat;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int strip_lo = warp * STRIP2;               // first interior column, relative to the tile
    const int i0 = t.i0 + strip_lo;
    const int w = min(STRIP2, nx - i0);
    const int h = min(TILE_Y, ny - t.j0);
    const int col = ((i0 - 2 + lane) % nx + nx) % nx;   // any nx >= 1
    const bool store = w > 0 && lane >= 2 && lane < w + 2;

    const R hfA = (R)(nA == 1 ? 0.5 * S.hf : S.hf);
    const R hfB = (R)S.hf;
    const R a = (R)S.a, bf = (R)S.bf;
    double pA = 0.0, pB = 0.0;

    if (w > 0) {
        const int j0 = t.j0;
        if (S.second_u) {
            // ---- sigma on u: v first ----
            // step A starts at row j0-1; its carried state needs row j0-2
            int jm2 = wrap2(j0 - 2, ny), jm1 = wrap2(j0 - 1, ny);
            unsigned g2 = (unsigned)(jm2 * nx + col), g1 = (unsigned)(jm1 * nx + col);
            R u_cur = su[g1];
            int m2 = mat[g2];
            R vxA_prev = svx[g2] - hfA * coef[3 * m2 + 1] * (u_cur - su[g2]);
            R uA_prev = 0, vyA_prev = 0, vxB_prev = 0;
            int m_prev = 0;
            // rows of step A: r = -1 .. h (j = j0 + r)
            for (int rb = -1; rb <= h; rb += ROWS2) {
                R un[ROWS2], vx[ROWS2], vy[ROWS2];
                int mt[ROWS2];
#pragma unroll
                for (int q = 0; q < ROWS2; ++q) {
                    int r = rb + q;
                    if (r <= h) {
                        int j = wrap2(j0 + r, ny);
                        unsigned g = (unsigned)(j * nx + col);
                        un[q] = su[(unsigned)(wrap2(j0 + r + 1, ny) * nx + col)];
                        vx[q] = svx[g];
                        vy[q] = svy[g];
                        mt[q] = mat[g];
                    }
                }
#pragma unroll
                for (int q = 0; q < ROWS2; ++q) {
                    int r = rb + q;
                    if (r > h) break;
                    int m = mt[q];
                    R cu = coef[3 * m], cvx = coef[3 * m + 1], cvy = coef[3 * m + 2];
                    // step A at row r
                    R vxA = vx[q] - hfA * cvx * (un[q] - u_cur);
                    R vyA = vy[q] + hfA * cvy * (sdn(u_cur) - u_cur);
                    R vyAl = sup(vyA);
                    R uA = a * u_cur + bf * cu * ((vyA - vyAl) - (vxA - vxA_prev));
                    if (!two) {
                        if (r >= 0 && r < h) {
                            if (store) {
                                unsigned g = (unsigned)((j0 + r) * nx + col);
                                du[g] = uA;
                                dvx[g] = vxA;
                                dvy[g] = vyA;
                            }
                            if (t.ne > 0) pA += project_row<R>(t, r, strip_lo, w, uA, vxA, vyA);
                        }
                    } else {
                        if (r >= 0 && r < h && t.ne > 0) pA += project_row<R>(t, r, strip_lo, w, uA, vxA, vyA);
                        if (r == 0) {
                            // new vx of step B one row above the tile
                            vxB_prev = vxA_prev - hfB * coef[3 * m_prev + 1] * (uA - uA_prev);
                        } else if (r >= 1) {
                            // step B at row r-1 (registers hold step A at rows r-1 and r)
                            int mp = m_prev;
                            R vxB = vxA_prev - hfB * coef[3 * mp + 1] * (uA - uA_prev);
                            R vyB = vyA_prev + hfB * coef[3 * mp + 2] * (sdn(uA_prev) - uA_prev);
                            R vyBl = sup(vyB);
                            R uB = a * uA_prev + bf * coef[3 * mp] * ((vyB - vyBl) - (vxB - vxB_prev));
                            if (store) {
                                unsigned g = (unsigned)((j0 + r - 1) * nx + col);
                                du[g] = uB;
                                dvx[g] = vxB;
                                dvy[g] = vyB;
                            }
                            if (t.ne > 0) pB += project_row<R>(t, r - 1, strip_lo, w, uB, vxB, vyB);
                            vxB_prev = vxB;
                        }
                    }
                    vxA_prev = vxA;
                    vyA_prev = vyA;
                    uA_prev = uA;
                    m_prev = m;
                    u_cur = un[q];
                }
            }
        } else {
            // ---- sigma on v: u first ----
            // step A: uA of rows j0-1 .. j0+h+1, vA of rows j0-1 .. j0+h; step B: uB of rows
            // j0 .. j0+h, vB of rows j0 .. j0+h-1
            int jm2 = wrap2(j0 - 2, ny), jm1 = wrap2(j0 - 1, ny);
            unsigned g2 = (unsigned)(jm2 * nx + col), g1 = (unsigned)(jm1 * nx + col);
            R vx_o = svx[g1], vy_o = svy[g1];        // old v of the current row (j0-1)
            int m_c = mat[g1];
            R uA_c = su[g1] + hfA * coef[3 * m_c] * ((vy_o - sup(vy_o)) - (vx_o - svx[g2]));
            R vxA_prev = 0, vyA_prev = 0, uB_prev = 0;
            int m_prev = 0;
            // iterate over row r = -1 .. h: load old row r+1, finish step A at row r
            for (int rb = -1; rb <= h; rb += ROWS2) {
                R un[ROWS2], vx[ROWS2], vy[ROWS2];
                int mt[ROWS2];
#pragma unroll
                for (int q = 0; q < ROWS2; ++q) {
                    int r = rb + q;
                    if (r <= h) {
                        unsigned g = (unsigned)(wrap2(j0 + r + 1, ny) * nx + col);
                        un[q] = su[g];
                        vx[q] = svx[g];
                        vy[q] = svy[g];
                        mt[q] = mat[g];
                    }
                }
#pragma unroll
                for (int q = 0; q < ROWS2; ++q) {
                    int r = rb + q;
                    if (r > h) break;
                    // step A: u of row r+1, then v of row r
                    R uA_n = un[q] + hfA * coef[3 * mt[q]] * ((vy[q] - sup(vy[q])) - (vx[q] - vx_o));
                    R vxA = a * vx_o - bf * coef[3 * m_c + 1] * (uA_n - uA_c);
                    R vyA = a * vy_o + bf * coef[3 * m_c + 2] * (sdn(uA_c) - uA_c);
                    if (!two) {
                        if (r >= 0 && r < h) {
                            if (store) {
                                unsigned g = (unsigned)((j0 + r) * nx + col);
                                du[g] = uA_c;
                                dvx[g] = vxA;
                                dvy[g] = vyA;
                            }
                            if (t.ne > 0) pA += project_row<R>(t, r, strip_lo, w, uA_c, vxA, vyA);
                        }
                    } else {
                        if (r >= 0 && r < h && t.ne > 0) pA += project_row<R>(t, r, strip_lo, w, uA_c, vxA, vyA);
                        if (r >= 0) {
                            // step B: u of row r (needs vA of rows r-1, r), then v of row r-1
                            R uB = uA_c + hfB * coef[3 * m_c] * ((vyA - sup(vyA)) - (vxA - vxA_prev));
                            if (r >= 1) {
                                int mp = m_prev;
                                R vxB = a * vxA_prev - bf * coef[3 * mp + 1] * (uB - uB_prev);
                                R vyB = a * vyA_prev + bf * coef[3 * mp + 2] * (sdn(uB_prev) - uB_prev);
                                if (store) {
                                    unsigned g = (unsigned)((j0 + r - 1) * nx + col);
                                    du[g] = uB_prev;
                                    dvx[g] = vxB;
                                    dvy[g] = vyB;
                                }
                                if (t.ne > 0) pB += project_row<R>(t, r - 1, strip_lo, w, uB_prev, vxB, vyB);
                            }
                            uB_prev = uB;
                        }
                    }
                    vxA_prev = vxA;
                    vyA_prev = vyA;
                    m_prev = m_c;
                    uA_c = uA_n;
                    vx_o = vx[q];
                    vy_o = vy[q];
                    m_c = mt[q];
                }
            }
        }
    }

    if (t.ne > 0) {
        for (int o = 16; o > 0; o >>= 1) {
            pA += __shfl_down_sync(0xffffffffu, pA, o);
            pB += __shfl_down_sync(0xffffffffu, pB, o);
        }
        if (lane == 0) {
            redA[warp] = pA;
            redB[warp] = pB;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double sA = 0.0, sB = 0.0;
            for (int q = 0; q < WARPS2; ++q) {
                sA += redA[q];
                sB += redB[q];
            }
            double c = S.gw[nA - 1] * sA + (two ? S.gw[nA] * sB : 0.0);
            atomicAdd(S.acc, c);
            double ct = (nA > S.tail_from ? S.gw[nA - 1] * sA : 0.0) + (two && nA + 1 > S.tail_from ? S.gw[nA] * sB : 0.0);
            if (ct != 0.0) atomicAdd(S.tail, ct);
        }
    }
}

}  // namespace

void launch_step2d_t2(int fp64, const DevSim2D *sims, const DevTile2 *tiles, int ntiles,
                      const int64_t *launch_base, int64_t launch_add, cudaStream_t st)
{
    if (ntiles <= 0) return;
    // three rows in flight per lane, six CTAs per SM: measured best among prefetch depths 2-6
    // and register caps for 4-8 resident CTAs
    if (fp64)
        k_step2d_t2<double, 3, 4><<<ntiles, WARPS2 * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
    else
        k_step2d_t2<float, 3, 6><<<ntiles, WARPS2 * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
}

}  // namespace cas
