// K leapfrog steps per launch for the two-dimensional (TM-form) simulations, K = 3.
//
// The update of step2d.cu and step2d_t2.cu (McCauley et al., arXiv:0906.5170: harmonic
// source J = delta(t) f_n on S, Yee leapfrog in a medium of conductivity sigma, surface
// functional weighted by w_n = 2 dt Im g(-n dt), Eq. (1)), fused over K consecutive steps
// n1 .. n1 + K - 1 so that every field is read and written once per K steps.
//
// A warp owns a strip of 32 - 2K interior columns plus K halo lanes on each side (after
// stage q the q outermost lanes of each side are stale).  It marches down the tile's rows
// with the stages pipelined: when stage 0 (the first step) is at row r, stage q is at row
// r - q, so stage q reads stage q - 1's newest row and the rows it kept in registers.  Stage
// q covers K - 1 - q rows above and below the tile (one row more for the field whose
// difference reaches back a row), so that the last stage is exact on the tile.  Shuffles
// give the x neighbours, carried registers the y neighbours.  Every stage's sigma group is
// projected on the fly (row-sorted entries, shuffle hand-over from the lane holding the
// entry's column).  Fields read buffer (L-1)&1 and write buffer L&1; a launch that holds
// fewer than K steps (the end of the run) stores every real stage as it passes a row, so the
// last real stage's values remain.
#include <cuda_runtime.h>

#include "kernels.h"

namespace cas {

namespace {

template <typename R>
__device__ __forceinline__ R kdn(R v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename R>
__device__ __forceinline__ R kup(R v) { return __shfl_up_sync(0xffffffffu, v, 1); }

template <bool B>
struct Flag {
    static constexpr bool value = B;
};

// any row index to [0, n)
__device__ __forceinline__ int wrapk(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// Projection of one tile row (entries rowptr[ly] .. rowptr[ly+1], loc = ly * TX + lx); a0/a1/a2
// are this lane's u, vx, vy at the row; lanes K .. K + w - 1 hold the strip's interior columns.
template <typename R, int TX, int K>
__device__ __forceinline__ double project_row_k(const DevTile2 &t, int ly, int strip_lo, int w, R a0, R a1, R a2)
{
    double part = 0.0;
    const int e0 = t.rowptr[ly], e1 = t.rowptr[ly + 1];
    for (int base = e0; base < e1; base += 32) {
        const int e = base + (int)(threadIdx.x & 31);
        int arr = 0, lx = -1;
        double wgt = 0.0;
        if (e < e1) {
            const DevEnt en = t.ents[e];
            arr = en.loc >> 16;
            lx = (en.loc & 0xffff) - ly * TX;
            wgt = en.w;
        }
        const int off = lx - strip_lo;
        const bool mine = lx >= 0 && off >= 0 && off < w;
        const int src = mine ? off + K : 0;
        const R v0 = __shfl_sync(0xffffffffu, a0, src);
        const R v1 = __shfl_sync(0xffffffffu, a1, src);
        const R v2 = __shfl_sync(0xffffffffu, a2, src);
        if (mine) part += wgt * (double)(arr == 0 ? v0 : (arr == 1 ? v1 : v2));
    }
    return part;
}

template <typename R, int K, int ROWS, int MINB>
__global__ void __launch_bounds__(WARPS_K * 32, MINB)
k_step2d_tk(const DevSim2D *__restrict__ sims, const DevTile2 *__restrict__ tiles,
            const int64_t *__restrict__ launch_base, int64_t launch_add)
{
    constexpr int STRIP = 32 - 2 * K;
    constexpr int TX = WARPS_K * STRIP;
    __shared__ double red[K][WARPS_K];
    const DevTile2 t = tiles[blockIdx.x];
    const DevSim2D &S = sims[t.sim];
    const int64_t L = *launch_base + launch_add - S.s0;
    const int64_t n1 = K * L - (K - 1);               // the step of stage 0
    if (L < 1 || n1 > S.T) return;
    const int ks = (int)(S.T - n1 + 1 < K ? S.T - n1 + 1 : K);   // stages that are real steps

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
    const int strip_lo = warp * STRIP;
    const int i0 = t.i0 + strip_lo;
    const int w = min(STRIP, nx - i0);
    const int h = min(TILE_Y, ny - t.j0);
    const int col = ((i0 - K + lane) % nx + nx) % nx;
    const bool store = w > 0 && lane >= K && lane < w + K;

    // the first group's step of stage 0 is a half step at n = 1 (the impulse sits at t = 0+)
    const R hf0 = (R)(n1 == 1 ? 0.5 * S.hf : S.hf), hf = (R)S.hf;
    const R a = (R)S.a, bf = (R)S.bf;
    // per material, the coefficients times their step factor: the first group's with hf, the
    // sigma group's with bf ((hf c) d is the (hf * c) * d of the unfused kernels bit for bit; at
    // stage 0 of the first launch the first group takes hf0 c = (hf c) / 2, exactly), padded to
    // four values so that one 16-byte shared load fetches a material's three coefficients
    struct alignas(4 * sizeof(R)) C4 {
        R c[4];
    };
    __shared__ C4 ctab4[256];
    R (*ctab)[4] = reinterpret_cast<R (*)[4]>(ctab4);
    for (int i = threadIdx.x; i < S.nmat; i += blockDim.x) {
        const R cu = coef[3 * i], cvx = coef[3 * i + 1], cvy = coef[3 * i + 2];
        ctab[i][0] = (S.second_u ? bf : hf) * cu;
        ctab[i][1] = (S.second_u ? hf : bf) * cvx;
        ctab[i][2] = (S.second_u ? hf : bf) * cvy;
    }
    __syncthreads();

    // FAST: a launch of K real steps that is not the run's first (the stored stage is K - 1 and no
    // coefficient is halved); a compile-time stored stage keeps the stage values in registers (a
    // run-time one made the compiler index them in local memory).  PROJ: the tile holds entries
    // of the surface functional.  The general path (the run's first and last launches) stores every
    // real stage as it passes a row and halves the first group's coefficients at stage 0 of step 1.
    auto march = [&](auto fast_tag, auto proj_tag) {
        constexpr bool FULL = decltype(fast_tag)::value;
        constexpr bool PROJ = decltype(proj_tag)::value;
        // the projection's partial sums live in the bodies that project (kept live through a body
        // that does not, they cost it registers)
        double p[K];
#pragma unroll
        for (int q = 0; q < K; ++q) p[q] = 0.0;
        if (w > 0) {
            const int j0 = t.j0;
            // rows of stage 0: r = -(K-1) .. h + K - 2 (relative to j0)
            const int r_first = -(K - 1), r_last = h + K - 2;
            if (S.second_u) {
                // ---- sigma on u: v first.  Stage q at row rho = r - q:
                //   vx_q(rho) = vx_{q-1}(rho) - h cvx (u_{q-1}(rho+1) - u_{q-1}(rho))
                //   vy_q(rho) = vy_{q-1}(rho) + h cvy (u_{q-1}(x+1, rho) - u_{q-1}(rho))
                //   u_q(rho)  = a u_{q-1}(rho) + bf cu ((vy_q(rho) - vy_q(x-1, rho)) - (vx_q(rho) - vx_q(rho-1)))
                // with q - 1 = -1 the buffer's values.  Carried: uo/vxo/vyo[q] = stage q at its previous row.
                R uo[K], vxo[K], vyo[K];
                int mh[K];   // material of row r - q
    #pragma unroll
                for (int q = 0; q < K; ++q) { uo[q] = (R)0; vxo[q] = (R)0; vyo[q] = (R)0; mh[q] = 0; }
                R u_cur;     // the buffer's u at row r
                {
                    const unsigned ga = (unsigned)(wrapk(j0 - K, ny) * nx + col), gb = (unsigned)(wrapk(j0 - K + 1, ny) * nx + col);
                    u_cur = su[gb];
                    vxo[0] = svx[ga] - hf0 * coef[3 * mat[ga] + 1] * (u_cur - su[ga]);   // vx of stage 0 at row -K
                }
                int jl = wrapk(j0 + r_first, ny);   // the next row to load, wrapped (advanced one row at a time)
                for (int rb = r_first; rb <= r_last; rb += ROWS) {
                    R un[ROWS], vxl[ROWS], vyl[ROWS];
                    int mt[ROWS];
    #pragma unroll
                    for (int i = 0; i < ROWS; ++i) {
                        const int r = rb + i;
                        if (r <= r_last) {
                            const int jn = jl + 1 == ny ? 0 : jl + 1;
                            const unsigned g = (unsigned)(jl * nx + col);
                            un[i] = su[(unsigned)(jn * nx + col)];
                            vxl[i] = svx[g];
                            vyl[i] = svy[g];
                            mt[i] = mat[g];
                            jl = jn;
                        }
                    }
    #pragma unroll
                    for (int i = 0; i < ROWS; ++i) {
                        const int r = rb + i;
                        if (r > r_last) break;
    #pragma unroll
                        for (int q = K - 1; q > 0; --q) mh[q] = mh[q - 1];
                        mh[0] = mt[i];
                        R un_[K], vxn[K], vyn[K];
    #pragma unroll
                        for (int q = 0; q < K; ++q) {
                            const int m = mh[q];
                            // hf c for the v group (hf0 c at stage 0 of the first launch), bf c_u
                            const R scale = !FULL && q == 0 && n1 == 1 ? (R)0.5 : (R)1;
                            const C4 cm = ctab4[m];
                            const R hcvx = cm.c[1] * scale, hcvy = cm.c[2] * scale, bcu = cm.c[0];
                            // inputs: stage q-1 at rows rho (carried) and rho + 1 (this iteration)
                            const R uin = q == 0 ? u_cur : uo[q - 1];
                            const R uin1 = q == 0 ? un[i] : un_[q - 1];
                            const R vxin = q == 0 ? vxl[i] : vxo[q - 1];
                            const R vyin = q == 0 ? vyl[i] : vyo[q - 1];
                            vxn[q] = vxin - hcvx * (uin1 - uin);
                            vyn[q] = vyin + hcvy * (kdn(uin) - uin);
                            un_[q] = a * uin + bcu * ((vyn[q] - kup(vyn[q])) - (vxn[q] - vxo[q]));
                            const int rho = r - q;
                            if ((FULL || q < ks) && rho >= 0 && rho < h) {
                                if ((FULL ? q == K - 1 : q < ks) && store) {
                                    const unsigned g = (unsigned)((j0 + rho) * nx + col);
                                    du[g] = un_[q];
                                    dvx[g] = vxn[q];
                                    dvy[g] = vyn[q];
                                }
                                if (PROJ && t.ne > 0) p[q] += project_row_k<R, TX, K>(t, rho, strip_lo, w, un_[q], vxn[q], vyn[q]);
                            }
                        }
    #pragma unroll
                        for (int q = 0; q < K; ++q) {
                            uo[q] = un_[q];
                            vxo[q] = vxn[q];
                            vyo[q] = vyn[q];
                        }
                        u_cur = un[i];
                    }
                }
            } else {
                // ---- sigma on v: u first.  Stage q at iteration r: u at row r - q + 1, then v at row r - q:
                //   u_q(rho+1) = u_{q-1}(rho+1) + h cu ((vy_{q-1}(rho+1) - vy_{q-1}(x-1, rho+1)) - (vx_{q-1}(rho+1) - vx_{q-1}(rho)))
                //   vx_q(rho) = a vx_{q-1}(rho) - bf cvx (u_q(rho+1) - u_q(rho))
                //   vy_q(rho) = a vy_{q-1}(rho) + bf cvy (u_q(x+1, rho) - u_q(rho))
                // Carried: uc[q] = u_q at row r - q (the row its v is made for), vxo/vyo[q] = v_q at row r - q - 1.
                R uc[K], vxo[K], vyo[K];
                int mh[K + 1];   // material of row r + 1 - i
    #pragma unroll
                for (int q = 0; q < K; ++q) { uc[q] = (R)0; vxo[q] = (R)0; vyo[q] = (R)0; }
    #pragma unroll
                for (int q = 0; q <= K; ++q) mh[q] = 0;
                R vx_c, vy_c;   // the buffer's v at row r
                {
                    const unsigned ga = (unsigned)(wrapk(j0 - K, ny) * nx + col), gb = (unsigned)(wrapk(j0 - K + 1, ny) * nx + col);
                    vx_c = svx[gb];
                    vy_c = svy[gb];
                    const int mb = mat[gb];
                    mh[0] = mb;
                    uc[0] = su[gb] + hf0 * coef[3 * mb] * ((vy_c - kup(vy_c)) - (vx_c - svx[ga]));   // u of stage 0 at row -(K-1)
                }
                int jl = wrapk(j0 + r_first + 1, ny);   // the next row to load, wrapped
                for (int rb = r_first; rb <= r_last; rb += ROWS) {
                    R un[ROWS], vxl[ROWS], vyl[ROWS];
                    int mt[ROWS];
    #pragma unroll
                    for (int i = 0; i < ROWS; ++i) {
                        const int r = rb + i;
                        if (r <= r_last) {
                            const unsigned g = (unsigned)(jl * nx + col);
                            jl = jl + 1 == ny ? 0 : jl + 1;
                            un[i] = su[g];
                            vxl[i] = svx[g];
                            vyl[i] = svy[g];
                            mt[i] = mat[g];
                        }
                    }
    #pragma unroll
                    for (int i = 0; i < ROWS; ++i) {
                        const int r = rb + i;
                        if (r > r_last) break;
    #pragma unroll
                        for (int q = K; q > 0; --q) mh[q] = mh[q - 1];
                        mh[0] = mt[i];
                        R unw[K], vxn[K], vyn[K];
    #pragma unroll
                        for (int q = 0; q < K; ++q) {
                            const R scale = !FULL && q == 0 && n1 == 1 ? (R)0.5 : (R)1;
                            // u at row r - q + 1 from stage q-1 at that row (u carried, v of this iteration) and v at row r - q
                            const R uin = q == 0 ? un[i] : uc[q - 1];
                            const R vxa = q == 0 ? vxl[i] : vxn[q - 1];
                            const R vya = q == 0 ? vyl[i] : vyn[q - 1];
                            const R vxb = q == 0 ? vx_c : vxo[q - 1];
                            const R vyb = q == 0 ? vy_c : vyo[q - 1];
                            const int mu = mh[q], mv = mh[q + 1];
                            const C4 cmv = ctab4[mv];
                            unw[q] = uin + ctab4[mu].c[0] * scale * ((vya - kup(vya)) - (vxa - vxb));
                            vxn[q] = a * vxb - cmv.c[1] * (unw[q] - uc[q]);
                            vyn[q] = a * vyb + cmv.c[2] * (kdn(uc[q]) - uc[q]);
                            const int rho = r - q;
                            if ((FULL || q < ks) && rho >= 0 && rho < h) {
                                if ((FULL ? q == K - 1 : q < ks) && store) {
                                    const unsigned g = (unsigned)((j0 + rho) * nx + col);
                                    du[g] = uc[q];
                                    dvx[g] = vxn[q];
                                    dvy[g] = vyn[q];
                                }
                                if (PROJ && t.ne > 0) p[q] += project_row_k<R, TX, K>(t, rho, strip_lo, w, uc[q], vxn[q], vyn[q]);
                            }
                        }
    #pragma unroll
                        for (int q = 0; q < K; ++q) {
                            uc[q] = unw[q];
                            vxo[q] = vxn[q];
                            vyo[q] = vyn[q];
                        }
                        vx_c = vxl[i];
                        vy_c = vyl[i];
                    }
                }
            }
        }
        // every warp of the CTA (one tile) runs the same body, so the barrier is uniform
        if (PROJ && t.ne > 0) {
    #pragma unroll
            for (int q = 0; q < K; ++q) {
                for (int o = 16; o > 0; o >>= 1) p[q] += __shfl_down_sync(0xffffffffu, p[q], o);
                if (lane == 0) red[q][warp] = p[q];
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double c = 0.0, ct = 0.0;
                for (int q = 0; q < ks; ++q) {
                    double s = 0.0;
                    for (int v = 0; v < WARPS_K; ++v) s += red[q][v];
                    const double cq = S.gw[n1 - 1 + q] * s;
                    c += cq;
                    if (n1 + q > S.tail_from) ct += cq;
                }
                atomicAdd(S.acc, c);
                if (ct != 0.0) atomicAdd(S.tail, ct);
            }
        }
    };
    if (ks == K && n1 != 1) {
        if (t.ne > 0) march(Flag<true>{}, Flag<true>{});
        else march(Flag<true>{}, Flag<false>{});
    } else {
        march(Flag<false>{}, Flag<true>{});
    }

}

}  // namespace

// FP32: rows whose loads are in flight together, resident CTAs per SM asked of the register allocator
#ifndef STEP2D_TK_ROWS
#define STEP2D_TK_ROWS 3
#endif
#ifndef STEP2D_TK_MINB
#define STEP2D_TK_MINB 8
#endif

void launch_step2d_t3(int fp64, const DevSim2D *sims, const DevTile2 *tiles, int ntiles,
                      const int64_t *launch_base, int64_t launch_add, cudaStream_t st)
{
    if (ntiles <= 0) return;
    if (fp64)
        k_step2d_tk<double, 3, 3, 4><<<ntiles, WARPS_K * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
    else
        k_step2d_tk<float, 3, STEP2D_TK_ROWS, STEP2D_TK_MINB><<<ntiles, WARPS_K * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
}

}  // namespace cas
