// Six-component leapfrog for two-dimensional cross-sections (d/dz -> i k_z,
// Sec. III B; Bloch-periodic cells, Sec. III D), both half steps in one pass.
//
// The update is the one of step6.cu (CPML of Sec. III B, Lorentz ADE of Eq. (9)
// continued onto the contour, surface functional weighted by w_n = 2 dt
// Im g(-n dt), Eq. (1)), organised like the TM-form kernel of step2d.cu: a CTA
// owns a TILE_X x TILE_Y tile of one simulation, each warp a strip of 30
// columns plus one halo lane per side, marching down the rows with x
// neighbours exchanged by shuffles and y neighbours carried in registers.
// Electric sources update H first (E of rows j and j+1 give H of row j), then
// E; magnetic sources update E one row ahead, then H.  Fields, CPML psi and
// Lorentz P ping-pong between two buffers by step parity, so that halo lanes
// recompute a neighbour's first half step from values nobody overwrites.
//
// Storage within one buffer is that of step6.cu: E_x..H_z planes of nx*ny
// elements (real and imaginary planes when complex), psi planes per PML axis
// over its two slabs, Lorentz P then P_prev per E component.
#include <cuda_runtime.h>

#include "kernels.h"

namespace cas {

namespace {

constexpr int STRIP6 = 30;
constexpr int WARPS6 = TILE_X / STRIP6;
static_assert(WARPS6 * STRIP6 == TILE_X, "tile width must be a multiple of the strip");

template <typename R, bool CPLX>
struct Z;

template <typename R>
struct Z<R, false> {
    R x;
    __device__ Z() : x(0) {}
    __device__ explicit Z(R a) : x(a) {}
    __device__ Z operator+(Z o) const { return Z(x + o.x); }
    __device__ Z operator-(Z o) const { return Z(x - o.x); }
    __device__ Z operator*(R s) const { return Z(x * s); }
    __device__ Z ph(R c, R) const { return Z(x * c); }                 // times (c + i s), s = 0 here
    __device__ Z dn() const { return Z(__shfl_down_sync(0xffffffffu, x, 1)); }
    __device__ Z up() const { return Z(__shfl_up_sync(0xffffffffu, x, 1)); }
};

template <typename R>
struct Z<R, true> {
    R x, y;
    __device__ Z() : x(0), y(0) {}
    __device__ Z(R a, R b) : x(a), y(b) {}
    __device__ Z operator+(Z o) const { return Z(x + o.x, y + o.y); }
    __device__ Z operator-(Z o) const { return Z(x - o.x, y - o.y); }
    __device__ Z operator*(R s) const { return Z(x * s, y * s); }
    __device__ Z ph(R c, R s) const { return Z(x * c - y * s, x * s + y * c); }
    __device__ Z ik(R k) const { return Z(-y * k, x * k); }            // i k F
    __device__ Z dn() const { return Z(__shfl_down_sync(0xffffffffu, x, 1), __shfl_down_sync(0xffffffffu, y, 1)); }
    __device__ Z up() const { return Z(__shfl_up_sync(0xffffffffu, x, 1), __shfl_up_sync(0xffffffffu, y, 1)); }
};

template <typename R, bool CPLX>
__device__ __forceinline__ Z<R, CPLX> ld(const R *p, int plane, size_t N, size_t g)
{
    if constexpr (CPLX) return Z<R, CPLX>(p[(size_t)(2 * plane) * N + g], p[(size_t)(2 * plane + 1) * N + g]);
    else return Z<R, CPLX>(p[(size_t)plane * N + g]);
}

template <typename R, bool CPLX>
__device__ __forceinline__ void st(R *p, int plane, size_t N, size_t g, Z<R, CPLX> v)
{
    if constexpr (CPLX) { p[(size_t)(2 * plane) * N + g] = v.x; p[(size_t)(2 * plane + 1) * N + g] = v.y; }
    else p[(size_t)plane * N + g] = v.x;
}

// One CPML-stretched difference: psi' = b psi + c d (written by the owner of the cell),
// returned value d / kappa + psi'.  prof holds b, c, 1/kappa, n entries each.
template <typename R, bool CPLX>
__device__ __forceinline__ Z<R, CPLX> cpml(Z<R, CPLX> d, const R *prof, int n, int pos, const R *pin, R *pout,
                                           int plane, size_t P, size_t gi, bool write)
{
    const R b = prof[pos], c = prof[n + pos], ik = prof[2 * n + pos];
    const Z<R, CPLX> p = ld<R, CPLX>(pin, plane, P, gi) * b + d * c;
    if (write) st<R, CPLX>(pout, plane, P, gi, p);
    return d * ik + p;
}

template <typename R, bool CPLX>
__global__ void __launch_bounds__(WARPS6 * 32)
k_march6(const DevSim6 *__restrict__ sims, const DevTile *__restrict__ tiles,
         const int64_t *__restrict__ launch_base, int64_t launch_add)
{
    using V = Z<R, CPLX>;
    __shared__ double red[WARPS6];
    const DevTile t = tiles[blockIdx.x];
    const DevSim6 &S = sims[t.sim];
    const int64_t n = *launch_base + launch_add - S.s0;
    if (n < 1 || n > S.T) return;
    const int nx = S.n[0], ny = S.n[1];
    const size_t N = (size_t)nx * ny;
    const int pin_par = (int)((n - 1) & 1), pout_par = (int)(n & 1);
    const R *fin = reinterpret_cast<const R *>(S.fields) + (size_t)pin_par * S.fhalf;
    R *fout = reinterpret_cast<R *>(S.fields) + (size_t)pout_par * S.fhalf;
    const R *coef = reinterpret_cast<const R *>(S.coef);
    const int dX = S.pml_d[0], dY = S.pml_d[1];
    const size_t PX = (size_t)S.slab[0], PY = (size_t)S.slab[1];
    const R *psi_in = S.psi ? reinterpret_cast<const R *>(S.psi) + (size_t)pin_par * S.psi_half : nullptr;
    R *psi_out = S.psi ? reinterpret_cast<R *>(S.psi) + (size_t)pout_par * S.psi_half : nullptr;
    const R *pxin = dX ? psi_in + S.psi_off[0] : nullptr;
    R *pxout = dX ? psi_out + S.psi_off[0] : nullptr;
    const R *pyin = dY ? psi_in + S.psi_off[1] : nullptr;
    R *pyout = dY ? psi_out + S.psi_off[1] : nullptr;
    const R *profx = dX ? reinterpret_cast<const R *>(S.pml) + S.pml_off[0] : nullptr;   // [half][b, c, 1/kappa][nx]
    const R *profy = dY ? reinterpret_cast<const R *>(S.pml) + S.pml_off[1] : nullptr;
    const R *lin = S.lor ? reinterpret_cast<const R *>(S.lor) + (size_t)pin_par * S.lor_half : nullptr;
    R *lout = S.lor ? reinterpret_cast<R *>(S.lor) + (size_t)pout_par * S.lor_half : nullptr;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i0 = t.i0 + warp * STRIP6;
    const int w = min(STRIP6, nx - i0);
    const int h = min(TILE_Y, ny - t.j0);
    const int col = ((i0 - 1 + lane) % nx + nx) % nx;     // lane 0: left halo, lane w + 1: right halo
    const bool own = w > 0 && lane >= 1 && lane <= w;
    const bool wrapR = col == nx - 1;                     // the right neighbour lies across the x wrap
    const bool wrapL = col == 0;                          // the left neighbour lies across the x wrap
    const bool inx = dX > 0 && (col < dX || col >= nx - dX);
    const int sx = col < dX ? col : col - (nx - 2 * dX);
    const R bxr = (R)S.bre[0], bxi = (R)S.bim[0], byr = (R)S.bre[1], byi = (R)S.bim[1];
    const R idx = (R)S.inv_dx;
    const R kA = (R)S.kzA, kB = (R)S.kzB, kc = (R)S.kz;
    const R a = (R)S.a, bs = (R)S.bs;
    const R hfirst = (R)(n == 1 ? 0.5 * S.dt : S.dt);
    const R dtl = (R)S.dt_full, sg = (R)S.sigma;

    // d/dz of a field of the set {Ex, Ey, Hz} (A) or {Ez, Hx, Hy} (B)
    auto dzA = [&](V f) -> V { if constexpr (CPLX) return f.ik(kc); else return f * kA; };
    auto dzB = [&](V f) -> V { if constexpr (CPLX) return f.ik(kc); else return f * kB; };
    auto right = [&](V f) -> V { V r = f.dn(); return wrapR ? r.ph(bxr, bxi) : r; };
    auto left = [&](V f) -> V { V l = f.up(); return wrapL ? l.ph(bxr, -bxi) : l; };
    auto rowp = [&](int j) { return j < 0 ? j + ny : (j >= ny ? j - ny : j); };

    // H at row j from E at rows j and j+1 (forward differences, half-site profiles)
    auto updH = [&](int j, int m, V ex, V ey, V ez, V exn, V ezn, V hx, V hy, V hz, R aa, R bb, bool wr,
                    V &hxo, V &hyo, V &hzo) {
        if (j + 1 >= ny) { exn = exn.ph(byr, byi); ezn = ezn.ph(byr, byi); }
        V dyEz = (ezn - ez) * idx, dyEx = (exn - ex) * idx;
        V dxEz = (right(ez) - ez) * idx, dxEy = (right(ey) - ey) * idx;
        if (inx) {
            const size_t gi = (size_t)j * (2 * dX) + sx;
            dxEz = cpml<R, CPLX>(dxEz, profx + 3 * nx, nx, col, pxin, pxout, 2, PX, gi, wr);   // H_y
            dxEy = cpml<R, CPLX>(dxEy, profx + 3 * nx, nx, col, pxin, pxout, 3, PX, gi, wr);   // H_z
        }
        if (dY > 0 && (j < dY || j >= ny - dY)) {
            const size_t gi = (size_t)(j < dY ? j : j - (ny - 2 * dY)) * nx + col;
            dyEx = cpml<R, CPLX>(dyEx, profy + 3 * ny, ny, j, pyin, pyout, 2, PY, gi, wr);   // H_z
            dyEz = cpml<R, CPLX>(dyEz, profy + 3 * ny, ny, j, pyin, pyout, 3, PY, gi, wr);   // H_x
        }
        const R *cm = coef + 6 * m;
        hxo = hx * aa - (dyEz - dzA(ey)) * (bb * cm[3]);
        hyo = hy * aa - (dzA(ex) - dxEz) * (bb * cm[4]);
        hzo = hz * aa - (dxEy - dyEx) * (bb * cm[5]);
    };
    // E at row j from H at rows j and j-1 (backward differences, integer-site profiles)
    auto updE = [&](int j, int m, V hx, V hy, V hz, V hxp, V hzp, V ex, V ey, V ez, R aa, R bb, bool wr,
                    bool first_e, size_t g, V &exo, V &eyo, V &ezo) {
        if (j - 1 < 0) { hxp = hxp.ph(byr, -byi); hzp = hzp.ph(byr, -byi); }
        V dyHz = (hz - hzp) * idx, dyHx = (hx - hxp) * idx;
        V dxHz = (hz - left(hz)) * idx, dxHy = (hy - left(hy)) * idx;
        if (inx) {
            const size_t gi = (size_t)j * (2 * dX) + sx;
            dxHz = cpml<R, CPLX>(dxHz, profx, nx, col, pxin, pxout, 0, PX, gi, wr);   // E_y
            dxHy = cpml<R, CPLX>(dxHy, profx, nx, col, pxin, pxout, 1, PX, gi, wr);   // E_z
        }
        if (dY > 0 && (j < dY || j >= ny - dY)) {
            const size_t gi = (size_t)(j < dY ? j : j - (ny - 2 * dY)) * nx + col;
            dyHx = cpml<R, CPLX>(dyHx, profy, ny, j, pyin, pyout, 0, PY, gi, wr);   // E_z
            dyHz = cpml<R, CPLX>(dyHz, profy, ny, j, pyin, pyout, 1, PY, gi, wr);   // E_x
        }
        const V c3[3] = {dyHz - dzB(hy), dzB(hx) - dxHz, dxHy - dyHx};
        const V e3[3] = {ex, ey, ez};
        V o3[3];
        const R *cm = coef + 6 * m;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const R de = lin ? (R)S.lorentz[6 * m + 2 * q] : (R)0;
            if (de != (R)0) {
                const R w0 = (R)S.lorentz[6 * m + 2 * q + 1];
                const R w2 = w0 * w0;
                const V p = ld<R, CPLX>(lin, q, N, g), pm = ld<R, CPLX>(lin, 3 + q, N, g);
                const V pn = first_e
                    ? (p * ((R)2 - w2 * dtl * dtl) + e3[q] * (de * w2 * dtl * dtl)) * (R)0.5
                    : (p * ((R)2 - w2 * dtl * dtl) - pm * ((R)1 - (R)0.5 * sg * dtl) + e3[q] * (de * w2 * dtl * dtl)) *
                          ((R)1 / ((R)1 + (R)0.5 * sg * dtl));
                if (wr) {
                    st<R, CPLX>(lout, q, N, g, pn);
                    st<R, CPLX>(lout, 3 + q, N, g, p);
                }
                o3[q] = e3[q] * aa + (p * aa - pn + c3[q] * bb) * cm[q];
            } else {
                o3[q] = e3[q] * aa + c3[q] * (bb * cm[q]);
            }
        }
        exo = o3[0];
        eyo = o3[1];
        ezo = o3[2];
    };
    auto put6 = [&](size_t g, V ex, V ey, V ez, V hx, V hy, V hz) {
        st<R, CPLX>(fout, 0, N, g, ex);
        st<R, CPLX>(fout, 1, N, g, ey);
        st<R, CPLX>(fout, 2, N, g, ez);
        st<R, CPLX>(fout, 3, N, g, hx);
        st<R, CPLX>(fout, 4, N, g, hy);
        st<R, CPLX>(fout, 5, N, g, hz);
    };

    if (w > 0) {
        const int j0 = t.j0;
        const int jm = rowp(j0 - 1);
        const size_t gm = (size_t)jm * nx + col, g0 = (size_t)j0 * nx + col;
        if (S.magnetic == 0) {
            // H (a = 1, b = h) then E (a, b_sigma).  Carried: E^n of row j, H^{n+1/2} of row j-1.
            V hxp, hyp, hzp;
            V ex = ld<R, CPLX>(fin, 0, N, g0), ey = ld<R, CPLX>(fin, 1, N, g0), ez = ld<R, CPLX>(fin, 2, N, g0);
            updH(jm, S.mat[gm], ld<R, CPLX>(fin, 0, N, gm), ld<R, CPLX>(fin, 1, N, gm), ld<R, CPLX>(fin, 2, N, gm), ex, ez,
                 ld<R, CPLX>(fin, 3, N, gm), ld<R, CPLX>(fin, 4, N, gm), ld<R, CPLX>(fin, 5, N, gm), (R)1, hfirst, false,
                 hxp, hyp, hzp);
            for (int r = 0; r < h; ++r) {
                const int j = j0 + r;
                const size_t g = (size_t)j * nx + col, gn = (size_t)rowp(j + 1) * nx + col;
                const V exn = ld<R, CPLX>(fin, 0, N, gn), eyn = ld<R, CPLX>(fin, 1, N, gn), ezn = ld<R, CPLX>(fin, 2, N, gn);
                const int m = S.mat[g];
                V hx, hy, hz;
                updH(j, m, ex, ey, ez, exn, ezn, ld<R, CPLX>(fin, 3, N, g), ld<R, CPLX>(fin, 4, N, g),
                     ld<R, CPLX>(fin, 5, N, g), (R)1, hfirst, own, hx, hy, hz);
                V ex1, ey1, ez1;
                updE(j, m, hx, hy, hz, hxp, hzp, ex, ey, ez, a, bs, own, n == 1, g, ex1, ey1, ez1);
                if (own) put6(g, ex1, ey1, ez1, hx, hy, hz);
                hxp = hx;
                hzp = hz;
                ex = exn;
                ey = eyn;
                ez = ezn;
            }
        } else {
            // E (a = 1, b = h) one row ahead, then H (a, b_sigma).  Carried: H^n of row j, E^{n+1} of row j.
            V hx = ld<R, CPLX>(fin, 3, N, g0), hy = ld<R, CPLX>(fin, 4, N, g0), hz = ld<R, CPLX>(fin, 5, N, g0);
            int m = S.mat[g0];
            V ex, ey, ez;
            updE(j0, m, hx, hy, hz, ld<R, CPLX>(fin, 3, N, gm), ld<R, CPLX>(fin, 5, N, gm), ld<R, CPLX>(fin, 0, N, g0),
                 ld<R, CPLX>(fin, 1, N, g0), ld<R, CPLX>(fin, 2, N, g0), (R)1, hfirst, own, false, g0, ex, ey, ez);
            for (int r = 0; r < h; ++r) {
                const int j = j0 + r, jn = rowp(j + 1);
                const size_t g = (size_t)j * nx + col, gn = (size_t)jn * nx + col;
                const V hxn = ld<R, CPLX>(fin, 3, N, gn), hyn = ld<R, CPLX>(fin, 4, N, gn), hzn = ld<R, CPLX>(fin, 5, N, gn);
                const int mn = S.mat[gn];
                V exn, eyn, ezn;   // E of row j + 1: psi and P written only for rows of this tile
                updE(jn, mn, hxn, hyn, hzn, hx, hz, ld<R, CPLX>(fin, 0, N, gn), ld<R, CPLX>(fin, 1, N, gn),
                     ld<R, CPLX>(fin, 2, N, gn), (R)1, hfirst, own && r + 1 < h, false, gn, exn, eyn, ezn);
                V hx1, hy1, hz1;
                updH(j, m, ex, ey, ez, exn, ezn, hx, hy, hz, a, bs, own, hx1, hy1, hz1);
                if (own) put6(g, ex, ey, ez, hx1, hy1, hz1);
                ex = exn;
                ey = eyn;
                ez = ezn;
                hx = hxn;
                hy = hyn;
                hz = hzn;
                m = mn;
            }
        }
    }

    if (t.ne > 0) {
        __syncthreads();   // the block's field writes are visible to the block
        double part = 0.0;
        for (int e = threadIdx.x; e < t.ne; e += blockDim.x) {
            const DevEnt en = t.ents[e];
            const int loc = en.loc & 0xffff, arr = (en.loc >> 16) & 7, im = (en.loc >> 19) & 1;
            const int ly = loc / TILE_X, lx = loc - ly * TILE_X;
            const size_t g = (size_t)(t.j0 + ly) * nx + t.i0 + lx;
            const size_t plane = CPLX ? (size_t)(2 * arr + im) : (size_t)arr;
            // Re(w v) = w_re v_re - w_im v_im: the imaginary weight enters with a minus sign
            part += (im ? -en.w : en.w) * (double)fout[plane * N + g];
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < WARPS6; ++q) s += red[q];
            const double c = S.gw[n - 1] * s;
            atomicAdd(S.acc, c);
            if (n > S.tail_from) atomicAdd(S.tail, c);
        }
    }
}

}  // namespace

void launch_march6(int fp64, int cplx, const DevSim6 *sims, const DevTile *tiles, int ntiles,
                   const int64_t *launch_base, int64_t launch_add, cudaStream_t st)
{
    if (ntiles <= 0) return;
    if (fp64) {
        if (cplx) k_march6<double, true><<<ntiles, WARPS6 * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
        else k_march6<double, false><<<ntiles, WARPS6 * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
    } else {
        if (cplx) k_march6<float, true><<<ntiles, WARPS6 * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
        else k_march6<float, false><<<ntiles, WARPS6 * 32, 0, st>>>(sims, tiles, launch_base, launch_add);
    }
}

}  // namespace cas
