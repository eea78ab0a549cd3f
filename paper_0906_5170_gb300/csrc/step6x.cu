// Six-component Yee half steps of three-dimensional simulations (Sec. III E),
// with CPML (Sec. III B), Bloch-periodic walls (Sec. III D) and Lorentz media of
// up to three undamped poles on the contour (Eq. (9); the silica model of
// Sec. III D), organised by x lines: every warp
// takes 32 consecutive x cells of one (y, z) line, so coordinates need no
// per-cell division, x neighbours come by shuffle (one explicit load at the
// segment edge or across the wrap), and y / z neighbours are coalesced row
// loads.  The update is the one of step6.cu: a step is two launches, the first
// group (H for J sources, E for K sources) with a = 1, b = h, then the sigma
// group fused with the surface projection and the FP64 accumulation of
// w_n s(n) (Eq. (1)).  Fields are updated in place (one buffer).
#include <cuda_runtime.h>

#include "casimir.h"
#include "kernels.h"

namespace cas {

namespace {

constexpr int WARPS3 = 8;                  // warps per CTA
constexpr int LPW3 = LINES3 / WARPS3;      // lines per warp
#ifndef UNROLL3
#define UNROLL3 2                          // lines of a warp in flight together
#endif
constexpr int kUnroll3 = UNROLL3;

template <typename R, bool CPLX>
struct W3;

template <typename R>
struct W3<R, false> {
    R x;
    __device__ W3() : x(0) {}
    __device__ explicit W3(R a) : x(a) {}
    __device__ W3 operator+(W3 o) const { return W3(x + o.x); }
    __device__ W3 operator-(W3 o) const { return W3(x - o.x); }
    __device__ W3 operator*(R s) const { return W3(x * s); }
    __device__ W3 ph(R c, R) const { return W3(x * c); }
    __device__ W3 dn() const { return W3(__shfl_down_sync(0xffffffffu, x, 1)); }
    __device__ W3 up() const { return W3(__shfl_up_sync(0xffffffffu, x, 1)); }
};

template <typename R>
struct W3<R, true> {
    R x, y;
    __device__ W3() : x(0), y(0) {}
    __device__ W3(R a, R b) : x(a), y(b) {}
    __device__ W3 operator+(W3 o) const { return W3(x + o.x, y + o.y); }
    __device__ W3 operator-(W3 o) const { return W3(x - o.x, y - o.y); }
    __device__ W3 operator*(R s) const { return W3(x * s, y * s); }
    __device__ W3 ph(R c, R s) const { return W3(x * c - y * s, x * s + y * c); }
    __device__ W3 dn() const { return W3(__shfl_down_sync(0xffffffffu, x, 1), __shfl_down_sync(0xffffffffu, y, 1)); }
    __device__ W3 up() const { return W3(__shfl_up_sync(0xffffffffu, x, 1), __shfl_up_sync(0xffffffffu, y, 1)); }
};

// planes of N elements (real, imaginary pairs when complex); 32-bit element offsets
template <typename R, bool CPLX>
__device__ __forceinline__ W3<R, CPLX> ld3(const R *p, int plane, unsigned N, unsigned g)
{
    if constexpr (CPLX) return W3<R, CPLX>(p[(2u * plane) * N + g], p[(2u * plane + 1u) * N + g]);
    else return W3<R, CPLX>(p[(unsigned)plane * N + g]);
}

template <typename R, bool CPLX>
__device__ __forceinline__ void st3(R *p, int plane, unsigned N, unsigned g, W3<R, CPLX> v)
{
    if constexpr (CPLX) { p[(2u * plane) * N + g] = v.x; p[(2u * plane + 1u) * N + g] = v.y; }
    else p[(unsigned)plane * N + g] = v.x;
}

// MINB: resident CTAs per SM asked of the register allocator; the kernel is latency-bound and
// gains from every extra warp (a few spilled words stay in L1)
template <typename R, bool CPLX, int MINB>
__global__ void __launch_bounds__(WARPS3 * 32, MINB)
k_line3(const DevSim6 *__restrict__ sims, const DevTile *__restrict__ tiles,
        const int64_t *__restrict__ launch_base, int64_t launch_add, int phase)
{
    using V = W3<R, CPLX>;
    __shared__ double red[WARPS3];
    __shared__ DevSim6 sS;
    const DevTile t = tiles[blockIdx.x];
    {
        // one copy of the simulation's descriptor per CTA (cheap shared reads in the loop)
        const int *src = reinterpret_cast<const int *>(sims + t.sim);
        int *dst = reinterpret_cast<int *>(&sS);
        for (int q = threadIdx.x; q < (int)(sizeof(DevSim6) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const DevSim6 &S = sS;
    const int64_t n = *launch_base + launch_add - S.s0;
    if (n < 1 || n > S.T) return;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const unsigned sy = (unsigned)nx, sz = (unsigned)nx * (unsigned)ny;
    const unsigned N = sz * (unsigned)nz;
    R *__restrict__ F = reinterpret_cast<R *>(S.fields);
    const R *__restrict__ coef = reinterpret_cast<const R *>(S.coef);
    const uint8_t *__restrict__ mat = S.mat;
    const bool updE = (phase == 0) == (S.magnetic != 0);
    const R a = phase == 0 ? (R)1 : (R)S.a;
    const R b = phase == 0 ? (R)(n == 1 ? 0.5 * S.dt : S.dt) : (R)S.bs;
    const bool first_e = S.magnetic == 0 && n == 1;    // Lorentz start of electric sources (their E group is phase 1)
    const R idx = (R)S.inv_dx;
    R *__restrict__ psi = reinterpret_cast<R *>(S.psi);
    const R *__restrict__ pml = reinterpret_cast<const R *>(S.pml);
    R *__restrict__ P = reinterpret_cast<R *>(S.lor);
    const R *__restrict__ lc = reinterpret_cast<const R *>(S.lorc);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = t.i0 + lane;
    const bool valid = x < nx;
    const int xc = valid ? x : nx - 1;
    const int line_end = min(t.j0 + LINES3, ny * nz);
    const bool inx = S.pml_d[0] > 0 && (xc < S.pml_d[0] || xc >= nx - S.pml_d[0]);
    const int cf = CPLX ? 2 : 1;
    const int dX = S.pml_d[0], dY = S.pml_d[1], dZ = S.pml_d[2];
    // psi planes of axis a start at psi + psi_off[a] and lie cf * slab[a] elements apart
    // (32-bit offsets: the planner sends only runs with 12 N < 2^32 here)
    const unsigned pstride[3] = {(unsigned)(cf * S.slab[0]), (unsigned)(cf * S.slab[1]), (unsigned)(cf * S.slab[2])};
    // stretched difference along axis ax at slab index si: psi' = b psi + c d, d / kappa + psi'
    auto stretch = [&](V d, int ax, const R *pr, int plane, unsigned si, bool wr) -> V {
        R *ps = psi + S.psi_off[ax] + plane * pstride[ax];
        V p;
        if constexpr (CPLX) p = V(ps[si], ps[S.slab[ax] + si]);
        else p = V(ps[si]);
        p = p * pr[0] + d * pr[1];
        if (wr) {
            if constexpr (CPLX) { ps[si] = p.x; ps[S.slab[ax] + si] = p.y; }
            else ps[si] = p.x;
        }
        return d * pr[2] + p;
    };
    // (y, z) of this warp's first line, then advanced by WARPS3 lines per iteration (no division in the loop)
    int y = (t.j0 + warp) % ny, z = (t.j0 + warp) / ny;

#pragma unroll kUnroll3
    for (int q = 0; q < LPW3; ++q) {
        const int line = t.j0 + warp + q * WARPS3;
        if (q > 0) {
            y += WARPS3;
            while (y >= ny) { y -= ny; ++z; }
        }
        if (line >= line_end) continue;                 // uniform over the warp
        const unsigned g = (unsigned)line * sy + (unsigned)xc;
        const bool iny = dY > 0 && (y < dY || y >= ny - dY);
        const bool inz = dZ > 0 && (z < dZ || z >= nz - dZ);
        if (updE) {
            // every load of the cell first: own E and H, backward neighbours (x by shuffle except at the
            // segment edge and the wrap), material
            const bool edge = lane == 0 || x == 0;
            V hyl_e, hzl_e;
            if (edge) {
                const unsigned gl = x == 0 ? g + (unsigned)(nx - 1) : g - 1u;
                hyl_e = ld3<R, CPLX>(F, 4, N, gl);
                hzl_e = ld3<R, CPLX>(F, 5, N, gl);
            }
            const V hx = ld3<R, CPLX>(F, 3, N, g), hy = ld3<R, CPLX>(F, 4, N, g), hz = ld3<R, CPLX>(F, 5, N, g);
            const unsigned gy = y == 0 ? g + (unsigned)(ny - 1) * sy : g - sy;
            V hxy = ld3<R, CPLX>(F, 3, N, gy), hzy = ld3<R, CPLX>(F, 5, N, gy);
            const unsigned gz = z == 0 ? g + (unsigned)(nz - 1) * sz : g - sz;
            V hxz = ld3<R, CPLX>(F, 3, N, gz), hyz = ld3<R, CPLX>(F, 4, N, gz);
            const V e3[3] = {ld3<R, CPLX>(F, 0, N, g), ld3<R, CPLX>(F, 1, N, g), ld3<R, CPLX>(F, 2, N, g)};
            const int m = mat[g];
            V hyl = hy.up(), hzl = hz.up();
            if (edge) {
                hyl = x == 0 ? hyl_e.ph((R)S.bre[0], -(R)S.bim[0]) : hyl_e;
                hzl = x == 0 ? hzl_e.ph((R)S.bre[0], -(R)S.bim[0]) : hzl_e;
            }
            if (y == 0) { hxy = hxy.ph((R)S.bre[1], -(R)S.bim[1]); hzy = hzy.ph((R)S.bre[1], -(R)S.bim[1]); }
            if (z == 0) { hxz = hxz.ph((R)S.bre[2], -(R)S.bim[2]); hyz = hyz.ph((R)S.bre[2], -(R)S.bim[2]); }
            V dyHz = (hz - hzy) * idx, dzHy = (hy - hyz) * idx, dzHx = (hx - hxz) * idx;
            V dxHz = (hz - hzl) * idx, dxHy = (hy - hyl) * idx, dyHx = (hx - hxy) * idx;
            if (inx) {
                const R *prx = pml + S.pml_off[0];
                const R pr[3] = {prx[xc], prx[nx + xc], prx[2 * nx + xc]};
                const int sxp = xc < dX ? xc : xc - (nx - 2 * dX);
                const unsigned six = (unsigned)line * (unsigned)(2 * dX) + (unsigned)sxp;
                dxHz = stretch(dxHz, 0, pr, 0, six, valid);    // E_y
                dxHy = stretch(dxHy, 0, pr, 1, six, valid);    // E_z
            }
            if (iny) {
                const R *pry = pml + S.pml_off[1];
                const R pr[3] = {pry[y], pry[ny + y], pry[2 * ny + y]};
                const int syp = y < dY ? y : y - (ny - 2 * dY);
                const unsigned siy = ((unsigned)z * (unsigned)(2 * dY) + (unsigned)syp) * sy + (unsigned)xc;
                dyHx = stretch(dyHx, 1, pr, 0, siy, valid);    // E_z
                dyHz = stretch(dyHz, 1, pr, 1, siy, valid);    // E_x
            }
            if (inz) {
                const R *prz = pml + S.pml_off[2];
                const R pr[3] = {prz[z], prz[nz + z], prz[2 * nz + z]};
                const int szp = z < dZ ? z : z - (nz - 2 * dZ);
                const unsigned siz = ((unsigned)szp * (unsigned)ny + (unsigned)y) * sy + (unsigned)xc;
                dzHy = stretch(dzHy, 2, pr, 0, siz, valid);    // E_x
                dzHx = stretch(dzHx, 2, pr, 1, siz, valid);    // E_y
            }
            const V c3[3] = {dyHz - dzHy, dzHx - dxHz, dxHy - dyHx};
            const R *cm = coef + 6 * m;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const V e = e3[k];
                V en = e * a + c3[k] * (b * cm[k]);
                if (P) {
                    const R *l4 = lc + 12 * S.npoles * m + 4 * k;
                    if (l4[2] != (R)0) {
                        // per pole q (present poles first): P_q' = [cp P_q - cpm P_q-prev + ce E] cd
                        // (unrolled to the largest pole count, so that every present pole's loads
                        // issue together)
                        V sp = c3[k] * b;
#pragma unroll
                        for (int q = 0; q < CASIMIR_MAX_POLES; ++q) {
                            const R *lq = l4 + 12 * q;
                            if (q > 0 && !(q < S.npoles && lq[2] != (R)0)) continue;
                            const R ce = lq[2];
                            const V p = ld3<R, CPLX>(P, 6 * q + k, N, g), pm = ld3<R, CPLX>(P, 6 * q + 3 + k, N, g);
                            const V pn = first_e ? (p * lq[0] + e * ce) * (R)0.5 : (p * lq[0] - pm * lq[1] + e * ce) * lq[3];
                            if (valid) {
                                st3<R, CPLX>(P, 6 * q + 3 + k, N, g, p);
                                st3<R, CPLX>(P, 6 * q + k, N, g, pn);
                            }
                            sp = sp + p * a - pn;
                        }
                        en = e * a + sp * cm[k];
                    }
                }
                if (valid) st3<R, CPLX>(F, k, N, g, en);
            }
        } else {
            // every load of the cell first: own E and H, forward neighbours, material
            const bool edge = lane == 31 || x >= nx - 1;
            V eyr_e, ezr_e;
            if (edge) {
                const unsigned gr = xc == nx - 1 ? g - (unsigned)(nx - 1) : g + 1u;
                eyr_e = ld3<R, CPLX>(F, 1, N, gr);
                ezr_e = ld3<R, CPLX>(F, 2, N, gr);
            }
            const V ex = ld3<R, CPLX>(F, 0, N, g), ey = ld3<R, CPLX>(F, 1, N, g), ez = ld3<R, CPLX>(F, 2, N, g);
            const unsigned gy = y == ny - 1 ? g - (unsigned)(ny - 1) * sy : g + sy;
            V exy = ld3<R, CPLX>(F, 0, N, gy), ezy = ld3<R, CPLX>(F, 2, N, gy);
            const unsigned gz = z == nz - 1 ? g - (unsigned)(nz - 1) * sz : g + sz;
            V exz = ld3<R, CPLX>(F, 0, N, gz), eyz = ld3<R, CPLX>(F, 1, N, gz);
            const V h3[3] = {ld3<R, CPLX>(F, 3, N, g), ld3<R, CPLX>(F, 4, N, g), ld3<R, CPLX>(F, 5, N, g)};
            const int m = mat[g];
            V eyr = ey.dn(), ezr = ez.dn();
            if (edge) {
                eyr = xc == nx - 1 ? eyr_e.ph((R)S.bre[0], (R)S.bim[0]) : eyr_e;
                ezr = xc == nx - 1 ? ezr_e.ph((R)S.bre[0], (R)S.bim[0]) : ezr_e;
            }
            if (y == ny - 1) { exy = exy.ph((R)S.bre[1], (R)S.bim[1]); ezy = ezy.ph((R)S.bre[1], (R)S.bim[1]); }
            if (z == nz - 1) { exz = exz.ph((R)S.bre[2], (R)S.bim[2]); eyz = eyz.ph((R)S.bre[2], (R)S.bim[2]); }
            V dyEz = (ezy - ez) * idx, dzEy = (eyz - ey) * idx, dzEx = (exz - ex) * idx;
            V dxEz = (ezr - ez) * idx, dxEy = (eyr - ey) * idx, dyEx = (exy - ex) * idx;
            if (inx) {
                const R *prx = pml + S.pml_off[0];
                const R pr[3] = {prx[3 * nx + xc], prx[4 * nx + xc], prx[5 * nx + xc]};
                const int sxp = xc < dX ? xc : xc - (nx - 2 * dX);
                const unsigned six = (unsigned)line * (unsigned)(2 * dX) + (unsigned)sxp;
                dxEz = stretch(dxEz, 0, pr, 2, six, valid);    // H_y
                dxEy = stretch(dxEy, 0, pr, 3, six, valid);    // H_z
            }
            if (iny) {
                const R *pry = pml + S.pml_off[1];
                const R pr[3] = {pry[3 * ny + y], pry[4 * ny + y], pry[5 * ny + y]};
                const int syp = y < dY ? y : y - (ny - 2 * dY);
                const unsigned siy = ((unsigned)z * (unsigned)(2 * dY) + (unsigned)syp) * sy + (unsigned)xc;
                dyEx = stretch(dyEx, 1, pr, 2, siy, valid);    // H_z
                dyEz = stretch(dyEz, 1, pr, 3, siy, valid);    // H_x
            }
            if (inz) {
                const R *prz = pml + S.pml_off[2];
                const R pr[3] = {prz[3 * nz + z], prz[4 * nz + z], prz[5 * nz + z]};
                const int szp = z < dZ ? z : z - (nz - 2 * dZ);
                const unsigned siz = ((unsigned)szp * (unsigned)ny + (unsigned)y) * sy + (unsigned)xc;
                dzEy = stretch(dzEy, 2, pr, 2, siz, valid);    // H_x
                dzEx = stretch(dzEx, 2, pr, 3, siz, valid);    // H_y
            }
            const V c3[3] = {dyEz - dzEy, dzEx - dxEz, dxEy - dyEx};
            const R *cm = coef + 6 * m;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (valid) st3<R, CPLX>(F, 3 + k, N, g, h3[k] * a - c3[k] * (b * cm[3 + k]));
        }
    }

    if (phase == 1 && t.ne > 0) {
        __syncthreads();   // the block's field writes are visible to the block
        double part = 0.0;
        for (int e = threadIdx.x; e < t.ne; e += blockDim.x) {
            const DevEnt en = t.ents[e];
            const int loc = en.loc & 0xffff, arr = (en.loc >> 16) & 7, im = (en.loc >> 19) & 1;
            const int lw = loc >> 5, lx = loc & 31;
            const unsigned g = (unsigned)(t.j0 + lw) * sy + (unsigned)(t.i0 + lx);
            const unsigned plane = CPLX ? (unsigned)(2 * arr + im) : (unsigned)arr;
            part += (im ? -en.w : en.w) * (double)F[plane * N + g];
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < WARPS3; ++w) s += red[w];
            const double c = S.gw[n - 1] * s;
            atomicAdd(S.acc, c);
            if (n > S.tail_from) atomicAdd(S.tail, c);
        }
    }
}

}  // namespace

void launch_line3(int fp64, int cplx, const DevSim6 *sims, const DevTile *tiles, int ntiles,
                  const int64_t *launch_base, int64_t launch_add, int phase, cudaStream_t st)
{
    if (ntiles <= 0) return;
    if (fp64) {
        if (cplx) k_line3<double, true, 4><<<ntiles, WARPS3 * 32, 0, st>>>(sims, tiles, launch_base, launch_add, phase);
        else k_line3<double, false, 6><<<ntiles, WARPS3 * 32, 0, st>>>(sims, tiles, launch_base, launch_add, phase);
    } else {
        if (cplx) k_line3<float, true, 6><<<ntiles, WARPS3 * 32, 0, st>>>(sims, tiles, launch_base, launch_add, phase);
        else k_line3<float, false, 8><<<ntiles, WARPS3 * 32, 0, st>>>(sims, tiles, launch_base, launch_add, phase);
    }
}

}  // namespace cas
