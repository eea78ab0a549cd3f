// Six-component Yee leapfrog for the simulations that need every field:
// two-dimensional cross-sections with k_z != 0 (Sec. III B), Bloch-periodic
// cells (Sec. III D) and full three-dimensional runs (Sec. III E), with CPML
// absorbing layers (Sec. III B) and single-pole Lorentz media continued onto
// the complex-frequency contour (Eq. (9), Sec. III B).
//
// Storage: E_x, E_y, E_z, H_x, H_y, H_z on the standard Yee sites, one plane of
// nx*ny*nz elements each (two planes, real and imaginary, for complex fields).
// Pure k_z runs keep real fields: with a real source the set {E_x, E_y, H_z}
// and i{E_z, H_x, H_y} stay real (or the other way round), so d/dz acts as
// +k_z on the source's set and -k_z on the other (kzA / kzB below).
//
// A step is two launches over every cell of every simulation: the first group
// (H for J sources, E for K sources) with a = 1, b = h, then the sigma group
// with a = (1 - sigma dt/2)/(1 + sigma dt/2), b = dt/(1 + sigma dt/2), fused
// with the surface projection and the FP64 accumulation of w_n s(n).
#include <cuda_runtime.h>

#include "kernels.h"

namespace cas {

namespace {

template <typename R, bool CPLX>
struct V;

template <typename R>
struct V<R, false> {
    R x;
    __device__ V() : x(0) {}
    __device__ explicit V(R a) : x(a) {}
    __device__ V operator+(V o) const { return V(x + o.x); }
    __device__ V operator-(V o) const { return V(x - o.x); }
    __device__ V scale(R s) const { return V(x * s); }
    __device__ V rot(R c, R s) const { return V(x * c); }     // times (c + i s), s = 0 for real fields
    __device__ V ikz(R kre) const { return V(x * kre); }      // real-phase d/dz
};

template <typename R>
struct V<R, true> {
    R x, y;
    __device__ V() : x(0), y(0) {}
    __device__ V(R a, R b) : x(a), y(b) {}
    __device__ V operator+(V o) const { return V(x + o.x, y + o.y); }
    __device__ V operator-(V o) const { return V(x - o.x, y - o.y); }
    __device__ V scale(R s) const { return V(x * s, y * s); }
    __device__ V rot(R c, R s) const { return V(x * c - y * s, x * s + y * c); }
    __device__ V ikz(R k) const { return V(-y * k, x * k); }   // i k F
};

template <typename R, bool CPLX>
struct Fields {
    R *p;
    size_t N;
    __device__ V<R, CPLX> get(int comp, size_t m) const
    {
        if constexpr (CPLX) return V<R, CPLX>(p[(2 * comp) * N + m], p[(2 * comp + 1) * N + m]);
        else return V<R, CPLX>(p[comp * N + m]);
    }
    __device__ void put(int comp, size_t m, V<R, CPLX> v) const
    {
        if constexpr (CPLX) { p[(2 * comp) * N + m] = v.x; p[(2 * comp + 1) * N + m] = v.y; }
        else p[comp * N + m] = v.x;
    }
};

// psi storage: per axis a, the two PML slabs along a (2 d cells) times the other axes
__device__ __forceinline__ size_t slab_index(const DevSim6 &S, int a, const int c[3])
{
    int d = S.pml_d[a];
    int s = c[a] < d ? c[a] : c[a] - (S.n[a] - 2 * d);
    int q[3] = {c[0], c[1], c[2]};
    q[a] = s;
    int dims[3] = {S.n[0], S.n[1], S.n[2]};
    dims[a] = 2 * d;
    return ((size_t)q[2] * dims[1] + q[1]) * dims[0] + q[0];
}

template <typename R, bool CPLX>
__device__ __forceinline__ V<R, CPLX> deriv(const DevSim6 &S, const Fields<R, CPLX> &F, int comp, int a,
                                            const int c[3], size_t m, bool forward)
{
    using Vt = V<R, CPLX>;
    Vt here = F.get(comp, m);
    if (a == 2 && S.dims == 2) {
        if constexpr (CPLX) return here.ikz((R)S.kz);
        else return here.ikz((comp == 0 || comp == 1 || comp == 5) ? (R)S.kzA : (R)S.kzB);
    }
    size_t stride = a == 0 ? 1 : (a == 1 ? (size_t)S.n[0] : (size_t)S.n[0] * S.n[1]);
    if (forward) {
        if (c[a] + 1 < S.n[a]) return (F.get(comp, m + stride) - here).scale((R)S.inv_dx);
        Vt o = F.get(comp, m - (size_t)(S.n[a] - 1) * stride).rot((R)S.bre[a], (R)S.bim[a]);
        return (o - here).scale((R)S.inv_dx);
    }
    if (c[a] > 0) return (here - F.get(comp, m - stride)).scale((R)S.inv_dx);
    Vt o = F.get(comp, m + (size_t)(S.n[a] - 1) * stride).rot((R)S.bre[a], -(R)S.bim[a]);
    return (here - o).scale((R)S.inv_dx);
}

template <typename R, bool CPLX>
__device__ __forceinline__ V<R, CPLX> stretch(const DevSim6 &S, V<R, CPLX> d, int a, int half, int pos,
                                              int psi_plane, const int c[3])
{
    if (a == 2 && S.dims == 2) return d;
    int dd = S.pml_d[a];
    if (dd == 0 || (pos >= dd && pos < S.n[a] - dd)) return d;
    const R *prof = reinterpret_cast<const R *>(S.pml) + S.pml_off[a] + (size_t)half * 3 * S.n[a];
    R b = prof[pos], cc = prof[S.n[a] + pos], ik = prof[2 * S.n[a] + pos];
    size_t si = slab_index(S, a, c);
    R *psi = reinterpret_cast<R *>(S.psi) + S.psi_off[a] + (size_t)psi_plane * (CPLX ? 2 : 1) * S.slab[a];
    V<R, CPLX> p;
    if constexpr (CPLX) p = V<R, CPLX>(psi[si], psi[S.slab[a] + si]);
    else p = V<R, CPLX>(psi[si]);
    p = p.scale(b) + d.scale(cc);
    if constexpr (CPLX) { psi[si] = p.x; psi[S.slab[a] + si] = p.y; }
    else psi[si] = p.x;
    return d.scale(ik) + p;
}

template <typename R, bool CPLX>
__global__ void __launch_bounds__(256)
k_full(const DevSim6 *__restrict__ sims, const DevTile6 *__restrict__ tiles,
       const int64_t *__restrict__ launch_base, int64_t launch_add, int phase)
{
    using Vt = V<R, CPLX>;
    __shared__ double red[8];
    const DevTile6 t = tiles[blockIdx.x];
    const DevSim6 &S = sims[t.sim];
    const int64_t n = *launch_base + launch_add - S.s0;
    if (n < 1 || n > S.T) return;
    const size_t N = (size_t)S.n[0] * S.n[1] * S.n[2];
    Fields<R, CPLX> F{reinterpret_cast<R *>(S.fields), N};
    const bool updE = (phase == 0) == (S.magnetic != 0);
    const R a = phase == 0 ? (R)1 : (R)S.a;
    const R b = phase == 0 ? (R)(n == 1 ? 0.5 * S.dt : S.dt) : (R)S.bs;
    const size_t m = t.cell0 + threadIdx.x;
    if (m < N && threadIdx.x < t.count) {
        int c3[3];
        const unsigned mm = (unsigned)m, nx = (unsigned)S.n[0], ny = (unsigned)S.n[1];
        const unsigned row = mm / nx;
        c3[0] = (int)(mm - row * nx);
        c3[1] = (int)(row % ny);
        c3[2] = (int)(row / ny);
        const int id = S.mat[m];
        const R *coef = reinterpret_cast<const R *>(S.coef) + 6 * id;
        if (updE) {
            for (int cpt = 0; cpt < 3; ++cpt) {
                int a1 = (cpt + 1) % 3, a2 = (cpt + 2) % 3;
                // (curl H)_c = d_{a1} H_{a2} - d_{a2} H_{a1}, backward differences, integer-site profiles
                Vt t1 = stretch<R, CPLX>(S, deriv<R, CPLX>(S, F, 3 + a2, a1, c3, m, false), a1, 0, c3[a1], (cpt == (a1 + 1) % 3) ? 0 : 1, c3);
                Vt t2 = stretch<R, CPLX>(S, deriv<R, CPLX>(S, F, 3 + a1, a2, c3, m, false), a2, 0, c3[a2], (cpt == (a2 + 1) % 3) ? 0 : 1, c3);
                Vt curl = t1 - t2;
                R ce = coef[cpt];
                Vt e = F.get(cpt, m);
                Vt enew;
                if (S.lor) {
                    const double *lt = S.lorentz + 6 * id + 2 * cpt;
                    R de = (R)lt[0];
                    if (de != (R)0) {
                        R w2 = (R)(lt[1] * lt[1]);
                        R dt = (R)S.dt_full, sg = (R)S.sigma;
                        Fields<R, CPLX> P{reinterpret_cast<R *>(S.lor), N};
                        Vt p = P.get(cpt, m), pm = P.get(3 + cpt, m);
                        Vt pn;
                        if (S.magnetic == 0 && n == 1)
                            pn = (p.scale((R)2 - w2 * dt * dt) + e.scale(de * w2 * dt * dt)).scale((R)0.5);
                        else
                            pn = (p.scale((R)2 - w2 * dt * dt) - pm.scale((R)1 - (R)0.5 * sg * dt) +
                                  e.scale(de * w2 * dt * dt)).scale((R)1 / ((R)1 + (R)0.5 * sg * dt));
                        P.put(3 + cpt, m, p);
                        P.put(cpt, m, pn);
                        enew = e.scale(a) + (p.scale(a) - pn + curl.scale(b)).scale(ce);
                    } else {
                        enew = e.scale(a) + curl.scale(b * ce);
                    }
                } else {
                    enew = e.scale(a) + curl.scale(b * ce);
                }
                F.put(cpt, m, enew);
            }
        } else {
            for (int cpt = 0; cpt < 3; ++cpt) {
                int a1 = (cpt + 1) % 3, a2 = (cpt + 2) % 3;
                // (curl E)_c = d_{a1} E_{a2} - d_{a2} E_{a1}, forward differences, half-site profiles
                Vt t1 = stretch<R, CPLX>(S, deriv<R, CPLX>(S, F, a2, a1, c3, m, true), a1, 1, c3[a1], 2 + ((cpt == (a1 + 1) % 3) ? 0 : 1), c3);
                Vt t2 = stretch<R, CPLX>(S, deriv<R, CPLX>(S, F, a1, a2, c3, m, true), a2, 1, c3[a2], 2 + ((cpt == (a2 + 1) % 3) ? 0 : 1), c3);
                Vt curl = t1 - t2;
                R ch = coef[3 + cpt];
                Vt hv = F.get(3 + cpt, m);
                F.put(3 + cpt, m, hv.scale(a) - curl.scale(b * ch));
            }
        }
    }
    if (phase == 1 && t.ne > 0) {
        __syncthreads();
        double part = 0.0;
        for (int e = threadIdx.x; e < t.ne; e += blockDim.x) {
            DevEnt6 en = t.ents[e];
            size_t g = t.cell0 + en.off;
            Vt v = F.get(en.arr, g);
            if constexpr (CPLX) part += en.wre * (double)v.x - en.wim * (double)v.y;
            else part += en.wre * (double)v.x;
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) red[warp] = part;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += red[q];
            double cc = S.gw[n - 1] * s;
            atomicAdd(S.acc, cc);
            if (n > S.tail_from) atomicAdd(S.tail, cc);
        }
    }
}

template <typename R>
__global__ void k_inject6(R *fields, const DevSrc6 *src, int nsrc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nsrc) {
        fields[src[i].idx_re] = (R)src[i].re;
        if (src[i].idx_im >= 0) fields[src[i].idx_im] = (R)src[i].im;
    }
}

}  // namespace

void launch_full(int fp64, int cplx, const DevSim6 *sims, const DevTile6 *tiles, int ntiles,
                 const int64_t *launch_base, int64_t launch_add, int phase, cudaStream_t st)
{
    if (ntiles <= 0) return;
    if (fp64) {
        if (cplx) k_full<double, true><<<ntiles, 256, 0, st>>>(sims, tiles, launch_base, launch_add, phase);
        else k_full<double, false><<<ntiles, 256, 0, st>>>(sims, tiles, launch_base, launch_add, phase);
    } else {
        if (cplx) k_full<float, true><<<ntiles, 256, 0, st>>>(sims, tiles, launch_base, launch_add, phase);
        else k_full<float, false><<<ntiles, 256, 0, st>>>(sims, tiles, launch_base, launch_add, phase);
    }
}

void launch_inject6(int fp64, void *fields, const DevSrc6 *src, int nsrc, cudaStream_t st)
{
    if (nsrc <= 0) return;
    int b = (nsrc + 255) / 256;
    if (fp64) k_inject6<double><<<b, 256, 0, st>>>(reinterpret_cast<double *>(fields), src, nsrc);
    else k_inject6<float><<<b, 256, 0, st>>>(reinterpret_cast<float *>(fields), src, nsrc);
}

}  // namespace cas
