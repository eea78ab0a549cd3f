// Six-component Yee leapfrog for the simulations that need every field:
// two-dimensional cross-sections with k_z != 0 (Sec. III B), Bloch-periodic
// cells (Sec. III D) and full three-dimensional runs (Sec. III E), with CPML
// absorbing layers (Sec. III B) and Lorentz media of up to three undamped poles
// continued onto the complex-frequency contour (Eq. (9), Sec. III B; the silica
// model of Sec. III D).
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

// Neighbour of cell (c) along axis a in direction dir (+1 forward, -1 backward): flat index,
// and whether the step wraps around (then the Bloch factor applies).
struct Nb {
    int64_t m;
    bool wrap;
};

template <int D>
__device__ __forceinline__ Nb nbr(const DevSim6 &S, const int c[3], int64_t m, int a, int dir)
{
    int64_t stride = a == 0 ? 1 : (a == 1 ? (int64_t)S.n[0] : (int64_t)S.n[0] * S.n[1]);
    if (dir > 0) {
        if (c[a] + 1 < S.n[a]) return Nb{m + stride, false};
        return Nb{m - (int64_t)(S.n[a] - 1) * stride, true};
    }
    if (c[a] > 0) return Nb{m - stride, false};
    return Nb{m + (int64_t)(S.n[a] - 1) * stride, true};
}

// d_a F at this cell: forward (H update) or backward (E update) difference, i k_z in 2D along z.
template <typename R, bool CPLX, int D>
__device__ __forceinline__ V<R, CPLX> dif(const DevSim6 &S, const Fields<R, CPLX> &F, int comp, int a,
                                          const int c[3], int64_t m, V<R, CPLX> here, bool forward)
{
    if (D == 2 && a == 2) {
        if constexpr (CPLX) return here.ikz((R)S.kz);
        else return here.ikz((comp == 0 || comp == 1 || comp == 5) ? (R)S.kzA : (R)S.kzB);
    }
    Nb q = nbr<D>(S, c, m, a, forward ? 1 : -1);
    V<R, CPLX> o = F.get(comp, q.m);
    if (q.wrap) o = o.rot((R)S.bre[a], forward ? (R)S.bim[a] : -(R)S.bim[a]);
    return (forward ? (o - here) : (here - o)).scale((R)S.inv_dx);
}

template <typename R, bool CPLX, int D>
__global__ void __launch_bounds__(256)
k_full(const DevSim6 *__restrict__ sims, const DevTile6 *__restrict__ tiles,
       const int64_t *__restrict__ launch_base, int64_t launch_add, int phase)
{
    using Vt = V<R, CPLX>;
    __shared__ double red[8];
    __shared__ DevSim6 sS;
    const DevTile6 t = tiles[blockIdx.x];
    {
        // one copy of the simulation's descriptor per CTA
        const int *src = reinterpret_cast<const int *>(sims + t.sim);
        int *dst = reinterpret_cast<int *>(&sS);
        for (int q = threadIdx.x; q < (int)(sizeof(DevSim6) / sizeof(int)); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const DevSim6 &S = sS;
    const int64_t n = *launch_base + launch_add - S.s0;
    if (n < 1 || n > S.T) return;
    const int64_t N = (int64_t)S.n[0] * S.n[1] * S.n[2];
    Fields<R, CPLX> F{reinterpret_cast<R *>(S.fields), (size_t)N};
    const bool updE = (phase == 0) == (S.magnetic != 0);
    const R a = phase == 0 ? (R)1 : (R)S.a;
    const R b = phase == 0 ? (R)(n == 1 ? 0.5 * S.dt : S.dt) : (R)S.bs;
#pragma unroll 2
    for (int r = 0; r < TILE6 / 256; ++r) {
    const int64_t m = t.cell0 + r * 256 + threadIdx.x;
    if (r * 256 + (int)threadIdx.x < t.count) {
        int c3[3];
        const unsigned mm = (unsigned)m, nx = (unsigned)S.n[0], ny = (unsigned)S.n[1];
        const unsigned row = mm / nx;
        c3[0] = (int)(mm - row * nx);
        c3[1] = (int)(row % ny);
        c3[2] = (int)(row / ny);
        bool inpml = false;
#pragma unroll
        for (int ax = 0; ax < D; ++ax)
            if (S.pml_d[ax] > 0 && (c3[ax] < S.pml_d[ax] || c3[ax] >= S.n[ax] - S.pml_d[ax])) inpml = true;
        const int id = S.mat[m];
        const R *coef = reinterpret_cast<const R *>(S.coef) + 6 * id;
        if (updE) {
            Vt h[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) h[q] = F.get(3 + q, m);
            Vt curl[3];
#pragma unroll
            for (int cpt = 0; cpt < 3; ++cpt) {
                const int a1 = (cpt + 1) % 3, a2 = (cpt + 2) % 3;
                // (curl H)_c = d_{a1} H_{a2} - d_{a2} H_{a1}, backward differences, integer-site profiles
                Vt t1 = dif<R, CPLX, D>(S, F, 3 + a2, a1, c3, m, h[a2], false);
                Vt t2 = dif<R, CPLX, D>(S, F, 3 + a1, a2, c3, m, h[a1], false);
                if (inpml) {
                    t1 = stretch<R, CPLX>(S, t1, a1, 0, c3[a1], (cpt == (a1 + 1) % 3) ? 0 : 1, c3);
                    t2 = stretch<R, CPLX>(S, t2, a2, 0, c3[a2], (cpt == (a2 + 1) % 3) ? 0 : 1, c3);
                }
                curl[cpt] = t1 - t2;
            }
#pragma unroll
            for (int cpt = 0; cpt < 3; ++cpt) {
                R ce = coef[cpt];
                Vt e = F.get(cpt, m);
                Vt enew;
                if (S.lor && S.lorentz[6 * S.npoles * id + 2 * cpt] != 0.0) {
                    // E' = a E + (a sum_q P_q - sum_q P_q' + b curl) / eps_inf
                    const R dt = (R)S.dt_full, sg = (R)S.sigma;
                    Fields<R, CPLX> P{reinterpret_cast<R *>(S.lor), (size_t)N};
                    Vt sp = curl[cpt].scale(b);
                    for (int q = 0; q < S.npoles; ++q) {
                        const double *lq = S.lorentz + 6 * (S.npoles * id + q) + 2 * cpt;
                        const R de = (R)lq[0];
                        if (de == (R)0) break;   // present poles come first
                        const R w2 = (R)(lq[1] * lq[1]);
                        Vt p = P.get(6 * q + cpt, m), pm = P.get(6 * q + 3 + cpt, m);
                        Vt pn;
                        if (S.magnetic == 0 && n == 1)
                            pn = (p.scale((R)2 - w2 * dt * dt) + e.scale(de * w2 * dt * dt)).scale((R)0.5);
                        else
                            pn = (p.scale((R)2 - w2 * dt * dt) - pm.scale((R)1 - (R)0.5 * sg * dt) +
                                  e.scale(de * w2 * dt * dt)).scale((R)1 / ((R)1 + (R)0.5 * sg * dt));
                        P.put(6 * q + 3 + cpt, m, p);
                        P.put(6 * q + cpt, m, pn);
                        sp = sp + p.scale(a) - pn;
                    }
                    enew = e.scale(a) + sp.scale(ce);
                } else {
                    enew = e.scale(a) + curl[cpt].scale(b * ce);
                }
                F.put(cpt, m, enew);
            }
        } else {
            Vt e[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) e[q] = F.get(q, m);
#pragma unroll
            for (int cpt = 0; cpt < 3; ++cpt) {
                const int a1 = (cpt + 1) % 3, a2 = (cpt + 2) % 3;
                // (curl E)_c = d_{a1} E_{a2} - d_{a2} E_{a1}, forward differences, half-site profiles
                Vt t1 = dif<R, CPLX, D>(S, F, a2, a1, c3, m, e[a2], true);
                Vt t2 = dif<R, CPLX, D>(S, F, a1, a2, c3, m, e[a1], true);
                if (inpml) {
                    t1 = stretch<R, CPLX>(S, t1, a1, 1, c3[a1], 2 + ((cpt == (a1 + 1) % 3) ? 0 : 1), c3);
                    t2 = stretch<R, CPLX>(S, t2, a2, 1, c3[a2], 2 + ((cpt == (a2 + 1) % 3) ? 0 : 1), c3);
                }
                Vt curl = t1 - t2;
                Vt hv = F.get(3 + cpt, m);
                F.put(3 + cpt, m, hv.scale(a) - curl.scale(b * coef[3 + cpt]));
            }
        }
    }
    }
    if (phase == 1 && t.ne > 0) {
        __syncthreads();
        double part = 0.0;
        for (int e = threadIdx.x; e < t.ne; e += blockDim.x) {
            DevEnt6 en = t.ents[e];
            int64_t g = t.cell0 + en.off;
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

void launch_full(int fp64, int cplx, int dims, const DevSim6 *sims, const DevTile6 *tiles, int ntiles,
                 const int64_t *launch_base, int64_t launch_add, int phase, cudaStream_t st)
{
    if (ntiles <= 0) return;
#define CAS_FULL(R, C, D) k_full<R, C, D><<<ntiles, 256, 0, st>>>(sims, tiles, launch_base, launch_add, phase)
    if (fp64) {
        if (cplx) { if (dims == 2) CAS_FULL(double, true, 2); else CAS_FULL(double, true, 3); }
        else { if (dims == 2) CAS_FULL(double, false, 2); else CAS_FULL(double, false, 3); }
    } else {
        if (cplx) { if (dims == 2) CAS_FULL(float, true, 2); else CAS_FULL(float, true, 3); }
        else { if (dims == 2) CAS_FULL(float, false, 2); else CAS_FULL(float, false, 3); }
    }
#undef CAS_FULL
}

void launch_inject6(int fp64, void *fields, const DevSrc6 *src, int nsrc, cudaStream_t st)
{
    if (nsrc <= 0) return;
    int b = (nsrc + 255) / 256;
    if (fp64) k_inject6<double><<<b, 256, 0, st>>>(reinterpret_cast<double *>(fields), src, nsrc);
    else k_inject6<float><<<b, 256, 0, st>>>(reinterpret_cast<float *>(fields), src, nsrc);
}

}  // namespace cas
