// Six-component leapfrog for two-dimensional cross-sections (d/dz -> i k_z,
// Sec. III B; Bloch-periodic cells, Sec. III D), both half steps in one pass.
//
// The update is the one of step6.cu (CPML of Sec. III B, Lorentz ADE of Eq. (9)
// continued onto the contour, surface functional weighted by w_n = 2 dt
// Im g(-n dt), Eq. (1)), organised as a row march: every warp owns a strip of
// MARCH_W columns and MARCH_H rows of one simulation (lane 0 and lane w + 1
// are halo columns), walks down the rows with x neighbours exchanged by
// shuffles and y neighbours carried in registers, and loads the next row's
// inputs while it computes the current one.  Electric sources update H first
// (E of rows j and j+1 give H of row j), then E; magnetic sources update E one
// row ahead, then H.  Fields, CPML psi and Lorentz P ping-pong between two
// buffers by step parity, so that halo lanes recompute a neighbour's first
// half step from values nobody overwrites.
//
// Storage within one buffer is that of step6.cu: E_x..H_z planes of nx*ny
// elements (real and imaginary planes when complex), psi planes per PML axis
// over its two slabs (planes 0, 1 for the E update, 2, 3 for the H update),
// per Lorentz pole, P then P_prev per E component.
#include <cuda_runtime.h>

#include "kernels.h"

namespace cas {

namespace {

constexpr int WARPS6 = 4;   // warps (strips) per CTA
#ifndef MARCH_PF
#define MARCH_PF 2
#endif
constexpr int PFMAX = MARCH_PF;   // upper bound of the prefetch depth of every variant

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

// Element offsets are 32-bit: a march run's buffer holds fewer than 2^32 elements (checked by the planner).
template <typename R, bool CPLX>
__device__ __forceinline__ Z<R, CPLX> ld(const R *__restrict__ p, int plane, unsigned N, unsigned g)
{
    if constexpr (CPLX) return Z<R, CPLX>(p[(2u * plane) * N + g], p[(2u * plane + 1u) * N + g]);
    else return Z<R, CPLX>(p[(unsigned)plane * N + g]);
}

template <typename R, bool CPLX>
__device__ __forceinline__ void st(R *__restrict__ p, int plane, unsigned N, unsigned g, Z<R, CPLX> v)
{
    if constexpr (CPLX) { p[(2u * plane) * N + g] = v.x; p[(2u * plane + 1u) * N + g] = v.y; }
    else p[(unsigned)plane * N + g] = v.x;
}

// The four Lorentz coefficients [cp, cpm, ce, cd] of one pole and component: a 16-byte aligned
// group of the table (one load in FP32, two in FP64)
template <typename R>
struct Four {
    R v[4];
};
__device__ __forceinline__ Four<float> ld4(const float *__restrict__ p)
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    return Four<float>{{a.x, a.y, a.z, a.w}};
}
__device__ __forceinline__ Four<double> ld4(const double *__restrict__ p)
{
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    return Four<double>{{a.x, a.y, b.x, b.y}};
}

// Asynchronous global -> shared copies of one element (cp.async, the thread's own data): the
// staged march keeps the rows in flight in shared memory instead of registers.
template <typename R>
__device__ __forceinline__ void cpa(R *sdst, const R *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    if constexpr (sizeof(R) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The inputs of one row step, loaded one row ahead.  Electric sources (row j):
// f = E(j+1), q = H(j), m, P(j), psi(j) of all four planes.  Magnetic sources:
// f = H(j+1), q = E(j+1) (old), m of row j+1, P(j+1), psi planes 0, 1 of row j+1
// and 2, 3 of row j.
// P and P_prev of pole q, component k at p[3 q + k], pm[3 q + k] (NPL poles: 0, 1 or 3).
template <typename R, bool CPLX, int NPL>
struct RowIn {
    static constexpr int NP = NPL > 0 ? NPL : 1;
    Z<R, CPLX> f[3], q[3];
    int m;
    Z<R, CPLX> p[3 * NP], pm[3 * NP];
    Z<R, CPLX> px[4], py[4];
    // staged rows: this lane's P values in the row's shared-memory slot (read where they are
    // used, so that the poles' state does not occupy registers); nullptr: p, pm above
    const R *lp = nullptr;
};

// CYL: cylindrical (r, z) lattice (Sec. III C), x = r from the symmetry axis, y = z, stored
// components (E_r, E_z, E_phi, H_r, H_z, H_phi) on the sites of (E_x, E_y, E_z, H_x, H_y, H_z);
// d/dphi -> i m in the real-phase form (kzA, kzB = +-m), per-lane radial factors.
// NPL: Lorentz poles the variant carries (0: no dispersive cell in the tile, 1: one pole at
// most, 3: up to three; a tile takes the smallest that covers its materials).
// PF: rows whose inputs are in flight ahead of the row being computed (1 or 2; 2 where the
// registers allow it without spilling, i.e. without the CPML planes)
// STG > 0: the inputs of the next STG rows are in flight in a per-warp shared-memory ring
// (cp.async of each lane's own elements, STG + 1 slots) instead of registers; PF is unused.
template <typename R, bool CPLX, bool PML, int NPL, int MINB, bool CYL = false, int PFREQ = 1, int STG = 0>
__global__ void __launch_bounds__(WARPS6 * 32, MINB)
k_march6(const DevSim6 *__restrict__ sims, const DevTile *__restrict__ tiles, int ntiles,
         const int64_t *__restrict__ launch_base, int64_t launch_add)
{
    using V = Z<R, CPLX>;
    using In = RowIn<R, CPLX, NPL>;
    constexpr bool LOR = NPL > 0;
    constexpr int PF6 = PFREQ < PFMAX ? PFREQ : PFMAX;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ti = blockIdx.x * WARPS6 + warp;
    if (ti >= ntiles) return;
    const DevTile t = tiles[ti];
    const DevSim6 &S = sims[t.sim];
    const int64_t n = *launch_base + launch_add - S.s0;
    if (n < 1 || n > S.T) return;
    const int nx = S.n[0], ny = S.n[1];
    const unsigned N = (unsigned)nx * (unsigned)ny;
    const int pin_par = (int)((n - 1) & 1), pout_par = (int)(n & 1);
    const R *__restrict__ fin = reinterpret_cast<const R *>(S.fields) + (size_t)pin_par * S.fhalf;
    R *__restrict__ fout = reinterpret_cast<R *>(S.fields) + (size_t)pout_par * S.fhalf;
    const R *__restrict__ coef = reinterpret_cast<const R *>(S.coef);
    const uint8_t *__restrict__ mat = S.mat;
    const int dX = PML ? S.pml_d[0] : 0, dY = PML ? S.pml_d[1] : 0;
    const unsigned PX = PML ? (unsigned)S.slab[0] : 0u, PY = PML ? (unsigned)S.slab[1] : 0u;
    const R *__restrict__ pxin = nullptr, *__restrict__ pyin = nullptr, *__restrict__ profy = nullptr;
    R *__restrict__ pxout = nullptr, *__restrict__ pyout = nullptr;
    if constexpr (PML) {
        const R *psi_in = reinterpret_cast<const R *>(S.psi) + (size_t)pin_par * S.psi_half;
        R *psi_out = reinterpret_cast<R *>(S.psi) + (size_t)pout_par * S.psi_half;
        pxin = psi_in + S.psi_off[0];
        pxout = psi_out + S.psi_off[0];
        pyin = psi_in + S.psi_off[1];
        pyout = psi_out + S.psi_off[1];
        profy = reinterpret_cast<const R *>(S.pml) + S.pml_off[1];   // [half][b, c, 1/kappa][ny]
    }
    const R *__restrict__ lin = nullptr, *__restrict__ lc = nullptr;
    R *__restrict__ lout = nullptr;
    if constexpr (LOR) {
        lin = reinterpret_cast<const R *>(S.lor) + (size_t)pin_par * S.lor_half;
        lout = reinterpret_cast<R *>(S.lor) + (size_t)pout_par * S.lor_half;
        lc = reinterpret_cast<const R *>(S.lorc);                    // [id][pole][3][cp, cpm, ce, cd]
    }
    const int np = LOR ? S.npoles : 0;

    const int i0 = t.i0;
    const int w = min(MARCH_W, nx - i0);
    const int h = min(S.tile_rows, ny - t.j0);
    const int col = ((i0 - 1 + lane) % nx + nx) % nx;     // lane 0: left halo, lane w + 1: right halo
    const bool own = lane >= 1 && lane <= w;
    const bool wrapR = col == nx - 1;                     // the right neighbour lies across the x wrap
    const bool wrapL = col == 0;                          // the left neighbour lies across the x wrap
    const bool inx = PML && dX > 0 && (col < dX || col >= nx - dX);
    const int sx = col < dX ? col : col - (nx - 2 * dX);
    // x profiles of this column: [b, c, 1/kappa] for the E update (integer sites) and the H update
    R xe[3] = {0, 0, 1}, xh[3] = {0, 0, 1};
    if (inx) {
        const R *pr = reinterpret_cast<const R *>(S.pml) + S.pml_off[0];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            xe[k] = pr[k * nx + col];
            xh[k] = pr[(3 + k) * nx + col];
        }
    }
    const R bxr = (R)S.bre[0], bxi = (R)S.bim[0], byr = (R)S.bre[1], byi = (R)S.bim[1];
    const R idx = (R)S.inv_dx;
    const R kA = (R)S.kzA, kB = (R)S.kzB, kc = (R)S.kz;
    const R a = (R)S.a, bs = (R)S.bs;
    const R hfirst = (R)(n == 1 ? 0.5 * S.dt : S.dt);
    const bool electric = S.magnetic == 0;
    const bool first_e = electric && n == 1;              // Lorentz start of electric sources
    // cylindrical radial factors of this lane's column i (r_i = i Delta, r_{i+1/2}, ...):
    //   (1/r) d(r E_phi)/dr at r_{i+1/2} = (ga E_phi(i+1) - gb E_phi(i)) / Delta,
    //   (1/r) d(r H_phi)/dr at r_i = (fa H_phi(i+1/2) - fb H_phi(i-1/2)) / Delta, on the axis
    //   Stokes over the disk of radius Delta/2: 4 H_phi(Delta/2) / Delta (fa = 4, fb = 0)
    R inv_ri = 0, inv_rh = 0, ga = 0, gb = 0, fa = 0, fb = 0;
    if constexpr (CYL) {
        // (Delta cancels from the ratios: each factor is one correctly rounded division of exact
        // operands in the run's precision, so FP32 runs need no FP64 arithmetic per thread)
        const R ci = (R)col, ch = ci + (R)0.5, ix = (R)S.inv_dx;
        inv_ri = col > 0 ? ix / ci : (R)0;
        inv_rh = ix / ch;
        ga = (ci + (R)1) / ch;
        gb = ci / ch;
        fa = col > 0 ? ch / ci : (R)4;
        fb = col > 0 ? (ci - (R)0.5) / ci : (R)0;
    }
    auto rowp = [&](int j) { return j < 0 ? j + ny : (j >= ny ? j - ny : j); };
    auto iny = [&](int j) { return PML && dY > 0 && (j < dY || j >= ny - dY); };
    auto gxi = [&](int j) { return (unsigned)(j * (2 * dX) + sx); };
    auto gyi = [&](int j) { return (unsigned)((j < dY ? j : j - (ny - 2 * dY)) * nx + col); };
    // the material's Lorentz coefficients (ce of pole 0 of component k nonzero: dispersive)
    auto disp = [&](int m, int k) -> bool { if constexpr (LOR) return lc[12 * np * m + 4 * k + 2] != (R)0; else return false; };

    // d/dz of a field of the set {Ex, Ey, Hz} (A) or {Ez, Hx, Hy} (B)
    auto dzA = [&](V f) -> V { if constexpr (CPLX) return f.ik(kc); else return f * kA; };
    auto dzB = [&](V f) -> V { if constexpr (CPLX) return f.ik(kc); else return f * kB; };
    auto right = [&](V f) -> V { V r = f.dn(); return wrapR ? r.ph(bxr, bxi) : r; };
    auto left = [&](V f) -> V { V l = f.up(); return wrapL ? l.ph(bxr, -bxi) : l; };
    // CPML-stretched difference: psi' = b psi + c d; d / kappa + psi'
    auto str = [&](V d, const R *pr, V psi, V &pn) -> V { pn = psi * pr[0] + d * pr[1]; return d * pr[2] + pn; };

    // loads of the psi planes of row j (lo..hi of 0..3) into px / py
    auto load_psi = [&](In &in, int j, int lo, int hi) {
        if constexpr (PML) {
            if (inx) {
                const unsigned g = gxi(j);
                for (int k = lo; k < hi; ++k) in.px[k] = ld<R, CPLX>(pxin, k, PX, g);
            }
            if (iny(j)) {
                const unsigned g = gyi(j);
                for (int k = lo; k < hi; ++k) in.py[k] = ld<R, CPLX>(pyin, k, PY, g);
            }
        }
    };
    // P of the poles material m has at cell g, per component (absent poles: never read)
    auto load_lor = [&](In &in, unsigned g, int m) {
        if constexpr (LOR) {
            const R *lm = lc + 12 * np * m;
#pragma unroll
            for (int q = 0; q < NPL; ++q)
#pragma unroll
                for (int k = 0; k < 3; ++k)
                    if (q < np && lm[12 * q + 4 * k + 2] != (R)0) {
                        in.p[3 * q + k] = ld<R, CPLX>(lin, 6 * q + k, N, g);
                        in.pm[3 * q + k] = ld<R, CPLX>(lin, 6 * q + 3 + k, N, g);
                    }
        }
    };

    // H at row j from E at rows j and j+1: new H, and the H-plane psi (2, 3) written when wr
    auto updH = [&](int j, int m, const V e[3], V exn, V ezn, const V hq[3], const V px[4], const V py[4],
                    R aa, R bb, bool wr, V ho[3]) {
        if (j + 1 >= ny) { exn = exn.ph(byr, byi); ezn = ezn.ph(byr, byi); }
        V dyEz = (ezn - e[2]) * idx, dyEx = (exn - e[0]) * idx;
        V dxEz = (right(e[2]) - e[2]) * idx, dxEy = (right(e[1]) - e[1]) * idx;
        if constexpr (PML) {
            if (inx) {
                V p2, p3;
                const R b2[3] = {xh[0], xh[1], xh[2]};
                dxEz = str(dxEz, b2, px[2], p2);   // H_y
                dxEy = str(dxEy, b2, px[3], p3);   // H_z
                if (wr) { const unsigned g = gxi(j); st<R, CPLX>(pxout, 2, PX, g, p2); st<R, CPLX>(pxout, 3, PX, g, p3); }
            }
            if (iny(j)) {
                const R pr[3] = {profy[3 * ny + j], profy[4 * ny + j], profy[5 * ny + j]};
                V p2, p3;
                dyEx = str(dyEx, pr, py[2], p2);   // H_z
                dyEz = str(dyEz, pr, py[3], p3);   // H_x
                if (wr) { const unsigned g = gyi(j); st<R, CPLX>(pyout, 2, PY, g, p2); st<R, CPLX>(pyout, 3, PY, g, p3); }
            }
        }
        const R *cm = coef + 6 * m;
        if constexpr (CYL) {
            // H_r = -(i m/r E_z - dE_phi/dz), H_z = -((1/r) d(r E_phi)/dr - i m/r E_r),
            // H_phi = -(dE_r/dz - dE_z/dr)
            const V dxEphi = (right(e[2]) * ga - e[2] * gb) * idx;
            ho[0] = hq[0] * aa - (e[1] * (kA * inv_ri) - dyEz) * (bb * cm[3]);
            ho[1] = hq[1] * aa - (dxEphi - e[0] * (kA * inv_rh)) * (bb * cm[4]);
            ho[2] = hq[2] * aa - (dyEx - dxEy) * (bb * cm[5]);
        } else {
            ho[0] = hq[0] * aa - (dyEz - dzA(e[1])) * (bb * cm[3]);
            ho[1] = hq[1] * aa - (dzA(e[0]) - dxEz) * (bb * cm[4]);
            ho[2] = hq[2] * aa - (dxEy - dyEx) * (bb * cm[5]);
        }
    };
    // E at row j from H at rows j and j-1: new E, the E-plane psi (0, 1) and P written when wr
    auto updE = [&](int j, int m, const V hh[3], V hxp, V hzp, const V eo[3], const In &in, R aa, R bb,
                    bool wr, unsigned g, V eo_new[3]) {
        if (j - 1 < 0) { hxp = hxp.ph(byr, -byi); hzp = hzp.ph(byr, -byi); }
        V dyHz = (hh[2] - hzp) * idx, dyHx = (hh[0] - hxp) * idx;
        V dxHz = (hh[2] - left(hh[2])) * idx, dxHy = (hh[1] - left(hh[1])) * idx;
        if constexpr (PML) {
            if (inx) {
                V p0, p1;
                dxHz = str(dxHz, xe, in.px[0], p0);   // E_y
                dxHy = str(dxHy, xe, in.px[1], p1);   // E_z
                if (wr) { const unsigned gg = gxi(j); st<R, CPLX>(pxout, 0, PX, gg, p0); st<R, CPLX>(pxout, 1, PX, gg, p1); }
            }
            if (iny(j)) {
                const R pr[3] = {profy[j], profy[ny + j], profy[2 * ny + j]};
                V p0, p1;
                dyHx = str(dyHx, pr, in.py[0], p0);   // E_z
                dyHz = str(dyHz, pr, in.py[1], p1);   // E_x
                if (wr) { const unsigned gg = gyi(j); st<R, CPLX>(pyout, 0, PY, gg, p0); st<R, CPLX>(pyout, 1, PY, gg, p1); }
            }
        }
        V c3[3];
        if constexpr (CYL) {
            // E_r: i m/r H_z - dH_phi/dz; E_z: (1/r) d(r H_phi)/dr - i m/r H_r; E_phi: dH_r/dz - dH_z/dr
            const V dxHphi = (hh[2] * fa - left(hh[2]) * fb) * idx;
            c3[0] = hh[1] * (kB * inv_rh) - dyHz;
            c3[1] = dxHphi - hh[0] * (kB * inv_ri);
            c3[2] = dyHx - dxHy;
        } else {
            c3[0] = dyHz - dzB(hh[1]);
            c3[1] = dzB(hh[0]) - dxHz;
            c3[2] = dxHy - dyHx;
        }
        const R *cm = coef + 6 * m;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if constexpr (LOR) {
                const R *l4 = lc + 12 * np * m + 4 * k;
                if (l4[2] != (R)0) {
                    // per pole: P^{n+1} = [cp P^n - cpm P^{n-1} + ce E^n] cd (the first electric step
                    // starts from rest); E^{n+1} = a E^n + (a sum P^n - sum P^{n+1} + b curl) / eps_inf
                    V sp = c3[k] * bb;
#pragma unroll
                    for (int q = 0; q < NPL; ++q) {
                        if (q > 0 && q >= np) continue;                      // beyond the plan's poles
                        const Four<R> lq = ld4(l4 + 12 * q);                 // cp, cpm, ce, cd
                        if (q > 0 && lq.v[2] == (R)0) continue;              // pole q absent here
                        const R ce = lq.v[2];
                        V p, pm;
                        if (STG > 0 && in.lp) {
                            // slot layout: P then P_prev of pole q, component k, each CF values 32 apart
                            const R *d = in.lp + 2 * (3 * q + k) * (CPLX ? 2 : 1) * 32;
                            if constexpr (CPLX) { p = V(d[0], d[32]); pm = V(d[64], d[96]); }
                            else { p = V(d[0]); pm = V(d[32]); }
                        } else {
                            p = in.p[3 * q + k];
                            pm = in.pm[3 * q + k];
                        }
                        const V pn = first_e ? (p * lq.v[0] + eo[k] * ce) * (R)0.5
                                             : (p * lq.v[0] - pm * lq.v[1] + eo[k] * ce) * lq.v[3];
                        if (wr) {
                            st<R, CPLX>(lout, 6 * q + k, N, g, pn);
                            st<R, CPLX>(lout, 6 * q + 3 + k, N, g, p);
                        }
                        sp = sp + p * aa - pn;
                    }
                    eo_new[k] = eo[k] * aa + sp * cm[k];
                    continue;
                }
            }
            eo_new[k] = eo[k] * aa + c3[k] * (bb * cm[k]);
        }
    };

    if (w > 0) {
        if constexpr (STG > 0) {
            // value slots of one staged row (in units of V): f[3], q[3], then P, P_prev per pole
            // and component, then the psi planes px[4], py[4]
            constexpr int CF = CPLX ? 2 : 1;
            constexpr int VF = 0, VQ = 3, VP = 6, VX = 6 + 6 * (NPL > 0 ? NPL : 0), VY = VX + 4;
            constexpr int NV = CF * (VX + (PML ? 8 : 0));
            extern __shared__ __align__(16) unsigned char smem6[];
            R *const ring = reinterpret_cast<R *>(smem6) + (size_t)warp * (STG + 1) * NV * 32 + lane;
            auto sg = [&](int slot, int v, const R *p, int plane, unsigned NN, unsigned g) {
                R *d = ring + (slot * NV + v * CF) * 32;
                if constexpr (CPLX) { cpa(d, p + (2u * plane) * NN + g); cpa(d + 32, p + (2u * plane + 1u) * NN + g); }
                else cpa(d, p + (unsigned)plane * NN + g);
            };
            auto fv = [&](int slot, int v) -> V {
                const R *d = ring + (slot * NV + v * CF) * 32;
                if constexpr (CPLX) return V(d[0], d[32]);
                else return V(d[0]);
            };
            // the same predicates as load_psi / load_lor
            auto stage_psi = [&](int slot, int j, int lo, int hi) {
                if constexpr (PML) {
                    if (inx) { const unsigned g = gxi(j); for (int k = lo; k < hi; ++k) sg(slot, VX + k, pxin, k, PX, g); }
                    if (iny(j)) { const unsigned g = gyi(j); for (int k = lo; k < hi; ++k) sg(slot, VY + k, pyin, k, PY, g); }
                }
            };
            auto fetch_psi = [&](int slot, In &in, int j, int lo, int hi) {
                if constexpr (PML) {
                    if (inx) for (int k = lo; k < hi; ++k) in.px[k] = fv(slot, VX + k);
                    if (iny(j)) for (int k = lo; k < hi; ++k) in.py[k] = fv(slot, VY + k);
                }
            };
            auto stage_lor = [&](int slot, unsigned g, int m) {
                if constexpr (LOR) {
                    const R *lm = lc + 12 * np * m;
#pragma unroll
                    for (int q = 0; q < NPL; ++q)
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            if (q < np && lm[12 * q + 4 * k + 2] != (R)0) {
                                sg(slot, VP + 2 * (3 * q + k), lin, 6 * q + k, N, g);
                                sg(slot, VP + 2 * (3 * q + k) + 1, lin, 6 * q + 3 + k, N, g);
                            }
                }
            };
            auto fetch_lor = [&](int slot, In &in, int m) {
                if constexpr (LOR) {
                    const R *lm = lc + 12 * np * m;
#pragma unroll
                    for (int q = 0; q < NPL; ++q)
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            if (q < np && lm[12 * q + 4 * k + 2] != (R)0) {
                                in.p[3 * q + k] = fv(slot, VP + 2 * (3 * q + k));
                                in.pm[3 * q + k] = fv(slot, VP + 2 * (3 * q + k) + 1);
                            }
                }
            };
            const int j0 = t.j0;
            const int jm = rowp(j0 - 1);
            const unsigned gm = (unsigned)(jm * nx + col), g0 = (unsigned)(j0 * nx + col);
            int mr[STG + 1];   // materials of the rows whose inputs are staged next (see below)
            if (electric) {
                // as the register path: H (a = 1, b = h) then E (a, b_sigma), E^n of row j and
                // H^{n+1/2} of row j-1 carried; mr[i] is the material of row j + i
                V e[3], hp[3];
                {
                    In in0;
                    const V em[3] = {ld<R, CPLX>(fin, 0, N, gm), ld<R, CPLX>(fin, 1, N, gm), ld<R, CPLX>(fin, 2, N, gm)};
                    const V hm[3] = {ld<R, CPLX>(fin, 3, N, gm), ld<R, CPLX>(fin, 4, N, gm), ld<R, CPLX>(fin, 5, N, gm)};
#pragma unroll
                    for (int k = 0; k < 3; ++k) e[k] = ld<R, CPLX>(fin, k, N, g0);
                    load_psi(in0, jm, 2, 4);
                    updH(jm, mat[gm], em, e[0], e[2], hm, in0.px, in0.py, (R)1, hfirst, false, hp);
                }
                auto stage_row = [&](int slot, int j, int m) {
                    const unsigned g = (unsigned)(j * nx + col), gn = (unsigned)(rowp(j + 1) * nx + col);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        sg(slot, VF + k, fin, k, N, gn);
                        sg(slot, VQ + k, fin, 3 + k, N, g);
                    }
                    stage_lor(slot, g, m);
                    stage_psi(slot, j, 0, 4);
                };
#pragma unroll
                for (int i = 0; i <= STG; ++i) mr[i] = i < h ? mat[g0 + i * nx] : 0;
#pragma unroll
                for (int i = 0; i < STG; ++i) {
                    if (i < h) stage_row(i, j0 + i, mr[i]);
                    cpa_commit();
                }
                int m_far = STG + 1 < h ? mat[g0 + (STG + 1) * nx] : 0;
                int slot = 0;
                for (int r = 0; r < h; ++r) {
                    const int j = j0 + r;
                    const unsigned g = (unsigned)(j * nx + col);
                    const int sl_in = slot == 0 ? STG : slot - 1;    // (r + STG) mod (STG + 1)
                    if (r + STG < h) stage_row(sl_in, j + STG, mr[STG]);
                    cpa_commit();
                    cpa_wait<STG>();
                    In cur;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        cur.f[k] = fv(slot, VF + k);
                        cur.q[k] = fv(slot, VQ + k);
                    }
                    cur.m = mr[0];
                    if constexpr (LOR) cur.lp = ring + (slot * NV + VP * CF) * 32;
                    fetch_psi(slot, cur, j, 0, 4);
#pragma unroll
                    for (int i = 0; i < STG; ++i) mr[i] = mr[i + 1];
                    mr[STG] = m_far;
                    if (r + STG + 2 < h) m_far = mat[g + (STG + 2) * nx];
                    slot = slot == STG ? 0 : slot + 1;
                    V hn[3], en[3];
                    updH(j, cur.m, e, cur.f[0], cur.f[2], cur.q, cur.px, cur.py, (R)1, hfirst, own, hn);
                    updE(j, cur.m, hn, hp[0], hp[2], e, cur, a, bs, own, g, en);
                    if (own) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            st<R, CPLX>(fout, k, N, g, en[k]);
                            st<R, CPLX>(fout, 3 + k, N, g, hn[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        hp[k] = hn[k];
                        e[k] = cur.f[k];
                    }
                }
            } else {
                // as the register path: E one row ahead, then H; mr[i] is the material of row j + 1 + i
                V hq[3], e[3];
                int m = mat[g0];
                {
                    In in0;
#pragma unroll
                    for (int k = 0; k < 3; ++k) hq[k] = ld<R, CPLX>(fin, 3 + k, N, g0);
                    const V eo[3] = {ld<R, CPLX>(fin, 0, N, g0), ld<R, CPLX>(fin, 1, N, g0), ld<R, CPLX>(fin, 2, N, g0)};
                    load_lor(in0, g0, m);
                    load_psi(in0, j0, 0, 2);
                    updE(j0, m, hq, ld<R, CPLX>(fin, 3, N, gm), ld<R, CPLX>(fin, 5, N, gm), eo, in0, (R)1, hfirst, own, g0, e);
                }
                auto stage_row = [&](int slot, int j, int mn) {
                    const int jn = rowp(j + 1);
                    const unsigned gn = (unsigned)(jn * nx + col);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        sg(slot, VF + k, fin, 3 + k, N, gn);
                        sg(slot, VQ + k, fin, k, N, gn);
                    }
                    stage_lor(slot, gn, mn);
                    stage_psi(slot, jn, 0, 2);
                    stage_psi(slot, j, 2, 4);
                };
#pragma unroll
                for (int i = 0; i <= STG; ++i) mr[i] = i < h ? mat[(unsigned)(rowp(j0 + 1 + i) * nx + col)] : 0;
#pragma unroll
                for (int i = 0; i < STG; ++i) {
                    if (i < h) stage_row(i, j0 + i, mr[i]);
                    cpa_commit();
                }
                int m_far = STG + 1 < h ? mat[(unsigned)(rowp(j0 + STG + 2) * nx + col)] : 0;
                int slot = 0;
                for (int r = 0; r < h; ++r) {
                    const int j = j0 + r, jn = rowp(j + 1);
                    const unsigned g = (unsigned)(j * nx + col), gn = (unsigned)(jn * nx + col);
                    const int sl_in = slot == 0 ? STG : slot - 1;
                    if (r + STG < h) stage_row(sl_in, j + STG, mr[STG]);
                    cpa_commit();
                    cpa_wait<STG>();
                    In cur;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        cur.f[k] = fv(slot, VF + k);
                        cur.q[k] = fv(slot, VQ + k);
                    }
                    cur.m = mr[0];
                    if constexpr (LOR) cur.lp = ring + (slot * NV + VP * CF) * 32;
                    fetch_psi(slot, cur, jn, 0, 2);
                    fetch_psi(slot, cur, j, 2, 4);
#pragma unroll
                    for (int i = 0; i < STG; ++i) mr[i] = mr[i + 1];
                    mr[STG] = m_far;
                    if (r + STG + 2 < h) m_far = mat[(unsigned)(rowp(j + STG + 3) * nx + col)];
                    slot = slot == STG ? 0 : slot + 1;
                    V en[3], hn[3];
                    updE(jn, cur.m, cur.f, hq[0], hq[2], cur.q, cur, (R)1, hfirst, own && r + 1 < h, gn, en);
                    updH(j, m, e, en[0], en[2], hq, cur.px, cur.py, a, bs, own, hn);
                    if (own) {
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            st<R, CPLX>(fout, k, N, g, e[k]);
                            st<R, CPLX>(fout, 3 + k, N, g, hn[k]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        e[k] = en[k];
                        hq[k] = cur.f[k];
                    }
                    m = cur.m;
                }
            }
        } else {
        const int j0 = t.j0;
        const int jm = rowp(j0 - 1);
        const unsigned gm = (unsigned)(jm * nx + col), g0 = (unsigned)(j0 * nx + col);
        In cur, nxt, nx2;
        if (electric) {
            // H (a = 1, b = h) then E (a, b_sigma).  Carried: E^n of row j, H^{n+1/2} of row j-1.
            // The material of row j+2 is loaded at row j, so that P of row j+1 loads only where dispersive.
            V e[3], hp[3];
            {
                In in0;
                const V em[3] = {ld<R, CPLX>(fin, 0, N, gm), ld<R, CPLX>(fin, 1, N, gm), ld<R, CPLX>(fin, 2, N, gm)};
                const V hm[3] = {ld<R, CPLX>(fin, 3, N, gm), ld<R, CPLX>(fin, 4, N, gm), ld<R, CPLX>(fin, 5, N, gm)};
#pragma unroll
                for (int k = 0; k < 3; ++k) e[k] = ld<R, CPLX>(fin, k, N, g0);
                load_psi(in0, jm, 2, 4);
                updH(jm, mat[gm], em, e[0], e[2], hm, in0.px, in0.py, (R)1, hfirst, false, hp);
            }
            auto load_row = [&](In &in, int j, int m) {
                const unsigned g = (unsigned)(j * nx + col), gn = (unsigned)(rowp(j + 1) * nx + col);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    in.f[k] = ld<R, CPLX>(fin, k, N, gn);
                    in.q[k] = ld<R, CPLX>(fin, 3 + k, N, g);
                }
                in.m = m;
                load_lor(in, g, m);
                load_psi(in, j, 0, 4);
            };
            load_row(cur, j0, mat[g0]);
            if (PF6 == 2 && h > 1) load_row(nxt, j0 + 1, mat[g0 + nx]);
            // material of the next row to load (row j0 + PF6), loaded one row before its fields
            int m_ahead = h > PF6 ? mat[g0 + PF6 * nx] : 0;
            for (int r = 0; r < h; ++r) {
                const int j = j0 + r;
                const unsigned g = (unsigned)(j * nx + col);
                if (r + PF6 < h) {
                    load_row(PF6 == 2 ? nx2 : nxt, j + PF6, m_ahead);
                    if (r + PF6 + 1 < h) m_ahead = mat[g + (PF6 + 1) * nx];
                }
                V hn[3], en[3];
                updH(j, cur.m, e, cur.f[0], cur.f[2], cur.q, cur.px, cur.py, (R)1, hfirst, own, hn);
                updE(j, cur.m, hn, hp[0], hp[2], e, cur, a, bs, own, g, en);
                if (own) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        st<R, CPLX>(fout, k, N, g, en[k]);
                        st<R, CPLX>(fout, 3 + k, N, g, hn[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    hp[k] = hn[k];
                    e[k] = cur.f[k];
                }
                cur = nxt;
                if (PF6 == 2) nxt = nx2;
            }
        } else {
            // E (a = 1, b = h) one row ahead, then H (a, b_sigma).  Carried: H^n of row j, E^{n+1} of row j.
            V hq[3], e[3];
            int m = mat[g0];
            {
                In in0;
#pragma unroll
                for (int k = 0; k < 3; ++k) hq[k] = ld<R, CPLX>(fin, 3 + k, N, g0);
                const V eo[3] = {ld<R, CPLX>(fin, 0, N, g0), ld<R, CPLX>(fin, 1, N, g0), ld<R, CPLX>(fin, 2, N, g0)};
                load_lor(in0, g0, m);
                load_psi(in0, j0, 0, 2);
                updE(j0, m, hq, ld<R, CPLX>(fin, 3, N, gm), ld<R, CPLX>(fin, 5, N, gm), eo, in0, (R)1, hfirst, own, g0, e);
            }
            // inputs of row step j: row j+1 (fields, material mn, P) and the H-plane psi of row j
            auto load_row = [&](In &in, int j, int mn) {
                const int jn = rowp(j + 1);
                const unsigned gn = (unsigned)(jn * nx + col);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    in.f[k] = ld<R, CPLX>(fin, 3 + k, N, gn);
                    in.q[k] = ld<R, CPLX>(fin, k, N, gn);
                }
                in.m = mn;
                load_lor(in, gn, mn);
                load_psi(in, jn, 0, 2);
                load_psi(in, j, 2, 4);
            };
            load_row(cur, j0, mat[(unsigned)(rowp(j0 + 1) * nx + col)]);
            if (PF6 == 2 && h > 1) load_row(nxt, j0 + 1, mat[(unsigned)(rowp(j0 + 2) * nx + col)]);
            // material of the row after the next one to load (its fields arrive one row later)
            int m_ahead = h > PF6 ? mat[(unsigned)(rowp(j0 + PF6 + 1) * nx + col)] : 0;
            for (int r = 0; r < h; ++r) {
                const int j = j0 + r, jn = rowp(j + 1);
                const unsigned g = (unsigned)(j * nx + col), gn = (unsigned)(jn * nx + col);
                if (r + PF6 < h) {
                    load_row(PF6 == 2 ? nx2 : nxt, j + PF6, m_ahead);
                    if (r + PF6 + 1 < h) m_ahead = mat[(unsigned)(rowp(j + PF6 + 2) * nx + col)];
                }
                V en[3], hn[3];
                // E of row j + 1: psi and P written only for rows of this strip
                updE(jn, cur.m, cur.f, hq[0], hq[2], cur.q, cur, (R)1, hfirst, own && r + 1 < h, gn, en);
                updH(j, m, e, en[0], en[2], hq, cur.px, cur.py, a, bs, own, hn);
                if (own) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        st<R, CPLX>(fout, k, N, g, e[k]);
                        st<R, CPLX>(fout, 3 + k, N, g, hn[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    e[k] = en[k];
                    hq[k] = cur.f[k];
                }
                m = cur.m;
                cur = nxt;
                if (PF6 == 2) nxt = nx2;
            }
        }
            }
    }

    if (t.ne > 0) {
        __syncwarp();   // the strip's field writes are visible to the warp
        double part = 0.0;
        for (int e = lane; e < t.ne; e += 32) {
            const DevEnt en = t.ents[e];
            const int loc = en.loc & 0xffff, arr = (en.loc >> 16) & 7, im = (en.loc >> 19) & 1;
            const int ly = loc / MARCH_W, lx = loc - ly * MARCH_W;
            const unsigned g = (unsigned)((t.j0 + ly) * nx + i0 + lx);
            const unsigned plane = CPLX ? (unsigned)(2 * arr + im) : (unsigned)arr;
            // Re(w v) = w_re v_re - w_im v_im: the imaginary weight enters with a minus sign
            part += (im ? -en.w : en.w) * (double)fout[plane * N + g];
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) {
            const double c = S.gw[n - 1] * part;
            atomicAdd(S.acc, c);
            if (n > S.tail_from) atomicAdd(S.tail, c);
        }
    }
}

// Rows staged ahead in shared memory (cp.async) by the non-cylindrical variants.  Measured on
// GB300 against the register prefetch: two staged rows move the FP32 real-field variants 5%
// faster (waveguides with CPML and a Lorentz pole) and the FP32 dispersive complex ones 8%
// (silicon/silica grating); four rows cost occupancy through shared memory (the complex Bloch
// grating 18% slower).  The FP32 complex non-dispersive variants (no gain) and the FP64 ones
// (bound by FP64 arithmetic, where the extra shared-memory reads only add instructions) keep
// the register prefetch.  At most MARCH_STG rows, within about 56 KB per CTA.
#ifndef MARCH_STG
#define MARCH_STG 2
#endif
constexpr int kStageBudget = 56 * 1024;

template <typename R, bool CPLX, bool PML, int NPL>
constexpr size_t slot_bytes()
{
    return (size_t)WARPS6 * 32 * (CPLX ? 2 : 1) * (6 + 6 * NPL + (PML ? 8 : 0)) * sizeof(R);
}

template <typename R, bool CPLX, bool PML, int NPL>
constexpr int stage_depth()
{
    if (sizeof(R) != 4 || (CPLX && NPL == 0) || MARCH_STG <= 0) return 0;
    const int fit = (int)(kStageBudget / slot_bytes<R, CPLX, PML, NPL>()) - 1;
    return fit < 1 ? 1 : (fit > MARCH_STG ? MARCH_STG : fit);
}

template <typename R, bool CPLX, bool PML, int NPL, int MINB, int PF>
struct Variant {
    static constexpr int STG = stage_depth<R, CPLX, PML, NPL>();
    static constexpr size_t SMEM = STG > 0 ? (STG + 1) * slot_bytes<R, CPLX, PML, NPL>() : 0;
    static cudaError_t prepare()
    {
        if (SMEM <= 48 * 1024) return cudaSuccess;
        return cudaFuncSetAttribute(k_march6<R, CPLX, PML, NPL, MINB, false, PF, STG>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    }
    static void launch(int grid, const DevSim6 *sims, const DevTile *tiles, int ntiles, const int64_t *lb, int64_t la,
                       cudaStream_t st)
    {
        k_march6<R, CPLX, PML, NPL, MINB, false, PF, STG><<<grid, WARPS6 * 32, SMEM, st>>>(sims, tiles, ntiles, lb, la);
    }
};

// MINB per variant (none, CPML, one pole, one pole + CPML, three poles, three poles + CPML):
// resident CTAs per SM asked of the register allocator
template <typename R, bool CPLX, int M0, int M1, int M2, int M3, int M4, int M5>
struct Variants {
    using V0 = Variant<R, CPLX, false, 0, M0, 2>;
    using V1 = Variant<R, CPLX, true, 0, M1, 1>;
    using V2 = Variant<R, CPLX, false, 1, M2, 2>;
    using V3 = Variant<R, CPLX, true, 1, M3, 1>;
    using V4 = Variant<R, CPLX, false, 3, M4, 1>;
    using V5 = Variant<R, CPLX, true, 3, M5, 1>;
    static cudaError_t prepare()
    {
        for (cudaError_t e : {V0::prepare(), V1::prepare(), V2::prepare(), V3::prepare(), V4::prepare(), V5::prepare()})
            if (e != cudaSuccess) return e;
        return cudaSuccess;
    }
    static void launch(int variant, const DevSim6 *sims, const DevTile *tiles, int ntiles, const int64_t *lb,
                       int64_t la, cudaStream_t st)
    {
        const int grid = (ntiles + WARPS6 - 1) / WARPS6;
        switch (variant) {
        case 0: V0::launch(grid, sims, tiles, ntiles, lb, la, st); break;
        case 1: V1::launch(grid, sims, tiles, ntiles, lb, la, st); break;
        case 2: V2::launch(grid, sims, tiles, ntiles, lb, la, st); break;
        case 3: V3::launch(grid, sims, tiles, ntiles, lb, la, st); break;
        case 4: V4::launch(grid, sims, tiles, ntiles, lb, la, st); break;
        default: V5::launch(grid, sims, tiles, ntiles, lb, la, st); break;
        }
    }
};

using VarD1 = Variants<double, true, 3, 2, 2, 1, 1, 1>;
using VarD0 = Variants<double, false, 4, 3, 3, 2, 2, 2>;
#ifndef MARCH_F1_M1
#define MARCH_F1_M1 4
#endif
#ifndef MARCH_F1_M45
#define MARCH_F1_M45 2
#endif
using VarF1 = Variants<float, true, 4, MARCH_F1_M1, 3, 3, MARCH_F1_M45, MARCH_F1_M45>;
using VarF0 = Variants<float, false, 7, 5, 6, 5, 4, 4>;

}  // namespace

void launch_march6_cyl(int fp64, const DevSim6 *sims, const DevTile *tiles, int ntiles,
                       const int64_t *launch_base, int64_t launch_add, cudaStream_t st)
{
    if (ntiles <= 0) return;
    const int grid = (ntiles + WARPS6 - 1) / WARPS6;
    // real fields without CPML or poles: the staging policy of the real-field variants
    constexpr int SD = stage_depth<double, false, false, 0>(), SF = stage_depth<float, false, false, 0>();
    constexpr size_t BD = SD > 0 ? (SD + 1) * slot_bytes<double, false, false, 0>() : 0;
    constexpr size_t BF = SF > 0 ? (SF + 1) * slot_bytes<float, false, false, 0>() : 0;
    static_assert(BD <= 48 * 1024 && BF <= 48 * 1024, "cylindrical march: no opt-in shared memory");
    if (fp64) k_march6<double, false, false, 0, 4, true, 2, SD><<<grid, WARPS6 * 32, BD, st>>>(sims, tiles, ntiles, launch_base, launch_add);
    else k_march6<float, false, false, 0, 6, true, 2, SF><<<grid, WARPS6 * 32, BF, st>>>(sims, tiles, ntiles, launch_base, launch_add);
}

void launch_march6(int fp64, int cplx, int variant, const DevSim6 *sims, const DevTile *tiles, int ntiles,
                   const int64_t *launch_base, int64_t launch_add, cudaStream_t st)
{
    if (ntiles <= 0) return;
    if (fp64) {
        if (cplx) VarD1::launch(variant, sims, tiles, ntiles, launch_base, launch_add, st);
        else VarD0::launch(variant, sims, tiles, ntiles, launch_base, launch_add, st);
    } else {
        if (cplx) VarF1::launch(variant, sims, tiles, ntiles, launch_base, launch_add, st);
        else VarF0::launch(variant, sims, tiles, ntiles, launch_base, launch_add, st);
    }
}

cudaError_t march6_prepare()
{
    for (cudaError_t e : {VarD1::prepare(), VarD0::prepare(), VarF1::prepare(), VarF0::prepare()})
        if (e != cudaSuccess) return e;
    return cudaSuccess;
}

}  // namespace cas
