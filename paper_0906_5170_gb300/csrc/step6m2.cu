// Two leapfrog steps per launch for two-dimensional six-component runs (k_z cross-sections of
// Sec. III B, Bloch-periodic cells of Sec. III D) with CPML (Sec. III B) and at most one
// undamped Lorentz pole per material (Eq. (9) on the contour).
//
// The update of the march in step6m.cu (curls with d/dz -> i k_z, or +-k_z on the real-phase
// split; wrapped neighbours times the Bloch factors; the stretched CPML differences psi' =
// b psi + c d, d / kappa + psi'; P' = [cp P - cpm P_prev + ce E] cd per pole, with the centred
// start of electric sources at n = 1), fused over two consecutive steps A = 2L-1 and B = 2L as
// in the cylindrical two-step march (step6c2.cu): a warp owns a strip of MARCH_W2 = 28 columns
// plus two halo lanes on each side (each step leaves one more outer lane stale) and marches down
// the tile's rows; electric sources update H then E, step B one row behind step A; magnetic
// sources update E one row ahead then H, step B's E at step A's H row.  Step A's CPML psi and
// Lorentz P of a row are kept in registers until step B reaches the row; fields, psi and P read
// buffer (L-1)&1 and write buffer L&1 (step B's values, or step A's when the launch holds one
// step).  The sigma group of both steps is projected from registers (row-sorted entries,
// shuffle hand-over; complex weights carry the imaginary part in bit 19).
#include <cuda_runtime.h>

#include "kernels.h"

namespace cas {

namespace {

constexpr int WARPS_M2 = 4;   // warps (strips) per CTA

template <bool B>
struct Flag {
    static constexpr bool value = B;
};

// resident CTAs per SM of each variant (registers without spills): real / complex fields,
// 0 = interior, 1 = CPML, 2 = Lorentz, 3 = both
// row steps whose inputs are staged ahead (0: register prefetch of the next row)
#ifndef MAR2_STG
#define MAR2_STG 1
#endif
#ifndef MAR2_R0
#define MAR2_R0 5
#endif
#ifndef MAR2_R1
#define MAR2_R1 4
#endif
#ifndef MAR2_R2
#define MAR2_R2 4
#endif
#ifndef MAR2_R3
#define MAR2_R3 3
#endif
#ifndef MAR2_C0
#define MAR2_C0 4
#endif
#ifndef MAR2_C1
#define MAR2_C1 3
#endif
#ifndef MAR2_C2
#define MAR2_C2 3
#endif
#ifndef MAR2_C3
#define MAR2_C3 2
#endif

template <typename R, bool CPLX>
struct Y;

template <typename R>
struct Y<R, false> {
    R x;
    __device__ Y() : x(0) {}
    __device__ explicit Y(R a) : x(a) {}
    __device__ Y operator+(Y o) const { return Y(x + o.x); }
    __device__ Y operator-(Y o) const { return Y(x - o.x); }
    __device__ Y operator*(R s) const { return Y(x * s); }
    __device__ Y ph(R c, R) const { return Y(x * c); }
    __device__ Y dn() const { return Y(__shfl_down_sync(0xffffffffu, x, 1)); }
    __device__ Y up() const { return Y(__shfl_up_sync(0xffffffffu, x, 1)); }
    __device__ Y from(int src) const { return Y(__shfl_sync(0xffffffffu, x, src)); }
};

template <typename R>
struct Y<R, true> {
    R x, y;
    __device__ Y() : x(0), y(0) {}
    __device__ Y(R a, R b) : x(a), y(b) {}
    __device__ Y operator+(Y o) const { return Y(x + o.x, y + o.y); }
    __device__ Y operator-(Y o) const { return Y(x - o.x, y - o.y); }
    __device__ Y operator*(R s) const { return Y(x * s, y * s); }
    __device__ Y ph(R c, R s) const { return Y(x * c - y * s, x * s + y * c); }
    __device__ Y ik(R k) const { return Y(-y * k, x * k); }
    __device__ Y dn() const { return Y(__shfl_down_sync(0xffffffffu, x, 1), __shfl_down_sync(0xffffffffu, y, 1)); }
    __device__ Y up() const { return Y(__shfl_up_sync(0xffffffffu, x, 1), __shfl_up_sync(0xffffffffu, y, 1)); }
    __device__ Y from(int src) const { return Y(__shfl_sync(0xffffffffu, x, src), __shfl_sync(0xffffffffu, y, src)); }
};

template <typename R, bool CPLX>
__device__ __forceinline__ Y<R, CPLX> ldy(const R *__restrict__ p, int plane, unsigned NN, unsigned g)
{
    if constexpr (CPLX) return Y<R, CPLX>(p[(2u * plane) * NN + g], p[(2u * plane + 1u) * NN + g]);
    else return Y<R, CPLX>(p[(unsigned)plane * NN + g]);
}

template <typename R, bool CPLX>
__device__ __forceinline__ void sty(R *__restrict__ p, int plane, unsigned NN, unsigned g, Y<R, CPLX> v)
{
    if constexpr (CPLX) { p[(2u * plane) * NN + g] = v.x; p[(2u * plane + 1u) * NN + g] = v.y; }
    else p[(unsigned)plane * NN + g] = v.x;
}

// Asynchronous global -> shared copy of one element (cp.async of the lane's own value): staged
// rows keep the inputs of the next STG row steps in flight in shared memory instead of registers.
template <typename R>
__device__ __forceinline__ void cpa(R *sdst, const R *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Projection of the sigma group's three components at tile row ly (entries rowptr[ly] ..
// rowptr[ly+1], loc = ly * MARCH_W2 + lx, the component in bits 16..18, bit 19 for the weight of
// the imaginary part): lanes 2 .. w + 1 hold the strip's columns.
template <typename R, bool CPLX>
__device__ __forceinline__ double project_row_m2(const DevTile2 &t, int ly, int w, int grp, Y<R, CPLX> v0,
                                                 Y<R, CPLX> v1, Y<R, CPLX> v2)
{
    double part = 0.0;
    const int e0 = t.rowptr[ly], e1 = t.rowptr[ly + 1];
    for (int base = e0; base < e1; base += 32) {
        const int e = base + (int)(threadIdx.x & 31);
        int c = 0, lx = -1, im = 0;
        double wgt = 0.0;
        if (e < e1) {
            const DevEnt en = t.ents[e];
            lx = (en.loc & 0xffff) - ly * MARCH_W2;
            c = ((en.loc >> 16) & 7) - grp;
            im = (en.loc >> 19) & 1;
            wgt = en.w;
        }
        const bool mine = lx >= 0 && lx < w;
        const int src = mine ? lx + 2 : 0;
        const Y<R, CPLX> a0 = v0.from(src), a1 = v1.from(src), a2 = v2.from(src);
        if (mine) {
            const Y<R, CPLX> v = c == 0 ? a0 : (c == 1 ? a1 : a2);
            if constexpr (CPLX) part += im ? -wgt * (double)v.y : wgt * (double)v.x;
            else part += wgt * (double)v.x;
        }
    }
    return part;
}

// CPML psi of one group at one row: the two x planes and the two y planes the group updates
template <typename R, bool CPLX>
struct Psi {
    Y<R, CPLX> x[2], y[2];
};

// LOR: one undamped Lorentz pole at most (P, P_prev per E component).
// STG > 0: the inputs of the next STG row steps (fields, CPML psi, P) are in flight in a per-lane
// shared-memory ring of STG + 1 slots, copied by cp.async; STG = 0: the next row's fields are
// prefetched into registers and psi and P are loaded where they are used.
template <typename R, bool CPLX, bool PML, bool LOR, int MINB, int STG>
__global__ void __launch_bounds__(WARPS_M2 * 32, MINB)
k_mar2(const DevSim6 *__restrict__ sims, const DevTile2 *__restrict__ tiles, int ntiles,
       const int64_t *__restrict__ launch_base, int64_t launch_add)
{
    using V = Y<R, CPLX>;
    using PS = Psi<R, CPLX>;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ti = blockIdx.x * WARPS_M2 + warp;
    if (ti >= ntiles) return;
    const DevTile2 t = tiles[ti];
    const DevSim6 &S = sims[t.sim];
    const int64_t L = *launch_base + launch_add - S.s0;
    const int64_t nA = 2 * L - 1;
    if (L < 1 || nA > S.T) return;
    const bool two = nA + 1 <= S.T;

    const int nx = S.n[0], ny = S.n[1];
    const unsigned N = (unsigned)nx * (unsigned)ny;   // 32-bit offsets: 12 max(1, poles) N < 2^32 (planner)
    const int pin = (int)((L - 1) & 1), pout = (int)(L & 1);
    const R *__restrict__ fin = reinterpret_cast<const R *>(S.fields) + (size_t)pin * S.fhalf;
    R *__restrict__ fout = reinterpret_cast<R *>(S.fields) + (size_t)pout * S.fhalf;
    const R *__restrict__ coef = reinterpret_cast<const R *>(S.coef);
    const uint8_t *__restrict__ mat = S.mat;
    int dX = 0, dY = 0;
    unsigned PX = 0u, PY = 0u;
    const R *__restrict__ pxin = nullptr, *__restrict__ pyin = nullptr, *__restrict__ profy = nullptr;
    R *__restrict__ pxout = nullptr, *__restrict__ pyout = nullptr;
    if constexpr (PML) {
        dX = S.pml_d[0];
        dY = S.pml_d[1];
        PX = (unsigned)S.slab[0];
        PY = (unsigned)S.slab[1];
        const R *psi_in = reinterpret_cast<const R *>(S.psi) + (size_t)pin * S.psi_half;
        R *psi_out = reinterpret_cast<R *>(S.psi) + (size_t)pout * S.psi_half;
        pxin = psi_in + S.psi_off[0];
        pxout = psi_out + S.psi_off[0];
        pyin = psi_in + S.psi_off[1];
        pyout = psi_out + S.psi_off[1];
        profy = reinterpret_cast<const R *>(S.pml) + S.pml_off[1];   // [half][b, c, 1/kappa][ny]
    }
    const R *__restrict__ lin = nullptr, *__restrict__ lc = nullptr;
    R *__restrict__ lout = nullptr;
    if constexpr (LOR) {
        lin = reinterpret_cast<const R *>(S.lor) + (size_t)pin * S.lor_half;
        lout = reinterpret_cast<R *>(S.lor) + (size_t)pout * S.lor_half;
        lc = reinterpret_cast<const R *>(S.lorc);                    // [id][pole][3][cp, cpm, ce, cd]
    }
    const int np = LOR ? S.npoles : 0;

    const int i0 = t.i0;
    const int w = min(MARCH_W2, nx - i0);
    const int h = min(S.tile_rows, ny - t.j0);
    const int col = ((i0 - 2 + lane) % nx + nx) % nx;   // lanes 0, 1 and w + 2, w + 3: halo columns
    const bool own = lane >= 2 && lane < w + 2;
    const bool wrapR = col == nx - 1, wrapL = col == 0;
    const bool inx = PML && dX > 0 && (col < dX || col >= nx - dX);
    const int sx = col < dX ? col : col - (nx - 2 * dX);
    R xe[3] = {0, 0, 1}, xh[3] = {0, 0, 1};   // x profiles of this column: E update, H update
    if constexpr (PML) {
        if (inx) {
            const R *pr = reinterpret_cast<const R *>(S.pml) + S.pml_off[0];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                xe[k] = pr[k * nx + col];
                xh[k] = pr[(3 + k) * nx + col];
            }
        }
    }
    const R bxr = (R)S.bre[0], bxi = (R)S.bim[0], byr = (R)S.bre[1], byi = (R)S.bim[1];
    const R idx = (R)S.inv_dx;
    const R kA = (R)S.kzA, kB = (R)S.kzB, kc = (R)S.kz;
    const R a = (R)S.a, bs = (R)S.bs;
    const R hA0 = (R)(nA == 1 ? 0.5 * S.dt : S.dt), hB0 = (R)S.dt;
    const bool electric = S.magnetic == 0;
    const bool firstA = electric && nA == 1;   // Lorentz start of electric sources (step A of the first launch)
    const int grp = electric ? 0 : 3;          // the measured (sigma) group

    auto wrow = [&](int j) { j %= ny; return j < 0 ? j + ny : j; };
    auto iny = [&](int j) { return PML && dY > 0 && (j < dY || j >= ny - dY); };
    auto gxi = [&](int j) { return (unsigned)(j * (2 * dX) + sx); };
    auto gyi = [&](int j) { return (unsigned)((j < dY ? j : j - (ny - 2 * dY)) * nx + col); };
    auto ldf = [&](int plane, int j) -> V { return ldy<R, CPLX>(fin, plane, N, (unsigned)(j * nx + col)); };
    auto dzA = [&](V f) -> V { if constexpr (CPLX) return f.ik(kc); else return f * kA; };
    auto dzB = [&](V f) -> V { if constexpr (CPLX) return f.ik(kc); else return f * kB; };
    auto right = [&](V f) -> V { V r = f.dn(); return wrapR ? r.ph(bxr, bxi) : r; };
    auto left = [&](V f) -> V { V l = f.up(); return wrapL ? l.ph(bxr, -bxi) : l; };
    auto str = [&](V d, const R *pr, V psi, V &pn) -> V { pn = psi * pr[0] + d * pr[1]; return d * pr[2] + pn; };
    // the psi a group reads at (wrapped) row j from the input buffer: planes lo, lo + 1 of x and y
    auto psi_in_row = [&](int j, int lo) -> PS {
        PS p;
        if constexpr (PML) {
            if (inx) { const unsigned g = gxi(j); p.x[0] = ldy<R, CPLX>(pxin, lo, PX, g); p.x[1] = ldy<R, CPLX>(pxin, lo + 1, PX, g); }
            if (iny(j)) { const unsigned g = gyi(j); p.y[0] = ldy<R, CPLX>(pyin, lo, PY, g); p.y[1] = ldy<R, CPLX>(pyin, lo + 1, PY, g); }
        }
        return p;
    };
    auto psi_store = [&](int j, int lo, const PS &p) {
        if constexpr (PML) {
            if (!own) return;
            if (inx) { const unsigned g = gxi(j); sty<R, CPLX>(pxout, lo, PX, g, p.x[0]); sty<R, CPLX>(pxout, lo + 1, PX, g, p.x[1]); }
            if (iny(j)) { const unsigned g = gyi(j); sty<R, CPLX>(pyout, lo, PY, g, p.y[0]); sty<R, CPLX>(pyout, lo + 1, PY, g, p.y[1]); }
        }
    };

    // staged rows: slot layout in values V of CF reals each, 32 apart per real: fields 0..5, then
    // psi x planes 0..3 and y planes 0..3 (CPML), then P, P_prev of E_x..E_z (Lorentz)
    constexpr int CF = CPLX ? 2 : 1;
    constexpr int VX = 6, VY = 10, VL = PML ? 14 : 6;
    constexpr int NV = CF * (VL + (LOR ? 6 : 0));
    constexpr int NSLOT = STG > 0 ? STG + 1 : 1;
    __shared__ __align__(16) R ring_s[STG > 0 ? WARPS_M2 * NSLOT * NV * 32 : 1];
    R *const ring = ring_s + (STG > 0 ? warp * NSLOT * NV * 32 + lane : 0);
    auto sg = [&](int sl, int v, const R *p, int plane, unsigned NN, unsigned g) {
        R *d = ring + (sl * NV + v * CF) * 32;
        if constexpr (CPLX) { cpa(d, p + (2u * plane) * NN + g); cpa(d + 32, p + (2u * plane + 1u) * NN + g); }
        else cpa(d, p + (unsigned)plane * NN + g);
    };
    auto fv = [&](int sl, int v) -> V {
        const R *d = ring + (sl * NV + v * CF) * 32;
        if constexpr (CPLX) return V(d[0], d[32]);
        else return V(d[0]);
    };
    auto disp = [&](int m, int k) -> bool { if constexpr (LOR) return lc[12 * np * m + 4 * k + 2] != (R)0; else return false; };
    // psi planes lo.. of x at row jx and of y at row jy into slot values VX + lo.., VY + lo..
    auto stage_psi = [&](int sl, int jx, int jy, int lo, int hi) {
        if constexpr (PML) {
            if (inx) { const unsigned g = gxi(jx); for (int q = lo; q < hi; ++q) sg(sl, VX + q, pxin, q, PX, g); }
            if (iny(jy)) { const unsigned g = gyi(jy); for (int q = lo; q < hi; ++q) sg(sl, VY + q, pyin, q, PY, g); }
        }
    };
    auto stage_lor = [&](int sl, int j, int m) {
        if constexpr (LOR) {
            const unsigned g = (unsigned)(j * nx + col);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (disp(m, k)) { sg(sl, VL + 2 * k, lin, k, N, g); sg(sl, VL + 2 * k + 1, lin, 3 + k, N, g); }
        }
    };
    // the psi of group planes lo, lo + 1 (x at row j's column, y at row j) from slot sl
    auto psi_slot = [&](int sl, int j, int lo) -> PS {
        PS p;
        if constexpr (PML) {
            if (inx) { p.x[0] = fv(sl, VX + lo); p.x[1] = fv(sl, VX + lo + 1); }
            if (iny(j)) { p.y[0] = fv(sl, VY + lo); p.y[1] = fv(sl, VY + lo + 1); }
        }
        return p;
    };
    auto lor_slot = [&](int sl, int m, V pp[3], V pm[3]) {
        if constexpr (LOR) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (disp(m, k)) { pp[k] = fv(sl, VL + 2 * k); pm[k] = fv(sl, VL + 2 * k + 1); }
                else { pp[k] = V(); pm[k] = V(); }
            }
        }
    };
    auto matw = [&](int row) -> int { return mat[(unsigned)(wrow(row) * nx + col)]; };

    // H at (wrapped) row j from E at rows j and j+1 (E_x, E_z of row j+1: exn, ezn); psi planes 2, 3
    auto updH = [&](int j, int m, const V e[3], V exn, V ezn, const V hq[3], R aa, R bb, const PS &pi, PS &po, V ho[3]) {
        if (j + 1 >= ny) { exn = exn.ph(byr, byi); ezn = ezn.ph(byr, byi); }
        V dyEz = (ezn - e[2]) * idx, dyEx = (exn - e[0]) * idx;
        V dxEz = (right(e[2]) - e[2]) * idx, dxEy = (right(e[1]) - e[1]) * idx;
        if constexpr (PML) {
            if (inx) {
                dxEz = str(dxEz, xh, pi.x[0], po.x[0]);   // H_y
                dxEy = str(dxEy, xh, pi.x[1], po.x[1]);   // H_z
            }
            if (iny(j)) {
                const R pr[3] = {profy[3 * ny + j], profy[4 * ny + j], profy[5 * ny + j]};
                dyEx = str(dyEx, pr, pi.y[0], po.y[0]);   // H_z
                dyEz = str(dyEz, pr, pi.y[1], po.y[1]);   // H_x
            }
        }
        const R *cm = coef + 6 * m;
        ho[0] = hq[0] * aa - (dyEz - dzA(e[1])) * (bb * cm[3]);
        ho[1] = hq[1] * aa - (dzA(e[0]) - dxEz) * (bb * cm[4]);
        ho[2] = hq[2] * aa - (dxEy - dyEx) * (bb * cm[5]);
    };
    // E at (wrapped) row j from H at rows j and j-1 (H_x, H_z of row j-1: hxp, hzp); psi planes 0, 1;
    // one pole per component: pp = P, pm = P_prev before the step, pn = P after it
    auto updE = [&](int j, int m, const V hh[3], V hxp, V hzp, const V eo[3], R aa, R bb, const PS &pi, PS &po,
                    const V pp[3], const V pm[3], bool first, V pn[3], V en[3]) {
        if (j - 1 < 0) { hxp = hxp.ph(byr, -byi); hzp = hzp.ph(byr, -byi); }
        V dyHz = (hh[2] - hzp) * idx, dyHx = (hh[0] - hxp) * idx;
        V dxHz = (hh[2] - left(hh[2])) * idx, dxHy = (hh[1] - left(hh[1])) * idx;
        if constexpr (PML) {
            if (inx) {
                dxHz = str(dxHz, xe, pi.x[0], po.x[0]);   // E_y
                dxHy = str(dxHy, xe, pi.x[1], po.x[1]);   // E_z
            }
            if (iny(j)) {
                const R pr[3] = {profy[j], profy[ny + j], profy[2 * ny + j]};
                dyHx = str(dyHx, pr, pi.y[0], po.y[0]);   // E_z
                dyHz = str(dyHz, pr, pi.y[1], po.y[1]);   // E_x
            }
        }
        const V c3[3] = {dyHz - dzB(hh[1]), dzB(hh[0]) - dxHz, dxHy - dyHx};
        const R *cm = coef + 6 * m;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if constexpr (LOR) {
                const R *lq = lc + 12 * np * m + 4 * k;
                if (lq[2] != (R)0) {
                    const R ce = lq[2];
                    pn[k] = first ? (pp[k] * lq[0] + eo[k] * ce) * (R)0.5 : (pp[k] * lq[0] - pm[k] * lq[1] + eo[k] * ce) * lq[3];
                    en[k] = eo[k] * aa + (c3[k] * bb + pp[k] * aa - pn[k]) * cm[k];
                    continue;
                }
                pn[k] = V();
            }
            en[k] = eo[k] * aa + c3[k] * (bb * cm[k]);
        }
    };
    // P and P_prev of (wrapped) row j from the input buffer (dispersive cells only)
    auto lor_in = [&](int j, int m, V pp[3], V pm[3]) {
        if constexpr (LOR) {
            const unsigned g = (unsigned)(j * nx + col);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (lc[12 * np * m + 4 * k + 2] != (R)0) {
                    pp[k] = ldy<R, CPLX>(lin, k, N, g);
                    pm[k] = ldy<R, CPLX>(lin, 3 + k, N, g);
                } else {
                    pp[k] = V();
                    pm[k] = V();
                }
            }
        }
    };
    auto lor_store = [&](int j, int m, const V pnew[3], const V pold[3]) {
        if constexpr (LOR) {
            if (!own) return;
            const unsigned g = (unsigned)(j * nx + col);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (lc[12 * np * m + 4 * k + 2] != (R)0) {
                    sty<R, CPLX>(lout, k, N, g, pnew[k]);
                    sty<R, CPLX>(lout, 3 + k, N, g, pold[k]);
                }
        }
    };
    auto store = [&](int j, const V e[3], const V hh[3]) {
        if (!own) return;
        const unsigned g = (unsigned)(j * nx + col);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sty<R, CPLX>(fout, k, N, g, e[k]);
            sty<R, CPLX>(fout, 3 + k, N, g, hh[k]);
        }
    };

    // the march, compiled with and without the projection of the sigma group (most tiles hold no
    // entries; their FP64 sums would otherwise stay live through the whole march)
    auto march = [&](auto proj_tag) {
        constexpr bool PROJ = decltype(proj_tag)::value;
        double pA = 0.0, pB = 0.0;
        const int j0 = t.j0;
        if (w > 0) {
            if (electric) {
                // carried: the buffer's E at row r, H_A at r-1, E_A at r-1, H_B at r-2 (+ materials), and
                // step A's psi (H and E groups) and P of row r-1, the buffer's P of row r-1
                V e0c[3], hAm[3], eAm[3], hBm[3];
                PS sHAm, sEAm;
                V pAm[3], p0m[3];
                int m_r, m_rm = 0;
                {
                    const int ja = wrow(j0 - 2), jb = wrow(j0 - 1);
                    const V ea[3] = {ldf(0, ja), ldf(1, ja), ldf(2, ja)};
                    const V ha[3] = {ldf(3, ja), ldf(4, ja), ldf(5, ja)};
    #pragma unroll
                    for (int k = 0; k < 3; ++k) e0c[k] = ldf(k, jb);
                    PS po;
                    updH(ja, mat[(unsigned)(ja * nx + col)], ea, e0c[0], e0c[2], ha, (R)1, hA0, psi_in_row(ja, 2), po, hAm);   // H_A(j0-2)
                    m_r = mat[(unsigned)(jb * nx + col)];
                }
                // inputs of iteration r: the buffer's E at row r+1, H at row r, material of row r+1
                V en_c[3], hq_c[3];
                int mn_c;
                int jr = wrow(j0 - 1), jp = wrow(j0 - 2);   // rows r and r-1, wrapped
                // staged rows: iteration r's slot holds E(r+1), H(r), psi and P of row r; mq[k] is the
                // material of row r + 1 + k (the rows staged ahead need theirs for the P copies)
                int mq[STG + 2];
                int sl = 0, js = 0, jq = 0;   // wrapped rows r + STG (staged next) and r + STG + 3 (its material next)
                auto stage_e = [&](int slot, int j, int m) {   // j: the staged iteration's row, wrapped
                    const int jn = j + 1 == ny ? 0 : j + 1;
                    const unsigned g = (unsigned)(j * nx + col), gn = (unsigned)(jn * nx + col);
    #pragma unroll
                    for (int k = 0; k < 3; ++k) { sg(slot, k, fin, k, N, gn); sg(slot, 3 + k, fin, 3 + k, N, g); }
                    stage_psi(slot, j, j, 0, 4);
                    stage_lor(slot, j, m);
                };
                if constexpr (STG > 0) {
    #pragma unroll
                    for (int k = 0; k < STG + 2; ++k) mq[k] = matw(j0 + k);
    #pragma unroll
                    for (int q = 0; q < STG; ++q) {
                        if (j0 - 1 + q <= j0 + h) stage_e(q, wrow(j0 - 1 + q), q == 0 ? m_r : mq[q - 1]);
                        cpa_commit();
                    }
                    mn_c = mq[0];
                    js = wrow(j0 - 1 + STG);
                    jq = wrow(j0 + STG + 2);
                } else {
                    const int jn = jr + 1 == ny ? 0 : jr + 1;
    #pragma unroll
                    for (int k = 0; k < 3; ++k) { en_c[k] = ldf(k, jn); hq_c[k] = ldf(3 + k, jr); }
                    mn_c = mat[(unsigned)(jn * nx + col)];
                }
                for (int r = j0 - 1; r <= j0 + h; ++r) {
                    const int jn = jr + 1 == ny ? 0 : jr + 1;
                    V en_n[3], hq_n[3];
                    int mn_n = 0;
                    PS piH, piE;
                    V p0r[3], pmr[3];
                    if constexpr (STG > 0) {
                        if (r + STG <= j0 + h) stage_e(sl == 0 ? STG : sl - 1, js, mq[STG - 1]);
                        cpa_commit();
                        cpa_wait<STG>();
    #pragma unroll
                        for (int k = 0; k < 3; ++k) { en_c[k] = fv(sl, k); hq_c[k] = fv(sl, 3 + k); }
                        piH = psi_slot(sl, jr, 2);
                        piE = psi_slot(sl, jr, 0);
                        lor_slot(sl, m_r, p0r, pmr);
                    } else {
                        if (r + 1 <= j0 + h) {   // the next iteration's inputs, loaded ahead
                            const int jnn = jn + 1 == ny ? 0 : jn + 1;
    #pragma unroll
                            for (int k = 0; k < 3; ++k) { en_n[k] = ldf(k, jnn); hq_n[k] = ldf(3 + k, jn); }
                            mn_n = mat[(unsigned)(jnn * nx + col)];
                        }
                        piH = psi_in_row(jr, 2);
                        piE = psi_in_row(jr, 0);
                        lor_in(jr, m_r, p0r, pmr);
                    }
                    V hA[3], eA[3], pAr[3];
                    PS sHA, sEA;
                    updH(jr, m_r, e0c, en_c[0], en_c[2], hq_c, (R)1, hA0, piH, sHA, hA);
                    updE(jr, m_r, hA, hAm[0], hAm[2], e0c, a, bs, piE, sEA, p0r, pmr, firstA, pAr, eA);
                    const bool inA = r >= j0 && r < j0 + h;
                    if (PROJ && inA && t.ne > 0) pA += project_row_m2<R, CPLX>(t, r - j0, w, grp, eA[0], eA[1], eA[2]);
                    if (!two) {
                        if (inA) {
                            store(jr, eA, hA);
                            psi_store(jr, 2, sHA);
                            psi_store(jr, 0, sEA);
                            lor_store(jr, m_r, pAr, p0r);
                        }
                    } else if (r == j0) {
                        PS po;
                        updH(jp, m_rm, eAm, eA[0], eA[2], hAm, (R)1, hB0, sHAm, po, hBm);   // H_B(j0-1)
                    } else if (r > j0) {
                        const int jm = jp;
                        V hB[3], eB[3], pBr[3];
                        PS sHB, sEB;
                        updH(jm, m_rm, eAm, eA[0], eA[2], hAm, (R)1, hB0, sHAm, sHB, hB);
                        updE(jm, m_rm, hB, hBm[0], hBm[2], eAm, a, bs, sEAm, sEB, pAm, p0m, false, pBr, eB);
                        if (r - 1 < j0 + h) {
                            store(jm, eB, hB);
                            psi_store(jm, 2, sHB);
                            psi_store(jm, 0, sEB);
                            lor_store(jm, m_rm, pBr, pAm);
                            if (PROJ && t.ne > 0) pB += project_row_m2<R, CPLX>(t, r - 1 - j0, w, grp, eB[0], eB[1], eB[2]);
                        }
    #pragma unroll
                        for (int k = 0; k < 3; ++k) hBm[k] = hB[k];
                    }
    #pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        eAm[k] = eA[k];
                        hAm[k] = hA[k];
                        e0c[k] = en_c[k];
                        if constexpr (STG == 0) { en_c[k] = en_n[k]; hq_c[k] = hq_n[k]; }
                        pAm[k] = pAr[k];
                        p0m[k] = p0r[k];
                    }
                    sHAm = sHA;
                    sEAm = sEA;
                    m_rm = m_r;
                    m_r = mn_c;
                    if constexpr (STG > 0) {
    #pragma unroll
                        for (int k = 0; k < STG + 1; ++k) mq[k] = mq[k + 1];
                        mq[STG + 1] = mat[(unsigned)(jq * nx + col)];
                        mn_c = mq[0];
                        sl = sl == STG ? 0 : sl + 1;
                        js = js + 1 == ny ? 0 : js + 1;
                        jq = jq + 1 == ny ? 0 : jq + 1;
                    } else {
                        mn_c = mn_n;
                    }
                    jp = jr;
                    jr = jn;
                }
            } else {
                // carried: E_A at row r, the buffer's H at row r, H_A at r-1, E_B at r-1 (+ materials),
                // step A's E psi and P of row r (made one iteration ahead), step A's H psi of row r-1
                V eAc[3], h0c[3], hAm[3], eBm[3];
                PS sEAc, sHAm;
                V pAc[3], p0c[3];
                int m_r, m_rm = 0;
                int jr = wrow(j0 - 1), jp = wrow(j0 - 2);   // rows r and r-1, wrapped
                {
                    const int ja = jp;
                    const V hb2[3] = {ldf(3, ja), ldf(4, ja), ldf(5, ja)};
                    const V e0[3] = {ldf(0, jr), ldf(1, jr), ldf(2, jr)};
    #pragma unroll
                    for (int k = 0; k < 3; ++k) h0c[k] = ldf(3 + k, jr);
                    m_r = mat[(unsigned)(jr * nx + col)];
                    V pm0[3];
                    lor_in(jr, m_r, p0c, pm0);
                    updE(jr, m_r, h0c, hb2[0], hb2[2], e0, (R)1, hA0, psi_in_row(jr, 0), sEAc, p0c, pm0, false, pAc, eAc);   // E_A(j0-1)
                }
                // inputs of iteration r: the buffer's H and E at row r+1, material of row r+1
                V hn_c[3], en_c[3];
                int mn_c;
                // staged rows: iteration r's slot holds H(r+1), E(r+1), the E-group psi and P of row r+1,
                // the H-group psi of row r; mq[k] is the material of row r + 1 + k
                int mq[STG + 2];
                int sl = 0, js = 0, jq = 0;   // wrapped rows r + STG (staged next) and r + STG + 3 (its material next)
                auto stage_m = [&](int slot, int j, int m) {   // j: the staged iteration's row, wrapped
                    const int jn = j + 1 == ny ? 0 : j + 1;
                    const unsigned gn = (unsigned)(jn * nx + col);
    #pragma unroll
                    for (int k = 0; k < 3; ++k) { sg(slot, k, fin, 3 + k, N, gn); sg(slot, 3 + k, fin, k, N, gn); }
                    stage_psi(slot, jn, jn, 0, 2);
                    stage_psi(slot, j, j, 2, 4);
                    stage_lor(slot, jn, m);
                };
                if constexpr (STG > 0) {
    #pragma unroll
                    for (int k = 0; k < STG + 2; ++k) mq[k] = matw(j0 + k);
    #pragma unroll
                    for (int q = 0; q < STG; ++q) {
                        if (j0 - 1 + q <= j0 + h) stage_m(q, wrow(j0 - 1 + q), mq[q]);
                        cpa_commit();
                    }
                    mn_c = mq[0];
                    js = wrow(j0 - 1 + STG);
                    jq = wrow(j0 + STG + 2);
                } else {
                    const int jn = jr + 1 == ny ? 0 : jr + 1;
    #pragma unroll
                    for (int k = 0; k < 3; ++k) { hn_c[k] = ldf(3 + k, jn); en_c[k] = ldf(k, jn); }
                    mn_c = mat[(unsigned)(jn * nx + col)];
                }
                for (int r = j0 - 1; r <= j0 + h; ++r) {
                    const int jn = jr + 1 == ny ? 0 : jr + 1;
                    V hn_n[3], en_n[3];
                    int mn_n = 0;
                    V eAn[3], hA[3], pAn[3], p0n[3], pmn[3];
                    PS sEAn, sHA, piE, piH;
                    if constexpr (STG > 0) {
                        if (r + STG <= j0 + h) stage_m(sl == 0 ? STG : sl - 1, js, mq[STG]);
                        cpa_commit();
                        cpa_wait<STG>();
    #pragma unroll
                        for (int k = 0; k < 3; ++k) { hn_c[k] = fv(sl, k); en_c[k] = fv(sl, 3 + k); }
                        piE = psi_slot(sl, jn, 0);
                        piH = psi_slot(sl, jr, 2);
                        lor_slot(sl, mn_c, p0n, pmn);
                    } else {
                        if (r + 1 <= j0 + h) {
                            const int jnn = jn + 1 == ny ? 0 : jn + 1;
    #pragma unroll
                            for (int k = 0; k < 3; ++k) { hn_n[k] = ldf(3 + k, jnn); en_n[k] = ldf(k, jnn); }
                            mn_n = mat[(unsigned)(jnn * nx + col)];
                        }
                        piE = psi_in_row(jn, 0);
                        piH = psi_in_row(jr, 2);
                        lor_in(jn, mn_c, p0n, pmn);
                    }
                    updE(jn, mn_c, hn_c, h0c[0], h0c[2], en_c, (R)1, hA0, piE, sEAn, p0n, pmn, false, pAn, eAn);   // E_A(r+1)
                    updH(jr, m_r, eAc, eAn[0], eAn[2], h0c, a, bs, piH, sHA, hA);          // H_A(r)
                    const bool inA = r >= j0 && r < j0 + h;
                    if (PROJ && inA && t.ne > 0) pA += project_row_m2<R, CPLX>(t, r - j0, w, grp, hA[0], hA[1], hA[2]);
                    if (!two) {
                        if (inA) {
                            store(jr, eAc, hA);
                            psi_store(jr, 0, sEAc);
                            psi_store(jr, 2, sHA);
                            lor_store(jr, m_r, pAc, p0c);
                        }
                    } else if (r >= j0) {
                        V eB[3], pBr[3];
                        PS sEB;
                        updE(jr, m_r, hA, hAm[0], hAm[2], eAc, (R)1, hB0, sEAc, sEB, pAc, p0c, false, pBr, eB);   // E_B(r)
                        if (r > j0) {
                            const int jm = jp;
                            V hB[3];
                            PS sHB;
                            updH(jm, m_rm, eBm, eB[0], eB[2], hAm, a, bs, sHAm, sHB, hB);    // H_B(r-1)
                            if (r - 1 < j0 + h) {
                                store(jm, eBm, hB);
                                psi_store(jm, 2, sHB);
                                if (PROJ && t.ne > 0) pB += project_row_m2<R, CPLX>(t, r - 1 - j0, w, grp, hB[0], hB[1], hB[2]);
                            }
                        }
                        if (r < j0 + h) {
                            psi_store(jr, 0, sEB);
                            lor_store(jr, m_r, pBr, pAc);
                        }
    #pragma unroll
                        for (int k = 0; k < 3; ++k) eBm[k] = eB[k];
                    }
    #pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        hAm[k] = hA[k];
                        eAc[k] = eAn[k];
                        h0c[k] = hn_c[k];
                        if constexpr (STG == 0) { hn_c[k] = hn_n[k]; en_c[k] = en_n[k]; }
                        pAc[k] = pAn[k];
                        p0c[k] = p0n[k];
                    }
                    sEAc = sEAn;
                    sHAm = sHA;
                    m_rm = m_r;
                    m_r = mn_c;
                    if constexpr (STG > 0) {
    #pragma unroll
                        for (int k = 0; k < STG + 1; ++k) mq[k] = mq[k + 1];
                        mq[STG + 1] = mat[(unsigned)(jq * nx + col)];
                        mn_c = mq[0];
                        sl = sl == STG ? 0 : sl + 1;
                        js = js + 1 == ny ? 0 : js + 1;
                        jq = jq + 1 == ny ? 0 : jq + 1;
                    } else {
                        mn_c = mn_n;
                    }
                    jp = jr;
                    jr = jn;
                }
            }
        }

        if (PROJ && t.ne > 0) {
            for (int o = 16; o > 0; o >>= 1) {
                pA += __shfl_down_sync(0xffffffffu, pA, o);
                pB += __shfl_down_sync(0xffffffffu, pB, o);
            }
            if (lane == 0) {
                const double c = S.gw[nA - 1] * pA + (two ? S.gw[nA] * pB : 0.0);
                atomicAdd(S.acc, c);
                const double ct = (nA > S.tail_from ? S.gw[nA - 1] * pA : 0.0) + (two && nA + 1 > S.tail_from ? S.gw[nA] * pB : 0.0);
                if (ct != 0.0) atomicAdd(S.tail, ct);
            }
        }
    };
    if (t.ne > 0) march(Flag<true>{});
    else march(Flag<false>{});
}

template <typename R, bool CPLX, bool PML, bool LOR, int MINB>
void launch_one(const DevSim6 *sims, const DevTile2 *tiles, int ntiles, const int64_t *lb, int64_t la, cudaStream_t st)
{
    // MAR2_STG staged rows while the ring stays within 48 KB of static shared memory per CTA
    constexpr int NV = (CPLX ? 2 : 1) * (6 + (PML ? 8 : 0) + (LOR ? 6 : 0));
    constexpr int STG = MAR2_STG == 0 ? 0 : (WARPS_M2 * (MAR2_STG + 1) * NV * 32 * 4 <= 48 * 1024 ? MAR2_STG : 1);
    k_mar2<R, CPLX, PML, LOR, MINB, STG><<<(ntiles + WARPS_M2 - 1) / WARPS_M2, WARPS_M2 * 32, 0, st>>>(sims, tiles, ntiles, lb, la);
}

}  // namespace

void launch_march6_2(int cplx, int variant, const DevSim6 *sims, const DevTile2 *tiles, int ntiles,
                     const int64_t *launch_base, int64_t launch_add, cudaStream_t st)
{
    if (ntiles <= 0) return;
    // variant: 1 = CPML planes present, + 2 = one Lorentz pole
    if (cplx) {
        switch (variant & 3) {
        case 0: launch_one<float, true, false, false, MAR2_C0>(sims, tiles, ntiles, launch_base, launch_add, st); break;
        case 1: launch_one<float, true, true, false, MAR2_C1>(sims, tiles, ntiles, launch_base, launch_add, st); break;
        case 2: launch_one<float, true, false, true, MAR2_C2>(sims, tiles, ntiles, launch_base, launch_add, st); break;
        default: launch_one<float, true, true, true, MAR2_C3>(sims, tiles, ntiles, launch_base, launch_add, st); break;
        }
    } else {
        switch (variant & 3) {
        case 0: launch_one<float, false, false, false, MAR2_R0>(sims, tiles, ntiles, launch_base, launch_add, st); break;
        case 1: launch_one<float, false, true, false, MAR2_R1>(sims, tiles, ntiles, launch_base, launch_add, st); break;
        case 2: launch_one<float, false, false, true, MAR2_R2>(sims, tiles, ntiles, launch_base, launch_add, st); break;
        default: launch_one<float, false, true, true, MAR2_R3>(sims, tiles, ntiles, launch_base, launch_add, st); break;
        }
    }
}

}  // namespace cas
