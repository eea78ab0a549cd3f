// Six-component Yee leapfrog of three-dimensional simulations (Sec. III E), with CPML
// (Sec. III B), Bloch-periodic walls (Sec. III D) and Lorentz media of up to three undamped
// poles continued onto the contour (Eq. (9); the silica model of Sec. III D): both half steps
// of one time step in a single pass over memory, fused with the surface projection and the
// FP64 accumulation of w_n s(n) (Eq. (1)).
//
// Column march.  Every warp owns a tile of COL3_W x COL3_H cells in (x, y) over a chunk of
// planes [z0, z1) and advances it on its own (no block-level barrier): lane l holds column
// x0 - 1 + l, and the warp walks the tile's rows plane after plane.  Call the update that goes
// first A (H for electric sources, E for magnetic ones, with a = 1 and b = dt, halved on step
// 1) and the sigma update B (measured by the surface functional).  A at a cell needs B_old at
// its neighbours on one side (J: x+1, y+1, z+1; K: x-1, y-1, z-1), B needs A_new on the other
// side.  So the warp marches in the direction of A's neighbours (J: rows and planes upwards;
// K: downwards): B_old of the next row is loaded one row ahead and becomes the row's own
// value, B_old of the next plane is loaded per row, A_new of the previous row stays in
// registers, and A_new of the previous plane waits in a per-lane shared-memory ring.  The
// first lane, one extra row per plane and one extra plane before the chunk compute A only
// (halo recomputation, nothing is exchanged between warps), so fields, CPML psi and Lorentz
// P ping-pong between two buffers by step parity (step n reads buffer (n-1)&1 and writes
// n&1).  x neighbours come by shuffle.  A row's inputs are loaded while the previous row
// computes.  Every value loaded from a cell beyond a periodic wall carries that wall's Bloch
// factor (psi and P included), so halo cells compute exactly the Bloch image of the owner's
// value; beyond a closed wall the wrapped neighbour is used, as on the other six-component
// kernels, where the wall's masked components make its value irrelevant.
#include <cuda_runtime.h>

#include "casimir.h"
#include "kernels.h"

namespace cas {

namespace {

constexpr int HR = COL3_H;      // rows of a tile

template <typename R, bool CPLX>
struct Q;

template <typename R>
struct Q<R, false> {
    R x;
    __device__ Q() : x(0) {}
    __device__ explicit Q(R a) : x(a) {}
    __device__ Q operator+(Q o) const { return Q(x + o.x); }
    __device__ Q operator-(Q o) const { return Q(x - o.x); }
    __device__ Q operator*(R s) const { return Q(x * s); }
    __device__ Q ph(R c, R) const { return Q(x * c); }
    __device__ Q dn() const { return Q(__shfl_down_sync(0xffffffffu, x, 1)); }
    __device__ Q up() const { return Q(__shfl_up_sync(0xffffffffu, x, 1)); }
};

template <typename R>
struct Q<R, true> {
    R x, y;
    __device__ Q() : x(0), y(0) {}
    __device__ Q(R a, R b) : x(a), y(b) {}
    __device__ Q operator+(Q o) const { return Q(x + o.x, y + o.y); }
    __device__ Q operator-(Q o) const { return Q(x - o.x, y - o.y); }
    __device__ Q operator*(R s) const { return Q(x * s, y * s); }
    __device__ Q ph(R c, R s) const { return Q(x * c - y * s, x * s + y * c); }
    __device__ Q dn() const { return Q(__shfl_down_sync(0xffffffffu, x, 1), __shfl_down_sync(0xffffffffu, y, 1)); }
    __device__ Q up() const { return Q(__shfl_up_sync(0xffffffffu, x, 1), __shfl_up_sync(0xffffffffu, y, 1)); }
};

// a field value as stored in shared memory (a shared array takes no constructor)
template <typename R, bool CPLX>
struct Raw {
    R v[CPLX ? 2 : 1];
    __device__ void operator=(const Q<R, CPLX> &q)
    {
        v[0] = q.x;
        if constexpr (CPLX) v[1] = q.y;
    }
    __device__ operator Q<R, CPLX>() const
    {
        if constexpr (CPLX) return Q<R, CPLX>(v[0], v[1]);
        else return Q<R, CPLX>(v[0]);
    }
};

// planes of N elements (real and imaginary planes when complex); 32-bit element offsets
// (the planner sends only runs with 12 max(1, poles) N < 2^32 here)
template <typename R, bool CPLX>
__device__ __forceinline__ Q<R, CPLX> ldq(const R *__restrict__ p, int plane, unsigned N, unsigned g)
{
    if constexpr (CPLX) return Q<R, CPLX>(p[(2u * plane) * N + g], p[(2u * plane + 1u) * N + g]);
    else return Q<R, CPLX>(p[(unsigned)plane * N + g]);
}

template <typename R, bool CPLX>
__device__ __forceinline__ void stq(R *__restrict__ p, int plane, unsigned N, unsigned g, Q<R, CPLX> v)
{
    if constexpr (CPLX) { p[(2u * plane) * N + g] = v.x; p[(2u * plane + 1u) * N + g] = v.y; }
    else p[(unsigned)plane * N + g] = v.x;
}

// Asynchronous copy of one element, global -> shared (cp.async: each lane stages its own
// values, so only the lane's own wait orders the copy before the read)
template <typename R>
__device__ __forceinline__ void cpa(R *sdst, const R *gsrc)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sdst);
    if constexpr (sizeof(R) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gsrc) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory"); }

// Staged inputs of a row step, per lane, in units of field values: B_old here (3), B_old at the
// next row (3), A_old here (3), B_old at the next plane (components 0, 1), and with CPML the
// psi of the A group (per axis, its two planes) and of the B group (likewise).
constexpr int ST_BO = 0, ST_BN = 3, ST_AO = 6, ST_BZ = 9, ST_PA = 11, ST_PB = 17;
constexpr int ST_VALUES_PML = 23, ST_VALUES = 11;

// warps (tiles) per CTA: four, or fewer where the staging slots and the ring of four warps
// would exceed 48 KB of shared memory
__host__ __device__ constexpr int col3_warps(int rsize, bool cplx, bool pml)
{
    const int per_warp = (2 * (pml ? ST_VALUES_PML : ST_VALUES) + 2 * COL3_H) * (cplx ? 2 : 1) * 32 * rsize;
    const int w = (48 * 1024) / per_warp;
    return w >= 4 ? 4 : (w >= 1 ? w : 1);
}

// Index i on an axis of n cells: the wrapped index and the side of the image it stands for
// (-1 below 0, 0 inside, +1 at n and above).  Indices more than one cell outside belong to
// lanes or rows whose results are never used; they are clamped into the grid.
struct Pos {
    int w;
    int side;
};
__device__ __forceinline__ Pos wrap(int i, int n)
{
    Pos p{i, 0};
    if (i < 0) { p.w = i + n; p.side = -1; }
    else if (i >= n) { p.w = i - n; p.side = 1; }
    p.w = p.w < 0 ? 0 : (p.w >= n ? n - 1 : p.w);
    return p;
}

// CPLX: complex fields (the only ones with Bloch factors other than 1: a real field's factors
// are all 1, since the planner makes every run with a complex factor complex)
template <typename R, bool CPLX, bool PML, int NPL, bool MAG, int MINB>
__global__ void __launch_bounds__(col3_warps((int)sizeof(R), CPLX, PML) * 32, MINB)
k_col3(const DevSim6 *__restrict__ sims, const DevTile *__restrict__ tiles, int ntiles,
       const int64_t *__restrict__ launch_base, int64_t launch_add)
{
    using V = Q<R, CPLX>;
    constexpr bool LOR = NPL > 0;
    constexpr int C3W = col3_warps((int)sizeof(R), CPLX, PML);
    __shared__ Raw<R, CPLX> ring[C3W][HR][2][32];   // A_new of the previous plane, components 0, 1
    constexpr int CF = CPLX ? 2 : 1;
    constexpr int NSV = PML ? ST_VALUES_PML : ST_VALUES;
    __shared__ R stage[C3W][2][NSV * CF][32];      // the current and the next row step's inputs
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ti = blockIdx.x * C3W + warp;
    if (ti >= ntiles) return;                       // no block-level barrier below
    const DevTile t = tiles[ti];
    const DevSim6 &S = sims[t.sim];
    const int64_t n = *launch_base + launch_add - S.s0;
    if (n < 1 || n > S.T) return;
    const int nx = S.n[0], ny = S.n[1], nz = S.n[2];
    const unsigned sy = (unsigned)nx, sz = (unsigned)nx * (unsigned)ny;
    const unsigned N = sz * (unsigned)nz;
    const int pin = (int)((n - 1) & 1), pout = (int)(n & 1);
    const R *__restrict__ Fi = reinterpret_cast<const R *>(S.fields) + (size_t)pin * S.fhalf;
    R *__restrict__ Fo = reinterpret_cast<R *>(S.fields) + (size_t)pout * S.fhalf;
    const R *__restrict__ coef = reinterpret_cast<const R *>(S.coef);
    const uint8_t *__restrict__ mat = S.mat;
    const R idx = (R)S.inv_dx;
    constexpr bool mag = MAG;                                // magnetic (K) sources
    constexpr int aBase = MAG ? 0 : 3, bBase = MAG ? 3 : 0;  // first plane of the A and B fields
    const R bA = (R)(n == 1 ? 0.5 * S.dt : S.dt);
    const R aB = (R)S.a, bB = (R)S.bs;
    const bool first_e = !MAG && n == 1;                    // Lorentz start of electric sources
    const R *__restrict__ Pi = nullptr;
    R *__restrict__ Po = nullptr;
    const R *__restrict__ lc = nullptr;
    if constexpr (LOR) {
        Pi = reinterpret_cast<const R *>(S.lor) + (size_t)pin * S.lor_half;
        Po = reinterpret_cast<R *>(S.lor) + (size_t)pout * S.lor_half;
        lc = reinterpret_cast<const R *>(S.lorc);
    }
    const R *__restrict__ psi_i = nullptr;
    R *__restrict__ psi_o = nullptr;
    const R *__restrict__ pml = nullptr;
    int dX = 0, dY = 0, dZ = 0;
    if constexpr (PML) {
        psi_i = reinterpret_cast<const R *>(S.psi) + (size_t)pin * S.psi_half;
        psi_o = reinterpret_cast<R *>(S.psi) + (size_t)pout * S.psi_half;
        pml = reinterpret_cast<const R *>(S.pml);
        dX = S.pml_d[0];
        dY = S.pml_d[1];
        dZ = S.pml_d[2];
    }

    // this lane's column
    const int x = t.i0 - 1 + lane;
    const Pos px = wrap(x, nx);
    const bool lane_own = lane >= 1 && lane <= COL3_W && x < nx;
    const bool inx = PML && dX > 0 && (px.w < dX || px.w >= nx - dX);
    const int sxp = px.w < dX ? px.w : px.w - (nx - 2 * dX);
    // rows q = 0 .. HR of a plane: q = 0 is the halo row; J rows ascend from y0 - 1, K rows
    // descend from y0 + HR; planes: J ascend from z0 (z0 - 1 first, A only), K descend from
    // z1 - 1 (z1 first, A only)
    const int dz = mag ? -1 : 1;
    auto rowy = [&](int q) { return mag ? t.j0 + HR - q : t.j0 - 1 + q; };
    const int np = t.z1 - t.z0;
    auto plz = [&](int p) { return mag ? t.z1 - 1 - p : t.z0 + p; };   // p = -1: the halo plane

    // Bloch factor of the image at (this lane, row side sy_, plane side sz_)
    auto bfac = [&](int sy_, int sz_, R &c, R &s) -> bool {
        if constexpr (!CPLX) {
            return false;
        } else {
            R pc = 1, ps = 0;
            const int side[3] = {px.side, sy_, sz_};
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (side[a]) {
                    const R fc = (R)S.bre[a], fs = (R)(side[a] * S.bim[a]);
                    const R nc = pc * fc - ps * fs, ns = pc * fs + ps * fc;
                    pc = nc;
                    ps = ns;
                }
            c = pc;
            s = ps;
            return pc != (R)1 || ps != (R)0;
        }
    };
    // slab index of PML axis ax for this lane at row py, plane pz (valid inside the slab)
    auto slab_index = [&](int ax, const Pos &py, const Pos &pz) -> unsigned {
        if (ax == 0) return ((unsigned)pz.w * (unsigned)ny + (unsigned)py.w) * (unsigned)(2 * dX) + (unsigned)sxp;
        if (ax == 1) {
            const int syp = py.w < dY ? py.w : py.w - (ny - 2 * dY);
            return ((unsigned)pz.w * (unsigned)(2 * dY) + (unsigned)syp) * sy + (unsigned)px.w;
        }
        const int szp = pz.w < dZ ? pz.w : pz.w - (nz - 2 * dZ);
        return ((unsigned)szp * (unsigned)ny + (unsigned)py.w) * sy + (unsigned)px.w;
    };
    auto in_slab = [&](int ax, const Pos &py, const Pos &pz) -> bool {
        if constexpr (!PML) return false;
        if (ax == 0) return inx;
        if (ax == 1) return dY > 0 && (py.w < dY || py.w >= ny - dY);
        return dZ > 0 && (pz.w < dZ || pz.w >= nz - dZ);
    };
    // psi planes of the A and B groups (J: A = H uses planes 2, 3; K: A = E uses planes 0, 1)
    constexpr int plA = MAG ? 0 : 2, plB = MAG ? 2 : 0;
    auto psi_ptr = [&](const R *base, int ax, int pl) -> const R * {
        return base + S.psi_off[ax] + (unsigned)pl * (unsigned)(CF * S.slab[ax]);
    };
    // stage one field value: component comp at (this lane, py, pz) into value slot v
    auto stage_f = [&](R (*st)[32], int v, int comp, const Pos &py, const Pos &pz) {
        const unsigned g = (unsigned)pz.w * sz + (unsigned)py.w * sy + (unsigned)px.w;
        if constexpr (CPLX) {
            cpa(&st[2 * v][lane], Fi + (2u * comp) * N + g);
            cpa(&st[2 * v + 1][lane], Fi + (2u * comp + 1u) * N + g);
        } else {
            cpa(&st[v][lane], Fi + (unsigned)comp * N + g);
        }
    };
    auto stage_p = [&](R (*st)[32], int v, const R *pp, unsigned slab, unsigned si) {
        if constexpr (CPLX) {
            cpa(&st[2 * v][lane], pp + si);
            cpa(&st[2 * v + 1][lane], pp + slab + si);
        } else {
            cpa(&st[v][lane], pp + si);
        }
    };
    // a staged value with the Bloch factor (c, s) of its cell applied
    auto unstage = [&](R (*st)[32], int v, bool ph, R c, R s) -> V {
        V r;
        if constexpr (CPLX) r = V(st[2 * v][lane], st[2 * v + 1][lane]);
        else r = V(st[v][lane]);
        if (ph) r = r.ph(c, s);
        return r;
    };

    // psi' = b psi + c d from the staged psi p (written to the output buffer at owned cells);
    // returns d / kappa + psi'
    auto stretch = [&](V d, int ax, const R *pr, int pl, unsigned si, V p, bool wr) -> V {
        p = p * pr[0] + d * pr[1];
        if (wr) {
            R *po = psi_o + S.psi_off[ax] + (unsigned)pl * (unsigned)(CF * S.slab[ax]);
            if constexpr (CPLX) { po[si] = p.x; po[S.slab[ax] + si] = p.y; }
            else po[si] = p.x;
        }
        return d * pr[2] + p;
    };

    // H group at (lane, py, pz): h' = a h - b (1/mu) curl E, forward differences; e: E here;
    // eyr, ezr: E_y, E_z at x+1; exy, ezy: E_x, E_z at y+1; exz, eyz: E_x, E_y at z+1
    auto updH = [&](const V h[3], const V e[3], V eyr, V ezr, V exy, V ezy, V exz, V eyz, int m, R a, R b,
                    const Pos &py, const Pos &pz, const V *ps, bool wr, V out[3]) {
        V dyEz = (ezy - e[2]) * idx, dzEy = (eyz - e[1]) * idx, dzEx = (exz - e[0]) * idx;
        V dxEz = (ezr - e[2]) * idx, dxEy = (eyr - e[1]) * idx, dyEx = (exy - e[0]) * idx;
        if constexpr (PML) {
            if (inx) {
                const R *prx = pml + S.pml_off[0];
                const R pr[3] = {prx[3 * nx + px.w], prx[4 * nx + px.w], prx[5 * nx + px.w]};
                const unsigned si = slab_index(0, py, pz);
                dxEz = stretch(dxEz, 0, pr, 2, si, ps[0], wr);    // H_y
                dxEy = stretch(dxEy, 0, pr, 3, si, ps[1], wr);    // H_z
            }
            if (in_slab(1, py, pz)) {
                const R *pry = pml + S.pml_off[1];
                const R pr[3] = {pry[3 * ny + py.w], pry[4 * ny + py.w], pry[5 * ny + py.w]};
                const unsigned si = slab_index(1, py, pz);
                dyEx = stretch(dyEx, 1, pr, 2, si, ps[2], wr);    // H_z
                dyEz = stretch(dyEz, 1, pr, 3, si, ps[3], wr);    // H_x
            }
            if (in_slab(2, py, pz)) {
                const R *prz = pml + S.pml_off[2];
                const R pr[3] = {prz[3 * nz + pz.w], prz[4 * nz + pz.w], prz[5 * nz + pz.w]};
                const unsigned si = slab_index(2, py, pz);
                dzEy = stretch(dzEy, 2, pr, 2, si, ps[4], wr);    // H_x
                dzEx = stretch(dzEx, 2, pr, 3, si, ps[5], wr);    // H_y
            }
        }
        const V c3[3] = {dyEz - dzEy, dzEx - dxEz, dxEy - dyEx};
        const R *cm = coef + 6 * m;
#pragma unroll
        for (int k = 0; k < 3; ++k) out[k] = h[k] * a - c3[k] * (b * cm[3 + k]);
    };

    // E group at (lane, py, pz): D' = a D + b curl H, backward differences, E = (D - sum_j P_j) / eps_inf;
    // h: H here; hyl, hzl: H_y, H_z at x-1; hxy, hzy: H_x, H_z at y-1; hxz, hyz: H_x, H_y at z-1
    auto updE = [&](const V e[3], const V h[3], V hyl, V hzl, V hxy, V hzy, V hxz, V hyz, int m, R a, R b, bool first,
                    const Pos &py, const Pos &pz, const V *ps, bool wr, V out[3]) {
        V dyHz = (h[2] - hzy) * idx, dzHy = (h[1] - hyz) * idx, dzHx = (h[0] - hxz) * idx;
        V dxHz = (h[2] - hzl) * idx, dxHy = (h[1] - hyl) * idx, dyHx = (h[0] - hxy) * idx;
        R c = 1, s = 0;
        bool ph = false;
        if constexpr (LOR) ph = bfac(py.side, pz.side, c, s);
        if constexpr (PML) {
            if (inx) {
                const R *prx = pml + S.pml_off[0];
                const R pr[3] = {prx[px.w], prx[nx + px.w], prx[2 * nx + px.w]};
                const unsigned si = slab_index(0, py, pz);
                dxHz = stretch(dxHz, 0, pr, 0, si, ps[0], wr);    // E_y
                dxHy = stretch(dxHy, 0, pr, 1, si, ps[1], wr);    // E_z
            }
            if (in_slab(1, py, pz)) {
                const R *pry = pml + S.pml_off[1];
                const R pr[3] = {pry[py.w], pry[ny + py.w], pry[2 * ny + py.w]};
                const unsigned si = slab_index(1, py, pz);
                dyHx = stretch(dyHx, 1, pr, 0, si, ps[2], wr);    // E_z
                dyHz = stretch(dyHz, 1, pr, 1, si, ps[3], wr);    // E_x
            }
            if (in_slab(2, py, pz)) {
                const R *prz = pml + S.pml_off[2];
                const R pr[3] = {prz[pz.w], prz[nz + pz.w], prz[2 * nz + pz.w]};
                const unsigned si = slab_index(2, py, pz);
                dzHy = stretch(dzHy, 2, pr, 0, si, ps[4], wr);    // E_x
                dzHx = stretch(dzHx, 2, pr, 1, si, ps[5], wr);    // E_y
            }
        }
        const V c3[3] = {dyHz - dzHy, dzHx - dxHz, dxHy - dyHx};
        const R *cm = coef + 6 * m;
        const unsigned g = (unsigned)pz.w * sz + (unsigned)py.w * sy + (unsigned)px.w;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            V en = e[k] * a + c3[k] * (b * cm[k]);
            if constexpr (LOR) {
                const R *l4 = lc + 12 * S.npoles * m + 4 * k;
                if (l4[2] != (R)0) {
                    // per pole q (present poles first): P_q' = [cp P_q - cpm P_q-prev + ce E] cd
                    V sp = c3[k] * b;
#pragma unroll
                    for (int q = 0; q < (NPL > 1 ? CASIMIR_MAX_POLES : 1); ++q) {
                        const R *lq = l4 + 12 * q;
                        if (q > 0 && !(q < S.npoles && lq[2] != (R)0)) continue;
                        const R ce = lq[2];
                        V p = ldq<R, CPLX>(Pi, 6 * q + k, N, g), pm = ldq<R, CPLX>(Pi, 6 * q + 3 + k, N, g);
                        if (ph) { p = p.ph(c, s); pm = pm.ph(c, s); }
                        const V pn = first ? (p * lq[0] + e[k] * ce) * (R)0.5 : (p * lq[0] - pm * lq[1] + e[k] * ce) * lq[3];
                        if (wr) {
                            stq<R, CPLX>(Po, 6 * q + 3 + k, N, g, p);
                            stq<R, CPLX>(Po, 6 * q + k, N, g, pn);
                        }
                        sp = sp + p * a - pn;
                    }
                    en = e[k] * a + sp * cm[k];
                }
            }
            out[k] = en;
        }
    };

    // Row steps in one flat sequence with one call site per update, so that every update inlines:
    // a virtual step (p = -1, q = 0) that only stages, the halo plane's rows q = 1 .. HR (A only,
    // into the ring), then the chunk's planes p = 0 .. np - 1 with rows q = 0 .. HR.  The inputs
    // of the next step are staged (cp.async into the lane's own slot) before the current step
    // computes; B_old here is the previous step's next-row value except where a plane starts.
    R (*stg)[NSV * CF][32] = stage[warp];
    V aPrev0, aPrev2;                 // A_new of the previous row, components 0 and 2
    V bNprev[3];                      // B_old of the next row, kept for the next step
    Raw<R, CPLX>(*rg)[2][32] = ring[warp];
    int p = -1, q = 0, slot = 0, m_cur = 0, m_nxt = 0;
    bool reuse_cur = false;
    for (;;) {
        int pn = p, qn = q + 1;
        if (qn > HR) { pn = p + 1; qn = 0; }
        const bool have = pn < np;
        const bool real_step = !(p < 0 && q == 0);
        const bool reuse = pn == p && real_step;
        if (have) {
            R (*st)[32] = stg[slot ^ 1];
            const Pos py = wrap(rowy(qn), ny), pyn = wrap(rowy(qn + 1), ny);
            const Pos pz = wrap(plz(pn), nz), pzn = wrap(plz(pn) + dz, nz);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (!reuse) stage_f(st, ST_BO + k, bBase + k, py, pz);
                stage_f(st, ST_BN + k, bBase + k, pyn, pz);
                stage_f(st, ST_AO + k, aBase + k, py, pz);
            }
            stage_f(st, ST_BZ, bBase, py, pzn);
            stage_f(st, ST_BZ + 1, bBase + 1, py, pzn);
            if constexpr (PML) {
#pragma unroll
                for (int ax = 0; ax < 3; ++ax)
                    if (in_slab(ax, py, pz)) {
                        const unsigned si = slab_index(ax, py, pz), sl = (unsigned)S.slab[ax];
                        stage_p(st, ST_PA + 2 * ax, psi_ptr(psi_i, ax, plA), sl, si);
                        stage_p(st, ST_PA + 2 * ax + 1, psi_ptr(psi_i, ax, plA + 1), sl, si);
                        stage_p(st, ST_PB + 2 * ax, psi_ptr(psi_i, ax, plB), sl, si);
                        stage_p(st, ST_PB + 2 * ax + 1, psi_ptr(psi_i, ax, plB + 1), sl, si);
                    }
            }
            m_nxt = mat[(unsigned)pz.w * sz + (unsigned)py.w * sy + (unsigned)px.w];
        }
        cpa_commit();
        if (real_step) {
            cpa_wait<1>();            // this step's copies have landed; the next step's may be in flight
            R (*st)[32] = stg[slot];
            const int y = rowy(q);
            const Pos py = wrap(y, ny), pz = wrap(plz(p), nz);
            R c = 1, s = 0;
            const bool ph = bfac(py.side, pz.side, c, s);
            V bO[3], bN[3], aO[3], bZ[2], psA[6], psB[6];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                bO[k] = reuse_cur ? bNprev[k] : unstage(st, ST_BO + k, ph, c, s);
                aO[k] = unstage(st, ST_AO + k, ph, c, s);
            }
            // B_old of the next row and of the next plane carry their own cells' Bloch factors
            {
                const Pos pyn = wrap(rowy(q + 1), ny), pzn = wrap(plz(p) + dz, nz);
                R c2 = 1, s2 = 0;
                const bool ph2 = bfac(pyn.side, pz.side, c2, s2);
#pragma unroll
                for (int k = 0; k < 3; ++k) bN[k] = unstage(st, ST_BN + k, ph2, c2, s2);
                const bool ph3 = bfac(py.side, pzn.side, c2, s2);
                bZ[0] = unstage(st, ST_BZ, ph3, c2, s2);
                bZ[1] = unstage(st, ST_BZ + 1, ph3, c2, s2);
            }
            if constexpr (PML) {
#pragma unroll
                for (int ax = 0; ax < 3; ++ax)
                    if (in_slab(ax, py, pz)) {
                        psA[2 * ax] = unstage(st, ST_PA + 2 * ax, ph, c, s);
                        psA[2 * ax + 1] = unstage(st, ST_PA + 2 * ax + 1, ph, c, s);
                        psB[2 * ax] = unstage(st, ST_PB + 2 * ax, ph, c, s);
                        psB[2 * ax + 1] = unstage(st, ST_PB + 2 * ax + 1, ph, c, s);
                    }
            }
            const bool own = p >= 0 && q >= 1 && lane_own && y < ny;
            V an[3];
            // A: J: H from E (x+1 by shuffle down); K: E from H (x-1 by shuffle up)
            if constexpr (!MAG) {
                const V x1 = bO[1].dn(), x2 = bO[2].dn();
                updH(aO, bO, x1, x2, bN[0], bN[2], bZ[0], bZ[1], m_cur, (R)1, bA, py, pz, psA, own, an);
            } else {
                const V x1 = bO[1].up(), x2 = bO[2].up();
                updE(aO, bO, x1, x2, bN[0], bN[2], bZ[0], bZ[1], m_cur, (R)1, bA, false, py, pz, psA, own, an);
            }
            // B: J: E from H_new (x-1 by shuffle up); K: H from E_new (x+1 by shuffle down)
            const V ax1 = MAG ? an[1].dn() : an[1].up(), ax2 = MAG ? an[2].dn() : an[2].up();
            if (p >= 0 && q >= 1) {
                const V az0 = rg[q - 1][0][lane], az1 = rg[q - 1][1][lane];
                V bn[3];
                if constexpr (!MAG)
                    updE(bO, an, ax1, ax2, aPrev0, aPrev2, az0, az1, m_cur, aB, bB, first_e, py, pz, psB, own, bn);
                else
                    updH(bO, an, ax1, ax2, aPrev0, aPrev2, az0, az1, m_cur, aB, bB, py, pz, psB, own, bn);
                if (own) {
                    const unsigned g = (unsigned)pz.w * sz + (unsigned)py.w * sy + (unsigned)px.w;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        stq<R, CPLX>(Fo, aBase + k, N, g, an[k]);
                        stq<R, CPLX>(Fo, bBase + k, N, g, bn[k]);
                    }
                }
            }
            if (q >= 1) {
                rg[q - 1][0][lane] = an[0];
                rg[q - 1][1][lane] = an[1];
            }
            aPrev0 = an[0];
            aPrev2 = an[2];
#pragma unroll
            for (int k = 0; k < 3; ++k) bNprev[k] = bN[k];
        }
        if (!have) break;
        m_cur = m_nxt;
        reuse_cur = reuse;
        slot ^= 1;
        p = pn;
        q = qn;
    }
    cpa_wait<0>();

    // surface functional of the sigma group (E for J sources, H for K sources), from the output
    // buffer: this warp wrote every entry's cell
    if (t.ne > 0) {
        __syncwarp();
        double part = 0.0;
        for (int e = lane; e < t.ne; e += 32) {
            const DevEnt en = t.ents[e];
            const int loc = en.loc & 0xffff, arr = (en.loc >> 16) & 7, im = (en.loc >> 19) & 1;
            const int ly = loc >> 5, lx = loc & 31;
            const unsigned g = (unsigned)en.pad * sz + (unsigned)(t.j0 + ly) * sy + (unsigned)(t.i0 + lx);
            const unsigned plane = CPLX ? (unsigned)(2 * arr + im) : (unsigned)arr;
            part += (im ? -en.w : en.w) * (double)Fo[plane * N + g];
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
        if (lane == 0) {
            const double c = S.gw[n - 1] * part;
            atomicAdd(S.acc, c);
            if (n > S.tail_from) atomicAdd(S.tail, c);
        }
    }
}

// resident CTAs per SM asked of the register allocator, per precision and field type
#ifndef COL3_MINB_FR
#define COL3_MINB_FR 8
#endif
#ifndef COL3_MINB_FRP
#define COL3_MINB_FRP 5
#endif
#ifndef COL3_MINB_FC
#define COL3_MINB_FC 6
#endif
#ifndef COL3_MINB_DR
#define COL3_MINB_DR 6
#endif
#ifndef COL3_MINB_DC
#define COL3_MINB_DC 4
#endif

// MINB: resident CTAs per SM asked of the register allocator (the CPML variants carry more state)
template <typename R, bool CPLX, bool PML, int NPL, bool MAG, int MINB>
void launch_one(const DevSim6 *sims, const DevTile *tiles, int ntiles, const int64_t *lb, int64_t la, cudaStream_t st)
{
    constexpr int w = col3_warps((int)sizeof(R), CPLX, PML);
    constexpr int mb = PML && sizeof(R) == 4 && !CPLX ? COL3_MINB_FRP : MINB;
    k_col3<R, CPLX, PML, NPL, MAG, mb><<<(ntiles + w - 1) / w, w * 32, 0, st>>>(sims, tiles, ntiles, lb, la);
}

template <typename R, bool CPLX, int MINB>
void launch_variants(int variant, const DevSim6 *sims, const DevTile *tiles, int ntiles, const int64_t *lb, int64_t la,
                     cudaStream_t st)
{
    switch (variant) {
    case 0: launch_one<R, CPLX, false, 0, false, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 1: launch_one<R, CPLX, true, 0, false, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 2: launch_one<R, CPLX, false, 1, false, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 3: launch_one<R, CPLX, true, 1, false, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 4: launch_one<R, CPLX, false, 3, false, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 5: launch_one<R, CPLX, true, 3, false, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 6: launch_one<R, CPLX, false, 0, true, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 7: launch_one<R, CPLX, true, 0, true, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 8: launch_one<R, CPLX, false, 1, true, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 9: launch_one<R, CPLX, true, 1, true, MINB>(sims, tiles, ntiles, lb, la, st); break;
    case 10: launch_one<R, CPLX, false, 3, true, MINB>(sims, tiles, ntiles, lb, la, st); break;
    default: launch_one<R, CPLX, true, 3, true, MINB>(sims, tiles, ntiles, lb, la, st); break;
    }
}

}  // namespace

void launch_col3(int fp64, int cplx, int variant, const DevSim6 *sims, const DevTile *tiles, int ntiles,
                 const int64_t *launch_base, int64_t launch_add, cudaStream_t st)
{
    if (ntiles <= 0) return;
    if (fp64) {
        if (cplx) launch_variants<double, true, COL3_MINB_DC>(variant, sims, tiles, ntiles, launch_base, launch_add, st);
        else launch_variants<double, false, COL3_MINB_DR>(variant, sims, tiles, ntiles, launch_base, launch_add, st);
    } else {
        if (cplx) launch_variants<float, true, COL3_MINB_FC>(variant, sims, tiles, ntiles, launch_base, launch_add, st);
        else launch_variants<float, false, COL3_MINB_FR>(variant, sims, tiles, ntiles, launch_base, launch_add, st);
    }
}

}  // namespace cas
