// Two leapfrog steps per launch for the rotationally symmetric (r, z) cross-sections with
// fields ~ exp(i m phi) (Sec. III C and the appendix on cylindrical coordinates).
//
// The update of the cylindrical march in step6m.cu (stored components E_r, E_z, E_phi, H_r,
// H_z, H_phi on the sites of E_x .. H_z, x = r from the axis, y = z, d/dphi -> +-m in the
// real-phase form, per-lane radial factors, the Stokes row on the axis), fused over two
// consecutive steps A = 2L-1 and B = 2L so that every field is read and written once per two
// steps.  A warp owns a strip of MARCH_W2 = 28 columns plus two halo lanes on each side (each
// step leaves one more outer lane stale) and marches down the tile's rows: electric sources
// update H then E, step B one row behind step A; magnetic sources update E one row ahead then
// H, step B's E at step A's H row.  The sigma group of both steps is projected from registers
// (row-sorted entries, shuffle hand-over).  Fields read buffer (L-1)&1 and write L&1; the
// last launch of an odd run holds step A alone.
#include <cuda_runtime.h>

#include "kernels.h"

namespace cas {

namespace {

constexpr int WARPS_C2 = 4;   // warps (strips) per CTA
// 1: the next iteration's field values staged by cp.async; 0: loaded into registers ahead
#ifndef CYL2_STG
#define CYL2_STG 1
#endif

template <typename R>
__device__ __forceinline__ R cdn(R v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename R>
__device__ __forceinline__ R cup(R v) { return __shfl_up_sync(0xffffffffu, v, 1); }

// Asynchronous copy of one element, global -> shared (cp.async of the lane's own value)
template <typename R>
__device__ __forceinline__ void cpa(R *sdst, const R *gsrc)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sdst);
    if constexpr (sizeof(R) == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gsrc) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Projection of the sigma group's three components at tile row ly (entries rowptr[ly] ..
// rowptr[ly+1], loc = ly * MARCH_W2 + lx, the component in bits 16..18): lanes 2 .. w + 1
// hold the strip's columns.
template <typename R>
__device__ __forceinline__ double project_row_c2(const DevTile2 &t, int ly, int w, int grp, R v0, R v1, R v2)
{
    double part = 0.0;
    const int e0 = t.rowptr[ly], e1 = t.rowptr[ly + 1];
    for (int base = e0; base < e1; base += 32) {
        const int e = base + (int)(threadIdx.x & 31);
        int c = 0, lx = -1;
        double wgt = 0.0;
        if (e < e1) {
            const DevEnt en = t.ents[e];
            lx = (en.loc & 0xffff) - ly * MARCH_W2;
            c = ((en.loc >> 16) & 7) - grp;
            wgt = en.w;
        }
        const bool mine = lx >= 0 && lx < w;
        const int src = mine ? lx + 2 : 0;
        const R a0 = __shfl_sync(0xffffffffu, v0, src);
        const R a1 = __shfl_sync(0xffffffffu, v1, src);
        const R a2 = __shfl_sync(0xffffffffu, v2, src);
        if (mine) part += wgt * (double)(c == 0 ? a0 : (c == 1 ? a1 : a2));
    }
    return part;
}

// STG = 1: the next iteration's six field values are copied by cp.async into a per-lane
// shared-memory ring of two slots while the current one computes; STG = 0: they are loaded
// into registers one iteration ahead
template <typename R, int MINB, int STG>
__global__ void __launch_bounds__(WARPS_C2 * 32, MINB)
k_cyl2(const DevSim6 *__restrict__ sims, const DevTile2 *__restrict__ tiles, int ntiles,
       const int64_t *__restrict__ launch_base, int64_t launch_add)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ti = blockIdx.x * WARPS_C2 + warp;
    if (ti >= ntiles) return;
    const DevTile2 t = tiles[ti];
    const DevSim6 &S = sims[t.sim];
    const int64_t L = *launch_base + launch_add - S.s0;
    const int64_t nA = 2 * L - 1;
    if (L < 1 || nA > S.T) return;
    const bool two = nA + 1 <= S.T;

    const int nx = S.n[0], ny = S.n[1];
    const unsigned N = (unsigned)nx * (unsigned)ny;   // 32-bit offsets: 12 N < 2^32 (checked by the planner)
    const R *__restrict__ fin = reinterpret_cast<const R *>(S.fields) + (size_t)((L - 1) & 1) * S.fhalf;
    R *__restrict__ fout = reinterpret_cast<R *>(S.fields) + (size_t)(L & 1) * S.fhalf;
    const R *__restrict__ coef = reinterpret_cast<const R *>(S.coef);
    const uint8_t *__restrict__ mat = S.mat;

    const int i0 = t.i0;
    const int w = min(MARCH_W2, nx - i0);
    const int h = min(S.tile_rows, ny - t.j0);
    const int col = ((i0 - 2 + lane) % nx + nx) % nx;   // lanes 0, 1 and w + 2, w + 3: halo columns
    const bool own = lane >= 2 && lane < w + 2;
    const bool wrapR = col == nx - 1, wrapL = col == 0;
    const R bxr = (R)S.bre[0], byr = (R)S.bre[1];   // real phases: PEC wall at r = R, z periodic or PEC
    const R idx = (R)S.inv_dx;
    const R kA = (R)S.kzA, kB = (R)S.kzB;
    const R a = (R)S.a, bs = (R)S.bs;
    const R hA0 = (R)(nA == 1 ? 0.5 * S.dt : S.dt), hB0 = (R)S.dt;
    const bool electric = S.magnetic == 0;
    const int grp = electric ? 0 : 3;   // the measured (sigma) group: E for J sources, H for K sources

    // radial factors of this lane's column i (r_i = i Delta, r_{i+1/2}); on the axis the Stokes
    // form 4 H_phi(Delta/2) / Delta (fa = 4, fb = 0)
    // (Delta cancels from the ratios: each factor is one correctly rounded division of exact
    // operands in the run's precision, so FP32 runs need no FP64 arithmetic per thread)
    const R ci = (R)col, ch = ci + (R)0.5, ix = (R)S.inv_dx;
    const R inv_ri = col > 0 ? ix / ci : (R)0, inv_rh = ix / ch;
    const R ga = (ci + (R)1) / ch, gb = ci / ch;
    const R fa = col > 0 ? ch / ci : (R)4, fb = col > 0 ? (ci - (R)0.5) / ci : (R)0;

    auto right = [&](R f) -> R { const R r = cdn(f); return wrapR ? r * bxr : r; };
    auto left = [&](R f) -> R { const R l = cup(f); return wrapL ? l * bxr : l; };
    // any row index to [0, ny)
    auto wrow = [&](int j) { j %= ny; return j < 0 ? j + ny : j; };
    auto ldr = [&](int plane, int j) -> R { return fin[(unsigned)plane * N + (unsigned)(j * nx + col)]; };
    // staged inputs: [slot][value][lane], six field values per iteration
    __shared__ __align__(16) R ring_s[STG > 0 ? WARPS_C2 : 1][2][6][32];
    auto sg = [&](int slot, int v, int plane, int j) { cpa(&ring_s[warp][slot][v][lane], fin + (unsigned)plane * N + (unsigned)(j * nx + col)); };
    auto fv = [&](int slot, int v) -> R { return ring_s[warp][slot][v][lane]; };

    // H at row j (wrapped) from E at rows j and j+1 (E_r, E_phi of row j+1: exn, ezn)
    auto updH = [&](int j, int m, const R e[3], R exn, R ezn, const R hq[3], R aa, R bb, R ho[3]) {
        if (j + 1 >= ny) { exn = exn * byr; ezn = ezn * byr; }
        const R dyEz = (ezn - e[2]) * idx, dyEx = (exn - e[0]) * idx;
        const R dxEy = (right(e[1]) - e[1]) * idx;
        const R dxEphi = (right(e[2]) * ga - e[2] * gb) * idx;
        const R *cm = coef + 6 * m;
        ho[0] = hq[0] * aa - (e[1] * (kA * inv_ri) - dyEz) * (bb * cm[3]);
        ho[1] = hq[1] * aa - (dxEphi - e[0] * (kA * inv_rh)) * (bb * cm[4]);
        ho[2] = hq[2] * aa - (dyEx - dxEy) * (bb * cm[5]);
    };
    // E at row j (wrapped) from H at rows j and j-1 (H_r, H_phi of row j-1: hxp, hzp)
    auto updE = [&](int j, int m, const R hh[3], R hxp, R hzp, const R eo[3], R aa, R bb, R en[3]) {
        if (j - 1 < 0) { hxp = hxp * byr; hzp = hzp * byr; }
        const R dyHz = (hh[2] - hzp) * idx, dyHx = (hh[0] - hxp) * idx;
        const R dxHy = (hh[1] - left(hh[1])) * idx;
        const R dxHphi = (hh[2] * fa - left(hh[2]) * fb) * idx;
        const R *cm = coef + 6 * m;
        const R c0 = hh[1] * (kB * inv_rh) - dyHz;
        const R c1 = dxHphi - hh[0] * (kB * inv_ri);
        const R c2 = dyHx - dxHy;
        en[0] = eo[0] * aa + c0 * (bb * cm[0]);
        en[1] = eo[1] * aa + c1 * (bb * cm[1]);
        en[2] = eo[2] * aa + c2 * (bb * cm[2]);
    };
    auto store = [&](int j, const R e[3], const R hh[3]) {
        if (!own) return;
        const unsigned g = (unsigned)(j * nx + col);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            fout[(unsigned)k * N + g] = e[k];
            fout[(unsigned)(3 + k) * N + g] = hh[k];
        }
    };

    double pA = 0.0, pB = 0.0;
    const int j0 = t.j0;
    if (w > 0) {
        if (electric) {
            // carried: the buffer's E at row r, H_A at r-1, E_A at r-1, H_B at r-2 (+ materials)
            R e0c[3], hAm[3], eAm[3] = {0, 0, 0}, hBm[3] = {0, 0, 0};
            int m_r, m_rm = 0;
            {
                const int ja = wrow(j0 - 2), jb = wrow(j0 - 1);
                const R ea[3] = {ldr(0, ja), ldr(1, ja), ldr(2, ja)};
                const R ha[3] = {ldr(3, ja), ldr(4, ja), ldr(5, ja)};
#pragma unroll
                for (int k = 0; k < 3; ++k) e0c[k] = ldr(k, jb);
                updH(ja, mat[(unsigned)(ja * nx + col)], ea, e0c[0], e0c[2], ha, (R)1, hA0, hAm);   // H_A(j0-2)
                m_r = mat[(unsigned)(jb * nx + col)];
            }
            // inputs of iteration r: the buffer's E at row r+1, H at row r, material of row r+1
            R en_c[3], hq_c[3];
            int mn_c;
            int jr = wrow(j0 - 1), jp = wrow(j0 - 2);   // rows r and r-1, wrapped
            // staged: slot `sl` holds this iteration's E(r+1) (values 0..2) and H(r) (3..5)
            int sl = 0;
            auto stage_e = [&](int slot, int j) {   // iteration of row j (wrapped)
                const int jn_ = j + 1 == ny ? 0 : j + 1;
#pragma unroll
                for (int k = 0; k < 3; ++k) { sg(slot, k, k, jn_); sg(slot, 3 + k, 3 + k, j); }
            };
            {
                const int jn = jr + 1 == ny ? 0 : jr + 1;
                if constexpr (STG > 0) {
                    stage_e(0, jr);
                    cpa_commit();
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) { en_c[k] = ldr(k, jn); hq_c[k] = ldr(3 + k, jr); }
                }
                mn_c = mat[(unsigned)(jn * nx + col)];
            }
            for (int r = j0 - 1; r <= j0 + h; ++r) {
                const int jn = jr + 1 == ny ? 0 : jr + 1;
                R en_n[3], hq_n[3];
                int mn_n = 0;
                if (r + 1 <= j0 + h) {   // the next iteration's inputs, loaded ahead
                    const int jnn = jn + 1 == ny ? 0 : jn + 1;
                    if constexpr (STG > 0) {
                        stage_e(sl ^ 1, jn);
                    } else {
#pragma unroll
                        for (int k = 0; k < 3; ++k) { en_n[k] = ldr(k, jnn); hq_n[k] = ldr(3 + k, jn); }
                    }
                    mn_n = mat[(unsigned)(jnn * nx + col)];
                }
                if constexpr (STG > 0) {
                    cpa_commit();
                    cpa_wait<1>();
#pragma unroll
                    for (int k = 0; k < 3; ++k) { en_c[k] = fv(sl, k); hq_c[k] = fv(sl, 3 + k); }
                    sl ^= 1;
                }
                R hA[3], eA[3];
                updH(jr, m_r, e0c, en_c[0], en_c[2], hq_c, (R)1, hA0, hA);
                updE(jr, m_r, hA, hAm[0], hAm[2], e0c, a, bs, eA);
                const bool inA = r >= j0 && r < j0 + h;
                if (inA && t.ne > 0) pA += project_row_c2<R>(t, r - j0, w, grp, eA[0], eA[1], eA[2]);
                if (!two) {
                    if (inA) store(jr, eA, hA);
                } else if (r == j0) {
                    updH(jp, m_rm, eAm, eA[0], eA[2], hAm, (R)1, hB0, hBm);   // H_B(j0-1)
                } else if (r > j0) {
                    const int jm = jp;
                    R hB[3], eB[3];
                    updH(jm, m_rm, eAm, eA[0], eA[2], hAm, (R)1, hB0, hB);
                    updE(jm, m_rm, hB, hBm[0], hBm[2], eAm, a, bs, eB);
                    if (r - 1 < j0 + h) {
                        store(jm, eB, hB);
                        if (t.ne > 0) pB += project_row_c2<R>(t, r - 1 - j0, w, grp, eB[0], eB[1], eB[2]);
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k) hBm[k] = hB[k];
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    eAm[k] = eA[k];
                    hAm[k] = hA[k];
                    e0c[k] = en_c[k];
                    if constexpr (STG == 0) {
                        en_c[k] = en_n[k];
                        hq_c[k] = hq_n[k];
                    }
                }
                m_rm = m_r;
                m_r = mn_c;
                mn_c = mn_n;
                jp = jr;
                jr = jn;
            }
        } else {
            // carried: E_A at row r, the buffer's H at row r, H_A at r-1, E_B at r-1 (+ materials)
            R eAc[3], h0c[3], hAm[3] = {0, 0, 0}, eBm[3] = {0, 0, 0};
            int m_r, m_rm = 0;
            int jr = wrow(j0 - 1), jp = wrow(j0 - 2);   // rows r and r-1, wrapped
            {
                const int ja = jp;
                const R hb2[3] = {ldr(3, ja), ldr(4, ja), ldr(5, ja)};
                const R e0[3] = {ldr(0, jr), ldr(1, jr), ldr(2, jr)};
#pragma unroll
                for (int k = 0; k < 3; ++k) h0c[k] = ldr(3 + k, jr);
                m_r = mat[(unsigned)(jr * nx + col)];
                updE(jr, m_r, h0c, hb2[0], hb2[2], e0, (R)1, hA0, eAc);   // E_A(j0-1)
            }
            // inputs of iteration r: the buffer's H and E at row r+1, material of row r+1
            R hn_c[3], en_c[3];
            int mn_c;
            // staged: slot `sl` holds this iteration's H(r+1) (values 0..2) and E(r+1) (3..5)
            int sl = 0;
            auto stage_m = [&](int slot, int jn_) {   // row r+1 (wrapped) of the staged iteration
#pragma unroll
                for (int k = 0; k < 3; ++k) { sg(slot, k, 3 + k, jn_); sg(slot, 3 + k, k, jn_); }
            };
            {
                const int jn = jr + 1 == ny ? 0 : jr + 1;
                if constexpr (STG > 0) {
                    stage_m(0, jn);
                    cpa_commit();
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) { hn_c[k] = ldr(3 + k, jn); en_c[k] = ldr(k, jn); }
                }
                mn_c = mat[(unsigned)(jn * nx + col)];
            }
            for (int r = j0 - 1; r <= j0 + h; ++r) {
                const int jn = jr + 1 == ny ? 0 : jr + 1;
                R hn_n[3], en_n[3];
                int mn_n = 0;
                if (r + 1 <= j0 + h) {
                    const int jnn = jn + 1 == ny ? 0 : jn + 1;
                    if constexpr (STG > 0) {
                        stage_m(sl ^ 1, jnn);
                    } else {
#pragma unroll
                        for (int k = 0; k < 3; ++k) { hn_n[k] = ldr(3 + k, jnn); en_n[k] = ldr(k, jnn); }
                    }
                    mn_n = mat[(unsigned)(jnn * nx + col)];
                }
                if constexpr (STG > 0) {
                    cpa_commit();
                    cpa_wait<1>();
#pragma unroll
                    for (int k = 0; k < 3; ++k) { hn_c[k] = fv(sl, k); en_c[k] = fv(sl, 3 + k); }
                    sl ^= 1;
                }
                R eAn[3], hA[3];
                updE(jn, mn_c, hn_c, h0c[0], h0c[2], en_c, (R)1, hA0, eAn);   // E_A(r+1)
                updH(jr, m_r, eAc, eAn[0], eAn[2], h0c, a, bs, hA);          // H_A(r)
                const bool inA = r >= j0 && r < j0 + h;
                if (inA && t.ne > 0) pA += project_row_c2<R>(t, r - j0, w, grp, hA[0], hA[1], hA[2]);
                if (!two) {
                    if (inA) store(jr, eAc, hA);
                } else if (r >= j0) {
                    R eB[3];
                    updE(jr, m_r, hA, hAm[0], hAm[2], eAc, (R)1, hB0, eB);   // E_B(r)
                    if (r > j0) {
                        const int jm = jp;
                        R hB[3];
                        updH(jm, m_rm, eBm, eB[0], eB[2], hAm, a, bs, hB);    // H_B(r-1)
                        if (r - 1 < j0 + h) {
                            store(jm, eBm, hB);
                            if (t.ne > 0) pB += project_row_c2<R>(t, r - 1 - j0, w, grp, hB[0], hB[1], hB[2]);
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 3; ++k) eBm[k] = eB[k];
                }
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    hAm[k] = hA[k];
                    eAc[k] = eAn[k];
                    h0c[k] = hn_c[k];
                    if constexpr (STG == 0) {
                        hn_c[k] = hn_n[k];
                        en_c[k] = en_n[k];
                    }
                }
                m_rm = m_r;
                m_r = mn_c;
                mn_c = mn_n;
                jp = jr;
                jr = jn;
            }
        }
    }

    if (t.ne > 0) {
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
}

}  // namespace

void launch_march6_cyl2(int fp64, const DevSim6 *sims, const DevTile2 *tiles, int ntiles,
                        const int64_t *launch_base, int64_t launch_add, cudaStream_t st)
{
    if (ntiles <= 0) return;
    const int grid = (ntiles + WARPS_C2 - 1) / WARPS_C2;
    if (fp64) k_cyl2<double, 4, CYL2_STG><<<grid, WARPS_C2 * 32, 0, st>>>(sims, tiles, ntiles, launch_base, launch_add);
    else k_cyl2<float, 5, CYL2_STG><<<grid, WARPS_C2 * 32, 0, st>>>(sims, tiles, ntiles, launch_base, launch_add);
}

}  // namespace cas
