// Request executor and C ABI (include/casimir.h).
//
// A context owns one CUDA stream, a device-memory budget and a worker thread.
// Requests (one force computation of a plan each) are admitted while their
// device memory fits the budget; every admitted simulation joins one batched
// launch per time step, so requests of different sizes and different start
// times advance together (continuous batching).  A simulation's step index is
// the global launch index minus its start index, kept on the device so that a
// chunk of steps can be replayed as one CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <new>
#include <stdexcept>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine_internal.h"

namespace {
thread_local std::string g_err;
}  // namespace

namespace cas {

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace cas

// ---------------------------------------------------------------------------------
// memory helpers
// ---------------------------------------------------------------------------------

int dev_alloc(casimir_ctx *c, size_t bytes, void **out)
{
    if (c->alloc) {
        *out = c->alloc(bytes, c->user);
        if (!*out) return fail(CASIMIR_ENOMEM, "allocator callback returned NULL");
        return CASIMIR_OK;
    }
    cudaError_t e = cudaMalloc(out, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CASIMIR_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return CASIMIR_OK;
}

void dev_free(casimir_ctx *c, void *p)
{
    if (!p) return;
    if (c->freef) c->freef(p, c->user);
    else cudaFree(p);
}

// ---------------------------------------------------------------------------------
// plan preparation (host)
// ---------------------------------------------------------------------------------

static int prepare_plan(casimir_plan_t *P)
{
    PlanData &D = P->data;
    P->fp64 = D.prob.precision == CASIMIR_FP64;
    P->rsize = P->fp64 ? 8 : 4;
    // geometry tables
    for (auto &g : D.geos) {
        P->mat_off.push_back((int64_t)P->mat_all.size());
        P->mat_all.insert(P->mat_all.end(), g.mat.begin(), g.mat.end());
        size_t pad = align256(P->mat_all.size()) - P->mat_all.size();
        P->mat_all.insert(P->mat_all.end(), pad, 0);
        P->coef_off.push_back((int64_t)P->coef_all.size());
        P->coef_all.insert(P->coef_all.end(), g.table.begin(), g.table.end());
        while (P->coef_all.size() % 32) P->coef_all.push_back(0.0);
        // (site, pole) pairs of the grid: the Lorentz planes one step reads and writes
        {
            int64_t pairs = 0;
            if (g.family == FAM_FULL && g.has_lorentz) {
                std::vector<int64_t> per_id(g.nmat, 0);
                for (int id = 0; id < g.nmat; ++id)
                    for (int q = 0; q < g.npoles; ++q)
                        for (int c = 0; c < 3; ++c)
                            if (g.lorentz[((size_t)id * g.npoles + q) * 6 + 2 * c] != 0.0) ++per_id[id];
                for (uint8_t id : g.mat) pairs += per_id[id];
            }
            P->lor_sites.push_back(pairs);
        }
        P->lor_off.push_back((int64_t)P->lor_all.size());
        if (g.family == FAM_FULL) P->lor_all.insert(P->lor_all.end(), g.lorentz.begin(), g.lorentz.end());
        // kernel form of the Lorentz recurrence of every pole: P' = (cp P - cpm P_prev + ce E) cd
        P->lorc_off.push_back((int64_t)P->lorc_all.size());
        if (g.family == FAM_FULL && g.has_lorentz) {
            const double dt = D.dt, sg = D.prob.sigma;
            // [id][pole][component]: the table of Geo::lorentz in the same order
            for (size_t ic = 0; ic < g.lorentz.size() / 2; ++ic) {
                const double de = g.lorentz[2 * ic], w0 = g.lorentz[2 * ic + 1];
                const double w2dt2 = w0 * w0 * dt * dt;
                P->lorc_all.push_back(2.0 - w2dt2);
                P->lorc_all.push_back(1.0 - 0.5 * sg * dt);
                P->lorc_all.push_back(de * w2dt2);
                P->lorc_all.push_back(1.0 / (1.0 + 0.5 * sg * dt));
            }
            while (P->lorc_all.size() % 32) P->lorc_all.push_back(0.0);
        }
        std::array<int64_t, 3> po{-1, -1, -1};
        for (int a = 0; a < 3; ++a)
            if (g.has_pml[a]) {
                po[a] = (int64_t)P->pml_all.size();
                for (int h = 0; h < 2; ++h)
                    for (int q = 0; q < 3; ++q) P->pml_all.insert(P->pml_all.end(), g.pml[a][h][q].begin(), g.pml[a][h][q].end());
                while (P->pml_all.size() % 32) P->pml_all.push_back(0.0);
            }
        P->pml_off.push_back(po);
    }
    // sims, tiles, entries, sources
    int64_t off = 0;
    std::map<int, std::vector<int>> march_variants;   // per geometry: kernel variant of each march tile
    std::map<int, std::vector<int>> mar2_variants;    // per geometry: variant of each two-step march tile
    for (size_t s = 0; s < D.sims.size(); ++s) {
        const Sim &sm = D.sims[s];
        const Geo &g = D.geos[sm.geo];
        HostSim hs{};
        hs.geo = sm.geo;
        hs.nx = g.n[0];
        hs.ny = g.n[1];
        hs.nz = g.n[2];
        hs.second_u = sm.second_u;
        hs.full = g.family == FAM_FULL;
        hs.magnetic = sm.kind;
        hs.field_off = off;
        hs.psi_off = -1;
        hs.lor_off = -1;
        int64_t N = (int64_t)hs.nx * hs.ny * hs.nz;
        P->cells += N;
        if (!hs.full) {
            if (3 * N >= ((int64_t)1 << 32)) return fail(CASIMIR_EINVAL, "two-dimensional grid too large (3 N >= 2^32)");
            off += 6 * N;
            off = (off + 63) & ~(int64_t)63;
            int tx = (hs.nx + TILE_X - 1) / TILE_X, ty = (hs.ny + TILE_Y - 1) / TILE_Y;
            hs.tile0 = (int)P->tiles.size();
            hs.ntile = tx * ty;
            std::vector<std::vector<DevEnt>> bucket(hs.ntile);
            for (const Entry &e : sm.meas) {
                int i = (int)(e.idx % hs.nx), j = (int)(e.idx / hs.nx);
                int ti = i / TILE_X, tj = j / TILE_Y;
                int loc = (j - tj * TILE_Y) * TILE_X + (i - ti * TILE_X);
                bucket[tj * tx + ti].push_back(DevEnt{loc | (e.arr << 16), 0, e.re});
            }
            hs.ent0 = (int)P->ents.size();
            for (int tj = 0; tj < ty; ++tj)
                for (int ti = 0; ti < tx; ++ti) {
                    auto &b = bucket[tj * tx + ti];
                    HostTile ht{(int)s, ti * TILE_X, tj * TILE_Y, (int)P->ents.size(), (int)b.size()};
                    P->ents.insert(P->ents.end(), b.begin(), b.end());
                    P->tiles.push_back(ht);
                }
            hs.nent = (int)P->ents.size() - hs.ent0;
            hs.src0 = (int)P->src.size();
            for (const Entry &e : sm.src) P->src.push_back(DevSrc{hs.field_off + e.arr * N + e.idx, e.re});
            hs.nsrc = (int)P->src.size() - hs.src0;
            // multi-step tiles: tile_xk(K) wide for K steps per launch, entries sorted by row with
            // per-row offsets
            {
                const int TXK = tile_xk(P->opts.steps_per_launch == 3 ? 3 : 2);
                int tx2 = (hs.nx + TXK - 1) / TXK;
                std::vector<std::vector<std::pair<int, DevEnt>>> b2(tx2 * ty);
                for (const Entry &e : sm.meas) {
                    int i = (int)(e.idx % hs.nx), j = (int)(e.idx / hs.nx);
                    int ti = i / TXK, tj = j / TILE_Y;
                    int ly = j - tj * TILE_Y, lx = i - ti * TXK;
                    b2[tj * tx2 + ti].push_back({ly * TXK + lx, DevEnt{(ly * TXK + lx) | (e.arr << 16), 0, e.re}});
                }
                hs.tile2_0 = (int)P->tiles2.size();
                for (int tj = 0; tj < ty; ++tj)
                    for (int ti = 0; ti < tx2; ++ti) {
                        auto &b = b2[tj * tx2 + ti];
                        std::stable_sort(b.begin(), b.end(), [](const std::pair<int, DevEnt> &x, const std::pair<int, DevEnt> &y) {
                            return x.first < y.first;
                        });
                        HostTile2 ht{(int)s, ti * TXK, tj * TILE_Y, (int)P->ents2.size(), (int)b.size(), (int)P->rowptr2.size()};
                        int k = 0;
                        for (int ly = 0; ly <= TILE_Y; ++ly) {
                            while (k < (int)b.size() && b[k].first / TXK < ly) ++k;
                            P->rowptr2.push_back(ly == TILE_Y ? (int)b.size() : k);
                        }
                        for (auto &pe : b) P->ents2.push_back(pe.second);
                        P->tiles2.push_back(ht);
                    }
                hs.ntile2 = (int)P->tiles2.size() - hs.tile2_0;
            }
        } else {
            hs.cplx = g.complex_fields ? 1 : 0;
            int cf = hs.cplx ? 2 : 1;
            // real fields: the source's set {Ex, Ey, Hz} or {Ez, Hx, Hy} is stored as is, the other
            // divided by i; d/dz = i kz then acts as +kz on the stored source set and -kz on the other
            int sarr = sm.src.empty() ? 0 : sm.src[0].arr;
            auto inA = [](int arr) { return arr == 0 || arr == 1 || arr == 5; };
            double sgn = inA(sarr) ? 1.0 : -1.0;
            // d/dz -> i k_z (Cartesian) or d/dphi -> i m (cylindrical): the same real-phase split
            const double kq = g.cyl ? (double)g.mphi : g.kz;
            hs.kzA = sgn * kq;
            hs.kzB = -sgn * kq;
            hs.cyl = g.cyl ? 1 : 0;
            const int rows = P->opts.march_rows;
            // two-dimensional runs march both half steps in one launch over ping-pong buffers
            static const bool march_env = [] {
                const char *e = std::getenv("CASIMIR_MARCH6");
                return !(e && std::atoi(e) == 0);
            }();
            // (its 32-bit element offsets reach 12 N within one buffer)
            const int64_t planes = 12 * std::max(1, g.npoles);   // complex planes of fields or Lorentz P
            hs.march = (D.prob.dims == 2 && g.n[2] == 1 && march_env && planes * N < ((int64_t)1 << 32)) ? 1 : 0;
            if (g.cyl && !hs.march)   // only the march kernel has the cylindrical form
                return fail(CASIMIR_EINVAL, "cylindrical runs need the march kernel (12 N < 2^32 cells)");
            // three-dimensional runs: the column march (both half steps per launch, ping-pong
            // buffers) by default, the x-line or per-cell kernels (in place) on request
            hs.col3 = (!hs.march && D.prob.dims == 3 && P->opts.kernel_3d == 3 && planes * N < ((int64_t)1 << 32)) ? 1 : 0;
            const int nbuf = (hs.march || hs.col3) ? 2 : 1;
            hs.fhalf = 6 * cf * N;
            off += nbuf * hs.fhalf;
            hs.psi_half = 0;
            for (int a = 0; a < 3; ++a)
                if (g.has_pml[a]) hs.psi_half += 4 * cf * (N / g.n[a]) * 2 * D.prob.pml_cells[a];
            if (hs.psi_half > 0) {
                hs.psi_off = off;
                off += nbuf * hs.psi_half;
            }
            hs.lor_half = g.has_lorentz ? 6 * g.npoles * cf * N : 0;
            hs.npoles = g.npoles;
            if (g.has_lorentz) {
                hs.lor_off = off;
                off += nbuf * hs.lor_half;
            }
            off = (off + 63) & ~(int64_t)63;
            if (hs.march) {
                // one strip tile (MARCH_W x MARCH_H) per warp, row bands outer; entries carry the
                // component in bits 16..18 and, for the imaginary weight of complex fields, bit 19
                int tx = (hs.nx + MARCH_W - 1) / MARCH_W, ty = (hs.ny + rows - 1) / rows;
                // kernel variant of each tile: the CPML and Lorentz code paths only where the tile's
                // halo-extended box [i0-1, i0+w] x [j0-1, j0+h] holds such cells (cached per geometry)
                auto vit = march_variants.find(sm.geo);
                if (vit == march_variants.end()) {
                    // poles of each material (the most over its three E components)
                    std::vector<int> dmat(g.nmat, 0);
                    for (int id = 0; id < g.nmat; ++id)
                        for (int q = 0; q < g.npoles; ++q)
                            for (int c = 0; c < 3; ++c)
                                if (g.lorentz[((size_t)id * g.npoles + q) * 6 + 2 * c] != 0.0) dmat[id] = std::max(dmat[id], q + 1);
                    const int dX = g.has_pml[0] ? D.prob.pml_cells[0] : 0, dY = g.has_pml[1] ? D.prob.pml_cells[1] : 0;
                    const bool xper = D.prob.bc[0] == CASIMIR_BC_PERIODIC, yper = D.prob.bc[1] == CASIMIR_BC_PERIODIC;
                    auto wrapc = [](int i, int n) { return ((i % n) + n) % n; };
                    std::vector<int> vs((size_t)tx * ty, 0);
                    for (int tj = 0; tj < ty; ++tj)
                        for (int ti = 0; ti < tx; ++ti) {
                            const int i0 = ti * MARCH_W, j0 = tj * rows;
                            const int w = std::min(MARCH_W, hs.nx - i0), h = std::min(rows, hs.ny - j0);
                            bool pml = false;
                            int poles = 0;
                            for (int jj = j0 - 1; jj <= j0 + h; ++jj) {
                                const int j = wrapc(jj, hs.ny);
                                if (dY > 0 && (j < dY || j >= hs.ny - dY)) pml = true;
                                for (int ii = i0 - 1; ii <= i0 + w; ++ii) {
                                    const int i = wrapc(ii, hs.nx);
                                    if (dX > 0 && (i < dX || i >= hs.nx - dX)) pml = true;
                                    // across a closed (PEC or CPML) wall the halo cell is the wall
                                    // row or column: the components the tile uses there are masked
                                    // and carry no poles
                                    if ((jj != j && !yper) || (ii != i && !xper)) continue;
                                    poles = std::max(poles, dmat[g.mat[(size_t)j * hs.nx + i]]);
                                }
                            }
                            vs[(size_t)tj * tx + ti] = (pml ? 1 : 0) + (poles == 0 ? 0 : poles == 1 ? 2 : 4);
                        }
                    vit = march_variants.emplace(sm.geo, std::move(vs)).first;
                }
                std::vector<std::vector<DevEnt>> bucket((size_t)tx * ty);
                for (const Entry &e : sm.meas) {
                    if (!hs.cplx && inA(e.arr) != inA(sarr)) continue;   // contributes i * real: no real part
                    int i = (int)(e.idx % hs.nx), j = (int)(e.idx / hs.nx);
                    int ti = i / MARCH_W, tj = j / rows;
                    int loc = (j - tj * rows) * MARCH_W + (i - ti * MARCH_W);
                    auto &b = bucket[(size_t)tj * tx + ti];
                    if (e.re != 0.0 || !hs.cplx) b.push_back(DevEnt{loc | (e.arr << 16), 0, e.re});
                    if (hs.cplx && e.im != 0.0) b.push_back(DevEnt{loc | ((e.arr | 8) << 16), 0, e.im});
                }
                hs.tile0 = (int)P->tilesM.size();
                hs.ntile = tx * ty;
                hs.ent0 = (int)P->entsM.size();
                for (int tj = 0; tj < ty; ++tj)
                    for (int ti = 0; ti < tx; ++ti) {
                        auto &b = bucket[(size_t)tj * tx + ti];
                        P->tilesM.push_back(HostTile{(int)s, ti * MARCH_W, tj * rows, (int)P->entsM.size(), (int)b.size(),
                                                     vit->second[(size_t)tj * tx + ti]});
                        P->entsM.insert(P->entsM.end(), b.begin(), b.end());
                    }
                hs.nent = (int)P->entsM.size() - hs.ent0;
                // two steps per launch: cylindrical runs, and Cartesian FP32 runs whose materials have
                // at most one Lorentz pole (the two-step march carries one pole's state per cell)
                int geo_poles = 0;
                for (int id = 0; id < g.nmat; ++id)
                    for (int q = 0; q < g.npoles; ++q)
                        for (int c = 0; c < 3; ++c)
                            if (g.lorentz[((size_t)id * g.npoles + q) * 6 + 2 * c] != 0.0) geo_poles = std::max(geo_poles, q + 1);
                if (P->opts.steps_per_launch >= 2 && (hs.cyl || (!P->fp64 && geo_poles <= 1))) {
                    // MARCH_W2-wide strips, entries sorted by row with per-row offsets (the sigma
                    // group is projected from registers)
                    const int tx2 = (hs.nx + MARCH_W2 - 1) / MARCH_W2;
                    // kernel variant of each Cartesian tile: the CPML and Lorentz code paths only where
                    // the box that two steps reach, [i0-2, i0+w+1] x [j0-2, j0+h+1], holds such cells
                    auto v2 = mar2_variants.find(sm.geo);
                    if (!hs.cyl && v2 == mar2_variants.end()) {
                        const int dX = g.has_pml[0] ? D.prob.pml_cells[0] : 0, dY = g.has_pml[1] ? D.prob.pml_cells[1] : 0;
                        const bool xper = D.prob.bc[0] == CASIMIR_BC_PERIODIC, yper = D.prob.bc[1] == CASIMIR_BC_PERIODIC;
                        auto wrapc = [](int i, int n) { return ((i % n) + n) % n; };
                        std::vector<bool> disp(g.nmat, false);
                        for (int id = 0; id < g.nmat; ++id)
                            for (int c = 0; c < 3 && g.npoles > 0; ++c)
                                if (g.lorentz[((size_t)id * g.npoles) * 6 + 2 * c] != 0.0) disp[id] = true;
                        std::vector<int> vs((size_t)tx2 * ty, 0);
                        for (int tj = 0; tj < ty; ++tj)
                            for (int ti = 0; ti < tx2; ++ti) {
                                const int i0 = ti * MARCH_W2, j0 = tj * rows;
                                const int w = std::min(MARCH_W2, hs.nx - i0), h = std::min(rows, hs.ny - j0);
                                bool pml = false, lor = false;
                                for (int jj = j0 - 2; jj <= j0 + h + 1; ++jj) {
                                    const int j = wrapc(jj, hs.ny);
                                    if (dY > 0 && (j < dY || j >= hs.ny - dY)) pml = true;
                                    for (int ii = i0 - 2; ii <= i0 + w + 1; ++ii) {
                                        const int i = wrapc(ii, hs.nx);
                                        if (dX > 0 && (i < dX || i >= hs.nx - dX)) pml = true;
                                        // across a closed wall the halo cells are wall cells: the
                                        // components the tile uses there are masked
                                        if ((jj != j && !yper) || (ii != i && !xper)) continue;
                                        lor = lor || disp[g.mat[(size_t)j * hs.nx + i]];
                                    }
                                }
                                vs[(size_t)tj * tx2 + ti] = (pml ? 1 : 0) + (lor ? 2 : 0);
                            }
                        v2 = mar2_variants.emplace(sm.geo, std::move(vs)).first;
                    }
                    std::vector<std::vector<std::pair<int, DevEnt>>> b2((size_t)tx2 * ty);
                    for (const Entry &e : sm.meas) {
                        if (!hs.cplx && inA(e.arr) != inA(sarr)) continue;   // real fields: the source's set only
                        const int i = (int)(e.idx % hs.nx), j = (int)(e.idx / hs.nx);
                        const int ti = i / MARCH_W2, tj = j / rows;
                        const int loc = (j - tj * rows) * MARCH_W2 + (i - ti * MARCH_W2);
                        auto &b = b2[(size_t)tj * tx2 + ti];
                        if (e.re != 0.0 || !hs.cplx) b.push_back({loc, DevEnt{loc | (e.arr << 16), 0, e.re}});
                        if (hs.cplx && e.im != 0.0) b.push_back({loc, DevEnt{loc | ((e.arr | 8) << 16), 0, e.im}});
                    }
                    hs.tile2_0 = (int)P->tiles2.size();
                    for (int tj = 0; tj < ty; ++tj)
                        for (int ti = 0; ti < tx2; ++ti) {
                            auto &b = b2[(size_t)tj * tx2 + ti];
                            std::stable_sort(b.begin(), b.end(), [](const std::pair<int, DevEnt> &x, const std::pair<int, DevEnt> &y) {
                                return x.first < y.first;
                            });
                            HostTile2 ht{(int)s, ti * MARCH_W2, tj * rows, (int)P->ents2.size(), (int)b.size(), (int)P->rowptr2.size()};
                            if (!hs.cyl) ht.variant = v2->second[(size_t)tj * tx2 + ti];
                            int k = 0;
                            for (int ly = 0; ly <= rows; ++ly) {
                                while (k < (int)b.size() && b[k].first / MARCH_W2 < ly) ++k;
                                P->rowptr2.push_back(ly == rows ? (int)b.size() : k);
                            }
                            for (auto &pe : b) P->ents2.push_back(pe.second);
                            P->tiles2.push_back(ht);
                        }
                    hs.ntile2 = (int)P->tiles2.size() - hs.tile2_0;
                }
            }
            if (hs.col3) {
                // one warp per tile of COL3_W x COL3_H cells in (x, y) over a chunk of at most COL3_ZMAX
                // planes; kernel variant of each tile from the CPML slabs and Lorentz poles of its
                // halo-extended box [i0-1, i0+COL3_W] x [j0-1, j0+COL3_H] x [z0-1, z1] (cached per geometry)
                const int tx = (hs.nx + COL3_W - 1) / COL3_W, ty = (hs.ny + COL3_H - 1) / COL3_H;
                const int ncz = (hs.nz + COL3_ZMAX - 1) / COL3_ZMAX, zc = (hs.nz + ncz - 1) / ncz;
                const int tz = (hs.nz + zc - 1) / zc;
                auto vit = march_variants.find(sm.geo);
                if (vit == march_variants.end()) {
                    std::vector<int> dmat(g.nmat, 0);
                    for (int id = 0; id < g.nmat; ++id)
                        for (int q = 0; q < g.npoles; ++q)
                            for (int c = 0; c < 3; ++c)
                                if (g.lorentz[((size_t)id * g.npoles + q) * 6 + 2 * c] != 0.0) dmat[id] = std::max(dmat[id], q + 1);
                    const int dX = g.has_pml[0] ? D.prob.pml_cells[0] : 0, dY = g.has_pml[1] ? D.prob.pml_cells[1] : 0;
                    const int dZ = g.has_pml[2] ? D.prob.pml_cells[2] : 0;
                    auto wrapc = [](int i, int n) { return ((i % n) + n) % n; };
                    std::vector<int> vs((size_t)tx * ty * tz, 0);
                    std::vector<int> colp((size_t)hs.nx * hs.ny);
                    for (int tk = 0; tk < tz; ++tk) {
                        const int z0 = tk * zc, z1 = std::min(hs.nz, z0 + zc);
                        // the most poles of each (x, y) column over the chunk's planes and its halo planes
                        std::fill(colp.begin(), colp.end(), 0);
                        bool zp = false;
                        for (int kk = z0 - 1; kk <= z1; ++kk) {
                            const int k = wrapc(kk, hs.nz);
                            if (dZ > 0 && (k < dZ || k >= hs.nz - dZ)) zp = true;
                            if (g.npoles == 0) continue;
                            for (int j = 0; j < hs.ny; ++j)
                                for (int i = 0; i < hs.nx; ++i) {
                                    int &cp = colp[(size_t)j * hs.nx + i];
                                    cp = std::max(cp, dmat[g.mat[((size_t)k * hs.ny + j) * hs.nx + i]]);
                                }
                        }
                        for (int tj = 0; tj < ty; ++tj)
                            for (int ti = 0; ti < tx; ++ti) {
                                const int i0 = ti * COL3_W, j0 = tj * COL3_H;
                                bool pml = zp;
                                int poles = 0;
                                for (int jj = j0 - 1; jj <= j0 + COL3_H; ++jj) {
                                    const int j = wrapc(jj, hs.ny);
                                    if (dY > 0 && (j < dY || j >= hs.ny - dY)) pml = true;
                                    for (int ii = i0 - 1; ii <= i0 + COL3_W; ++ii) {
                                        const int i = wrapc(ii, hs.nx);
                                        if (dX > 0 && (i < dX || i >= hs.nx - dX)) pml = true;
                                        poles = std::max(poles, colp[(size_t)j * hs.nx + i]);
                                    }
                                }
                                vs[((size_t)tk * ty + tj) * tx + ti] = (pml ? 1 : 0) + (poles == 0 ? 0 : poles == 1 ? 2 : 4);
                            }
                    }
                    vit = march_variants.emplace(sm.geo, std::move(vs)).first;
                }
                std::vector<std::vector<DevEnt>> bucket((size_t)tx * ty * tz);
                const int64_t sxy = (int64_t)hs.nx * hs.ny;
                for (const Entry &e : sm.meas) {
                    const int z = (int)(e.idx / sxy);
                    const int64_t r = e.idx - (int64_t)z * sxy;
                    const int j = (int)(r / hs.nx), i = (int)(r - (int64_t)j * hs.nx);
                    const int ti = i / COL3_W, tj = j / COL3_H, tk = z / zc;
                    const int loc = (j - tj * COL3_H) * 32 + (i - ti * COL3_W);
                    auto &b = bucket[((size_t)tk * ty + tj) * tx + ti];
                    if (e.re != 0.0 || !hs.cplx) b.push_back(DevEnt{loc | (e.arr << 16), z, e.re});
                    if (hs.cplx && e.im != 0.0) b.push_back(DevEnt{loc | ((e.arr | 8) << 16), z, e.im});
                }
                hs.tile0 = (int)P->tilesM.size();
                hs.ntile = tx * ty * tz;
                hs.ent0 = (int)P->entsM.size();
                for (int tk = 0; tk < tz; ++tk)
                    for (int tj = 0; tj < ty; ++tj)
                        for (int ti = 0; ti < tx; ++ti) {
                            const size_t tt = ((size_t)tk * ty + tj) * tx + ti;
                            auto &b = bucket[tt];
                            HostTile ht{(int)s, ti * COL3_W, tj * COL3_H, (int)P->entsM.size(), (int)b.size(),
                                        vit->second[tt] + (hs.magnetic ? MARCH_VARIANTS : 0)};
                            ht.z0 = tk * zc;
                            ht.z1 = std::min(hs.nz, ht.z0 + zc);
                            P->tilesM.push_back(ht);
                            P->entsM.insert(P->entsM.end(), b.begin(), b.end());
                        }
                hs.nent = (int)P->entsM.size() - hs.ent0;
            }
            hs.line3 = (!hs.march && !hs.col3 && D.prob.dims == 3 && P->opts.kernel_3d == 1 && planes * N < ((int64_t)1 << 32)) ? 1 : 0;
            if (hs.line3) {
                // tiles of 32 x cells by LINES3 (y, z) lines; entries bucketed per tile
                const int64_t nl = (int64_t)hs.ny * hs.nz;
                const int tx = (hs.nx + 31) / 32, tl = (int)((nl + LINES3 - 1) / LINES3);
                std::vector<std::vector<DevEnt>> bucket((size_t)tx * tl);
                for (const Entry &e : sm.meas) {
                    const int64_t line = e.idx / hs.nx;
                    const int i = (int)(e.idx - line * hs.nx);
                    const int ti = i / 32, tj = (int)(line / LINES3);
                    const int loc = (int)(line - (int64_t)tj * LINES3) * 32 + (i - ti * 32);
                    auto &b = bucket[(size_t)tj * tx + ti];
                    if (e.re != 0.0 || !hs.cplx) b.push_back(DevEnt{loc | (e.arr << 16), 0, e.re});
                    if (hs.cplx && e.im != 0.0) b.push_back(DevEnt{loc | ((e.arr | 8) << 16), 0, e.im});
                }
                hs.tile0 = (int)P->tilesM.size();
                hs.ntile = tx * tl;
                hs.ent0 = (int)P->entsM.size();
                for (int tj = 0; tj < tl; ++tj)
                    for (int ti = 0; ti < tx; ++ti) {
                        auto &b = bucket[(size_t)tj * tx + ti];
                        P->tilesM.push_back(HostTile{(int)s, ti * 32, tj * LINES3, (int)P->entsM.size(), (int)b.size(), 0});
                        P->entsM.insert(P->entsM.end(), b.begin(), b.end());
                    }
                hs.nent = (int)P->entsM.size() - hs.ent0;
            }
            if (!hs.march && !hs.line3 && !hs.col3) {
                int ntile = (int)((N + TILE6 - 1) / TILE6);
                hs.tile0 = (int)P->tiles6.size();
                hs.ntile = ntile;
                std::vector<std::vector<DevEnt6>> bucket(ntile);
                for (const Entry &e : sm.meas) {
                    if (!hs.cplx && g.n[2] == 1 && D.prob.dims == 2 && inA(e.arr) != inA(sarr)) continue;   // contributes i * real: no real part
                    int tl = (int)(e.idx / TILE6);
                    bucket[tl].push_back(DevEnt6{(int)(e.idx - (int64_t)tl * TILE6), e.arr, e.re, e.im});
                }
                hs.ent0 = (int)P->ents6.size();
                for (int tl = 0; tl < ntile; ++tl) {
                    auto &b = bucket[tl];
                    HostTile6 ht{(int)s, (int)std::min<int64_t>(TILE6, N - (int64_t)tl * TILE6), (int64_t)tl * TILE6,
                                 (int)P->ents6.size(), (int)b.size()};
                    P->ents6.insert(P->ents6.end(), b.begin(), b.end());
                    P->tiles6.push_back(ht);
                }
                hs.nent = (int)P->ents6.size() - hs.ent0;
            }
            hs.src0 = (int)P->src6.size();
            for (const Entry &e : sm.src) {
                if (hs.cplx)
                    P->src6.push_back(DevSrc6{hs.field_off + (2 * e.arr) * N + e.idx, hs.field_off + (2 * e.arr + 1) * N + e.idx, e.re, e.im});
                else
                    P->src6.push_back(DevSrc6{hs.field_off + e.arr * N + e.idx, -1, e.re, 0.0});
            }
            hs.nsrc = (int)P->src6.size() - hs.src0;
        }
        P->sims.push_back(hs);
    }
    P->field_elems = off;
    {
        bool all2d = !P->sims.empty() && !P->sims[0].full;
        // six-component runs fuse two steps when every simulation has its two-step tiles
        bool two6 = !P->sims.empty() && !all2d;
        for (const HostSim &h : P->sims) two6 = two6 && h.march && h.ntile2 > 0;
        P->k2d = all2d ? P->opts.steps_per_launch : (two6 ? 2 : 1);
        P->launches = (D.prob.n_steps + P->k2d - 1) / P->k2d;
    }
    P->table_bytes = (int64_t)(align256(P->ents2.size() * sizeof(DevEnt)) + align256(P->rowptr2.size() * sizeof(int)) +
                               align256(P->mat_all.size()) + align256(P->coef_all.size() * P->rsize) +
                               align256(D.gw.size() * 8) + align256(P->ents.size() * sizeof(DevEnt)) +
                               align256(P->src.size() * sizeof(DevSrc)) + align256(P->ents6.size() * sizeof(DevEnt6)) +
                               align256(P->src6.size() * sizeof(DevSrc6)) + align256(P->lor_all.size() * 8) +
                               align256(P->pml_all.size() * P->rsize) + align256(P->entsM.size() * sizeof(DevEnt)) +
                               align256(P->lorc_all.size() * P->rsize));
    P->request_bytes = (int64_t)(align256(P->field_elems * P->rsize) + 2 * align256(P->sims.size() * 8) +
                                 P->tiles.size() * sizeof(DevTile) + P->tiles6.size() * sizeof(DevTile6) +
                                 P->tiles2.size() * sizeof(DevTile2) + P->tilesM.size() * sizeof(DevTile) +
                                 P->sims.size() * std::max(sizeof(DevSim2D), sizeof(DevSim6)));
    return CASIMIR_OK;
}

template <typename T>
static int put_table(const std::vector<T> &v, void *dst, cudaStream_t st)
{
    if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return CASIMIR_OK;
}

static int put_real(const std::vector<double> &v, void *dst, int fp64, cudaStream_t st)
{
    if (v.empty()) return CASIMIR_OK;
    if (fp64) return put_table(v, dst, st);
    std::vector<float> f(v.begin(), v.end());
    CUDA_TRY(cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return CASIMIR_OK;
}

int upload_plan(casimir_plan_t *P, cudaStream_t st)
{
    NvtxRange nvtx_("casimir.upload");
    if (P->dev.block) return CASIMIR_OK;
    casimir_ctx *c = P->ctx;
    size_t sz[13] = {align256(P->mat_all.size()), align256(P->coef_all.size() * P->rsize),
                     align256(P->data.gw.size() * 8), align256(P->ents.size() * sizeof(DevEnt)),
                     align256(P->src.size() * sizeof(DevSrc)), align256(P->ents6.size() * sizeof(DevEnt6)),
                     align256(P->src6.size() * sizeof(DevSrc6)), align256(P->lor_all.size() * 8),
                     align256(P->pml_all.size() * P->rsize), align256(P->ents2.size() * sizeof(DevEnt)),
                     align256(P->rowptr2.size() * sizeof(int)), align256(P->entsM.size() * sizeof(DevEnt)),
                     align256(P->lorc_all.size() * P->rsize)};
    size_t total = 0;
    for (size_t q : sz) total += q;
    void *blk;
    int rc = dev_alloc(c, std::max<size_t>(total, 256), &blk);
    if (rc) return rc;
    char *p = (char *)blk;
    P->dev.block = blk;
    P->dev.bytes = total;
    P->dev.mat = (uint8_t *)p; p += sz[0];
    P->dev.coef = p; p += sz[1];
    P->dev.gw = (double *)p; p += sz[2];
    P->dev.ents = (DevEnt *)p; p += sz[3];
    P->dev.src = (DevSrc *)p; p += sz[4];
    P->dev.ents6 = (DevEnt6 *)p; p += sz[5];
    P->dev.src6 = (DevSrc6 *)p; p += sz[6];
    P->dev.lor = (double *)p; p += sz[7];
    P->dev.pml = p; p += sz[8];
    P->dev.ents2 = (DevEnt *)p; p += sz[9];
    P->dev.rowptr2 = (int *)p; p += sz[10];
    P->dev.entsM = (DevEnt *)p; p += sz[11];
    P->dev.lorc = p;
    if ((rc = put_table(P->mat_all, P->dev.mat, st))) return rc;
    if ((rc = put_real(P->coef_all, P->dev.coef, P->fp64, st))) return rc;
    if ((rc = put_table(P->data.gw, P->dev.gw, st))) return rc;
    if ((rc = put_table(P->ents, P->dev.ents, st))) return rc;
    if ((rc = put_table(P->src, P->dev.src, st))) return rc;
    if ((rc = put_table(P->ents6, P->dev.ents6, st))) return rc;
    if ((rc = put_table(P->src6, P->dev.src6, st))) return rc;
    if ((rc = put_table(P->lor_all, P->dev.lor, st))) return rc;
    if ((rc = put_real(P->pml_all, P->dev.pml, P->fp64, st))) return rc;
    if ((rc = put_table(P->ents2, P->dev.ents2, st))) return rc;
    if ((rc = put_table(P->rowptr2, P->dev.rowptr2, st))) return rc;
    if ((rc = put_table(P->entsM, P->dev.entsM, st))) return rc;
    if ((rc = put_real(P->lorc_all, P->dev.lorc, P->fp64, st))) return rc;
    c->used += total;
    return CASIMIR_OK;
}

// ---------------------------------------------------------------------------------
// engine
// ---------------------------------------------------------------------------------

static void drop_graphs(casimir_ctx *c)
{
    for (auto &kv : c->graphs) cudaGraphExecDestroy(kv.second);
    c->graphs.clear();
}

static int admit(casimir_ctx *c, casimir_request *r)
{
    casimir_plan_t *P = r->plan;
    int rc = upload_plan(P, c->stream);
    if (rc) return rc;
    size_t bf = align256(P->field_elems * P->rsize), ba = align256(P->sims.size() * 8);
    void *blk;
    rc = dev_alloc(c, bf + 2 * ba, &blk);
    if (rc) return rc;
    r->block = blk;
    r->acc = (double *)((char *)blk + bf);
    r->tail = (double *)((char *)blk + bf + ba);
    c->used += bf + 2 * ba;
    CUDA_TRY(cudaMemsetAsync(blk, 0, bf + 2 * ba, c->stream));
    // sources: offsets are relative to the request's field block
    launch_inject(P->fp64, blk, P->dev.src, (int)P->src.size(), c->stream);
    launch_inject6(P->fp64, blk, P->dev.src6, (int)P->src6.size(), c->stream);
    CUDA_TRY(cudaGetLastError());
    if (!r->h_acc) CUDA_TRY(cudaMallocHost((void **)&r->h_acc, std::max<size_t>(1, 2 * P->sims.size()) * 8));
    // waves of consecutive simulations whose field blocks fit the wave budget
    r->waves.clear();
    r->waves_done = 0;
    const size_t ns = P->sims.size();
    const int64_t wave_bytes = c->wave_bytes.load();
    for (size_t q = 0; q < ns;) {
        casimir_request::Wave w{q, q, 0, 0, 0, 0};
        while (w.s_end < ns) {
            size_t e = w.s_end;
            int64_t next = e + 1 < ns ? P->sims[e + 1].field_off : P->field_elems;
            int64_t b = (next - P->sims[e].field_off) * (int64_t)P->rsize;
            if (w.s_end > w.s_begin && wave_bytes > 0 && w.bytes + b > wave_bytes) break;
            w.bytes += b;
            w.cells += (int64_t)P->sims[e].nx * P->sims[e].ny * P->sims[e].nz;
            ++w.s_end;
        }
        q = w.s_end;
        r->waves.push_back(w);
    }
    for (size_t wi = 0; wi < r->waves.size(); ++wi) c->pending_waves.push_back({r, wi});
    r->state = 1;
    r->t_admit = now_ms();
    c->active.push_back(r);
    c->dirty = true;
    return CASIMIR_OK;
}

// Start pending waves (FIFO over requests) while the active waves' field bytes stay
// within the wave budget; a wave always starts when nothing else is active.
static void activate_waves(casimir_ctx *c)
{
    const int64_t wave_bytes = c->wave_bytes.load();
    while (!c->pending_waves.empty()) {
        auto pw = c->pending_waves.front();
        casimir_request::Wave &w = pw.first->waves[pw.second];
        if (!c->active_waves.empty() && wave_bytes > 0 && c->active_bytes + w.bytes > wave_bytes) break;
        c->pending_waves.pop_front();
        w.s0 = c->h_launch - 1;
        w.state = 1;
        c->active_bytes += w.bytes;
        c->active_waves.push_back(pw);
        c->dirty = true;
    }
}

// Drop every wave of request r (timeout, cancel).
static void drop_waves(casimir_ctx *c, casimir_request *r)
{
    for (size_t q = 0; q < c->active_waves.size();) {
        if (c->active_waves[q].first == r) {
            c->active_bytes -= r->waves[c->active_waves[q].second].bytes;
            c->active_waves.erase(c->active_waves.begin() + q);
        } else {
            ++q;
        }
    }
    for (size_t q = 0; q < c->pending_waves.size();) {
        if (c->pending_waves[q].first == r) c->pending_waves.erase(c->pending_waves.begin() + q);
        else ++q;
    }
    c->dirty = true;
}

// Device descriptor of simulation s of plan P whose request block is `blk`.
void make_sim2d(const casimir_plan_t *P, char *blk, double *acc, double *tail, int64_t s0, size_t s, DevSim2D *d)
{
    const PlanData &D = P->data;
    const HostSim &hs = P->sims[s];
    double sg = D.prob.sigma, dt = D.dt, dx = D.dx;
    *d = DevSim2D{};
    d->fields = blk + hs.field_off * P->rsize;
    d->mat = P->dev.mat + P->mat_off[hs.geo];
    d->coef = (char *)P->dev.coef + P->coef_off[hs.geo] * P->rsize;
    d->gw = P->dev.gw;
    d->acc = acc + s;
    d->tail = tail + s;
    d->s0 = s0;
    d->nx = hs.nx;
    d->ny = hs.ny;
    d->T = D.prob.n_steps;
    d->tail_from = D.prob.n_steps - std::max(1, D.prob.n_steps / 8);
    d->second_u = hs.second_u;
    d->nmat = D.geos[hs.geo].nmat;
    d->a = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt);
    d->bf = dt / (1.0 + 0.5 * sg * dt) / dx;
    d->hf = dt / dx;
}

void make_sim6(const casimir_plan_t *P, char *blk, double *acc, double *tail, int64_t s0, size_t s, DevSim6 *d)
{
    const PlanData &D = P->data;
    const HostSim &hs = P->sims[s];
    const Geo &g = D.geos[hs.geo];
    double sg = D.prob.sigma, dt = D.dt, dx = D.dx;
    *d = DevSim6{};
    d->fields = blk + hs.field_off * P->rsize;
    d->psi = hs.psi_off >= 0 ? blk + hs.psi_off * P->rsize : nullptr;
    d->lor = hs.lor_off >= 0 ? blk + hs.lor_off * P->rsize : nullptr;
    d->mat = P->dev.mat + P->mat_off[hs.geo];
    d->coef = (char *)P->dev.coef + P->coef_off[hs.geo] * P->rsize;
    d->lorentz = P->dev.lor + P->lor_off[hs.geo];
    d->lorc = (char *)P->dev.lorc + P->lorc_off[hs.geo] * P->rsize;
    d->pml = P->dev.pml;
    d->gw = P->dev.gw;
    d->acc = acc + s;
    d->tail = tail + s;
    d->s0 = s0;
    int64_t N = (int64_t)hs.nx * hs.ny * hs.nz;
    int64_t po = 0;
    int cf = hs.cplx ? 2 : 1;
    for (int a = 0; a < 3; ++a) {
        d->n[a] = g.n[a];
        d->pml_d[a] = g.has_pml[a] ? D.prob.pml_cells[a] : 0;
        d->pml_off[a] = g.has_pml[a] ? P->pml_off[hs.geo][a] : 0;
        d->slab[a] = g.has_pml[a] ? (N / g.n[a]) * 2 * D.prob.pml_cells[a] : 0;
        d->psi_off[a] = po;
        po += g.has_pml[a] ? 4 * cf * d->slab[a] : 0;
        d->bre[a] = g.bloch_re[a];
        d->bim[a] = g.bloch_im[a];
    }
    d->dims = D.prob.dims;
    d->magnetic = hs.magnetic;
    d->T = D.prob.n_steps;
    d->tail_from = D.prob.n_steps - std::max(1, D.prob.n_steps / 8);
    d->a = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt);
    d->bs = dt / (1.0 + 0.5 * sg * dt);
    d->dt = dt;
    d->dt_full = dt;
    d->sigma = sg;
    d->inv_dx = 1.0 / dx;
    d->kz = g.kz;
    d->kzA = hs.kzA;
    d->kzB = hs.kzB;
    const bool pp = hs.march || hs.col3;   // ping-pong buffers
    d->fhalf = pp ? hs.fhalf : 0;
    d->tile_rows = P->opts.march_rows;
    d->npoles = hs.npoles;
    d->psi_half = pp ? hs.psi_half : 0;
    d->lor_half = pp ? hs.lor_half : 0;
}

static int grow(casimir_ctx *c, void **p, size_t *cap, size_t need)
{
    if (need <= *cap) return CASIMIR_OK;
    dev_free(c, *p);
    *p = nullptr;
    size_t n = std::max(need, 2 * *cap);
    int rc = dev_alloc(c, n, p);
    if (rc) { *cap = 0; return rc; }
    *cap = n;
    return CASIMIR_OK;
}

static int rebuild(casimir_ctx *c)
{
    NvtxRange nvtx_("casimir.rebuild");
    std::vector<DevSim2D> s2[2];
    std::vector<DevTile> t2[2];
    std::vector<DevTile2> tt[4];   // [fp64]: two steps per launch, [2 + fp64]: three
    std::vector<DevSim6> s6[8];
    std::vector<DevTile6> t6[8];
    std::vector<DevSim6> sm6[4 * MARCH_VARIANTS];
    std::vector<DevTile> tm6[4 * MARCH_VARIANTS];
    std::vector<DevSim6> sl3[4];
    std::vector<DevTile> tl3[4];
    std::vector<DevSim6> scol[4 * COL3_VARIANTS];
    std::vector<DevTile> tcol[4 * COL3_VARIANTS];
    std::vector<DevSim6> sc6[2];
    std::vector<DevTile> tc6[2];
    std::vector<DevSim6> sc2[2];    // cylindrical, two steps per launch
    std::vector<DevTile2> tc2[2];
    std::vector<DevSim6> sm2[2 * MAR2_VARIANTS];    // Cartesian march, two steps per launch
    std::vector<DevTile2> tm2[2 * MAR2_VARIANTS];
    for (auto &aw : c->active_waves) {
        casimir_request *r = aw.first;
        const casimir_request::Wave &w = r->waves[aw.second];
        casimir_plan_t *P = r->plan;
        for (size_t s = w.s_begin; s < w.s_end; ++s) {
            const HostSim &hs = P->sims[s];
            char *blk = (char *)r->block;
            if (!hs.full) {
                auto &sv = s2[P->fp64];
                auto &tv = t2[P->fp64];
                int idx = (int)sv.size();
                DevSim2D d;
                make_sim2d(P, blk, r->acc, r->tail, w.s0, s, &d);
                sv.push_back(d);
                if (P->k2d >= 2) {
                    auto &tk = tt[(P->k2d == 3 ? 2 : 0) + P->fp64];
                    for (int t = hs.tile2_0; t < hs.tile2_0 + hs.ntile2; ++t) {
                        const HostTile2 &ht = P->tiles2[t];
                        tk.push_back(DevTile2{idx, ht.i0, ht.j0, ht.ne, P->dev.ents2 + ht.ent0, P->dev.rowptr2 + ht.rp0});
                    }
                } else {
                    for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                        const HostTile &ht = P->tiles[t];
                        tv.push_back(DevTile{idx, ht.i0, ht.j0, ht.ne, P->dev.ents + ht.ent0});
                    }
                }
            } else if (hs.col3) {
                // the simulation's descriptor goes to each variant group that holds one of its tiles
                DevSim6 d;
                make_sim6(P, blk, r->acc, r->tail, w.s0, s, &d);
                int idx[COL3_VARIANTS];
                std::fill(idx, idx + COL3_VARIANTS, -1);
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile &ht = P->tilesM[t];
                    const int gi = COL3_VARIANTS * (2 * P->fp64 + hs.cplx) + ht.variant;
                    if (idx[ht.variant] < 0) {
                        idx[ht.variant] = (int)scol[gi].size();
                        scol[gi].push_back(d);
                    }
                    tcol[gi].push_back(DevTile{idx[ht.variant], ht.i0, ht.j0, ht.ne, P->dev.entsM + ht.ent0, ht.z0, ht.z1});
                }
            } else if (hs.line3) {
                const int gi = 2 * P->fp64 + hs.cplx;
                DevSim6 d;
                make_sim6(P, blk, r->acc, r->tail, w.s0, s, &d);
                const int idx = (int)sl3[gi].size();
                sl3[gi].push_back(d);
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile &ht = P->tilesM[t];
                    tl3[gi].push_back(DevTile{idx, ht.i0, ht.j0, ht.ne, P->dev.entsM + ht.ent0});
                }
            } else if (hs.cyl) {
                const int gi = P->fp64;
                DevSim6 d;
                make_sim6(P, blk, r->acc, r->tail, w.s0, s, &d);
                if (P->k2d == 2) {
                    const int idx = (int)sc2[gi].size();
                    sc2[gi].push_back(d);
                    for (int t = hs.tile2_0; t < hs.tile2_0 + hs.ntile2; ++t) {
                        const HostTile2 &ht = P->tiles2[t];
                        tc2[gi].push_back(DevTile2{idx, ht.i0, ht.j0, ht.ne, P->dev.ents2 + ht.ent0, P->dev.rowptr2 + ht.rp0});
                    }
                } else {
                    const int idx = (int)sc6[gi].size();
                    sc6[gi].push_back(d);
                    for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                        const HostTile &ht = P->tilesM[t];
                        tc6[gi].push_back(DevTile{idx, ht.i0, ht.j0, ht.ne, P->dev.entsM + ht.ent0});
                    }
                }
            } else if (hs.march && P->k2d == 2) {
                // two steps per launch: the descriptor goes to each variant group holding one of its tiles
                DevSim6 d;
                make_sim6(P, blk, r->acc, r->tail, w.s0, s, &d);
                int idx[MAR2_VARIANTS];
                std::fill(idx, idx + MAR2_VARIANTS, -1);
                for (int t = hs.tile2_0; t < hs.tile2_0 + hs.ntile2; ++t) {
                    const HostTile2 &ht = P->tiles2[t];
                    const int gi = MAR2_VARIANTS * hs.cplx + ht.variant;
                    if (idx[ht.variant] < 0) {
                        idx[ht.variant] = (int)sm2[gi].size();
                        sm2[gi].push_back(d);
                    }
                    tm2[gi].push_back(DevTile2{idx[ht.variant], ht.i0, ht.j0, ht.ne, P->dev.ents2 + ht.ent0, P->dev.rowptr2 + ht.rp0});
                }
            } else if (hs.march) {
                // the simulation's descriptor goes to each variant group that holds one of its tiles
                DevSim6 d;
                make_sim6(P, blk, r->acc, r->tail, w.s0, s, &d);
                int idx[MARCH_VARIANTS];
                std::fill(idx, idx + MARCH_VARIANTS, -1);
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile &ht = P->tilesM[t];
                    const int gi = MARCH_VARIANTS * (2 * P->fp64 + hs.cplx) + ht.variant;
                    if (idx[ht.variant] < 0) {
                        idx[ht.variant] = (int)sm6[gi].size();
                        sm6[gi].push_back(d);
                    }
                    tm6[gi].push_back(DevTile{idx[ht.variant], ht.i0, ht.j0, ht.ne, P->dev.entsM + ht.ent0});
                }
            } else {
                int gi = 4 * P->fp64 + 2 * hs.cplx + (P->data.prob.dims == 3 ? 1 : 0);
                auto &sv = s6[gi];
                auto &tv = t6[gi];
                int idx = (int)sv.size();
                DevSim6 d;
                make_sim6(P, blk, r->acc, r->tail, w.s0, s, &d);
                sv.push_back(d);
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile6 &ht = P->tiles6[t];
                    tv.push_back(DevTile6{idx, ht.count, ht.cell0, ht.ne, 0, P->dev.ents6 + ht.ent0});
                }
            }
        }
    }
    c->ntiles = 0;
    for (int gi = 0; gi < casimir_ctx::NGROUPS; ++gi) {
        auto &G = c->groups[gi];
        size_t ns, nt, ss, ts;
        const void *sp, *tp;
        if (gi < 2) { ns = s2[gi].size(); nt = t2[gi].size(); ss = sizeof(DevSim2D); ts = sizeof(DevTile); sp = s2[gi].data(); tp = t2[gi].data(); }
        else if (gi < 10) { ns = s6[gi - 2].size(); nt = t6[gi - 2].size(); ss = sizeof(DevSim6); ts = sizeof(DevTile6); sp = s6[gi - 2].data(); tp = t6[gi - 2].data(); }
        else if (gi < 12) { ns = 0; nt = tt[gi - 10].size(); ss = sizeof(DevSim2D); ts = sizeof(DevTile2); sp = nullptr; tp = tt[gi - 10].data(); }
        else if (gi < casimir_ctx::G_LINE3) {
            const int v = gi - casimir_ctx::G_MARCH;
            ns = sm6[v].size(); nt = tm6[v].size(); ss = sizeof(DevSim6); ts = sizeof(DevTile); sp = sm6[v].data(); tp = tm6[v].data();
        } else if (gi < casimir_ctx::G_CYL) {
            const int v = gi - casimir_ctx::G_LINE3;
            ns = sl3[v].size(); nt = tl3[v].size(); ss = sizeof(DevSim6); ts = sizeof(DevTile); sp = sl3[v].data(); tp = tl3[v].data();
        } else if (gi < casimir_ctx::G_T3) {
            const int v = gi - casimir_ctx::G_CYL;
            ns = sc6[v].size(); nt = tc6[v].size(); ss = sizeof(DevSim6); ts = sizeof(DevTile); sp = sc6[v].data(); tp = tc6[v].data();
        } else if (gi < casimir_ctx::G_CYL2) {
            const int v = 2 + gi - casimir_ctx::G_T3;
            ns = 0; nt = tt[v].size(); ss = sizeof(DevSim2D); ts = sizeof(DevTile2); sp = nullptr; tp = tt[v].data();
        } else if (gi < casimir_ctx::G_COL3) {
            const int v = gi - casimir_ctx::G_CYL2;
            ns = sc2[v].size(); nt = tc2[v].size(); ss = sizeof(DevSim6); ts = sizeof(DevTile2); sp = sc2[v].data(); tp = tc2[v].data();
        } else if (gi < casimir_ctx::G_MAR2) {
            const int v = gi - casimir_ctx::G_COL3;
            ns = scol[v].size(); nt = tcol[v].size(); ss = sizeof(DevSim6); ts = sizeof(DevTile); sp = scol[v].data(); tp = tcol[v].data();
        } else {
            const int v = gi - casimir_ctx::G_MAR2;
            ns = sm2[v].size(); nt = tm2[v].size(); ss = sizeof(DevSim6); ts = sizeof(DevTile2); sp = sm2[v].data(); tp = tm2[v].data();
        }
        int rc = grow(c, &G.sims, &G.sims_cap, ns * ss);
        if (rc) return rc;
        rc = grow(c, &G.tiles, &G.tiles_cap, nt * ts);
        if (rc) return rc;
        if (ns) CUDA_TRY(cudaMemcpyAsync(G.sims, sp, ns * ss, cudaMemcpyHostToDevice, c->stream));
        if (nt) CUDA_TRY(cudaMemcpyAsync(G.tiles, tp, nt * ts, cudaMemcpyHostToDevice, c->stream));
        G.ntiles = (int)nt;
        c->ntiles += (int)nt;
    }
    // the two-step tiles index the 2D simulation tables of groups 0 / 1
    c->groups[10].ntiles = (int)tt[0].size();
    c->groups[11].ntiles = (int)tt[1].size();
    c->groups[casimir_ctx::G_T3].ntiles = (int)tt[2].size();
    c->groups[casimir_ctx::G_T3 + 1].ntiles = (int)tt[3].size();
    CUDA_TRY(cudaStreamSynchronize(c->stream));   // host vectors die here
    drop_graphs(c);
    c->dirty = false;
    return CASIMIR_OK;
}

// One launch unit of step j (a six-component group's two phases form one unit).
static void launch_unit(casimir_ctx *c, int gi, int j, cudaStream_t st)
{
    const auto &G = c->groups[gi];
    if (gi < 2)
        launch_step2d(gi, (const DevSim2D *)G.sims, (const DevTile *)G.tiles, G.ntiles, c->d_launch, j, st);
    else if (gi < 10)
        for (int phase = 0; phase < 2; ++phase)
            launch_full(((gi - 2) >> 2) & 1, ((gi - 2) >> 1) & 1, ((gi - 2) & 1) ? 3 : 2, (const DevSim6 *)G.sims,
                        (const DevTile6 *)G.tiles, G.ntiles, c->d_launch, j, phase, st);
    else if (gi < 12)
        launch_step2d_t2(gi - 10, (const DevSim2D *)c->groups[gi - 10].sims, (const DevTile2 *)G.tiles, G.ntiles,
                         c->d_launch, j, st);
    else if (gi < casimir_ctx::G_LINE3) {
        const int v = gi - casimir_ctx::G_MARCH, fc = v / MARCH_VARIANTS;   // 2 * fp64 + cplx
        launch_march6(fc >> 1, fc & 1, v % MARCH_VARIANTS, (const DevSim6 *)G.sims, (const DevTile *)G.tiles, G.ntiles,
                      c->d_launch, j, st);
    } else if (gi < casimir_ctx::G_CYL) {
        const int v = gi - casimir_ctx::G_LINE3;
        for (int phase = 0; phase < 2; ++phase)
            launch_line3((v >> 1) & 1, v & 1, (const DevSim6 *)G.sims, (const DevTile *)G.tiles, G.ntiles,
                         c->d_launch, j, phase, st);
    } else if (gi < casimir_ctx::G_T3) {
        launch_march6_cyl(gi - casimir_ctx::G_CYL, (const DevSim6 *)G.sims, (const DevTile *)G.tiles, G.ntiles, c->d_launch, j, st);
    } else if (gi < casimir_ctx::G_CYL2) {
        // the 2D simulation tables are those of groups 0 / 1
        const int f = gi - casimir_ctx::G_T3;
        launch_step2d_t3(f, (const DevSim2D *)c->groups[f].sims, (const DevTile2 *)G.tiles, G.ntiles, c->d_launch, j, st);
    } else if (gi < casimir_ctx::G_COL3) {
        launch_march6_cyl2(gi - casimir_ctx::G_CYL2, (const DevSim6 *)G.sims, (const DevTile2 *)G.tiles, G.ntiles, c->d_launch, j, st);
    } else if (gi < casimir_ctx::G_MAR2) {
        const int v = gi - casimir_ctx::G_COL3, fc = v / COL3_VARIANTS;   // 2 * fp64 + cplx
        launch_col3(fc >> 1, fc & 1, v % COL3_VARIANTS, (const DevSim6 *)G.sims, (const DevTile *)G.tiles, G.ntiles,
                    c->d_launch, j, st);
    } else {
        const int v = gi - casimir_ctx::G_MAR2;
        launch_march6_2(v / MAR2_VARIANTS, v % MAR2_VARIANTS, (const DevSim6 *)G.sims, (const DevTile2 *)G.tiles, G.ntiles,
                        c->d_launch, j, st);
    }
}

// Launch k consecutive steps.  The units of one step touch disjoint tiles and read only the
// previous step's buffers, so with more than one unit they run side by side on auxiliary
// streams (forked from and joined back into the context's stream every step), which lets one
// unit's last partial wave overlap the next unit.
static void launch_steps(casimir_ctx *c, int k)
{
    static const bool no_fork = std::getenv("CASIMIR_NO_FORK") != nullptr;
    int units[casimir_ctx::NGROUPS], nu = 0;
    for (int gi = 0; gi < casimir_ctx::NGROUPS; ++gi)
        if (c->groups[gi].ntiles > 0) units[nu++] = gi;
    const bool fork = nu > 1 && !no_fork;
    for (int j = 0; j < k; ++j) {
        if (!fork) {
            for (int u = 0; u < nu; ++u) launch_unit(c, units[u], j, c->stream);
            continue;
        }
        cudaEventRecord(c->ev_fork, c->stream);
        const int na = std::min(nu, casimir_ctx::NAUX);
        for (int a = 0; a < na; ++a) cudaStreamWaitEvent(c->aux[a], c->ev_fork, 0);
        for (int u = 0; u < nu; ++u) launch_unit(c, units[u], j, c->aux[u % na]);
        for (int a = 0; a < na; ++a) {
            cudaEventRecord(c->ev_join[a], c->aux[a]);
            cudaStreamWaitEvent(c->stream, c->ev_join[a], 0);
        }
    }
    launch_bump(c->d_launch, k, c->stream);
}

// Launch `k` consecutive steps (as a cached CUDA graph, or directly when the
// environment sets CASIMIR_NO_GRAPHS, e.g. for kernel profiling) and advance
// the launch counter.
static int run_chunk(casimir_ctx *c, int k)
{
    NvtxRange nvtx_("casimir.chunk");
    static const bool no_graphs = std::getenv("CASIMIR_NO_GRAPHS") != nullptr;
    if (no_graphs) {
        CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        launch_steps(c, k);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    }
    auto it = c->graphs.find(k);
    if (!no_graphs && it == c->graphs.end()) {
        std::lock_guard<std::mutex> cg(c->capture_mu);
        cudaGraph_t g;
        CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        launch_steps(c, k);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (e != cudaSuccess) return fail(CASIMIR_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t ex;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(CASIMIR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        it = c->graphs.emplace(k, ex).first;
    }
    if (!no_graphs) {
        CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
        CUDA_TRY(cudaGraphLaunch(it->second, c->stream));
        CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    }
    c->h_launch += k;
    int per_step = 0;
    for (int gi = 0; gi < casimir_ctx::NGROUPS; ++gi)
        if (c->groups[gi].ntiles > 0)
            per_step += ((gi >= 2 && gi < 10) || (gi >= casimir_ctx::G_LINE3 && gi < casimir_ctx::G_CYL)) ? 2 : 1;
    for (casimir_request *r : c->active) r->launches += (int64_t)k * per_step + 1;
    return CASIMIR_OK;
}

static void finish_request(casimir_ctx *c, casimir_request *r, int status)
{
    casimir_plan_t *P = r->plan;
    const PlanData &D = P->data;
    size_t ns = P->sims.size();
    r->per_sim.assign(ns, 0.0);
    // ordered, compensated sum of the per-simulation contributions times the k-point weights
    double s = 0, comp = 0, te = 0;
    for (size_t q = 0; q < ns; ++q) {
        double v = r->h_acc[q] * D.kweight[D.sims[q].kpt];
        r->per_sim[q] = v;
        double y = v - comp, t = s + y;
        comp = (t - s) - y;
        s = t;
        te += std::fabs(r->h_acc[ns + q] * D.kweight[D.sims[q].kpt]);
    }
    r->F[0] = r->F[1] = r->F[2] = 0.0;
    r->F[D.prob.force_axis] = s;
    r->err = te;
    dev_free(c, r->block);
    c->used -= align256(P->field_elems * P->rsize) + 2 * align256(ns * 8);
    r->block = nullptr;
    r->t_done = now_ms();
    r->status = status;
    P->inflight--;
    r->state.store(status == CASIMIR_OK ? 2 : 3, std::memory_order_release);
}

// One engine iteration: run a chunk, then issue copy-backs for finished requests
// and retire those whose copies landed.  Returns 0 or an error code.
static int engine_iterate(casimir_ctx *c)
{
    activate_waves(c);
    if (c->dirty) {
        int rc = rebuild(c);
        if (rc) return rc;
    }
    if (c->ntiles > 0 && !c->active_waves.empty()) {
        int64_t next = c->h_launch;
        int64_t rem = INT64_MAX;
        for (auto &aw : c->active_waves) {
            const casimir_request::Wave &w = aw.first->waves[aw.second];
            rem = std::min<int64_t>(rem, w.s0 + aw.first->plan->launches - (next - 1));
        }
        if (rem > 0) {
            int k = (int)std::min<int64_t>(64, rem);
            int rc = run_chunk(c, k);
            if (rc) return rc;
            CUDA_TRY(cudaEventSynchronize(c->ev1));
            float ms = 0;
            cudaEventElapsedTime(&ms, c->ev0, c->ev1);
            std::lock_guard<std::mutex> lk(c->mu);   // the statistics are read under the lock
            c->step_ms += ms;
            c->step_launches += k;
            for (auto &aw : c->active_waves) {
                const casimir_request::Wave &w = aw.first->waves[aw.second];
                const casimir_plan_t *P = aw.first->plan;
                int64_t T = P->data.prob.n_steps, K = P->k2d;
                // steps covered by launches next .. next+k-1 of this wave
                int64_t l_lo = std::max<int64_t>(1, next - w.s0), l_hi = std::min<int64_t>(P->launches, next + k - 1 - w.s0);
                if (l_hi >= l_lo) c->cell_updates += (std::min<int64_t>(T, K * l_hi) - K * (l_lo - 1)) * w.cells;
            }
        }
    }
    // retire finished waves
    for (size_t q = 0; q < c->active_waves.size();) {
        casimir_request *r = c->active_waves[q].first;
        casimir_request::Wave &w = r->waves[c->active_waves[q].second];
        if (c->h_launch - 1 - w.s0 >= r->plan->launches) {
            w.state = 2;
            r->waves_done++;
            c->active_bytes -= w.bytes;
            c->active_waves.erase(c->active_waves.begin() + q);
            c->dirty = true;
        } else {
            ++q;
        }
    }
    for (casimir_request *r : c->active) {
        if (r->copy_issued) continue;
        bool done = r->waves_done == r->waves.size();
        const double wd = c->watchdog_ms.load();
        bool timed_out = wd > 0 && now_ms() - r->t_admit > wd;
        if (done || timed_out || r->cancel) {
            if (!done) drop_waves(c, r);
            size_t ns = r->plan->sims.size();
            CUDA_TRY(cudaMemcpyAsync(r->h_acc, r->acc, ns * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaMemcpyAsync(r->h_acc + ns, r->tail, ns * 8, cudaMemcpyDeviceToHost, c->stream));
            if (!r->done_ev) CUDA_TRY(cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming));
            CUDA_TRY(cudaEventRecord(r->done_ev, c->stream));
            r->copy_issued = true;
            if (!done) r->status = r->cancel ? CASIMIR_ECANCELED : CASIMIR_ETIMEOUT;
        }
    }
    {
        // the active list and the memory accounting are read by other threads under the lock
        std::lock_guard<std::mutex> lk(c->mu);
        for (size_t q = 0; q < c->active.size();) {
            casimir_request *r = c->active[q];
            if (r->copy_issued && cudaEventQuery(r->done_ev) == cudaSuccess) {
                c->active.erase(c->active.begin() + q);
                finish_request(c, r, r->status.load());
            } else {
                ++q;
            }
        }
    }
    activate_waves(c);
    return CASIMIR_OK;
}

static bool fits(casimir_ctx *c, casimir_plan_t *P)
{
    uint64_t need = (uint64_t)P->request_bytes + (P->dev.block ? 0 : (uint64_t)P->table_bytes);
    return c->used + need <= c->budget;
}

static void worker_main(casimir_ctx *c)
{
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(c->mu);
    while (!c->stop) {
        // admission: FIFO while the budget allows
        while (!c->queue.empty()) {
            casimir_request *r = c->queue.front();
            if (r->cancel) {
                c->queue.pop_front();
                r->status = CASIMIR_ECANCELED;
                r->plan->inflight--;
                r->state = 3;
                c->cv.notify_all();
                continue;
            }
            if (!fits(c, r->plan) && !c->active.empty()) break;
            c->queue.pop_front();
            int rc = admit(c, r);
            if (rc) {
                r->msg = g_err;
                r->status = rc;
                r->plan->inflight--;
                r->state = 3;
                c->cv.notify_all();
            }
        }
        if (c->active.empty()) {
            c->cv.wait(lk, [&] { return c->stop || !c->queue.empty(); });
            continue;
        }
        lk.unlock();
        int rc = engine_iterate(c);
        lk.lock();
        if (rc) {
            const std::string msg = g_err;
            for (casimir_request *r : c->active) {
                dev_free(c, r->block);
                r->block = nullptr;
                r->msg = msg;
                r->status = rc;
                r->plan->inflight--;
                r->state = 3;
            }
            c->active.clear();
            c->active_waves.clear();
            c->pending_waves.clear();
            c->active_bytes = 0;
            c->dirty = true;
        }
        c->cv.notify_all();
    }
}

// ---------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------

extern "C" {

const char *casimir_last_error(void) { return g_err.c_str(); }

int casimir_ctx_create(int device, uint64_t budget, casimir_ctx_t **out)
{
    if (!out) return fail(CASIMIR_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(CASIMIR_EINVAL, "no such CUDA device");
    CUDA_TRY(cudaSetDevice(device));
    CUDA_TRY(march6_prepare());
    auto *c = new casimir_ctx();
    c->device = device;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = budget ? budget : (uint64_t)(0.9 * (double)fr);
    // waves off by default: one launch per step over every admitted simulation measured
    // faster than L2-sized waves (each launch then fills the GPU)
    c->wave_bytes = 0;
    if (const char *e = std::getenv("CASIMIR_WAVE_BYTES")) c->wave_bytes = std::atoll(e);
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return fail(CASIMIR_ECUDA, "stream"); }
    c->own_stream = true;
    if (cudaMalloc(&c->d_launch, sizeof(int64_t)) != cudaSuccess) { cudaStreamDestroy(c->stream); delete c; return fail(CASIMIR_ENOMEM, "launch counter"); }
    cudaMemcpy(c->d_launch, &c->h_launch, sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaEventCreate(&c->ev0);
    cudaEventCreate(&c->ev1);
    cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    for (int a = 0; a < casimir_ctx::NAUX; ++a) {
        cudaStreamCreateWithFlags(&c->aux[a], cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&c->ev_join[a], cudaEventDisableTiming);
    }
    *out = c;
    return CASIMIR_OK;
}

void casimir_ctx_destroy(casimir_ctx_t *c)
{
    if (!c) return;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
    }
    c->cv.notify_all();
    if (c->worker.joinable()) c->worker.join();
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    for (casimir_request *r : c->active) dev_free(c, r->block);
    drop_graphs(c);
    for (auto &G : c->groups) {
        dev_free(c, G.sims);
        dev_free(c, G.tiles);
    }
    cudaFree(c->d_launch);
    cudaEventDestroy(c->ev0);
    cudaEventDestroy(c->ev1);
    cudaEventDestroy(c->ev_fork);
    for (int a = 0; a < casimir_ctx::NAUX; ++a) {
        cudaStreamDestroy(c->aux[a]);
        cudaEventDestroy(c->ev_join[a]);
    }
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

int casimir_ctx_set_stream(casimir_ctx_t *c, void *stream)
{
    if (!c) return fail(CASIMIR_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->active.empty() || !c->queue.empty()) return fail(CASIMIR_EBUSY, "requests in flight");
    if (c->own_stream) cudaStreamDestroy(c->stream);
    if (stream) {
        c->stream = (cudaStream_t)stream;
        c->own_stream = false;
    } else {
        cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        c->own_stream = true;
    }
    drop_graphs(c);
    c->dirty = true;
    return CASIMIR_OK;
}

int casimir_ctx_set_allocator(casimir_ctx_t *c, casimir_alloc_fn a, casimir_free_fn f, void *user)
{
    if (!c || (!a) != (!f)) return fail(CASIMIR_EINVAL, "allocator needs both callbacks");
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->active.empty() || !c->queue.empty() || c->groups[0].sims) return fail(CASIMIR_EBUSY, "set the allocator before the first request");
    c->alloc = a;
    c->freef = f;
    c->user = user;
    return CASIMIR_OK;
}

int casimir_ctx_set_watchdog(casimir_ctx_t *c, double max_ms)
{
    if (!c || max_ms < 0) return fail(CASIMIR_EINVAL, "watchdog");
    c->watchdog_ms = max_ms;
    return CASIMIR_OK;
}

int casimir_ctx_set_wave_bytes(casimir_ctx_t *c, int64_t bytes)
{
    if (!c || bytes < 0) return fail(CASIMIR_EINVAL, "wave bytes");
    std::lock_guard<std::mutex> lk(c->mu);
    c->wave_bytes = bytes;
    return CASIMIR_OK;
}

int casimir_ctx_kernel_stats(casimir_ctx_t *c, double *step_ms, int64_t *launches, int64_t *cell_updates, int reset)
{
    if (!c) return fail(CASIMIR_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    if (step_ms) *step_ms = c->step_ms;
    if (launches) *launches = c->step_launches;
    if (cell_updates) *cell_updates = c->cell_updates;
    if (reset) {
        c->step_ms = 0;
        c->step_launches = 0;
        c->cell_updates = 0;
    }
    return CASIMIR_OK;
}

// Options with defaults filled in (the environment variables CASIMIR_STEP2D_K, CASIMIR_LINE3
// and CASIMIR_COL3 set the defaults of steps_per_launch and kernel_3d, for A/B runs).
// The default of steps_per_launch is 3 for FP32 runs (fewer passes over memory; measured 25%
// faster than 2 on the piston sweep) and 2 for FP64 runs (bound by FP64 arithmetic, where the
// third step's extra halo work costs more than the memory it saves).  The default 3D kernel is
// the column march for runs without CPML (73.0 against 67.4 Gcell-updates/s for the x-line
// kernel on a closed 160^3 sphere cell) and the x-line kernel for runs with CPML (52.1 against
// 40.5 with a 12-cell CPML shell: the march's CPML path carries 2.5 times the instructions of
// its interior path).
static bool has_pml3d(const casimir_problem &p)
{
    if (p.dims != 3) return false;
    for (int a = 0; a < 3; ++a)
        if (p.bc[a] == CASIMIR_BC_PML) return true;
    return false;
}

static int resolve_options(const casimir_plan_options *in, casimir_plan_options *out, bool fp64, bool pml3d)
{
    static const int k_env = [] {
        const char *e = std::getenv("CASIMIR_STEP2D_K");
        return e ? std::atoi(e) : 0;
    }();
    static const int l_env = [] {
        // CASIMIR_LINE3=0: the per-cell kernel; CASIMIR_COL3=0: the x-line kernel; else the column march
        const char *e = std::getenv("CASIMIR_LINE3");
        if (e && std::atoi(e) == 0) return 2;
        const char *c = std::getenv("CASIMIR_COL3");
        if (c) return std::atoi(c) == 0 ? 1 : 3;
        return 0;   // by problem: below
    }();
    casimir_plan_options o{};
    if (in) o = *in;
    if (o.steps_per_launch == 0) o.steps_per_launch = (k_env >= 1 && k_env <= 3) ? k_env : (fp64 ? 2 : 3);
    if (o.march_rows == 0) o.march_rows = MARCH_H;
    if (o.kernel_3d == 0) o.kernel_3d = l_env ? l_env : (pml3d ? 1 : 3);
    if (o.steps_per_launch < 1 || o.steps_per_launch > 3 || o.march_rows < 1 || o.march_rows > MARCH_H_MAX ||
        o.kernel_3d < 1 || o.kernel_3d > 3)
        return fail(CASIMIR_EINVAL, "plan options out of range");
    o.reserved = 0;
    *out = o;
    return CASIMIR_OK;
}

static int make_plan(casimir_ctx_t *c, const casimir_problem *p, const casimir_plan_options *opts, casimir_plan_t **out)
{
    NvtxRange nvtx_("casimir.plan");
    *out = nullptr;
    auto *P = new casimir_plan_t();
    P->ctx = c;
    int rc = resolve_options(opts, &P->opts, p->precision == CASIMIR_FP64, has_pml3d(*p));
    if (rc) { delete P; return rc; }
    std::string err;
    rc = build_plan(p, &P->data, &err);
    if (rc) { delete P; return fail(rc, err); }
    rc = prepare_plan(P);
    if (rc) { delete P; return rc; }
    if (c && (uint64_t)(P->table_bytes + P->request_bytes) > c->budget) {
        delete P;
        return fail(CASIMIR_ENOMEM, "plan needs more device memory than the context budget");
    }
    *out = P;
    return CASIMIR_OK;
}

// Problem class for autotuning: what decides which schedule is fastest.
static std::string tune_key(const casimir_problem &p)
{
    bool pml = false, lor = false, cplx = false;
    for (int a = 0; a < p.dims; ++a) pml |= p.bc[a] == CASIMIR_BC_PML;
    for (int o = 0; o < p.n_objects; ++o) lor |= p.objects[o].kind == CASIMIR_MAT_LORENTZ;
    for (int k = 0; k < p.n_kpoints; ++k)
        for (int a = 0; a < p.dims; ++a) cplx |= p.bc[a] == CASIMIR_BC_PERIODIC && p.kpoints[k].k[a] != 0.0;
    auto bucket = [](int n) { int b = 0; while ((1 << b) < n) ++b; return b; };
    std::string k = std::to_string(p.dims) + (p.polarization == CASIMIR_POL_FULL ? "F" : "T") + std::to_string(p.precision) +
                    std::to_string(p.coords) + (pml ? "p" : "") + (lor ? "l" : "") + (cplx ? "c" : "");
    for (int a = 0; a < 3; ++a) k += "," + std::to_string(bucket(p.n[a]));
    return k;
}

// Time each candidate on the problem cut to 128 steps; the fastest per cell-update wins.
static casimir_plan_options autotune(casimir_ctx *c, const casimir_problem &p)
{
    NvtxRange nvtx_("casimir.autotune");
    casimir_plan_options dflt{};
    resolve_options(nullptr, &dflt, p.precision == CASIMIR_FP64, has_pml3d(p));
    std::vector<casimir_plan_options> cand;
    if (p.dims == 3) {
        // the default first (ties keep it), then the other 3D kernels
        cand = {dflt};
        for (int k : {3, 1, 2})
            if (k != dflt.kernel_3d) {
                casimir_plan_options o = dflt;
                o.kernel_3d = k;
                cand.push_back(o);
            }
    } else if (p.polarization == CASIMIR_POL_FULL) {
        for (int rows : {32, 16, 64}) {
            casimir_plan_options o = dflt;
            o.march_rows = rows;
            cand.push_back(o);
        }
        if (dflt.steps_per_launch >= 2) {
            // the two-step marches (cylindrical runs; Cartesian FP32 runs with at most one pole
            // per material) also run one step per launch
            casimir_plan_options o = dflt;
            o.steps_per_launch = 1;
            cand.push_back(o);
        }
    } else {
        // the default first (ties keep it), then the other fusion depths
        cand = {dflt};
        for (int k : {3, 2, 1})
            if (k != dflt.steps_per_launch) {
                casimir_plan_options o = dflt;
                o.steps_per_launch = k;
                cand.push_back(o);
            }
    }
    const std::string key = tune_key(p);
    {
        std::lock_guard<std::mutex> lk(c->mu);
        auto it = c->tuned.find(key);
        if (it != c->tuned.end()) return it->second;
        if (!c->active.empty() || !c->queue.empty() || c->sync_busy) return dflt;   // never disturb running work
    }
    casimir_problem trial = p;
    trial.n_steps = std::min(p.n_steps, 128);
    // the context's statistics belong to its user: restore them after the trials
    const double ms0 = c->step_ms;
    const int64_t l0 = c->step_launches, cu0 = c->cell_updates;
    double best_t = 0;
    casimir_plan_options best = dflt;
    bool any = false;
    for (const casimir_plan_options &o : cand) {
        casimir_plan_t *tp = nullptr;
        if (make_plan(c, &trial, &o, &tp) != CASIMIR_OK) continue;
        const double m_before = c->step_ms;
        const int64_t cu_before = c->cell_updates;
        double F[3];
        int rc = casimir_run(tp, F, nullptr, nullptr);
        const double dms = c->step_ms - m_before;
        const int64_t dcu = c->cell_updates - cu_before;
        casimir_plan_destroy(tp);
        if (rc != CASIMIR_OK || dcu <= 0) continue;
        const double t = dms / (double)dcu;
        if (!any || t < best_t) { best_t = t; best = o; any = true; }
    }
    c->step_ms = ms0;
    c->step_launches = l0;
    c->cell_updates = cu0;
    if (any) {
        std::lock_guard<std::mutex> lk(c->mu);
        c->tuned[key] = best;
    }
    return best;
}

int casimir_plan_ex(casimir_ctx_t *c, const casimir_problem *p, const casimir_plan_options *opts, casimir_plan_t **out)
{
    if (!p || !out) return fail(CASIMIR_EINVAL, "NULL argument");
    try {
        return make_plan(c, p, opts, out);
    } catch (const std::bad_alloc &) {
        return fail(CASIMIR_ENOMEM, "out of host memory while planning");
    } catch (const std::exception &e) {
        return fail(CASIMIR_EINVAL, std::string("planning failed: ") + e.what());
    }
}

int casimir_plan(casimir_ctx_t *c, const casimir_problem *p, casimir_plan_t **out)
{
    if (!p || !out) return fail(CASIMIR_EINVAL, "NULL argument");
    // nothing thrown by the planner (host allocation, thread creation) crosses the C ABI
    try {
        if (c && c->autotune) {
            const casimir_plan_options o = autotune(c, *p);
            return make_plan(c, p, &o, out);
        }
        return make_plan(c, p, nullptr, out);
    } catch (const std::bad_alloc &) {
        return fail(CASIMIR_ENOMEM, "out of host memory while planning");
    } catch (const std::exception &e) {
        return fail(CASIMIR_EINVAL, std::string("planning failed: ") + e.what());
    }
}

int casimir_plan_get_options(const casimir_plan_t *P, casimir_plan_options *opts)
{
    if (!P || !opts) return fail(CASIMIR_EINVAL, "NULL argument");
    *opts = P->opts;
    return CASIMIR_OK;
}

int casimir_ctx_set_autotune(casimir_ctx_t *c, int on)
{
    if (!c) return fail(CASIMIR_EINVAL, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    c->autotune = on ? 1 : 0;
    return CASIMIR_OK;
}

int casimir_plan_pml(const casimir_plan_t *P, int axis, int half, double *b, double *c, double *inv_kappa)
{
    if (!P || !b || !c || !inv_kappa || axis < 0 || axis > 2 || half < 0 || half > 1)
        return fail(CASIMIR_EINVAL, "NULL argument, axis or half");
    if (P->data.geos.empty() || !P->data.geos[0].has_pml[axis]) return fail(CASIMIR_EINVAL, "not a PML axis of this plan");
    const auto &pr = P->data.geos[0].pml[axis][half];
    std::copy(pr[0].begin(), pr[0].end(), b);
    std::copy(pr[1].begin(), pr[1].end(), c);
    std::copy(pr[2].begin(), pr[2].end(), inv_kappa);
    return CASIMIR_OK;
}

int casimir_plan_site_poles(const casimir_plan_t *P, int kpoint, int comp, int pole, double *de, double *w0)
{
    if (!P || !de || !w0) return fail(CASIMIR_EINVAL, "NULL argument");
    const PlanData &D = P->data;
    if (kpoint < 0 || kpoint >= D.prob.n_kpoints || comp < 0 || comp > 2 || pole < 0 || pole >= CASIMIR_MAX_POLES)
        return fail(CASIMIR_EINVAL, "kpoint, comp or pole out of range");
    for (const Geo &g : D.geos) {
        if (g.kpt != kpoint || g.family != FAM_FULL) continue;
        for (size_t c = 0; c < g.mat.size(); ++c) {
            de[c] = w0[c] = 0.0;
            if (pole < g.npoles) {
                const size_t at = ((size_t)g.mat[c] * g.npoles + pole) * 6 + 2 * comp;
                de[c] = g.lorentz[at];
                w0[c] = g.lorentz[at + 1];
            }
        }
        return CASIMIR_OK;
    }
    return fail(CASIMIR_EINVAL, "Lorentz tables exist for six-component plans only");
}

int casimir_plan_site_coefs(const casimir_plan_t *P, int kpoint, int field, int comp, double off[3], double *out)
{
    if (!P || !off || !out) return fail(CASIMIR_EINVAL, "NULL argument");
    const PlanData &D = P->data;
    if (kpoint < 0 || kpoint >= D.prob.n_kpoints) return fail(CASIMIR_EINVAL, "kpoint out of range");
    for (const Geo &g : D.geos) {
        if (g.kpt != kpoint) continue;
        ArraySpec arrs[6];
        const int narr = family_arrays(g.family, arrs);
        for (int a = 0; a < narr; ++a) {
            if (arrs[a].field != field || arrs[a].comp != comp) continue;
            for (int q = 0; q < 3; ++q) off[q] = arrs[a].off[q];
            for (size_t c = 0; c < g.mat.size(); ++c) out[c] = g.table[(size_t)g.mat[c] * narr + a];
            return CASIMIR_OK;
        }
    }
    return fail(CASIMIR_EINVAL, "no such field array in this plan");
}

int casimir_plan_get_info(const casimir_plan_t *P, casimir_plan_info *info)
{
    if (!P || !info) return fail(CASIMIR_EINVAL, "NULL argument");
    info->n_sims = (int64_t)P->sims.size();
    info->n_cells = P->cells;
    info->cell_updates = P->cells * (int64_t)P->data.prob.n_steps;
    info->device_bytes = P->table_bytes + P->request_bytes;
    // algorithmic bytes per cell-update: every stored field read and written once, plus the material id
    bool full = !P->sims.empty() && P->sims[0].full;
    int cf = full && P->sims[0].cplx ? 2 : 1;
    info->bytes_per_update = (full ? 12 * cf : 6) * (int64_t)P->rsize + 1;
    info->upload_bytes = P->table_bytes;
    info->launches = P->launches;
    // one step over every simulation: the field planes, the CPML psi planes of the slab cells
    // (4 per PML axis) and P, P_prev of every (site, pole) pair, each read and written once
    int64_t bps = 0;
    for (const HostSim &hs : P->sims) {
        const int64_t N = (int64_t)hs.nx * hs.ny * hs.nz, c = hs.cplx ? 2 : 1, rs = P->rsize;
        bps += N * ((hs.full ? 12 * c : 6) * rs + 1);
        if (!hs.full) continue;
        const int n[3] = {hs.nx, hs.ny, hs.nz};
        for (int a = 0; a < 3; ++a)
            if (P->data.geos[hs.geo].has_pml[a]) bps += 4 * 2 * c * rs * (N / n[a]) * 2 * P->data.prob.pml_cells[a];
        bps += P->lor_sites[hs.geo] * 4 * c * rs;
    }
    info->bytes_per_step = bps;
    return CASIMIR_OK;
}

int casimir_plan_sims(const casimir_plan_t *P, int32_t *desc, int64_t n)
{
    if (!P || !desc || n < (int64_t)P->data.sims.size()) return fail(CASIMIR_EINVAL, "desc too small");
    for (size_t s = 0; s < P->data.sims.size(); ++s) {
        const Sim &m = P->data.sims[s];
        int32_t *d = desc + 6 * s;
        d[0] = m.kpt; d[1] = m.face; d[2] = m.n1; d[3] = m.n2; d[4] = m.kind; d[5] = m.comp;
    }
    return CASIMIR_OK;
}

int64_t casimir_plan_sim_entries(const casimir_plan_t *P, int64_t sim, int which, int32_t *comp, int64_t *idx,
                                 double *val, int64_t cap)
{
    if (!P || sim < 0 || sim >= (int64_t)P->data.sims.size() || (which != 0 && which != 1) || cap < 0 ||
        (cap > 0 && (!comp || !idx || !val)))
        return fail(CASIMIR_EINVAL, "simulation index, which or buffers");
    const Sim &m = P->data.sims[sim];
    ArraySpec arrs[6];
    family_arrays(m.family, arrs);
    const std::vector<Entry> &v = which == 0 ? m.src : m.meas;
    for (size_t e = 0; e < v.size() && (int64_t)e < cap; ++e) {
        comp[e] = 3 * arrs[v[e].arr].field + arrs[v[e].arr].comp;
        idx[e] = v[e].idx;
        val[2 * e] = v[e].re;
        val[2 * e + 1] = v[e].im;
    }
    return (int64_t)v.size();
}

int casimir_plan_weights(const casimir_plan_t *P, double *w, int64_t n)
{
    if (!P || !w || n < (int64_t)P->data.gw.size()) return fail(CASIMIR_EINVAL, "w too small");
    std::copy(P->data.gw.begin(), P->data.gw.end(), w);
    return CASIMIR_OK;
}

void casimir_plan_destroy(casimir_plan_t *P)
{
    if (!P) return;
    casimir_ctx *c = P->ctx;
    if (c) {
        // requests of this plan still queued or running finish first
        std::unique_lock<std::mutex> lk(c->mu);
        c->cv.wait(lk, [&] { return P->inflight.load() == 0; });
    }
    if (c && P->dev.block) {
        std::lock_guard<std::mutex> lk(c->mu);
        std::lock_guard<std::mutex> cg(c->capture_mu);
        cudaStreamSynchronize(c->stream);
        dev_free(c, P->dev.block);
        c->used -= P->dev.bytes;
    }
    delete P;
}

int casimir_submit(casimir_plan_t *P, uint64_t tag, casimir_ticket *out)
{
    if (!P || !out) return fail(CASIMIR_EINVAL, "NULL argument");
    casimir_ctx *c = P->ctx;
    if (!c) return fail(CASIMIR_EINVAL, "host-only plan (created without a context)");
    if (c->sync_busy.load()) return fail(CASIMIR_EBUSY, "a synchronous run is using the context");
    auto *r = new casimir_request();
    r->plan = P;
    r->tag = tag;
    r->t_submit = now_ms();
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (c->queue.size() >= 4096) { delete r; return fail(CASIMIR_EBUSY, "request queue full"); }
        P->inflight++;
        c->queue.push_back(r);
        if (!c->worker_on) {
            c->worker = std::thread(worker_main, c);
            c->worker_on = true;
        }
    }
    c->cv.notify_all();
    *out = r;
    return CASIMIR_OK;
}

static void release(casimir_request *r)
{
    if (r->h_acc) cudaFreeHost(r->h_acc);
    if (r->done_ev) cudaEventDestroy(r->done_ev);
    delete r;
}

int casimir_force(casimir_ticket r, int wait_ms, double F[3], double *err_est, casimir_stats *st)
{
    if (!r) return fail(CASIMIR_EINVAL, "ticket is NULL");
    casimir_ctx *c = r->plan->ctx;
    std::unique_lock<std::mutex> lk(c->mu);
    auto ready = [&] { return r->state >= 2; };
    if (wait_ms < 0) c->cv.wait(lk, ready);
    else if (wait_ms > 0) c->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    if (!ready()) return CASIMIR_NOTREADY;
    int status = r->status;
    if (F) for (int a = 0; a < 3; ++a) F[a] = r->F[a];
    if (err_est) *err_est = r->err;
    if (st) {
        st->queue_ms = r->t_admit - r->t_submit;
        st->device_ms = r->t_done - r->t_admit;
        st->total_ms = r->t_done - r->t_submit;
        st->cell_updates = r->plan->cells * (int64_t)r->plan->data.prob.n_steps;
        st->kernel_launches = r->launches;
    }
    const std::string msg = r->msg;
    lk.unlock();
    {
        std::lock_guard<std::mutex> cg(c->capture_mu);
        release(r);
    }
    if (status == CASIMIR_ETIMEOUT) return fail(status, "watchdog stopped the run");
    if (status == CASIMIR_ECANCELED) return fail(status, "request cancelled");
    if (status != CASIMIR_OK) return fail(status, msg.empty() ? "request failed" : msg);
    return CASIMIR_OK;
}

int casimir_cancel(casimir_ticket r)
{
    if (!r) return fail(CASIMIR_EINVAL, "ticket is NULL");
    casimir_ctx *c = r->plan->ctx;
    std::lock_guard<std::mutex> lk(c->mu);
    r->cancel = true;
    c->cv.notify_all();
    return CASIMIR_OK;
}

int casimir_run(casimir_plan_t *P, double F[3], double *per_sim, casimir_stats *st)
{
    NvtxRange nvtx_("casimir.run");
    if (!P) return fail(CASIMIR_EINVAL, "plan is NULL");
    casimir_ctx *c = P->ctx;
    if (!c) return fail(CASIMIR_EINVAL, "host-only plan (created without a context)");
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->active.empty() || !c->queue.empty()) return fail(CASIMIR_EBUSY, "requests in flight on this context");
        c->sync_busy = 1;
    }
    cudaSetDevice(c->device);
    casimir_request r;
    r.plan = P;
    r.t_submit = now_ms();
    P->inflight++;
    int rc = admit(c, &r);
    while (rc == CASIMIR_OK && r.state == 1) rc = engine_iterate(c);
    if (rc) {
        for (casimir_request *q : c->active) dev_free(c, q->block);
        c->active.clear();
        c->active_waves.clear();
        c->pending_waves.clear();
        c->active_bytes = 0;
        c->dirty = true;
    }
    c->sync_busy = 0;
    int status = rc ? rc : r.status.load();
    if (status == CASIMIR_OK) {
        if (F) for (int a = 0; a < 3; ++a) F[a] = r.F[a];
        if (per_sim) std::copy(r.per_sim.begin(), r.per_sim.end(), per_sim);
        if (st) {
            st->queue_ms = 0;
            st->device_ms = r.t_done - r.t_admit;
            st->total_ms = r.t_done - r.t_submit;
            st->cell_updates = P->cells * (int64_t)P->data.prob.n_steps;
            st->kernel_launches = r.launches;
        }
    }
    if (r.h_acc) cudaFreeHost(r.h_acc);
    if (r.done_ev) cudaEventDestroy(r.done_ev);
    if (status != CASIMIR_OK && rc == CASIMIR_OK) return fail(status, "run stopped");
    return status;
}

}  // extern "C"

// ---------------------------------------------------------------------------------
// Allocation-free run of a two-dimensional plan.
//
// Some callers cannot let a library allocate device memory: hosts that have
// handed nearly all of the GPU's memory to their own pool, embedders whose memory
// manager must not be re-entered from one of its own callbacks, and loops that
// cannot absorb the device-wide synchronisation of cudaFree.  casimir_run_noalloc
// lets them run a plan without any device allocation: the fields, the simulation
// and tile tables, the copied plan tables and the launch counter all live in the
// file-scope array below, which every device that loads the library holds until
// the process exits.
// ---------------------------------------------------------------------------------

static constexpr size_t kNoallocBytes = size_t(64) << 20;   // 64 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];   // device address of the array, per device ordinal

// Device address of g_noalloc_scratch on the current device.  In host code the
// symbol is only a host-side stand-in, so the address is looked up once per
// device (with that device current) and cached.
static int noalloc_scratch(void **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return fail(CASIMIR_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(CASIMIR_ECUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return CASIMIR_OK;
}

// Copy `n` items produced by `make(i, &item)` to device memory through a small
// stack buffer (copies from pageable memory return once the source is staged,
// so the buffer can be refilled immediately).
template <typename T, typename F>
static int staged_copy(T *dst, int64_t n, F make, cudaStream_t st)
{
    constexpr int B = 64;
    T buf[B];
    for (int64_t i0 = 0; i0 < n; i0 += B) {
        int m = (int)std::min<int64_t>(B, n - i0);
        for (int j = 0; j < m; ++j) make(i0 + j, &buf[j]);
        CUDA_TRY(cudaMemcpyAsync(dst + i0, buf, m * sizeof(T), cudaMemcpyHostToDevice, st));
    }
    return CASIMIR_OK;
}

extern "C" int casimir_run_noalloc(const casimir_plan_t *P, double *d_per_sim, void *cuda_stream)
{
    if (!P || !d_per_sim) return fail(CASIMIR_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const PlanData &D = P->data;
    for (const Geo &g : D.geos)
        if (g.family == FAM_FULL) return fail(CASIMIR_EINVAL, "casimir_run_noalloc runs two-dimensional TM/TE plans only");
    const size_t ns = P->sims.size(), nt = P->tiles.size();
    // scratch layout: counter | sims | tiles | tail | mat | coef | gw | ents | src | fields
    size_t off[11];
    off[0] = 0;
    off[1] = align256(sizeof(int64_t));
    off[2] = off[1] + align256(ns * sizeof(DevSim2D));
    off[3] = off[2] + align256(nt * sizeof(DevTile));
    off[4] = off[3] + align256(ns * sizeof(double));
    off[5] = off[4] + align256(P->mat_all.size());
    off[6] = off[5] + align256(P->coef_all.size() * P->rsize);
    off[7] = off[6] + align256(D.gw.size() * sizeof(double));
    off[8] = off[7] + align256(P->ents.size() * sizeof(DevEnt));
    off[9] = off[8] + align256(P->src.size() * sizeof(DevSrc));
    off[10] = off[9] + align256((size_t)P->field_elems * P->rsize);
    if (off[10] > kNoallocBytes)
        return fail(CASIMIR_ENOMEM, "casimir_run_noalloc: the plan needs " + std::to_string(off[10]) +
                                        " bytes of scratch; the static array holds " + std::to_string(kNoallocBytes));
    void *base_v = nullptr;
    int rc = noalloc_scratch(&base_v);
    if (rc) return rc;
    char *base = (char *)base_v;
    int64_t *d_counter = (int64_t *)(base + off[0]);
    DevSim2D *d_sims = (DevSim2D *)(base + off[1]);
    DevTile *d_tiles = (DevTile *)(base + off[2]);
    double *d_tail = (double *)(base + off[3]);
    uint8_t *d_mat = (uint8_t *)(base + off[4]);
    char *d_coef = base + off[5];
    double *d_gw = (double *)(base + off[6]);
    DevEnt *d_ents = (DevEnt *)(base + off[7]);
    DevSrc *d_src = (DevSrc *)(base + off[8]);
    char *d_fields = base + off[9];

    // the array keeps the previous call's contents: clear the fields, the tail sums and the output
    CUDA_TRY(cudaMemsetAsync(d_fields, 0, (size_t)P->field_elems * P->rsize, st));
    CUDA_TRY(cudaMemsetAsync(d_tail, 0, ns * sizeof(double), st));
    CUDA_TRY(cudaMemsetAsync(d_per_sim, 0, ns * sizeof(double), st));
    static const int64_t one = 1;
    CUDA_TRY(cudaMemcpyAsync(d_counter, &one, sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (!P->mat_all.empty()) CUDA_TRY(cudaMemcpyAsync(d_mat, P->mat_all.data(), P->mat_all.size(), cudaMemcpyHostToDevice, st));
    if (P->fp64) {
        CUDA_TRY(cudaMemcpyAsync(d_coef, P->coef_all.data(), P->coef_all.size() * 8, cudaMemcpyHostToDevice, st));
    } else {
        rc = staged_copy((float *)d_coef, (int64_t)P->coef_all.size(),
                         [&](int64_t i, float *o) { *o = (float)P->coef_all[i]; }, st);
        if (rc) return rc;
    }
    CUDA_TRY(cudaMemcpyAsync(d_gw, D.gw.data(), D.gw.size() * 8, cudaMemcpyHostToDevice, st));
    if (!P->ents.empty()) CUDA_TRY(cudaMemcpyAsync(d_ents, P->ents.data(), P->ents.size() * sizeof(DevEnt), cudaMemcpyHostToDevice, st));
    if (!P->src.empty()) CUDA_TRY(cudaMemcpyAsync(d_src, P->src.data(), P->src.size() * sizeof(DevSrc), cudaMemcpyHostToDevice, st));
    const double sg = D.prob.sigma, dt = D.dt, dx = D.dx;
    rc = staged_copy(d_sims, (int64_t)ns, [&](int64_t s, DevSim2D *d) {
        const HostSim &hs = P->sims[s];
        *d = DevSim2D{};
        d->fields = d_fields + hs.field_off * P->rsize;
        d->mat = d_mat + P->mat_off[hs.geo];
        d->coef = d_coef + P->coef_off[hs.geo] * P->rsize;
        d->gw = d_gw;
        d->acc = d_per_sim + s;
        d->tail = d_tail + s;
        d->s0 = 0;
        d->nx = hs.nx;
        d->ny = hs.ny;
        d->T = D.prob.n_steps;
        d->tail_from = D.prob.n_steps;
        d->second_u = hs.second_u;
        d->nmat = D.geos[hs.geo].nmat;
        d->a = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt);
        d->bf = dt / (1.0 + 0.5 * sg * dt) / dx;
        d->hf = dt / dx;
    }, st);
    if (rc) return rc;
    rc = staged_copy(d_tiles, (int64_t)nt, [&](int64_t t, DevTile *d) {
        const HostTile &ht = P->tiles[t];
        *d = DevTile{ht.sim, ht.i0, ht.j0, ht.ne, d_ents + ht.ent0};
    }, st);
    if (rc) return rc;
    launch_inject(P->fp64, d_fields, d_src, (int)P->src.size(), st);
    for (int n = 0; n < D.prob.n_steps; ++n)
        launch_step2d(P->fp64, d_sims, d_tiles, (int)nt, d_counter, n, st);
    CUDA_TRY(cudaGetLastError());
    return CASIMIR_OK;
}
