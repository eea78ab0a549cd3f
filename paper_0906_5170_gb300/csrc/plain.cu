// The plain execution of a plan, kept as the comparison point for the batched
// executor: one run at a time -- a run being the simulations of one k-point,
// harmonic and polarisation family (every face and source component) -- with
// the field updates of each time step launched for that run alone, a separate
// projection launch per step, and no CUDA graph.  The field updates are the
// one-step kernels (where the batched path fuses two or three steps into one
// launch, it runs the fused kernels of the same update), so the two differ in
// scheduling, not in arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <tuple>
#include <vector>

#include "engine_internal.h"

namespace {

struct PlainEnt {
    int64_t idx_re, idx_im;   // element offsets from the simulation's block (idx_im < 0: real)
    double wre, wim;
};

struct PlainSim {
    int64_t parity_stride;    // 2D fields ping-pong between two buffers; 0 for in-place updates
    int ent0, ne;
    double *acc;
};

// one block per simulation of the run
template <typename R>
__global__ void k_project(const R *base, const PlainSim *sims, const PlainEnt *all, const double *gw, int n)
{
    __shared__ double red[8];
    const PlainSim ps = sims[blockIdx.x];
    const R *f = base + (n & 1) * ps.parity_stride;
    const PlainEnt *ents = all + ps.ent0;
    const int ne = ps.ne;
    double *acc = ps.acc;
    double part = 0.0;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        PlainEnt en = ents[e];
        part += en.wre * (double)f[en.idx_re];
        if (en.idx_im >= 0) part -= en.wim * (double)f[en.idx_im];
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *acc += gw[n - 1] * s;
    }
}

// strip tiles a run needs before the plain path takes the march kernel for it: four CTAs of four
// warps on each of the 152 SMs
constexpr int64_t kPlainMarchTiles = 4 * 4 * 152;

struct Free {
    casimir_ctx *c;
    void *p;
    ~Free() { dev_free(c, p); }
};

}  // namespace

extern "C" int casimir_run_plain(casimir_plan_t *P, double F[3], double *per_sim, casimir_stats *st)
{
    NvtxRange nvtx_("casimir.run_plain");
    if (!P) return fail(CASIMIR_EINVAL, "plan is NULL");
    casimir_ctx *c = P->ctx;
    if (!c) return fail(CASIMIR_EINVAL, "host-only plan (created without a context)");
    {
        std::lock_guard<std::mutex> lk(c->mu);
        if (!c->active.empty() || !c->queue.empty()) return fail(CASIMIR_EBUSY, "requests in flight on this context");
        c->sync_busy = 1;
    }
    struct Busy {
        casimir_ctx *c;
        ~Busy() { c->sync_busy = 0; }
    } busy{c};
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    double t0 = now_ms();
    int rc = upload_plan(P, s);
    if (rc) return rc;
    const PlanData &D = P->data;
    const size_t ns = P->sims.size();
    size_t bf = align256(P->field_elems * P->rsize), ba = align256(ns * 8);
    void *blk = nullptr;
    rc = dev_alloc(c, bf + 2 * ba + 256, &blk);
    if (rc) return rc;
    Free guard{c, blk};
    char *b = (char *)blk;
    double *acc = (double *)(b + bf), *tail = (double *)(b + bf + ba);
    int64_t *d_counter = (int64_t *)(b + bf + 2 * ba);
    CUDA_TRY(cudaMemsetAsync(blk, 0, bf + 2 * ba, s));
    launch_inject(P->fp64, blk, P->dev.src, (int)P->src.size(), s);
    launch_inject6(P->fp64, blk, P->dev.src6, (int)P->src6.size(), s);
    static const int64_t one = 1;
    CUDA_TRY(cudaMemcpyAsync(d_counter, &one, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    int64_t launches = 2;
    // runs: the simulations of one k-point, harmonic and family, in order of first appearance
    std::vector<std::vector<size_t>> runs;
    {
        std::map<std::tuple<int, int, int, int>, size_t> at;
        for (size_t q = 0; q < ns; ++q) {
            const Sim &m = D.sims[q];
            auto key = std::make_tuple(m.kpt, m.n1, m.n2, m.family);
            auto it = at.find(key);
            if (it == at.end()) {
                at.emplace(key, runs.size());
                runs.push_back({q});
            } else {
                runs[it->second].push_back(q);
            }
        }
    }
    std::vector<DevSim2D> s2;
    std::vector<DevSim6> s6;
    std::vector<DevTile> t2;
    std::vector<DevTile> tv[COL3_VARIANTS];     // march and column-march tiles by kernel variant
    int voff[COL3_VARIANTS + 1] = {};
    std::vector<DevTile6> t6;
    std::vector<PlainEnt> pe;
    std::vector<PlainSim> ps;
    for (auto &run : runs) {
        s2.clear(); s6.clear(); t2.clear(); t6.clear(); pe.clear(); ps.clear();
        for (auto &v : tv) v.clear();
        bool full = P->sims[run[0]].full;
        // A two-dimensional six-component run uses the march kernel only when its strip tiles can
        // fill the GPU; a small run alone is latency-bound there (each warp walks its rows in
        // sequence) and goes faster through the one-thread-per-cell kernel, in place on buffer 0.
        bool march = P->sims[run[0]].march;
        const bool line3 = P->sims[run[0]].line3;
        const bool col3 = P->sims[run[0]].col3;
        const bool cylr = P->sims[run[0]].cyl;   // only the march kernel has the cylindrical form
        if (march) {
            int64_t nt = 0;
            for (size_t q : run) nt += P->sims[q].ntile;
            static const int64_t thr = [] {
                const char *e = std::getenv("CASIMIR_PLAIN_MARCH_TILES");
                return e ? (int64_t)std::atoll(e) : kPlainMarchTiles;
            }();
            march = nt >= thr || cylr;
        }
        int cplx = P->sims[run[0]].cplx;
        for (size_t q : run) {
            const HostSim &hs = P->sims[q];
            int64_t N = (int64_t)hs.nx * hs.ny * hs.nz;
            PlainSim one{hs.full ? (march || col3 ? hs.fhalf : 0) : 3 * N, (int)pe.size(), 0, acc + q};
            if (!hs.full) {
                DevSim2D d;
                make_sim2d(P, b, acc, tail, 0, q, &d);
                int idx = (int)s2.size();
                s2.push_back(d);
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile &ht = P->tiles[t];
                    t2.push_back(DevTile{idx, ht.i0, ht.j0, 0, nullptr});      // projection runs separately
                    for (int e = ht.ent0; e < ht.ent0 + ht.ne; ++e) {
                        const DevEnt &en = P->ents[e];
                        int loc = en.loc & 0xffff, arr = en.loc >> 16;
                        int ly = loc / TILE_X, lx = loc - ly * TILE_X;
                        int64_t g = (int64_t)arr * N + (int64_t)(ht.j0 + ly) * hs.nx + ht.i0 + lx;
                        pe.push_back(PlainEnt{hs.field_off + g, -1, en.w, 0.0});
                    }
                }
            } else if (hs.col3) {
                DevSim6 d;
                make_sim6(P, b, acc, tail, 0, q, &d);
                int idx = (int)s6.size();
                s6.push_back(d);
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile &ht = P->tilesM[t];
                    tv[ht.variant].push_back(DevTile{idx, ht.i0, ht.j0, 0, nullptr, ht.z0, ht.z1});   // projection runs separately
                    for (int e = ht.ent0; e < ht.ent0 + ht.ne; ++e) {
                        const DevEnt &en = P->entsM[e];
                        int loc = en.loc & 0xffff, arr = (en.loc >> 16) & 7, im = (en.loc >> 19) & 1;
                        int64_t plane = hs.cplx ? 2 * arr + im : arr;
                        int64_t g = plane * N + ((int64_t)en.pad * hs.ny + ht.j0 + (loc >> 5)) * hs.nx + ht.i0 + (loc & 31);
                        pe.push_back(PlainEnt{hs.field_off + g, -1, im ? -en.w : en.w, 0.0});
                    }
                }
            } else if (hs.line3) {
                DevSim6 d;
                make_sim6(P, b, acc, tail, 0, q, &d);
                int idx = (int)s6.size();
                s6.push_back(d);
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile &ht = P->tilesM[t];
                    t2.push_back(DevTile{idx, ht.i0, ht.j0, 0, nullptr});      // projection runs separately
                    for (int e = ht.ent0; e < ht.ent0 + ht.ne; ++e) {
                        const DevEnt &en = P->entsM[e];
                        int loc = en.loc & 0xffff, arr = (en.loc >> 16) & 7, im = (en.loc >> 19) & 1;
                        int64_t plane = hs.cplx ? 2 * arr + im : arr;
                        int64_t g = plane * N + (int64_t)(ht.j0 + (loc >> 5)) * hs.nx + ht.i0 + (loc & 31);
                        pe.push_back(PlainEnt{hs.field_off + g, -1, im ? -en.w : en.w, 0.0});
                    }
                }
            } else if (hs.march && !march) {
                // march layout run through the two-phase kernel: buffer 0 only, whole-cell tiles
                DevSim6 d;
                make_sim6(P, b, acc, tail, 0, q, &d);
                int idx = (int)s6.size();
                s6.push_back(d);
                for (int64_t c0 = 0; c0 < N; c0 += TILE6)
                    t6.push_back(DevTile6{idx, (int)std::min<int64_t>(TILE6, N - c0), c0, 0, 0, nullptr});
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile &ht = P->tilesM[t];
                    for (int e = ht.ent0; e < ht.ent0 + ht.ne; ++e) {
                        const DevEnt &en = P->entsM[e];
                        int loc = en.loc & 0xffff, arr = (en.loc >> 16) & 7, im = (en.loc >> 19) & 1;
                        int ly = loc / MARCH_W, lx = loc - ly * MARCH_W;
                        int64_t plane = hs.cplx ? 2 * arr + im : arr;
                        int64_t g = plane * N + (int64_t)(ht.j0 + ly) * hs.nx + ht.i0 + lx;
                        pe.push_back(PlainEnt{hs.field_off + g, -1, im ? -en.w : en.w, 0.0});
                    }
                }
            } else if (hs.march) {
                DevSim6 d;
                make_sim6(P, b, acc, tail, 0, q, &d);
                int idx = (int)s6.size();
                s6.push_back(d);
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile &ht = P->tilesM[t];
                    tv[ht.variant].push_back(DevTile{idx, ht.i0, ht.j0, 0, nullptr});   // projection runs separately
                    for (int e = ht.ent0; e < ht.ent0 + ht.ne; ++e) {
                        const DevEnt &en = P->entsM[e];
                        int loc = en.loc & 0xffff, arr = (en.loc >> 16) & 7, im = (en.loc >> 19) & 1;
                        int ly = loc / MARCH_W, lx = loc - ly * MARCH_W;
                        int64_t plane = hs.cplx ? 2 * arr + im : arr;
                        int64_t g = plane * N + (int64_t)(ht.j0 + ly) * hs.nx + ht.i0 + lx;
                        pe.push_back(PlainEnt{hs.field_off + g, -1, im ? -en.w : en.w, 0.0});
                    }
                }
            } else {
                DevSim6 d;
                make_sim6(P, b, acc, tail, 0, q, &d);
                int idx = (int)s6.size();
                s6.push_back(d);
                int cf = hs.cplx ? 2 : 1;
                for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                    const HostTile6 &ht = P->tiles6[t];
                    t6.push_back(DevTile6{idx, ht.count, ht.cell0, 0, 0, nullptr});
                    for (int e = ht.ent0; e < ht.ent0 + ht.ne; ++e) {
                        const DevEnt6 &en = P->ents6[e];
                        int64_t cell = ht.cell0 + en.off;
                        int64_t re = hs.field_off + (int64_t)(cf * en.arr) * N + cell;
                        int64_t im = hs.cplx ? hs.field_off + (int64_t)(2 * en.arr + 1) * N + cell : -1;
                        pe.push_back(PlainEnt{re, im, en.wre, en.wim});
                    }
                }
            }
            one.ne = (int)pe.size() - one.ent0;
            ps.push_back(one);
        }
        if (march || col3) {
            const int nv = col3 ? COL3_VARIANTS : MARCH_VARIANTS;
            for (int v = 0; v < nv; ++v) {
                voff[v] = (int)t2.size();
                t2.insert(t2.end(), tv[v].begin(), tv[v].end());
            }
            voff[nv] = (int)t2.size();
        }
        void *d_sim = nullptr, *d_tiles = nullptr, *d_pe = nullptr, *d_ps = nullptr;
        size_t bsim = align256(full ? s6.size() * sizeof(DevSim6) : s2.size() * sizeof(DevSim2D));
        size_t btil = align256(full && !march && !line3 && !col3 ? t6.size() * sizeof(DevTile6) : t2.size() * sizeof(DevTile));
        size_t bpe = align256(std::max<size_t>(1, pe.size()) * sizeof(PlainEnt));
        size_t bps = align256(ps.size() * sizeof(PlainSim));
        void *rb = nullptr;
        rc = dev_alloc(c, bsim + btil + bpe + bps, &rb);
        if (rc) return rc;
        Free rguard{c, rb};
        d_sim = rb;
        d_tiles = (char *)rb + bsim;
        d_pe = (char *)rb + bsim + btil;
        d_ps = (char *)rb + bsim + btil + bpe;
        if (full) {
            CUDA_TRY(cudaMemcpyAsync(d_sim, s6.data(), s6.size() * sizeof(DevSim6), cudaMemcpyHostToDevice, s));
            if (march || line3 || col3)
                CUDA_TRY(cudaMemcpyAsync(d_tiles, t2.data(), t2.size() * sizeof(DevTile), cudaMemcpyHostToDevice, s));
            else
                CUDA_TRY(cudaMemcpyAsync(d_tiles, t6.data(), t6.size() * sizeof(DevTile6), cudaMemcpyHostToDevice, s));
        } else {
            CUDA_TRY(cudaMemcpyAsync(d_sim, s2.data(), s2.size() * sizeof(DevSim2D), cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(d_tiles, t2.data(), t2.size() * sizeof(DevTile), cudaMemcpyHostToDevice, s));
        }
        if (!pe.empty()) CUDA_TRY(cudaMemcpyAsync(d_pe, pe.data(), pe.size() * sizeof(PlainEnt), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(d_ps, ps.data(), ps.size() * sizeof(PlainSim), cudaMemcpyHostToDevice, s));
        for (int n = 1; n <= D.prob.n_steps; ++n) {
            if (!full) {
                launch_step2d(P->fp64, (const DevSim2D *)d_sim, (const DevTile *)d_tiles, (int)t2.size(), d_counter, n - 1, s);
                ++launches;
            } else if (col3) {
                for (int v = 0; v < COL3_VARIANTS; ++v)
                    if (voff[v + 1] > voff[v]) {
                        launch_col3(P->fp64, cplx, v, (const DevSim6 *)d_sim, (const DevTile *)d_tiles + voff[v],
                                    voff[v + 1] - voff[v], d_counter, n - 1, s);
                        ++launches;
                    }
            } else if (line3) {
                for (int phase = 0; phase < 2; ++phase)
                    launch_line3(P->fp64, cplx, (const DevSim6 *)d_sim, (const DevTile *)d_tiles, (int)t2.size(), d_counter, n - 1, phase, s);
                launches += 2;
            } else if (march) {
                if (cylr) {
                    launch_march6_cyl(P->fp64, (const DevSim6 *)d_sim, (const DevTile *)d_tiles, voff[MARCH_VARIANTS], d_counter, n - 1, s);
                    ++launches;
                }
                for (int v = 0; v < MARCH_VARIANTS && !cylr; ++v)
                    if (voff[v + 1] > voff[v]) {
                        launch_march6(P->fp64, cplx, v, (const DevSim6 *)d_sim, (const DevTile *)d_tiles + voff[v],
                                      voff[v + 1] - voff[v], d_counter, n - 1, s);
                        ++launches;
                    }
            } else {
                for (int phase = 0; phase < 2; ++phase)
                    launch_full(P->fp64, cplx, D.prob.dims, (const DevSim6 *)d_sim, (const DevTile6 *)d_tiles, (int)t6.size(), d_counter, n - 1, phase, s);
                launches += 2;
            }
            if (P->fp64)
                k_project<double><<<(int)ps.size(), 256, 0, s>>>((const double *)b, (const PlainSim *)d_ps, (const PlainEnt *)d_pe, P->dev.gw, n);
            else
                k_project<float><<<(int)ps.size(), 256, 0, s>>>((const float *)b, (const PlainSim *)d_ps, (const PlainEnt *)d_pe, P->dev.gw, n);
            ++launches;
        }
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(s));   // the run's tables are freed and the host vectors reused
    }
    std::vector<double> h(ns);
    CUDA_TRY(cudaMemcpy(h.data(), acc, ns * 8, cudaMemcpyDeviceToHost));
    double sum = 0, comp = 0;
    for (size_t q = 0; q < ns; ++q) {
        double v = h[q] * D.kweight[D.sims[q].kpt];
        if (per_sim) per_sim[q] = v;
        double y = v - comp, t = sum + y;
        comp = (t - sum) - y;
        sum = t;
    }
    if (F) {
        F[0] = F[1] = F[2] = 0.0;
        F[D.prob.force_axis] = sum;
    }
    if (st) {
        st->queue_ms = 0;
        st->total_ms = st->device_ms = now_ms() - t0;
        st->cell_updates = P->cells * (int64_t)D.prob.n_steps;
        st->kernel_launches = launches;
    }
    return CASIMIR_OK;
}
