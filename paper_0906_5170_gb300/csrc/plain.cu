// The plain execution of a plan, kept as the comparison point for the batched
// executor: one simulation at a time, one launch per half of each time step
// group and one separate projection launch per step, no CUDA graph.  The field
// updates are the same kernels the batched path uses, so the two differ only
// in how the work is scheduled.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "engine_internal.h"

namespace {

struct PlainEnt {
    int64_t idx_re, idx_im;   // element offsets from the simulation's block (idx_im < 0: real)
    double wre, wim;
};

template <typename R>
__global__ void k_project(const R *base, int64_t parity_stride, const PlainEnt *ents, int ne,
                          const double *gw, int n, double *acc)
{
    __shared__ double red[8];
    const R *f = base + (n & 1) * parity_stride;
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

}  // namespace

extern "C" int casimir_run_plain(casimir_plan_t *P, double F[3], double *per_sim, casimir_stats *st)
{
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
    size_t max_tiles = 1, max_ents = 1;
    for (const HostSim &hs : P->sims) {
        max_tiles = std::max<size_t>(max_tiles, hs.ntile);
        max_ents = std::max<size_t>(max_ents, hs.nent);
    }
    size_t bf = align256(P->field_elems * P->rsize), ba = align256(ns * 8);
    size_t bs = align256(std::max(sizeof(DevSim2D), sizeof(DevSim6)));
    size_t bt = align256(max_tiles * std::max(sizeof(DevTile), sizeof(DevTile6)));
    size_t be = align256(max_ents * sizeof(PlainEnt));
    void *blk = nullptr;
    rc = dev_alloc(c, bf + 2 * ba + bs + bt + be + 256, &blk);
    if (rc) return rc;
    struct Free {
        casimir_ctx *c;
        void *p;
        ~Free() { dev_free(c, p); }
    } guard{c, blk};
    char *b = (char *)blk;
    double *acc = (double *)(b + bf), *tail = (double *)(b + bf + ba);
    void *d_sim = b + bf + 2 * ba;
    void *d_tiles = b + bf + 2 * ba + bs;
    PlainEnt *d_ents = (PlainEnt *)(b + bf + 2 * ba + bs + bt);
    int64_t *d_counter = (int64_t *)(b + bf + 2 * ba + bs + bt + be);
    CUDA_TRY(cudaMemsetAsync(blk, 0, bf + 2 * ba, s));
    launch_inject(P->fp64, blk, P->dev.src, (int)P->src.size(), s);
    launch_inject6(P->fp64, blk, P->dev.src6, (int)P->src6.size(), s);
    static const int64_t one = 1;
    CUDA_TRY(cudaMemcpyAsync(d_counter, &one, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    int64_t launches = 2;
    std::vector<DevTile> t2;
    std::vector<DevTile6> t6;
    std::vector<PlainEnt> pe;
    for (size_t q = 0; q < ns; ++q) {
        const HostSim &hs = P->sims[q];
        int64_t N = (int64_t)hs.nx * hs.ny * hs.nz;
        pe.clear();
        if (!hs.full) {
            DevSim2D d;
            make_sim2d(P, b, acc, tail, 0, q, &d);
            t2.clear();
            for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                const HostTile &ht = P->tiles[t];
                t2.push_back(DevTile{0, ht.i0, ht.j0, 0, nullptr});      // projection runs separately
                for (int e = ht.ent0; e < ht.ent0 + ht.ne; ++e) {
                    const DevEnt &en = P->ents[e];
                    int loc = en.loc & 0xffff, arr = en.loc >> 16;
                    int ly = loc / TILE_X, lx = loc - ly * TILE_X;
                    int64_t g = (int64_t)arr * N + (int64_t)(ht.j0 + ly) * hs.nx + ht.i0 + lx;
                    pe.push_back(PlainEnt{hs.field_off + g, -1, en.w, 0.0});
                }
            }
            CUDA_TRY(cudaMemcpyAsync(d_sim, &d, sizeof(d), cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(d_tiles, t2.data(), t2.size() * sizeof(DevTile), cudaMemcpyHostToDevice, s));
        } else {
            DevSim6 d;
            make_sim6(P, b, acc, tail, 0, q, &d);
            t6.clear();
            int cf = hs.cplx ? 2 : 1;
            for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                const HostTile6 &ht = P->tiles6[t];
                t6.push_back(DevTile6{0, ht.count, ht.cell0, 0, 0, nullptr});
                for (int e = ht.ent0; e < ht.ent0 + ht.ne; ++e) {
                    const DevEnt6 &en = P->ents6[e];
                    int64_t cell = ht.cell0 + en.off;
                    int64_t re = hs.field_off + (int64_t)(cf * en.arr) * N + cell;
                    int64_t im = hs.cplx ? hs.field_off + (int64_t)(2 * en.arr + 1) * N + cell : -1;
                    pe.push_back(PlainEnt{re, im, en.wre, en.wim});
                }
            }
            CUDA_TRY(cudaMemcpyAsync(d_sim, &d, sizeof(d), cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(d_tiles, t6.data(), t6.size() * sizeof(DevTile6), cudaMemcpyHostToDevice, s));
        }
        if (!pe.empty()) CUDA_TRY(cudaMemcpyAsync(d_ents, pe.data(), pe.size() * sizeof(PlainEnt), cudaMemcpyHostToDevice, s));
        // 2D fields ping-pong between two buffers of 3N; the six-component fields update in place
        int64_t stride = hs.full ? 0 : 3 * N;
        for (int n = 1; n <= D.prob.n_steps; ++n) {
            if (!hs.full) {
                launch_step2d(P->fp64, (const DevSim2D *)d_sim, (const DevTile *)d_tiles, (int)t2.size(), d_counter, n - 1, s);
                ++launches;
            } else {
                for (int phase = 0; phase < 2; ++phase)
                    launch_full(P->fp64, hs.cplx, (const DevSim6 *)d_sim, (const DevTile6 *)d_tiles, (int)t6.size(), d_counter, n - 1, phase, s);
                launches += 2;
            }
            if (!pe.empty()) {
                if (P->fp64)
                    k_project<double><<<1, 256, 0, s>>>((const double *)b, stride, d_ents, (int)pe.size(), P->dev.gw, n, acc + q);
                else
                    k_project<float><<<1, 256, 0, s>>>((const float *)b, stride, d_ents, (int)pe.size(), P->dev.gw, n, acc + q);
                ++launches;
            }
        }
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(s));   // the host descriptor vectors are reused for the next simulation
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
