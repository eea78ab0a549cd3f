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
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "casimir.h"
#include "kernels.h"
#include "plan.h"

using namespace cas;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) return fail(CASIMIR_ECUDA, std::string(#expr ": ") + cudaGetErrorString(e_)); \
    } while (0)

double now_ms()
{
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

// ---------------------------------------------------------------------------------
// host-side device tables of a plan
// ---------------------------------------------------------------------------------

struct HostSim {
    int geo;
    int nx, ny;
    int second_u;
    int64_t field_off;     // element offset of this sim's 6 arrays inside the request's field block
    int tile0, ntile;      // range in the plan's tile list
    int ent0, nent;        // range in the plan's entry list (bucketed by tile)
    int src0, nsrc;        // range in the plan's source list
};

struct HostTile {
    int sim, i0, j0, ent0, ne;
};

struct DevPlan {           // device copies of a plan's static tables (kept while the plan lives)
    uint8_t *mat = nullptr;
    void *coef = nullptr;
    double *gw = nullptr;
    DevEnt *ents = nullptr;
    DevSrc *src = nullptr;
    size_t bytes = 0;
    void *block = nullptr;
};

struct casimir_ctx;

struct casimir_plan {
    casimir_ctx *ctx = nullptr;
    PlanData data;
    int fp64 = 0;
    size_t rsize = 4;
    std::vector<HostSim> sims;
    std::vector<HostTile> tiles;
    std::vector<DevEnt> ents;
    std::vector<DevSrc> src;
    std::vector<int64_t> mat_off;     // per geo, bytes
    std::vector<int64_t> coef_off;    // per geo, elements
    std::vector<uint8_t> mat_all;
    std::vector<double> coef_all;
    int64_t field_elems = 0;          // per request
    int64_t cells = 0;
    int64_t table_bytes = 0;
    int64_t request_bytes = 0;
    DevPlan dev;
    std::atomic<int> inflight{0};
};

struct casimir_request {
    casimir_plan_t *plan = nullptr;
    uint64_t tag = 0;
    std::atomic<int> state{0};   // 0 queued, 1 running, 2 done, 3 failed
    std::atomic<int> status{0};
    std::atomic<bool> cancel{false};
    double F[3] = {0, 0, 0};
    double err = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int64_t s0 = 0;
    int64_t launches = 0;
    void *block = nullptr;   // fields, acc, tail
    double *acc = nullptr, *tail = nullptr;
    double *h_acc = nullptr;  // pinned copy-back (acc then tail)
    cudaEvent_t done_ev = nullptr;
    bool copy_issued = false;
    std::vector<double> per_sim;
};

struct casimir_ctx {
    int device = 0;
    uint64_t budget = 0;
    uint64_t used = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    casimir_alloc_fn alloc = nullptr;
    casimir_free_fn freef = nullptr;
    void *user = nullptr;
    double watchdog_ms = 0;
    int64_t *d_launch = nullptr;
    int64_t h_launch = 1;            // index of the next launch
    // active set
    std::vector<casimir_request *> active;
    DevSim2D *d_sims = nullptr;
    DevTile *d_tiles = nullptr;
    size_t sims_cap = 0, tiles_cap = 0;
    int ntiles = 0;
    int fp64_active = -1;
    bool dirty = true;
    std::map<int, cudaGraphExec_t> graphs;    // per chunk length, for the current active set
    // statistics
    double step_ms = 0;
    int64_t step_launches = 0;
    int64_t cell_updates = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // worker
    std::mutex mu;
    std::condition_variable cv;
    std::deque<casimir_request *> queue;
    std::thread worker;
    bool worker_on = false;
    bool stop = false;
    std::atomic<int> sync_busy{0};
};

// ---------------------------------------------------------------------------------
// memory helpers
// ---------------------------------------------------------------------------------

static int dev_alloc(casimir_ctx *c, size_t bytes, void **out)
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

static void dev_free(casimir_ctx *c, void *p)
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
    for (auto &g : D.geos)
        if (g.family == FAM_FULL) return fail(CASIMIR_EINVAL, "polarization FULL (k_z, Bloch, 3D) is not supported by this build");
    // geometry tables
    for (auto &g : D.geos) {
        P->mat_off.push_back((int64_t)P->mat_all.size());
        P->mat_all.insert(P->mat_all.end(), g.mat.begin(), g.mat.end());
        size_t pad = align256(P->mat_all.size()) - P->mat_all.size();
        P->mat_all.insert(P->mat_all.end(), pad, 0);
        P->coef_off.push_back((int64_t)P->coef_all.size());
        P->coef_all.insert(P->coef_all.end(), g.table.begin(), g.table.end());
        while (P->coef_all.size() % 32) P->coef_all.push_back(0.0);
    }
    // sims, tiles, entries, sources
    int64_t off = 0;
    for (size_t s = 0; s < D.sims.size(); ++s) {
        const Sim &sm = D.sims[s];
        const Geo &g = D.geos[sm.geo];
        HostSim hs{};
        hs.geo = sm.geo;
        hs.nx = g.n[0];
        hs.ny = g.n[1];
        hs.second_u = sm.second_u;
        hs.field_off = off;
        int64_t N = (int64_t)hs.nx * hs.ny;
        off += 6 * N;
        off = (off + 63) & ~(int64_t)63;
        P->cells += N;
        int tx = (hs.nx + TILE_X - 1) / TILE_X, ty = (hs.ny + TILE_Y - 1) / TILE_Y;
        hs.tile0 = (int)P->tiles.size();
        hs.ntile = tx * ty;
        // bucket measurement entries by tile
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
        P->sims.push_back(hs);
    }
    P->field_elems = off;
    P->table_bytes = (int64_t)(align256(P->mat_all.size()) + align256(P->coef_all.size() * P->rsize) +
                               align256(D.gw.size() * 8) + align256(P->ents.size() * sizeof(DevEnt)) +
                               align256(P->src.size() * sizeof(DevSrc)));
    P->request_bytes = (int64_t)(align256(P->field_elems * P->rsize) + 2 * align256(P->sims.size() * 8) +
                                 P->tiles.size() * sizeof(DevTile) + P->sims.size() * sizeof(DevSim2D));
    return CASIMIR_OK;
}

static int upload_plan(casimir_plan_t *P, cudaStream_t st)
{
    if (P->dev.block) return CASIMIR_OK;
    casimir_ctx *c = P->ctx;
    size_t b_mat = align256(P->mat_all.size()), b_coef = align256(P->coef_all.size() * P->rsize),
           b_gw = align256(P->data.gw.size() * 8), b_ent = align256(P->ents.size() * sizeof(DevEnt)),
           b_src = align256(P->src.size() * sizeof(DevSrc));
    size_t total = b_mat + b_coef + b_gw + b_ent + b_src;
    void *blk;
    int rc = dev_alloc(c, total, &blk);
    if (rc) return rc;
    char *p = (char *)blk;
    P->dev.block = blk;
    P->dev.bytes = total;
    P->dev.mat = (uint8_t *)p;
    p += b_mat;
    P->dev.coef = p;
    p += b_coef;
    P->dev.gw = (double *)p;
    p += b_gw;
    P->dev.ents = (DevEnt *)p;
    p += b_ent;
    P->dev.src = (DevSrc *)p;
    CUDA_TRY(cudaMemcpyAsync(P->dev.mat, P->mat_all.data(), P->mat_all.size(), cudaMemcpyHostToDevice, st));
    if (P->fp64) {
        CUDA_TRY(cudaMemcpyAsync(P->dev.coef, P->coef_all.data(), P->coef_all.size() * 8, cudaMemcpyHostToDevice, st));
    } else {
        std::vector<float> f(P->coef_all.begin(), P->coef_all.end());
        CUDA_TRY(cudaMemcpyAsync(P->dev.coef, f.data(), f.size() * 4, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    CUDA_TRY(cudaMemcpyAsync(P->dev.gw, P->data.gw.data(), P->data.gw.size() * 8, cudaMemcpyHostToDevice, st));
    if (!P->ents.empty())
        CUDA_TRY(cudaMemcpyAsync(P->dev.ents, P->ents.data(), P->ents.size() * sizeof(DevEnt), cudaMemcpyHostToDevice, st));
    if (!P->src.empty())
        CUDA_TRY(cudaMemcpyAsync(P->dev.src, P->src.data(), P->src.size() * sizeof(DevSrc), cudaMemcpyHostToDevice, st));
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
    CUDA_TRY(cudaGetLastError());
    if (!r->h_acc) CUDA_TRY(cudaMallocHost((void **)&r->h_acc, std::max<size_t>(1, 2 * P->sims.size()) * 8));
    r->s0 = c->h_launch - 1;
    r->state = 1;
    r->t_admit = now_ms();
    c->active.push_back(r);
    c->dirty = true;
    return CASIMIR_OK;
}

static int rebuild(casimir_ctx *c)
{
    std::vector<DevSim2D> sims;
    std::vector<DevTile> tiles;
    int fp64 = -1;
    for (casimir_request *r : c->active) {
        casimir_plan_t *P = r->plan;
        if (fp64 < 0) fp64 = P->fp64;
        int base = (int)sims.size();
        const PlanData &D = P->data;
        double sg = D.prob.sigma, dt = D.dt, dx = D.dx;
        for (size_t s = 0; s < P->sims.size(); ++s) {
            const HostSim &hs = P->sims[s];
            DevSim2D d{};
            d.fields = (char *)r->block + hs.field_off * P->rsize;
            d.mat = P->dev.mat + P->mat_off[hs.geo];
            d.coef = (char *)P->dev.coef + P->coef_off[hs.geo] * P->rsize;
            d.gw = P->dev.gw;
            d.acc = r->acc + s;
            d.tail = r->tail + s;
            d.s0 = r->s0;
            d.nx = hs.nx;
            d.ny = hs.ny;
            d.T = D.prob.n_steps;
            d.tail_from = D.prob.n_steps - std::max(1, D.prob.n_steps / 8);
            d.second_u = hs.second_u;
            d.a = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt);
            d.bf = dt / (1.0 + 0.5 * sg * dt) / dx;
            d.hf = dt / dx;
            sims.push_back(d);
            for (int t = hs.tile0; t < hs.tile0 + hs.ntile; ++t) {
                const HostTile &ht = P->tiles[t];
                tiles.push_back(DevTile{base + (int)s, ht.i0, ht.j0, ht.ne, P->dev.ents + ht.ent0});
            }
        }
    }
    if (sims.size() > c->sims_cap) {
        dev_free(c, c->d_sims);
        size_t cap = std::max<size_t>(sims.size(), 2 * c->sims_cap);
        void *p;
        int rc = dev_alloc(c, cap * sizeof(DevSim2D), &p);
        if (rc) return rc;
        c->d_sims = (DevSim2D *)p;
        c->sims_cap = cap;
    }
    if (tiles.size() > c->tiles_cap) {
        dev_free(c, c->d_tiles);
        size_t cap = std::max<size_t>(tiles.size(), 2 * c->tiles_cap);
        void *p;
        int rc = dev_alloc(c, cap * sizeof(DevTile), &p);
        if (rc) return rc;
        c->d_tiles = (DevTile *)p;
        c->tiles_cap = cap;
    }
    if (!sims.empty()) CUDA_TRY(cudaMemcpyAsync(c->d_sims, sims.data(), sims.size() * sizeof(DevSim2D), cudaMemcpyHostToDevice, c->stream));
    if (!tiles.empty()) CUDA_TRY(cudaMemcpyAsync(c->d_tiles, tiles.data(), tiles.size() * sizeof(DevTile), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));   // host vectors die here
    c->ntiles = (int)tiles.size();
    c->fp64_active = fp64;
    drop_graphs(c);
    c->dirty = false;
    return CASIMIR_OK;
}

// Launch `k` consecutive steps (as a cached CUDA graph) and advance the launch counter.
static int run_chunk(casimir_ctx *c, int k)
{
    auto it = c->graphs.find(k);
    if (it == c->graphs.end()) {
        cudaGraph_t g;
        CUDA_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        for (int j = 0; j < k; ++j) launch_step2d(c->fp64_active, c->d_sims, c->d_tiles, c->ntiles, c->d_launch, j, c->stream);
        launch_bump(c->d_launch, k, c->stream);
        cudaError_t e = cudaStreamEndCapture(c->stream, &g);
        if (e != cudaSuccess) return fail(CASIMIR_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t ex;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(CASIMIR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        it = c->graphs.emplace(k, ex).first;
    }
    CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    CUDA_TRY(cudaGraphLaunch(it->second, c->stream));
    CUDA_TRY(cudaEventRecord(c->ev1, c->stream));
    c->h_launch += k;
    for (casimir_request *r : c->active) r->launches += k + 1;
    return CASIMIR_OK;
}

// Publish a request's result.  The state store is the last access to *r: once
// it is visible, casimir_force may release the request.
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
    if (c->dirty) {
        int rc = rebuild(c);
        if (rc) return rc;
    }
    if (c->ntiles > 0) {
        int64_t next = c->h_launch;
        int64_t rem = INT64_MAX;
        for (casimir_request *r : c->active)
            if (!r->copy_issued) rem = std::min<int64_t>(rem, r->s0 + r->plan->data.prob.n_steps - (next - 1));
        if (rem != INT64_MAX && rem > 0) {
            int k = (int)std::min<int64_t>(64, rem);
            int rc = run_chunk(c, k);
            if (rc) return rc;
            CUDA_TRY(cudaEventSynchronize(c->ev1));
            float ms = 0;
            cudaEventElapsedTime(&ms, c->ev0, c->ev1);
            c->step_ms += ms;
            c->step_launches += k;
            for (casimir_request *r : c->active) {
                int64_t n_lo = std::max<int64_t>(1, next - r->s0), n_hi = std::min<int64_t>(r->plan->data.prob.n_steps, next + k - 1 - r->s0);
                if (n_hi >= n_lo) c->cell_updates += (n_hi - n_lo + 1) * r->plan->cells;
            }
        }
    }
    bool changed = false;
    for (casimir_request *r : c->active) {
        if (r->copy_issued) continue;
        bool done = c->h_launch - 1 - r->s0 >= r->plan->data.prob.n_steps;
        bool timed_out = c->watchdog_ms > 0 && now_ms() - r->t_admit > c->watchdog_ms;
        if (done || timed_out || r->cancel) {
            size_t ns = r->plan->sims.size();
            CUDA_TRY(cudaMemcpyAsync(r->h_acc, r->acc, ns * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(cudaMemcpyAsync(r->h_acc + ns, r->tail, ns * 8, cudaMemcpyDeviceToHost, c->stream));
            if (!r->done_ev) CUDA_TRY(cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming));
            CUDA_TRY(cudaEventRecord(r->done_ev, c->stream));
            r->copy_issued = true;
            if (!done) r->status = r->cancel ? CASIMIR_ECANCELED : CASIMIR_ETIMEOUT;
            changed = true;
        }
    }
    for (size_t q = 0; q < c->active.size();) {
        casimir_request *r = c->active[q];
        if (r->copy_issued && cudaEventQuery(r->done_ev) == cudaSuccess) {
            c->active.erase(c->active.begin() + q);
            finish_request(c, r, r->status.load());
            changed = true;
        } else {
            ++q;
        }
    }
    if (changed) c->dirty = true;
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
            std::string msg = g_err;
            for (casimir_request *r : c->active) {
                dev_free(c, r->block);
                r->block = nullptr;
                r->status = rc;
                r->plan->inflight--;
                r->state = 3;
            }
            c->active.clear();
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
    auto *c = new casimir_ctx();
    c->device = device;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    c->budget = budget ? budget : (uint64_t)(0.9 * (double)fr);
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return fail(CASIMIR_ECUDA, "stream"); }
    c->own_stream = true;
    if (cudaMalloc(&c->d_launch, sizeof(int64_t)) != cudaSuccess) { cudaStreamDestroy(c->stream); delete c; return fail(CASIMIR_ENOMEM, "launch counter"); }
    cudaMemcpy(c->d_launch, &c->h_launch, sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaEventCreate(&c->ev0);
    cudaEventCreate(&c->ev1);
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
    dev_free(c, c->d_sims);
    dev_free(c, c->d_tiles);
    cudaFree(c->d_launch);
    cudaEventDestroy(c->ev0);
    cudaEventDestroy(c->ev1);
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
    if (!c->active.empty() || !c->queue.empty() || c->d_sims) return fail(CASIMIR_EBUSY, "set the allocator before the first request");
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

int casimir_plan(casimir_ctx_t *c, const casimir_problem *p, casimir_plan_t **out)
{
    if (!p || !out) return fail(CASIMIR_EINVAL, "NULL argument");
    *out = nullptr;
    auto *P = new casimir_plan_t();
    P->ctx = c;
    std::string err;
    int rc = build_plan(p, &P->data, &err);
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

int casimir_plan_get_info(const casimir_plan_t *P, casimir_plan_info *info)
{
    if (!P || !info) return fail(CASIMIR_EINVAL, "NULL argument");
    info->n_sims = (int64_t)P->sims.size();
    info->n_cells = P->cells;
    info->cell_updates = P->cells * (int64_t)P->data.prob.n_steps;
    info->device_bytes = P->table_bytes + P->request_bytes;
    info->bytes_per_update = 6 * (int64_t)P->rsize + 1;
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
    lk.unlock();
    release(r);
    if (status != CASIMIR_OK) return fail(status, status == CASIMIR_ETIMEOUT ? "watchdog stopped the run" : "request failed");
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
// Some callers may not allocate device memory at all: code running while a
// CUDA graph is being captured (cudaMalloc is not permitted inside a capture),
// hosts that hand the library a fixed memory reservation, or embedders whose
// allocator must not be re-entered from a library.  casimir_run_noalloc lets
// them run a plan without any device allocation: the fields, the simulation
// and tile tables, the copied plan tables and the launch counter all live in
// the file-scope array below, allocated once per device when the library is
// loaded and held until the process exits.
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
