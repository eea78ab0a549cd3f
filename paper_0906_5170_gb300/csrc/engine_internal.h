// Internal host-side structures shared by the executor translation units.
#pragma once
#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>

#include <array>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "casimir.h"
#include "kernels.h"
#include "plan.h"

namespace cas {
int fail(int code, const std::string &msg);
double now_ms();
size_t align256(size_t b);
}  // namespace cas

// NVTX ranges around the executor's phases (plan, upload, batch rebuild, chunk, autotune
// trials, plain runs), visible to profilers; header-only NVTX v3, inert without a tool.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess) return cas::fail(CASIMIR_ECUDA, std::string(#expr ": ") + cudaGetErrorString(e_)); \
    } while (0)

using namespace cas;

struct HostSim {
    int geo;
    int nx, ny, nz;
    int second_u;
    int full;              // six-component fields
    int march;             // two-dimensional six-component run on the march kernel (ping-pong buffers)
    int line3;             // three-dimensional run on the x-line kernel (tiles in tilesM)
    int col3;              // three-dimensional run on the column-march kernel (tiles in tilesM, ping-pong buffers)
    int cyl;               // cylindrical (r, z) run on the march kernel's cylindrical variant
    int cplx;              // complex fields (Bloch phase)
    int magnetic;
    double kzA, kzB;       // real-phase d/dz factors (two-dimensional k_z runs)
    int64_t field_off;     // element offset of this sim's block inside the request's field block
    int64_t psi_off;       // element offset of its CPML planes (full kernel, -1: none)
    int64_t lor_off;       // element offset of its Lorentz planes (full kernel, -1: none)
    int64_t fhalf, psi_half, lor_half;   // march runs: elements of one buffer of fields, psi, Lorentz planes
    int npoles = 0;        // Lorentz poles in use (6 planes each)
    int tile0, ntile;      // range in the plan's tile list (2D and march runs) or tile6 list (full)
    int tile2_0, ntile2;   // range in the plan's two-step tile list (2D)
    int ent0, nent;        // range in the plan's entry list (bucketed by tile)
    int src0, nsrc;        // range in the plan's source list
};

struct HostTile {
    int sim, i0, j0, ent0, ne;
    int variant = 0;       // march tiles: 1 = touches CPML, + 2 (4) = the most Lorentz poles of its cells is 1 (> 1)
    int z0 = 0, z1 = 0;    // column-march tiles: planes [z0, z1)
};

struct HostTile2 {
    int sim, i0, j0, ent0, ne, rp0;
    int variant = 0;       // two-step march tiles of Cartesian runs: 1 = touches CPML, + 2 = Lorentz cells
};

struct HostTile6 {
    int sim, count;
    int64_t cell0;
    int ent0, ne;
};

struct DevPlan {           // device copies of a plan's static tables (kept while the plan lives)
    uint8_t *mat = nullptr;
    void *coef = nullptr;
    double *gw = nullptr;
    DevEnt *ents = nullptr;
    DevSrc *src = nullptr;
    DevEnt6 *ents6 = nullptr;
    DevEnt *entsM = nullptr;
    DevSrc6 *src6 = nullptr;
    DevEnt *ents2 = nullptr;
    int *rowptr2 = nullptr;
    double *lor = nullptr;
    void *lorc = nullptr;
    void *pml = nullptr;
    size_t bytes = 0;
    void *block = nullptr;
};

struct casimir_ctx;

struct casimir_plan {
    casimir_ctx *ctx = nullptr;
    PlanData data;
    casimir_plan_options opts{};      // resolved execution options (no zero fields)
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
    std::vector<HostTile2> tiles2;    // multi-step kernel tiles (tile_xk(k2d) wide), entries sorted by row
    std::vector<DevEnt> ents2;
    std::vector<int> rowptr2;
    int64_t launches = 0;             // launches a request needs (ceil(T/k2d))
    int k2d = 1;                      // time steps per launch of the 2D kernel (1, 2 or 3)
    std::vector<HostTile6> tiles6;
    std::vector<HostTile> tilesM;     // march kernel strip tiles (MARCH_W x MARCH_H) with their entries
    std::vector<DevEnt> entsM;
    std::vector<DevEnt6> ents6;
    std::vector<DevSrc6> src6;
    std::vector<int64_t> lor_sites;   // per geo: (E site, present pole) pairs over the grid
    std::vector<double> lor_all;      // per geo [id][pole][6]
    std::vector<int64_t> lor_off;     // per geo, elements
    std::vector<double> lorc_all;     // per geo [id][pole][3][4] kernel Lorentz coefficients
    std::vector<int64_t> lorc_off;    // per geo, elements
    std::vector<double> pml_all;      // per geo, per PML axis [half][b, c, 1/kappa][n_a]
    std::vector<std::array<int64_t, 3>> pml_off;   // per geo and axis, elements (-1: no PML)
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
    std::string msg;          // why the request failed (the worker's error message)
    // the request's simulations run in waves (contiguous ranges in plan order)
    struct Wave {
        size_t s_begin, s_end;
        int64_t s0;            // launch index of step 0 once active
        int64_t bytes, cells;
        int state;             // 0 pending, 1 active, 2 done
    };
    std::vector<Wave> waves;
    size_t waves_done = 0;
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
    std::atomic<double> watchdog_ms{0};   // set by callers, read by the worker
    int64_t *d_launch = nullptr;
    int64_t h_launch = 1;            // index of the next launch
    // active set
    std::vector<casimir_request *> active;
    // launch groups: [0, 1] the 2D kernel in FP32 / FP64; [2 + 4*fp64 + 2*cplx + (dims == 3)]
    // the six-component kernel; [10, 11] the two-step 2D kernel in FP32 / FP64;
    // [G_MARCH + MARCH_VARIANTS * (2*fp64 + cplx) + variant] the six-component march kernel of
    // two-dimensional runs; [G_LINE3 + 2*fp64 + cplx] the x-line kernel of three-dimensional
    // runs; [G_CYL + fp64] the cylindrical march kernel
    static constexpr int G_MARCH = 12;
    static constexpr int G_LINE3 = G_MARCH + 4 * MARCH_VARIANTS;
    static constexpr int G_CYL = G_LINE3 + 4;
    static constexpr int G_T3 = G_CYL + 2;          // [G_T3 + fp64] the three-step 2D kernel
    static constexpr int G_CYL2 = G_T3 + 2;         // [G_CYL2 + fp64] the two-step cylindrical march
    // [G_COL3 + COL3_VARIANTS * (2*fp64 + cplx) + variant] the column march of 3D runs
    static constexpr int G_COL3 = G_CYL2 + 2;
    // [G_MAR2 + MAR2_VARIANTS * cplx + variant] the two-step march of Cartesian 2D runs (FP32)
    static constexpr int G_MAR2 = G_COL3 + 4 * COL3_VARIANTS;
    static constexpr int NGROUPS = G_MAR2 + 2 * MAR2_VARIANTS;
    struct Group {
        void *sims = nullptr, *tiles = nullptr;
        size_t sims_cap = 0, tiles_cap = 0;
        int ntiles = 0;
    } groups[NGROUPS];
    int ntiles = 0;                   // over all groups
    // waves: simulations are activated in groups whose field bytes fit `wave_bytes`
    // (0: a whole request at once), so that the active working set can stay in L2
    std::atomic<int64_t> wave_bytes{0};
    int64_t active_bytes = 0;
    std::vector<std::pair<casimir_request *, size_t>> active_waves;
    std::deque<std::pair<casimir_request *, size_t>> pending_waves;
    bool dirty = true;
    std::map<int, cudaGraphExec_t> graphs;    // per chunk length, for the current active set
    // statistics
    double step_ms = 0;
    int64_t step_launches = 0;
    int64_t cell_updates = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // auxiliary streams for the launch units of one step (forked and joined every step)
    static constexpr int NAUX = 6;
    cudaStream_t aux[NAUX] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[NAUX] = {};
    // worker
    std::mutex mu;
    // Held while the worker captures a chunk graph on `stream`, and by calls from other
    // threads that synchronise that stream or free device or pinned memory: an operation on
    // a stream under capture is not permitted and would invalidate the capture.
    std::mutex capture_mu;
    std::condition_variable cv;
    std::deque<casimir_request *> queue;
    std::thread worker;
    bool worker_on = false;
    bool stop = false;
    std::atomic<int> sync_busy{0};
    // autotuning: chosen options per problem class
    int autotune = 0;
    std::map<std::string, casimir_plan_options> tuned;
};


int dev_alloc(casimir_ctx *c, size_t bytes, void **out);
void make_sim2d(const casimir_plan_t *P, char *blk, double *acc, double *tail, int64_t s0, size_t s, DevSim2D *d);
void make_sim6(const casimir_plan_t *P, char *blk, double *acc, double *tail, int64_t s0, size_t s, DevSim6 *d);
int upload_plan(casimir_plan_t *P, cudaStream_t st);
void dev_free(casimir_ctx *c, void *p);
