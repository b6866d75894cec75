// C ABI of the library (declared in include/sdeb.h): argument validation,
// device buffers owned by the context, the call-order state machine and the
// kernel launches.  Every function returns a status; nothing throws.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "em_internal.h"
#include "sdeb_rtc.h"
#include "sdeb.h"

using namespace sdeb;

struct sdeb_ctx {
    sdeb_problem pb;
    int32_t units = 0;
    size_t elem = 0;          // 4 or 8
    int device = 0;
    Layout layout{1, 1};
    void *d_params = nullptr;
    size_t params_bytes = 0;
    void *d_x = nullptr;
    float *d_comp = nullptr;
    void *d_frames = nullptr;
    int64_t nframes = 0;
    void *d_ckpt = nullptr;
    float *d_ckpt_comp = nullptr;
    int64_t nckpt = 0;
    int64_t ckpt_int = 0;         // checkpoint interval kept (<= pb.ckpt_every; see checkpoint_interval)
    int32_t adj_records = SDEB_RECORDS_AUTO;  // sdeb_set_adjoint_records
    uint8_t *d_flags = nullptr;
    void *d_seg = nullptr;        // adjoint: replayed phases and normals of one segment
    void *d_gradp = nullptr;      // adjoint: per-orbit parameter gradients (shared params)
    bool params_set = false;
    int64_t k_current = 0;
    std::string err;
    RtcModule *rtc = nullptr;             // user-defined model: its run-time compiled kernel
    // ---- batch contexts (sdeb_create_batch) ----
    bool is_batch = false;
    std::vector<sdeb_problem> probs;
    std::vector<BatchInstance> inst;      // host copy of the instance table
    int64_t batch_params_bytes = 0, batch_state_elems = 0, batch_frame_elems = 0, batch_items = 0;
    std::vector<Layout> inst_layout;
    double batch_chain_frac = 0.5;        // longest chain allowed, as a fraction of the work per sub-partition
    int num_sms = 1;
    BatchInstance *d_inst = nullptr;
    BatchItem *d_items = nullptr;
    BatchTask *d_tasks = nullptr;
    int *d_head = nullptr;
    int32_t ntasks = 0, team_items = 0;
    int grid = 0;
    int grid_cap = 1;                     // resident blocks of the batch kernel on this device
    cudaStream_t capture_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool batch_done = false;
};

namespace {

thread_local std::string g_last_error;

sdeb_status fail(sdeb_ctx *ctx, sdeb_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    g_last_error = buf;
    return s;
}

sdeb_status cuda_fail(sdeb_ctx *ctx, cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(ctx, SDEB_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(ctx, SDEB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

// An NVTX range over a host call (integration, gradient, batch, moments,
// tuning), so a timeline tool shows which library call enqueued which
// kernels.  NVTX v3 is header-only: without an attached tool a range costs a
// branch.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Host-side fault injection for failure-detection tests, nothing on the
// device: SDEB_FAULT="alloc:<k>" makes the k-th allocation of a context's
// buffers in this process (counted from 0) fail as out of memory,
// "launch:<k>" makes the k-th forward launch of an integrate call
// (sdeb_integrate, sdeb_integrate_range) fail without launching; the layout
// tuner's trial launches are not counted.  Read once, at the first
// allocation or launch; any other value injects nothing.
struct FaultPlan {
    long alloc_at = -1, launch_at = -1;
    std::atomic<long> allocs{0}, launches{0};
    FaultPlan() {
        const char *v = std::getenv("SDEB_FAULT");
        if (!v) return;
        long k = -1;
        if (std::sscanf(v, "alloc:%ld", &k) == 1 && k >= 0) alloc_at = k;
        else if (std::sscanf(v, "launch:%ld", &k) == 1 && k >= 0) launch_at = k;
    }
};

FaultPlan &fault_plan() {
    static FaultPlan plan;
    return plan;
}

bool inject_alloc_fault() {
    FaultPlan &f = fault_plan();
    return f.alloc_at >= 0 && f.allocs.fetch_add(1) == f.alloc_at;
}

bool inject_launch_fault() {
    FaultPlan &f = fault_plan();
    return f.launch_at >= 0 && f.launches.fetch_add(1) == f.launch_at;
}

bool model_shape(int32_t model, int32_t n, int32_t &m, int32_t &d, int32_t &units) {
    switch (model) {
    case SDEB_KURAMOTO: m = n; d = n + 2; units = n; return true;
    case SDEB_KURAMOTO_PAPER: m = n; d = 2 * n + 1; units = n; return true;
    case SDEB_FHN_NET:
        if (n % 2) return false;
        m = n / 2; d = 6; units = n / 2; return true;
    case SDEB_OU:
    case SDEB_GBM: m = n; d = 2; units = n; return true;
    case SDEB_LINEAR_ODE: m = 0; d = 1; units = n; return true;
    default: return false;
    }
}

bool mul_ok(int64_t a, int64_t b, int64_t &out) {
    if (a < 0 || b < 0) return false;
    if (a != 0 && b > INT64_MAX / a) return false;
    out = a * b;
    return true;
}

void free_buffers(sdeb_ctx *c) {
    cudaFree(c->d_params);
    cudaFree(c->d_x);
    cudaFree(c->d_comp);
    cudaFree(c->d_frames);
    cudaFree(c->d_ckpt);
    cudaFree(c->d_ckpt_comp);
    cudaFree(c->d_flags);
    cudaFree(c->d_seg);
    cudaFree(c->d_gradp);
    c->d_seg = c->d_gradp = nullptr;
    cudaFree(c->d_inst);
    cudaFree(c->d_items);
    cudaFree(c->d_tasks);
    cudaFree(c->d_head);
    c->d_inst = nullptr;
    c->d_items = nullptr;
    c->d_tasks = nullptr;
    c->d_head = nullptr;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    c->graph = nullptr;
    c->capture_stream = nullptr;
    c->d_params = c->d_x = c->d_frames = c->d_ckpt = nullptr;
    c->d_comp = c->d_ckpt_comp = nullptr;
    c->d_flags = nullptr;
    rtc_release(c->rtc);
    c->rtc = nullptr;
}

sdeb_status validate(const sdeb_problem *pb, int32_t &units) {
    if (!pb) return fail(nullptr, SDEB_EINVAL, "problem is NULL");
    int32_t m = 0, d = 0;
    if (pb->n <= 0) return fail(nullptr, SDEB_EINVAL, "n must be positive (got %d)", pb->n);
    if (pb->model == SDEB_USER) {
        if (pb->n > SDEB_USER_MAX_N || pb->m < 0 || pb->m > SDEB_USER_MAX_M || pb->d < 0)
            return fail(nullptr, SDEB_EINVAL, "a user model needs 1 <= n <= %d, 0 <= m <= %d, d >= 0",
                        SDEB_USER_MAX_N, SDEB_USER_MAX_M);
        if (pb->flags & (SDEB_FLAG_MILSTEIN | kImplicitFlags))
            return fail(nullptr, SDEB_EUNSUPPORTED, "user models integrate by Euler-Maruyama or SDEB_FLAG_RK4");
        if (pb->ckpt_every != 0) return fail(nullptr, SDEB_EUNSUPPORTED, "user models keep no checkpoints");
        m = pb->m;
        d = pb->d;
        units = pb->n;
    } else if (!model_shape(pb->model, pb->n, m, d, units))
        return fail(nullptr, SDEB_EINVAL, "unknown model %d or n=%d invalid for it", pb->model, pb->n);
    if (pb->m != m || pb->d != d)
        return fail(nullptr, SDEB_EINVAL, "model %d with n=%d needs m=%d d=%d (got m=%d d=%d)", pb->model,
                    pb->n, m, d, pb->m, pb->d);
    if (pb->orbits <= 0) return fail(nullptr, SDEB_EINVAL, "orbits must be positive");
    if (!(pb->dt > 0.0) || !std::isfinite(pb->dt)) return fail(nullptr, SDEB_EINVAL, "dt must be positive and finite");
    if (!std::isfinite(pb->t0)) return fail(nullptr, SDEB_EINVAL, "t0 must be finite");
    if (pb->steps < 0 || pb->steps > 0xffffffffLL)
        return fail(nullptr, SDEB_EINVAL, "steps must be in [0, 2^32)");
    if (pb->stride < 1 || pb->stride > 0xffffffffLL)
        return fail(nullptr, SDEB_EINVAL, "stride must be in [1, 2^32)");
    if (pb->precision != SDEB_FP32_KAHAN && pb->precision != SDEB_FP64)
        return fail(nullptr, SDEB_EINVAL, "unknown precision %d", pb->precision);
    if (pb->ckpt_every < 0) return fail(nullptr, SDEB_EINVAL, "ckpt_every must be >= 0");
    if (pb->flags & ~(uint32_t)(SDEB_FLAG_SHARED_PARAMS | SDEB_FLAG_NO_FRAMES | kSchemeFlags))
        return fail(nullptr, SDEB_EINVAL, "unknown flag bits 0x%x", pb->flags);
    if (!scheme_flags_valid(pb->flags))
        return fail(nullptr, SDEB_EINVAL,
                    "SDEB_FLAG_MILSTEIN, SDEB_FLAG_RK4, SDEB_FLAG_IMPLICIT_EULER and SDEB_FLAG_IMPLICIT_MIDPOINT "
                    "are exclusive");
    if (pb->reserved != 0) return fail(nullptr, SDEB_EINVAL, "reserved field must be 0");
    if (pb->orbit_offset < 0 || pb->orbit_offset + pb->orbits > 0x100000000LL)
        return fail(nullptr, SDEB_EINVAL, "orbit_offset + orbits must not exceed 2^32");
    Layout l;
    if (!default_layout(units, l))
        return fail(nullptr, SDEB_EUNSUPPORTED, "more than 256 units per orbit is not supported");
    return SDEB_OK;
}

// Layouts with a forward kernel for the model (and, for the Kuramoto models,
// an adjoint kernel): the default set for every model, the tuning set for
// the phase models.
bool layout_instantiated(int32_t model, Layout l) {
    static const Layout kDefault[] = {{1, 1}, {1, 2}, {1, 4}, {1, 8}, {2, 8}, {4, 8}, {8, 8}, {16, 8}, {32, 8}};
    static const Layout kTuning[] = {{2, 4}, {4, 4}, {8, 4}, {16, 4}, {32, 4}, {4, 16}, {8, 16}};
    for (const Layout &d : kDefault)
        if (d.G == l.G && d.P == l.P) return true;
    if (model == SDEB_KURAMOTO)
        for (const Layout &d : kTuning)
            if (d.G == l.G && d.P == l.P) return true;
    return false;
}

cudaError_t launch_forward(const ForwardArgs &a, Layout l, bool fp64, cudaStream_t s) {
    if (inject_launch_fault()) return cudaErrorLaunchFailure;
    return launch_forward_any(a, l, fp64, s);
}

// ---- batch planning ---------------------------------------------------------

// Time of one step of a lane group, in ns, as measured on the 4096-instance
// workload with three resident blocks per SM (median over the tasks of each
// kind, from a per-task timeline): a packed warp with P = 8 / 4 units per
// lane 650 / 425, a 64-lane team with 4 units per lane 388, a team with 2
// units per lane 227 (128 lanes) to 249 (64).  A packed warp's step is not
// much shorter with fewer units per lane (2 and 1: 385 and 390): with other
// warps on its SM sub-partition its rate is set by the issue slots it gets,
// while a team spreads an item's units over two or four sub-partitions,
// shares its Philox blocks between lane pairs and adds its sums with one
// redux per warp instead of a five-level scan.  A single-warp item (2 units
// per lane, sums by one redux, no barrier) is taken at a team's 240.  An
// item's chain is steps x this time, its work that times the lanes it holds
// (a single-warp item holds the whole warp).
double batch_step_cost(int P, bool team) {
    if (team) return P == 4 ? 388.0 : 240.0;
    return P == 8 ? 650.0 : P == 4 ? 425.0 : 240.0;
}

// Where an item runs: a packed warp with P = 8 or 4 units per lane on
// ceil(units / P) <= 32 lanes, a warp of its own (P = 2, up to 64 units),
// or a team of 64 lanes (P = 4 for more than 64 units, P = 2 for 65 to 128)
// or 128 lanes (P = 2, more than 128 units).  An item takes the layout of
// least total work (lanes x per-step cost) among those whose sequential
// chain, steps x per-step cost, stays within chain_max, else the layout
// with the shortest chain.  A small item alone on a warp leaves lanes idle,
// but its chain is the shortest it can have, which is what the longest
// instances of small n need.
struct ItemLayout {
    int lanes = 0, P = 0;
    bool team = false;
    bool solo = false;   // a warp of its own (lanes: those holding units)
};

ItemLayout choose_item_layout(int units, uint32_t steps, double chain_max) {
    ItemLayout cand[6];
    int nc = 0;
    for (int P : {8, 4})
        if ((units + P - 1) / P <= 32) cand[nc++] = {(units + P - 1) / P, P, false, false};
    if (units <= 64) cand[nc++] = {(units + 1) / 2, 2, false, true};
    if (units > 64 && units <= 256) cand[nc++] = {64, 4, true, false};
    if (units > 64 && units <= 128) cand[nc++] = {64, 2, true, false};
    if (units > 128 && units <= 256) cand[nc++] = {128, 2, true, false};
    ItemLayout best, shortest;
    double best_work = 0.0, shortest_chain = 0.0;
    for (int c = 0; c < nc; ++c) {
        const double per_step = batch_step_cost(cand[c].P, cand[c].team);
        const double chain = (double)steps * per_step, work = chain * (cand[c].solo ? 32 : cand[c].lanes);
        if (chain <= chain_max && (best.P == 0 || work < best_work)) {
            best = cand[c];
            best_work = work;
        }
        if (shortest.P == 0 || chain < shortest_chain) {
            shortest = cand[c];
            shortest_chain = chain;
        }
    }
    return best.P != 0 ? best : shortest;
}

struct BatchPlan {
    std::vector<BatchItem> items;
    std::vector<BatchTask> tasks;
    std::vector<Layout> inst_layout;   // (lanes per item, units per lane) of every instance
    int32_t team_items = 0;
};

BatchPlan plan_batch(const std::vector<BatchInstance> &inst, double chain_frac, int num_sms) {
    double total_warp_time = 0.0;   // the whole batch in packed warps of 8 units per lane
    for (const BatchInstance &b : inst)
        total_warp_time += (double)b.steps * b.orbits * b.units * batch_step_cost(8, false) / 8.0 / 32.0;
    const double chain_max = chain_frac * total_warp_time / (4.0 * std::max(1, num_sms));
    struct Cand {
        int32_t instance, orbit;
        uint32_t steps;
        int lanes;
    };
    std::vector<Cand> packed[9];               // by units per lane (8 or 4)
    std::vector<Cand> solo;                    // single-warp items (2 units per lane)
    std::vector<Cand> team64[5], team128[5];   // by units per lane (2 or 4)
    BatchPlan plan;
    plan.inst_layout.resize(inst.size());
    for (int32_t i = 0; i < (int32_t)inst.size(); ++i) {
        const ItemLayout l = choose_item_layout(inst[i].units, inst[i].steps, chain_max);
        plan.inst_layout[(size_t)i] = {l.lanes, l.P};
        for (int64_t o = 0; o < inst[i].orbits; ++o) {
            const Cand c{i, (int32_t)o, inst[i].steps, l.lanes};
            if (l.solo) solo.push_back(c);
            else if (!l.team) packed[l.P].push_back(c);
            else if (l.lanes == 128) team128[l.P].push_back(c);
            else team64[l.P].push_back(c);
        }
    }
    struct Costed {
        BatchTask task;
        double cost;
    };
    std::vector<Costed> tasks;
    auto by_steps = [](const Cand &a, const Cand &b) { return a.steps > b.steps; };
    for (int P : {2, 4}) {
        for (const Cand &c : team128[P]) {
            BatchTask t{};
            t.kind = kBatchTeam128;
            t.team_p = P;
            t.item[0] = (int32_t)plan.items.size();
            t.item[1] = -1;
            plan.items.push_back({c.instance, c.orbit});
            tasks.push_back({t, (double)c.steps * batch_step_cost(P, true)});
            ++plan.team_items;
        }
        std::vector<Cand> &v = team64[P];
        std::stable_sort(v.begin(), v.end(), by_steps);
        for (size_t q = 0; q < v.size(); q += 2) {
            BatchTask t{};
            t.kind = kBatchTeam64;
            t.team_p = P;
            t.item[0] = (int32_t)plan.items.size();
            plan.items.push_back({v[q].instance, v[q].orbit});
            t.item[1] = -1;
            if (q + 1 < v.size()) {
                t.item[1] = (int32_t)plan.items.size();
                plan.items.push_back({v[q + 1].instance, v[q + 1].orbit});
            }
            tasks.push_back({t, (double)v[q].steps * batch_step_cost(P, true)});
            plan.team_items += t.item[1] >= 0 ? 2 : 1;
        }
    }
    // Packed warps: items sorted by steps are cut into buckets whose step
    // counts lie within a factor kBucket (a warp steps until its longest
    // item ends), and each bucket is packed first-fit by decreasing lanes.
    const double kBucket = 1.2;
    struct CostedWarp {
        BatchWarpTask wt;
        double cost;
    };
    std::vector<CostedWarp> warps;
    for (int P : {8, 4}) {
        std::vector<Cand> &v = packed[P];
        std::stable_sort(v.begin(), v.end(), by_steps);
        for (size_t b0 = 0; b0 < v.size();) {
            size_t b1 = b0;
            while (b1 < v.size() && (double)v[b1].steps * kBucket >= (double)v[b0].steps) ++b1;
            std::vector<Cand> bucket(v.begin() + (std::ptrdiff_t)b0, v.begin() + (std::ptrdiff_t)b1);
            std::stable_sort(bucket.begin(), bucket.end(), [](const Cand &a, const Cand &b) { return a.lanes > b.lanes; });
            std::vector<std::vector<Cand>> bins;
            std::vector<int> used;
            for (const Cand &c : bucket) {
                size_t w = 0;
                while (w < bins.size() && used[w] + c.lanes > 32) ++w;
                if (w == bins.size()) {
                    bins.emplace_back();
                    used.push_back(0);
                }
                bins[w].push_back(c);
                used[w] += c.lanes;
            }
            for (const std::vector<Cand> &bin : bins) {
                BatchWarpTask wt{};
                wt.p = (int16_t)P;
                wt.first = (int32_t)plan.items.size();
                wt.count = (int16_t)bin.size();
                wt.kmax = 0;
                for (const Cand &c : bin) {
                    plan.items.push_back({c.instance, c.orbit});
                    wt.kmax = std::max(wt.kmax, c.steps);
                }
                warps.push_back({wt, (double)wt.kmax * batch_step_cost(P, false)});
            }
            b0 = b1;
        }
    }
    for (const Cand &c : solo) {
        BatchWarpTask wt{};
        wt.p = 2;
        wt.first = (int32_t)plan.items.size();
        wt.count = 1;
        wt.kmax = c.steps;
        plan.items.push_back({c.instance, c.orbit});
        warps.push_back({wt, (double)c.steps * batch_step_cost(2, false)});
    }
    std::stable_sort(warps.begin(), warps.end(), [](const CostedWarp &a, const CostedWarp &b) { return a.cost > b.cost; });
    for (size_t w = 0; w < warps.size(); w += 4) {
        BatchTask t{};
        t.kind = kBatchWarps;
        t.item[0] = t.item[1] = -1;
        double cost = 0.0;
        for (size_t q = 0; q < 4 && w + q < warps.size(); ++q) {
            t.warp[q] = warps[w + q].wt;
            cost = std::max(cost, warps[w + q].cost);
        }
        tasks.push_back({t, cost});
    }
    std::stable_sort(tasks.begin(), tasks.end(), [](const Costed &a, const Costed &b) { return a.cost > b.cost; });
    for (const Costed &c : tasks) plan.tasks.push_back(c.task);
    return plan;
}

// Upload a plan into the context's tables (sized for the largest plan).
sdeb_status upload_plan(sdeb_ctx *c, const BatchPlan &plan) {
    cudaFree(c->d_items);
    cudaFree(c->d_tasks);
    c->d_items = nullptr;
    c->d_tasks = nullptr;
    cudaError_t e = cudaMalloc((void **)&c->d_items, sizeof(BatchItem) * std::max<size_t>(1, plan.items.size()));
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_tasks, sizeof(BatchTask) * std::max<size_t>(1, plan.tasks.size()));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_items, plan.items.data(), sizeof(BatchItem) * plan.items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_tasks, plan.tasks.data(), sizeof(BatchTask) * plan.tasks.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(c, e, "batch plan upload");
    }
    c->ntasks = (int32_t)plan.tasks.size();
    c->team_items = plan.team_items;
    c->inst_layout = plan.inst_layout;
    c->grid = std::max(1, std::min<int>(c->ntasks, c->grid_cap));
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    return SDEB_OK;
}

BatchArgs batch_args(const sdeb_ctx *c, void *x, float *comp, void *frames, uint8_t *flags) {
    BatchArgs a{};
    a.inst = c->d_inst;
    a.items = c->d_items;
    a.tasks = c->d_tasks;
    a.ntasks = c->ntasks;
    a.head = c->d_head;
    a.params = c->d_params;
    a.x = x;
    a.comp = comp;
    a.frames = frames;
    a.flags = flags;
    a.keys = philox_key_schedule(c->pb.seed);
    a.ninst = (int32_t)c->inst.size();
    a.nitems = c->batch_items;
    a.state_elems = c->batch_state_elems;
    a.frame_elems = c->batch_frame_elems;
    a.param_elems = c->batch_params_bytes / (int64_t)c->elem;
    a.check = check_word();
    return a;
}

sdeb_status integrate_batch(sdeb_ctx *c, cudaStream_t s) {
    NvtxRange nvtx_range("sdeb_integrate (batch)");
    if (!c->params_set) return fail(c, SDEB_ESTATE, "sdeb_set_params has not been called");
    if (c->batch_done) return fail(c, SDEB_ESTATE, "batch already integrated; call sdeb_set_params to rerun");
    cudaError_t e = cudaSuccess;
    if (c->graph == nullptr) {
        // one graph: reset the queue head, run the persistent kernel
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaMemsetAsync(c->d_head, 0, sizeof(int), c->capture_stream);
            if (e1 == cudaSuccess)
                e1 = launch_batch(batch_args(c, c->d_x, c->d_comp, c->d_frames, c->d_flags), c->grid,
                                  c->pb.precision == SDEB_FP64, c->capture_stream);
            e = cudaStreamEndCapture(c->capture_stream, &g);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->graph = nullptr;
            return cuda_fail(c, e, "batch graph capture");
        }
    }
    e = cudaGraphLaunch(c->graph, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(c, e, "batch graph launch");
    }
    c->batch_done = true;
    c->k_current = c->pb.steps;
    return SDEB_OK;
}

// Times the whole batch for each candidate plan -- chain budget (a fraction
// of the average work per SM sub-partition) x resident blocks per SM (fewer
// resident warps leave the long chains more issue slots) -- on private
// copies of the state, without frames, and keeps the fastest.
sdeb_status autotune_batch(sdeb_ctx *c, cudaStream_t s) {
    if (!c->params_set || c->batch_done)
        return fail(c, SDEB_ESTATE, "call sdeb_autotune after sdeb_set_params and before integrating");
    const bool fp64 = c->pb.precision == SDEB_FP64;
    const size_t sb = (size_t)c->batch_state_elems * c->elem;
    void *tx = nullptr;
    float *tc = nullptr;
    uint8_t *tf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&tx, sb);
    if (e == cudaSuccess && !fp64) e = cudaMalloc((void **)&tc, (size_t)c->batch_state_elems * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&tf, (size_t)c->batch_items);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double best_frac = c->batch_chain_frac;
    int best_grid = c->grid_cap;
    float best_ms = 1e30f;
    bool first = true;
    const int cap = c->grid_cap;
    for (double frac : {0.125, 0.18, 0.25, 0.35, 0.5, 0.7, 1.0, 2.0})
      for (int per_sm : {2, 3, 4, 5}) {
        if (e != cudaSuccess) break;
        c->grid_cap = std::min(cap, per_sm * c->num_sms);
        if (upload_plan(c, plan_batch(c->inst, frac, c->num_sms)) != SDEB_OK) {
            e = cudaErrorUnknown;
            break;
        }
        float ms = 0.0f;
        for (int rep = 0; rep < (first ? 2 : 1) && e == cudaSuccess; ++rep) {
            e = cudaMemcpyAsync(tx, c->d_x, sb, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess && tc) e = cudaMemsetAsync(tc, 0, (size_t)c->batch_state_elems * 4, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_head, 0, sizeof(int), s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) e = launch_batch(batch_args(c, tx, tc, nullptr, tf), c->grid, fp64, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        }
        first = false;
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best_frac = frac;
            best_grid = c->grid_cap;
        }
      }
    c->grid_cap = best_grid;
    cudaFree(tx);
    cudaFree(tc);
    cudaFree(tf);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(c, e, "batch autotune");
    }
    c->batch_chain_frac = best_frac;
    return upload_plan(c, plan_batch(c->inst, best_frac, c->num_sms));
}

// Validates the problems of a batch and lays out their instances in the
// concatenated buffers (host only, no CUDA call).
struct BatchLayoutSums {
    int64_t p_off = 0, x_off = 0, f_off = 0, o_off = 0;
    int32_t max_n = 0;
    int64_t max_steps = 0;
};

sdeb_status build_batch_instances(const sdeb_problem *pbs, int32_t count, std::vector<BatchInstance> &inst,
                                  BatchLayoutSums &sums) {
    if (!pbs || count <= 0) return fail(nullptr, SDEB_EINVAL, "pbs must hold count >= 1 problems");
    inst.assign((size_t)count, BatchInstance{});
    int64_t &p_off = sums.p_off, &x_off = sums.x_off, &f_off = sums.f_off, &o_off = sums.o_off;
    int32_t &max_n = sums.max_n;
    int64_t &max_steps = sums.max_steps;
    for (int32_t i = 0; i < count; ++i) {
        const sdeb_problem &pb = pbs[i];
        int32_t units = 0;
        sdeb_status st = validate(&pb, units);
        if (st != SDEB_OK) return fail(nullptr, st, "instance %d: %s", i, g_last_error.c_str());
        if (pb.model != SDEB_KURAMOTO)
            return fail(nullptr, SDEB_EUNSUPPORTED, "instance %d: batches run the SDEB_KURAMOTO model", i);
        if (pb.precision != pbs[0].precision || pb.seed != pbs[0].seed)
            return fail(nullptr, SDEB_EINVAL, "instance %d: precision and seed must match instance 0", i);
        if (pb.ckpt_every != 0) return fail(nullptr, SDEB_EUNSUPPORTED, "instance %d: no checkpoints in a batch", i);
        if (pb.flags & (SDEB_FLAG_RK4 | kImplicitFlags))
            return fail(nullptr, SDEB_EUNSUPPORTED, "instance %d: batches run Euler-Maruyama", i);
        if (pb.orbits > 0x7fffffffLL) return fail(nullptr, SDEB_EINVAL, "instance %d: too many orbits", i);
        const bool shared = pb.flags & SDEB_FLAG_SHARED_PARAMS;
        const bool frames = !(pb.flags & SDEB_FLAG_NO_FRAMES);
        BatchInstance &b = inst[(size_t)i];
        b.n = pb.n;
        b.units = units;
        b.d = pb.d;
        b.param_stride = shared ? 0 : pb.d;
        b.steps = (uint32_t)pb.steps;
        b.stride = (uint32_t)pb.stride;
        b.orbit_offset = (uint32_t)pb.orbit_offset;
        b.has_frames = frames ? 1u : 0u;
        b.orbits = pb.orbits;
        b.x_off = x_off;
        b.p_off = p_off;
        b.f_off = f_off;
        b.o_off = o_off;
        b.dt = pb.dt;
        p_off += (shared ? 1 : pb.orbits) * pb.d;
        x_off += pb.orbits * pb.n;
        if (frames) f_off += (pb.steps / pb.stride + 1) * pb.orbits * pb.n;
        o_off += pb.orbits;
        max_n = std::max(max_n, pb.n);
        max_steps = std::max<int64_t>(max_steps, pb.steps);
    }
    return SDEB_OK;
}

sdeb_status create_context(const sdeb_problem *pb, int32_t units, sdeb_ctx **out);

}  // namespace

namespace sdeb {
// Lets other translation units set the text sdeb_last_error(NULL) returns.
void record_error(const char *msg) { g_last_error = msg; }
}  // namespace sdeb

extern "C" {

const char *sdeb_status_string(sdeb_status s) {
    switch (s) {
    case SDEB_OK: return "ok";
    case SDEB_EINVAL: return "invalid argument";
    case SDEB_ENOMEM: return "out of memory";
    case SDEB_ECUDA: return "CUDA error";
    case SDEB_ETIMEOUT: return "device wait timed out";
    case SDEB_ESTATE: return "call order violated";
    case SDEB_EUNSUPPORTED: return "unsupported";
    case SDEB_ENONFINITE: return "non-finite state";
    case SDEB_EBOUNDS: return "bounds check failed";
    default: return "unknown status";
    }
}

const char *sdeb_last_error(const sdeb_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_last_error.c_str();
}

sdeb_status sdeb_create(const sdeb_problem *pb, sdeb_ctx **out) {
    if (!out) return fail(nullptr, SDEB_EINVAL, "out is NULL");
    *out = nullptr;
    int32_t units = 0;
    sdeb_status st = validate(pb, units);
    if (st != SDEB_OK) return st;
    if (pb->model == SDEB_USER)
        return fail(nullptr, SDEB_EINVAL, "a user-defined model needs its source: use sdeb_create_user");
    return create_context(pb, units, out);
}

sdeb_status sdeb_create_user(const sdeb_problem *pb, const char *source, sdeb_ctx **out) {
    if (!out) return fail(nullptr, SDEB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!source) return fail(nullptr, SDEB_EINVAL, "source is NULL");
    int32_t units = 0;
    sdeb_status st = validate(pb, units);
    if (st != SDEB_OK) return st;
    if (pb->model != SDEB_USER) return fail(nullptr, SDEB_EINVAL, "sdeb_create_user needs model SDEB_USER");
    RtcModule *m = nullptr;
    std::string log;
    st = rtc_build(*pb, source, &m, log);
    if (st != SDEB_OK) return fail(nullptr, st, "user model: %s", log.c_str());
    sdeb_ctx *c = nullptr;
    st = create_context(pb, units, &c);
    if (st != SDEB_OK) {
        rtc_release(m);
        return st;
    }
    c->rtc = m;
    *out = c;
    return SDEB_OK;
}

}  // extern "C"

namespace {

// Checkpoint interval of a context that keeps checkpoints for sdeb_grad.
// The adjoint replays one segment (the steps between two checkpoints) and
// keeps a record of each step for its reverse sweep.  Segments of
// kSmemSegment steps keep the records in the shared memory of the thread
// that writes and reads them; that interval is taken whenever its
// checkpoints fit a quarter of the device memory.  Otherwise the records go
// through a global buffer of 2 n + 2 elements per orbit and step; with every
// resident orbit's segment at once in flight, a segment of ckpt_every steps
// can outgrow the L2 cache and make the buffer an HBM round trip, so the
// interval is cut to ckpt_every / m (m <= 16, so at most 16x the
// checkpoints asked for) until the in-flight buffer fits 60 % of the L2.
constexpr int64_t kSmemSegment = 8;

int64_t checkpoint_interval(const sdeb_problem *pb, int32_t units, size_t elem, int device) {
    const int64_t every = pb->ckpt_every;
    const bool adjoint = every > 0 && (pb->model == SDEB_KURAMOTO || pb->model == SDEB_KURAMOTO_PAPER);
    if (!adjoint || every <= kSmemSegment) return every;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
        const double nck = (double)((pb->steps + kSmemSegment - 1) / kSmemSegment + 1);
        const double bytes = nck * (double)pb->orbits * (double)pb->n * (double)elem * (elem == 4 ? 2.0 : 1.0);
        if (bytes <= (double)total_b / 4.0) return kSmemSegment;
    } else {
        cudaGetLastError();
    }
    int l2 = 0, sms = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || l2 <= 0 || sms <= 0) {
        cudaGetLastError();
        return every;
    }
    Layout l;
    default_layout(units, l);
    const int64_t resident = std::min<int64_t>(pb->orbits, (int64_t)sms * 2048 / l.G);
    const double per_step = (double)resident * (pb->n + 1) * 2.0 * (double)elem;
    const int64_t fit = std::max<int64_t>(1, (int64_t)(0.6 * (double)l2 / per_step));
    if (fit >= every) return every;
    const int64_t m = std::min<int64_t>(16, (every + fit - 1) / fit);
    int64_t interval = (every + m - 1) / m;
    // a multiple of the FP32 forward's compensation period when possible:
    // the periods then never split at a checkpoint
    if (interval > (int64_t)kCompPeriod) interval -= interval % kCompPeriod;
    return interval;
}

sdeb_status create_context(const sdeb_problem *pb, int32_t units, sdeb_ctx **out) {
    const size_t elem = pb->precision == SDEB_FP64 ? 8 : 4;
    const bool shared = pb->flags & SDEB_FLAG_SHARED_PARAMS;
    int64_t state_elems, param_elems, frame_elems = 0, ckpt_elems = 0, seg_elems = 0, gradp_elems = 0;
    const bool adjoint = pb->ckpt_every > 0 && (pb->model == SDEB_KURAMOTO || pb->model == SDEB_KURAMOTO_PAPER);
    int device = 0;
    cudaError_t e0 = cudaGetDevice(&device);
    if (e0 != cudaSuccess) return cuda_fail(nullptr, e0, "cudaGetDevice");
    const int64_t ckpt_int = checkpoint_interval(pb, units, elem, device);
    int64_t nframes = (pb->flags & SDEB_FLAG_NO_FRAMES) ? 0 : pb->steps / pb->stride + 1;
    int64_t nckpt = ckpt_int > 0 ? (pb->steps + ckpt_int - 1) / ckpt_int + 1 : 0;
    if (!mul_ok(pb->orbits, pb->n, state_elems) || !mul_ok(shared ? 1 : pb->orbits, pb->d, param_elems) ||
        !mul_ok(nframes, state_elems, frame_elems) || !mul_ok(nckpt, state_elems, ckpt_elems) ||
        !mul_ok(adjoint ? 2 * ckpt_int : 0, state_elems + pb->orbits, seg_elems) ||
        !mul_ok(adjoint && shared ? pb->orbits : 0, pb->d, gradp_elems) ||
        frame_elems > INT64_MAX / 8 || ckpt_elems > INT64_MAX / 8 || seg_elems > INT64_MAX / 8)
        return fail(nullptr, SDEB_EINVAL, "problem size overflows");

    sdeb_ctx *c = new (std::nothrow) sdeb_ctx;
    if (!c) return fail(nullptr, SDEB_ENOMEM, "host allocation failed");
    c->pb = *pb;
    c->units = units;
    c->elem = elem;
    c->nframes = nframes;
    c->nckpt = nckpt;
    c->ckpt_int = ckpt_int;
    default_layout(units, c->layout);
    c->device = device;
    cudaError_t e = cudaSuccess;
    c->params_bytes = (size_t)param_elems * elem;
    struct {
        void **p;
        size_t bytes;
        const char *what;
    } allocs[] = {
        {&c->d_params, c->params_bytes, "parameters"},
        {&c->d_x, (size_t)state_elems * elem, "state"},
        {(void **)&c->d_comp, elem == 4 ? (size_t)state_elems * 4 : 0, "compensation"},
        {&c->d_frames, (size_t)frame_elems * elem, "frames"},
        {&c->d_ckpt, (size_t)ckpt_elems * elem, "checkpoints"},
        {(void **)&c->d_ckpt_comp, elem == 4 ? (size_t)ckpt_elems * 4 : 0, "checkpoint compensation"},
        {(void **)&c->d_flags, (size_t)pb->orbits, "flags"},
        {&c->d_seg, (size_t)seg_elems * elem, "adjoint segment buffer"},
        {&c->d_gradp, (size_t)gradp_elems * elem, "per-orbit gradients"},
    };
    for (auto &a : allocs) {
        if (a.bytes == 0) continue;
        e = inject_alloc_fault() ? cudaErrorMemoryAllocation : cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            sdeb_status s = cuda_fail(nullptr, e, a.what);
            free_buffers(c);
            delete c;
            return s;
        }
    }
    *out = c;
    return SDEB_OK;
}

}  // namespace

extern "C" {

void sdeb_destroy(sdeb_ctx *ctx) {
    if (!ctx) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    free_buffers(ctx);
    cudaSetDevice(prev);
    delete ctx;
}

// Memory kinds of the copy calls' host-side buffers (SDEB_MEM_*).
static bool mem_kind_valid(int32_t k) { return k == SDEB_MEM_HOST || k == SDEB_MEM_DEVICE || k == SDEB_MEM_HOST_ASYNC; }

// The copy of a read call to dst (SDEB_MEM_*): device to device, or to host
// memory, waited for unless SDEB_MEM_HOST_ASYNC.
static cudaError_t read_copy(void *dst, const void *src, size_t bytes, int32_t dst_kind, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes,
                                    dst_kind == SDEB_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && dst_kind == SDEB_MEM_HOST) e = cudaStreamSynchronize(s);
    return e;
}

sdeb_status sdeb_set_params(sdeb_ctx *ctx, const void *params, const void *x0, int32_t on_device,
                            void *stream) {
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (!params || !x0) return fail(ctx, SDEB_EINVAL, "params and x0 must not be NULL");
    if (!mem_kind_valid(on_device)) return fail(ctx, SDEB_EINVAL, "on_device %d is not SDEB_MEM_*", on_device);
    const cudaStream_t s = as_stream(stream);
    const cudaMemcpyKind kind = on_device == SDEB_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (ctx->is_batch) {
        const size_t sb = (size_t)ctx->batch_state_elems * ctx->elem;
        cudaError_t e = cudaMemcpyAsync(ctx->d_params, params, (size_t)ctx->batch_params_bytes, kind, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_x, x0, sb, kind, s);
        if (e == cudaSuccess && ctx->d_comp) e = cudaMemsetAsync(ctx->d_comp, 0, (size_t)ctx->batch_state_elems * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->d_flags, 0, (size_t)ctx->batch_items, s);
        if (e == cudaSuccess && on_device == SDEB_MEM_HOST) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->params_set = false;
            return cuda_fail(ctx, e, "sdeb_set_params copy");
        }
        ctx->params_set = true;
        ctx->batch_done = false;
        ctx->k_current = 0;
        return SDEB_OK;
    }
    const size_t state_bytes = (size_t)ctx->pb.orbits * ctx->pb.n * ctx->elem;
    cudaError_t e = cudaMemcpyAsync(ctx->d_params, params, ctx->params_bytes, kind, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->d_x, x0, state_bytes, kind, s);
    if (e == cudaSuccess && ctx->d_comp) e = cudaMemsetAsync(ctx->d_comp, 0, state_bytes, s);
    if (e == cudaSuccess && ctx->d_frames)
        e = cudaMemcpyAsync(ctx->d_frames, ctx->d_x, state_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && ctx->d_ckpt)
        e = cudaMemcpyAsync(ctx->d_ckpt, ctx->d_x, state_bytes, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && ctx->d_ckpt_comp) e = cudaMemsetAsync(ctx->d_ckpt_comp, 0, state_bytes, s);
    if (e == cudaSuccess && ctx->d_flags) e = cudaMemsetAsync(ctx->d_flags, 0, (size_t)ctx->pb.orbits, s);
    if (e == cudaSuccess && on_device == SDEB_MEM_HOST) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->params_set = false;
        return cuda_fail(ctx, e, "sdeb_set_params copy");
    }
    ctx->params_set = true;
    ctx->k_current = 0;
    return SDEB_OK;
}

sdeb_status sdeb_integrate_range(sdeb_ctx *ctx, int64_t k_begin, int64_t k_end, void *stream) {
    NvtxRange nvtx_range("sdeb_integrate_range");
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return fail(ctx, SDEB_EUNSUPPORTED, "a batch integrates whole horizons (sdeb_integrate)");
    if (!ctx->params_set) return fail(ctx, SDEB_ESTATE, "sdeb_set_params has not been called");
    if (k_begin != ctx->k_current)
        return fail(ctx, SDEB_ESTATE, "k_begin=%lld but the state is at step %lld", (long long)k_begin,
                    (long long)ctx->k_current);
    if (k_end < k_begin || k_end > ctx->pb.steps)
        return fail(ctx, SDEB_EINVAL, "k_end=%lld outside [k_begin, steps]", (long long)k_end);
    if (k_end == k_begin) return SDEB_OK;
    if (ctx->rtc) {
        UserArgs u{};
        u.params = ctx->d_params;
        u.param_stride = (ctx->pb.flags & SDEB_FLAG_SHARED_PARAMS) ? 0 : ctx->pb.d;
        u.x = ctx->d_x;
        u.comp = ctx->d_comp;
        u.frames = ctx->d_frames;
        u.orbits = ctx->pb.orbits;
        u.t0 = ctx->pb.t0;
        u.dt = ctx->pb.dt;
        u.k_begin = (uint32_t)k_begin;
        u.k_end = (uint32_t)k_end;
        u.stride = (uint32_t)ctx->pb.stride;
        u.orbit_offset = (uint32_t)ctx->pb.orbit_offset;
        u.flags = ctx->d_flags;
        u.keys = philox_key_schedule(ctx->pb.seed);
        u.nframes = ctx->nframes;
        u.check = check_word();
        cudaError_t e = rtc_launch(ctx->rtc, u, as_stream(stream));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "user model kernel launch");
        ctx->k_current = k_end;
        return SDEB_OK;
    }
    ForwardArgs a{};
    a.model = ctx->pb.model;
    a.n = ctx->pb.n;
    a.units = ctx->units;
    a.orbits = ctx->pb.orbits;
    a.params = ctx->d_params;
    a.param_stride = (ctx->pb.flags & SDEB_FLAG_SHARED_PARAMS) ? 0 : ctx->pb.d;
    a.x = ctx->d_x;
    a.comp = ctx->d_comp;
    a.frames = ctx->d_frames;
    a.nframes = ctx->nframes;
    a.ckpt = ctx->d_ckpt;
    a.ckpt_comp = ctx->d_ckpt_comp;
    a.ckpt_every = (uint32_t)ctx->ckpt_int;
    a.k_begin = (uint32_t)k_begin;
    a.k_end = (uint32_t)k_end;
    a.stride = (uint32_t)ctx->pb.stride;
    a.orbit_offset = (uint32_t)ctx->pb.orbit_offset;
    a.dt = ctx->pb.dt;
    a.flags = ctx->d_flags;
    a.keys = philox_key_schedule(ctx->pb.seed);
    a.nckpt = ctx->nckpt;
    a.check = check_word();
    a.milstein = (ctx->pb.flags & SDEB_FLAG_MILSTEIN) ? 1 : 0;
    a.rk4 = (ctx->pb.flags & SDEB_FLAG_RK4) ? 1 : 0;
    a.implicit = implicit_kind(ctx->pb.flags);
    cudaError_t e = launch_forward(a, ctx->layout, ctx->pb.precision == SDEB_FP64, as_stream(stream));
    if (e == cudaErrorNotSupported)
        return fail(ctx, SDEB_EUNSUPPORTED, "no kernel for model %d with layout G=%d P=%d", a.model,
                    ctx->layout.G, ctx->layout.P);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "forward kernel launch");
    ctx->k_current = k_end;
    return SDEB_OK;
}

sdeb_status sdeb_integrate(sdeb_ctx *ctx, void *stream) {
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return integrate_batch(ctx, as_stream(stream));
    if (ctx->params_set && ctx->k_current != 0)
        return fail(ctx, SDEB_ESTATE, "state is at step %lld; call sdeb_set_params to restart",
                    (long long)ctx->k_current);
    return sdeb_integrate_range(ctx, 0, ctx->pb.steps, stream);
}

sdeb_status sdeb_read_orbits(sdeb_ctx *ctx, void *dst, size_t dst_bytes, int64_t frame_begin,
                             int64_t frame_count, int32_t dst_on_device, void *stream) {
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return fail(ctx, SDEB_EUNSUPPORTED, "use sdeb_batch_read on a batch");
    if (!dst) return fail(ctx, SDEB_EINVAL, "dst is NULL");
    if (!mem_kind_valid(dst_on_device)) return fail(ctx, SDEB_EINVAL, "dst_on_device %d is not SDEB_MEM_*", dst_on_device);
    if (!ctx->d_frames) return fail(ctx, SDEB_ESTATE, "context was created without frames");
    if (!ctx->params_set) return fail(ctx, SDEB_ESTATE, "sdeb_set_params has not been called");
    if (frame_begin < 0 || frame_count < 0 || frame_begin + frame_count > ctx->nframes)
        return fail(ctx, SDEB_EINVAL, "frames [%lld, %lld) outside [0, %lld)", (long long)frame_begin,
                    (long long)(frame_begin + frame_count), (long long)ctx->nframes);
    if (frame_count > 0 && (frame_begin + frame_count - 1) * ctx->pb.stride > ctx->k_current)
        return fail(ctx, SDEB_ESTATE, "frame %lld is past the current step %lld",
                    (long long)(frame_begin + frame_count - 1), (long long)ctx->k_current);
    const size_t frame_bytes = (size_t)ctx->pb.orbits * ctx->pb.n * ctx->elem;
    if (dst_bytes != frame_bytes * (size_t)frame_count)
        return fail(ctx, SDEB_EINVAL, "dst_bytes=%zu, expected %zu", dst_bytes, frame_bytes * (size_t)frame_count);
    if (frame_count == 0) return SDEB_OK;
    const cudaStream_t s = as_stream(stream);
    cudaError_t e = read_copy(dst, static_cast<char *>(ctx->d_frames) + frame_bytes * frame_begin, dst_bytes,
                              dst_on_device, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "sdeb_read_orbits copy");
    }
    return SDEB_OK;
}

sdeb_status sdeb_read_final(sdeb_ctx *ctx, void *dst, size_t dst_bytes, int32_t dst_on_device, void *stream) {
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return fail(ctx, SDEB_EUNSUPPORTED, "use sdeb_batch_read on a batch");
    if (!dst) return fail(ctx, SDEB_EINVAL, "dst is NULL");
    if (!mem_kind_valid(dst_on_device)) return fail(ctx, SDEB_EINVAL, "dst_on_device %d is not SDEB_MEM_*", dst_on_device);
    if (!ctx->params_set) return fail(ctx, SDEB_ESTATE, "sdeb_set_params has not been called");
    const size_t bytes = (size_t)ctx->pb.orbits * ctx->pb.n * ctx->elem;
    if (dst_bytes != bytes) return fail(ctx, SDEB_EINVAL, "dst_bytes=%zu, expected %zu", dst_bytes, bytes);
    const cudaStream_t s = as_stream(stream);
    cudaError_t e;
    if (!ctx->rtc && delayed_compensation(ctx->pb.model, ctx->pb.precision, ctx->pb.flags)) {
        // the stored pair (x, c) of a resumable state: its value is x - c
        const int64_t count = ctx->pb.orbits * ctx->pb.n;
        if (dst_on_device == SDEB_MEM_DEVICE) {
            e = launch_state_value(static_cast<const float *>(ctx->d_x), ctx->d_comp, count, static_cast<float *>(dst), s);
        } else {
            void *tmp = nullptr;
            e = cudaMallocAsync(&tmp, bytes, s);
            if (e == cudaSuccess)
                e = launch_state_value(static_cast<const float *>(ctx->d_x), ctx->d_comp, count, static_cast<float *>(tmp), s);
            if (e == cudaSuccess) e = read_copy(dst, tmp, bytes, dst_on_device, s);
            if (tmp) {
                cudaError_t ef = cudaFreeAsync(tmp, s);
                if (e == cudaSuccess) e = ef;
            }
        }
    } else {
        e = read_copy(dst, ctx->d_x, bytes, dst_on_device, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "sdeb_read_final copy");
    }
    return SDEB_OK;
}

sdeb_status sdeb_frame_moments(sdeb_ctx *ctx, int64_t frame_begin, int64_t frame_count, double *mom,
                               size_t mom_bytes, double *rmom, size_t rmom_bytes, int32_t dst_on_device,
                               void *stream) {
    NvtxRange nvtx_range("sdeb_frame_moments");
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return fail(ctx, SDEB_EUNSUPPORTED, "moments are per context, not per batch");
    if (!mom && !rmom) return fail(ctx, SDEB_EINVAL, "mom and rmom are both NULL");
    if (!mem_kind_valid(dst_on_device)) return fail(ctx, SDEB_EINVAL, "dst_on_device %d is not SDEB_MEM_*", dst_on_device);
    const bool phase = ctx->pb.model == SDEB_KURAMOTO || ctx->pb.model == SDEB_KURAMOTO_PAPER;
    if (rmom && !phase) return fail(ctx, SDEB_EUNSUPPORTED, "the order parameter needs a phase model");
    if (!ctx->d_frames) return fail(ctx, SDEB_ESTATE, "context was created without frames");
    if (!ctx->params_set) return fail(ctx, SDEB_ESTATE, "sdeb_set_params has not been called");
    if (frame_begin < 0 || frame_count < 0 || frame_begin + frame_count > ctx->nframes)
        return fail(ctx, SDEB_EINVAL, "frames [%lld, %lld) outside [0, %lld)", (long long)frame_begin,
                    (long long)(frame_begin + frame_count), (long long)ctx->nframes);
    if (frame_count > 0 && (frame_begin + frame_count - 1) * ctx->pb.stride > ctx->k_current)
        return fail(ctx, SDEB_ESTATE, "frame %lld is past the current step %lld",
                    (long long)(frame_begin + frame_count - 1), (long long)ctx->k_current);
    const int n = ctx->pb.n;
    if (mom && mom_bytes != (size_t)frame_count * n * 2 * sizeof(double))
        return fail(ctx, SDEB_EINVAL, "mom_bytes=%zu, expected %zu", mom_bytes,
                    (size_t)frame_count * n * 2 * sizeof(double));
    if (rmom && rmom_bytes != (size_t)frame_count * 2 * sizeof(double))
        return fail(ctx, SDEB_EINVAL, "rmom_bytes=%zu, expected %zu", rmom_bytes,
                    (size_t)frame_count * 2 * sizeof(double));
    if (frame_count == 0) return SDEB_OK;
    const cudaStream_t s = as_stream(stream);
    const bool fp64 = ctx->pb.precision == SDEB_FP64;
    const bool to_host = dst_on_device != SDEB_MEM_DEVICE;
    const FrameMomentsPlan plan = frame_moments_plan(ctx->pb.orbits, n, frame_count);
    void *scratch = nullptr;
    cudaError_t e = cudaMallocAsync(&scratch, plan.partial_bytes + (to_host ? plan.out_bytes : 0), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "sdeb_frame_moments scratch");
    }
    double *stage = to_host ? reinterpret_cast<double *>(static_cast<char *>(scratch) + plan.partial_bytes) : nullptr;
    for (int64_t f = 0; f < frame_count && e == cudaSuccess; f += plan.frames_per_pass) {
        const int64_t cnt = std::min<int64_t>(plan.frames_per_pass, frame_count - f);
        double *st = mom ? (to_host ? stage : mom + f * n * 2) : nullptr;
        double *rt = rmom ? (to_host ? stage + cnt * n * 2 : rmom + f * 2) : nullptr;
        e = launch_frame_moments_pass(ctx->d_frames, fp64, ctx->pb.orbits, n, frame_begin + f, cnt, ctx->nframes, plan,
                                      scratch,
                                      st, rt, s);
        if (e == cudaSuccess && to_host && mom)
            e = cudaMemcpyAsync(mom + f * n * 2, st, (size_t)cnt * n * 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && to_host && rmom)
            e = cudaMemcpyAsync(rmom + f * 2, rt, (size_t)cnt * 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    }
    cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = ef;
    if (e == cudaSuccess && dst_on_device == SDEB_MEM_HOST) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "sdeb_frame_moments");
    }
    return SDEB_OK;
}

sdeb_status sdeb_orbit_flags(sdeb_ctx *ctx, uint8_t *dst, void *stream) {
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (!dst) return fail(ctx, SDEB_EINVAL, "dst is NULL");
    if (!ctx->params_set) return fail(ctx, SDEB_ESTATE, "sdeb_set_params has not been called");
    const cudaStream_t s = as_stream(stream);
    cudaError_t e = cudaMemcpyAsync(dst, ctx->d_flags, (size_t)ctx->pb.orbits, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "sdeb_orbit_flags copy");
    }
    return SDEB_OK;
}

sdeb_status sdeb_set_layout(sdeb_ctx *ctx, int32_t lanes_per_orbit, int32_t units_per_lane) {
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return fail(ctx, SDEB_EUNSUPPORTED, "a batch chooses layouts per instance (sdeb_autotune)");
    if (ctx->rtc) return fail(ctx, SDEB_EUNSUPPORTED, "a user model runs one thread per orbit");
    const int G = lanes_per_orbit, P = units_per_lane;
    if (!(G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32) || P < 1 || P > 16 ||
        (G > 1 && P % 4 != 0) || (int64_t)G * P < ctx->units)
        return fail(ctx, SDEB_EINVAL, "layout G=%d P=%d invalid for %d units", G, P, ctx->units);
    if (ctx->params_set && ctx->k_current != 0)
        return fail(ctx, SDEB_ESTATE, "set the layout before integrating");
    if (!layout_instantiated(ctx->pb.model, {G, P}))
        return fail(ctx, SDEB_EUNSUPPORTED, "no kernel for model %d with G=%d P=%d", ctx->pb.model, G, P);
    ctx->layout = {G, P};
    return SDEB_OK;
}

sdeb_status sdeb_autotune(sdeb_ctx *ctx, int64_t trial_steps, void *stream) {
    NvtxRange nvtx_range("sdeb_autotune");
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return autotune_batch(ctx, as_stream(stream));
    if (!ctx->params_set || ctx->k_current != 0)
        return fail(ctx, SDEB_ESTATE, "call sdeb_autotune after sdeb_set_params and before integrating");
    if (ctx->rtc) return SDEB_OK;  // a user model has one kernel shape: one thread per orbit
    // A context that keeps checkpoints for sdeb_grad is tuned for forward +
    // adjoint, each timed per step: the forward over trial_steps steps, the
    // adjoint over whole segments covering at least 64 steps (at most 1024)
    // from checkpoints that are copies of checkpoint 0 (the one
    // sdeb_set_params has written; the integration overwrites them).
    const bool tune_adjoint = ctx->d_seg != nullptr && !(ctx->pb.flags & (kSchemeFlags));
    if (trial_steps <= 0) trial_steps = 64;
    if (tune_adjoint) trial_steps = std::min<int64_t>(std::max<int64_t>(trial_steps, 64), 1024);
    if (trial_steps > ctx->pb.steps) trial_steps = ctx->pb.steps;
    if (trial_steps == 0) return SDEB_OK;
    int64_t adj_steps = 0;
    if (tune_adjoint) {
        const int64_t segs = std::max<int64_t>(1, std::min<int64_t>(1024, std::max<int64_t>(64, ctx->ckpt_int)) /
                                                      ctx->ckpt_int);
        adj_steps = std::min<int64_t>(segs * ctx->ckpt_int, ctx->pb.steps);
    }
    static const Layout kCandidates[] = {{1, 1}, {1, 2}, {1, 4}, {1, 8}, {2, 4}, {2, 8}, {4, 4}, {4, 8}, {4, 16},
                                         {8, 4}, {8, 8}, {8, 16}, {16, 4}, {16, 8}, {32, 4}, {32, 8}};
    const cudaStream_t s = as_stream(stream);
    const size_t state_bytes = (size_t)ctx->pb.orbits * ctx->pb.n * ctx->elem;
    void *tx = nullptr;
    float *tc = nullptr;
    uint8_t *tf = nullptr;
    void *t_dl = nullptr, *t_dp = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&tx, state_bytes);
    if (e == cudaSuccess && ctx->d_comp) e = cudaMalloc((void **)&tc, (size_t)ctx->pb.orbits * ctx->pb.n * 4);
    if (e == cudaSuccess) e = cudaMalloc((void **)&tf, (size_t)ctx->pb.orbits);
    if (e == cudaSuccess && tune_adjoint) e = cudaMalloc(&t_dl, state_bytes);
    if (e == cudaSuccess && tune_adjoint) e = cudaMemsetAsync(t_dl, 0, state_bytes, s);
    if (e == cudaSuccess && tune_adjoint) e = cudaMalloc(&t_dp, (size_t)ctx->pb.orbits * ctx->pb.d * ctx->elem);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    Layout best = ctx->layout;
    float best_ms = 1e30f;
    for (const Layout &l : kCandidates) {
        if (e != cudaSuccess) break;
        // lanes x units must cover the orbit and waste at most half of it
        const int64_t cover = (int64_t)l.G * l.P;
        if (cover < ctx->units || (cover > 4 && cover > 2 * (int64_t)ctx->units)) continue;
        if (!layout_instantiated(ctx->pb.model, l)) continue;
        ForwardArgs a{};
        a.model = ctx->pb.model;
        a.n = ctx->pb.n;
        a.units = ctx->units;
        a.orbits = ctx->pb.orbits;
        a.params = ctx->d_params;
        a.param_stride = (ctx->pb.flags & SDEB_FLAG_SHARED_PARAMS) ? 0 : ctx->pb.d;
        a.x = tx;
        a.comp = tc;
        a.k_begin = 0;
        a.k_end = (uint32_t)trial_steps;
        a.stride = (uint32_t)ctx->pb.stride;
        a.orbit_offset = (uint32_t)ctx->pb.orbit_offset;
        a.dt = ctx->pb.dt;
        a.flags = tf;
        a.keys = philox_key_schedule(ctx->pb.seed);
        a.nckpt = ctx->nckpt;
        a.check = check_word();
        a.milstein = (ctx->pb.flags & SDEB_FLAG_MILSTEIN) ? 1 : 0;
        a.rk4 = (ctx->pb.flags & SDEB_FLAG_RK4) ? 1 : 0;
        a.implicit = implicit_kind(ctx->pb.flags);
        float ms = 0.0f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run warms up
            e = cudaMemcpyAsync(tx, ctx->d_x, state_bytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess && tc) e = cudaMemsetAsync(tc, 0, (size_t)ctx->pb.orbits * ctx->pb.n * 4, s);
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            // trial launches are not counted by the fault injection (SDEB_FAULT)
            if (e == cudaSuccess) e = launch_forward_any(a, l, ctx->pb.precision == SDEB_FP64, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        }
        if (e == cudaSuccess && tune_adjoint) {
            AdjointArgs g{};
            g.model = ctx->pb.model;
            g.n = ctx->pb.n;
            g.units = ctx->units;
            g.d = ctx->pb.d;
            g.orbits = ctx->pb.orbits;
            g.params = ctx->d_params;
            g.param_stride = a.param_stride;
            g.ckpt = ctx->d_ckpt;
            g.ckpt_comp = ctx->d_ckpt_comp;
            g.ckpt_every = (uint32_t)ctx->ckpt_int;
            g.steps = (uint32_t)adj_steps;
            g.orbit_offset = a.orbit_offset;
            g.dt = ctx->pb.dt;
            g.seg = ctx->d_seg;
            g.dL_dxK = t_dl;
            g.dL_dp = t_dp;
            g.keys = a.keys;
            g.nckpt = ctx->nckpt;
            g.check = a.check;
            g.records = ctx->adj_records;
            float ms_adj = 0.0f;
            // checkpoints 1 .. of the trial: copies of checkpoint 0
            const int64_t ck_used = (adj_steps + ctx->ckpt_int - 1) / ctx->ckpt_int;
            for (int64_t c = 1; c < ck_used && e == cudaSuccess; ++c) {
                e = cudaMemcpyAsync(static_cast<char *>(ctx->d_ckpt) + c * state_bytes, ctx->d_ckpt, state_bytes,
                                    cudaMemcpyDeviceToDevice, s);
                if (e == cudaSuccess && ctx->d_ckpt_comp)
                    e = cudaMemsetAsync(reinterpret_cast<char *>(ctx->d_ckpt_comp) + c * ((size_t)ctx->pb.orbits *
                                        ctx->pb.n * 4), 0, (size_t)ctx->pb.orbits * ctx->pb.n * 4, s);
            }
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                e = cudaEventRecord(e0, s);
                if (e == cudaSuccess) e = launch_adjoint(g, l, ctx->pb.precision == SDEB_FP64, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_adj, e0, e1);
            }
            ms = ms / (float)trial_steps + ms_adj / (float)adj_steps;   // per step, forward + adjoint
        }
        if (e == cudaErrorNotSupported) {
            e = cudaSuccess;
            cudaGetLastError();
            continue;
        }
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = l;
        }
    }
    cudaFree(tx);
    cudaFree(tc);
    cudaFree(tf);
    cudaFree(t_dl);
    cudaFree(t_dp);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "sdeb_autotune");
    }
    ctx->layout = best;
    return SDEB_OK;
}

sdeb_status sdeb_set_adjoint_records(sdeb_ctx *ctx, int32_t mode) {
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return fail(ctx, SDEB_EINVAL, "a batch has no adjoint");
    if (mode != SDEB_RECORDS_AUTO && mode != SDEB_RECORDS_GLOBAL && mode != SDEB_RECORDS_SHARED)
        return fail(ctx, SDEB_EINVAL, "records mode %d is not SDEB_RECORDS_AUTO, _GLOBAL or _SHARED", mode);
    ctx->adj_records = mode;
    return SDEB_OK;
}

sdeb_status sdeb_get_checkpoint_interval(const sdeb_ctx *ctx, int64_t *steps) {
    if (!ctx || !steps) return fail(nullptr, SDEB_EINVAL, "ctx and steps must not be NULL");
    *steps = ctx->is_batch ? 0 : ctx->ckpt_int;
    return SDEB_OK;
}

sdeb_status sdeb_get_layout(const sdeb_ctx *ctx, int32_t *lanes_per_orbit, int32_t *units_per_lane) {
    if (!ctx || !lanes_per_orbit || !units_per_lane) return fail(nullptr, SDEB_EINVAL, "NULL argument");
    *lanes_per_orbit = ctx->layout.G;
    *units_per_lane = ctx->layout.P;
    return SDEB_OK;
}

sdeb_status sdeb_frames_device_ptr(sdeb_ctx *ctx, void **ptr, size_t *bytes) {
    if (!ctx || !ptr || !bytes) return fail(ctx, SDEB_EINVAL, "NULL argument");
    *ptr = ctx->d_frames;
    if (ctx->is_batch)
        *bytes = ctx->d_frames ? (size_t)ctx->batch_frame_elems * ctx->elem : 0;
    else
        *bytes = ctx->d_frames ? (size_t)ctx->nframes * ctx->pb.orbits * ctx->pb.n * ctx->elem : 0;
    return SDEB_OK;
}

sdeb_status sdeb_grad(sdeb_ctx *ctx, const void *dL_dxK, void *dL_dp, void *dL_dx0, void *stream) {
    NvtxRange nvtx_range("sdeb_grad");
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (ctx->is_batch) return fail(ctx, SDEB_EUNSUPPORTED, "the adjoint is not available on batches");
    if (!dL_dxK || !dL_dp) return fail(ctx, SDEB_EINVAL, "dL_dxK and dL_dp must not be NULL");
    if (ctx->pb.model != SDEB_KURAMOTO && ctx->pb.model != SDEB_KURAMOTO_PAPER)
        return fail(ctx, SDEB_EUNSUPPORTED, "the adjoint is implemented for the Kuramoto models");
    if (ctx->pb.ckpt_every <= 0) return fail(ctx, SDEB_ESTATE, "context was created with ckpt_every = 0");
    if (ctx->pb.flags & kSchemeFlags)
        return fail(ctx, SDEB_EUNSUPPORTED, "sdeb_grad is the adjoint of the Euler-Maruyama step");
    if (!ctx->params_set || ctx->k_current != ctx->pb.steps)
        return fail(ctx, SDEB_ESTATE, "integrate to step %lld first (state is at %lld)", (long long)ctx->pb.steps,
                    (long long)ctx->k_current);
    const bool shared = ctx->pb.flags & SDEB_FLAG_SHARED_PARAMS;
    AdjointArgs a{};
    a.model = ctx->pb.model;
    a.n = ctx->pb.n;
    a.units = ctx->units;
    a.d = ctx->pb.d;
    a.orbits = ctx->pb.orbits;
    a.params = ctx->d_params;
    a.param_stride = shared ? 0 : ctx->pb.d;
    a.ckpt = ctx->d_ckpt;
    a.ckpt_comp = ctx->d_ckpt_comp;
    a.ckpt_every = (uint32_t)ctx->ckpt_int;
    a.steps = (uint32_t)ctx->pb.steps;
    a.orbit_offset = (uint32_t)ctx->pb.orbit_offset;
    a.dt = ctx->pb.dt;
    a.seg = ctx->d_seg;
    a.dL_dxK = dL_dxK;
    a.dL_dp = shared ? ctx->d_gradp : dL_dp;
    a.dL_dx0 = dL_dx0;
    a.keys = philox_key_schedule(ctx->pb.seed);
    a.nckpt = ctx->nckpt;
    a.check = check_word();
    a.records = ctx->adj_records;
    const bool fp64 = ctx->pb.precision == SDEB_FP64;
    const cudaStream_t s = as_stream(stream);
    cudaError_t e = launch_adjoint(a, ctx->layout, fp64, s);
    if (e == cudaErrorNotSupported)
        return fail(ctx, SDEB_EUNSUPPORTED, "no adjoint kernel for layout G=%d P=%d%s", ctx->layout.G,
                    ctx->layout.P, ctx->adj_records == SDEB_RECORDS_SHARED ? " with records in shared memory" : "");
    if (e == cudaSuccess && shared) e = launch_sum_over_orbits(ctx->d_gradp, ctx->pb.orbits, ctx->pb.d, fp64, dL_dp, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint kernel launch");
    return SDEB_OK;
}

sdeb_status sdeb_create_batch(const sdeb_problem *pbs, int32_t count, sdeb_ctx **out) {
    if (!out) return fail(nullptr, SDEB_EINVAL, "out is NULL");
    *out = nullptr;
    std::vector<BatchInstance> inst;
    BatchLayoutSums sums;
    sdeb_status st0 = build_batch_instances(pbs, count, inst, sums);
    if (st0 != SDEB_OK) return st0;
    const int64_t p_off = sums.p_off, x_off = sums.x_off, f_off = sums.f_off, o_off = sums.o_off;
    const int32_t max_n = sums.max_n;
    const int64_t max_steps = sums.max_steps;
    sdeb_ctx *c = new (std::nothrow) sdeb_ctx;
    if (!c) return fail(nullptr, SDEB_ENOMEM, "host allocation failed");
    c->is_batch = true;
    c->probs.assign(pbs, pbs + count);
    c->inst = inst;
    c->pb = pbs[0];
    c->pb.n = max_n;
    c->pb.steps = max_steps;
    c->pb.orbits = o_off;
    c->elem = pbs[0].precision == SDEB_FP64 ? 8 : 4;
    c->batch_params_bytes = p_off * (int64_t)c->elem;
    c->batch_state_elems = x_off;
    c->batch_frame_elems = f_off;
    c->batch_items = o_off;
    cudaError_t e = cudaGetDevice(&c->device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_params, (size_t)c->batch_params_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_x, (size_t)x_off * c->elem);
    if (e == cudaSuccess && c->elem == 4) e = cudaMalloc((void **)&c->d_comp, (size_t)x_off * 4);
    if (e == cudaSuccess && f_off > 0) e = cudaMalloc(&c->d_frames, (size_t)f_off * c->elem);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_flags, (size_t)o_off);
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_inst, sizeof(BatchInstance) * inst.size());
    if (e == cudaSuccess) e = cudaMalloc((void **)&c->d_head, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_inst, inst.data(), sizeof(BatchInstance) * inst.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        sdeb_status st = cuda_fail(nullptr, e, "sdeb_create_batch");
        free_buffers(c);
        delete c;
        return st;
    }
    c->num_sms = sms > 0 ? sms : 1;
    c->grid_cap = c->num_sms * batch_blocks_per_sm(c->elem == 8);
    sdeb_status st = upload_plan(c, plan_batch(c->inst, c->batch_chain_frac, c->num_sms));
    if (st != SDEB_OK) {
        free_buffers(c);
        delete c;
        return fail(nullptr, st, "batch plan upload failed");
    }
    *out = c;
    return SDEB_OK;
}

sdeb_status sdeb_batch_read(sdeb_ctx *ctx, int32_t instance, int32_t what, void *dst, size_t dst_bytes,
                            int32_t dst_on_device, void *stream) {
    if (!ctx) return fail(nullptr, SDEB_EINVAL, "ctx is NULL");
    if (!ctx->is_batch) return fail(ctx, SDEB_EINVAL, "not a batch context");
    if (!dst) return fail(ctx, SDEB_EINVAL, "dst is NULL");
    if (!mem_kind_valid(dst_on_device)) return fail(ctx, SDEB_EINVAL, "dst_on_device %d is not SDEB_MEM_*", dst_on_device);
    if (instance < 0 || instance >= (int32_t)ctx->inst.size())
        return fail(ctx, SDEB_EINVAL, "instance %d outside [0, %d)", instance, (int)ctx->inst.size());
    if (!ctx->batch_done) return fail(ctx, SDEB_ESTATE, "integrate the batch first");
    const BatchInstance &b = ctx->inst[(size_t)instance];
    const void *src = nullptr;
    size_t bytes = 0;
    if (what == 0) {
        if (!b.has_frames) return fail(ctx, SDEB_ESTATE, "instance %d has no frames", instance);
        bytes = (size_t)((b.steps / b.stride + 1) * b.orbits * b.n) * ctx->elem;
        src = static_cast<const char *>(ctx->d_frames) + (size_t)b.f_off * ctx->elem;
    } else if (what == 1) {
        bytes = (size_t)(b.orbits * b.n) * ctx->elem;
        src = static_cast<const char *>(ctx->d_x) + (size_t)b.x_off * ctx->elem;
    } else {
        return fail(ctx, SDEB_EINVAL, "what must be 0 (frames) or 1 (final state)");
    }
    if (dst_bytes != bytes) return fail(ctx, SDEB_EINVAL, "dst_bytes=%zu, expected %zu", dst_bytes, bytes);
    const cudaStream_t s = as_stream(stream);
    cudaError_t e = read_copy(dst, src, bytes, dst_on_device, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(ctx, e, "sdeb_batch_read copy");
    }
    return SDEB_OK;
}

sdeb_status sdeb_batch_info(const sdeb_ctx *ctx, int32_t *tasks, int32_t *team_items, int32_t *grid) {
    if (!ctx || !ctx->is_batch || !tasks || !team_items || !grid)
        return fail(nullptr, SDEB_EINVAL, "batch context and outputs required");
    *tasks = ctx->ntasks;
    *team_items = ctx->team_items;
    *grid = ctx->grid;
    return SDEB_OK;
}

sdeb_status sdeb_batch_set_schedule(sdeb_ctx *ctx, double chain_fraction) {
    if (!ctx || !ctx->is_batch) return fail(nullptr, SDEB_EINVAL, "batch context required");
    if (!(chain_fraction > 0.0) || !std::isfinite(chain_fraction))
        return fail(ctx, SDEB_EINVAL, "chain_fraction must be positive and finite");
    if (ctx->params_set && ctx->batch_done)
        return fail(ctx, SDEB_ESTATE, "set the schedule before integrating (after sdeb_set_params)");
    ctx->batch_chain_frac = chain_fraction;
    return upload_plan(ctx, plan_batch(ctx->inst, chain_fraction, ctx->num_sms));
}

sdeb_status sdeb_batch_plan(const sdeb_problem *pbs, int32_t count, double chain_fraction, int32_t num_sms,
                            int32_t *lanes, int32_t *units_per_lane, int64_t total_orbits, int32_t *item_task,
                            int32_t *item_slot, int32_t *item_lane0, int32_t *ntasks) {
    if (!(chain_fraction > 0.0) || !std::isfinite(chain_fraction))
        return fail(nullptr, SDEB_EINVAL, "chain_fraction must be positive and finite");
    if (num_sms < 1) return fail(nullptr, SDEB_EINVAL, "num_sms must be >= 1");
    std::vector<BatchInstance> inst;
    BatchLayoutSums sums;
    sdeb_status st = build_batch_instances(pbs, count, inst, sums);
    if (st != SDEB_OK) return st;
    const bool per_item = item_task || item_slot || item_lane0;
    if (per_item && total_orbits != sums.o_off)
        return fail(nullptr, SDEB_EINVAL, "total_orbits is %lld, the batch holds %lld orbits", (long long)total_orbits,
                    (long long)sums.o_off);
    const BatchPlan plan = plan_batch(inst, chain_fraction, num_sms);
    for (int32_t i = 0; i < count; ++i) {
        if (lanes) lanes[i] = plan.inst_layout[(size_t)i].G;
        if (units_per_lane) units_per_lane[i] = plan.inst_layout[(size_t)i].P;
    }
    if (ntasks) *ntasks = (int32_t)plan.tasks.size();
    if (!per_item) return SDEB_OK;
    auto place = [&](int32_t item, int32_t t, int32_t slot, int32_t lane0) {
        const BatchItem &it = plan.items[(size_t)item];
        const int64_t g = inst[(size_t)it.instance].o_off + it.orbit;
        if (item_task) item_task[g] = t;
        if (item_slot) item_slot[g] = slot;
        if (item_lane0) item_lane0[g] = lane0;
    };
    for (int32_t t = 0; t < (int32_t)plan.tasks.size(); ++t) {
        const BatchTask &task = plan.tasks[(size_t)t];
        if (task.kind == kBatchWarps) {
            for (int w = 0; w < 4; ++w) {
                const BatchWarpTask &wt = task.warp[w];
                int32_t lane = 0;
                for (int j = 0; j < wt.count; ++j) {
                    place(wt.first + j, t, w, lane);
                    lane += (inst[(size_t)plan.items[(size_t)(wt.first + j)].instance].units + wt.p - 1) / wt.p;
                }
            }
        } else if (task.kind == kBatchTeam128) {
            place(task.item[0], t, 6, 0);
        } else {
            for (int h = 0; h < 2; ++h)
                if (task.item[h] >= 0) place(task.item[h], t, 4 + h, 0);
        }
    }
    return SDEB_OK;
}

sdeb_status sdeb_batch_layout(const sdeb_ctx *ctx, int32_t instance, int32_t *lanes, int32_t *units_per_lane) {
    if (!ctx || !ctx->is_batch || !lanes || !units_per_lane)
        return fail(nullptr, SDEB_EINVAL, "batch context and outputs required");
    if (instance < 0 || instance >= (int32_t)ctx->inst_layout.size())
        return fail(nullptr, SDEB_EINVAL, "instance %d out of range", instance);
    *lanes = ctx->inst_layout[(size_t)instance].G;
    *units_per_lane = ctx->inst_layout[(size_t)instance].P;
    return SDEB_OK;
}

sdeb_status sdeb_philox_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t b0, int64_t nb, uint32_t o0,
                             int64_t no, uint32_t stream_id, uint32_t *out, void *stream) {
    if (nk < 0 || nb < 0 || no < 0) return fail(nullptr, SDEB_EINVAL, "negative extent");
    if (nk > 0x100000000LL || nb > 0x100000000LL || no > 0x100000000LL)
        return fail(nullptr, SDEB_EINVAL, "extent beyond the 32-bit counter range");
    int64_t t;
    if (!mul_ok(nk, nb, t) || !mul_ok(t, no, t) || t > INT64_MAX / 16)
        return fail(nullptr, SDEB_EINVAL, "size overflows");
    if (t > 0 && !out) return fail(nullptr, SDEB_EINVAL, "out is NULL");
    cudaError_t e = launch_philox_fill(seed, k0, nk, b0, nb, o0, no, stream_id, out, as_stream(stream));
    return e == cudaSuccess ? SDEB_OK : cuda_fail(nullptr, e, "philox_fill launch");
}

sdeb_status sdeb_normals_fill(uint64_t seed, uint32_t k0, int64_t nk, uint32_t o0, int64_t no, int32_t m,
                              int32_t precision, void *out, void *stream) {
    if (nk < 0 || no < 0 || m < 0) return fail(nullptr, SDEB_EINVAL, "negative extent");
    if (nk > 0x100000000LL || no > 0x100000000LL)
        return fail(nullptr, SDEB_EINVAL, "extent beyond the 32-bit counter range");
    if (precision != SDEB_FP32_KAHAN && precision != SDEB_FP64)
        return fail(nullptr, SDEB_EINVAL, "unknown precision %d", precision);
    int64_t t;
    if (!mul_ok(nk, no, t) || !mul_ok(t, m, t) || t > INT64_MAX / 8)
        return fail(nullptr, SDEB_EINVAL, "size overflows");
    if (t > 0 && !out) return fail(nullptr, SDEB_EINVAL, "out is NULL");
    cudaError_t e = launch_normals_fill(seed, k0, nk, o0, no, m, precision == SDEB_FP64, out, as_stream(stream));
    return e == cudaSuccess ? SDEB_OK : cuda_fail(nullptr, e, "normals_fill launch");
}

sdeb_status sdeb_order_param(const void *theta, int64_t orbits, int32_t n, int32_t precision, void *r,
                             void *dr, void *stream) {
    if (orbits < 0 || n <= 0) return fail(nullptr, SDEB_EINVAL, "orbits >= 0 and n > 0 required");
    if (precision != SDEB_FP32_KAHAN && precision != SDEB_FP64)
        return fail(nullptr, SDEB_EINVAL, "unknown precision %d", precision);
    if (orbits > 0 && (!theta || !r)) return fail(nullptr, SDEB_EINVAL, "theta and r must not be NULL");
    cudaError_t e = launch_order_param(theta, orbits, n, precision == SDEB_FP64, r, dr, as_stream(stream));
    return e == cudaSuccess ? SDEB_OK : cuda_fail(nullptr, e, "order_param launch");
}

}  // extern "C"
