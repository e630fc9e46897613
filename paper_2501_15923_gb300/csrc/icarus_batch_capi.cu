// icarus_batch_capi.cu -- host side of the batched ensemble (include/icarus.h, icarus_batch_*):
// member contexts, work-item tables, the tile autotuner, and the one-launch-per-step graph.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <map>
#include <tuple>
#include <vector>

#include "icarus_batch.cuh"
#include "icarus_ctx.h"

using namespace icarus;

struct icarus_batch {
    std::vector<icarus_ctx *> members;
    std::vector<int> versions;
    std::vector<int> cfg_r, cfg_t;
    icarus_options opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    BatchOps ops{};
    Member *d_members = nullptr;
    long long *d_off = nullptr;
    BarrierState *d_bar = nullptr;
    size_t members_cap = 0;
    int blocks = 0;
    cudaGraphExec_t graph = nullptr;
    bool use_graph = true;
    bool dirty = true;
    long long spin_limit = 4000000000LL;
    int mode = ICARUS_BATCH_CONCURRENT;   // members' steps as graph branches (default: measured fastest)
    int pcfg_r = 2, pcfg_t = 1;           // the per-phase form's flux tiles (one per direction, all members)
    // concurrent form: lanes of members whose steps run as parallel branches of one graph
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_events;  // [0]: fork; [1 + l]: join of lane l
    long long items[BPH_N] = {};          // work items of each phase over all members
    std::map<std::tuple<int, int, int>, std::pair<int, int>> tune_cache;   // grid shape -> (cfg_r, cfg_t)
};

namespace {

#define BCK(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return report_error(ICARUS_ECUDA, cudaGetErrorString(e_));            \
    } while (0)

void *balloc(icarus_batch *b, size_t bytes)
{
    // batch-level tables live in the first member's context (released with it)
    return ctx_alloc(b->members[0], bytes);
}

template <int D, int BX, int BY> void tiles_of(const Params &P, int *t, long long *items)
{
    int nx, ny, nz;
    flux_tiles<D, BX, BY>(P, nx, ny, nz);
    t[0] = nx; t[1] = ny; t[2] = nz;
    *items = (long long)nx * ny * nz;
}

int build_tables(icarus_batch *b)
{
    const int n = (int)b->members.size();
    std::vector<Member> hm(n);
    std::vector<long long> off((size_t)BPH_N * (n + 1), 0);
    for (int m = 0; m < n; ++m) {
        icarus_ctx *c = b->members[m];
        Member &M = hm[m];
        M.P = c->P;
        M.U = c->U; M.U1 = c->U1; M.W = c->W; M.W1 = c->W1;
        M.F1 = c->F1; M.F2 = c->F2; M.F3 = c->F3; M.divB = c->divB;
        // per-member tiles in the persistent kernel; one choice for the ensemble in the per-phase form
        M.cfg_r = b->mode == ICARUS_BATCH_PHASES ? b->pcfg_r : b->cfg_r[m];
        M.cfg_t = b->mode == ICARUS_BATCH_PHASES ? b->pcfg_t : b->cfg_t[m];
        if (M.cfg_r == 0) tiles_of<0, 128, 2>(M.P, M.tr, &M.items_r);
        else if (M.cfg_r == 1) tiles_of<0, 64, 4>(M.P, M.tr, &M.items_r);
        else tiles_of<0, 32, 8>(M.P, M.tr, &M.items_r);
        if (M.cfg_t == 0) { tiles_of<1, 16, 16>(M.P, M.tt, &M.items_t); tiles_of<2, 16, 16>(M.P, M.tp, &M.items_p); }
        else { tiles_of<1, 32, 8>(M.P, M.tt, &M.items_t); tiles_of<2, 32, 8>(M.P, M.tp, &M.items_p); }
        const Params &P = M.P;
        auto chunks = [](long long x) { return (x + BATCH_THREADS - 1) / BATCH_THREADS; };
        long long it[BPH_N];
        it[BPH_BND1] = chunks((long long)P.n2 * P.n3);
        it[BPH_BND2] = chunks((long long)P.p1 * P.n3);
        it[BPH_BND3] = chunks((long long)P.p1 * P.p2);
        it[BPH_FLUX] = M.items_r + M.items_t + M.items_p;
        it[BPH_DIVB] = P.divb == 1 ? chunks((long long)(P.n1 + 2) * (P.n2 + 2) * (P.n3 + 2)) : 0;
        it[BPH_UPD] = chunks((long long)P.n1 * P.n2 * P.n3);
        it[BPH_PROBE] = P.n_probes > 0 ? 1 : 0;
        it[BPH_FR] = M.items_r;
        it[BPH_FT] = M.items_t;
        it[BPH_FP] = M.items_p;
        for (int ph = 0; ph < BPH_N; ++ph) off[(size_t)ph * (n + 1) + m + 1] = off[(size_t)ph * (n + 1) + m] + it[ph];
        b->versions[m] = c->p_version;
    }
    if (!b->d_members) {
        b->d_members = (Member *)balloc(b, sizeof(Member) * n);
        b->d_off = (long long *)balloc(b, sizeof(long long) * off.size());
        b->d_bar = (BarrierState *)balloc(b, sizeof(BarrierState));
        if (!b->d_members || !b->d_off || !b->d_bar) return report_error(ICARUS_ENOMEM, "batch table allocation failed");
        BCK(cudaMemsetAsync(b->d_bar, 0, sizeof(BarrierState), b->stream));
    }
    for (int ph = 0; ph < BPH_N; ++ph) b->items[ph] = off[(size_t)ph * (n + 1) + n];
    BCK(cudaMemcpyAsync(b->d_members, hm.data(), sizeof(Member) * n, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaMemcpyAsync(b->d_off, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return ICARUS_OK;
}

int enqueue(icarus_batch *b)
{
    BatchArgs A;
    A.m = b->d_members;
    A.off = b->d_off;
    A.n = (int)b->members.size();
    A.bar = b->d_bar;
    A.spin_limit = b->spin_limit;
    if (b->mode == ICARUS_BATCH_PHASES) {
        BCK(b->ops.launch_phases(A, b->items, b->pcfg_r, b->pcfg_t, b->stream));
        return ICARUS_OK;
    }
    // the barrier counters start from zero at every step (the error word is kept)
    BCK(cudaMemsetAsync(b->d_bar, 0, 2 * sizeof(unsigned int), b->stream));
    BCK(b->ops.launch(A, b->blocks, b->stream));
    return ICARUS_OK;
}

// concurrent form: every member's own step kernels (the single solver's, each launch with the
// member's parameters) captured on one of up to kLanes parallel streams, members assigned to the
// least-loaded lane in decreasing order of cells, joined into one graph per ensemble step
constexpr int kLanes = 16;

int capture_concurrent(icarus_batch *b, cudaGraph_t *g)
{
    const int n = (int)b->members.size();
    const int L = n < kLanes ? n : kLanes;
    while ((int)b->lanes.size() < L) {
        cudaStream_t st;
        BCK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b->lanes.push_back(st);
    }
    while ((int)b->lane_events.size() < L + 1) {
        cudaEvent_t e;
        BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->lane_events.push_back(e);
    }
    std::vector<int> order(n);
    for (int m = 0; m < n; ++m) order[m] = m;
    auto cells = [&](int m) { const Params &P = b->members[m]->P; return (long long)P.n1 * P.n2 * P.n3; };
    std::sort(order.begin(), order.end(), [&](int x, int y) { return cells(x) > cells(y); });
    std::vector<long long> load(L, 0);
    std::vector<std::vector<int>> lane_members(L);
    for (int m : order) {
        int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane_members[l].push_back(m);
        load[l] += cells(m);
    }
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->lane_events[0], b->stream);
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        e = cudaStreamWaitEvent(b->lanes[l], b->lane_events[0], 0);
        for (int m : lane_members[l]) enqueue_step_on(b->members[m], b->lanes[l]);
        if (e == cudaSuccess) e = cudaEventRecord(b->lane_events[1 + l], b->lanes[l]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->lane_events[1 + l], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(b->stream, g);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return report_error(ICARUS_ECUDA, cudaGetErrorString(e != cudaSuccess ? e : e2));
    return ICARUS_OK;
}

int prepare(icarus_batch *b)
{
    bool changed = b->dirty;
    for (size_t m = 0; m < b->members.size(); ++m)
        if (b->versions[m] != b->members[m]->p_version) changed = true;
    if (!changed) return ICARUS_OK;
    for (icarus_ctx *c : b->members)
        if (!c->have_state) return report_error(ICARUS_ESTATE, "every member needs a state (icarus_set_boundary / icarus_set_state)");
    int rc = build_tables(b);
    if (rc) return rc;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    if (b->mode == ICARUS_BATCH_CONCURRENT) {
        cudaGraph_t g;
        rc = capture_concurrent(b, &g);
        if (rc) return rc;
        cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return report_error(ICARUS_ECUDA, cudaGetErrorString(e));
        b->dirty = false;
        return ICARUS_OK;
    }
    if (b->use_graph) {
        cudaGraph_t g;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            int erc = enqueue(b);
            cudaError_t e = cudaStreamEndCapture(b->stream, &g);
            if (erc == 0 && e == cudaSuccess) {
                if (cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) b->graph = nullptr;
                cudaGraphDestroy(g);
            }
        }
        cudaGetLastError();
        if (!b->graph) b->use_graph = false;   // cooperative node not capturable here: launch directly
    }
    b->dirty = false;
    return ICARUS_OK;
}

}  // namespace

extern "C" {

int icarus_batch_init(int n_members, const icarus_grid *grids, double gamma, double omega_rot,
                      const icarus_options *opts, icarus_batch **out)
{
    if (n_members < 1 || !grids || !opts || !out) return report_error(ICARUS_EINVAL, "bad argument");
    if (n_members > ICARUS_BATCH_MAX_MEMBERS) return report_error(ICARUS_EINVAL, "too many members (ICARUS_BATCH_MAX_MEMBERS)");
    if (opts->flux == ICARUS_FLUX_HLLD) return report_error(ICARUS_EINVAL, "the batched form supports the TVDLF and HLL fluxes only");
    if (opts->tracer) return report_error(ICARUS_EINVAL, "the batched form carries no CME tracer");
    if (opts->divb == ICARUS_DIVB_GLM) return report_error(ICARUS_EINVAL, "the batched form has no GLM div-B control");
    if (opts->divb == ICARUS_DIVB_POWELL) return report_error(ICARUS_EINVAL, "the batched form has no Powell source");
    icarus_batch *b = new icarus_batch();
    b->opts = *opts;
    if (opts->cuda_stream) b->stream = (cudaStream_t)opts->cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return report_error(ICARUS_ECUDA, "stream creation failed");
        }
        b->own_stream = true;
    }
    b->ops = opts->precision == ICARUS_FP64 ? batch_ops_fp64()
           : (opts->precision == ICARUS_FP32 ? batch_ops_fp32() : batch_ops_mixed());
    icarus_options mo = *opts;
    mo.cuda_stream = b->stream;
    for (int m = 0; m < n_members; ++m) {
        icarus_ctx *c = nullptr;
        int rc = icarus_init(&grids[m], gamma, omega_rot, &mo, &c);
        if (rc) {
            for (icarus_ctx *x : b->members) icarus_destroy(x);
            if (b->own_stream) cudaStreamDestroy(b->stream);
            delete b;
            return rc;
        }
        b->members.push_back(c);
        b->versions.push_back(-1);
        b->cfg_r.push_back(0);
        b->cfg_t.push_back(0);
    }
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = b->ops.blocks_per_sm(n_members);
    if (per_sm < 1) {
        icarus_batch_destroy(b);
        return report_error(ICARUS_ECUDA, "batched kernel cannot be resident (occupancy 0)");
    }
    b->blocks = per_sm * nsm;
    *out = b;
    return ICARUS_OK;
}

int icarus_batch_member(icarus_batch *b, int m, icarus_ctx **ctx)
{
    if (!b || !ctx || m < 0 || m >= (int)b->members.size()) return report_error(ICARUS_EINVAL, "bad member index");
    *ctx = b->members[m];
    return ICARUS_OK;
}

// the per-phase form's autotuner: for each direction, every tile candidate times the flux launch
// over all members (reps launches after an untimed one, on the members' current primitives)
static int autotune_phases(icarus_batch *b, int reps)
{
    for (icarus_ctx *c : b->members)
        if (!c->have_state) return report_error(ICARUS_ESTATE, "autotune needs member states");
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    int best[2] = {b->pcfg_r, b->pcfg_t};
    for (int grp = 0; grp < 2; ++grp) {          // 0: r faces; 1: theta and phi faces (one shape code)
        float best_ms = 1e30f;
        for (int cfg = 0; cfg < (grp == 0 ? NCFG_R : NCFG_T); ++cfg) {
            if (grp == 0) b->pcfg_r = cfg; else b->pcfg_t = cfg;
            int rc = build_tables(b);
            if (rc) return rc;
            BatchArgs A{};
            A.m = b->d_members; A.off = b->d_off; A.n = (int)b->members.size();
            for (int q = 0; q <= reps; ++q) {
                if (q == 1) BCK(cudaEventRecord(e0, b->stream));
                if (grp == 0) BCK(b->ops.launch_flux_dir(A, 0, cfg, b->items[BPH_FR], 1, b->stream));
                else {
                    BCK(b->ops.launch_flux_dir(A, 1, cfg, b->items[BPH_FT], 1, b->stream));
                    BCK(b->ops.launch_flux_dir(A, 2, cfg, b->items[BPH_FP], 1, b->stream));
                }
            }
            BCK(cudaEventRecord(e1, b->stream));
            BCK(cudaEventSynchronize(e1));
            float ms = 0.f;
            BCK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best_ms) { best_ms = ms; best[grp] = cfg; }
        }
        if (grp == 0) b->pcfg_r = best[0]; else b->pcfg_t = best[1];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->dirty = true;
    return ICARUS_OK;
}

int icarus_batch_autotune(icarus_batch *b, int reps)
{
    if (!b || reps < 1) return report_error(ICARUS_EINVAL, "bad argument");
    if (b->mode == ICARUS_BATCH_PHASES) return autotune_phases(b, reps);
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    for (size_t m = 0; m < b->members.size(); ++m) {
        icarus_ctx *c = b->members[m];
        const Params &P = c->P;
        auto key = std::make_tuple(P.n1, P.n2, P.n3);
        auto hit = b->tune_cache.find(key);
        if (hit == b->tune_cache.end()) {
            if (!c->have_state) return report_error(ICARUS_ESTATE, "autotune needs member states");
            float best_r = 1e30f, best_t = 1e30f;
            int cr = 0, ct = 0;
            for (int cfg = 0; cfg < NCFG_R + NCFG_T; ++cfg) {
                const bool is_r = cfg < NCFG_R;
                const int v = is_r ? cfg : cfg - NCFG_R;
                // one untimed launch, then reps timed ones
                for (int q = 0; q <= reps; ++q) {
                    if (q == 1) BCK(cudaEventRecord(e0, b->stream));
                    if (is_r) b->ops.flux_variant(P, 0, v, c->W, c->F1, b->stream);
                    else {
                        b->ops.flux_variant(P, 1, v, c->W, c->F2, b->stream);
                        b->ops.flux_variant(P, 2, v, c->W, c->F3, b->stream);
                    }
                }
                BCK(cudaEventRecord(e1, b->stream));
                BCK(cudaEventSynchronize(e1));
                float ms = 0.f;
                BCK(cudaEventElapsedTime(&ms, e0, e1));
                if (is_r && ms < best_r) { best_r = ms; cr = v; }
                if (!is_r && ms < best_t) { best_t = ms; ct = v; }
            }
            hit = b->tune_cache.emplace(key, std::make_pair(cr, ct)).first;
        }
        b->cfg_r[m] = hit->second.first;
        b->cfg_t[m] = hit->second.second;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BCK(cudaGetLastError());
    b->dirty = true;
    return ICARUS_OK;
}

int icarus_batch_set_mode(icarus_batch *b, int mode)
{
    if (!b || (mode != ICARUS_BATCH_PERSISTENT && mode != ICARUS_BATCH_PHASES && mode != ICARUS_BATCH_CONCURRENT))
        return report_error(ICARUS_EINVAL, "mode must be ICARUS_BATCH_PERSISTENT, _PHASES or _CONCURRENT");
    if (b->mode != mode) b->dirty = true;
    b->mode = mode;
    return ICARUS_OK;
}

int icarus_batch_tiles(icarus_batch *b, int m, int *cfg)
{
    if (!b || !cfg || m < 0 || m >= (int)b->members.size()) return report_error(ICARUS_EINVAL, "bad argument");
    cfg[0] = b->mode == ICARUS_BATCH_PHASES ? b->pcfg_r : b->cfg_r[m];
    cfg[1] = b->mode == ICARUS_BATCH_PHASES ? b->pcfg_t : b->cfg_t[m];
    return ICARUS_OK;
}

int icarus_batch_set_tiles(icarus_batch *b, int m, int cfg_r, int cfg_t)
{
    if (!b || m < 0 || m >= (int)b->members.size() || cfg_r < 0 || cfg_r >= NCFG_R || cfg_t < 0 || cfg_t >= NCFG_T)
        return report_error(ICARUS_EINVAL, "bad argument");
    b->cfg_r[m] = cfg_r;
    b->cfg_t[m] = cfg_t;
    if (b->mode == ICARUS_BATCH_PHASES) {      // one shape for the whole ensemble in this form
        b->pcfg_r = cfg_r;
        b->pcfg_t = cfg_t;
    }
    b->dirty = true;
    return ICARUS_OK;
}

int icarus_batch_step(icarus_batch *b, int n)
{
    if (!b || n < 0) return report_error(ICARUS_EINVAL, "bad argument");
    int rc = prepare(b);
    if (rc) return rc;
    for (int q = 0; q < n; ++q) {
        if (b->graph) BCK(cudaGraphLaunch(b->graph, b->stream));
        else {
            rc = enqueue(b);
            if (rc) return rc;
        }
    }
    return ICARUS_OK;
}

int icarus_batch_barrier_selftest(int blocks, int absent, long long spin_limit)
{
    if (blocks < 1 || blocks > 64 || absent >= blocks || spin_limit < 1)
        return report_error(ICARUS_EINVAL, "blocks in [1, 64], absent < blocks, spin_limit >= 1");
    BarrierState *bar = nullptr;
    BCK(cudaMalloc(&bar, sizeof(BarrierState)));
    BCK(cudaMemset(bar, 0, sizeof(BarrierState)));
    BatchArgs A{};
    A.bar = bar;
    A.spin_limit = spin_limit;
    k_barrier_selftest<<<blocks, 32>>>(A, absent);
    cudaError_t e = cudaDeviceSynchronize();
    BarrierState s{};
    if (e == cudaSuccess) e = cudaMemcpy(&s, bar, sizeof s, cudaMemcpyDeviceToHost);
    cudaFree(bar);
    if (e != cudaSuccess) return report_error(ICARUS_ECUDA, cudaGetErrorString(e));
    if (s.err) return report_error(ICARUS_ETIMEOUT, "the barrier wait gave up (a block never arrived)");
    return ICARUS_OK;
}

int icarus_batch_status(icarus_batch *b)
{
    if (!b) return report_error(ICARUS_EINVAL, "NULL batch");
    if (b->d_bar) {
        BarrierState s;
        BCK(cudaMemcpyAsync(&s, b->d_bar, sizeof s, cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
        if (s.err) return report_error(ICARUS_ETIMEOUT, "a grid barrier of the batched step gave up waiting");
    }
    for (icarus_ctx *c : b->members) {
        int rc = icarus_status(c, nullptr);
        if (rc) return rc;
    }
    return ICARUS_OK;
}

int icarus_batch_info(icarus_batch *b, int *info)
{
    if (!b || !info) return report_error(ICARUS_EINVAL, "bad argument");
    info[0] = (int)b->members.size();
    info[1] = b->blocks;
    info[2] = b->graph != nullptr;
    info[3] = b->mode;
    return ICARUS_OK;
}

void *icarus_batch_stream(icarus_batch *b) { return b ? (void *)b->stream : nullptr; }

int icarus_batch_destroy(icarus_batch *b)
{
    if (!b) return ICARUS_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaStream_t st : b->lanes) cudaStreamDestroy(st);
    for (cudaEvent_t e : b->lane_events) cudaEventDestroy(e);
    // members other than the first, then the first (it owns the batch tables)
    for (size_t m = b->members.size(); m-- > 0;) icarus_destroy(b->members[m]);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return ICARUS_OK;
}

}  // extern "C"
