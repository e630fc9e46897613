// icarus_ctx.h -- the solver context behind the opaque icarus_ctx handle (host side)
#pragma once
#include <string>
#include <vector>

#include "../../include/icarus.h"
#include "icarus_internal.cuh"
#include "icarus_ops.h"

struct icarus_ctx {
    icarus::Params P{};
    icarus::Ops ops{};
    icarus_grid grid{};
    icarus_options opts{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<void *> allocs;
    void *U = nullptr, *U1 = nullptr, *W = nullptr, *W1 = nullptr;
    void *F1 = nullptr, *F2 = nullptr, *F3 = nullptr, *divB = nullptr;
    void *T = nullptr, *T1 = nullptr, *C = nullptr, *C1 = nullptr;   // CME tracer: rho c (state type), c
    void *Psi = nullptr, *Psi1 = nullptr, *FP1 = nullptr, *FP2 = nullptr, *FP3 = nullptr;   // GLM psi, its face fluxes
    double *metric = nullptr, *stage_buf = nullptr;
    icarus::Scalars *sc = nullptr;
    double *maps = nullptr, *tmaps = nullptr, *cme = nullptr, *traj = nullptr, *ring = nullptr;
    size_t maps_cap = 0, tmaps_cap = 0, cme_cap = 0, traj_cap = 0;
    double *maps_raw = nullptr;     // the caller's maps as given (SI), scaled to code units on the device
    size_t maps_raw_cap = 0;
    double *hstage = nullptr;       // pinned host staging of the small boundary tables (times, CMEs)
    int *hstatus = nullptr;         // host-mapped copy of the status word, written by each step
    void *snapU = nullptr, *snapT = nullptr, *snapC = nullptr, *snapPsi = nullptr;   // icarus_step_recover's snapshot
    size_t hstage_cap = 0;
    bool have_state = false, have_boundary = false;
    cudaGraphExec_t graph = nullptr;
    long long ring_tail = 0;
    double t0, p0, b0, omega_code, gm_code;
    int launches_per_step = 0;
    int p_version = 0;      // bumped whenever P changes (the batched form re-reads it)
    std::vector<double> colvec_host;
};

namespace icarus {
// allocate through the context's allocator (tracked, released by icarus_destroy)
void *ctx_alloc(icarus_ctx *c, size_t bytes);
// enqueue one time step of the context on stream s (not captured, no graph)
void enqueue_step_on(icarus_ctx *c, cudaStream_t s);
}  // namespace icarus
