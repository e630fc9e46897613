// icarus_ops.h -- per-precision launcher table (one instantiation per precision mode)
#pragma once
#include <cstddef>
#include <cuda_runtime.h>

#include "../../include/icarus.h"

namespace icarus {
struct Params;
struct Ops {
    void (*fill_ghosts)(const Params &, void *U, void *W, int stage, cudaStream_t);
    void (*fluxes)(const Params &, const void *W, void *F1, void *F2, void *F3, cudaStream_t);
    void (*flux_dir)(const Params &, int dir, const void *W, void *F, cudaStream_t);
    void (*divb)(const Params &, const void *W, void *divB, cudaStream_t);
    void (*update)(const Params &, int stage, const void *Us, const void *Ws, void *Uo, void *Wo,
                   const void *F1, const void *F2, const void *F3, const void *divB, cudaStream_t);
    void (*cfl)(const Params &, const void *W, cudaStream_t);
    void (*probe)(const Params &, const void *W, cudaStream_t);
    void (*prims)(const Params &, const void *U, void *W, cudaStream_t);
    void (*init_state)(const Params &, void *U, void *W, double r_in, cudaStream_t);
    void (*pack)(const Params &, const void *U, double *out, cudaStream_t);
    void (*unpack)(const Params &, void *U, const double *in, cudaStream_t);
    // one whole stage (fluxes, div B, update) in a single kernel; null where not available
    void (*fused_stage)(const Params &, int stage, const void *Us, const void *Ws, void *Uo, void *Wo, cudaStream_t);
    // the stage update with the r-face fluxes computed inside it (the theta / phi fluxes and div B
    // from the separate kernels); null where not available
    void (*update_rf)(const Params &, int stage, const void *Us, const void *Ws, void *Uo, void *Wo, const void *F2,
                      const void *F3, const void *divB, cudaStream_t);
    // GLM div-B control: psi ghosts; the three flux kernels with the (B_n, psi) face step; the psi
    // stage update (after the MHD update); psi from / to host-layout doubles
    void (*glm_ghost)(const Params &, void *Psi, cudaStream_t);
    void (*fluxes_glm)(const Params &, const void *W, const void *Psi, void *F1, void *F2, void *F3, void *FP1, void *FP2,
                       void *FP3, cudaStream_t);
    void (*glm_update)(const Params &, int stage, const void *Ps, void *Po, const void *FP1, const void *FP2,
                       const void *FP3, cudaStream_t);
    void (*psi_copy)(const Params &, void *Psi, double *buf, int to_psi, cudaStream_t);
    // CME tracer: ghost values of c at the stage time; the stage update of rho c (after update);
    // c of the interior from / to host-layout doubles [n3][n2][n1] (staged on the device)
    void (*tracer_ghost)(const Params &, void *C, int stage, cudaStream_t);
    void (*tracer_update)(const Params &, int stage, const void *C, const void *F1, const void *F2, const void *F3,
                          const void *Ts, void *To, const void *Unew, void *Cout, cudaStream_t);
    void (*tracer_set)(const Params &, const double *c, const void *U, void *T, void *C, cudaStream_t);
    void (*tracer_get)(const Params &, const void *T, const void *U, double *c, cudaStream_t);
    size_t ts_size, tw_size;
};
int report_error(int code, const char *msg);
// validation of a grid description (EINVAL and a message for what icarus_init rejects)
int check_grid(const icarus_grid *g);
Ops ops_fp64();
Ops ops_fp32();
Ops ops_mixed();
}  // namespace icarus
