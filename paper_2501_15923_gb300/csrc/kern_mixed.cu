// kern_mixed.cu -- instantiation of the hot-path kernels for the mixed precision mode, with the
// fused single-kernel stage and the update that forms the r-face fluxes itself (single-precision
// arithmetic)
#include "icarus_fused.cuh"
namespace icarus {
Ops ops_mixed()
{
    Ops o = Launch<double, float>::make();
    FusedLaunch<double>::prepare();
    o.fused_stage = FusedLaunch<double>::stage;
    o.update_rf = Launch<double, float>::update_rf;
    return o;
}
}  // namespace icarus
