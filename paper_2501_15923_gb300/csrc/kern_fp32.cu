// kern_fp32.cu -- instantiation of the hot-path kernels for the fp32 precision mode, with the
// fused single-kernel stage and the update that forms the r-face fluxes itself (single-precision
// arithmetic)
#include "icarus_fused.cuh"
namespace icarus {
Ops ops_fp32()
{
    Ops o = Launch<float, float>::make();
    FusedLaunch<float>::prepare();
    o.fused_stage = FusedLaunch<float>::stage;
    o.update_rf = Launch<float, float>::update_rf;
    return o;
}
}  // namespace icarus
