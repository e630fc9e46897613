// kern_fp32.cu -- instantiation of the hot-path kernels for the fp32 precision mode, with the
// fused single-kernel stage (single-precision arithmetic)
#include "icarus_fused.cuh"
namespace icarus {
Ops ops_fp32()
{
    Ops o = Launch<float, float>::make();
    FusedLaunch<float>::prepare();
    o.fused_stage = FusedLaunch<float>::stage;
    o.fused_blocks = FusedLaunch<float>::blocks;
    return o;
}
}  // namespace icarus
