// kern_fp32.cu -- instantiation of the hot-path kernels for the fp32 precision mode
#include "icarus_kernels.cuh"
namespace icarus {
Ops ops_fp32() { return Launch<float, float>::make(); }
}  // namespace icarus
