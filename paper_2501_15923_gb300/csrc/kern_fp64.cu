// kern_fp64.cu -- instantiation of the hot-path kernels for the fp64 precision mode
#include "icarus_kernels.cuh"
namespace icarus {
Ops ops_fp64() { return Launch<double, double>::make(); }
}  // namespace icarus
