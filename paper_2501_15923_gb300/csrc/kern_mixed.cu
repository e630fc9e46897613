// kern_mixed.cu -- instantiation of the hot-path kernels for the mixed precision mode
#include "icarus_kernels.cuh"
namespace icarus {
Ops ops_mixed() { return Launch<double, float>::make(); }
}  // namespace icarus
