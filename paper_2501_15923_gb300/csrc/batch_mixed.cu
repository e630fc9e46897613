// batch_mixed.cu -- instantiation of the batched-ensemble kernels for the mixed precision mode
#include "icarus_batch.cuh"
namespace icarus {
BatchOps batch_ops_mixed() { return BatchLaunch<double, float>::make(); }
}  // namespace icarus
