// batch_fp64.cu -- instantiation of the batched-ensemble kernels for the fp64 precision mode
#include "icarus_batch.cuh"
namespace icarus {
BatchOps batch_ops_fp64() { return BatchLaunch<double, double>::make(); }
}  // namespace icarus
