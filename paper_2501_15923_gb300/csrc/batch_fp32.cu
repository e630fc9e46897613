// batch_fp32.cu -- instantiation of the batched-ensemble kernels for the fp32 precision mode
#include "icarus_batch.cuh"
namespace icarus {
BatchOps batch_ops_fp32() { return BatchLaunch<float, float>::make(); }
}  // namespace icarus
