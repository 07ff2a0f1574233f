// The precision form's cluster kernels (opts.precision = 1): the same kernel bodies as the FP64 translation
// units, compiled with GCAMPS_TC = 1 so that their CTA-level Grams run on the tensor cores (tcgen05 TF32
// with a three-term split, the accumulator in TMEM, operands staged in dynamic shared memory).
// This unit: the gate-list kernels; gcamps_engine_tc_ops.cu holds the single-step and scoring kernels.
#define GCAMPS_TC 1
#include "gcamps_device.cuh"

namespace gcx {
namespace {

__global__ void __launch_bounds__(kThreads, kMinCtas) k_run_tc(Engine e, const gcamps_op* ops, const int32_t* begin) {
  const int c = blockIdx.x / e.csize;
  run_body(e, ops, begin[c], begin[c + 1], c, blockIdx.x % e.csize);
}

__global__ void __launch_bounds__(kThreads, kMinCtas) k_run_all_tc(Engine e, const gcamps_op* ops, int nops) {
  run_body(e, ops, 0, nops, blockIdx.x / e.csize, blockIdx.x % e.csize);
}

}  // namespace

cudaError_t launch_run_tc(const Engine& e, const gcamps_op* ops_dev, const int32_t* begin_dev, cudaStream_t st) {
  return launch_cluster(k_run_tc, e, st, e, ops_dev, begin_dev);
}

cudaError_t launch_run_all_tc(const Engine& e, const gcamps_op* ops_dev, int nops, cudaStream_t st) {
  return launch_cluster(k_run_all_tc, e, st, e, ops_dev, nops);
}

}  // namespace gcx
