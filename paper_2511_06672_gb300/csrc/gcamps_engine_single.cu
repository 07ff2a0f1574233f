// Single-operation launches of libgcamps (arxiv 2511.06672, Sec. 3): one Clifford gate, one non-Clifford
// step or one disentangling sweep on every circuit of a handle.

#include "gcamps_device.cuh"

namespace gcx {
namespace {

__global__ void __launch_bounds__(kThreads, kMinCtas) k_single(Engine e, gcamps_op op) { single_body(e, op); }

}  // namespace

cudaError_t launch_single(const Engine& e, const gcamps_op& op, cudaStream_t st) {
  if (e.precision) return launch_single_tc(e, op, st);
  return launch_cluster(k_single, e, st, e, op);
}

}  // namespace gcx
