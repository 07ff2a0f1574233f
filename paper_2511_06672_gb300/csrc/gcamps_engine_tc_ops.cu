// The precision form's cluster kernels (opts.precision = 1): the same kernel bodies as the FP64 translation
// units, compiled with GCAMPS_TC = 1 so that their CTA-level Grams run on the tensor cores (tcgen05 TF32
// with a three-term split, the accumulator in TMEM, operands staged in dynamic shared memory).
// This unit: the single-step and scoring kernels (the gate-list kernels are in gcamps_engine_tc.cu).
#define GCAMPS_TC 1
#include "gcamps_device.cuh"

namespace gcx {
namespace {

__global__ void __launch_bounds__(kThreads, kMinCtas) k_single_tc(Engine e, gcamps_op op) { single_body(e, op); }

__global__ void __launch_bounds__(kThreads, kMinCtas) k_score_theta_tc(Engine e, const double2* th, int cl, int cr,
                                                                      double* out_s2, double* out_vn,
                                                                      int* out_choice) {
  score_theta_body(e, th, cl, cr, out_s2, out_vn, out_choice);
}

}  // namespace

cudaError_t launch_single_tc(const Engine& e, const gcamps_op& op, cudaStream_t st) {
  return launch_cluster(k_single_tc, e, st, e, op);
}

cudaError_t launch_score_theta_tc(const Engine& e, const double2* th, int cl, int cr, double* s2, double* vn,
                                  int* choice, cudaStream_t st) {
  return launch_cluster(k_score_theta_tc, e, st, e, th, cl, cr, s2, vn, choice);
}

}  // namespace gcx
