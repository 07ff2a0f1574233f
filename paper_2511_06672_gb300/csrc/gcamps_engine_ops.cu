// All-circuits launches of libgcamps (arxiv 2511.06672, Sec. 3) and the Schmidt-value readout of one bond
// (Sec. 2.4); the single-operation launch is in gcamps_engine_single.cu.

#include "gcamps_device.cuh"

namespace gcx {
namespace {

__global__ void __launch_bounds__(kThreads, kMinCtas) k_run_all(Engine e, const gcamps_op* ops, int nops) {
  run_body(e, ops, 0, nops, blockIdx.x / e.csize, blockIdx.x % e.csize);
}


// Schmidt values of one bond: move the centre next to it and take the singular values.
__global__ void __launch_bounds__(kThreads) k_schmidt(Engine e, int c, int bond, double* sv, int* cnt) {
  __shared__ Smem s;
  Ctx C = make_ctx(e, c);
  init_tau(s, e.d);
  move_center(s, C, bond);
  const int cl = C.dims[bond], cr = C.dims[bond + 1];
  Factor F = svd_factor(s, C, site_ptr(C, bond), cl * e.d, cr, 1 << 30, false);
  (void)F;
  const int m = cl * e.d < cr ? cl * e.d : cr;
  for (int i = threadIdx.x; i < m; i += blockDim.x) sv[i] = C.sing[i];
  if (threadIdx.x == 0) *cnt = m;
}


}  // namespace

cudaError_t launch_run_all(const Engine& e, const gcamps_op* ops_dev, int nops, cudaStream_t st) {
  if (e.precision) return launch_run_all_tc(e, ops_dev, nops, st);
  return launch_cluster(k_run_all, e, st, e, ops_dev, nops);
}

cudaError_t launch_schmidt(const Engine& e, int circuit, int bond, double* s_dev, int* cnt_dev, cudaStream_t st) {
  k_schmidt<<<1, kThreads, 0, st>>>(e, circuit, bond, s_dev, cnt_dev);
  return cudaGetLastError();
}

}  // namespace gcx
