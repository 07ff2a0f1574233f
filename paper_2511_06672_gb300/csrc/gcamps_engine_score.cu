// Class scoring on a given two-site tensor (arxiv 2511.06672, Sec. 3): the handle-based kernel and the
// variant whose working memory is a static device array of the library (no allocation).

#include "gcamps_device.cuh"

namespace gcx {
namespace {

// Scores of every class on a caller-provided theta (score_theta_body).
__global__ void __launch_bounds__(kThreads, kMinCtas) k_score_theta(Engine e, const double2* th, int cl, int cr,
                                                                   double* out_s2, double* out_vn, int* out_choice) {
  score_theta_body(e, th, cl, cr, out_s2, out_vn, out_choice);
}

// FP32 von Neumann estimates of every class on a caller-provided theta, with their error bounds (the pruning
// step of the disentangler, vn_est32), one class per CTA of the first circuit's cluster.
__global__ void __launch_bounds__(kThreads, kMinCtas) k_estimate_theta(Engine e, const double2* th, int cl, int cr,
                                                                      double* out_est, double* out_bd) {
  __shared__ Smem s;
  const int c = blockIdx.x / e.csize, rank = blockIdx.x % e.csize;
  if (c != 0) return;   // the whole cluster of every other circuit leaves together
  Ctx C = make_ctx(e, c, rank);
  const int d = C.d, dd = d * d;
  if (rank == 0)
    for (int i = threadIdx.x; i < cl * dd * cr; i += blockDim.x) C.th32[i] = make_float2((float)th[i].x, (float)th[i].y);
  cluster_sync();
  float2* ws = reinterpret_cast<float2*>(C.cta + e.cl.block);
  const int rows = cl * d, cols = d * cr;
  const double bound = vn_est_bound(d, rows < cols ? rows : cols, rows < cols ? cols : rows);
  for (int k = rank; k < C.K; k += C.csize) {
    float est = 0.f;
    BlockGroup g{&s, (int)threadIdx.x, (int)blockDim.x};
    const bool ok = vn_est32(g, C, C.th32, cl, cr, e.candU32 + (long long)k * dd * dd, ws, s.hv, s.hw, kBTri,
                             s.btri32, kBTri, &est, (float*)nullptr, (float*)nullptr);
    if (threadIdx.x == 0) {
      out_est[k] = est;
      out_bd[k] = ok ? bound : 1e300;
    }
    __syncthreads();
  }
  cluster_sync();
}

}  // namespace

cudaError_t launch_estimate_theta(const Engine& e, const double2* th, int cl, int cr, double* est, double* bd,
                                  cudaStream_t st) {
  return launch_cluster(k_estimate_theta, e, st, e, th, cl, cr, est, bd);
}

cudaError_t launch_score_theta(const Engine& e, const double2* th, int cl, int cr, double* s2, double* vn,
                               int* choice, cudaStream_t st) {
  if (e.precision) return launch_score_theta_tc(e, th, cl, cr, s2, vn, choice, st);
  return launch_cluster(k_score_theta, e, st, e, th, cl, cr, s2, vn, choice);
}

// ------------------------------------------------------ class scores without device allocation
// gcamps_score_theta_noalloc runs the scoring and the class choice of k_score_theta with all of its
// scratch in the static array below instead of a handle's allocation.  Per CTA: kWarps warp-level
// buffers of kSmallStride entries and one CTA-level buffer (theta' of up to kStaticSide^2 entries,
// its Gram, eigenvalue arrays); then the last-visit score record, the status words and the FP32 copy
// of theta used by the screen.
constexpr long long kStaticTcap = (long long)kStaticSide * kStaticSide;
constexpr long long kStaticCtaRaw = (long long)kWarps * kSmallStride + 2 * kStaticTcap + kStaticSide + 64;
constexpr long long kStaticCta = (kStaticCtaRaw + 15) / 16 * 16;                  // 256-byte multiples
constexpr long long kStaticScores = ((3LL * kMaxK + 2 + 2LL * kSmall + 1) / 2 + 15) / 16 * 16;
constexpr long long kStaticMeta = 16;                                             // >= M_COUNT ints
constexpr long long kStaticTh32 = ((kStaticTcap + 1) / 2 + 15) / 16 * 16;          // float2 pairs
constexpr long long kStaticWords = kStaticCluster * kStaticCta + kStaticScores + kStaticMeta + kStaticTh32;
static_assert(2 * kStaticMeta >= M_COUNT, "status words");
static_assert(kStaticWords * 16 == 1696256, "scratch size stated in gcamps.h");
// 1,696,256 bytes, held by every device that loads the library.  Calls reuse it and it keeps the
// last call's contents; only the status words must start at zero, and each call clears them itself.
static __device__ __align__(256) double2 g_static_scratch[kStaticWords];
// Class unitaries for d = 2 then d = 3 ([K][d^4]) and their images ([K][20]), set once per device.
static __device__ __align__(256) double2 g_static_candU[kStaticK2 * 16 + kStaticK3 * 81];
static __device__ __align__(256) float2 g_static_candU32[kStaticK2 * 16 + kStaticK3 * 81];
static __device__ __align__(256) int32_t g_static_candImg[(kStaticK2 + kStaticK3) * 20];

// Device addresses of the arrays above, per device (host code only sees host-side stand-ins under
// their names).
struct StaticPtrs {
  double2* scratch;
  double2* candU;
  float2* candU32;
  int32_t* candImg;
};
static StaticPtrs g_static_ptrs[kStaticMaxDevices];

// The same steps as k_score_theta for one theta; the cluster is the only one of the launch.
__global__ void __launch_bounds__(kThreads, kMinCtas) k_score_theta_static(Engine e, const double2* th, int cl, int cr,
                                                                 double* out_s2, double* out_vn,
                                                                 int32_t* out_choice) {
  __shared__ Smem s;
  const int rank = blockIdx.x % e.csize;
  Ctx C = {};
  C.e = &e;
  C.c = 0;
  C.rank = rank;
  C.csize = e.csize;
  C.d = e.d;
  C.K = e.K;
  C.cta = e.cscr + (long long)rank * e.cl.total;
  C.meta = e.meta;
  C.th32 = reinterpret_cast<float2*>(e.cscr + kStaticCluster * kStaticCta + kStaticScores + kStaticMeta);
  Smem* lead = cg::this_cluster().map_shared_rank(&s, 0);
  init_tau(s, e.d);
  if (rank == 0 && threadIdx.x < M_COUNT) C.meta[threadIdx.x] = 0;   // status of this call only
  cluster_sync();
  score_classes(s, lead, C, th, cl, cr, nullptr, C.K, kExact);
  cluster_sync();
  if (rank == 0)
    for (int k = threadIdx.x; k < C.K; k += blockDim.x) {
      out_s2[k] = s.s2[k];
      out_vn[k] = s.vn[k];
    }
  cluster_sync();
  int nev = 0;
  const int kb = select_class(s, lead, C, th, cl, cr, &nev);
  cluster_sync();
  if (rank == 0 && threadIdx.x == 0) {
    out_choice[0] = kb;
    out_choice[1] = nev;
    out_choice[2] = C.meta[M_STATUS];
  }
}

cudaError_t static_setup(int device, const double* u2, const int32_t* img2, const double* u3,
                         const int32_t* img3) {
  if (device < 0 || device >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  StaticPtrs p = {};
  cudaError_t ce = cudaGetSymbolAddress(reinterpret_cast<void**>(&p.scratch), g_static_scratch);
  if (ce == cudaSuccess) ce = cudaGetSymbolAddress(reinterpret_cast<void**>(&p.candU), g_static_candU);
  if (ce == cudaSuccess) ce = cudaGetSymbolAddress(reinterpret_cast<void**>(&p.candU32), g_static_candU32);
  if (ce == cudaSuccess) {
    float u32[2 * (kStaticK2 * 16 + kStaticK3 * 81)];
    for (int i = 0; i < 2 * kStaticK2 * 16; ++i) u32[i] = (float)u2[i];
    for (int i = 0; i < 2 * kStaticK3 * 81; ++i) u32[2 * kStaticK2 * 16 + i] = (float)u3[i];
    ce = cudaMemcpyToSymbol(g_static_candU32, u32, sizeof u32, 0);
  }
  if (ce == cudaSuccess) ce = cudaGetSymbolAddress(reinterpret_cast<void**>(&p.candImg), g_static_candImg);
  if (ce == cudaSuccess) ce = cudaMemcpyToSymbol(g_static_candU, u2, sizeof(double2) * kStaticK2 * 16, 0);
  if (ce == cudaSuccess)
    ce = cudaMemcpyToSymbol(g_static_candU, u3, sizeof(double2) * kStaticK3 * 81, sizeof(double2) * kStaticK2 * 16);
  if (ce == cudaSuccess) ce = cudaMemcpyToSymbol(g_static_candImg, img2, sizeof(int32_t) * kStaticK2 * 20, 0);
  if (ce == cudaSuccess)
    ce = cudaMemcpyToSymbol(g_static_candImg, img3, sizeof(int32_t) * kStaticK3 * 20, sizeof(int32_t) * kStaticK2 * 20);
  if (ce == cudaSuccess) g_static_ptrs[device] = p;
  return ce;
}

cudaError_t launch_score_theta_static(int device, int d, double tie_tol, const double2* th, int cl, int cr,
                                      double* s2, double* vn, int32_t* choice, cudaStream_t st) {
  if (device < 0 || device >= kStaticMaxDevices) return cudaErrorInvalidDevice;
  const StaticPtrs& p = g_static_ptrs[device];
  if (!p.scratch || !p.candU || !p.candU32 || !p.candImg) return cudaErrorInitializationError;
  Engine e = {};
  e.d = d;
  e.K = d == 2 ? kStaticK2 : kStaticK3;
  e.batch = 1;
  e.csize = kStaticCluster;
  e.tie_tol = tie_tol;
  e.tcap = kStaticTcap;
  e.wcap = kStaticTcap;
  e.scap = kStaticTcap;
  e.cscr = p.scratch;
  e.cl.warp = 0;
  e.cl.block = (long long)kWarps * kSmallStride;
  e.cl.total = kStaticCta;
  e.lastsc = reinterpret_cast<double*>(p.scratch + kStaticCluster * kStaticCta);
  e.meta = reinterpret_cast<int*>(p.scratch + kStaticCluster * kStaticCta + kStaticScores);
  e.candU = p.candU + (d == 2 ? 0 : kStaticK2 * 16);
  e.candU32 = p.candU32 + (d == 2 ? 0 : kStaticK2 * 16);
  e.candImg = p.candImg + (d == 2 ? 0 : kStaticK2 * 20);
  return launch_cluster(k_score_theta_static, e, st, e, th, cl, cr, s2, vn, choice);
}


}  // namespace gcx
