// Internal layout shared by the host side (gcamps_host.cpp) and the device engine
// (gcamps_engine.cu) of libgcamps.  Not part of the public C ABI (include/gcamps.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "gcamps.h"

namespace gcx {

constexpr int kThreads = 256;             // threads per CTA; a cluster of CTAs runs one circuit
constexpr int kClusterJacobiMin = 24;     // SVD splits of bond visits with at least this many Jacobi columns use the cluster
constexpr int kTcMaxM = 128;               // tensor-core Grams: at most this many rows (one M = 128 tile)
constexpr int kTcCols = 256;               // TMEM columns each engine CTA allocates for them
// their staging buffers: hi and lo parts of A (128 rows) and B (up to 256 rows) for 16 real K columns, plus
// alignment
constexpr int kTcSmemBytes = 2 * 2 * (16 + 32) * 256 + 1024;
constexpr double kMixedTieTol = 1e-5;      // tie tolerance of the precision form (FP32 contractions)
constexpr int kMinCtas = 2;               // resident CTAs per SM the engine kernels are compiled for (128 registers)
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCluster = 16;           // CTAs per circuit (thread-block cluster)
constexpr int kSmall = 729;               // warp-level scoring when theta' and its Gram fit this many entries
constexpr int kSmallStride = 2 * kSmall + 64;
constexpr int kMaxN = 128;                // qudits per circuit
constexpr int kMaxK = 90;                 // disentangler classes (d = 3)
constexpr int kDecCap = 1 << 16;          // decisions recorded per circuit
constexpr int kDStats = 8;                // doubles of counters per circuit (dstats)

// meta[] words per circuit
enum Meta { M_OC = 0, M_F, M_L, M_STATUS, M_NDEC, M_WEYL_R, M_HAVE_SPAN, M_DIAG_WHERE, M_DIAG_A, M_DIAG_B,
            M_NSNAP, M_SNAPOFF, M_COUNT };

// Adjoint snapshots: header of snapshot k of circuit c at snap_hdr + (c snap_max + k) kSnapHdr:
// [0] arena offset, [1] gate site, [2] phase r of its string, [3] first decision index of the
// disentangling after it, [kSnapDims ..] bond dimensions (n + 1), then the string (x | z, 2 n).
constexpr int kSnapDims = 8;
constexpr int kSnapHdr = 400;
static_assert(kSnapDims + (kMaxN + 1) + 2 * kMaxN <= kSnapHdr, "snapshot header");
// stats: S_VN counts exact von Neumann evaluations (the rest were excluded by the Renyi-2 bound)
// stats[] counters per circuit (int64)
enum Stat { S_T = 0, S_CLIFF, S_BONDS, S_CANDS, S_ACC, S_SWEEPS, S_MAXCHI, S_VN, S_SVD, S_JSWEEPS, S_JMAX,
            S_QR, S_COUNT };
// prof[] counters per circuit (int64, the layout gcamps_get_profile documents): SM cycles of the leader CTA
// per phase, then per bond-visit size bucket (m = min(chi_l d, d chi_r) <= 9, 27, 54, 81, larger) the
// visits, their cycles, their exact (FP64) evaluations and their FP32 von Neumann estimates; the cycles
// and count of the warp-level exact evaluations run by the leader's first warp; the phase cycles of each
// bucket's visits; and (P_CURB, internal) 1 + the bucket of the visit in progress, 0 outside visits.
enum Prof { P_CLIFF = 0, P_MPO, P_CENTER, P_THETA, P_SCREEN, P_EST, P_EXACT, P_DECIDE, P_APPLYQ, P_SPLIT,
            P_QRMOVE, P_LEAD_EXACT_CYC, P_VISITS = 12, P_VCYC = 17, P_VEXACT = 22, P_VEST = 27,
            P_LEAD_EXACT_N = 32, P_BPHASE = 33, P_XPARTS = 88, P_SMID = 160, P_CURB = 191, P_COUNT = 192 };
constexpr int kProfSmids = 16;   // 1 + the SM id of cluster ranks 0..15 in the last gate-list launch
constexpr int kProfPhases = 11;
constexpr int kProfBuckets = 5;
// parts of the leader's own exact evaluations: [P_XPARTS + 6 (5 g + b) + j], g = 0 warp-level, 1 CTA-level,
// b the size bucket, j = 0 count, 1 cycles, 2 theta' and Gram, 3 Householder reduction, 4 eigenvalues,
// 5 entropy
constexpr int kXParts = 6;
static_assert(P_BPHASE + kProfBuckets * kProfPhases <= P_XPARTS, "bucket phase words fit");
static_assert(P_XPARTS + 2 * kProfBuckets * kXParts <= P_SMID, "exact-part words fit");
static_assert(P_SMID + 16 <= P_CURB, "SM id words fit");
static_assert(P_COUNT == GCAMPS_PROF_WORDS, "profile layout stated in gcamps.h");

// Scratch areas of one circuit, as element offsets (double2) from its scratch base.
struct ScratchLayout {
  long long theta;   // two-site tensor / MPO output staging         [tcap]
  long long b;       // Jacobi working matrix                          [tcap]
  long long w;       // accumulated Jacobi rotations                   [wcap]
  long long u;       // left factor                                    [tcap]
  long long vh;      // right factor                                   [tcap]
  long long tmp;     // matmul staging                                 [tcap]
  long long total;   // elements per circuit
};

// Scratch of one CTA (circuit c, cluster rank r at index c * csize + r): kWarps warp-level scoring
// buffers of kSmallStride entries, then one block-level scoring buffer (theta' [tcap], Gram [wcap],
// eigenvalue arrays).
struct CtaLayout {
  long long warp;    // 0
  long long block;   // kWarps * kSmallStride
  long long total;
};

struct Engine {
  int n, d, K, chi_max, batch, max_sweeps, maxdim, csize;   // n: largest qudit count of the batch
  int score_kind;                 // 0 von Neumann, 1 Renyi-2, 2 weight rank then von Neumann
  int jacobi_cap;                 // most sweeps of one Jacobi SVD before GCAMPS_ENOCONV (60)
  int exact_cta_min_m;            // warp-level-size exact evaluations one per CTA from this m on (10)
  int precision;                  // 0 FP64 contractions; 1 FP32 contractions (tensor cores at CTA-level sizes)
  int tc_smem;                    // dynamic shared memory of the engine kernels (bytes; 0 without tensor cores)
  double cutoff, tie_tol, strict_weight;
  long long tcap;                 // elements of the largest two-site matrix
  long long wcap;                 // elements of the largest Jacobi rotation matrix
  long long scap;                 // elements of the largest scored theta' (and Gram): (d chi_max)^2
  // per-circuit state, circuit c at base + c * stride
  uint8_t* tab;     long long tab_stride;   // fwd exps | fwd phase | inv exps | inv phase
  const int* nq;                            // [batch] qudits of each circuit (<= n)
  double2* mps;                             // site slots of all circuits
  const long long* mps_base;                // [batch] offset of each circuit's slots in mps
  const long long* site_off;                // [batch][n+1] slot offsets within the circuit's block
  const int* bond_bound;                    // [batch][n+1] Schmidt-rank bound d^min(b, n_c-b) of bond b
  int* dims;                                // [batch][n+1]
  int* meta;                                // [batch][M_COUNT]
  long long* stats;                         // [batch][S_COUNT]
  long long* prof;                          // [batch][P_COUNT]
  double* dstats;                           // [batch][kDStats]: discarded weight, FP64 scoring flops, FP32 screen flops,
                                            // tensor-core Gram flops, algorithmic scoring flops
  int* dec;                                 // [batch][kDecCap][2]
  // replay (null when unused): circuit c with replay_n[c] > 0 applies the recorded (bond, class) pairs
  // replay[c][k] at its bond visits in order instead of choosing
  const int* replay;                        // [batch][kDecCap][2]
  const int* replay_n;                      // [batch]
  int8_t* weyl;                             // [batch][2n]
  double* lastsc;                           // [batch][3 * kMaxK + 2 + 2 * kSmall]: s2 | vn | evaluated | chi_l, chi_r | theta of the last visit
  double2* scr;     ScratchLayout sl;       // per-circuit scratch, stride sl.total
  double2* cscr;    CtaLayout cl;           // per-CTA scratch, stride cl.total
  double* sing;     long long sing_stride;  // singular values / eigenvalues
  int* iscr;        long long iscr_stride;  // permutation scratch
  const double2* candU;                     // [K][d^4] class unitaries, row-major
  const float2* candU32;                    // [K][d^4] the same in FP32 (screening)
  // adjoint snapshots (null when the handle keeps none): per circuit an arena of snap_stride entries
  double2* snap;    long long snap_stride;
  int* snap_hdr;    int snap_max;           // [batch + 1][snap_max][kSnapHdr]
  double* snap_ph;                          // [batch + 1][snap_max][4] gate phases
  const int32_t* candImg;                   // [K][20] class images
};

// Host -> device entry points implemented in gcamps_engine.cu.
cudaError_t launch_run(const Engine& e, const gcamps_op* ops_dev, const int32_t* begin_dev,
                       cudaStream_t st);
cudaError_t launch_single(const Engine& e, const gcamps_op& op, cudaStream_t st);
cudaError_t launch_reset(const Engine& e, cudaStream_t st);
cudaError_t launch_expect(const Engine& e, int circuit, const int8_t* xz_dev, double2* out_dev,
                          cudaStream_t st);
cudaError_t launch_statevector(const Engine& e, int circuit, double2* out_dev, long long dim,
                               const int32_t* ys_dev, long long nys, void* work, cudaStream_t st);
cudaError_t launch_score_theta(const Engine& e, const double2* th, int cl, int cr, double* s2, double* vn,
                               int* choice, cudaStream_t st);
// The precision form's variants of the cluster kernels (compiled with the tensor-core Gram).
cudaError_t launch_run_tc(const Engine& e, const gcamps_op* ops_dev, const int32_t* begin_dev, cudaStream_t st);
cudaError_t launch_run_all_tc(const Engine& e, const gcamps_op* ops_dev, int nops, cudaStream_t st);
cudaError_t launch_single_tc(const Engine& e, const gcamps_op& op, cudaStream_t st);
cudaError_t launch_score_theta_tc(const Engine& e, const double2* th, int cl, int cr, double* s2, double* vn,
                                  int* choice, cudaStream_t st);
// <M1|M2> of circuit c1 of e1 and circuit c2 of e2 (same n and d; transfer matrices, FP64, scratch of c1).
cudaError_t launch_overlap(const Engine& e1, int c1, const Engine& e2, int c2, double2* out_dev, cudaStream_t st);
cudaError_t launch_estimate_theta(const Engine& e, const double2* th, int cl, int cr, double* est, double* bd,
                                  cudaStream_t st);
cudaError_t launch_schmidt(const Engine& e, int circuit, int bond, double* s_dev, int* cnt_dev,
                           cudaStream_t st);
// Adjoint gradient of Re<W> for circuit cf, using circuit slot cb as the backward workspace:
// xz_dev = W's exponents (x | z, 2 n int8); grad_dev receives d doubles per recorded gate.
cudaError_t launch_adjoint(const Engine& e, int cf, int cb, const int8_t* xz_dev, double* grad_dev, cudaStream_t st);

// gcamps_score_theta_noalloc: class scores with every scratch word in static device memory of this
// library (no allocation).  theta is at most kStaticSide x kStaticSide (rows chi_l d, columns
// d chi_r); kStaticCluster CTAs score it.
constexpr int kStaticSide = 81;
static_assert(kStaticSide == GCAMPS_NOALLOC_MAX_SIDE, "limit stated in gcamps.h");
constexpr int kStaticCluster = 4;
constexpr int kStaticMaxDevices = 64;
constexpr int kStaticK2 = 20, kStaticK3 = 90;   // classes for d = 2, 3
// One-time setup for `device`, which must be current: the static arrays' device addresses (checked)
// and the class tables (unitaries [K][d^4] complex, images [K][20]) of d = 2 and d = 3, copied
// synchronously.
cudaError_t static_setup(int device, const double* u2, const int32_t* img2, const double* u3,
                         const int32_t* img3);
// Launches the scoring of theta (device memory) on stream st with the static scratch of `device`
// (static_setup done).  s2, vn: K doubles; choice: class, exact evaluations, status.
cudaError_t launch_score_theta_static(int device, int d, double tie_tol, const double2* th, int cl, int cr,
                                      double* s2, double* vn, int32_t* choice, cudaStream_t st);

}  // namespace gcx
