// Device side of libgcamps shared by its kernel translation units (the GCAMPS non-Clifford step,
// arxiv 2511.06672, Sec. 3, on sm_103a): state layout, complex helpers, tableau updates, the
// factorisations, the MPO step, class scoring and the disentangling sweeps.  Each .cu file that
// includes it instantiates a few kernels, so the heavy kernels compile in parallel.
#pragma once

// GCAMPS_TC = 1 in the translation unit of the precision form's kernels: its CTA-level Grams run on the
// tensor cores (tcgen05, TMEM, dynamic shared memory).  The FP64 kernels are compiled without any of it.
#ifndef GCAMPS_TC
#define GCAMPS_TC 0
#endif

//
// One CTA runs one circuit.  A launch processes a whole gate list for every circuit of the
// batch, so the control flow of the method (support span of the commuted Weyl string, bond
// dimensions after truncation, the disentangler decision at every bond) stays on the device and
// no host round trip separates two steps.
//
// Layout of a circuit in device memory (see gcamps_internal.h):
//   tableau   fwd exps [2n][2n] | fwd phase [2n] | inv exps [2n][2n] | inv phase [2n]  (uint8)
//             rows 0..n-1: C Z_j C^dag (fwd) / C^dag Z_j C (inv); rows n..2n-1: the X_j images;
//             columns x_0..x_{n-1} | z_0..z_{n-1}; phase in units of tau = exp(i pi/d), mod 2d.
//   MPS       site j in its own slot, compact row-major (a, s, b) with the current bond dims
//             dims[j] x d x dims[j+1]; complex128.
//   scratch   two-site tensor, Jacobi buffers, matmul staging, per-warp scoring buffers.
//
// All arithmetic on the MPS is complex128 (FP64), the precision the paper's simulator uses
// (Sec. 4.1.2); the tableau is exact integer arithmetic mod d / mod 2d.

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstdint>

#include "gcamps_internal.h"

namespace gcx {
namespace {

namespace cg = cooperative_groups;

// Classes are scored with the Renyi-2 bound first when the Gram has more rows than this.
constexpr int kPruneMin = 1;
// CTA-level eigenvalue multisection keeps the tridiagonal in shared memory up to this size.
constexpr int kBTri = 256;

// (i, j), j <= i, of entry t of the row-major packed lower triangle (t = i (i + 1) / 2 + j).
__device__ __forceinline__ void tri_index(int t, int& i, int& j) {
  int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > t) --r;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  i = r;
  j = t - r * (r + 1) / 2;
}

// ------------------------------------------------------------------------------ complex helpers
__device__ __forceinline__ double2 cz() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
// acc + a * b
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a) * b
__device__ __forceinline__ double2 cfmac(double2 a, double2 b, double2 acc) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
__device__ __forceinline__ double cabs2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
// FP32 complex: acc + a b and acc + a conj(b)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
  return acc;
}
__device__ __forceinline__ float2 ffmac2(float2 a, float2 b, float2 acc) {
  acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
  acc.y = fmaf(a.y, b.x, fmaf(-a.x, b.y, acc.y));
  return acc;
}
// x / |x|, and 1 for x = 0.  A subnormal x is first scaled by 2^600 (exact): its modulus carries only
// a few significant bits, so the plain quotient has a modulus visibly different from 1 and a
// Householder reflector built with it is no longer unitary.
__device__ __forceinline__ double2 unit_phase(double2 x) {
  if (x.x == 0.0 && x.y == 0.0) return make_double2(1.0, 0.0);
  if (fabs(x.x) < 0x1p-900 && fabs(x.y) < 0x1p-900) {
    x.x *= 0x1p600;
    x.y *= 0x1p600;
  }
  const double ax = hypot(x.x, x.y);
  return make_double2(x.x / ax, x.y / ax);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Four warp sums at once by reduce-scatter: after the xor-16 and xor-8 levels each lane holds one running
// sum (a in lanes 0-7, b in 8-15, c in 16-23, d in 24-31), three more levels finish it, four shuffles
// broadcast: 6 FP64 adds instead of 20 (each holds an SM sub-partition's FP64 pipe for 64 cycles).
__device__ __forceinline__ void warp_sum4(double& a, double& b, double& c, double& d) {
  const int lane = threadIdx.x & 31;
  const bool h16 = lane & 16, h8 = lane & 8;
  double k0 = h16 ? c : a, k1 = h16 ? d : b;
  k0 += __shfl_xor_sync(0xffffffffu, h16 ? a : c, 16);
  k1 += __shfl_xor_sync(0xffffffffu, h16 ? b : d, 16);
  double v = h8 ? k1 : k0;
  v += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  a = __shfl_sync(0xffffffffu, v, 0);
  b = __shfl_sync(0xffffffffu, v, 8);
  c = __shfl_sync(0xffffffffu, v, 16);
  d = __shfl_sync(0xffffffffu, v, 24);
}
__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// -------------------------------------------------------------------------- per-CTA workspace
struct Smem {
  uint8_t lut[81 * 5];        // conjugation table of the current two-qudit Clifford
  int img[20];                // its generator images, 4 x (x0, z0, x1, z1, r)
  int inv[20];                // images of its inverse
  uint8_t src[4][2 * kMaxN];  // rows read by a row product
  int srcr[4];
  double s2[kMaxK];           // Renyi-2 entropy per class (cluster leader)
  double vn[kMaxK];           // von Neumann entropy per class (cluster leader)
  uint8_t evald[kMaxK];       // vn[k] valid
  int list[kMaxK];            // classes to evaluate next (cluster leader)
  int nlist;
  int rank0;                  // numerical rank of the identity class's Gram (cluster leader; -1 = none)
  int ord[kMaxK];             // rank of each class in ascending S2 (cluster leader)
  double s2lo[kMaxK];         // lower bound of S2 from the FP32 screen (cluster leader)
  double vest[kMaxK];         // FP32 von Neumann estimate per class (cluster leader)
  double vbd[kMaxK];          // its error bound: |vest - S_vN| <= vbd (cluster leader)
  uint8_t estd[kMaxK];        // vest[k] valid
  int rk[kMaxK];              // weight rank of each exactly evaluated class (cluster leader)
  double wtri[kWarps][64];    // per warp: tridiagonal diagonal [0, 32) | off-diagonal squared [32, 64)
  float wtri32[kWarps][64];   // the same in FP32
  double btri[2 * kBTri];     // CTA-level: diagonal | off-diagonal squared
  float btri32[2 * kBTri];
  float2 hv[kBTri], hw[kBTri];  // FP32 Householder reduction: reflector v and w = p - K v of the current column
  // the second half-CTA group's copies (two FP32 estimates at once, HalfGroup) and both halves' partial sums
  float2 hv2[kBTri], hw2[kBTri];
  float btri32b[2 * kBTri];
  float redh[2][kWarps / 2];
  float2 whv[kWarps][32], whw[kWarps][32];   // the same per warp (warp-level estimates, m <= 32)
  int bcast;
  int jmode, jm, jn;          // cluster split of a bond visit: 0 none, 2 cluster Jacobi; its matrix shape (leader)
  int jflag[2];               // cluster Jacobi: a rotation happened in the sweep of this parity (leader)
  double jfro;                // cluster Jacobi: |B|_F^2 (leader)
  double red[kWarps * 4];
  double2 coef[4];            // MPO term coefficients c_m tau^{...}
  double2 tau[6];             // tau^k, k < 2d
  int flag;
  int ival[8];
  double dval[4];
  double pub;                 // BlockGroup::publish
  uint64_t tc_mbar;           // tensor-core Gram: completion barrier of its MMAs
  uint32_t tc_tmem;           // its TMEM accumulator (column base)
  uint32_t tc_commits;        // commits on tc_mbar so far (its phase parity)
};

struct Ctx {
  const Engine* e;
  int c, n, d, K;
  int rank, csize;            // position in the circuit's cluster; rank 0 leads
  double2* cta;               // this CTA's scoring scratch
  float2* th32;               // FP32 copy of the two-site tensor being scored
  const long long* site_off;  // this circuit's slot offsets
  const int* bond_bound;      // this circuit's Schmidt-rank bounds
  uint8_t *fx, *fr, *ix, *ir;
  double2* mps;
  int* dims;
  int* meta;
  long long* stats;
  long long* prof;
  double* dstats;
  int* dec;
  int8_t* weyl;
  double2* scr;
  double* sing;
  int* perm;
};

__device__ __forceinline__ double2* site_ptr(const Ctx& C, int j) { return C.mps + C.site_off[j]; }

__device__ Ctx make_ctx(const Engine& e, int c, int rank = 0) {
  Ctx C;
  C.e = &e;
  C.c = c;
  C.rank = rank;
  C.csize = e.csize;
  C.cta = e.cscr + ((long long)c * e.csize + rank) * e.cl.total;
  C.th32 = reinterpret_cast<float2*>(e.scr + (long long)c * e.sl.total + e.sl.tmp);
  const int n = e.nq[c];   // the circuit's tableau is stored compactly in its n_max-sized slot
  C.n = n;
  C.d = e.d;
  C.K = e.K;
  uint8_t* t = e.tab + (long long)c * e.tab_stride;
  C.fx = t;
  C.fr = t + 4 * n * n;
  C.ix = C.fr + 2 * n;
  C.ir = C.ix + 4 * n * n;
  C.mps = e.mps + e.mps_base[c];
  C.site_off = e.site_off + (long long)c * (e.n + 1);
  C.bond_bound = e.bond_bound + (long long)c * (e.n + 1);
  C.dims = e.dims + (long long)c * (e.n + 1);
  C.meta = e.meta + (long long)c * M_COUNT;
  C.stats = e.stats + (long long)c * S_COUNT;
  C.prof = e.prof ? e.prof + (long long)c * P_COUNT : nullptr;
  C.dstats = e.dstats + (long long)c * kDStats;
  C.dec = e.dec + (long long)c * kDecCap * 2;
  C.weyl = e.weyl + (long long)c * 2 * e.n;
  C.scr = e.scr + (long long)c * e.sl.total;
  C.sing = e.sing + (long long)c * e.sing_stride;
  C.perm = e.iscr + (long long)c * e.iscr_stride;
  return C;
}

// Phase timers (gcamps_get_profile): thread 0 of the leader CTA reads clock64 after the phase's barrier.
__device__ __forceinline__ bool prof_thread(const Ctx& C) { return C.prof && C.rank == 0 && threadIdx.x == 0; }
__device__ __forceinline__ long long prof_start(const Ctx& C) { return prof_thread(C) ? clock64() : 0; }
__device__ __forceinline__ void prof_lap(const Ctx& C, int slot, long long& t) {
  if (prof_thread(C)) {
    const long long now = clock64();
    C.prof[slot] += now - t;
    const long long cb = C.prof[P_CURB];
    if (cb > 0) C.prof[P_BPHASE + (cb - 1) * kProfPhases + slot] += now - t;
    t = now;
  }
}
__device__ __forceinline__ int prof_bucket(int m) { return m <= 9 ? 0 : (m <= 27 ? 1 : (m <= 54 ? 2 : (m <= 81 ? 3 : 4))); }

__device__ void set_status(const Ctx& C, int code) {
  if (C.meta[M_STATUS] == 0) C.meta[M_STATUS] = code;
}

// First failure of a circuit: which routine (1 = Jacobi SVD, 2 = tridiagonal eigenvalues) and the
// matrix shape it had, for gcamps_last_error.
__device__ void set_failure(const Ctx& C, int code, int where, int a, int b) {
  if (C.meta[M_STATUS] == 0) {
    C.meta[M_STATUS] = code;
    C.meta[M_DIAG_WHERE] = where;
    C.meta[M_DIAG_A] = a;
    C.meta[M_DIAG_B] = b;
  }
}

static_assert((kWarps & (kWarps - 1)) == 0 && kWarps <= 32, "block_sum's shuffle tree");
__device__ double block_sum(double v, Smem& s) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) s.red[w] = v;
  __syncthreads();
  // the kWarps partial sums by a shuffle tree (three FP64 adds per warp instead of kWarps)
  double t = l < kWarps ? s.red[l] : 0.0;
#pragma unroll
  for (int o = kWarps / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return __shfl_sync(0xffffffffu, t, 0);
}

// FP32 sums for the FP32 paths (the screen and the estimates): GB300 runs FP64 adds on a narrow pipe, so
// reductions of FP32 data stay in FP32.
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ float block_sum_f(float v, Smem& s) {
  v = warp_sum_f(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  float* red = reinterpret_cast<float*>(s.red);
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) t += red[i];
  return t;
}

__device__ void block_copy(double2* dst, const double2* src, long long count) {
  for (long long i = threadIdx.x; i < count; i += blockDim.x) dst[i] = src[i];
}

// C[M x N] = A[M x K] * B[K x N], row-major, no aliasing.
__device__ void block_matmul(double2* Cm, const double2* A, const double2* B, int M, int K, int N) {
  const long long total = (long long)M * N;
  for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int r = (int)(idx / N), col = (int)(idx % N);
    const double2* a = A + (long long)r * K;
    double2 acc = cz();
    for (int k = 0; k < K; ++k) acc = cfma(a[k], B[(long long)k * N + col], acc);
    Cm[idx] = acc;
  }
}

// ------------------------------------------------------------------------- tableau (Sec. 2.3)
// Images are normalised to 4 x (x0, z0, x1, z1, r); for one qudit only generators 0, 1 are used
// and x1 = z1 = 0.

// lut[v] = exponents and phase of G W(v) G^dag for every local exponent vector v, where
// W(v) = X_q0^v0 Z_q0^v1 X_q1^v2 Z_q1^v3 and the images of the generators are s.img.  The product of
// images is accumulated with the Weyl rule  (tau^r W(a))(tau^r' W(b)) = tau^{r+r'+2 sum z(a) x(b)} W(a+b).
__device__ void lut_build(Smem& s, int nq, int d) {
  const int ng = 2 * nq;
  int nent = d * d;
  if (nq == 2) nent *= d * d;
  for (int v = threadIdx.x; v < nent; v += blockDim.x) {
    int dig[4] = {0, 0, 0, 0};
    int t = v;
    for (int k = ng - 1; k >= 0; --k) {
      dig[k] = t % d;
      t /= d;
    }
    int ax0 = 0, az0 = 0, ax1 = 0, az1 = 0, r = 0;
    for (int k = 0; k < ng; ++k) {
      const int* g = s.img + 5 * k;
      for (int p = 0; p < dig[k]; ++p) {
        r += g[4] + 2 * (az0 * g[0] + az1 * g[2]);
        ax0 = (ax0 + g[0]) % d;
        az0 = (az0 + g[1]) % d;
        ax1 = (ax1 + g[2]) % d;
        az1 = (az1 + g[3]) % d;
      }
    }
    uint8_t* o = s.lut + 5 * v;
    o[0] = (uint8_t)ax0;
    o[1] = (uint8_t)az0;
    o[2] = (uint8_t)ax1;
    o[3] = (uint8_t)az1;
    o[4] = (uint8_t)(r % (2 * d));
  }
  __syncthreads();
  // Inverse images: the unique v with G W(v) G^dag = tau^delta g_k gives G^dag g_k G = tau^{-delta} W(v).
  for (int v = threadIdx.x; v < nent; v += blockDim.x) {
    const uint8_t* o = s.lut + 5 * v;
    int hit = -1, cnt = 0;
    for (int k = 0; k < 4; ++k) {
      if (o[k]) {
        ++cnt;
        hit = (o[k] == 1) ? k : -2;
      }
    }
    if (cnt == 1 && hit >= 0 && hit < ng) {
      int dig[4] = {0, 0, 0, 0};
      int t = v;
      for (int k = ng - 1; k >= 0; --k) {
        dig[k] = t % d;
        t /= d;
      }
      int* w = s.inv + 5 * hit;
      for (int k = 0; k < 4; ++k) w[k] = dig[k];
      w[4] = (2 * d - o[4]) % (2 * d);
    }
  }
  __syncthreads();
}

// Conjugate every row of a tableau by the Clifford of s.lut on sites q0 (, q1).
__device__ void tab_apply_lut(Smem& s, uint8_t* X, uint8_t* R, int n, int d, int q0, int q1, int nq) {
  for (int row = threadIdx.x; row < 2 * n; row += blockDim.x) {
    uint8_t* e = X + (long long)row * 2 * n;
    int v = e[q0] * d + e[n + q0];
    if (nq == 2) v = (v * d + e[q1]) * d + e[n + q1];
    const uint8_t* o = s.lut + 5 * v;
    e[q0] = o[0];
    e[n + q0] = o[1];
    if (nq == 2) {
      e[q1] = o[2];
      e[n + q1] = o[3];
    }
    R[row] = (uint8_t)((R[row] + o[4]) % (2 * d));
  }
  __syncthreads();
}

// Replace the rows of the generators on (q0, q1) by products of the old rows: row(g_k) becomes
// tau^{r_k} prod_g row(g)^{v_k[g]} for the images (v_k, r_k) in s.inv (generator order
// X_q0, Z_q0, X_q1, Z_q1; row of X_q is n + q, of Z_q is q).
__device__ void tab_rowprod(Smem& s, uint8_t* X, uint8_t* R, int n, int d, int q0, int q1, int nq) {
  const int ng = 2 * nq;
  const int rowlen = 2 * n;
  for (int i = threadIdx.x; i < ng * rowlen; i += blockDim.x) {
    const int g = i / rowlen, j = i % rowlen;
    const int q = (g >> 1) ? q1 : q0;
    const int row = (g & 1) ? q : n + q;
    s.src[g][j] = X[(long long)row * rowlen + j];
  }
  if (threadIdx.x < ng) {
    const int g = threadIdx.x;
    const int q = (g >> 1) ? q1 : q0;
    s.srcr[g] = R[(g & 1) ? q : n + q];
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < ng) {
    constexpr int kPer = (kMaxN + 31) / 32;
    int ax[kPer], az[kPer];
#pragma unroll
    for (int t = 0; t < kPer; ++t) ax[t] = az[t] = 0;
    int r = s.inv[5 * w + 4];
    for (int g = 0; g < ng; ++g) {
      const int pw = s.inv[5 * w + g];
      for (int p = 0; p < pw; ++p) {
        int loc = 0;
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
          const int j = lane + 32 * t;
          if (j < n) loc += az[t] * s.src[g][j];
        }
        r += s.srcr[g] + 2 * warp_sum_int(loc);
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
          const int j = lane + 32 * t;
          if (j < n) {
            ax[t] = (ax[t] + s.src[g][j]) % d;
            az[t] = (az[t] + s.src[g][n + j]) % d;
          }
        }
      }
    }
    const int q = (w >> 1) ? q1 : q0;
    const int row = (w & 1) ? q : n + q;
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int j = lane + 32 * t;
      if (j < n) {
        X[(long long)row * rowlen + j] = (uint8_t)ax[t];
        X[(long long)row * rowlen + n + j] = (uint8_t)az[t];
      }
    }
    if (lane == 0) R[row] = (uint8_t)(((r % (2 * d)) + 2 * d) % (2 * d));
  }
  __syncthreads();
}

__device__ void load_images(Smem& s, const int32_t* img, int nq) {
  if (threadIdx.x < 20) {
    int v = 0;
    const int k = threadIdx.x / 5, f = threadIdx.x % 5;
    if (nq == 2) {
      v = img[threadIdx.x];
    } else if (k < 2) {
      if (f == 0) v = img[3 * k + 0];
      else if (f == 1) v = img[3 * k + 1];
      else if (f == 4) v = img[3 * k + 2];
    }
    s.img[threadIdx.x] = v;
    s.inv[threadIdx.x] = 0;
  }
  __syncthreads();
}

// C <- G C (Sec. 3, top loop of Fig. 3).  Forward rows are conjugated by G; the rows of the
// inverse tableau for G's sites become products of old rows via the images of G^{-1}.
__device__ void apply_clifford(Smem& s, const Ctx& C, int q0, int q1, const int32_t* img) {
  const int nq = (q1 < 0) ? 1 : 2;
  load_images(s, img, nq);
  lut_build(s, nq, C.d);
  tab_apply_lut(s, C.fx, C.fr, C.n, C.d, q0, q1, nq);
  tab_rowprod(s, C.ix, C.ir, C.n, C.d, q0, q1, nq);
  if (threadIdx.x == 0) C.stats[S_CLIFF] += 1;
}

// C <- C Q^dag (Sec. 3): the inverse rows are conjugated by Q, the forward rows of Q's sites
// become products of old rows via the images of Q^{-1}.
__device__ void fold_candidate(Smem& s, const Ctx& C, int k, int q0) {
  load_images(s, C.e->candImg + 20 * k, 2);
  lut_build(s, 2, C.d);
  tab_apply_lut(s, C.ix, C.ir, C.n, C.d, q0, q0 + 1, 2);
  tab_rowprod(s, C.fx, C.fr, C.n, C.d, q0, q0 + 1, 2);
}

// --------------------------------------------------------- one-sided Jacobi SVD (block level)
// Orthogonalises the n columns of B (m x n, column-major) by complex Jacobi rotations applied
// from the right, accumulating them in W (n x n, column-major, starts as I):  B_in W = B_out.
// Round-robin ordering: in each round the n/2 column pairs are disjoint and handled by the
// warps in parallel.  A pair is rotated while |b_i^H b_j| > 1e-14 |b_i| |b_j|, unless one of the
// two columns is numerically zero (|b|^2 <= 1e-30 |B|_F^2): the direction of such a column is
// rounding noise, rotating it never settles, and its singular value lies below any truncation
// cutoff.  Returns the number of sweeps, or -1 if `max_sweeps` were not enough.
__device__ int jacobi_orthogonalize(Smem& s, double2* B, int m, int n, double2* W, int max_sweeps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long i = threadIdx.x; i < (long long)n * n; i += blockDim.x)
    W[i] = ((i % n) == (i / n)) ? make_double2(1.0, 0.0) : cz();
  double fro = 0;
  for (long long i = threadIdx.x; i < (long long)m * n; i += blockDim.x) fro += cabs2(B[i]);
  fro = block_sum(fro, s);
  const double zero_col = 1e-30 * fro;
  const long long zc_bits = __double_as_longlong(zero_col);
  if (threadIdx.x == 0) s.flag = 0;
  __syncthreads();
  if (n <= 1) return 0;
  const int N = n + (n & 1);
  const int npairs = N / 2;
  const double tol2 = 1e-28;   // rotate while |b_i^H b_j| > 1e-14 |b_i| |b_j|
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < N - 1; ++round) {
      for (int p = warp; p < npairs; p += kWarps) {
        const int pa = (p == 0) ? 0 : 1 + ((p - 1 + round) % (N - 1));
        const int qa = 1 + ((N - 2 - p + round) % (N - 1));
        int i = pa < qa ? pa : qa, j = pa < qa ? qa : pa;
        if (j >= n) continue;
        double2* bi = B + (long long)i * m;
        double2* bj = B + (long long)j * m;
        double al = 0, be = 0, gr = 0, gi = 0;
        for (int r = lane; r < m; r += 32) {
          const double2 x = bi[r], y = bj[r];
          al = fma(x.x, x.x, fma(x.y, x.y, al));
          be = fma(y.x, y.x, fma(y.y, y.y, be));
          gr = fma(x.x, y.x, fma(x.y, y.y, gr));   // Re conj(x) y
          gi = fma(x.x, y.y, fma(-x.y, y.x, gi));  // Im conj(x) y
        }
        warp_sum4(al, be, gr, gi);
        // al, be >= 0: compared as integers (off the FP64 pipe)
        if (__double_as_longlong(al) <= zc_bits || __double_as_longlong(be) <= zc_bits) continue;
        const double g2 = fma(gr, gr, gi * gi);
        if (!(g2 > tol2 * al * be) || g2 < 1e-290) continue;   // |gamma| <= tol sqrt(al be)
        const double ig = rsqrt(g2);                            // 1 / |gamma|
        const double zeta = (be - al) * 0.5 * ig;
        const double t = fabs(zeta) < 1e150 ? copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)))
                                            : 0.5 / zeta;
        const double cs = rsqrt(fma(t, t, 1.0));
        const double sn = cs * t;
        const double2 e = make_double2(gr * ig, gi * ig);      // gamma / |gamma|
        const double2 se = cscale(e, sn), sec = cscale(cconj(e), sn);
        // b_i' = cs b_i - sn conj(e) b_j ; b_j' = sn e b_i + cs b_j
        for (int r = lane; r < m; r += 32) {
          const double2 x = bi[r], y = bj[r];
          bi[r] = csub(cscale(x, cs), cmul(sec, y));
          bj[r] = cadd(cmul(se, x), cscale(y, cs));
        }
        double2* wi = W + (long long)i * n;
        double2* wj = W + (long long)j * n;
        for (int r = lane; r < n; r += 32) {
          const double2 x = wi[r], y = wj[r];
          wi[r] = csub(cscale(x, cs), cmul(sec, y));
          wj[r] = cadd(cmul(se, x), cscale(y, cs));
        }
        if (lane == 0) s.flag = 1;
      }
      __syncthreads();
    }
    const int rotated = s.flag;
    __syncthreads();
    if (threadIdx.x == 0) s.flag = 0;
    __syncthreads();
    if (!rotated) return sweep + 1;
  }
  return -1;
}

__device__ __forceinline__ void cluster_sync() { cg::this_cluster().sync(); }

// jacobi_orthogonalize on the whole cluster of the circuit: the same rotations, pair order and stopping
// rule, with the column pairs of each round spread over the warps of every CTA and a cluster barrier between
// rounds (its release / acquire orders the global writes of one round before the reads of the next; B and W
// are read through L2).  On entry (after a cluster barrier) the leader has set W = I, lead->jfro = |B|_F^2 and
// lead->jflag[0] = lead->jflag[1] = 0.  Every CTA returns the number of sweeps, or -1 if max_sweeps were not
// enough.
__device__ __noinline__ int jacobi_cluster(Smem* lead, const Ctx& C, double2* B, int m, int n, double2* W, int max_sweeps) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (n <= 1) return 0;
  const double zero_col = 1e-30 * lead->jfro;
  const long long zc_bits = __double_as_longlong(zero_col);
  const int N = n + (n & 1);
  const int npairs = N / 2;
  const double tol2 = 1e-28;
  const int gw = C.rank * kWarps + warp, nw = C.csize * kWarps;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    bool any = false;
    for (int round = 0; round < N - 1; ++round) {
      for (int p = gw; p < npairs; p += nw) {
        const int pa = (p == 0) ? 0 : 1 + ((p - 1 + round) % (N - 1));
        const int qa = 1 + ((N - 2 - p + round) % (N - 1));
        const int i = pa < qa ? pa : qa, j = pa < qa ? qa : pa;
        if (j >= n) continue;
        double2* bi = B + (long long)i * m;
        double2* bj = B + (long long)j * m;
        double al = 0, be = 0, gr = 0, gi = 0;
        for (int r = lane; r < m; r += 32) {
          const double2 x = __ldcg(bi + r), y = __ldcg(bj + r);
          al = fma(x.x, x.x, fma(x.y, x.y, al));
          be = fma(y.x, y.x, fma(y.y, y.y, be));
          gr = fma(x.x, y.x, fma(x.y, y.y, gr));
          gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
        }
        warp_sum4(al, be, gr, gi);
        if (__double_as_longlong(al) <= zc_bits || __double_as_longlong(be) <= zc_bits) continue;
        const double g2 = fma(gr, gr, gi * gi);
        if (!(g2 > tol2 * al * be) || g2 < 1e-290) continue;
        const double ig = rsqrt(g2);
        const double zeta = (be - al) * 0.5 * ig;
        const double t = fabs(zeta) < 1e150 ? copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)))
                                            : 0.5 / zeta;
        const double cs = rsqrt(fma(t, t, 1.0));
        const double sn = cs * t;
        const double2 e = make_double2(gr * ig, gi * ig);
        const double2 se = cscale(e, sn), sec = cscale(cconj(e), sn);
        for (int r = lane; r < m; r += 32) {
          const double2 x = __ldcg(bi + r), y = __ldcg(bj + r);
          __stcg(bi + r, csub(cscale(x, cs), cmul(sec, y)));
          __stcg(bj + r, cadd(cmul(se, x), cscale(y, cs)));
        }
        double2* wi = W + (long long)i * n;
        double2* wj = W + (long long)j * n;
        for (int r = lane; r < n; r += 32) {
          const double2 x = __ldcg(wi + r), y = __ldcg(wj + r);
          __stcg(wi + r, csub(cscale(x, cs), cmul(sec, y)));
          __stcg(wj + r, cadd(cmul(se, x), cscale(y, cs)));
        }
        any = true;
      }
      cluster_sync();
    }
    // a rotation anywhere in the cluster: OR into the leader's flag of this sweep's parity
    if (lane == 0 && any) atomicOr(&lead->jflag[sweep & 1], 1);
    cluster_sync();
    const int rotated = lead->jflag[sweep & 1];
    // the other parity is set only after the next sweep's rounds (cluster barriers the leader passes too)
    if (C.rank == 0 && threadIdx.x == 0) lead->jflag[(sweep + 1) & 1] = 0;
    if (!rotated) return sweep + 1;
  }
  return -1;
}

// Singular values of the orthogonalised columns, sorted descending: sing[i] = |b_perm[i]|.
__device__ void sorted_column_norms(const double2* B, int m, int n, double* sv_tmp, double* sing, int* perm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = warp; j < n; j += kWarps) {
    double a = 0;
    for (int r = lane; r < m; r += 32) a += cabs2(B[(long long)j * m + r]);
    a = warp_sum(a);
    if (lane == 0) sv_tmp[j] = sqrt(a);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double v = sv_tmp[j];
    int rank = 0;
    for (int i = 0; i < n; ++i) {
      const double u = sv_tmp[i];
      rank += (u > v) || (u == v && i < j);
    }
    perm[rank] = j;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) sing[j] = sv_tmp[perm[j]];
  __syncthreads();
}

// Factor M (rows x cols, row-major) = U S Vh keeping the k largest singular values with
// s_i > cutoff * s_0 (at most cap, at least one).  U: rows x k, Vh: k x cols, both row-major in
// scratch; S in C.sing[0..k).  If renorm, S is rescaled to unit norm.  Returns k; *disc gets the
// discarded weight sum_{i>=k} s_i^2.
struct Factor {
  double2* U;
  double2* Vh;
  int k;
  double disc;
};

__device__ __noinline__ int block_qr(Smem& s, double2* B, int m, int n, double2* Q, double2* R, double* beta, double2* rdiag);

// When the long side is at least twice the short one, the long side is first reduced by a QR
// (B = Q R) and the Jacobi rotations act on the n x n factor R; the long factor is then Q times
// the orthogonalised columns of R.  The steps are svd_prepare (B and the QR), the Jacobi rotations
// (jacobi_orthogonalize on this CTA, or jacobi_cluster on the circuit's cluster) and svd_finish.
struct SvdPrep {
  bool tall, precond;
  int m, n, mm;   // B is m x n (column-major); the rotations act on its first mm rows (mm = n after the QR)
};

__device__ __noinline__ SvdPrep svd_prepare(Smem& s, const Ctx& C, const double2* M, int rows, int cols) {
  const Engine& e = *C.e;
  double2* B = C.scr + e.sl.b;
  double2* Vh = C.scr + e.sl.vh;
  double2* Qb = C.scr + e.sl.tmp;
  SvdPrep p;
  p.tall = rows >= cols;
  p.m = p.tall ? rows : cols;
  p.n = p.tall ? cols : rows;
  // B = M (tall) or M^H (wide), column-major m x n
  for (long long idx = threadIdx.x; idx < (long long)rows * cols; idx += blockDim.x) {
    const int r = (int)(idx / cols), c = (int)(idx % cols);
    if (p.tall) B[(long long)c * p.m + r] = M[idx];
    else B[(long long)r * p.m + c] = cconj(M[idx]);
  }
  __syncthreads();
  p.precond = p.n > 1 && p.m >= 2 * p.n;
  p.mm = p.m;
  if (p.precond) {
    block_qr(s, B, p.m, p.n, Qb, Vh, C.sing, reinterpret_cast<double2*>(C.sing + e.sing_stride / 2));
    __syncthreads();
    for (long long idx = threadIdx.x; idx < (long long)p.n * p.n; idx += blockDim.x) {
      const int i = (int)(idx / p.n), c = (int)(idx % p.n);
      B[(long long)c * p.n + i] = Vh[idx];
    }
    __syncthreads();
    p.mm = p.n;
  }
  return p;
}

__device__ __noinline__ Factor svd_finish(Smem& s, const Ctx& C, const SvdPrep& p, int sweeps, int rows, int cols,
                                          int cap, bool renorm) {
  const Engine& e = *C.e;
  double2* B = C.scr + e.sl.b;
  double2* W = C.scr + e.sl.w;
  double2* U = C.scr + e.sl.u;
  double2* Vh = C.scr + e.sl.vh;
  double2* Qb = C.scr + e.sl.tmp;
  double* sing = C.sing;
  double* svt = C.sing + e.sing_stride / 2;
  int* perm = C.perm;
  const bool tall = p.tall, precond = p.precond;
  const int m = p.m, n = p.n;
  if (threadIdx.x == 0) {
    if (sweeps < 0) set_failure(C, GCAMPS_ENOCONV, 1, rows, cols);
    const int sw = sweeps < 0 ? e.jacobi_cap : sweeps;
    C.stats[S_SVD] += 1;
    C.stats[S_JSWEEPS] += sw;
    if (sw > C.stats[S_JMAX]) C.stats[S_JMAX] = sw;
  }
  sorted_column_norms(B, p.mm, n, svt, sing, perm);
  // rank rule
  if (threadIdx.x == 0) {
    int k = 0;
    const double s0 = sing[0];
    if (s0 > 0) {
      while (k < n && sing[k] > e.cutoff * s0) ++k;
    }
    if (k > cap) k = cap;
    if (k < 1) k = 1;
    double kept = 0, drop = 0;
    for (int i = 0; i < n; ++i) (i < k ? kept : drop) += sing[i] * sing[i];
    s.ival[0] = k;
    s.dval[0] = drop;
    s.dval[1] = (renorm && kept > 0) ? 1.0 / sqrt(kept) : 1.0;
  }
  __syncthreads();
  const int k = s.ival[0];
  const double scale = s.dval[1];
  Factor F;
  F.U = U;
  F.Vh = Vh;
  F.k = k;
  F.disc = s.dval[0];
  // X[:, i] = (long side) orthogonalised column perm[i] / sigma_i, an m-vector
  for (long long idx = threadIdx.x; idx < (long long)m * k; idx += blockDim.x) {
    const int r = (int)(idx / k), i = (int)(idx % k);
    const int pj = perm[i];
    const double sv = sing[i];
    double2 x = cz();
    if (sv > 0) {
      if (precond) {
        const double2* col = B + (long long)pj * n;
        for (int t = 0; t < n; ++t) x = cfma(Qb[(long long)t * m + r], col[t], x);
      } else {
        x = B[(long long)pj * m + r];
      }
      x = cscale(x, 1.0 / sv);
    }
    if (tall) U[idx] = x;                              // U[r][i], r < rows
    else Vh[(long long)i * cols + r] = cconj(x);       // Vh[i][r], r < cols
  }
  if (tall) {
    for (long long idx = threadIdx.x; idx < (long long)k * cols; idx += blockDim.x) {
      const int i = (int)(idx / cols), c = (int)(idx % cols);
      Vh[idx] = cconj(W[(long long)perm[i] * n + c]);
    }
  } else {
    for (long long idx = threadIdx.x; idx < (long long)rows * k; idx += blockDim.x) {
      const int r = (int)(idx / k), i = (int)(idx % k);
      U[idx] = W[(long long)perm[i] * n + r];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) sing[i] *= scale;
  __syncthreads();
  return F;
}

// Factor M (rows x cols, row-major) = U S Vh keeping the k largest singular values with
// s_i > cutoff * s_0 (at most cap, at least one), on this CTA alone.
__device__ __noinline__ Factor svd_factor(Smem& s, const Ctx& C, const double2* M, int rows, int cols, int cap,
                                          bool renorm) {
  const Engine& e = *C.e;
  const SvdPrep p = svd_prepare(s, C, M, rows, cols);
  const int sweeps = jacobi_orthogonalize(s, C.scr + e.sl.b, p.mm, p.n, C.scr + e.sl.w, e.jacobi_cap);
  return svd_finish(s, C, p, sweeps, rows, cols, cap, renorm);
}

// ------------------------------------------------------------ Householder QR (block level)
// Reduced QR of B (m x n, column-major, overwritten): B = Q R with k = min(m, n); Q (m x k,
// column-major) in Q, R (k x n, row-major) in R.  Reflector k is H = I - beta v v^H with
// v = x + e^{i arg x_0} |x| e_1 on rows k..m-1 (x = column k), so H x = -e^{i arg x_0} |x| e_1.
// Columns handled by warps in parallel; no rank decision (the reduced Q keeps k columns).
__device__ __noinline__ int block_qr(Smem& s, double2* B, int m, int n, double2* Q, double2* R, double* beta, double2* rdiag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k = m < n ? m : n;
  // columns whose remaining part is below 1e-15 |B|_F are left unreflected (the reflector would
  // underflow); R keeps their diagonal entry and drops the rest (<= 1e-15 |B|_F)
  double fro = 0;
  for (long long i = threadIdx.x; i < (long long)m * n; i += blockDim.x) fro += cabs2(B[i]);
  fro = block_sum(fro, s);
  const double tiny = 1e-30 * fro;
  for (int j = 0; j < k; ++j) {
    double2* x = B + (long long)j * m;
    double nrm2 = 0;
    for (int r = j + threadIdx.x; r < m; r += blockDim.x) nrm2 += cabs2(x[r]);
    nrm2 = block_sum(nrm2, s);
    // the column's scalars on thread 0 alone (as in group_tridiag), published as beta (0: left unreflected)
    if (threadIdx.x == 0) {
      const double2 x0 = x[j];
      if (nrm2 <= tiny) {
        beta[j] = 0.0;
        rdiag[j] = x0;
        s.pub = 0.0;
      } else {
        const double s0 = fma(x0.x, x0.x, x0.y * x0.y);
        const bool fast = s0 > 0x1p-1000 && s0 < 0x1p+1000;
        const double rs = fast ? rsqrt(s0) : 0.0;
        const double ax0 = fast ? s0 * rs : hypot(x0.x, x0.y);
        const double alpha = sqrt(nrm2);
        const double2 ph = fast ? make_double2(x0.x * rs, x0.y * rs) : unit_phase(x0);
        const double b = 1.0 / (alpha * (alpha + ax0));
        x[j] = make_double2(x0.x + ph.x * alpha, x0.y + ph.y * alpha);
        beta[j] = b;
        rdiag[j] = make_double2(-ph.x * alpha, -ph.y * alpha);
        s.pub = b;
      }
    }
    __syncthreads();
    const double bt = s.pub;
    if (bt == 0.0) {
      __syncthreads();
      continue;
    }
    for (int c = j + 1 + warp; c < n; c += kWarps) {
      double2* y = B + (long long)c * m;
      double wr = 0, wi = 0;   // w = v^H y
      for (int r = j + lane; r < m; r += 32) {
        const double2 v = x[r], t = y[r];
        wr = fma(v.x, t.x, fma(v.y, t.y, wr));
        wi = fma(v.x, t.y, fma(-v.y, t.x, wi));
      }
      wr = warp_sum(wr) * bt;
      wi = warp_sum(wi) * bt;
      const double2 w = make_double2(wr, wi);
      for (int r = j + lane; r < m; r += 32) y[r] = csub(y[r], cmul(x[r], w));
    }
    __syncthreads();
  }
  // R (k x n, row-major)
  for (long long idx = threadIdx.x; idx < (long long)k * n; idx += blockDim.x) {
    const int i = (int)(idx / n), c = (int)(idx % n);
    R[idx] = (c < i) ? cz() : (c == i ? rdiag[i] : B[(long long)c * m + i]);
  }
  // Q = H_0 ... H_{k-1} [I_k; 0]
  for (long long idx = threadIdx.x; idx < (long long)m * k; idx += blockDim.x) {
    const int r = (int)(idx % m), c = (int)(idx / m);
    Q[idx] = (r == c) ? make_double2(1.0, 0.0) : cz();
  }
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double bt = beta[j];
    if (bt == 0.0) continue;
    const double2* x = B + (long long)j * m;
    for (int c = j + warp; c < k; c += kWarps) {
      double2* y = Q + (long long)c * m;
      double wr = 0, wi = 0;
      for (int r = j + lane; r < m; r += 32) {
        const double2 v = x[r], t = y[r];
        wr = fma(v.x, t.x, fma(v.y, t.y, wr));
        wi = fma(v.x, t.y, fma(-v.y, t.x, wi));
      }
      wr = warp_sum(wr) * bt;
      wi = warp_sum(wi) * bt;
      const double2 w = make_double2(wr, wi);
      for (int r = j + lane; r < m; r += 32) y[r] = csub(y[r], cmul(x[r], w));
    }
    __syncthreads();
  }
  return k;
}

// ---------------------------------------------------------------- canonical-form moves (Sec. 2.4)
__device__ void note_chi(const Ctx& C, int k) {
  if (threadIdx.x == 0 && k > C.stats[S_MAXCHI]) C.stats[S_MAXCHI] = k;
}

// Centre j -> j+1 without truncation (Sec. 2.4 canonical form): A_j = Q R (reduced QR of the
// (chi_l d) x chi_r matrix), A_j <- Q, A_{j+1} <- R A_{j+1}; the bond keeps min(chi_l d, chi_r).
__device__ void move_right(Smem& s, const Ctx& C, int j) {
  const Engine& e = *C.e;
  const int d = C.d;
  const int cl = C.dims[j], cr = C.dims[j + 1], cr2 = C.dims[j + 2];
  double2* A = site_ptr(C, j);
  double2* A2 = site_ptr(C, j + 1);
  double2* B = C.scr + e.sl.b;
  double2* Q = C.scr + e.sl.u;
  double2* R = C.scr + e.sl.vh;
  double2* tmp = C.scr + e.sl.tmp;
  const int m = cl * d, n = cr;
  for (long long idx = threadIdx.x; idx < (long long)m * n; idx += blockDim.x) {
    const int r = (int)(idx / n), c = (int)(idx % n);
    B[(long long)c * m + r] = A[idx];
  }
  __syncthreads();
  const int k = block_qr(s, B, m, n, Q, R, C.sing, reinterpret_cast<double2*>(C.sing + e.sing_stride / 2));
  if (threadIdx.x == 0) C.stats[S_QR] += 1;
  __syncthreads();
  for (long long idx = threadIdx.x; idx < (long long)m * k; idx += blockDim.x) {
    const int r = (int)(idx / k), c = (int)(idx % k);
    A[idx] = Q[(long long)c * m + r];
  }
  block_matmul(tmp, R, A2, k, n, d * cr2);
  __syncthreads();
  block_copy(A2, tmp, (long long)k * d * cr2);
  if (threadIdx.x == 0) {
    C.dims[j + 1] = k;
    C.meta[M_OC] = j + 1;
  }
  __syncthreads();
}

// Centre j -> j-1 without truncation: M = A_j (chi_l x d chi_r) = L Q from the QR of M^H
// (M^H = Q' R', M = R'^H Q'^H); A_j <- Q'^H, A_{j-1} <- A_{j-1} R'^H.
__device__ void move_left_qr(Smem& s, const Ctx& C, int j) {
  const Engine& e = *C.e;
  const int d = C.d;
  const int cl = C.dims[j], cr = C.dims[j + 1], cl2 = C.dims[j - 1];
  double2* A = site_ptr(C, j);
  double2* A0 = site_ptr(C, j - 1);
  double2* B = C.scr + e.sl.b;
  double2* Q = C.scr + e.sl.u;
  double2* R = C.scr + e.sl.vh;
  double2* tmp = C.scr + e.sl.tmp;
  double2* RH = C.scr + e.sl.w;
  const int m = d * cr, n = cl;   // M^H is m x n
  for (long long idx = threadIdx.x; idx < (long long)n * m; idx += blockDim.x) {
    const int a = (int)(idx / m), c = (int)(idx % m);      // M[a][c]
    B[(long long)a * m + c] = cconj(A[idx]);
  }
  __syncthreads();
  const int k = block_qr(s, B, m, n, Q, R, C.sing, reinterpret_cast<double2*>(C.sing + e.sing_stride / 2));
  if (threadIdx.x == 0) C.stats[S_QR] += 1;
  __syncthreads();
  for (long long idx = threadIdx.x; idx < (long long)k * m; idx += blockDim.x) {
    const int i = (int)(idx / m), c = (int)(idx % m);
    A[idx] = cconj(Q[(long long)i * m + c]);
  }
  for (long long idx = threadIdx.x; idx < (long long)n * k; idx += blockDim.x) {
    const int a = (int)(idx / k), i = (int)(idx % k);
    RH[idx] = cconj(R[(long long)i * n + a]);
  }
  __syncthreads();
  block_matmul(tmp, A0, RH, cl2 * d, n, k);
  __syncthreads();
  block_copy(A0, tmp, (long long)cl2 * d * k);
  if (threadIdx.x == 0) {
    C.dims[j] = k;
    C.meta[M_OC] = j - 1;
  }
  __syncthreads();
}

// Centre j -> j-1: A_j = U S Vh, A_j <- Vh, A_{j-1} <- A_{j-1} U S.  With truncation (cap, renorm)
// this is one step of the right-to-left compression sweep.
// The truncated SVD of M with its Jacobi rotations on the whole cluster when lead is given (the leader's
// shared memory, seen from the leader) and the matrix has at least kClusterJacobiMin Jacobi columns: the
// leader publishes the request (jmode 2 and the shape) and meets the cluster at one barrier, then every CTA
// runs jacobi_cluster.  Called by the leader only, while the other CTAs serve such requests (run_op).
__device__ Factor svd_factor_cluster(Smem& s, Smem* lead, const Ctx& C, const double2* M, int rows, int cols,
                                     int cap, bool renorm) {
  const Engine& e = *C.e;
  const SvdPrep p = svd_prepare(s, C, M, rows, cols);
  double2* B = C.scr + e.sl.b;
  double2* W = C.scr + e.sl.w;
  int sweeps;
  if (lead == nullptr || C.csize <= 1 || p.n < kClusterJacobiMin) {
    sweeps = jacobi_orthogonalize(s, B, p.mm, p.n, W, e.jacobi_cap);
  } else {
    for (long long idx = threadIdx.x; idx < (long long)p.n * p.n; idx += blockDim.x)
      W[idx] = ((idx % p.n) == (idx / p.n)) ? make_double2(1.0, 0.0) : cz();
    double fro = 0;
    for (long long idx = threadIdx.x; idx < (long long)p.mm * p.n; idx += blockDim.x) fro += cabs2(B[idx]);
    fro = block_sum(fro, s);
    if (threadIdx.x == 0) {
      s.jfro = fro;
      s.jflag[0] = s.jflag[1] = 0;
      s.jm = p.mm;
      s.jn = p.n;
      s.jmode = 2;
    }
    __syncthreads();
    cluster_sync();
    sweeps = jacobi_cluster(lead, C, B, p.mm, p.n, W, e.jacobi_cap);
  }
  return svd_finish(s, C, p, sweeps, rows, cols, cap, renorm);
}

__device__ double move_left(Smem& s, const Ctx& C, int j, int cap, bool renorm, Smem* lead = nullptr) {
  const int d = C.d;
  const int cl = C.dims[j], cr = C.dims[j + 1], cl2 = C.dims[j - 1];
  double2* A = site_ptr(C, j);
  double2* A0 = site_ptr(C, j - 1);
  const int bb = C.bond_bound[j];
  Factor F = lead ? svd_factor_cluster(s, lead, C, A, cl, d * cr, cap < bb ? cap : bb, renorm)
                  : svd_factor(s, C, A, cl, d * cr, cap < bb ? cap : bb, renorm);
  const int k = F.k;
  block_copy(A, F.Vh, (long long)k * d * cr);
  for (long long idx = threadIdx.x; idx < (long long)cl * k; idx += blockDim.x)
    F.U[idx] = cscale(F.U[idx], C.sing[idx % k]);
  __syncthreads();
  double2* tmp = C.scr + C.e->sl.tmp;
  block_matmul(tmp, A0, F.U, cl2 * d, cl, k);
  __syncthreads();
  block_copy(A0, tmp, (long long)cl2 * d * k);
  if (threadIdx.x == 0) {
    C.dims[j] = k;
    C.meta[M_OC] = j - 1;
  }
  __syncthreads();
  return F.disc;
}

__device__ void move_center(Smem& s, const Ctx& C, int target) {
  while (true) {
    const int oc = C.meta[M_OC];
    __syncthreads();
    if (oc < target) move_right(s, C, oc);
    else if (oc > target) move_left_qr(s, C, oc);
    else break;
  }
}

// ------------------------------------------------- non-Clifford step (Sec. 2.3.1, Sec. 2.4, Sec. 3)
// sum_m c_m P^m for a Weyl string P = tau^r (x)_j X_j^{x_j} Z_j^{z_j} (row: x in [0, n), z in [n, 2n))
// and base coefficients c_m in s.coef[0..d), applied to the circuit's MPS as an MPO of bond dimension
// d that is diagonal in m, over the support span [f, l] of P, then [f, l] recompressed (Sec. 2.4).
// (X^a Z^b)_{s s'} = omega^{b s'} delta_{s, s'+a}, so each MPO tensor is a gather with phases.
// record: this is the circuit's non-Clifford step (span, string and counters are kept); the adjoint
// passes false.  The identity string (f > l) sets EINVAL.
// lead: the leader's shared memory when the other CTAs of the cluster serve cluster-Jacobi requests during
// the step (run_op); null for a leader-only compression
__device__ __noinline__ void mpo_apply(Smem& s, const Ctx& C, const uint8_t* row, int r, bool record,
                                       Smem* lead = nullptr) {
  const int n = C.n, d = C.d;
  // support span and sum_j x_j z_j
  if (threadIdx.x == 0) {
    s.ival[0] = n;
    s.ival[1] = -1;
    s.ival[2] = 0;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int x = row[j], z = row[n + j];
    if (record) {
      C.weyl[j] = (int8_t)x;
      C.weyl[n + j] = (int8_t)z;
    }
    if (x | z) {
      atomicMin(&s.ival[0], j);
      atomicMax(&s.ival[1], j);
    }
    if (x * z) atomicAdd(&s.ival[2], x * z);
  }
  __syncthreads();
  const int f = s.ival[0], l = s.ival[1];
  const int sxz = s.ival[2] % d;
  __syncthreads();
  if (f > l) {  // a row of a valid tableau is never the identity
    if (threadIdx.x == 0) set_status(C, GCAMPS_EINVAL);
    __syncthreads();
    return;
  }
  if (threadIdx.x == 0) {
    if (record) {
      C.meta[M_WEYL_R] = r;
      C.meta[M_F] = f;
      C.meta[M_L] = l;
      C.meta[M_HAVE_SPAN] = 1;
      C.stats[S_T] += 1;
    }
    // the phase of P^m: (tau^r W)^m = tau^{r m} omega^{sxz m(m-1)/2} W(m x, m z)
    for (int m = 0; m < d; ++m) {
      const int ph = (r * m + 2 * sxz * (m * (m - 1) / 2)) % (2 * d);
      s.coef[m] = cmul(s.coef[m], s.tau[ph]);
    }
  }
  __syncthreads();
  // centre into [f, l]
  {
    int oc = C.meta[M_OC];
    __syncthreads();
    const int target = oc < f ? f : (oc > l ? l : oc);
    move_center(s, C, target);
  }
  double2* stage = C.scr + C.e->sl.theta;
  for (int j = f; j <= l; ++j) {
    const int cl = C.dims[j], cr = C.dims[j + 1];
    const int x = row[j], z = row[n + j];
    const double2* A = site_ptr(C, j);
    const bool first = (j == f), last = (j == l);
    const int ml = (first ? 1 : d), mr = (last ? 1 : d);
    const int ncl = cl * ml, ncr = cr * mr;
    const long long total = (long long)ncl * d * ncr;
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int B = (int)(idx % ncr);
      const int sidx = (int)((idx / ncr) % d);
      const int Aa = (int)(idx / ((long long)ncr * d));
      double2 v = cz();
      if (f == l) {
        for (int m = 0; m < d; ++m) {
          const int am = (m * x) % d, bm = (m * z) % d;
          const int sp = (sidx - am + d) % d;
          const double2 ph = s.tau[(2 * bm * sp) % (2 * d)];
          v = cadd(v, cmul(s.coef[m], cmul(ph, A[((long long)Aa * d + sp) * cr + B])));
        }
      } else {
        const int ml_idx = first ? -1 : Aa / cl;
        const int mr_idx = last ? -1 : B / cr;
        const int a = first ? Aa : Aa % cl;
        const int b = last ? B : B % cr;
        int m = first ? mr_idx : ml_idx;
        if (!first && !last && ml_idx != mr_idx) m = -1;
        if (m >= 0) {
          const int am = (m * x) % d, bm = (m * z) % d;
          const int sp = (sidx - am + d) % d;
          v = cmul(s.tau[(2 * bm * sp) % (2 * d)], A[((long long)a * d + sp) * cr + b]);
          if (first) v = cmul(s.coef[m], v);
        }
      }
      stage[idx] = v;
    }
    __syncthreads();
    block_copy(site_ptr(C, j), stage, total);
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int j = f + 1; j <= l; ++j) C.dims[j] *= d;
  __syncthreads();
  if (l > f) {
    // canonicalise [f, l] left to right from f, then truncate right to left
    if (threadIdx.x == 0) C.meta[M_OC] = f;
    __syncthreads();
    for (int j = f; j < l; ++j) move_right(s, C, j);
    double disc = 0;
    for (int j = l; j > f; --j) {
      disc += move_left(s, C, j, C.e->chi_max, true, lead);
      note_chi(C, C.dims[j]);
    }
    if (threadIdx.x == 0) {
      C.dstats[0] += disc;
      if (C.e->strict_weight > 0 && disc > C.e->strict_weight) set_status(C, GCAMPS_ECHI);
    }
  }
  __syncthreads();
}

// Snapshot of the MPS right after non-Clifford gate k (for the adjoint): the site tensors packed in the
// circuit's arena, and a header with the arena offset, the gate's site, the string's phase r, the
// first decision index of the disentangling that follows, the bond dimensions and the string.
__device__ void take_snapshot(Smem& s, const Ctx& C, int site, const double* phases) {
  const Engine& e = *C.e;
  const int n = C.n, d = C.d;
  const int k = C.meta[M_NSNAP];
  long long need = 0;
  for (int j = 0; j < n; ++j) need += (long long)C.dims[j] * d * C.dims[j + 1];
  const long long off = C.meta[M_SNAPOFF];
  __syncthreads();
  if (k >= e.snap_max || off + need > e.snap_stride) {
    if (threadIdx.x == 0) set_status(C, GCAMPS_ESNAP);
    __syncthreads();
    return;
  }
  int* hd = e.snap_hdr + ((long long)C.c * e.snap_max + k) * kSnapHdr;
  double2* dst = e.snap + (long long)C.c * e.snap_stride + off;
  long long pos = 0;
  for (int j = 0; j < n; ++j) {
    const long long nel = (long long)C.dims[j] * d * C.dims[j + 1];
    block_copy(dst + pos, site_ptr(C, j), nel);
    pos += nel;
  }
  const uint8_t* row = C.ix + (long long)site * 2 * n;
  for (int j = threadIdx.x; j <= n; j += blockDim.x) hd[kSnapDims + j] = C.dims[j];
  for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) hd[kSnapDims + kMaxN + 1 + j] = row[j];
  if (threadIdx.x == 0) {
    hd[0] = (int)off;
    hd[1] = site;
    hd[2] = C.ir[site];
    hd[3] = C.meta[M_NDEC];
    double* ph = e.snap_ph + ((long long)C.c * e.snap_max + k) * 4;
    for (int j = 0; j < d; ++j) ph[j] = phases[j];
    C.meta[M_NSNAP] = k + 1;
    C.meta[M_SNAPOFF] = (int)(off + need);
  }
  __syncthreads();
}

// Diagonal non-Clifford gate diag(e^{i phases[j]}) on `site`: P = C^dag Z_site C is row `site` of the
// inverse tableau; diag(t) = sum_m c_m Z^m with c_m = (1/d) sum_j t_j omega^{-mj}; C^dag diag(t) C =
// sum_m c_m P^m goes through mpo_apply.
__device__ void apply_nonclifford(Smem& s, Smem* lead, const Ctx& C, int site, const double* phases) {
  const int n = C.n, d = C.d;
  if (threadIdx.x == 0)
    for (int m = 0; m < d; ++m) {
      double re = 0, im = 0;
      for (int j = 0; j < d; ++j) {
        double sn, cs;
        sincos(phases[j] - 2.0 * CUDART_PI * (double)(m * j) / d, &sn, &cs);
        re += cs;
        im += sn;
      }
      s.coef[m] = make_double2(re / d, im / d);
    }
  __syncthreads();
  mpo_apply(s, C, C.ix + (long long)site * 2 * n, C.ir[site], true, lead);
  if (C.e->snap && C.meta[M_STATUS] == 0) take_snapshot(s, C, site, phases);
}

// --------------------------------------------------------------- candidate scoring (Sec. 3)
// The same routines run on a warp (small problems, one class per warp) or on a whole CTA (large
// problems, one class per CTA); the group type supplies the thread index, barrier and reduction.
struct WarpGroup {
  int tid;
  static constexpr int n = 32;
  __device__ void sync() const { __syncwarp(); }
  __device__ double sum(double v) const { return warp_sum(v); }
  __device__ float sumf(float v) const { return warp_sum_f(v); }
  __device__ double bcast(double v) const { return __shfl_sync(0xffffffffu, v, 0); }
  // thread 0's v (after its memory writes) to every thread of the group
  __device__ double publish(double v) const {
    __syncwarp();
    return __shfl_sync(0xffffffffu, v, 0);
  }
};
// Half a CTA: kThreads / 2 threads (warps 0-3 or 4-7, one warp per SM sub-partition), synchronised by the
// named barrier 1 + half, with its own partial-sum slots; two halves score two classes at once.
struct HalfGroup {
  Smem* s;
  int tid, n, half;
  __device__ void sync() const {   // immediate barrier ids: a register id would reserve all sixteen
    if (half == 0) asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
    else asm volatile("bar.sync 2, %0;" ::"r"(n) : "memory");
  }
  __device__ float sumf(float v) const {
    v = warp_sum_f(v);
    const int w = tid >> 5, l = tid & 31;
    sync();
    if (l == 0) s->redh[half][w] = v;
    sync();
    float t = l < kWarps / 2 ? s->redh[half][l] : 0.f;
#pragma unroll
    for (int o = kWarps / 4; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return __shfl_sync(0xffffffffu, t, 0);
  }
};
static_assert(kThreads == 32 * kWarps && kWarps >= 4, "two half-CTA groups of whole warps");

struct BlockGroup {
  Smem* s;
  int tid, n;
  __device__ void sync() const { __syncthreads(); }
  __device__ double sum(double v) const { return block_sum(v, *s); }
  __device__ float sumf(float v) const { return block_sum_f(v, *s); }
  __device__ double bcast(double v) const {
    __syncthreads();
    if (tid == 0) s->dval[2] = v;
    __syncthreads();
    const double r = s->dval[2];
    __syncthreads();
    return r;
  }
  // thread 0's v (after its memory writes) to every thread of the CTA, one barrier; the caller keeps
  // two publishes apart by at least one more barrier (no thread still reads the previous value)
  __device__ double publish(double v) const {
    if (tid == 0) s->pub = v;
    __syncthreads();
    return s->pub;
  }
};

// Householder reduction of a Hermitian m x m matrix (row-major, full storage, overwritten) to a
// real symmetric tridiagonal (diag dg, off-diagonal magnitudes od).  A column whose entries below
// the subdiagonal have norm below 1e-16 |A|_F is taken as already reduced (dropping them moves
// eigenvalues by at most that much).  Column k below the diagonal keeps the reflector v, row k right
// of it p and w.
template <class Grp>
__device__ void group_tridiag(const Grp& g, double2* A, int m, double* dg, double* od) {
  double fro2 = 0;
  for (int idx = g.tid; idx < m * m; idx += g.n) fro2 += cabs2(A[idx]);
  fro2 = g.sum(fro2);
  for (int k = 0; k + 2 < m; ++k) {
    const int r = m - k - 1;
    // the tail below x0 is summed on its own: |x|^2 - |x0|^2 cancels when x0 dominates and would
    // hide a small tail (which, inside a degenerate eigenspace, moves eigenvalues at first order)
    double tail2 = 0;
    for (int i = 1 + g.tid; i < r; i += g.n) tail2 += cabs2(A[(long long)(k + 1 + i) * m + k]);
    tail2 = g.sum(tail2);
    // the step's scalars on thread 0 alone (every warp computing them would put each FP64 pipe through
    // them twice): |x0|, alpha = |x|, the reflector's head x0 + phase(x0) alpha, h = v^H v / 2; published
    // as 1 / h, or -1 for a column that is already reduced
    double pub = 0.0;
    if (g.tid == 0) {
      const double2 x0 = A[(long long)(k + 1) * m + k];
      // |x0|^2 in the normal range: one reciprocal square root gives |x0| and the phase x0 / |x0| (each
      // within two units of the last place); outside it, hypot and unit_phase with their rescaling
      const double s0 = fma(x0.x, x0.x, x0.y * x0.y);
      const bool fast = s0 > 0x1p-1000 && s0 < 0x1p+1000;
      const double rs = fast ? rsqrt(s0) : 0.0;
      const double ax0 = fast ? s0 * rs : hypot(x0.x, x0.y);
      dg[k] = A[(long long)k * m + k].x;
      if (tail2 <= 1e-32 * fro2) {
        od[k] = ax0;
        pub = -1.0;
      } else {
        const double alpha = sqrt(tail2 + ax0 * ax0);
        const double2 ph = fast ? make_double2(x0.x * rs, x0.y * rs) : unit_phase(x0);
        A[(long long)(k + 1) * m + k] = make_double2(x0.x + ph.x * alpha, x0.y + ph.y * alpha);
        od[k] = alpha;
        pub = 1.0 / (alpha * (alpha + ax0));
      }
    }
    const double hinv = g.publish(pub);
    if (hinv < 0.0) {
      g.sync();
      continue;
    }
    // p = A v / h: kc lanes of one warp share a row (kc a power of two, kc r <= group size), each summing
    // every kc-th column, then a shuffle tree; every thread runs the same passes, so the shuffles see
    // full warps
    // kc chosen for the FP64 pipes: per pass of g.n / kc rows, the busiest pipe issues (its warps) x
    // (4 ceil(r / kc) + 2 log2 kc) FP64 instructions
    int kc = 1;
    {
      int best = 1 << 30;
      for (int q = 1, lg = 0; q <= 32 && q <= r; q *= 2, ++lg) {
        const int rif = g.n / q;
        if (rif < 1) break;
        int cost = 0;
        for (int b0 = 0; b0 < r; b0 += rif) {
          const int rows_p = r - b0 < rif ? r - b0 : rif;
          const int warps = (rows_p * q + 31) / 32;
          cost += ((warps + 3) / 4) * (4 * ((r + q - 1) / q) + 2 * lg);
        }
        if (cost < best) {
          best = cost;
          kc = q;
        }
      }
    }
    const int rows_in_flight = g.n / kc;
    for (int base = 0; base < r; base += rows_in_flight) {
      const int i = base + g.tid / kc, c = g.tid & (kc - 1);
      double2 acc = cz();
      if (i < r) {
        const double2* arow = A + (long long)(k + 1 + i) * m + (k + 1);
        for (int j = c; j < r; j += kc) acc = cfma(arow[j], A[(long long)(k + 1 + j) * m + k], acc);
      }
      for (int o = kc >> 1; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (i < r && c == 0) A[(long long)k * m + k + 1 + i] = cscale(acc, hinv);
    }
    g.sync();
    double kr = 0;
    for (int i = g.tid; i < r; i += g.n) {
      const double2 v = A[(long long)(k + 1 + i) * m + k], p = A[(long long)k * m + k + 1 + i];
      kr += v.x * p.x + v.y * p.y;
    }
    kr = g.sum(kr) * 0.5 * hinv;
    g.sync();
    for (int i = g.tid; i < r; i += g.n) {
      const double2 v = A[(long long)(k + 1 + i) * m + k], p = A[(long long)k * m + k + 1 + i];
      A[(long long)k * m + k + 1 + i] = make_double2(p.x - kr * v.x, p.y - kr * v.y);
    }
    g.sync();
    for (int idx = g.tid; idx < r * (r + 1) / 2; idx += g.n) {
      int i, j;
      tri_index(idx, i, j);
      const double2 vi = A[(long long)(k + 1 + i) * m + k], vj = A[(long long)(k + 1 + j) * m + k];
      const double2 wi = A[(long long)k * m + k + 1 + i], wj = A[(long long)k * m + k + 1 + j];
      // a - (vi conj(wj) + wi conj(vj)), as eight fused multiply-adds
      double2* a = A + (long long)(k + 1 + i) * m + (k + 1 + j);
      double2 nv = *a;
      nv.x = fma(-vi.x, wj.x, fma(-vi.y, wj.y, fma(-wi.x, vj.x, fma(-wi.y, vj.y, nv.x))));
      nv.y = fma(-vi.y, wj.x, fma(vi.x, wj.y, fma(-wi.y, vj.x, fma(wi.x, vj.y, nv.y))));
      *a = nv;
      if (j != i) A[(long long)(k + 1 + j) * m + (k + 1 + i)] = cconj(nv);
    }
    g.sync();
  }
  if (g.tid == 0) {
    if (m >= 2) {
      dg[m - 2] = A[(long long)(m - 2) * m + (m - 2)].x;
      const double2 e = A[(long long)(m - 1) * m + (m - 2)];
      od[m - 2] = hypot(e.x, e.y);
    }
    dg[m - 1] = A[(long long)(m - 1) * m + (m - 1)].x;
  }
  g.sync();
}

// Integer key with the order of the double v (no NaN): sorting keys sorts values, off the FP64 pipe.
__device__ __forceinline__ long long order_key(double v) {
  const long long b = __double_as_longlong(v);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}

// The smallest value of v over the warp, compared through order_key (integer work only).
__device__ __forceinline__ double warp_min_double(double v) {
  long long k = order_key(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long o2 = __shfl_xor_sync(0xffffffffu, k, o);
    k = o2 < k ? o2 : k;
  }
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffLL));
}
__device__ __forceinline__ int warp_min_int(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// Called by one whole warp: appends to list[start..] every k in [k0, K) with flag(k), in increasing k;
// returns the new length (the same on every lane).
template <class F>
__device__ __forceinline__ int warp_list(int* list, int start, int K, int k0, F flag) {
  const int lane = threadIdx.x & 31;
  int cnt = start;
  for (int base = k0; base < K; base += 32) {
    const int k = base + lane;
    const bool f = k < K && flag(k);
    const unsigned b = __ballot_sync(0xffffffffu, f);
    if (f) list[cnt + __popc(b & ((1u << lane) - 1u))] = k;
    cnt += __popc(b);
  }
  return cnt;
}

// Number of eigenvalues below x of the symmetric tridiagonal (dg, e2 = off-diagonal squared): the
// number of sign changes along the leading principal minors f_0 = 1, f_1, ..., f_m of T - x I,
// f_{i+1} = (d_i - x) f_i - e2_{i-1} f_{i-1} (Sturm sequence; a sign change is a negative LDL^T pivot
// f_{i+1} / f_i, Sylvester's law of inertia).  A minor that is exactly zero counts as a negative pivot
// (its sign is taken opposite to the previous one).  The pair (f_i, f_{i+1}) is rescaled by 2^-+500
// whenever the larger leaves [2^-500, 2^500]; scaling by a positive power of two changes no sign.
// Three FP64 instructions per step; the sign and exponent tests are integer operations.
__device__ __forceinline__ int sturm_count(const double* dg, const double* e2, int m, double x) {
  double f0 = 1.0, f1 = dg[0] - x;
  long long b1 = __double_as_longlong(f1);
  unsigned s1 = (b1 & 0x7fffffffffffffffLL) == 0 ? 1u : (unsigned)((unsigned long long)b1 >> 63);
  int cnt = (int)s1;
  for (int i = 1; i < m; ++i) {
    double f2 = fma(dg[i] - x, f1, -e2[i - 1] * f0);
    const long long b2 = __double_as_longlong(f2);
    const int ex1 = (int)((b1 >> 52) & 0x7ff), ex2 = (int)((b2 >> 52) & 0x7ff);
    const int ex = ex1 > ex2 ? ex1 : ex2;
    const bool out = ex > 1023 + 500 || ex < 1023 - 500;
    // a warp-uniform branch around the (rare) rescaling: predicated FP64 multiplies would still occupy
    // the FP64 pipe on every step
    if (__any_sync(__activemask(), out)) {
      if (ex > 1023 + 500) {
        f1 *= 3.054936363499605e-151;   // 2^-500
        f2 *= 3.054936363499605e-151;
      } else if (ex < 1023 - 500) {
        f1 *= 3.273390607896142e+150;   // 2^500
        f2 *= 3.273390607896142e+150;
      }
    }
    const long long c2 = __double_as_longlong(f2);
    const unsigned s2 = (c2 & 0x7fffffffffffffffLL) == 0 ? (s1 ^ 1u) : (unsigned)((unsigned long long)c2 >> 63);
    cnt += (int)(s2 != s1);
    s1 = s2;
    f0 = f1;
    f1 = f2;
    b1 = c2;
  }
  return cnt;
}

// det(T - x) and its derivative in x by the same three-term recurrence (f_i = (d_i - x) f_{i-1} -
// e_{i-1}^2 f_{i-2}, f'_i = (d_i - x) f'_{i-1} - f_{i-1} - e_{i-1}^2 f'_{i-2}), the four running values
// rescaled together by 2^-+500 when their largest exponent leaves [2^-500, 2^500]: f / f' is unchanged.
__device__ __forceinline__ void sturm_newton(const double* dg, const double* e2, int m, double x, double& f,
                                             double& fp) {
  double f0 = 1.0, f1 = dg[0] - x, g0 = 0.0, g1 = -1.0;
  for (int i = 1; i < m; ++i) {
    const double t = dg[i] - x;
    double f2 = fma(t, f1, -e2[i - 1] * f0);
    double g2 = fma(t, g1, -fma(e2[i - 1], g0, f1));
    const int ea = (int)((__double_as_longlong(f1) >> 52) & 0x7ff), eb = (int)((__double_as_longlong(f2) >> 52) & 0x7ff);
    const int ec = (int)((__double_as_longlong(g1) >> 52) & 0x7ff), ed = (int)((__double_as_longlong(g2) >> 52) & 0x7ff);
    const int ex = max(max(ea, eb), max(ec, ed));
    if (__any_sync(__activemask(), ex > 1023 + 500 || ex < 1023 - 500)) {   // rare: see sturm_count
      if (ex > 1023 + 500) {
        f1 *= 3.054936363499605e-151;   // 2^-500
        f2 *= 3.054936363499605e-151;
        g1 *= 3.054936363499605e-151;
        g2 *= 3.054936363499605e-151;
      } else if (ex < 1023 - 500) {
        f1 *= 3.273390607896142e+150;   // 2^500
        f2 *= 3.273390607896142e+150;
        g1 *= 3.273390607896142e+150;
        g2 *= 3.273390607896142e+150;
      }
    }
    f0 = f1;
    f1 = f2;
    g0 = g1;
    g1 = g2;
  }
  f = f1;
  fp = g1;
}

// FP32 version of sturm_count (rescaling by 2^-+40 outside [2^-40, 2^40]); it is exact for a matrix
// within a few FP32 units of T, which bounds the bracket it gives (see tridiag_bisect).
__device__ __forceinline__ int sturm_count32(const float* dg, const float* e2, int m, float x) {
  float f0 = 1.0f, f1 = dg[0] - x;
  int b1 = __float_as_int(f1);
  unsigned s1 = (b1 & 0x7fffffff) == 0 ? 1u : ((unsigned)b1 >> 31);
  int cnt = (int)s1;
  for (int i = 1; i < m; ++i) {
    float f2 = fmaf(dg[i] - x, f1, -e2[i - 1] * f0);
    const int b2 = __float_as_int(f2);
    const int ex1 = (b1 >> 23) & 0xff, ex2 = (b2 >> 23) & 0xff;
    const int ex = ex1 > ex2 ? ex1 : ex2;
    if (ex > 127 + 40) {
      f1 *= 9.094947017729282e-13f;   // 2^-40
      f2 *= 9.094947017729282e-13f;
    } else if (ex < 127 - 40) {
      f1 *= 1099511627776.0f;         // 2^40
      f2 *= 1099511627776.0f;
    }
    const int c2 = __float_as_int(f2);
    const unsigned s2 = (c2 & 0x7fffffff) == 0 ? (s1 ^ 1u) : ((unsigned)c2 >> 31);
    cnt += (int)(s2 != s1);
    s1 = s2;
    f0 = f1;
    f1 = f2;
    b1 = c2;
  }
  return cnt;
}

// Eigenvalues of a positive semidefinite tridiagonal (the reduced Gram) by multisection, P lanes per
// eigenvalue (see below): eigenvalue j (ascending) is where the Sturm count passes j.  The spectrum
// lies in [0, tr] (span = |tr|); each eigenvalue is located within 2^-50 span (an entropy error below
// 1e-12 for the Gram sizes used here).
//   sh, sh32: shared arrays of 2 cap entries for (diagonal | off-diagonal squared), or null.  With them
//   (m <= cap) FP32 steps worth 24 halvings first bracket eigenvalue j; since an FP32 Sturm count is
//   exact for a matrix within 8 FP32 units of span of T, the bracket padded by 40 units holds it, which
//   two FP64 counts confirm (else the full interval is used), and FP64 steps worth 33 halvings finish.
//   Without them, FP64 steps worth 50 halvings of [0, span] on the global arrays.
// Off-diagonal squares are at least 1e-300 span^2 (1e-20 span^2 in FP32), which moves no eigenvalue
// by more than 1e-150 span (1e-10 span, inside the FP32 padding) and keeps an exactly zero minor from
// zeroing the rest of the sequence.  od is overwritten with its squares; ev receives the m eigenvalues.
// m <= 2 in closed form.
template <class Grp>
__device__ void tridiag_bisect(const Grp& g, const double* dg, double* od, int m, double* ev, double* sh,
                               float* sh32, int cap) {
  if (m <= 2) {
    if (g.tid == 0) {
      if (m == 1) {
        ev[0] = dg[0];
      } else {
        const double mean = 0.5 * (dg[0] + dg[1]), r = hypot(0.5 * (dg[0] - dg[1]), od[0]);
        ev[0] = mean - r;
        ev[1] = mean + r;
      }
    }
    g.sync();
    return;
  }
  double tr = 0;
  for (int i = g.tid; i < m; i += g.n) tr += dg[i];
  tr = g.sum(tr);
  const double span = fabs(tr) + 1e-300;
  const double e2min = 1e-300 * span * span;
  const double gl = -4.440892098500626e-16 * span, gu = tr + 4.440892098500626e-16 * span;
  const bool fast = sh != nullptr && m <= cap;
  const double* D = dg;
  const double* E = od;
  if (fast) {
    const float e2min32 = (float)(1e-20 * span * span);
    for (int i = g.tid; i < m; i += g.n) {
      sh[i] = dg[i];
      sh32[i] = (float)dg[i];
      if (i + 1 < m) {
        const double e2 = fmax(od[i] * od[i], e2min);
        sh[cap + i] = e2;
        sh32[cap + i] = fmaxf((float)e2, e2min32);
      }
    }
    D = sh;
    E = sh + cap;
  } else {
    for (int i = g.tid; i + 1 < m; i += g.n) od[i] = fmax(od[i] * od[i], e2min);
  }
  g.sync();
  // Multisection: P lanes of a warp share eigenvalue j and count at P interior points of its
  // interval, which then shrinks by P + 1 per step (P as large as the group's warps allow).  All
  // lanes of a warp run the same number of steps (the group's outcome is combined by a ballot).
  // P is chosen for the FP64 pipes, not the lanes: a warp's Sturm step issues 3 FP64 instructions (64 cycles
  // of its sub-partition's pipe each) whatever its active lanes, and takes about 340 cycles alone (latency);
  // warps w, w + 4 of a CTA share one pipe.  The cost of P: passes over the eigenvalues x FP64 steps for P x
  // max(192 x the busiest pipe's warps, 340) (ties to the larger P)
  const int nw = (g.n + 31) / 32;
  constexpr int kIt64[9] = {0, 33, 21, 17, 15, 13, 12, 11, 11};   // ceil(33 / log2(P + 1))
  int P = 1;
  {
    int best = 1 << 30;
    for (int p = 8; p >= 1; --p) {
      const int pw = 32 / p, need = (m + pw - 1) / pw, passes = (need + nw - 1) / nw;
      const int busiest = passes > 1 ? (nw + 3) / 4 : (need + 3) / 4;
      const int cost = passes * kIt64[p] * max(192 * busiest, 340);
      if (cost < best) {
        best = cost;
        P = p;
      }
    }
  }
  const int per_warp = 32 / P;
  const int lane = g.tid & 31, warp = g.tid >> 5;
  const int grp = lane / P, pidx = lane % P;
  const unsigned gmask = ((1u << P) - 1u) << (grp < per_warp ? grp * P : 0);
  constexpr double kLog2[9] = {0.0, 1.0, 1.584962500721156, 2.0, 2.321928094887362, 2.584962500721156,
                               2.807354922057604, 3.0, 3.169925001442312};
  const int it32 = (int)ceil(24.0 / kLog2[P] - 1e-9);
  const int it64 = (int)ceil(33.0 / kLog2[P] - 1e-9);
  const int itfull = (int)ceil(50.0 / kLog2[P] - 1e-9);
  for (int base = 0; base < m; base += nw * per_warp) {
    const int jr = base + warp * per_warp + grp;
    const bool active = grp < per_warp && jr < m;
    const int j = active ? jr : 0;
    double lo = gl, hi = gu;
    int nit = itfull;
    if (fast) {
      float lo32 = (float)gl, hi32 = (float)gu;
      for (int it = 0; it < it32; ++it) {
        const float step = (hi32 - lo32) / (float)(P + 1);
        const float x = lo32 + (float)(pidx + 1) * step;
        const bool flag = active && sturm_count32(sh32, sh32 + cap, m, x) > j;
        const unsigned bits = (__ballot_sync(0xffffffffu, flag) & gmask) >> (grp < per_warp ? grp * P : 0);
        const int ps = bits ? __ffs(bits) - 1 : P;
        const float nlo = ps == 0 ? lo32 : lo32 + (float)ps * step;
        const float nhi = ps == P ? hi32 : lo32 + (float)(ps + 1) * step;
        lo32 = nlo;
        hi32 = nhi;
      }
      const double pad = 40.0 * 5.960464477539063e-08 * span;   // 40 FP32 units
      const double a = (double)lo32 - pad, b = (double)hi32 + pad;
      // FP64 counts at the padded ends (lane 0 of the group at a, lane 1 at b): ca <= j < cb confirms the
      // bracket, and cb - ca eigenvalues lie in it
      const int g0 = (lane / P) * P;
      int ca = 0, cb = m;
      if (P == 1) {
        if (active) {
          ca = sturm_count(D, E, m, a);
          cb = sturm_count(D, E, m, b);
        }
      } else {
        int c = 0;
        if (active && pidx < 2) c = sturm_count(D, E, m, pidx == 0 ? a : b);
        ca = __shfl_sync(0xffffffffu, c, g0);
        cb = __shfl_sync(0xffffffffu, c, g0 + 1);
      }
      if (__all_sync(0xffffffffu, !active || (ca <= j && cb > j))) {
        lo = a;
        hi = b;
        nit = it64;
      }
      // at m > 27 the small eigenvalues of decaying spectra share their FP32 brackets and the Newton
      // attempt below rarely verifies: the multisection alone is cheaper there
      if (m <= 27 && nit == it64) {
        // Newton steps on det(T - x) from the bracket's midpoint, the step times k = cb - ca (the root is
        // k-fold when the bracket holds a cluster far tighter than itself), kept inside [a, b].  Their
        // result stands for every eigenvalue of the warp if FP64 counts place each within tol = 2^-51 span
        // of it (the guarantee the multisection gives); otherwise the multisection below runs.
        const double tol = 4.440892098500626e-16 * span;
        const double k = active ? (double)(cb - ca) : 1.0;
        double x = active ? 0.5 * (a + b) : 0.0;
        bool bad = false;
        for (int it = 0; it < 4; ++it) {
          double f, fp;
          sturm_newton(D, E, m, x, f, fp);
          const double stp = k * f / fp;
          if (!(fabs(stp) < 1e300)) bad = true;   // f' = 0 or a non-finite value
          const double xn = bad ? x : fmin(fmax(x - stp, a), b);
          const bool conv = fabs(xn - x) <= 0.25 * tol;
          x = xn;
          if (__all_sync(0xffffffffu, !active || bad || conv)) break;
        }
        int vlo = 0, vhi = m;
        if (P == 1) {
          if (active && !bad) {
            vlo = sturm_count(D, E, m, x - tol);
            vhi = sturm_count(D, E, m, x + tol);
          }
        } else {
          int c = 0;
          if (active && pidx < 2) c = sturm_count(D, E, m, pidx == 0 ? x - tol : x + tol);
          vlo = __shfl_sync(0xffffffffu, c, g0);
          vhi = __shfl_sync(0xffffffffu, c, g0 + 1);
        }
        if (__all_sync(0xffffffffu, !active || (!bad && vlo <= j && vhi > j))) {
          if (active && pidx == 0) ev[j] = x;
          continue;
        }
      }
    }
    for (int it = 0; it < nit; ++it) {
      const double step = (hi - lo) / (double)(P + 1);
      const double x = lo + (double)(pidx + 1) * step;
      const bool flag = active && sturm_count(D, E, m, x) > j;
      const unsigned bits = (__ballot_sync(0xffffffffu, flag) & gmask) >> (grp < per_warp ? grp * P : 0);
      const int ps = bits ? __ffs(bits) - 1 : P;
      const double nlo = ps == 0 ? lo : lo + (double)ps * step;
      const double nhi = ps == P ? hi : lo + (double)(ps + 1) * step;
      lo = nlo;
      hi = nhi;
    }
    if (active && pidx == 0) ev[j] = 0.5 * (lo + hi);
  }
  g.sync();
}

struct Score {
  double s2, vn;
  int rank;   // eigenvalues above max(1e-12, 4 cutoff^2) tr G (von Neumann evaluations only)
  bool ok;
};

// One class Q on theta: theta' = Q theta over (a, s) x (t, b); its Gram G on the smaller side (lower
// triangle computed, mirrored); the Renyi-2 entropy S2 = -ln(|G|_F^2 / tr(G)^2); and, if asked, the
// von Neumann entropy -sum p ln p from the eigenvalues of G (p = lambda / tr G).  S2 <= S_vN always.
template <class Grp>
__device__ void gram_fp32(const Grp& g, const Ctx& C, const float2* X, int rows, int cols, float2* G);
template <class Grp>
__device__ __forceinline__ Score score_spectrum(const Grp& g, const Ctx& C, double2* G, int m, double tr, double fro,
                                                bool want_vn, double* dg, double* od, double* tri, float* tri32,
                                                int tricap, long long* xw = nullptr);

// The precision form's class evaluation: theta' = Q theta and its Gram in FP32 (tensor cores at CTA level),
// promoted to FP64 for the reduction, the eigenvalues and the score.  Kept out of line so that the FP64 path
// compiles as on its own.
template <class Grp>
__device__ __noinline__ Score score_class_fp32(const Grp& g, const Ctx& C, int cl, int cr, const float2* Q32,
                                               double2* ws, long long gram_off, bool want_vn, double* tri,
                                               float* tri32, int tricap) {
  const int d = C.d, dd = d * d;
  const int rows = cl * d, cols = d * cr;
  const int m = rows < cols ? rows : cols;
  double2* tp = ws;
  double2* G = ws + gram_off;
  double* dg = reinterpret_cast<double*>(G + (long long)m * m);
  double* od = dg + m;
  float2* X32 = reinterpret_cast<float2*>(tp);
  float2* G32 = X32 + (long long)rows * cols;
  for (int idx = g.tid; idx < rows * cols; idx += g.n) {
    const int rr = idx / cols, col = idx % cols;
    const int a = rr / d, sd = rr % d, t = col / cr, b = col % cr;
    const float2* q = Q32 + (sd * d + t) * dd;
    const float2* th = C.th32 + (long long)a * dd * cr + b;
    float2 acc = make_float2(0.f, 0.f);
    for (int v = 0; v < dd; ++v) acc = ffma2(q[v], th[(long long)v * cr], acc);
    X32[idx] = acc;
  }
  g.sync();
  gram_fp32(g, C, X32, rows, cols, G32);
  double tr = 0, fro = 0;
  for (int idx = g.tid; idx < m * m; idx += g.n) {
    const double2 v = make_double2((double)G32[idx].x, (double)G32[idx].y);
    G[idx] = v;
    if (idx / m == idx % m) tr += v.x;
    fro += cabs2(v);
  }
  tr = g.sum(tr);
  fro = g.sum(fro);
  return score_spectrum(g, C, G, m, tr, fro, want_vn, dg, od, tri, tri32, tricap);
}

template <class Grp>
__device__ Score score_class(const Grp& g, const Ctx& C, const double2* theta, int cl, int cr, const double2* Q,
                             const float2* Q32, double2* ws, long long gram_off, bool want_vn, double* tri,
                             float* tri32, int tricap) {
  const int d = C.d, dd = d * d;
  const int rows = cl * d, cols = d * cr;
  const int m = rows < cols ? rows : cols;
  double2* tp = ws;
  double2* G = ws + gram_off;
  double* dg = reinterpret_cast<double*>(G + (long long)m * m);
  double* od = dg + m;
  if (C.e->precision && m > kPruneMin && Q != C.e->candU)
    return score_class_fp32(g, C, cl, cr, Q32, ws, gram_off, want_vn, tri, tri32, tricap);
  // the leader's own exact evaluations, timed part by part (thread 0: warp 0's or the CTA's)
  long long* xw = (want_vn && C.prof && C.rank == 0 && threadIdx.x == 0)
                      ? C.prof + P_XPARTS + kXParts * (kProfBuckets * (g.n > 32 ? 1 : 0) + prof_bucket(m))
                      : nullptr;
  const long long tx0 = xw ? clock64() : 0;
  for (long long idx = g.tid; idx < (long long)rows * cols; idx += g.n) {
    const int rr = (int)(idx / cols), col = (int)(idx % cols);
    const int a = rr / d, sd = rr % d, t = col / cr, b = col % cr;
    const double2* q = Q + (sd * d + t) * dd;
    const double2* th = theta + (long long)a * dd * cr + b;
    double2 acc = cz();
    for (int u = 0; u < dd; ++u) acc = cfma(q[u], th[(long long)u * cr], acc);
    tp[idx] = acc;
  }
  g.sync();
  double tr = 0, fro = 0;
  const int ntri = m * (m + 1) / 2;
  for (int idx = g.tid; idx < ntri; idx += g.n) {
    int i, j;
    tri_index(idx, i, j);
    double2 acc = cz();
    if (rows <= cols) {
      const double2* ri = tp + (long long)i * cols;
      const double2* rj = tp + (long long)j * cols;
      for (int c = 0; c < cols; ++c) acc = cfmac(rj[c], ri[c], acc);   // sum_c ri conj(rj)
    } else {
      for (int r = 0; r < rows; ++r) acc = cfmac(tp[(long long)r * cols + i], tp[(long long)r * cols + j], acc);
    }
    G[(long long)i * m + j] = acc;
    if (i == j) {
      tr += acc.x;
      fro += acc.x * acc.x;
    } else {
      G[(long long)j * m + i] = cconj(acc);
      fro += 2.0 * cabs2(acc);
    }
  }
  tr = g.sum(tr);
  fro = g.sum(fro);
  if (xw) xw[2] += clock64() - tx0;
  const Score sc = score_spectrum(g, C, G, m, tr, fro, want_vn, dg, od, tri, tri32, tricap, xw);
  if (xw) {
    xw[0] += 1;
    xw[1] += clock64() - tx0;
  }
  return sc;
}

// S2 from the Gram's trace and squared Frobenius norm, and (want_vn) the von Neumann entropy and weight rank
// from its eigenvalues (FP64 Householder reduction, multisection).
template <class Grp>
__device__ __forceinline__ Score score_spectrum(const Grp& g, const Ctx& C, double2* G, int m, double tr, double fro,
                                                bool want_vn, double* dg, double* od, double* tri, float* tri32,
                                                int tricap, long long* xw) {
  Score sc;
  sc.ok = true;
  sc.s2 = (tr > 0.0 && fro > 0.0) ? -log(fro / (tr * tr)) : 0.0;
  sc.vn = sc.s2;
  sc.rank = -1;
  if (!want_vn) return sc;
  g.sync();
  long long tx = xw ? clock64() : 0;
  group_tridiag(g, G, m, dg, od);
  if (xw) {
    const long long now = clock64();
    xw[3] += now - tx;
    tx = now;
  }
  double* ev = reinterpret_cast<double*>(G);   // G is dead after the reduction
  tridiag_bisect(g, dg, od, m, ev, tri, tri32, tricap);
  if (xw) {
    const long long now = clock64();
    xw[4] += now - tx;
    tx = now;
  }
  // entropy -sum p ln p (p = lambda / tr) and the numerical rank, summed over the group
  double tot = 0;
  for (int i = g.tid; i < m; i += g.n) tot += fmax(ev[i], 0.0);
  tot = g.sum(tot);
  double ent = 0.0, rk = 0.0;
  if (tot > 0) {
    const double inv = 1.0 / tot;
    const double rthr = fmax(1e-12, 4.0 * C.e->cutoff * C.e->cutoff);
    for (int i = g.tid; i < m; i += g.n) {
      const double p = fmax(ev[i], 0.0) * inv;
      if (p > 0) ent -= p * log(p);
      if (p > rthr) rk += 1.0;
    }
  }
  sc.vn = g.sum(ent);
  sc.rank = (int)g.sum(rk);
  sc.ok = true;
  if (xw) xw[5] += clock64() - tx;
  return sc;
}

// Renyi-2 entropy of class Q on theta in FP32, and a lower bound on the exact value.  theta' = Q theta
// (FP32 inputs, d^2-term sums) is off by at most e1 |theta|_F with e1 = d (d^2 + 6) u (u = 2^-24),
// and the Gram on the smaller side (sums of 2M + 4 rounded terms, M the longer side) by at most
// (2M + 4) u |theta'|_F^2, so |G^ - G|_F <= eta tr G with eta = 2 e1 + e1^2 + (2M + 4) u (1 + e1)^2;
// the same bound holds for the trace.  Then |ln |G^|_F - ln |G|_F| <= eta tr / |G|_F <= eta sqrt(m) and
// |ln tr^ - ln tr| <= eta, so |S2^ - S2| <= 2 eta sqrt(m) + 2 eta.  The lower bound subtracts twice that
// plus the rounding of the partial sums.  Outside 1e-12 < tr < 1e12 (where FP32 squares of the Gram
// entries could underflow or overflow and break the bound) the lower bound is 0 (S2 >= 0).
template <class Grp>
__device__ void s2_fp32(const Grp& g, const Ctx& C, const float2* th, int cl, int cr, const float2* Q, float2* X,
                        double* s2_out, double* lo_out) {
  const int d = C.d, dd = d * d;
  const int rows = cl * d, cols = d * cr;
  const int m = rows < cols ? rows : cols, M = rows < cols ? cols : rows;
  for (int idx = g.tid; idx < rows * cols; idx += g.n) {
    const int rr = idx / cols, col = idx % cols;
    const int a = rr / d, sd = rr % d, t = col / cr, b = col % cr;
    const float2* q = Q + (sd * d + t) * dd;
    const float2* tp = th + (long long)a * dd * cr + b;
    float2 acc = make_float2(0.f, 0.f);
    for (int v = 0; v < dd; ++v) acc = ffma2(q[v], tp[(long long)v * cr], acc);
    X[idx] = acc;
  }
  g.sync();
  float tr = 0.f, fro = 0.f;
  const int ntri = m * (m + 1) / 2;
  for (int idx = g.tid; idx < ntri; idx += g.n) {
    int i, j;
    tri_index(idx, i, j);
    float2 acc = make_float2(0.f, 0.f);
    if (rows <= cols) {
      const float2* ri = X + (long long)i * cols;
      const float2* rj = X + (long long)j * cols;
      for (int c = 0; c < cols; ++c) acc = ffmac2(ri[c], rj[c], acc);
    } else {
      for (int r = 0; r < rows; ++r) acc = ffmac2(X[(long long)r * cols + i], X[(long long)r * cols + j], acc);
    }
    if (i == j) {
      tr += acc.x;
      fro = fmaf(acc.x, acc.x, fro);
    } else {
      fro = fmaf(2.f * acc.x, acc.x, fmaf(2.f * acc.y, acc.y, fro));
    }
  }
  // group sums and the final logarithms in FP32 (valid on the group's first thread, the one that stores
  // them); their rounding is inside the bound: 96 u for the sums and 4 u (|ln fro| + 2 |ln tr| + 2) for logf
  tr = g.sumf(tr);
  fro = g.sumf(fro);
  if (g.tid != 0) return;
  float s2 = 0.f, lo = 0.f;
  if (tr > 1e-12f && tr < 1e12f && fro > 0.f) {
    const float u = 5.9604645e-08f;
    const float e1 = d * (dd + 6) * u;
    const float eta = (2.f * e1 + e1 * e1 + (2.f * M + 4.f) * u * (1.f + e1) * (1.f + e1)) * 1.0001f;
    const float lf = logf(fro), lt = logf(tr);
    const float delta = 4.f * eta * sqrtf((float)m) * 1.0001f + 4.f * eta + ((float)m * m / 16.f + 112.f) * u +
                        4.f * u * (fabsf(lf) + 2.f * fabsf(lt) + 2.f);
    s2 = 2.f * lt - lf;
    lo = s2 - delta;
  }
  *s2_out = s2;
  *lo_out = lo;
}

// ------------------------------------------- FP32 von Neumann estimate with an error bound (Sec. 3 score)
// Bound on |S^ - S_vN| for vn_est32 on a class of a theta with m = min side, M = max side.  The Gram of the
// FP32 theta' is within eta tr G of the exact one (as for the screen); scaling it to unit trace adds u; the
// FP32 Householder reduction is backward stable, its eigenvalues being those of G^ + E, modelled here as
// |E|_F <= 2 m^2 u |G^|_F (m - 2 reflectors, each applied on both sides within about m u of the matrix
// norm), with |G^|_F <= (1 + eta) tr G; the FP32 multisection adds at most 9 u tr per eigenvalue.  By
// Hoffman-Wielandt and Cauchy-Schwarz the l1 distance of the spectra is at most sqrt(m) times the Frobenius
// error; normalising by the estimated sum at most doubles it, so the trace distance of the normalised
// spectra is T <= sqrt(m) (eta + u + 2 m^2 u (1 + eta)) + 9 m u, and Fannes-Audenaert gives
// |S^ - S| <= T ln(m - 1) + H2(T).  The bound used is twice that with ln m (room for the rounding of S^
// itself); 1e300 (no information) when T >= 1/2.
__device__ double vn_est_bound(int d, int m, int M) {
  // evaluated in FP32 (off the narrow FP64 pipe) and rounded up by 0.1 %, far more than its rounding error
  const float u = 5.9604645e-08f;
  const float e1 = d * (d * d + 6) * u;
  const float eta = 2.f * e1 + e1 * e1 + (2.f * M + 4.f) * u * (1.f + e1) * (1.f + e1);
  const float T = (sqrtf((float)m) * (eta + u + 2.f * (float)m * (float)m * u * (1.f + eta)) + 9.f * m * u) * 1.001f;
  if (!(T < 0.5f)) return 1e300;
  const float h2 = T > 0.f ? -T * logf(T) - (1.f - T) * log1pf(-T) : 0.f;
  return (double)(2.f * (T * logf((float)(m > 1 ? m : 2)) + h2) * 1.001f);
}

__device__ __forceinline__ float fabs2f(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// Householder reduction of a Hermitian m x m matrix (FP32, row-major, full storage, overwritten) to a real
// symmetric tridiagonal (diag dg, off-diagonal magnitudes od) on a warp or a CTA; the reflections of
// group_tridiag, arranged for latency: the reflector v and w = p - K v live in shared memory (hv, hw: at
// least m - 1 entries), the product p = A v is taken as p_i = sum_j conj(A_ji) v_j (consecutive rows,
// coalesced) with four independent accumulators, and the rank-2 update covers the whole trailing block, a
// warp per row.  A column whose part below the subdiagonal has norm below 1e-10 |A|_F is taken as reduced
// (far below FP32 rounding).
template <class Grp>
__device__ void tridiag32(const Grp& g, float2* A, int m, float* dg, float* od, float2* hv, float2* hw) {
  const int tid = g.tid, nt = g.n, lane = tid & 31, wid = tid >> 5, nwarps = (nt + 31) >> 5;
  float fro2 = 0.f;
  for (int idx = tid; idx < m * m; idx += nt) fro2 += fabs2f(A[idx]);
  fro2 = g.sumf(fro2);
  for (int k = 0; k + 2 < m; ++k) {
    const int r = m - k - 1;
    float tail2 = 0.f;
    for (int i = tid; i < r; i += nt) {
      const float2 x = A[(long long)(k + 1 + i) * m + k];
      hv[i] = x;
      if (i > 0) tail2 += fabs2f(x);
    }
    g.sync();
    tail2 = g.sumf(tail2);
    const float2 x0 = hv[0];
    const float ax0 = hypotf(x0.x, x0.y);
    if (tid == 0) dg[k] = A[(long long)k * m + k].x;
    if (tail2 <= 1e-20f * fro2) {
      if (tid == 0) od[k] = ax0;
      g.sync();
      continue;
    }
    const float alpha = sqrtf(fmaf(ax0, ax0, tail2));
    const float2 ph = ax0 > 0.f ? make_float2(x0.x / ax0, x0.y / ax0) : make_float2(1.f, 0.f);
    const float hinv = 1.f / (alpha * (alpha + ax0));   // 2 / v^H v
    g.sync();
    if (tid == 0) hv[0] = make_float2(fmaf(ph.x, alpha, x0.x), fmaf(ph.y, alpha, x0.y));
    g.sync();
    // p_i = hinv sum_j conj(A_(k+1+j),(k+1+i)) v_j: thread i walks down column k+1+i
    for (int i = tid; i < r; i += nt) {
      const float2* col = A + (long long)(k + 1) * m + (k + 1 + i);
      float ax[4] = {0.f, 0.f, 0.f, 0.f}, ay[4] = {0.f, 0.f, 0.f, 0.f};
      int j = 0;
      for (; j + 4 <= r; j += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 a = col[(long long)(j + u) * m], v = hv[j + u];
          ax[u] = fmaf(a.x, v.x, fmaf(a.y, v.y, ax[u]));    // Re conj(a) v
          ay[u] = fmaf(a.x, v.y, fmaf(-a.y, v.x, ay[u]));   // Im conj(a) v
        }
      }
      for (; j < r; ++j) {
        const float2 a = col[(long long)j * m], v = hv[j];
        ax[0] = fmaf(a.x, v.x, fmaf(a.y, v.y, ax[0]));
        ay[0] = fmaf(a.x, v.y, fmaf(-a.y, v.x, ay[0]));
      }
      hw[i] = make_float2(((ax[0] + ax[1]) + (ax[2] + ax[3])) * hinv, ((ay[0] + ay[1]) + (ay[2] + ay[3])) * hinv);
    }
    g.sync();
    float kr = 0.f;
    for (int i = tid; i < r; i += nt) {
      const float2 v = hv[i], p = hw[i];
      kr = fmaf(v.x, p.x, fmaf(v.y, p.y, kr));
    }
    const float krf = g.sumf(kr) * 0.5f * hinv;
    for (int i = tid; i < r; i += nt) {
      const float2 v = hv[i], p = hw[i];
      hw[i] = make_float2(fmaf(-krf, v.x, p.x), fmaf(-krf, v.y, p.y));
    }
    g.sync();
    // A22 <- A22 - v w^H - w v^H, a warp per row, lanes along the row
    for (int i = wid; i < r; i += nwarps) {
      const float2 vi = hv[i], wi = hw[i];
      float2* arow = A + (long long)(k + 1 + i) * m + (k + 1);
      for (int j = lane; j < r; j += 32) {
        const float2 vj = hv[j], wj = hw[j];
        float2 nv = arow[j];
        nv.x = fmaf(-vi.x, wj.x, fmaf(-vi.y, wj.y, fmaf(-wi.x, vj.x, fmaf(-wi.y, vj.y, nv.x))));
        nv.y = fmaf(-vi.y, wj.x, fmaf(vi.x, wj.y, fmaf(-wi.y, vj.x, fmaf(wi.x, vj.y, nv.y))));
        arow[j] = nv;
      }
    }
    if (tid == 0) od[k] = alpha;
    g.sync();
  }
  if (tid == 0) {
    if (m >= 2) {
      dg[m - 2] = A[(long long)(m - 2) * m + (m - 2)].x;
      const float2 e = A[(long long)(m - 1) * m + (m - 2)];
      od[m - 2] = hypotf(e.x, e.y);
    }
    dg[m - 1] = A[(long long)(m - 1) * m + (m - 1)].x;
  }
  g.sync();
}

// Eigenvalues of a real symmetric tridiagonal (dg, off-diagonal magnitudes od; od is overwritten with its
// squares) in FP32 on a warp or a CTA: multisection on FP32 Sturm counts, P lanes per eigenvalue, over
// [-R, R] (R >= spectral radius) until the bracket is below R 2^-24; ev receives the m eigenvalues
// (ascending).  sh: 2 cap shared floats used when m <= cap.
template <class Grp>
__device__ void tridiag_eig32(const Grp& g, const float* dg, float* od, int m, float* ev, float* sh, int cap) {
  const int tid = g.tid, nt = g.n;
  if (m <= 2) {
    if (tid == 0) {
      if (m == 1) {
        ev[0] = dg[0];
      } else {
        const float mean = 0.5f * (dg[0] + dg[1]), r = hypotf(0.5f * (dg[0] - dg[1]), od[0]);
        ev[0] = mean - r;
        ev[1] = mean + r;
      }
    }
    g.sync();
    return;
  }
  // [-R, R] with R the Frobenius norm of T (it bounds the spectral radius), widened by 0.1 % for its rounding
  float f2 = 0.f;
  for (int i = tid; i < m; i += nt) f2 = fmaf(dg[i], dg[i], i + 1 < m ? fmaf(2.f * od[i], od[i], f2) : f2);
  const float R = sqrtf(g.sumf(f2)) * 1.001f + 1e-30f;
  const float e2min = 1e-20f * R * R;
  const bool fast = m <= cap;
  float* D = fast ? sh : const_cast<float*>(dg);
  float* E = fast ? sh + cap : od;
  for (int i = tid; i < m; i += nt) {
    const float e2 = i + 1 < m ? fmaxf(od[i] * od[i], e2min) : 0.f;
    if (fast) D[i] = dg[i];
    E[i] = e2;
  }
  g.sync();
  const int nw = (nt + 31) / 32;
  int P = 1;
  for (int p = 8; p >= 1; --p)
    if (nw * (32 / p) >= m) {
      P = p;
      break;
    }
  const int per_warp = 32 / P;
  const int lane = tid & 31, warp = tid >> 5;
  const int grp = lane / P, pidx = lane % P;
  const unsigned gmask = ((1u << P) - 1u) << (grp < per_warp ? grp * P : 0);
  constexpr float kLog2f[9] = {0.f, 1.f, 1.5849625f, 2.f, 2.3219281f, 2.5849625f, 2.8073549f, 3.f, 3.169925f};
  const int it32 = (int)ceilf(25.0f / kLog2f[P] - 1e-4f);   // 2R shrinks to below R 2^-24
  for (int base = 0; base < m; base += nw * per_warp) {
    const int jr = base + warp * per_warp + grp;
    const bool active = grp < per_warp && jr < m;
    const int j = active ? jr : 0;
    float lo = -R, hi = R;
    for (int it = 0; it < it32; ++it) {
      const float step = (hi - lo) / (float)(P + 1);
      const float x = lo + (float)(pidx + 1) * step;
      const bool flag = active && sturm_count32(D, E, m, x) > j;
      const unsigned bits = (__ballot_sync(0xffffffffu, flag) & gmask) >> (grp < per_warp ? grp * P : 0);
      const int ps = bits ? __ffs(bits) - 1 : P;
      const float nlo = ps == 0 ? lo : lo + (float)ps * step;
      const float nhi = ps == P ? hi : lo + (float)(ps + 1) * step;
      lo = nlo;
      hi = nhi;
    }
    if (active && pidx == 0) ev[j] = 0.5f * (lo + hi);
  }
  g.sync();
}

// FP32 estimate of the von Neumann entropy of class Q on theta (a warp or a CTA), whose error vn_est_bound
// bounds: theta' = Q theta and its Gram on the smaller side in FP32, scaled to unit trace, tridiagonalised
// and its eigenvalues found in FP32; -sum p ln p of the eigenvalues clipped at 0 and normalised by their
// sum, in FP32 (its rounding, of order m u ln m, is covered by the factor 2 of the bound).  From the same
// Gram, the Renyi-2 entropy and its lower bound as s2_fp32 computes them (s2 may be NULL).  Returns false
// (no estimate; s2 and its bound still set) outside 1e-12 < tr G < 1e12, the FP32 range of the Gram's
// squares, or for m above the reflector buffers (hcap).  Values are valid on the group's first thread.
// ws: rows cols + m^2 + 3 m float2 of scratch; sh: 2 shcap floats of shared memory.
template <class Grp>
__device__ __noinline__ bool vn_est32(const Grp& g, const Ctx& C, const float2* th, int cl, int cr, const float2* Q,
                                      float2* ws, float2* hv, float2* hw, int hcap, float* sh, int shcap,
                                      float* est_out, float* s2_out, float* s2lo_out) {
  const int d = C.d, dd = d * d;
  const int rows = cl * d, cols = d * cr;
  const int m = rows < cols ? rows : cols, M = rows < cols ? cols : rows;
  const int tid = g.tid, nt = g.n;
  float2* X = ws;
  float2* G = ws + (long long)rows * cols;
  float* dg = reinterpret_cast<float*>(G + (long long)m * m);
  float* od = dg + m;
  float* ev = od + m;
  for (int idx = tid; idx < rows * cols; idx += nt) {
    const int rr = idx / cols, col = idx % cols;
    const int a = rr / d, sd = rr % d, t = col / cr, b = col % cr;
    const float2* q = Q + (sd * d + t) * dd;
    const float2* tp = th + (long long)a * dd * cr + b;
    float2 acc = make_float2(0.f, 0.f);
    for (int v = 0; v < dd; ++v) acc = ffma2(q[v], tp[(long long)v * cr], acc);
    X[idx] = acc;
  }
  g.sync();
  float tr = 0.f, fro = 0.f;
  const int ntri = m * (m + 1) / 2;
  for (int idx = tid; idx < ntri; idx += nt) {
    int i, j;
    tri_index(idx, i, j);
    float2 acc = make_float2(0.f, 0.f);
    if (rows <= cols) {
      const float2* ri = X + (long long)i * cols;
      const float2* rj = X + (long long)j * cols;
      for (int c = 0; c < cols; ++c) acc = ffmac2(ri[c], rj[c], acc);
    } else {
      for (int r = 0; r < rows; ++r) acc = ffmac2(X[(long long)r * cols + i], X[(long long)r * cols + j], acc);
    }
    G[(long long)i * m + j] = acc;
    if (i == j) {
      tr += acc.x;
      fro = fmaf(acc.x, acc.x, fro);
    } else {
      G[(long long)j * m + i] = make_float2(acc.x, -acc.y);
      fro = fmaf(2.f * acc.x, acc.x, fmaf(2.f * acc.y, acc.y, fro));
    }
  }
  tr = g.sumf(tr);
  fro = g.sumf(fro);
  const bool in_range = tr > 1e-12f && tr < 1e12f && fro > 0.f;
  if (s2_out && tid == 0) {   // the screen's value and lower bound (s2_fp32)
    float s2 = 0.f, lo = 0.f;
    if (in_range) {
      const float u = 5.9604645e-08f;
      const float e1 = d * (dd + 6) * u;
      const float eta = (2.f * e1 + e1 * e1 + (2.f * M + 4.f) * u * (1.f + e1) * (1.f + e1)) * 1.0001f;
      const float lf = logf(fro), lt = logf(tr);
      const float delta = 4.f * eta * sqrtf((float)m) * 1.0001f + 4.f * eta + ((float)m * m / 16.f + 112.f) * u +
                          4.f * u * (fabsf(lf) + 2.f * fabsf(lt) + 2.f);
      s2 = 2.f * lt - lf;
      lo = s2 - delta;
    }
    *s2_out = s2;
    *s2lo_out = lo;
  }
  if (!in_range || m - 1 > hcap) return false;
  const float sc = 1.f / tr;
  for (int idx = tid; idx < m * m; idx += nt) G[idx] = make_float2(G[idx].x * sc, G[idx].y * sc);
  g.sync();
  tridiag32(g, G, m, dg, od, hv, hw);
  tridiag_eig32(g, dg, od, m, ev, sh, shcap);
  float tot = 0.f;
  for (int i = tid; i < m; i += nt) tot += fmaxf(ev[i], 0.f);
  tot = g.sumf(tot);
  float ent = 0.f;
  if (tot > 0.f) {
    const float inv = 1.f / tot;
    for (int i = tid; i < m; i += nt) {
      const float p = fmaxf(ev[i], 0.f) * inv;
      if (p > 0.f) ent = fmaf(-p, logf(p), ent);
    }
  }
  ent = g.sumf(ent);
  *est_out = ent;
  return true;
}

// ------------------------------------------------------------ tensor-core Gram (tcgen05, kind::tf32)
// G = X X^H (rows <= cols) or X^T conj(X) (rows > cols), m x m on the smaller side, of X (rows x cols
// complex FP32, row-major) as one real product D = A B^T on the tensor cores: A (128 x 2K) holds the m rows
// of X as interleaved (re, im), B (N x 2K, N = 2m padded to 16) holds them and, in rows m..2m-1, the rows
// times i ((-im, re)), so that D[i][j] = Re G_ij and D[i][m + j] = Im G_ij.  Each operand value a is split
// as a_hi + a_lo with a_hi = tf32(a) and a_lo = tf32(a - a_hi); a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// (three MMAs per K step) has error at most 3 2^-22 |a b|, and the FP32 accumulation in TMEM adds at most
// 2 u per addition (u = 2^-24), so |G^ - G|_ij <= (3 2^-22 + (4K + 16) u) sum_c |x_ic| |x_jc|.
// Operands are staged KC real columns at a time into dynamic shared memory in the canonical K-major layout
// without swizzling: core matrices of 8 rows x 16 bytes, 128 bytes apart along K (leading byte offset) and
// 256 bytes apart along the rows (stride byte offset), one block per MMA K step of 8.  One thread issues the
// MMAs and commits them to tc_mbar; every thread waits for that barrier (bounded; on a timeout the circuit's
// status becomes GCAMPS_ENOCONV and the Gram is not used) before the stage is overwritten.  The accumulator
// (128 lanes x N columns of FP32) is read back with tcgen05.ld into G (FP32).  Needs m <= kTcMaxM and the
// kernel's TMEM (tc_tmem, kTcCols columns) and dynamic shared memory (tc_smem bytes).
#if GCAMPS_TC
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         ((uint64_t)1 << 46);
}
__device__ __forceinline__ float tf32_round(float a) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(a));
  return __uint_as_float(r);
}
__device__ __forceinline__ void umma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
               :: "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// bounded wait for phase `parity` of the mbarrier; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.b32 %0, 1, 0, q;\n}"
                 : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}
// Set-up of a CTA that uses gram_tc: its mbarrier and TMEM columns (warp 0 allocates).  Every thread calls it.
__device__ void tc_setup(Smem& s) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(&s.tc_mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s.tc_commits = 0;
  }
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&s.tc_tmem)), "r"(kTcCols));
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
}
__device__ void tc_teardown(Smem& s) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(s.tc_tmem), "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
}
// Real K columns staged per round: 16 (hi and lo parts of A and B, at most 48 KB), small enough to leave
// most of the SM's L1 to the engine's global-memory scratch.
__device__ __host__ __forceinline__ int tc_kc(int npad) { return 16; }

__device__ __noinline__ bool gram_tc(Smem& s, const Ctx& C, const float2* X, int rows, int cols, float2* G) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const bool wide = rows <= cols;
  const int m = wide ? rows : cols, Kc = wide ? cols : rows;
  const int Kr = 2 * Kc, npad = (2 * m + 15) / 16 * 16;
  const int KC = tc_kc(npad);
  const int asz = (KC / 8) * (128 / 8) * 256, bsz = (KC / 8) * (npad / 8) * 256;   // bytes per part
  uint8_t* Ahi = dsm;
  uint8_t* Alo = Ahi + asz;
  uint8_t* Bhi = Alo + asz;
  uint8_t* Blo = Bhi + bsz;
  const float* Xf = reinterpret_cast<const float*>(X);
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  const uint32_t tmem = s.tc_tmem, mbar = smem_addr(&s.tc_mbar);
  uint32_t commits = s.tc_commits;
  bool ok = true;
  // value (row, kk) of A (rows < m are X's rows as (re, im) pairs; 0 beyond)
  auto aval = [&](int row, int kk) -> float {
    if (row >= m || kk >= Kr) return 0.f;
    const int c = kk >> 1;
    return wide ? Xf[((long long)row * cols + c) * 2 + (kk & 1)] : Xf[((long long)c * cols + row) * 2 + (kk & 1)];
  };
  for (int k0 = 0; k0 < Kr; k0 += KC) {
    // stage the quads (4 consecutive K values of one row) of A and B, hi and lo parts
    const int qa = 128 * (KC / 4), qb = npad * (KC / 4);
    for (int q = tid; q < qa + qb; q += nt) {
      const bool isA = q < qa;
      const int qq = isA ? q : q - qa;
      const int row = qq / (KC / 4), quad = qq % (KC / 4);
      const int kk = k0 + 4 * quad;
      float v[4];
      if (isA || row < m) {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = aval(row, kk + u);
      } else if (row < 2 * m) {   // the row times i: (re, im) -> (-im, re)
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
          const float re = aval(row - m, kk + u), im = aval(row - m, kk + u + 1);
          v[u] = -im;
          v[u + 1] = re;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = 0.f;
      }
      float4 hi, lo;
      hi.x = tf32_round(v[0]);
      hi.y = tf32_round(v[1]);
      hi.z = tf32_round(v[2]);
      hi.w = tf32_round(v[3]);
      lo.x = tf32_round(v[0] - hi.x);
      lo.y = tf32_round(v[1] - hi.y);
      lo.z = tf32_round(v[2] - hi.z);
      lo.w = tf32_round(v[3] - hi.w);
      const int R = isA ? 128 : npad;
      const int off = (quad >> 1) * (R / 8) * 256 + (row >> 3) * 256 + (quad & 1) * 128 + (row & 7) * 16;
      *reinterpret_cast<float4*>((isA ? Ahi : Bhi) + off) = hi;
      *reinterpret_cast<float4*>((isA ? Alo : Blo) + off) = lo;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int t = 0; t < KC / 8; ++t) {
        const uint64_t ah = umma_desc(smem_addr(Ahi + t * (128 / 8) * 256)), al = umma_desc(smem_addr(Alo + t * (128 / 8) * 256));
        const uint64_t bh = umma_desc(smem_addr(Bhi + t * (npad / 8) * 256)), bl = umma_desc(smem_addr(Blo + t * (npad / 8) * 256));
        umma_tf32(tmem, ah, bl, idesc, (k0 > 0 || t > 0) ? 1u : 0u);
        umma_tf32(tmem, al, bh, idesc, 1u);
        umma_tf32(tmem, ah, bh, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
    }
    ok = mbar_wait(mbar, commits & 1) && ok;
    ++commits;
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  // epilogue: warps w and w + 4 share TMEM lanes 32 (w % 4) .. + 31 and split the columns
  const int row = 32 * (warp & 3) + lane;
  const int half = npad / 2, c0 = (warp >> 2) * half;
  float* Gf = reinterpret_cast<float*>(G);
  for (int cc = c0; cc < c0 + half; cc += 8) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)cc));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    if (row < m)
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = cc + u;
        if (j < m) Gf[2 * ((long long)row * m + j)] = __uint_as_float(r[u]);
        else if (j < 2 * m) Gf[2 * ((long long)row * m + (j - m)) + 1] = __uint_as_float(r[u]);
      }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0) {
    s.tc_commits = commits;
    if (C.dstats) C.dstats[3] += 8.0 * m * m * Kc;   // algorithmic flops of the complex Gram
  }
  if (!ok && tid == 0) set_failure(C, GCAMPS_ENOCONV, 3, rows, cols);
  __syncthreads();
  return ok;
}
#else
__device__ __forceinline__ void tc_setup(Smem&) {}
__device__ __forceinline__ void tc_teardown(Smem&) {}
#endif  // GCAMPS_TC

// The full m x m Gram (smaller side) of X (rows x cols complex FP32) in FP32: SIMT on a warp; on a CTA the
// tensor cores (gram_tc) when the kernel set them up and m <= kTcMaxM, else SIMT.
__device__ void gram_fp32_simt(int tid, int nt, const float2* X, int rows, int cols, float2* G) {
  const int m = rows < cols ? rows : cols;
  for (int idx = tid; idx < m * (m + 1) / 2; idx += nt) {
    int i, j;
    tri_index(idx, i, j);
    float2 acc = make_float2(0.f, 0.f);
    if (rows <= cols) {
      const float2* ri = X + (long long)i * cols;
      const float2* rj = X + (long long)j * cols;
      for (int c = 0; c < cols; ++c) acc = ffmac2(ri[c], rj[c], acc);
    } else {
      for (int r = 0; r < rows; ++r) acc = ffmac2(X[(long long)r * cols + i], X[(long long)r * cols + j], acc);
    }
    G[(long long)i * m + j] = acc;
    if (i != j) G[(long long)j * m + i] = make_float2(acc.x, -acc.y);
  }
}
template <>
__device__ void gram_fp32<WarpGroup>(const WarpGroup& g, const Ctx& C, const float2* X, int rows, int cols, float2* G) {
  gram_fp32_simt(g.tid, g.n, X, rows, cols, G);
  g.sync();
}
template <>
__device__ void gram_fp32<BlockGroup>(const BlockGroup& g, const Ctx& C, const float2* X, int rows, int cols,
                                      float2* G) {
#if GCAMPS_TC
  const int m = rows < cols ? rows : cols;
  if (C.e->tc_smem > 0 && m <= kTcMaxM && gram_tc(*g.s, C, X, rows, cols, G)) return;
#endif
  gram_fp32_simt(g.tid, g.n, X, rows, cols, G);
  g.sync();
}

// Scores classes list[0..cnt) (all K classes if list is null) on the whole cluster: small problems
// one class per warp, large ones one class per CTA.  Results go to the leader CTA's shared memory.
// mode kExact: S2 and S_vN in FP64; kScreen: S2 in FP32 with its lower bound (lead->s2lo).
// kS2Exact: S2 in FP64 only (class 0 still gets kExact: its eigenvalues certify QR moves).
// kEstimate: the FP32 von Neumann estimate and its bound (lead->vest, lead->vbd; CTA-level sizes only).
enum ScoreMode { kExact = 0, kScreen = 1, kS2Exact = 2, kEstimate = 3 };
__device__ void score_classes(Smem& s, Smem* lead, const Ctx& C, const double2* theta, int cl, int cr,
                              const int* list, int cnt, int mode) {
  const Engine& e = *C.e;
  const int d = C.d, dd = d * d;
  const int rows = cl * d, cols = d * cr;
  const int m = rows < cols ? rows : cols;
  // exact evaluations at warp-level sizes run one per CTA when the list has no more entries than the
  // cluster has CTAs and m >= exact_cta_min_m: a CTA spreads one evaluation over its four FP64 pipes
  const bool cta_exact = mode == kExact && cnt <= C.csize && m >= e.exact_cta_min_m;
  const bool small = (long long)rows * cols <= kSmall && m * m <= kSmall && !cta_exact;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (small) {
    WarpGroup g{lane};
    double2* ws = C.cta + e.cl.warp + (long long)warp * kSmallStride;
    // consecutive list entries go to different CTAs, then to different warps: the first 4 csize
    // entries land on distinct FP64 pipes (SM sub-partitions)
    const int gw = warp * C.csize + C.rank, nw = C.csize * kWarps;
    for (int t = gw; t < cnt; t += nw) {
      const int k = list ? list[t] : t;
      if (mode == kEstimate) {
        float est = 0.f, v = 0.f, lo = 0.f;
        const bool ok = vn_est32(g, C, C.th32, cl, cr, e.candU32 + (long long)k * dd * dd, reinterpret_cast<float2*>(ws),
                                 s.whv[warp], s.whw[warp], 32, s.wtri32[warp], 32, &est, &v, &lo);
        if (lane == 0) {
          lead->s2[k] = v;
          lead->s2lo[k] = lo;
          lead->vest[k] = est;
          lead->vbd[k] = ok ? lead->dval[3] : 1e300;   // the visit's bound (select_class), or none
          lead->estd[k] = 1;
        }
        continue;
      }
      if (mode == kScreen) {
        double v, lo;
        s2_fp32(g, C, C.th32, cl, cr, e.candU32 + (long long)k * dd * dd, reinterpret_cast<float2*>(ws), &v, &lo);
        if (lane == 0) {
          lead->s2[k] = v;
          lead->s2lo[k] = lo;
        }
        continue;
      }
      const bool want_vn = mode == kExact || k == 0;
      const long long t0 = (C.prof && C.rank == 0 && warp == 0 && lane == 0) ? clock64() : 0;
      const Score sc = score_class(g, C, theta, cl, cr, e.candU + (long long)k * dd * dd,
                                   e.candU32 + (long long)k * dd * dd, ws, kSmall, want_vn, s.wtri[warp],
                                   s.wtri32[warp], 32);
      if (C.prof && C.rank == 0 && warp == 0 && lane == 0 && want_vn) {   // the leader's own exact evaluations
        C.prof[P_LEAD_EXACT_CYC] += clock64() - t0;
        C.prof[P_LEAD_EXACT_N] += 1;
      }
      if (lane == 0) {
        lead->s2[k] = sc.s2;
        lead->evald[k] = 1;
        lead->vn[k] = want_vn ? sc.vn : CUDART_NAN;
        lead->rk[k] = sc.rank;
        if (k == 0) lead->rank0 = sc.rank;
        if (!sc.ok) set_failure(C, GCAMPS_ENOCONV, 2, rows, cols);
      }
    }
  } else {
    BlockGroup g{&s, (int)threadIdx.x, (int)blockDim.x};
    double2* ws = C.cta + e.cl.block;
    // FP32 estimates of more classes than the cluster has CTAs: two at once per CTA, one per half (each
    // half's scratch after the other's, when both fit the CTA-level buffer of 2 scap + 64 complex doubles)
    const long long half_off = ((long long)rows * cols + (long long)m * m + 2LL * m + 63) & ~31LL;   // float2
    if (mode == kEstimate && cnt > C.csize && half_off <= 2 * e.scap + 64) {
      const int half = (int)threadIdx.x / (kThreads / 2);
      HalfGroup hg{&s, (int)threadIdx.x % (kThreads / 2), kThreads / 2, half};
      float2* wsh = reinterpret_cast<float2*>(ws) + half * half_off;
      for (int t = C.rank + half * C.csize; t < cnt; t += 2 * C.csize) {
        const int k = list ? list[t] : t;
        float est = 0.f;
        const bool ok = vn_est32(hg, C, C.th32, cl, cr, e.candU32 + (long long)k * dd * dd, wsh,
                                 half ? s.hv2 : s.hv, half ? s.hw2 : s.hw, kBTri, half ? s.btri32b : s.btri32,
                                 kBTri, &est, (float*)nullptr, (float*)nullptr);
        if (hg.tid == 0) {
          lead->vest[k] = est;
          lead->vbd[k] = ok ? lead->dval[3] : 1e300;   // the visit's bound (select_class), or none
          lead->estd[k] = 1;
        }
        hg.sync();
      }
      __syncthreads();
      return;
    }
    for (int t = C.rank; t < cnt; t += C.csize) {
      const int k = list ? list[t] : t;
      if (mode == kScreen) {
        double v, lo;
        s2_fp32(g, C, C.th32, cl, cr, e.candU32 + (long long)k * dd * dd, reinterpret_cast<float2*>(ws), &v, &lo);
        if (threadIdx.x == 0) {
          lead->s2[k] = v;
          lead->s2lo[k] = lo;
        }
        __syncthreads();
        continue;
      }
      if (mode == kEstimate) {
        float est = 0.f;
        const bool ok = vn_est32(g, C, C.th32, cl, cr, e.candU32 + (long long)k * dd * dd,
                                 reinterpret_cast<float2*>(ws), s.hv, s.hw, kBTri, s.btri32, kBTri, &est,
                                 (float*)nullptr, (float*)nullptr);
        if (threadIdx.x == 0) {
          lead->vest[k] = est;
          lead->vbd[k] = ok ? lead->dval[3] : 1e300;   // the visit's bound (select_class), or none
          lead->estd[k] = 1;
        }
        __syncthreads();
        continue;
      }
      const bool want_vn = mode == kExact || k == 0;
      const Score sc = score_class(g, C, theta, cl, cr, e.candU + (long long)k * dd * dd,
                                   e.candU32 + (long long)k * dd * dd, ws, e.scap, want_vn, s.btri, s.btri32, kBTri);
      if (threadIdx.x == 0) {
        lead->s2[k] = sc.s2;
        lead->evald[k] = 1;
        lead->vn[k] = want_vn ? sc.vn : CUDART_NAN;
        lead->rk[k] = sc.rank;
        if (k == 0) lead->rank0 = sc.rank;
        if (!sc.ok) set_failure(C, GCAMPS_ENOCONV, 2, rows, cols);
      }
      __syncthreads();
    }
  }
}


// ---------------------------------------------------------------- disentangling sweeps (Sec. 3)
// One bond.  The leader CTA forms theta = A_i A_{i+1}; the cluster scores the classes; the leader
// decides, applies and splits.  With the Renyi-2 bound (S2 <= S_vN): phase A gives S2 of every class
// from an FP32 screen with a rigorous lower bound s2lo (s2_fp32), and the passes below use s2lo;
// the first pass evaluates S_vN of the identity and of the classes with the smallest S2 (as many as the
// cluster evaluates at once), giving an upper bound B on the best entropy; the second pass evaluates every
// other class with S2 <= B + tie_tol (usually none: they are a prefix of the S2 order).  A class left out
// has S_vN >= S2 > best + tie_tol, so the decision equals the one from evaluating every class.
// Cluster-wide choice of the class for one theta (shape chi_l x d x d x chi_r in global memory,
// readable by every CTA).  Returns the chosen class on the leader (-1 on the other CTAs); the
// leader's s.vn / s.evald hold the evaluated entropies and *nev their count.
// The decision over the exactly evaluated classes of the leader's shared memory (select_class), and the
// record of the visit's scores; -1 on the other CTAs.
__device__ int decide_class(Smem& s, const Ctx& C, const double2* theta, int cl, int cr, int* nev_out, long long& tp) {
  const Engine& e = *C.e;
  const bool leader = C.rank == 0;
  const int d = C.d, kind = e.score_kind;
  const int rows = cl * d, cols = d * cr;
  if (!leader) return -1;
  if (threadIdx.x < 32) {
    // the decision over the exactly evaluated classes, on the first warp: key = S_vN (kind 0), S2 (kind 1),
    // or the weight rank first and S_vN second (kind 2); ties within tie_tol go to the lowest index, and a
    // class is applied only if it beats the identity
    const int lane = threadIdx.x;
    int nev = 0, rmin = 1 << 30;
    for (int k = lane; k < C.K; k += 32)
      if (s.evald[k]) {
        ++nev;
        rmin = min(rmin, s.rk[k]);
      }
    nev = warp_sum_int(nev);
    rmin = warp_min_int(rmin);
    auto key = [&](int k) { return kind == 1 ? s.s2[k] : s.vn[k]; };
    auto in = [&](int k) { return s.evald[k] && (kind != 2 || s.rk[k] == rmin); };
    double b = 1e300;
    for (int k = lane; k < C.K; k += 32)
      if (in(k)) b = fmin(b, key(k));
    const double best = warp_min_double(b) + e.tie_tol;
    int kb = 0;
    for (int base = 0; base < C.K; base += 32) {
      const int k = base + lane;
      const unsigned hit = __ballot_sync(0xffffffffu, k < C.K && in(k) && key(k) <= best);
      if (hit) {
        kb = base + __ffs(hit) - 1;
        break;
      }
    }
    if (lane == 0) {
      const bool better = (kind == 2 && s.rk[kb] < s.rk[0]) || key(kb) < key(0) - e.tie_tol;
      s.ival[4] = better ? kb : 0;
      s.ival[5] = nev;
    }
  }
  {
    double* out = e.lastsc + (long long)C.c * (3 * kMaxK + 2 + 2 * kSmall);
    for (int k = threadIdx.x; k < C.K; k += blockDim.x) {
      out[k] = s.s2[k];
      out[kMaxK + k] = s.vn[k];
      out[2 * kMaxK + k] = s.evald[k];
    }
    if (threadIdx.x == 0) {
      out[3 * kMaxK] = cl;
      out[3 * kMaxK + 1] = cr;
    }
    if ((long long)rows * cols <= kSmall)
      for (int k = threadIdx.x; k < rows * cols; k += blockDim.x) {
        out[3 * kMaxK + 2 + 2 * k] = theta[k].x;
        out[3 * kMaxK + 3 + 2 * k] = theta[k].y;
      }
  }
  __syncthreads();
  prof_lap(C, P_DECIDE, tp);
  *nev_out = s.ival[5];
  return s.ival[4];
}

__device__ int select_class(Smem& s, Smem* lead, const Ctx& C, const double2* theta, int cl, int cr, int* nev_out) {
  long long tp = prof_start(C);
  const Engine& e = *C.e;
  const bool leader = C.rank == 0;
  const int d = C.d;
  const int rows = cl * d, cols = d * cr;
  const int m = rows < cols ? rows : cols;
  const bool prune = m > kPruneMin;
  const bool small = (long long)rows * cols <= kSmall && m * m <= kSmall;
  const int kind = e.score_kind;
  // The von Neumann score prunes with FP32 estimates whose error bound depends on the shape only: the leader
  // computes it once, published with the FP32 copy of theta by the barrier below.
  const bool est_kind = prune && kind == 0;
  if (leader && threadIdx.x == 0) {
    s.ival[6] = 0;
    if (est_kind) s.dval[3] = vn_est_bound(d, m, rows < cols ? cols : rows);
  }
  if (prune) {   // FP32 copy of theta for the screen, shared by the cluster
    if (leader)
      for (int i = threadIdx.x; i < rows * cols; i += blockDim.x)
        C.th32[i] = make_float2((float)theta[i].x, (float)theta[i].y);
    cluster_sync();
  }
  if (est_kind && small && lead->dval[3] < 1.0) {
    // Warp-level sizes: one pass gives every class its FP32 von Neumann estimate (and its Renyi-2 value and
    // bound, from the same Gram); exact FP64 entropies only for the identity and the classes whose estimate
    // interval reaches down to U + tie_tol, U the smallest upper bound.  A class left out has S_vN above
    // U + tie_tol >= best + tie_tol (the class that set U is evaluated exactly), so the decision equals
    // evaluating every class.
    score_classes(s, lead, C, theta, cl, cr, nullptr, C.K, kEstimate);
    cluster_sync();
    prof_lap(C, P_EST, tp);
    if (leader && threadIdx.x < 32) {   // the leader's first warp builds the exact list
      double u = 1e300;
      for (int k = threadIdx.x; k < C.K; k += 32) {
        s.evald[k] = 0;
        u = fmin(u, s.vest[k] + s.vbd[k]);
      }
      const double U = warp_min_double(u) + e.tie_tol + 1e-12;
      if (threadIdx.x == 0) s.list[0] = 0;
      const int cnt = warp_list(s.list, 1, C.K, 1, [&](int k) { return s.vest[k] - s.vbd[k] <= U; });
      if (threadIdx.x == 0) {
        s.nlist = cnt;
        s.ival[6] = C.K;
      }
    }
    cluster_sync();
    score_classes(s, lead, C, theta, cl, cr, lead->list, lead->nlist, kExact);
    cluster_sync();
    prof_lap(C, P_EXACT, tp);
    return decide_class(s, C, theta, cl, cr, nev_out, tp);
  }
  score_classes(s, lead, C, theta, cl, cr, nullptr, C.K, prune ? kScreen : kExact);
  cluster_sync();
  prof_lap(C, prune ? P_SCREEN : P_EXACT, tp);
  // weight-rank threshold (the same as the QR-move certificate) and the rank lower bound from S2:
  // the weights above tau carry at least 1 - m tau of the trace, so sum p^2 >= (1 - m tau)^2 / rank and
  // rank >= exp(S2 + 2 ln(1 - m tau)) >= exp(S2 - 2.01 m tau)
  const double tau_w = fmax(1e-12, 4.0 * e.cutoff * e.cutoff);
  auto rank_lo = [&](int k) -> int {
    const double x = s.s2lo[k] - 2.01 * m * tau_w;
    if (!(x > 0.0) || m * tau_w >= 0.25) return 0;
    return (int)ceil(exp(x) * (1.0 - 1e-12));
  };
  // FP32 von Neumann estimates (kind 0, CTA-level sizes whose estimate bound is informative): the identity and
  // the classes of smallest S2 lower bound get estimates first (one per CTA), giving an upper bound U on the
  // best entropy; then every class whose S2 lower bound is within tie_tol of U; then exact FP64 entropies
  // only for the identity and the classes whose estimate interval reaches down to U + tie_tol.  A class left
  // out has S_vN >= S2 lower bound or >= its estimate's lower bound, either above U + tie_tol >= best +
  // tie_tol (the class that set U is evaluated exactly), so the decision equals evaluating every class.
  // the estimate bound depends on the shape only: computed once, on the leader, and read from its shared
  // memory by every CTA after the next cluster barrier
  const bool estimate = est_kind && !small && lead->dval[3] < 1.0;
  if (estimate) {
    if (leader) {
      const int L = C.csize - 1;
      for (int k = threadIdx.x; k < C.K; k += blockDim.x) {
        s.evald[k] = 0;
        s.estd[k] = 0;
        const long long bk = order_key(s.s2lo[k]);
        int r = 0;
        for (int q = 0; q < C.K; ++q) {
          const long long bq = order_key(s.s2lo[q]);
          r += (bq < bk) || (bq == bk && q < k);
        }
        s.ord[k] = r;
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        if (threadIdx.x == 0) s.list[0] = 0;
        const int cnt = warp_list(s.list, 1, C.K, 1, [&](int k) { return s.ord[k] < L; });
        if (threadIdx.x == 0) s.nlist = cnt;
      }
    }
    cluster_sync();
    score_classes(s, lead, C, theta, cl, cr, lead->list, lead->nlist, kEstimate);
    cluster_sync();
    if (leader && threadIdx.x < 32) {
      double u = 1e300;
      for (int k = threadIdx.x; k < C.K; k += 32)
        if (s.estd[k]) u = fmin(u, s.vest[k] + s.vbd[k]);
      const double U = warp_min_double(u) + e.tie_tol + 1e-12;
      const int cnt = warp_list(s.list, 0, C.K, 0, [&](int k) { return !s.estd[k] && s.s2lo[k] <= U; });
      if (threadIdx.x == 0) s.nlist = cnt;
    }
    cluster_sync();
    score_classes(s, lead, C, theta, cl, cr, lead->list, lead->nlist, kEstimate);
    cluster_sync();
    prof_lap(C, P_EST, tp);
    if (leader && threadIdx.x < 32) {
      double u = 1e300;
      int nest = 0;
      for (int k = threadIdx.x; k < C.K; k += 32)
        if (s.estd[k]) {
          u = fmin(u, s.vest[k] + s.vbd[k]);
          ++nest;
        }
      const double U = warp_min_double(u) + e.tie_tol + 1e-12;
      nest = warp_sum_int(nest);
      if (threadIdx.x == 0) s.list[0] = 0;
      const int cnt = warp_list(s.list, 1, C.K, 1, [&](int k) { return s.estd[k] && s.vest[k] - s.vbd[k] <= U; });
      if (threadIdx.x == 0) {
        s.nlist = cnt;
        s.ival[6] = nest;
      }
    }
    cluster_sync();
    score_classes(s, lead, C, theta, cl, cr, lead->list, lead->nlist, kExact);
    cluster_sync();
    prof_lap(C, P_EXACT, tp);
  } else if (prune) {
    if (kind == 1) {
      // Renyi-2 score: exact S2 for every class whose lower bound is within tie_tol of the smallest
      // upper bound (upper = screen value + the same margin), and for the identity
      if (leader && threadIdx.x == 0) {
        double ub = 1e300;
        for (int k = 0; k < C.K; ++k) {
          s.evald[k] = 0;
          ub = fmin(ub, 2.0 * s.s2[k] - s.s2lo[k]);
        }
        int cnt = 1;
        s.list[0] = 0;
        for (int k = 1; k < C.K; ++k)
          if (s.s2lo[k] <= ub + e.tie_tol + 1e-12) s.list[cnt++] = k;
        s.nlist = cnt;
      }
      cluster_sync();
      score_classes(s, lead, C, theta, cl, cr, lead->list, lead->nlist, kS2Exact);
      cluster_sync();
    } else {
      if (leader) {
        // first pass: the identity and the classes of smallest S2 lower bound, one per FP64 pipe of the
        // cluster (warp-level scoring) or one per CTA (CTA-level scoring)
        const int L = (small ? 4 * C.csize : C.csize) - 1;
        for (int k = threadIdx.x; k < C.K; k += blockDim.x) {
          s.evald[k] = 0;
          const long long bk = order_key(s.s2lo[k]);
          int r = 0;
          for (int q = 0; q < C.K; ++q) {
            const long long bq = order_key(s.s2lo[q]);
            r += (bq < bk) || (bq == bk && q < k);
          }
          s.ord[k] = r;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
          int cnt = 1;
          s.list[0] = 0;
          for (int k = 1; k < C.K; ++k)
            if (s.ord[k] < L) s.list[cnt++] = k;
          s.nlist = cnt;
        }
      }
      cluster_sync();
      score_classes(s, lead, C, theta, cl, cr, lead->list, lead->nlist, kExact);
      cluster_sync();
      if (leader && threadIdx.x == 0) {
        // second pass: every class the bounds cannot exclude.  Kind 0: S2 lower bound within tie_tol of the
        // best exact entropy.  Kind 2: rank bound below the best exact rank, or equal to it with the S2
        // bound within tie_tol of the best entropy among the classes of that rank.
        int rmin = 1 << 30;
        if (kind == 2)
          for (int k = 0; k < C.K; ++k)
            if (s.evald[k] && s.rk[k] < rmin) rmin = s.rk[k];
        double bound = 1e300;
        for (int k = 0; k < C.K; ++k)
          if (s.evald[k] && (kind != 2 || s.rk[k] == rmin)) bound = fmin(bound, s.vn[k]);
        int cnt = 0;
        for (int k = 0; k < C.K; ++k) {
          if (s.evald[k]) continue;
          bool need = s.s2lo[k] <= bound + e.tie_tol + 1e-12;
          if (kind == 2) {
            const int rl = rank_lo(k);
            need = rl < rmin || (rl == rmin && need);
          }
          if (need) s.list[cnt++] = k;
        }
        s.nlist = cnt;
      }
      cluster_sync();
      score_classes(s, lead, C, theta, cl, cr, lead->list, lead->nlist, kExact);
      cluster_sync();
    }
    prof_lap(C, P_EXACT, tp);
  }
  return decide_class(s, C, theta, cl, cr, nev_out, tp);
}

__device__ void visit_bond(Smem& s, Smem* lead, const Ctx& C, int i, bool ltr, int* accepted) {
  const Engine& e = *C.e;
  const bool leader = C.rank == 0;
  const int d = C.d, dd = d * d;
  double2* theta = C.scr + e.sl.theta;
  double2* tmp = C.scr + e.sl.tmp;
  const long long tv = prof_start(C);
  long long tp = tv;
  if (prof_thread(C)) {
    const int ml = C.dims[i] * d, mr = d * C.dims[i + 2];
    C.prof[P_CURB] = 1 + prof_bucket(ml < mr ? ml : mr);
  }
  if (leader) {
    const int cl0 = C.dims[i], ch = C.dims[i + 1], cr0 = C.dims[i + 2];
    block_matmul(theta, site_ptr(C, i), site_ptr(C, i + 1), cl0 * d, ch, d * cr0);
    if (threadIdx.x == 0) s.rank0 = -1;
  }
  cluster_sync();
  prof_lap(C, P_THETA, tp);
  const int cl = C.dims[i], cr = C.dims[i + 2];
  const int rows = cl * d, cols = d * cr;
  const int m = rows < cols ? rows : cols;
  int nev = 0;
  // Splits with many Jacobi columns run their rotations on the whole cluster: the other CTAs wait for the
  // leader's choice (a QR move or such a split) at one more cluster barrier.
  const bool big = C.csize > 1 && m >= kClusterJacobiMin;
  if (e.replay && e.replay_n[C.c] > 0) {
    // replay: the recorded class of this visit (every CTA reads the same list; a visit past its end or at
    // another bond invalidates the circuit)
    if (leader && threadIdx.x == 0) {
      const int nd = C.meta[M_NDEC];
      const int* rp = e.replay + ((long long)C.c * kDecCap + nd) * 2;
      int kb = 0;
      if (nd >= e.replay_n[C.c] || nd >= kDecCap || rp[0] != i) set_status(C, GCAMPS_EINVAL);
      else kb = rp[1];
      s.ival[4] = (kb >= 0 && kb < C.K) ? kb : 0;
      s.ival[6] = 0;
      s.rank0 = -1;   // no certificate: the visit splits by SVD
    }
    __syncthreads();
    nev = -1;
  }
  const int kbsel = nev < 0 ? (leader ? s.ival[4] : -1)
                            : select_class(s, lead, C, theta, cl, cr, &nev);
  if (nev < 0) nev = 0;
  if (!leader) {
    if (!big) return;
    cluster_sync();
    if (lead->jmode == 2) jacobi_cluster(lead, C, C.scr + e.sl.b, lead->jm, lead->jn, C.scr + e.sl.w, e.jacobi_cap);
    return;
  }
  tp = prof_start(C);
  // visit counters of the size bucket; the visit's cycles are added when it ends
  if (prof_thread(C)) {
    const int b = prof_bucket(m);
    C.prof[P_VISITS + b] += 1;
    C.prof[P_VEXACT + b] += nev;
    C.prof[P_VEST + b] += s.ival[6];
  }
  if (threadIdx.x == 0) {
    const int kb = kbsel;
    C.stats[S_BONDS] += 1;
    C.stats[S_CANDS] += C.K;
    C.stats[S_VN] += nev;
    {
      const double R = rows, Cc = cols, mm = m, M = rows < cols ? cols : rows;
      const double per_class = 8.0 * dd * R * Cc + 4.0 * mm * (mm + 1.0) * M;
      const double tri = (16.0 / 3.0) * mm * mm * mm;
      // exact evaluations, FP64 (Renyi-2 scores need no eigenvalues except the identity's)
      C.dstats[1] += e.score_kind == 1 ? nev * per_class + tri : nev * (per_class + tri);
      if (m > kPruneMin) C.dstats[4] += C.K * (per_class + tri);   // every class scored exactly (the algorithm)
      if (m > kPruneMin) C.dstats[2] += C.K * per_class;                // FP32 screen of every class
    }
    const int nd = C.meta[M_NDEC];
    if (nd < kDecCap) {
      C.dec[2 * nd] = i;
      C.dec[2 * nd + 1] = kb;
    }
    C.meta[M_NDEC] = nd + 1;
  }
  __syncthreads();
  const int kb = s.ival[4];
  if (kb != 0) {
    const double2* Q = e.candU + (long long)kb * dd * dd;
    const long long total = (long long)cl * dd * cr;
    for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int b = (int)(idx % cr), u = (int)((idx / cr) % dd);
      const long long a = idx / ((long long)cr * dd);
      double2 acc = cz();
      for (int v = 0; v < dd; ++v) acc = cfma(Q[u * dd + v], theta[(a * dd + v) * cr + b], acc);
      tmp[idx] = acc;
    }
    __syncthreads();
    block_copy(theta, tmp, total);
    __syncthreads();
    fold_candidate(s, C, kb, i);
    if (threadIdx.x == 0) C.stats[S_ACC] += 1;
    ++*accepted;
  }
  prof_lap(C, P_APPLYQ, tp);
  const int bb = C.bond_bound[i + 1];
  const int cap = e.chi_max < bb ? e.chi_max : bb;
  // Nothing applied and the identity class's Gram has exactly chi eigenvalues above
  // max(1e-12, 4 cutoff^2) tr (theta has rank <= chi, the bond dimension): every one of those
  // Schmidt values is above 1e-6 s_0 and above the cutoff, so the truncated SVD would keep the bond
  // as it is.  A QR move of the centre gives the same state and bond dimension without it.
  const int chim = C.dims[i + 1];
  if (kb == 0 && s.rank0 == chim && chim <= cap) {
    if (big) {   // release the other CTAs
      if (threadIdx.x == 0) s.jmode = 0;
      __syncthreads();
      cluster_sync();
    }
    if (ltr) move_right(s, C, i);
    else move_left_qr(s, C, i + 1);
    note_chi(C, chim);
    __syncthreads();
    prof_lap(C, P_QRMOVE, tp);
    if (prof_thread(C)) {
      C.prof[P_VCYC + prof_bucket(m)] += clock64() - tv;
      C.prof[P_CURB] = 0;
    }
    return;
  }
  Factor F;
  if (big) {
    const SvdPrep p = svd_prepare(s, C, theta, rows, cols);
    double2* B = C.scr + e.sl.b;
    double2* W = C.scr + e.sl.w;
    for (long long idx = threadIdx.x; idx < (long long)p.n * p.n; idx += blockDim.x)
      W[idx] = ((idx % p.n) == (idx / p.n)) ? make_double2(1.0, 0.0) : cz();
    double fro = 0;
    for (long long idx = threadIdx.x; idx < (long long)p.mm * p.n; idx += blockDim.x) fro += cabs2(B[idx]);
    fro = block_sum(fro, s);
    if (threadIdx.x == 0) {
      s.jfro = fro;
      s.jflag[0] = s.jflag[1] = 0;
      s.jm = p.mm;
      s.jn = p.n;
      s.jmode = 2;
    }
    __syncthreads();
    cluster_sync();
    const int sweeps = jacobi_cluster(lead, C, B, p.mm, p.n, W, e.jacobi_cap);
    F = svd_finish(s, C, p, sweeps, rows, cols, cap, true);
  } else {
    F = svd_factor(s, C, theta, rows, cols, cap, true);
  }
  const int k = F.k;
  if (ltr) {
    for (long long idx = threadIdx.x; idx < (long long)k * d * cr; idx += blockDim.x)
      F.Vh[idx] = cscale(F.Vh[idx], C.sing[idx / (d * cr)]);
  } else {
    for (long long idx = threadIdx.x; idx < (long long)cl * d * k; idx += blockDim.x)
      F.U[idx] = cscale(F.U[idx], C.sing[idx % k]);
  }
  __syncthreads();
  block_copy(site_ptr(C, i), F.U, (long long)cl * d * k);
  block_copy(site_ptr(C, i + 1), F.Vh, (long long)k * d * cr);
  if (threadIdx.x == 0) {
    C.dims[i + 1] = k;
    C.meta[M_OC] = ltr ? i + 1 : i;
    C.dstats[0] += F.disc;
  }
  note_chi(C, k);
  __syncthreads();
  prof_lap(C, P_SPLIT, tp);
  if (prof_thread(C)) {
    C.prof[P_VCYC + prof_bucket(m)] += clock64() - tv;
    C.prof[P_CURB] = 0;
  }
}

// Alternating sweeps over the bonds of the last span; every CTA of the cluster runs the loop, only
// the leader touches the MPS and the tableau.
// sweep_cap > 0 overrides the handle's max_sweeps for this call; visit_cap > 0 stops after that
// many bond visits (the centre is then left where the last split put it).
__device__ void disentangle(Smem& s, Smem* lead, const Ctx& C, int sweep_cap, int visit_cap) {
  cluster_sync();
  if (C.meta[M_STATUS] != 0) return;   // a failed circuit does no further work
  if (!C.meta[M_HAVE_SPAN]) return;
  const int f = C.meta[M_F], l = C.meta[M_L];
  if (l <= f) return;
  const int max_sweeps = sweep_cap > 0 ? sweep_cap : C.e->max_sweeps;
  int visits = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    const bool ltr = (sweep & 1) == 0;
    long long tp = prof_start(C);
    if (C.rank == 0) move_center(s, C, ltr ? f : l);
    prof_lap(C, P_CENTER, tp);
    int acc = 0;
    bool capped = false;
    for (int t = 0; t < l - f; ++t) {
      if (visit_cap > 0 && visits >= visit_cap) {
        capped = true;
        break;
      }
      const int i = ltr ? f + t : l - 1 - t;
      visit_bond(s, lead, C, i, ltr, &acc);
      ++visits;
    }
    if (capped) break;
    if (C.rank == 0 && threadIdx.x == 0) {
      C.stats[S_SWEEPS] += 1;
      s.bcast = acc;
    }
    cluster_sync();
    const int acc_all = lead->bcast;
    const int failed = C.meta[M_STATUS];
    cluster_sync();   // every CTA has read bcast and the status before either changes
    if (acc_all == 0 || failed != 0) break;
  }
}

__device__ void init_tau(Smem& s, int d) {
  if (threadIdx.x < 2 * d) {
    double sn, cs;
    sincospi((double)threadIdx.x / d, &sn, &cs);
    s.tau[threadIdx.x] = make_double2(cs, sn);
  }
  __syncthreads();
}

// Clifford and non-Clifford steps touch only the leader's state; disentangling uses the cluster.
__device__ void run_op(Smem& s, Smem* lead, const Ctx& C, const gcamps_op& op) {
  long long tp = prof_start(C);
  switch (op.kind) {
    case GCAMPS_OP_CLIFFORD:
      if (C.rank == 0) apply_clifford(s, C, op.q0, op.q1, op.img);
      prof_lap(C, P_CLIFF, tp);
      break;
    case GCAMPS_OP_NONCLIFFORD:
      // the leader applies the MPO; its compression SVDs with many Jacobi columns rotate on the whole
      // cluster: the other CTAs serve its requests until it releases them, on every path, with jmode 0 at
      // one last barrier (each request is one barrier plus jacobi_cluster's, the same on every CTA)
      if (C.rank == 0) {
        if (C.meta[M_STATUS] == 0) apply_nonclifford(s, C.csize > 1 ? lead : nullptr, C, op.q0, op.phases);
        if (C.csize > 1) {
          if (threadIdx.x == 0) s.jmode = 0;
          __syncthreads();
          cluster_sync();
        }
      } else {
        for (;;) {
          cluster_sync();
          if (lead->jmode != 2) break;
          jacobi_cluster(lead, C, C.scr + C.e->sl.b, lead->jm, lead->jn, C.scr + C.e->sl.w, C.e->jacobi_cap);
        }
      }
      prof_lap(C, P_MPO, tp);
      break;
    case GCAMPS_OP_DISENTANGLE:
      disentangle(s, lead, C, op.q0, op.q1);
      break;
    default:
      break;
  }
  __syncthreads();
}

// P' = C^dag W C for W = (x)_j X_j^{x_j} Z_j^{z_j} (xz = x | z): the inverse-tableau rows multiplied in
// the order of W with the Weyl product rule; exponents into acc_x, acc_z and the phase (units of tau)
// into *acc_r, all in shared memory.
__device__ void conj_weyl(Smem& s, const Ctx& C, const int8_t* xz, int* acc_x, int* acc_z, int* acc_r) {
  const int n = C.n, d = C.d;
  for (int j = threadIdx.x; j < n; j += blockDim.x) acc_x[j] = acc_z[j] = 0;
  if (threadIdx.x == 0) *acc_r = 0;
  __syncthreads();
  for (int q = 0; q < n; ++q) {
    for (int kind = 0; kind < 2; ++kind) {
      const int pw = kind == 0 ? xz[q] : xz[n + q];
      const int rowi = kind == 0 ? n + q : q;
      const uint8_t* R = C.ix + (long long)rowi * 2 * n;
      for (int p = 0; p < pw; ++p) {
        double loc = 0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) loc += acc_z[j] * R[j];
        const int tot = (int)llround(block_sum(loc, s));
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
          acc_x[j] = (acc_x[j] + R[j]) % d;
          acc_z[j] = (acc_z[j] + R[n + j]) % d;
        }
        if (threadIdx.x == 0) *acc_r = (*acc_r + C.ir[rowi] + 2 * tot) % (2 * d);
        __syncthreads();
      }
    }
  }
}



// ------------------------------------------------------------ bodies of the cluster kernels
// Each is the whole kernel: the FP64 translation units and the precision form's (GCAMPS_TC = 1) wrap them
// in kernels of their own.  One thread-block cluster of e.csize CTAs per circuit.
__device__ __forceinline__ void run_body(const Engine& e, const gcamps_op* ops, int first, int stop, int c, int rank) {
  __shared__ Smem s;
  Ctx C = make_ctx(e, c, rank);
  Smem* lead = cg::this_cluster().map_shared_rank(&s, 0);
  init_tau(s, e.d);
  if (C.prof && threadIdx.x == 0 && rank < kProfSmids) {   // where the cluster's CTAs run (1 + SM id)
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    C.prof[P_SMID + rank] = 1 + (long long)sm;
  }
  if (GCAMPS_TC && e.tc_smem) tc_setup(s);
  for (int i = first; i < stop; ++i) run_op(s, lead, C, ops[i]);
  cluster_sync();
  if (GCAMPS_TC && e.tc_smem) tc_teardown(s);
}

__device__ __forceinline__ void single_body(const Engine& e, const gcamps_op& op) {
  __shared__ Smem s;
  const int c = blockIdx.x / e.csize, rank = blockIdx.x % e.csize;
  Ctx C = make_ctx(e, c, rank);
  Smem* lead = cg::this_cluster().map_shared_rank(&s, 0);
  init_tau(s, e.d);
  if (GCAMPS_TC && e.tc_smem) tc_setup(s);
  run_op(s, lead, C, op);
  cluster_sync();
  if (GCAMPS_TC && e.tc_smem) tc_teardown(s);
}

// Scores of every class on a caller-provided theta (chi_l, d, d, chi_r), through the same cluster code as the
// disentangler: S2 and S_vN of all classes (no pruning), then the disentangler's own choice.
__device__ __forceinline__ void score_theta_body(const Engine& e, const double2* th, int cl, int cr, double* out_s2,
                                                 double* out_vn, int* out_choice) {
  __shared__ Smem s;
  const int c = blockIdx.x / e.csize, rank = blockIdx.x % e.csize;
  Ctx C = make_ctx(e, c, rank);
  Smem* lead = cg::this_cluster().map_shared_rank(&s, 0);
  init_tau(s, e.d);
  if (GCAMPS_TC && e.tc_smem) tc_setup(s);
  if (rank == 0)   // the FP32 copy of theta (the precision form's contractions read it)
    for (int i = threadIdx.x; i < cl * e.d * e.d * cr; i += blockDim.x)
      C.th32[i] = make_float2((float)th[i].x, (float)th[i].y);
  cluster_sync();
  score_classes(s, lead, C, th, cl, cr, nullptr, C.K, kExact);
  cluster_sync();
  if (c == 0 && rank == 0)
    for (int k = threadIdx.x; k < C.K; k += blockDim.x) {
      out_s2[k] = s.s2[k];
      out_vn[k] = s.vn[k];
    }
  cluster_sync();
  int nev = 0;
  const int kb = select_class(s, lead, C, th, cl, cr, &nev);
  if (c == 0 && rank == 0 && threadIdx.x == 0) {
    out_choice[0] = kb;
    out_choice[1] = nev;
  }
  cluster_sync();
  if (GCAMPS_TC && e.tc_smem) tc_teardown(s);
}
}  // namespace

// ---------------------------------------------------------------------------- host launchers
// Engine kernels are launched with one thread-block cluster of e.csize CTAs per circuit.
template <typename... KArgs, typename... Args>
cudaError_t launch_cluster(void (*kern)(KArgs...), const Engine& e, cudaStream_t st, Args... args) {
  if (e.csize > 8) {
    cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (a != cudaSuccess) return a;
  }
  if (e.tc_smem > 0) {
    cudaError_t a = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, e.tc_smem);
    if (a != cudaSuccess) return a;
    // a shared-memory carveout for two such CTAs per SM, the rest of the SM's 256 KB left to L1
    cudaFuncAttributes fa;
    a = cudaFuncGetAttributes(&fa, kern);
    if (a != cudaSuccess) return a;
    const int pct = (int)((2.0 * (fa.sharedSizeBytes + e.tc_smem + 1024) * 100.0) / (228.0 * 1024.0)) + 1;
    a = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct > 100 ? 100 : pct);
    if (a != cudaSuccess) return a;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(e.batch * e.csize), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)e.tc_smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)e.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace gcx
