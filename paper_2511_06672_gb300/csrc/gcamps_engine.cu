// Engine launch of libgcamps (arxiv 2511.06672, Sec. 3): the gate-list kernel k_run, the reset and
// the readout kernels (<W>, dense state vector).

#include "gcamps_device.cuh"

namespace gcx {
namespace {

__global__ void __launch_bounds__(kThreads, kMinCtas) k_run(Engine e, const gcamps_op* ops, const int32_t* begin) {
  const int c = blockIdx.x / e.csize;
  run_body(e, ops, begin[c], begin[c + 1], c, blockIdx.x % e.csize);
}


// |0...0> with C = I, counters cleared.
__global__ void __launch_bounds__(kThreads) k_reset(Engine e) {
  Ctx C = make_ctx(e, blockIdx.x);
  const int n = C.n, d = e.d;
  for (int i = threadIdx.x; i < 4 * n * n; i += blockDim.x) {
    const int row = i / (2 * n), col = i % (2 * n);
    // row j < n: Z_j -> z column n + j; row n + j: X_j -> x column j
    const uint8_t v = (row < n) ? (col == n + row) : (col == row - n);
    C.fx[i] = v;
    C.ix[i] = v;
  }
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) {
    C.fr[i] = 0;
    C.ir[i] = 0;
    C.weyl[i] = 0;
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double2* A = site_ptr(C, j);
    for (int sidx = 0; sidx < d; ++sidx) A[sidx] = make_double2(sidx == 0 ? 1.0 : 0.0, 0.0);
  }
  for (int j = threadIdx.x; j <= n; j += blockDim.x) C.dims[j] = 1;
  if (threadIdx.x < M_COUNT) C.meta[threadIdx.x] = 0;
  if (threadIdx.x < S_COUNT) C.stats[threadIdx.x] = (threadIdx.x == S_MAXCHI) ? 1 : 0;
  if (C.prof && threadIdx.x < P_COUNT) C.prof[threadIdx.x] = 0;
  if (threadIdx.x < kDStats) C.dstats[threadIdx.x] = 0.0;
}

// ------------------------------------------------------------------------------ readouts
// <MPS| P' |MPS> with P' = C^dag W C = tau^r (x)_j X^{a_j} Z^{b_j}: the inverse-tableau rows are
// multiplied in the order of W = prod_j X_j^{x_j} Z_j^{z_j}, then transfer matrices left to right.

__global__ void __launch_bounds__(kThreads) k_expect(Engine e, int c, const int8_t* xz, double2* out) {
  __shared__ Smem s;
  __shared__ int acc_x[kMaxN], acc_z[kMaxN];
  __shared__ int acc_r;
  Ctx C = make_ctx(e, c);
  init_tau(s, e.d);
  const int n = C.n, d = e.d;
  conj_weyl(s, C, xz, acc_x, acc_z, &acc_r);
  // transfer matrices: E (chi x chi) starts as [[1]]
  double2* E = C.scr + e.sl.b;
  double2* T = C.scr + e.sl.tmp;
  double2* E2 = C.scr + e.sl.u;
  if (threadIdx.x == 0) E[0] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int cl = C.dims[j], cr = C.dims[j + 1];
    const double2* A = site_ptr(C, j);
    const int a_j = acc_x[j], b_j = acc_z[j];
    // T[a, s, b'] = sum_{a'} E[a, a'] (X^a Z^b A)[a', s, b'],  (X^a Z^b A)[a', s, b'] = omega^{b (s-a)} A[a', s-a, b']
    for (long long idx = threadIdx.x; idx < (long long)cl * d * cr; idx += blockDim.x) {
      const int bp = (int)(idx % cr), sd = (int)((idx / cr) % d), a = (int)(idx / ((long long)cr * d));
      const int sp = (sd - a_j + d) % d;
      const double2 ph = s.tau[(2 * b_j * sp) % (2 * d)];
      double2 acc = cz();
      for (int ap = 0; ap < cl; ++ap) acc = cfma(E[(long long)a * cl + ap], A[((long long)ap * d + sp) * cr + bp], acc);
      T[idx] = cmul(ph, acc);
    }
    __syncthreads();
    // E'[b, b'] = sum_{a, s} conj(A[a, s, b]) T[a, s, b']
    for (long long idx = threadIdx.x; idx < (long long)cr * cr; idx += blockDim.x) {
      const int b = (int)(idx / cr), bp = (int)(idx % cr);
      double2 acc = cz();
      for (int a = 0; a < cl; ++a)
        for (int sd = 0; sd < d; ++sd)
          acc = cfmac(A[((long long)a * d + sd) * cr + b], T[((long long)a * d + sd) * cr + bp], acc);
      E2[idx] = acc;
    }
    __syncthreads();
    block_copy(E, E2, (long long)cr * cr);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = cmul(s.tau[acc_r], E[0]);
}

// Dense MPS vector mv[x] (d^n entries): contraction left to right through two ping-pong buffers
// of dim * maxdim entries each (the partial contraction over sites 0..j has d^{j+1} chi_{j+1}).
__global__ void __launch_bounds__(kThreads) k_mps_dense(Engine e, int c, double2* mv, double2* bufa, double2* bufb, long long dim) {
  Ctx C = make_ctx(e, c);
  const int n = C.n, d = e.d;
  double2* cur = bufa;
  double2* nxt = bufb;
  long long rowsn = d;
  int chi = C.dims[1];
  block_copy(cur, site_ptr(C, 0), (long long)d * chi);
  __syncthreads();
  for (int j = 1; j < n; ++j) {
    const int cr = C.dims[j + 1];
    block_matmul(nxt, cur, site_ptr(C, j), (int)rowsn, chi, d * cr);
    __syncthreads();
    double2* t = cur;
    cur = nxt;
    nxt = t;
    rowsn *= d;
    chi = cr;
  }
  block_copy(mv, cur, dim);
}

// For every basis label x: W_x = prod_j D_j^{x_j} = tau^rho W(a, b) from the destabilizer rows.
__global__ void k_weyl_of_labels(Engine e, int c, long long dim, int* aidx, uint8_t* bdig, int* rho) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= dim) return;
  Ctx C = make_ctx(e, c);
  const int n = C.n, d = e.d;
  int ax[kMaxN], az[kMaxN];
  for (int j = 0; j < n; ++j) ax[j] = az[j] = 0;
  int r = 0;
  long long t = x;
  int digs[kMaxN];
  for (int j = n - 1; j >= 0; --j) {
    digs[j] = (int)(t % d);
    t /= d;
  }
  for (int q = 0; q < n; ++q) {
    const uint8_t* R = C.fx + (long long)(n + q) * 2 * n;
    for (int p = 0; p < digs[q]; ++p) {
      int dot = 0;
      for (int j = 0; j < n; ++j) dot += az[j] * R[j];
      r += C.fr[n + q] + 2 * dot;
      for (int j = 0; j < n; ++j) {
        ax[j] = (ax[j] + R[j]) % d;
        az[j] = (az[j] + R[n + j]) % d;
      }
    }
  }
  int ai = 0;
  for (int j = 0; j < n; ++j) {
    ai = ai * d + ax[j];
    bdig[x * n + j] = (uint8_t)az[j];
  }
  aidx[x] = ai;
  rho[x] = r % (2 * d);
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// C|0>: common +1 eigenvector of the stabilizer rows, by projecting a fixed pseudo-random vector
// with prod_j (1/d) sum_m S_j^m, then normalising.  One CTA.
__global__ void __launch_bounds__(kThreads) k_stab_state(Engine e, int c, long long dim, double2* v, double2* w) {
  __shared__ Smem s;
  Ctx C = make_ctx(e, c);
  init_tau(s, e.d);
  const int n = C.n, d = e.d;
  for (long long y = threadIdx.x; y < dim; y += blockDim.x) {
    const unsigned long long h = mix64((unsigned long long)y * 2 + 1);
    const unsigned long long g = mix64((unsigned long long)y * 2 + 2);
    v[y] = make_double2((double)(h >> 11) / 9007199254740992.0 - 0.5, (double)(g >> 11) / 9007199254740992.0 - 0.5);
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const uint8_t* R = C.fx + (long long)j * 2 * n;
    const int r = C.fr[j];
    // S^m = tau^{r m + 2 sxz m(m-1)/2} W(m x, m z); (W(a,b) v)(y) = omega^{b.(y-a)} v(y-a)
    int sxz = 0;
    for (int q = 0; q < n; ++q) sxz += R[q] * R[n + q];
    for (long long y = threadIdx.x; y < dim; y += blockDim.x) {
      double2 acc = cz();
      for (int m = 0; m < d; ++m) {
        long long src = 0;
        int dot = 0;
        long long t = y;
        long long pw = 1;
        for (int q = n - 1; q >= 0; --q) {
          const int yq = (int)(t % d);
          t /= d;
          const int aq = (m * R[q]) % d, bq = (m * R[n + q]) % d;
          const int sq = (yq - aq + d) % d;
          dot += bq * sq;
          src += sq * pw;
          pw *= d;
        }
        const int ph = (r * m + 2 * (sxz % d) * (m * (m - 1) / 2) + 2 * dot) % (2 * d);
        acc = cfma(s.tau[ph], v[src], acc);
      }
      w[y] = cscale(acc, 1.0 / d);
    }
    __syncthreads();
    block_copy(v, w, dim);
    __syncthreads();
  }
  double nrm = 0;
  for (long long y = threadIdx.x; y < dim; y += blockDim.x) nrm += cabs2(v[y]);
  nrm = block_sum(nrm, s);
  const double inv = nrm > 0 ? 1.0 / sqrt(nrm) : 0.0;
  for (long long y = threadIdx.x; y < dim; y += blockDim.x) v[y] = cscale(v[y], inv);
}

// psi(y) = sum_x M_x tau^{rho(x)} omega^{b(x).(y - a(x))} s0(y - a(x)) for the requested labels y.
__global__ void k_apply_clifford_dense(Engine e, int c, long long dim, const double2* mv, const double2* s0,
                                       const int* aidx, const uint8_t* bdig, const int* rho,
                                       const int32_t* ys, long long nys, double2* out) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nys) return;
  const int n = e.nq[c], d = e.d;
  const long long y = ys ? ys[t] : t;
  int yd[kMaxN];
  {
    long long u = y;
    for (int j = n - 1; j >= 0; --j) {
      yd[j] = (int)(u % d);
      u /= d;
    }
  }
  double2 tau_t[6];
  for (int k = 0; k < 2 * d; ++k) {
    double sn, cs;
    sincospi((double)k / d, &sn, &cs);
    tau_t[k] = make_double2(cs, sn);
  }
  double2 acc = cz();
  for (long long x = 0; x < dim; ++x) {
    const double2 mx = mv[x];
    if (mx.x == 0.0 && mx.y == 0.0) continue;
    int ai = aidx[x];
    long long src = 0, pw = 1;
    int dot = 0;
    for (int j = n - 1; j >= 0; --j) {
      const int aj = ai % d;
      ai /= d;
      const int sj = (yd[j] - aj + d) % d;
      dot += bdig[x * n + j] * sj;
      src += sj * pw;
      pw *= d;
    }
    const double2 sv = s0[src];
    if (sv.x == 0.0 && sv.y == 0.0) continue;
    const int ph = (rho[x] + 2 * dot) % (2 * d);
    acc = cfma(cmul(mx, tau_t[ph]), sv, acc);
  }
  out[t] = acc;
}


// <M1|M2> for circuit c1 of e1 and circuit c2 of e2 (same n and d; Sec. 2.4 MPS): transfer matrices
// E[a1][a2] from the left, T[a1][s][b2] = sum_a2 E[a1][a2] B[a2][s][b2], then
// E'[b1][b2] = sum_{a1, s} conj(A[a1][s][b1]) T[a1][s][b2]; FP64, one CTA, scratch of circuit c1.
__global__ void __launch_bounds__(kThreads) k_overlap(Engine e1, int c1, Engine e2, int c2, double2* out) {
  const Ctx A = make_ctx(e1, c1), B = make_ctx(e2, c2);
  const int n = A.n, d = e1.d;
  double2* E = A.scr + e1.sl.b;
  double2* T = A.scr + e1.sl.tmp;
  if (threadIdx.x == 0) E[0] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int la = A.dims[j], ra = A.dims[j + 1], lb = B.dims[j], rb = B.dims[j + 1];
    const double2* Aj = site_ptr(A, j);
    const double2* Bj = site_ptr(B, j);
    for (long long idx = threadIdx.x; idx < (long long)la * d * rb; idx += blockDim.x) {
      const int a1 = (int)(idx / (d * rb)), sb = (int)(idx % (d * rb));
      double2 acc = cz();
      for (int a2 = 0; a2 < lb; ++a2) acc = cfma(E[(long long)a1 * lb + a2], Bj[(long long)a2 * d * rb + sb], acc);
      T[idx] = acc;
    }
    __syncthreads();
    for (long long idx = threadIdx.x; idx < (long long)ra * rb; idx += blockDim.x) {
      const int b1 = (int)(idx / rb), b2 = (int)(idx % rb);
      double2 acc = cz();
      for (int as = 0; as < la * d; ++as) acc = cfmac(Aj[(long long)as * ra + b1], T[(long long)as * rb + b2], acc);
      E[idx] = acc;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = E[0];
}

}  // namespace

cudaError_t launch_overlap(const Engine& e1, int c1, const Engine& e2, int c2, double2* out_dev, cudaStream_t st) {
  k_overlap<<<1, kThreads, 0, st>>>(e1, c1, e2, c2, out_dev);
  return cudaGetLastError();
}

cudaError_t launch_run(const Engine& e, const gcamps_op* ops_dev, const int32_t* begin_dev, cudaStream_t st) {
  if (e.precision) return launch_run_tc(e, ops_dev, begin_dev, st);
  return launch_cluster(k_run, e, st, e, ops_dev, begin_dev);
}

cudaError_t launch_reset(const Engine& e, cudaStream_t st) {
  k_reset<<<e.batch, kThreads, 0, st>>>(e);
  return cudaGetLastError();
}

cudaError_t launch_expect(const Engine& e, int circuit, const int8_t* xz_dev, double2* out_dev, cudaStream_t st) {
  k_expect<<<1, kThreads, 0, st>>>(e, circuit, xz_dev, out_dev);
  return cudaGetLastError();
}

// work layout: bufa[dim * maxdim] | bufb[dim * maxdim] | mv[dim] | s0[dim] | w[dim] | aidx[dim] |
// rho[dim] | bdig[dim * n]
cudaError_t launch_statevector(const Engine& e, int circuit, double2* out_dev, long long dim,
                               const int32_t* ys_dev, long long nys, void* work, cudaStream_t st) {
  const long long nbuf = dim * (long long)e.maxdim;
  double2* bufa = reinterpret_cast<double2*>(work);
  double2* bufb = bufa + nbuf;
  double2* mv = bufb + nbuf;
  double2* s0 = mv + dim;
  double2* w = s0 + dim;
  int* aidx = reinterpret_cast<int*>(w + dim);
  int* rho = aidx + dim;
  uint8_t* bdig = reinterpret_cast<uint8_t*>(rho + dim);
  k_mps_dense<<<1, kThreads, 0, st>>>(e, circuit, mv, bufa, bufb, dim);
  const int blk = 128;
  k_weyl_of_labels<<<(unsigned)((dim + blk - 1) / blk), blk, 0, st>>>(e, circuit, dim, aidx, bdig, rho);
  k_stab_state<<<1, kThreads, 0, st>>>(e, circuit, dim, s0, w);
  k_apply_clifford_dense<<<(unsigned)((nys + blk - 1) / blk), blk, 0, st>>>(e, circuit, dim, mv, s0, aidx, bdig, rho,
                                                                          ys_dev, nys, out_dev);
  return cudaGetLastError();
}

}  // namespace gcx
