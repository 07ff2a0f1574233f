// Adjoint phase gradient of libgcamps (through the MPO applications of Sec. 3).

#include "gcamps_device.cuh"

namespace gcx {
namespace {

// ---------------------------------------------------------------- adjoint phase gradient
// <B| W(m a, m b) |M> for two MPS on the same n sites, W(a, b) = (x)_j X_j^{a_j} Z_j^{b_j} (no phase):
// B's sites through site_ptr(CB, j) and CB.dims, M packed at mbase with bond dimensions mdims and
// site offsets moff.  Transfer matrices E[a, a'] left to right, scratch in CB.
__device__ double2 overlap_weyl(Smem& s, const Ctx& CB, const double2* mbase, const int* mdims,
                                const long long* moff, const uint8_t* row, int mp) {
  const Engine& e = *CB.e;
  const int n = CB.n, d = CB.d;
  double2* E = CB.scr + e.sl.b;
  double2* T = CB.scr + e.sl.tmp;
  double2* E2 = CB.scr + e.sl.u;
  if (threadIdx.x == 0) E[0] = make_double2(1.0, 0.0);
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const int bl = CB.dims[j], br = CB.dims[j + 1], ml = mdims[j], mr = mdims[j + 1];
    const double2* A = site_ptr(CB, j);
    const double2* M = mbase + moff[j];
    const int ax = (mp * row[j]) % d, bz = (mp * row[n + j]) % d;
    // T[a, s, b'] = sum_{a'} E[a, a'] omega^{bz (s - ax)} M[a', s - ax, b']
    for (long long idx = threadIdx.x; idx < (long long)bl * d * mr; idx += blockDim.x) {
      const int bp = (int)(idx % mr), sd = (int)((idx / mr) % d), a = (int)(idx / ((long long)mr * d));
      const int sp = (sd - ax + d) % d;
      double2 acc = cz();
      for (int ap = 0; ap < ml; ++ap) acc = cfma(E[(long long)a * ml + ap], M[((long long)ap * d + sp) * mr + bp], acc);
      T[idx] = cmul(s.tau[(2 * bz * sp) % (2 * d)], acc);
    }
    __syncthreads();
    // E'[b, b'] = sum_{a, s} conj(A[a, s, b]) T[a, s, b']
    for (long long idx = threadIdx.x; idx < (long long)br * mr; idx += blockDim.x) {
      const int b = (int)(idx / mr), bp = (int)(idx % mr);
      double2 acc = cz();
      for (int a = 0; a < bl; ++a)
        for (int sd = 0; sd < d; ++sd)
          acc = cfmac(A[((long long)a * d + sd) * br + b], T[((long long)a * d + sd) * mr + bp], acc);
      E2[idx] = acc;
    }
    __syncthreads();
    block_copy(E, E2, (long long)br * mr);
    __syncthreads();
  }
  const double2 v = E[0];
  __syncthreads();
  return v;
}

// theta <- Q_q^dag theta on sites (i, i+1) of CB's MPS (undoing an applied disentangler), split by SVD
// with the centre left at i + 1.
__device__ void undo_disentangler(Smem& s, const Ctx& CB, int i, int q) {
  const Engine& e = *CB.e;
  const int d = CB.d, dd = d * d;
  move_center(s, CB, i);
  const int cl = CB.dims[i], ch = CB.dims[i + 1], cr = CB.dims[i + 2];
  double2* theta = CB.scr + e.sl.theta;
  double2* tmp = CB.scr + e.sl.tmp;
  block_matmul(theta, site_ptr(CB, i), site_ptr(CB, i + 1), cl * d, ch, d * cr);
  __syncthreads();
  const double2* Q = e.candU + (long long)q * dd * dd;
  const long long total = (long long)cl * dd * cr;
  for (long long idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int b = (int)(idx % cr), u = (int)((idx / cr) % dd);
    const long long a = idx / ((long long)cr * dd);
    double2 acc = cz();
    for (int v = 0; v < dd; ++v) acc = cfmac(Q[v * dd + u], theta[(a * dd + v) * cr + b], acc);   // conj(Q[v][u])
    tmp[idx] = acc;
  }
  __syncthreads();
  block_copy(theta, tmp, total);
  __syncthreads();
  const int bb = CB.bond_bound[i + 1];
  Factor F = svd_factor(s, CB, theta, cl * d, d * cr, e.chi_max < bb ? e.chi_max : bb, false);
  const int k = F.k;
  for (long long idx = threadIdx.x; idx < (long long)k * d * cr; idx += blockDim.x)
    F.Vh[idx] = cscale(F.Vh[idx], CB.sing[idx / (d * cr)]);
  __syncthreads();
  block_copy(site_ptr(CB, i), F.U, (long long)cl * d * k);
  block_copy(site_ptr(CB, i + 1), F.Vh, (long long)k * d * cr);
  if (threadIdx.x == 0) {
    CB.dims[i + 1] = k;
    CB.meta[M_OC] = i + 1;
  }
  __syncthreads();
}

// d Re<W> / d phi_{k,j} for every recorded non-Clifford gate k of circuit cf (gate k =
// diag(e^{i phi_{k,j}})), by the adjoint method in the forward run's own Clifford frames:
//   lambda_K = O psi with O = (W + W^dag)/2 = C (P + P^dag)/2 C^dag, P = C^dag W C (final frame);
//   for k = K-1 .. 0: undo the disentanglers applied after gate k (Q^dag, reverse order), which puts
//   lambda in the frame C'_k of gate k's MPO; take g_{k,j} = -2 Im <lambda| Pi_j |phi_k> with
//   phi_k = snapshot k and Pi_j = (1/d) sum_m omega^{-mj} P_k^m (P_k = gate k's string); apply
//   D_k^dag = sum_m c_m(-phi) P_k^m.  Cliffords between gates only change the frame.
// Circuit slot cb holds lambda (its first n sites).  grad: d doubles per gate.
__global__ void __launch_bounds__(kThreads, kMinCtas) k_adjoint(Engine e, int cf, int cb, const int8_t* xz, double* grad) {
  __shared__ Smem s;
  __shared__ int ax[kMaxN], az[kMaxN], ar;
  __shared__ uint8_t row[2 * kMaxN];
  __shared__ long long moff[kMaxN + 1];
  Ctx F = make_ctx(e, cf);
  Ctx B = make_ctx(e, cb);
  const int n = F.n, d = e.d;
  B.n = n;   // the workspace slot has room for n_max >= n sites
  init_tau(s, d);
  for (int j = 0; j < n; ++j) block_copy(site_ptr(B, j), site_ptr(F, j), (long long)F.dims[j] * d * F.dims[j + 1]);
  for (int j = threadIdx.x; j <= n; j += blockDim.x) B.dims[j] = F.dims[j];
  if (threadIdx.x < M_COUNT) B.meta[threadIdx.x] = 0;
  if (threadIdx.x < kDStats) B.dstats[threadIdx.x] = 0.0;
  __syncthreads();
  if (threadIdx.x == 0) B.meta[M_OC] = F.meta[M_OC];
  conj_weyl(s, F, xz, ax, az, &ar);
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    row[j] = (uint8_t)ax[j];
    row[n + j] = (uint8_t)az[j];
  }
  if (threadIdx.x == 0) {
    for (int m = 0; m < d; ++m) s.coef[m] = cz();
    s.coef[1].x += 0.5;
    s.coef[d - 1].x += 0.5;   // P^(d-1) = P^dag
  }
  __syncthreads();
  bool has_w = false;
  for (int j = 0; j < n; ++j) has_w |= (row[j] | row[n + j]) != 0;
  if (has_w) mpo_apply(s, B, row, ar, false);
  const int K = F.meta[M_NSNAP];
  const int ndec = F.meta[M_NDEC];
  for (int k = K - 1; k >= 0 && B.meta[M_STATUS] == 0; --k) {
    const int* hd = e.snap_hdr + ((long long)cf * e.snap_max + k) * kSnapHdr;
    const int dec0 = hd[3];
    const int dec1 = k + 1 < K ? hd[kSnapHdr + 3] : ndec;
    if (dec1 > kDecCap) {
      if (threadIdx.x == 0) set_status(B, GCAMPS_EINVAL);
      __syncthreads();
      break;
    }
    for (int idx = dec1 - 1; idx >= dec0; --idx) {
      const int bond = F.dec[2 * idx], q = F.dec[2 * idx + 1];
      if (q) undo_disentangler(s, B, bond, q);
    }
    // gate k's string, phase and snapshot
    for (int j = threadIdx.x; j < 2 * n; j += blockDim.x) row[j] = (uint8_t)hd[kSnapDims + kMaxN + 1 + j];
    if (threadIdx.x == 0) {
      long long o = 0;
      for (int j = 0; j < n; ++j) {
        moff[j] = o;
        o += (long long)hd[kSnapDims + j] * d * hd[kSnapDims + j + 1];
      }
      int sxz = 0;
      for (int j = 0; j < n; ++j) sxz += row[j] * row[n + j];
      s.ival[6] = sxz % d;
    }
    __syncthreads();
    const int rk = hd[2], sxz = s.ival[6];
    const double2* mbase = e.snap + (long long)cf * e.snap_stride + hd[0];
    double2 proj[3] = {cz(), cz(), cz()};
    for (int m = 0; m < d; ++m) {
      const double2 ov = overlap_weyl(s, B, mbase, hd + kSnapDims, moff, row, m);
      const double2 pm = cmul(s.tau[(rk * m + 2 * sxz * (m * (m - 1) / 2)) % (2 * d)], ov);   // <B|P^m|M>
      for (int j = 0; j < d; ++j) proj[j] = cadd(proj[j], cscale(cmul(s.tau[(2 * d - (2 * m * j) % (2 * d)) % (2 * d)], pm), 1.0 / d));
    }
    if (threadIdx.x == 0)
      for (int j = 0; j < d; ++j) grad[(long long)k * d + j] = -2.0 * proj[j].y;
    // D_k^dag = sum_m c_m(-phi) P_k^m
    const double* ph = e.snap_ph + ((long long)cf * e.snap_max + k) * 4;
    if (threadIdx.x == 0)
      for (int m = 0; m < d; ++m) {
        double re = 0, im = 0;
        for (int j = 0; j < d; ++j) {
          double sn, cs;
          sincos(-ph[j] - 2.0 * CUDART_PI * (double)(m * j) / d, &sn, &cs);
          re += cs;
          im += sn;
        }
        s.coef[m] = make_double2(re / d, im / d);
      }
    __syncthreads();
    mpo_apply(s, B, row, rk, false);
  }
}

}  // namespace

cudaError_t launch_adjoint(const Engine& e, int cf, int cb, const int8_t* xz_dev, double* grad_dev, cudaStream_t st) {
  k_adjoint<<<1, kThreads, 0, st>>>(e, cf, cb, xz_dev, grad_dev);
  return cudaGetLastError();
}

}  // namespace gcx
