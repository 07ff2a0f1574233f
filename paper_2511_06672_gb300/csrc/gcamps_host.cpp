// Host side of libgcamps: the C ABI of include/gcamps.h, argument validation, device memory,
// and the one-time construction of the two-qudit disentangler classes (Sec. 3, Sec. 3.1).
//
// Nothing here computes a step of the simulation: every call enqueues kernels of
// gcamps_engine.cu on the handle's stream.  The host code only (a) checks arguments, (b) builds
// per-d constant tables once (the symplectic group Sp(4, F_d), its classes modulo single-qudit
// Cliffords, the class unitaries), and (c) moves inputs and outputs.

#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "gcamps_internal.h"

namespace gcx {
cudaError_t launch_run_all(const Engine& e, const gcamps_op* ops_dev, int nops, cudaStream_t st);
}

using gcx::Engine;
using cplx = std::complex<double>;

namespace {

// ------------------------------------------------------------------ symplectic group Sp(4, F_d)
// A 4x4 matrix over F_d is stored as 16 base-d digits, row-major, most significant first, so the
// numeric order of codes is the lexicographic order of the row-major entries.  Column k holds the
// exponents (x_q0, z_q0, x_q1, z_q1) of the image of generator k (X_q0, Z_q0, X_q1, Z_q1).
using Mat4 = std::array<int, 16>;

uint64_t encode(const Mat4& m, int d) {
  uint64_t c = 0;
  for (int i = 0; i < 16; ++i) c = c * d + (uint64_t)m[i];
  return c;
}
Mat4 decode(uint64_t c, int d) {
  Mat4 m{};
  for (int i = 15; i >= 0; --i) {
    m[i] = (int)(c % d);
    c /= d;
  }
  return m;
}
Mat4 matmul4(const Mat4& a, const Mat4& b, int d) {
  Mat4 r{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      int s = 0;
      for (int k = 0; k < 4; ++k) s += a[4 * i + k] * b[4 * k + j];
      r[4 * i + j] = s % d;
    }
  return r;
}
Mat4 from_columns(const int cols[4][4]) {
  Mat4 m{};
  for (int c = 0; c < 4; ++c)
    for (int r = 0; r < 4; ++r) m[4 * r + c] = cols[c][r];
  return m;
}

// Lambda(u, v) = sum_q z_q(u) x_q(v) - x_q(u) z_q(v)  (W(u) W(v) = omega^Lambda W(v) W(u)).
int lam(const int* u, const int* v, int nq, int d) {
  int s = 0;
  for (int q = 0; q < nq; ++q) s += u[2 * q + 1] * v[2 * q] - u[2 * q] * v[2 * q + 1];
  return ((s % d) + d) % d;
}

struct Tables {
  int d = 0;
  std::vector<uint64_t> sp4;                 // sorted codes
  std::vector<Mat4> reps;                    // class representatives, class 0 = identity
  std::vector<int32_t> img;                  // [K][20]
  std::vector<double> u;                     // [K][d^4][2] unitaries
};

// BFS closure of the generators H_0, S_0, H_1, S_1, SUM_01 (Table 1) acting by left
// multiplication; the Clifford group modulo Weyl shifts and phases is Sp(4, F_d).
std::vector<uint64_t> enumerate_sp4(int d) {
  const int m1 = d - 1;
  const int H0[4][4] = {{0, 1, 0, 0}, {m1, 0, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  const int S0[4][4] = {{1, 1, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  const int H1[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 0, 1}, {0, 0, m1, 0}};
  const int S1[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 1}, {0, 0, 0, 1}};
  const int SUM[4][4] = {{1, 0, 1, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, m1, 0, 1}};
  const Mat4 gens[5] = {from_columns(H0), from_columns(S0), from_columns(H1), from_columns(S1),
                        from_columns(SUM)};
  uint64_t space = 1;
  for (int i = 0; i < 16; ++i) space *= d;
  std::vector<uint8_t> seen(space / 8 + 1, 0);
  Mat4 id{};
  for (int i = 0; i < 4; ++i) id[5 * i] = 1;
  std::vector<uint64_t> out;
  std::vector<Mat4> frontier{id};
  const uint64_t c0 = encode(id, d);
  seen[c0 >> 3] |= (uint8_t)(1u << (c0 & 7));
  out.push_back(c0);
  while (!frontier.empty()) {
    std::vector<Mat4> next;
    for (const Mat4& m : frontier)
      for (const Mat4& g : gens) {
        const Mat4 p = matmul4(g, m, d);
        const uint64_t c = encode(p, d);
        if (seen[c >> 3] & (1u << (c & 7))) continue;
        seen[c >> 3] |= (uint8_t)(1u << (c & 7));
        out.push_back(c);
        next.push_back(p);
      }
    frontier.swap(next);
  }
  std::sort(out.begin(), out.end());
  return out;
}

int std_phase(const int* v, int d) {
  if (d % 2) return 0;
  return (v[0] * v[1] + v[2] * v[3]) % (2 * d);
}

// Images (x0, z0, x1, z1, r) of the generators for  W(shift) U_S.
void images_of(const Mat4& s, const int* shift, int d, int32_t* img) {
  for (int k = 0; k < 4; ++k) {
    int v[4];
    for (int r = 0; r < 4; ++r) v[r] = s[4 * r + k];
    const int ph = std_phase(v, d) + 2 * lam(shift, v, 2, d);
    for (int r = 0; r < 4; ++r) img[5 * k + r] = v[r];
    img[5 * k + 4] = ph % (2 * d);
  }
}

// Dense matrix of tau^r X^x0 Z^z0 (x) X^x1 Z^z1 (qudit 0 most significant).
std::vector<cplx> weyl_dense(const int32_t* w, int d) {
  const int D = d * d;
  std::vector<cplx> m(D * D, 0.0);
  const double pi = 3.14159265358979323846;
  for (int yp = 0; yp < D; ++yp) {
    const int y0 = yp / d, y1 = yp % d;
    const int o0 = (y0 + w[0]) % d, o1 = (y1 + w[2]) % d;
    const int ph = w[4] + 2 * (w[1] * y0 + w[3] * y1);   // tau units
    m[(o0 * d + o1) * D + yp] = std::polar(1.0, pi * (double)(ph % (2 * d)) / d);
  }
  return m;
}

std::vector<cplx> mm(const std::vector<cplx>& a, const std::vector<cplx>& b, int D) {
  std::vector<cplx> r(D * D, 0.0);
  for (int i = 0; i < D; ++i)
    for (int k = 0; k < D; ++k) {
      const cplx aik = a[i * D + k];
      if (aik == 0.0) continue;
      for (int j = 0; j < D; ++j) r[i * D + j] += aik * b[k * D + j];
    }
  return r;
}

// The Clifford with the given generator images: U|00> = v, the common +1 eigenvector of the
// images of Z_0, Z_1 (first entry above 1e-8 in modulus made real positive);
// U|y0 y1> = Ximg_0^{y0} Ximg_1^{y1} v.
std::vector<cplx> unitary_from_images(const int32_t* img, int d) {
  const int D = d * d;
  std::vector<cplx> proj(D * D, 0.0);
  for (int i = 0; i < D; ++i) proj[i * D + i] = 1.0;
  for (int q = 0; q < 2; ++q) {
    const std::vector<cplx> z = weyl_dense(img + 5 * (2 * q + 1), d);
    std::vector<cplx> acc(D * D, 0.0), p(D * D, 0.0);
    for (int i = 0; i < D; ++i) p[i * D + i] = 1.0;
    for (int m = 0; m < d; ++m) {
      for (int i = 0; i < D * D; ++i) acc[i] += p[i];
      p = mm(p, z, D);
    }
    for (auto& a : acc) a /= (double)d;
    proj = mm(proj, acc, D);
  }
  int best = 0;
  double bn = -1;
  for (int c = 0; c < D; ++c) {
    double s = 0;
    for (int r = 0; r < D; ++r) s += std::norm(proj[r * D + c]);
    if (s > bn + 1e-12) {
      bn = s;
      best = c;
    }
  }
  std::vector<cplx> v(D);
  double nrm = 0;
  for (int r = 0; r < D; ++r) {
    v[r] = proj[r * D + best];
    nrm += std::norm(v[r]);
  }
  nrm = std::sqrt(nrm);
  for (auto& a : v) a /= nrm;
  for (int r = 0; r < D; ++r)
    if (std::abs(v[r]) > 1e-8) {
      const cplx ph = std::abs(v[r]) / v[r];
      for (auto& a : v) a *= ph;
      break;
    }
  const std::vector<cplx> x0 = weyl_dense(img + 0, d), x1 = weyl_dense(img + 10, d);
  std::vector<cplx> u(D * D, 0.0);
  for (int y = 0; y < D; ++y) {
    std::vector<cplx> col = v;
    const int reps[2] = {y / d, y % d};
    for (int q = 0; q < 2; ++q)
      for (int t = 0; t < reps[q]; ++t) {
        const std::vector<cplx>& x = q ? x1 : x0;
        std::vector<cplx> nc(D, 0.0);
        for (int i = 0; i < D; ++i)
          for (int j = 0; j < D; ++j) nc[i] += x[i * D + j] * col[j];
        col.swap(nc);
      }
    for (int i = 0; i < D; ++i) u[i * D + y] = col[i];
  }
  return u;
}

// Classes {(L_0 (+) L_1) S} of Sp(4, F_d) under single-qudit symplectic maps applied after S.
// Representative: lexicographically smallest member; the identity class is represented by the
// identity and listed first, the others in representative order.
void build_tables(Tables& t, int d) {
  t.d = d;
  t.sp4 = enumerate_sp4(d);
  std::vector<Mat4> sl2;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b)
      for (int c = 0; c < d; ++c)
        for (int e = 0; e < d; ++e)
          if (((a * e - b * c) % d + d) % d == 1) {
            Mat4 m{};
            m[0] = a;
            m[1] = b;
            m[4] = c;
            m[5] = e;
            sl2.push_back(m);
          }
  std::vector<Mat4> blocks;
  for (const Mat4& a : sl2)
    for (const Mat4& b : sl2) {
      Mat4 m{};
      m[0] = a[0];
      m[1] = a[1];
      m[4] = a[4];
      m[5] = a[5];
      m[10] = b[0];
      m[11] = b[1];
      m[14] = b[4];
      m[15] = b[5];
      blocks.push_back(m);
    }
  std::vector<int> cls(t.sp4.size(), -1);
  std::vector<Mat4> reps;
  for (size_t i = 0; i < t.sp4.size(); ++i) {
    if (cls[i] >= 0) continue;
    const Mat4 s = decode(t.sp4[i], d);
    const int id = (int)reps.size();
    reps.push_back(s);
    for (const Mat4& b : blocks) {
      const uint64_t c = encode(matmul4(b, s, d), d);
      const size_t pos = (size_t)(std::lower_bound(t.sp4.begin(), t.sp4.end(), c) - t.sp4.begin());
      cls[pos] = id;
    }
  }
  Mat4 id{};
  for (int i = 0; i < 4; ++i) id[5 * i] = 1;
  const size_t ipos = (size_t)(std::lower_bound(t.sp4.begin(), t.sp4.end(), encode(id, d)) - t.sp4.begin());
  const int idc = cls[ipos];
  t.reps.clear();
  t.reps.push_back(id);
  for (int c = 0; c < (int)reps.size(); ++c)
    if (c != idc) t.reps.push_back(reps[c]);
  const int K = (int)t.reps.size();
  const int D = d * d;
  t.img.assign((size_t)K * 20, 0);
  t.u.assign((size_t)K * D * D * 2, 0.0);
  const int zero[4] = {0, 0, 0, 0};
  for (int k = 0; k < K; ++k) {
    images_of(t.reps[k], zero, d, &t.img[(size_t)k * 20]);
    const std::vector<cplx> u = unitary_from_images(&t.img[(size_t)k * 20], d);
    for (int i = 0; i < D * D; ++i) {
      t.u[((size_t)k * D * D + i) * 2] = u[i].real();
      t.u[((size_t)k * D * D + i) * 2 + 1] = u[i].imag();
    }
  }
}

Tables g_tables[4];
std::once_flag g_once[4];

const Tables& tables(int d) {
  std::call_once(g_once[d], [d] { build_tables(g_tables[d], d); });
  return g_tables[d];
}

// Symplectic images with phases of order d.  nq = 1: img[3k..3k+2] = (x, z, r).
bool valid_images(const int32_t* img, int nq, int d, std::string* why) {
  int v[4][5];
  for (int k = 0; k < 2 * nq; ++k) {
    for (int f = 0; f < 5; ++f) v[k][f] = 0;
    if (nq == 2) {
      for (int f = 0; f < 5; ++f) v[k][f] = img[5 * k + f];
    } else {
      v[k][0] = img[3 * k];
      v[k][1] = img[3 * k + 1];
      v[k][4] = img[3 * k + 2];
    }
    for (int f = 0; f < 4; ++f)
      if (v[k][f] < 0 || v[k][f] >= d) {
        *why = "image exponent out of range [0, d)";
        return false;
      }
    if (v[k][4] < 0 || v[k][4] >= 2 * d) {
      *why = "image phase out of range [0, 2d)";
      return false;
    }
    if (d % 2) {
      if (v[k][4] % 2) {
        *why = "odd d: image phase must be a power of omega (even in units of tau)";
        return false;
      }
    } else {
      const int xz = v[k][0] * v[k][1] + v[k][2] * v[k][3];
      if ((v[k][4] + xz) % 2) {
        *why = "d = 2: image must be Hermitian (phase + x.z even)";
        return false;
      }
    }
  }
  for (int i = 0; i < 2 * nq; ++i)
    for (int j = 0; j < 2 * nq; ++j) {
      int ei[4] = {0, 0, 0, 0}, ej[4] = {0, 0, 0, 0};
      ei[i] = 1;
      ej[j] = 1;
      if (lam(v[i], v[j], nq, d) != lam(ei, ej, nq, d)) {
        *why = "images are not symplectic";
        return false;
      }
    }
  return true;
}

}  // namespace

// ------------------------------------------------------------------------------------ handle
struct gcamps {
  Engine e{};
  std::vector<int> nq;                 // qudits of each circuit
  std::vector<long long> site_off;     // [batch][n_max + 1] slot offsets within a circuit's block
  std::vector<long long> mps_base;     // [batch] offset of each circuit's block
  int nmin = 0;                        // smallest qudit count of the batch
  int csize_alloc = 0;                 // cluster size the per-CTA scratch was laid out for
  double* grad_dev = nullptr;          // adjoint output (snapshot_max_gates x 4 doubles)
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  void* dev_block = nullptr;      // one allocation for everything but the op buffer
  gcamps_op* ops_dev = nullptr;
  size_t ops_cap = 0;
  int32_t* begin_dev = nullptr;
  int8_t* xz_dev = nullptr;
  double2* out_dev = nullptr;
  double* schmidt_dev = nullptr;
  int* cnt_dev = nullptr;
  int* replay_dev = nullptr;           // [batch][kDecCap][2] recorded decisions to replay
  int* replay_n_dev = nullptr;         // [batch] their counts (0: choose)
};

namespace {

int fail(gcamps_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int cuda_fail(gcamps_t* h, cudaError_t e, const char* where) {
  return fail(h, GCAMPS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GC_CUDA(h, call)                                     \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_fail((h), _e, #call); \
  } while (0)

// Shape limits of a handle: every matrix the engine works on (two-site tensor, Jacobi rotations,
// scored theta' and its Gram) has at most 2^31 - 1 entries, so 32-bit element indices cannot wrap;
// bond capacities d chi are checked first, at a size whose squares cannot overflow 64 bits.
constexpr long long kMaxMatrixEntries = 2147483647LL;
constexpr long long kMaxBondCap = 1LL << 20;

long long sat_pow(int d, int k, long long cap) {
  long long v = 1;
  for (int i = 0; i < k; ++i) {
    v *= d;
    if (v >= cap) return cap;
  }
  return v;
}

int device_status(gcamps_t* h) {
  std::vector<int> meta((size_t)h->e.batch * gcx::M_COUNT);
  cudaError_t e = cudaMemcpyAsync(meta.data(), h->e.meta, meta.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                  h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "device status");
  for (int c = 0; c < h->e.batch; ++c) {
    const int* mc = &meta[(size_t)c * gcx::M_COUNT];
    const int s = mc[gcx::M_STATUS];
    if (s) {
      char buf[192];
      const int where = mc[gcx::M_DIAG_WHERE];
      snprintf(buf, sizeof buf, "device status %d on circuit %d (%s; %s, matrix %d x %d)", s, c,
               s == GCAMPS_ENOCONV ? "iteration cap reached" : (s == GCAMPS_ECHI ? "chi_max bound" : "invalid state"),
               where == 1 ? "Jacobi SVD" : (where == 2 ? "tridiagonal eigenvalues" : "-"), mc[gcx::M_DIAG_A],
               mc[gcx::M_DIAG_B]);
      return fail(h, s, buf);
    }
  }
  return GCAMPS_OK;
}

}  // namespace

extern "C" {

void gcamps_default_opts(gcamps_opts* o) {
  if (!o) return;
  o->cutoff = 1e-12;
  o->max_sweeps = 8;
  o->score_kind = 0;
  o->precision = 0;
  o->tie_tol = 1e-10;
  o->strict_weight = 0.0;
  o->cuda_stream = nullptr;
  o->cluster_size = 8;
  o->snapshot_entries = 0;
  o->snapshot_max_gates = 0;
}

int gcamps_num_candidates(int d) {
  if (d != 2 && d != 3) return -1;
  return (int)tables(d).reps.size();
}

// Images of the named gates, worked out from their definitions (Sec. 2.3) with Z X = omega X Z:
// H X H^dag = Z and H Z H^dag = X^{-1} for the DFT H; S X S^dag = omega^{j} on |j> -> |j+1>, i.e. X Z
// (tau X Z = Y for d = 2); SUM maps X_c -> X_c X_t and Z_t -> Z_c^{-1} Z_t; X Z X^dag = omega^{-1} Z;
// Z X Z^dag = omega X.  Phases in units of tau (omega = tau^2).
int gcamps_named_images(int d, int gate, int32_t* img, int32_t* nq) {
  if ((d != 2 && d != 3) || !img) return GCAMPS_EINVAL;
  const int m1 = d - 1, two_d = 2 * d;
  auto one = [&](int xx, int xz, int xr, int zx, int zz, int zr) {
    const int32_t v[6] = {xx, xz, xr, zx, zz, zr};
    std::memcpy(img, v, sizeof v);
    if (nq) *nq = 1;
    return GCAMPS_OK;
  };
  switch (gate) {
    case GCAMPS_GATE_H: return one(0, 1, 0, m1, 0, 0);
    case GCAMPS_GATE_S: return one(1, 1, d == 2 ? 1 : 0, 0, 1, 0);
    case GCAMPS_GATE_X: return one(1, 0, 0, 0, 1, two_d - 2);
    case GCAMPS_GATE_Z: return one(1, 0, 2, 0, 1, 0);
    case GCAMPS_GATE_SUM: {
      // images of X_c, Z_c, X_t, Z_t as (x_c, z_c, x_t, z_t, phase)
      const int32_t v[20] = {1, 0, 1, 0, 0,   0, 1, 0, 0, 0,   0, 0, 1, 0, 0,   0, m1, 0, 1, 0};
      std::memcpy(img, v, sizeof v);
      if (nq) *nq = 2;
      return GCAMPS_OK;
    }
    default: return GCAMPS_EINVAL;
  }
}

int gcamps_sp4_images(int d, int64_t sp_index, const int32_t* shift, int32_t* img) {
  if ((d != 2 && d != 3) || !img) return GCAMPS_EINVAL;
  const Tables& t = tables(d);
  if (sp_index < 0 || (uint64_t)sp_index >= t.sp4.size()) return GCAMPS_EINVAL;
  int sh[4] = {0, 0, 0, 0};
  if (shift)
    for (int i = 0; i < 4; ++i) {
      if (shift[i] < 0 || shift[i] >= d) return GCAMPS_EINVAL;
      sh[i] = shift[i];
    }
  images_of(decode(t.sp4[(size_t)sp_index], d), sh, d, img);
  return GCAMPS_OK;
}

int gcamps_candidate(int d, int k, int32_t* img, double* u) {
  if ((d != 2 && d != 3) || !img) return GCAMPS_EINVAL;
  const Tables& t = tables(d);
  if (k < 0 || k >= (int)t.reps.size()) return GCAMPS_EINVAL;
  std::memcpy(img, &t.img[(size_t)k * 20], 20 * sizeof(int32_t));
  if (u) {
    const size_t dd = (size_t)d * d * d * d * 2;
    std::memcpy(u, &t.u[(size_t)k * dd], dd * sizeof(double));
  }
  return GCAMPS_OK;
}

int gcamps_create(int n, int d, int chi_max, const gcamps_opts* o, gcamps_t** out) {
  return gcamps_create_batch(1, n, d, chi_max, o, out);
}

int gcamps_create_batch(int batch, int n, int d, int chi_max, const gcamps_opts* o, gcamps_t** out) {
  if (!out) return GCAMPS_EINVAL;
  *out = nullptr;
  if (batch < 1 || n < 2 || n > gcx::kMaxN) return GCAMPS_EINVAL;
  const std::vector<int32_t> nv((size_t)batch, n);
  return gcamps_create_batch_uneven(batch, nv.data(), d, chi_max, o, out);
}

int gcamps_batch_create(int count, const int32_t* n, int d, int chi_max, const gcamps_opts* o, gcamps_t** out) {
  return gcamps_create_batch_uneven(count, n, d, chi_max, o, out);
}

int gcamps_create_batch_uneven(int batch, const int32_t* nqs, int d, int chi_max, const gcamps_opts* o,
                               gcamps_t** out) {
  if (!out) return GCAMPS_EINVAL;
  *out = nullptr;
  if (batch < 1 || !nqs || (d != 2 && d != 3) || chi_max < 1) return GCAMPS_EINVAL;
  int n = 0;
  for (int c = 0; c < batch; ++c) {
    if (nqs[c] < 2 || nqs[c] > gcx::kMaxN) return GCAMPS_EINVAL;
    n = std::max(n, (int)nqs[c]);
  }
  gcamps_opts opts;
  gcamps_default_opts(&opts);
  if (o) opts = *o;
  if (!(opts.cutoff >= 0.0) || opts.max_sweeps < 0 || opts.score_kind < 0 || opts.score_kind > 2 ||
      opts.precision < 0 || opts.precision > 1 || opts.snapshot_entries < 0 || opts.snapshot_max_gates < 0 ||
      (opts.snapshot_entries > 0) != (opts.snapshot_max_gates > 0) || opts.snapshot_entries > (1LL << 31) - 1 ||
      !(opts.tie_tol >= 0.0))
    return GCAMPS_EINVAL;
  if (opts.cluster_size == 0) opts.cluster_size = 8;
  if (opts.cluster_size < 1 || opts.cluster_size > gcx::kMaxCluster)
    return GCAMPS_EINVAL;
  gcamps_t* h = new (std::nothrow) gcamps;
  if (!h) return GCAMPS_ENOMEM;
  const Tables& tb = tables(d);
  Engine& e = h->e;
  e.n = n;
  e.d = d;
  e.K = (int)tb.reps.size();
  e.chi_max = chi_max;
  e.batch = batch;
  e.max_sweeps = opts.max_sweeps;
  e.score_kind = opts.score_kind;
  e.jacobi_cap = 60;
  e.exact_cta_min_m = 10;
  e.precision = opts.precision;
  e.tc_smem = opts.precision ? gcx::kTcSmemBytes : 0;
  e.cutoff = opts.cutoff;
  // FP32 contractions resolve scores to about 1e-6 nats: ties are taken at least that wide
  e.tie_tol = opts.precision ? std::max(opts.tie_tol, gcx::kMixedTieTol) : opts.tie_tol;
  e.strict_weight = opts.strict_weight;
  // bond capacities of each circuit: after the MPO a bond holds at most d * min(chi_max, Schmidt
  // bound); slots of each circuit's sites laid out back to back, circuits one after another
  // with adjoint snapshots one more circuit slot (index batch, n_max qudits) holds the backward state
  const bool snap = opts.snapshot_entries > 0;
  const int nslots = batch + (snap ? 1 : 0);
  h->nq.assign(nqs, nqs + batch);
  if (snap) h->nq.push_back(n);
  h->nmin = *std::min_element(nqs, nqs + batch);
  h->site_off.assign((size_t)nslots * (n + 1), 0);
  h->mps_base.assign((size_t)nslots, 0);
  std::vector<int> bound((size_t)nslots * (n + 1), 1);
  long long maxdim = 1, tcap = 1, mps_total = 0;
  for (int c = 0; c < nslots; ++c) {
    const int nc = h->nq[c];
    std::vector<long long> cap(nc + 1, 1);
    for (int b = 1; b < nc; ++b) {
      const long long sb = sat_pow(d, std::min(b, nc - b), 1LL << 30);
      bound[(size_t)c * (n + 1) + b] = (int)sb;
      cap[b] = d * std::min<long long>(chi_max, sb);
      maxdim = std::max(maxdim, cap[b]);
    }
    if (maxdim > kMaxBondCap) {   // the products below stay far from overflow
      delete h;
      return GCAMPS_EINVAL;
    }
    long long* off = &h->site_off[(size_t)c * (n + 1)];
    for (int j = 0; j < nc; ++j) {
      const long long sz = cap[j] * d * cap[j + 1];
      off[j + 1] = off[j] + sz;
      tcap = std::max(tcap, sz);
      if (j + 2 <= nc) tcap = std::max(tcap, cap[j] * d * d * cap[j + 2]);
    }
    for (int j = nc + 1; j <= n; ++j) off[j] = off[nc];
    h->mps_base[c] = mps_total;
    mps_total += (off[nc] + 31) / 32 * 32;   // 512-byte aligned circuit blocks
  }
  e.maxdim = (int)maxdim;
  const long long maxm = (long long)d * maxdim;
  e.tcap = tcap;
  e.wcap = maxm * maxm;
  gcx::ScratchLayout& sl = e.sl;
  sl.theta = 0;
  sl.b = sl.theta + tcap;
  sl.w = sl.b + tcap;
  sl.u = sl.w + e.wcap;
  sl.vh = sl.u + tcap;
  sl.tmp = sl.vh + tcap;
  sl.total = sl.tmp + tcap;
  e.csize = opts.cluster_size;
  h->csize_alloc = opts.cluster_size;
  gcx::CtaLayout& cly = e.cl;
  cly.warp = 0;
  cly.block = (long long)gcx::kWarps * gcx::kSmallStride;
  // CTA-level scoring sees theta only after compression (every bond <= chi_max), so theta' and its
  // Gram hold at most (d chi_max)^2 entries each
  const long long sside = (long long)d * std::min<long long>(chi_max, maxdim);
  e.scap = sside * sside;
  cly.total = cly.block + 2 * e.scap + sside + 64;
  if (tcap > kMaxMatrixEntries || e.wcap > kMaxMatrixEntries || e.scap > kMaxMatrixEntries) {
    delete h;
    return GCAMPS_EINVAL;
  }
  e.tab_stride = 2LL * (4LL * n * n + 2LL * n);

  e.sing_stride = 4 * maxm + 128;   // singular values | sort scratch / QR betas | QR diagonal
  e.iscr_stride = maxm + 64;
  // one device block, carved up
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t bytes = 0;
  const size_t o_tab = bytes;
  bytes = align(bytes + (size_t)nslots * e.tab_stride);
  const size_t o_mps = bytes;
  bytes = align(bytes + (size_t)mps_total * sizeof(double2));
  const size_t o_off = bytes;
  bytes = align(bytes + (size_t)nslots * (n + 1) * sizeof(long long));
  const size_t o_bound = bytes;
  bytes = align(bytes + (size_t)nslots * (n + 1) * sizeof(int));
  const size_t o_nq = bytes;
  bytes = align(bytes + (size_t)nslots * sizeof(int));
  const size_t o_base = bytes;
  bytes = align(bytes + (size_t)nslots * sizeof(long long));
  const size_t o_dims = bytes;
  bytes = align(bytes + (size_t)nslots * (n + 1) * sizeof(int));
  const size_t o_meta = bytes;
  bytes = align(bytes + (size_t)nslots * gcx::M_COUNT * sizeof(int));
  const size_t o_stats = bytes;
  bytes = align(bytes + (size_t)nslots * gcx::S_COUNT * sizeof(long long));
  const size_t o_prof = bytes;
  bytes = align(bytes + (size_t)nslots * gcx::P_COUNT * sizeof(long long));
  const size_t o_dstats = bytes;
  bytes = align(bytes + (size_t)nslots * gcx::kDStats * sizeof(double));
  const size_t o_dec = bytes;
  bytes = align(bytes + (size_t)nslots * gcx::kDecCap * 2 * sizeof(int));
  const size_t o_weyl = bytes;
  bytes = align(bytes + (size_t)nslots * 2 * n);
  const size_t o_last = bytes;
  bytes = align(bytes + (size_t)nslots * (3 * gcx::kMaxK + 2 + 2 * gcx::kSmall) * sizeof(double));
  const size_t o_scr = bytes;
  bytes = align(bytes + (size_t)nslots * sl.total * sizeof(double2));
  const size_t o_cscr = bytes;
  bytes = align(bytes + (size_t)nslots * e.csize * cly.total * sizeof(double2));
  const size_t o_sing = bytes;
  bytes = align(bytes + (size_t)nslots * e.sing_stride * sizeof(double));
  const size_t o_iscr = bytes;
  bytes = align(bytes + (size_t)nslots * e.iscr_stride * sizeof(int));
  const size_t o_candU = bytes;
  const int D = d * d;
  bytes = align(bytes + (size_t)e.K * D * D * sizeof(double2));
  const size_t o_candU32 = bytes;
  bytes = align(bytes + (size_t)e.K * D * D * sizeof(float2));
  const size_t o_candI = bytes;
  bytes = align(bytes + (size_t)e.K * 20 * sizeof(int32_t));
  const size_t o_snap = bytes;
  if (snap) bytes = align(bytes + (size_t)batch * opts.snapshot_entries * sizeof(double2));
  const size_t o_shdr = bytes;
  if (snap) bytes = align(bytes + (size_t)batch * opts.snapshot_max_gates * gcx::kSnapHdr * sizeof(int));
  const size_t o_sph = bytes;
  if (snap) bytes = align(bytes + (size_t)batch * opts.snapshot_max_gates * 4 * sizeof(double));
  const size_t o_grad = bytes;
  if (snap) bytes = align(bytes + (size_t)opts.snapshot_max_gates * 4 * sizeof(double));
  const size_t o_aux = bytes;
  bytes = align(bytes + (size_t)(gcx::kMaxN * 2 + 64) + 4096);
  if (opts.cuda_stream) {
    h->stream = (cudaStream_t)opts.cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return GCAMPS_ECUDA;
    }
    h->own_stream = true;
  }
  if (cudaMalloc(&h->dev_block, bytes) != cudaSuccess) {
    cudaGetLastError();
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return GCAMPS_ENOMEM;
  }
  char* base = (char*)h->dev_block;
  e.tab = (uint8_t*)(base + o_tab);
  e.mps = (double2*)(base + o_mps);
  e.site_off = (const long long*)(base + o_off);
  e.bond_bound = (const int*)(base + o_bound);
  e.nq = (const int*)(base + o_nq);
  e.mps_base = (const long long*)(base + o_base);
  e.dims = (int*)(base + o_dims);
  e.meta = (int*)(base + o_meta);
  e.stats = (long long*)(base + o_stats);
  e.prof = (long long*)(base + o_prof);
  e.dstats = (double*)(base + o_dstats);
  e.dec = (int*)(base + o_dec);
  e.weyl = (int8_t*)(base + o_weyl);
  e.lastsc = (double*)(base + o_last);
  e.scr = (double2*)(base + o_scr);
  e.cscr = (double2*)(base + o_cscr);
  e.sing = (double*)(base + o_sing);
  e.iscr = (int*)(base + o_iscr);
  e.candU = (const double2*)(base + o_candU);
  e.candU32 = (const float2*)(base + o_candU32);
  if (snap) {
    e.snap = (double2*)(base + o_snap);
    e.snap_stride = opts.snapshot_entries;
    e.snap_hdr = (int*)(base + o_shdr);
    e.snap_max = opts.snapshot_max_gates;
    e.snap_ph = (double*)(base + o_sph);
    h->grad_dev = (double*)(base + o_grad);
  }
  e.candImg = (const int32_t*)(base + o_candI);
  h->xz_dev = (int8_t*)(base + o_aux);
  h->out_dev = (double2*)(base + o_aux + align(gcx::kMaxN * 2));
  h->cnt_dev = (int*)(h->out_dev + 2);
  cudaError_t ce = cudaMemcpyAsync((void*)e.site_off, h->site_off.data(), h->site_off.size() * sizeof(long long),
                                   cudaMemcpyHostToDevice, h->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void*)e.bond_bound, bound.data(), bound.size() * sizeof(int), cudaMemcpyHostToDevice,
                         h->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void*)e.nq, h->nq.data(), h->nq.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void*)e.mps_base, h->mps_base.data(), h->mps_base.size() * sizeof(long long),
                         cudaMemcpyHostToDevice, h->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void*)e.candU, tb.u.data(), tb.u.size() * sizeof(double), cudaMemcpyHostToDevice,
                         h->stream);
  const std::vector<float> u32(tb.u.begin(), tb.u.end());   // lives until the synchronisation below
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void*)e.candU32, u32.data(), u32.size() * sizeof(float), cudaMemcpyHostToDevice,
                         h->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync((void*)e.candImg, tb.img.data(), tb.img.size() * sizeof(int32_t),
                         cudaMemcpyHostToDevice, h->stream);
  if (ce == cudaSuccess) ce = gcx::launch_reset(e, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (ce != cudaSuccess) {
    gcamps_destroy(h);
    return GCAMPS_ECUDA;
  }
  *out = h;
  return GCAMPS_OK;
}

void gcamps_destroy(gcamps_t* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->dev_block) cudaFree(h->dev_block);
  if (h->ops_dev) cudaFree(h->ops_dev);
  if (h->begin_dev) cudaFree(h->begin_dev);
  if (h->schmidt_dev) cudaFree(h->schmidt_dev);
  if (h->replay_dev) cudaFree(h->replay_dev);
  if (h->replay_n_dev) cudaFree(h->replay_n_dev);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char* gcamps_last_error(gcamps_t* h) { return h ? h->err.c_str() : "null handle"; }

int gcamps_apply_clifford(gcamps_t* h, int q0, int q1, const int32_t* img) {
  if (!h) return GCAMPS_EINVAL;
  const int n = h->nmin;   // applied to every circuit
  if (!img || q0 < 0 || q0 >= n || q1 >= n || q1 == q0 || q1 < -1)
    return fail(h, GCAMPS_EINVAL, "bad qudit indices or null images");
  const int nq = q1 < 0 ? 1 : 2;
  std::string why;
  if (!valid_images(img, nq, h->e.d, &why)) return fail(h, GCAMPS_EINVAL, why);
  gcamps_op op;
  std::memset(&op, 0, sizeof op);
  op.kind = GCAMPS_OP_CLIFFORD;
  op.q0 = q0;
  op.q1 = q1;
  std::memcpy(op.img, img, sizeof(int32_t) * (nq == 2 ? 20 : 6));
  GC_CUDA(h, gcx::launch_single(h->e, op, h->stream));
  return GCAMPS_OK;
}

int gcamps_apply_named(gcamps_t* h, int gate, int q0, int q1) {
  if (!h) return GCAMPS_EINVAL;
  int32_t img[20];
  int32_t nq = 0;
  if (gcamps_named_images(h->e.d, gate, img, &nq)) return fail(h, GCAMPS_EINVAL, "unknown named gate");
  if ((nq == 1) != (q1 == -1)) return fail(h, GCAMPS_EINVAL, "q1 must be -1 for one-qudit gates, a qudit for SUM");
  return gcamps_apply_clifford(h, q0, q1, img);
}

int gcamps_apply_nonclifford(gcamps_t* h, int site, const double* phases) {
  if (!h) return GCAMPS_EINVAL;
  if (!phases || site < 0 || site >= h->nmin) return fail(h, GCAMPS_EINVAL, "bad site or null phases");
  gcamps_op op;
  std::memset(&op, 0, sizeof op);
  op.kind = GCAMPS_OP_NONCLIFFORD;
  op.q0 = site;
  op.q1 = -1;
  for (int j = 0; j < h->e.d; ++j) {
    if (!std::isfinite(phases[j])) return fail(h, GCAMPS_EINVAL, "non-finite phase");
    op.phases[j] = phases[j];
  }
  GC_CUDA(h, gcx::launch_single(h->e, op, h->stream));
  return GCAMPS_OK;
}

int gcamps_disentangle(gcamps_t* h, gcamps_stats* st) {
  if (!h) return GCAMPS_EINVAL;
  gcamps_op op;
  std::memset(&op, 0, sizeof op);
  op.kind = GCAMPS_OP_DISENTANGLE;
  GC_CUDA(h, gcx::launch_single(h->e, op, h->stream));
  if (st) return gcamps_get_stats(h, 0, st);
  return GCAMPS_OK;
}

// Ops i in [0, nops) run on circuits with at least n qudits.
static int validate_ops(gcamps_t* h, const gcamps_op* ops, int nops, int n) {
  std::string why;
  for (int i = 0; i < nops; ++i) {
    const gcamps_op& op = ops[i];
    switch (op.kind) {
      case GCAMPS_OP_CLIFFORD: {
        if (op.q0 < 0 || op.q0 >= n || op.q1 >= n || op.q1 == op.q0 || op.q1 < -1)
          return fail(h, GCAMPS_EINVAL, "op " + std::to_string(i) + ": bad qudits");
        if (!valid_images(op.img, op.q1 < 0 ? 1 : 2, h->e.d, &why))
          return fail(h, GCAMPS_EINVAL, "op " + std::to_string(i) + ": " + why);
        break;
      }
      case GCAMPS_OP_NONCLIFFORD:
        if (op.q0 < 0 || op.q0 >= n) return fail(h, GCAMPS_EINVAL, "op " + std::to_string(i) + ": bad site");
        for (int j = 0; j < h->e.d; ++j)
          if (!std::isfinite(op.phases[j])) return fail(h, GCAMPS_EINVAL, "non-finite phase");
        break;
      case GCAMPS_OP_DISENTANGLE:
        break;
      default:
        return fail(h, GCAMPS_EINVAL, "op " + std::to_string(i) + ": unknown kind");
    }
  }
  return GCAMPS_OK;
}

int gcamps_run(gcamps_t* h, const gcamps_op* ops, int nops, const int32_t* begin) {
  if (!h || nops < 0 || (nops > 0 && !ops)) return GCAMPS_EINVAL;
  if (begin) {
    if (begin[0] != 0) return fail(h, GCAMPS_EINVAL, "begin[0] must be 0");
    for (int c = 0; c < h->e.batch; ++c)
      if (begin[c + 1] < begin[c] || begin[c + 1] > nops) return fail(h, GCAMPS_EINVAL, "bad begin offsets");
  }
  int rc = GCAMPS_OK;
  if (begin) {
    for (int c = 0; c < h->e.batch && !rc; ++c)
      rc = validate_ops(h, ops + begin[c], begin[c + 1] - begin[c], h->nq[c]);
  } else {
    rc = validate_ops(h, ops, nops, h->nmin);
  }
  if (rc) return rc;
  if (nops == 0) return GCAMPS_OK;
  if ((size_t)nops > h->ops_cap) {
    if (h->ops_dev) {
      cudaStreamSynchronize(h->stream);
      cudaFree(h->ops_dev);
      h->ops_dev = nullptr;
    }
    size_t cap = 1024;
    while (cap < (size_t)nops) cap *= 2;
    if (cudaMalloc(&h->ops_dev, cap * sizeof(gcamps_op)) != cudaSuccess) {
      cudaGetLastError();
      h->ops_cap = 0;
      return fail(h, GCAMPS_ENOMEM, "op buffer");
    }
    h->ops_cap = cap;
  }
  GC_CUDA(h, cudaMemcpyAsync(h->ops_dev, ops, (size_t)nops * sizeof(gcamps_op), cudaMemcpyHostToDevice, h->stream));
  if (begin) {
    if (!h->begin_dev) GC_CUDA(h, cudaMalloc(&h->begin_dev, (size_t)(h->e.batch + 1) * sizeof(int32_t)));
    GC_CUDA(h, cudaMemcpyAsync(h->begin_dev, begin, (size_t)(h->e.batch + 1) * sizeof(int32_t),
                               cudaMemcpyHostToDevice, h->stream));
    GC_CUDA(h, gcx::launch_run(h->e, h->ops_dev, h->begin_dev, h->stream));
  } else {
    GC_CUDA(h, gcx::launch_run_all(h->e, h->ops_dev, nops, h->stream));
  }
  return GCAMPS_OK;
}

int gcamps_run_device(gcamps_t* h, const gcamps_op* ops_dev, const int32_t* begin_dev) {
  if (!h || !ops_dev || !begin_dev) return GCAMPS_EINVAL;
  GC_CUDA(h, gcx::launch_run(h->e, ops_dev, begin_dev, h->stream));
  return GCAMPS_OK;
}

int gcamps_num_qudits(gcamps_t* h, int circuit) {
  if (!h || circuit < 0 || circuit >= h->e.batch) return -1;
  return h->nq[circuit];
}

int gcamps_set_jacobi_cap(gcamps_t* h, int sweeps) {
  if (!h) return GCAMPS_EINVAL;
  if (sweeps < 1 || sweeps > 1000) return fail(h, GCAMPS_EINVAL, "Jacobi sweep cap outside 1..1000");
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  h->e.jacobi_cap = sweeps;
  return GCAMPS_OK;
}

int gcamps_set_exact_cta(gcamps_t* h, int min_m) {
  if (!h) return GCAMPS_EINVAL;
  if (min_m < 0) return fail(h, GCAMPS_EINVAL, "negative size threshold");
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  h->e.exact_cta_min_m = min_m;
  return GCAMPS_OK;
}

int gcamps_set_cluster_size(gcamps_t* h, int cluster_size) {
  if (!h) return GCAMPS_EINVAL;
  if (cluster_size < 1 || cluster_size > h->csize_alloc)
    return fail(h, GCAMPS_EINVAL, "cluster size must be 1 up to the one the handle was created with");
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  h->e.csize = cluster_size;
  return GCAMPS_OK;
}

int gcamps_sync(gcamps_t* h) {
  if (!h) return GCAMPS_EINVAL;
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  return device_status(h);
}

int gcamps_reset(gcamps_t* h) {
  if (!h) return GCAMPS_EINVAL;
  GC_CUDA(h, gcx::launch_reset(h->e, h->stream));
  return GCAMPS_OK;
}

static int check_circuit(gcamps_t* h, int circuit) {
  if (!h) return GCAMPS_EINVAL;
  if (circuit < 0 || circuit >= h->e.batch) return fail(h, GCAMPS_EINVAL, "circuit index out of range");
  return GCAMPS_OK;
}

int gcamps_batch_expect_weyl(gcamps_t* h, int circuit, const int32_t* x, const int32_t* z, double* re, double* im) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  const int n = h->nq[circuit], d = h->e.d;
  if (!x || !z || !re || !im) return fail(h, GCAMPS_EINVAL, "null argument");
  std::vector<int8_t> xz(2 * n);
  for (int j = 0; j < n; ++j) {
    if (x[j] < 0 || x[j] >= d || z[j] < 0 || z[j] >= d) return fail(h, GCAMPS_EINVAL, "exponent out of range");
    xz[j] = (int8_t)x[j];
    xz[n + j] = (int8_t)z[j];
  }
  GC_CUDA(h, cudaMemcpyAsync(h->xz_dev, xz.data(), 2 * n, cudaMemcpyHostToDevice, h->stream));
  GC_CUDA(h, gcx::launch_expect(h->e, circuit, h->xz_dev, h->out_dev, h->stream));
  double2 r;
  GC_CUDA(h, cudaMemcpyAsync(&r, h->out_dev, sizeof r, cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  *re = r.x;
  *im = r.y;
  return device_status(h);
}

int gcamps_expect_gradient(gcamps_t* h, int circuit, const int32_t* x, const int32_t* z, double* value,
                           double* grad, int32_t cap_gates, int32_t* ngates) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  if (!h->e.snap) return fail(h, GCAMPS_EINVAL, "handle created without snapshots (opts.snapshot_entries)");
  const int n = h->nq[circuit], d = h->e.d;
  if (!x || !z || !value || !ngates || cap_gates < 0 || (cap_gates > 0 && !grad))
    return fail(h, GCAMPS_EINVAL, "null argument");
  double re = 0, im = 0;
  rc = gcamps_batch_expect_weyl(h, circuit, x, z, &re, &im);   // also checks x, z and the device status
  if (rc) return rc;
  *value = re;
  int meta[gcx::M_COUNT];
  GC_CUDA(h, cudaMemcpyAsync(meta, h->e.meta + (long long)circuit * gcx::M_COUNT, sizeof meta, cudaMemcpyDeviceToHost,
                             h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  const int K = meta[gcx::M_NSNAP];
  *ngates = K;
  std::vector<int8_t> xz(2 * n);
  for (int j = 0; j < n; ++j) {
    xz[j] = (int8_t)x[j];
    xz[n + j] = (int8_t)z[j];
  }
  GC_CUDA(h, cudaMemcpyAsync(h->xz_dev, xz.data(), xz.size(), cudaMemcpyHostToDevice, h->stream));
  const int ws = h->e.batch;   // workspace slot
  GC_CUDA(h, gcx::launch_adjoint(h->e, circuit, ws, h->xz_dev, h->grad_dev, h->stream));
  int wmeta[gcx::M_COUNT];
  double wdisc = 0.0;
  GC_CUDA(h, cudaMemcpyAsync(wmeta, h->e.meta + (long long)ws * gcx::M_COUNT, sizeof wmeta, cudaMemcpyDeviceToHost,
                             h->stream));
  GC_CUDA(h, cudaMemcpyAsync(&wdisc, h->e.dstats + (long long)ws * gcx::kDStats, sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
  const int ncopy = std::min(K, (int)cap_gates);
  std::vector<double> g((size_t)std::max(ncopy, 1) * d);
  if (ncopy > 0)
    GC_CUDA(h, cudaMemcpyAsync(g.data(), h->grad_dev, (size_t)ncopy * d * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  if (wmeta[gcx::M_STATUS]) return fail(h, wmeta[gcx::M_STATUS], "adjoint pass failed (device status)");
  // the backward state carries the observable evolved back through the later gates and can need
  // more bond dimension than the forward state: if chi_max made it discard weight, the gradient is
  // not exact
  if (wdisc > 1e-16)
    return fail(h, GCAMPS_ECHI, "adjoint pass truncated (discarded weight " + std::to_string(wdisc) +
                                    "): raise chi_max");
  if (ncopy > 0) std::memcpy(grad, g.data(), (size_t)ncopy * d * sizeof(double));
  return GCAMPS_OK;
}

static int statevector_impl(gcamps_t* h, int circuit, const int32_t* ys, long long nys, double* re, double* im) {
  const int n = h->nq[circuit], d = h->e.d;
  long long dim = 1;
  for (int j = 0; j < n; ++j) {
    dim *= d;
    if (dim > (1LL << 20)) return fail(h, GCAMPS_EINVAL, "d^n above 2^20: dense readout not supported");
  }
  const long long nbuf = dim * (long long)h->e.maxdim;
  const size_t bytes = (size_t)(2 * nbuf + 3 * dim) * sizeof(double2) + (size_t)dim * (2 * sizeof(int) + n) + 256;
  void* work = nullptr;
  if (cudaMalloc(&work, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, GCAMPS_ENOMEM, "statevector workspace");
  }
  int32_t* ys_dev = nullptr;
  double2* out = nullptr;
  cudaError_t ce = cudaMalloc(&out, (size_t)nys * sizeof(double2));
  if (ce == cudaSuccess && ys) ce = cudaMalloc(&ys_dev, (size_t)nys * sizeof(int32_t));
  if (ce == cudaSuccess && ys)
    ce = cudaMemcpyAsync(ys_dev, ys, (size_t)nys * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream);
  if (ce == cudaSuccess) ce = gcx::launch_statevector(h->e, circuit, out, dim, ys_dev, nys, work, h->stream);
  std::vector<double2> host((size_t)nys);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(host.data(), out, (size_t)nys * sizeof(double2), cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  cudaFree(work);
  if (out) cudaFree(out);
  if (ys_dev) cudaFree(ys_dev);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "statevector");
  for (long long i = 0; i < nys; ++i) {
    re[i] = host[(size_t)i].x;
    im[i] = host[(size_t)i].y;
  }
  return device_status(h);
}

int gcamps_statevector(gcamps_t* h, int circuit, double* re, double* im) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  if (!re || !im) return fail(h, GCAMPS_EINVAL, "null output");
  long long dim = 1;
  for (int j = 0; j < h->nq[circuit]; ++j) {
    dim *= h->e.d;
    if (dim > (1LL << 20)) return fail(h, GCAMPS_EINVAL, "d^n above 2^20: dense readout not supported");
  }
  return statevector_impl(h, circuit, nullptr, dim, re, im);
}

int gcamps_batch_amplitude(gcamps_t* h, int circuit, const int32_t* digits, double* re, double* im) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  if (!digits || !re || !im) return fail(h, GCAMPS_EINVAL, "null argument");
  long long y = 0;
  for (int j = 0; j < h->nq[circuit]; ++j) {
    if (digits[j] < 0 || digits[j] >= h->e.d) return fail(h, GCAMPS_EINVAL, "digit out of range");
    y = y * h->e.d + digits[j];
    if (y > (1LL << 30)) return fail(h, GCAMPS_EINVAL, "d^n above 2^20: dense readout not supported");
  }
  const int32_t yy = (int32_t)y;
  return statevector_impl(h, circuit, &yy, 1, re, im);
}

int gcamps_batch_get_tableau(gcamps_t* h, int circuit, uint8_t* exps, uint8_t* phase) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  const int n = h->nq[circuit];
  const uint8_t* t = h->e.tab + (long long)circuit * h->e.tab_stride;
  if (exps) GC_CUDA(h, cudaMemcpyAsync(exps, t, 4 * n * n, cudaMemcpyDeviceToHost, h->stream));
  if (phase) GC_CUDA(h, cudaMemcpyAsync(phase, t + 4 * n * n, 2 * n, cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  return device_status(h);
}

int gcamps_get_inverse_tableau(gcamps_t* h, int circuit, uint8_t* exps, uint8_t* phase) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  const int n = h->nq[circuit];
  const uint8_t* t = h->e.tab + (long long)circuit * h->e.tab_stride + 4 * n * n + 2 * n;
  if (exps) GC_CUDA(h, cudaMemcpyAsync(exps, t, 4 * n * n, cudaMemcpyDeviceToHost, h->stream));
  if (phase) GC_CUDA(h, cudaMemcpyAsync(phase, t + 4 * n * n, 2 * n, cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  return device_status(h);
}

int gcamps_batch_get_bond_dims(gcamps_t* h, int circuit, int32_t* chi) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  if (!chi) return fail(h, GCAMPS_EINVAL, "null output");
  const int n = h->nq[circuit];
  std::vector<int> dims(n + 1);
  GC_CUDA(h, cudaMemcpyAsync(dims.data(), h->e.dims + (long long)circuit * (h->e.n + 1), (n + 1) * sizeof(int),
                             cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int j = 0; j < n - 1; ++j) chi[j] = dims[j + 1];
  return device_status(h);
}

// The single-circuit forms of the contract (circuit 0 of the handle).
int gcamps_expect_weyl(gcamps_t* h, const int32_t* x, const int32_t* z, double* re, double* im) {
  return gcamps_batch_expect_weyl(h, 0, x, z, re, im);
}
int gcamps_amplitude(gcamps_t* h, const int32_t* digits, double* re, double* im) {
  return gcamps_batch_amplitude(h, 0, digits, re, im);
}
int gcamps_get_tableau(gcamps_t* h, uint8_t* exps, uint8_t* phase) { return gcamps_batch_get_tableau(h, 0, exps, phase); }
int gcamps_get_bond_dims(gcamps_t* h, int32_t* chi) { return gcamps_batch_get_bond_dims(h, 0, chi); }

int gcamps_get_schmidt(gcamps_t* h, int circuit, int bond, double* s, int32_t* count) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  if (!s || !count || bond < 0 || bond >= h->nq[circuit] - 1) return fail(h, GCAMPS_EINVAL, "bad bond or null output");
  if (!h->schmidt_dev) GC_CUDA(h, cudaMalloc(&h->schmidt_dev, (size_t)(h->e.d * h->e.maxdim + 64) * sizeof(double)));
  GC_CUDA(h, gcx::launch_schmidt(h->e, circuit, bond, h->schmidt_dev, h->cnt_dev, h->stream));
  int cnt = 0;
  GC_CUDA(h, cudaMemcpyAsync(&cnt, h->cnt_dev, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  GC_CUDA(h, cudaMemcpy(s, h->schmidt_dev, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToHost));
  *count = cnt;
  return device_status(h);
}

int gcamps_get_site(gcamps_t* h, int circuit, int site, double* t, int64_t cap, int32_t* dims) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  const int n = h->nq[circuit];
  if (site < 0 || site >= n || !dims) return fail(h, GCAMPS_EINVAL, "bad site or null dims");
  int dd[2];
  GC_CUDA(h, cudaMemcpyAsync(dd, h->e.dims + (long long)circuit * (h->e.n + 1) + site, 2 * sizeof(int),
                             cudaMemcpyDeviceToHost, h->stream));
  const long long off = h->mps_base[circuit] + h->site_off[(size_t)circuit * (h->e.n + 1) + site];
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  dims[0] = dd[0];
  dims[1] = h->e.d;
  dims[2] = dd[1];
  const long long nel = (long long)dd[0] * h->e.d * dd[1];
  if (t) {
    if (cap < nel) return fail(h, GCAMPS_EINVAL, "site buffer too small");
    GC_CUDA(h, cudaMemcpy(t, h->e.mps + off, (size_t)nel * sizeof(double2),
                          cudaMemcpyDeviceToHost));
  }
  return device_status(h);
}

int gcamps_get_last_weyl(gcamps_t* h, int circuit, int32_t* x, int32_t* z, int32_t* r) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  const int n = h->nq[circuit];
  std::vector<int8_t> w(2 * n);
  std::vector<int> meta(gcx::M_COUNT);
  GC_CUDA(h, cudaMemcpyAsync(w.data(), h->e.weyl + (long long)circuit * 2 * h->e.n, 2 * n, cudaMemcpyDeviceToHost,
                             h->stream));
  GC_CUDA(h, cudaMemcpyAsync(meta.data(), h->e.meta + (long long)circuit * gcx::M_COUNT, gcx::M_COUNT * sizeof(int),
                             cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int j = 0; j < n; ++j) {
    if (x) x[j] = w[j];
    if (z) z[j] = w[n + j];
  }
  if (r) *r = meta[gcx::M_WEYL_R];
  return device_status(h);
}

int gcamps_get_stats(gcamps_t* h, int circuit, gcamps_stats* st) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  if (!st) return fail(h, GCAMPS_EINVAL, "null output");
  long long s[gcx::S_COUNT];
  double ds[gcx::kDStats];
  int meta[gcx::M_COUNT];
  GC_CUDA(h, cudaMemcpyAsync(s, h->e.stats + (long long)circuit * gcx::S_COUNT, sizeof s, cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaMemcpyAsync(ds, h->e.dstats + (long long)circuit * gcx::kDStats, sizeof ds, cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaMemcpyAsync(meta, h->e.meta + (long long)circuit * gcx::M_COUNT, sizeof meta, cudaMemcpyDeviceToHost,
                             h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  st->t_gates = s[gcx::S_T];
  st->clifford_gates = s[gcx::S_CLIFF];
  st->bonds_visited = s[gcx::S_BONDS];
  st->candidates_scored = s[gcx::S_CANDS];
  st->accepted = s[gcx::S_ACC];
  st->sweeps = s[gcx::S_SWEEPS];
  st->vn_evaluations = s[gcx::S_VN];
  st->svd_calls = s[gcx::S_SVD];
  st->jacobi_sweeps = s[gcx::S_JSWEEPS];
  st->jacobi_max_sweeps = s[gcx::S_JMAX];
  st->qr_calls = s[gcx::S_QR];
  st->max_chi = (int32_t)s[gcx::S_MAXCHI];
  st->status = meta[gcx::M_STATUS];
  st->discarded_weight = ds[0];
  st->scoring_flops = ds[1];
  st->screen_flops = ds[2];
  st->tensor_flops = ds[3];
  st->algorithmic_flops = ds[4];
  return device_status(h);
}

int gcamps_set_replay(gcamps_t* h, int circuit, const int32_t* pairs, int32_t count) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  if (count < 0 || count > gcx::kDecCap || (count > 0 && !pairs)) return fail(h, GCAMPS_EINVAL, "bad replay list");
  for (int k = 0; k < count; ++k)
    if (pairs[2 * k] < 0 || pairs[2 * k] > h->nq[circuit] - 2 || pairs[2 * k + 1] < 0 || pairs[2 * k + 1] >= h->e.K)
      return fail(h, GCAMPS_EINVAL, "replay pair out of range");
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  if (!h->replay_dev) {
    const size_t nb = (size_t)h->e.batch * gcx::kDecCap * 2 * sizeof(int);
    if (cudaMalloc(&h->replay_dev, nb) != cudaSuccess || cudaMalloc(&h->replay_n_dev, h->e.batch * sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, GCAMPS_ENOMEM, "replay buffers");
    }
    GC_CUDA(h, cudaMemset(h->replay_n_dev, 0, h->e.batch * sizeof(int)));
    h->e.replay = h->replay_dev;
    h->e.replay_n = h->replay_n_dev;
  }
  if (count > 0)
    GC_CUDA(h, cudaMemcpy(h->replay_dev + (size_t)circuit * gcx::kDecCap * 2, pairs, (size_t)count * 2 * sizeof(int),
                          cudaMemcpyHostToDevice));
  GC_CUDA(h, cudaMemcpy(h->replay_n_dev + circuit, &count, sizeof(int), cudaMemcpyHostToDevice));
  return GCAMPS_OK;
}

int gcamps_overlap(gcamps_t* h1, int circuit1, gcamps_t* h2, int circuit2, double* re, double* im) {
  int rc = check_circuit(h1, circuit1);
  if (rc) return rc;
  rc = check_circuit(h2, circuit2);
  if (rc) return fail(h1, rc, "second handle or circuit invalid");
  if (!re || !im) return fail(h1, GCAMPS_EINVAL, "null output");
  if (h1->nq[circuit1] != h2->nq[circuit2] || h1->e.d != h2->e.d || h1->e.maxdim != h2->e.maxdim)
    return fail(h1, GCAMPS_EINVAL, "overlap needs the same n, d and chi_max");
  GC_CUDA(h1, cudaStreamSynchronize(h2->stream));
  GC_CUDA(h1, gcx::launch_overlap(h1->e, circuit1, h2->e, circuit2, h1->out_dev, h1->stream));
  double2 v;
  GC_CUDA(h1, cudaMemcpyAsync(&v, h1->out_dev, sizeof v, cudaMemcpyDeviceToHost, h1->stream));
  GC_CUDA(h1, cudaStreamSynchronize(h1->stream));
  *re = v.x;
  *im = v.y;
  rc = device_status(h1);
  return rc ? rc : device_status(h2);
}

int gcamps_get_profile(gcamps_t* h, int circuit, int64_t* out, int32_t cap, int32_t* count) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  if (cap < 0 || (cap > 0 && !out)) return fail(h, GCAMPS_EINVAL, "bad profile buffer");
  long long p[gcx::P_COUNT];
  GC_CUDA(h, cudaMemcpyAsync(p, h->e.prof + (long long)circuit * gcx::P_COUNT, sizeof p, cudaMemcpyDeviceToHost,
                             h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int i = 0; i < cap && i < gcx::P_COUNT; ++i) out[i] = p[i];
  if (count) *count = gcx::P_COUNT;
  return device_status(h);
}

int gcamps_score_theta(gcamps_t* h, int chi_l, int chi_r, const double* theta, double* s2, double* vn,
                       int32_t* choice) {
  if (!h) return GCAMPS_EINVAL;
  const int d = h->e.d;
  if (!theta || !s2 || !vn || chi_l < 1 || chi_r < 1 || chi_l > h->e.maxdim / d || chi_r > h->e.maxdim / d)
    return fail(h, GCAMPS_EINVAL, "bad theta shape or null pointer");
  const size_t nel = (size_t)chi_l * d * d * chi_r;
  double2* th = nullptr;
  double* out = nullptr;
  cudaError_t ce = cudaMalloc(&th, nel * sizeof(double2));
  if (ce == cudaSuccess) ce = cudaMalloc(&out, (2 * gcx::kMaxK + 2) * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(th, theta, nel * sizeof(double2), cudaMemcpyHostToDevice, h->stream);
  int* ch_dev = reinterpret_cast<int*>(out + 2 * gcx::kMaxK);
  if (ce == cudaSuccess)
    ce = gcx::launch_score_theta(h->e, th, chi_l, chi_r, out, out + gcx::kMaxK, ch_dev, h->stream);
  std::vector<double> host(2 * gcx::kMaxK + 2);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(host.data(), out, host.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (th) cudaFree(th);
  if (out) cudaFree(out);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "score_theta");
  for (int k = 0; k < h->e.K; ++k) {
    s2[k] = host[k];
    vn[k] = host[gcx::kMaxK + k];
  }
  if (choice) std::memcpy(choice, &host[2 * gcx::kMaxK], 2 * sizeof(int32_t));
  return device_status(h);
}

int gcamps_estimate_theta(gcamps_t* h, int chi_l, int chi_r, const double* theta, double* est, double* bound) {
  if (!h) return GCAMPS_EINVAL;
  const int d = h->e.d;
  if (!theta || !est || !bound || chi_l < 1 || chi_r < 1 || chi_l > h->e.maxdim / d || chi_r > h->e.maxdim / d)
    return fail(h, GCAMPS_EINVAL, "bad theta shape or null pointer");
  const size_t nel = (size_t)chi_l * d * d * chi_r;
  double2* th = nullptr;
  double* out = nullptr;
  cudaError_t ce = cudaMalloc(&th, nel * sizeof(double2));
  if (ce == cudaSuccess) ce = cudaMalloc(&out, 2 * gcx::kMaxK * sizeof(double));
  if (ce == cudaSuccess) ce = cudaMemcpyAsync(th, theta, nel * sizeof(double2), cudaMemcpyHostToDevice, h->stream);
  if (ce == cudaSuccess)
    ce = gcx::launch_estimate_theta(h->e, th, chi_l, chi_r, out, out + gcx::kMaxK, h->stream);
  std::vector<double> host(2 * gcx::kMaxK);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(host.data(), out, host.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
  if (th) cudaFree(th);
  if (out) cudaFree(out);
  if (ce != cudaSuccess) return cuda_fail(h, ce, "estimate_theta");
  for (int k = 0; k < h->e.K; ++k) {
    est[k] = host[k];
    bound[k] = host[gcx::kMaxK + k];
  }
  return device_status(h);
}

int gcamps_score_theta_noalloc(int d, int chi_l, int chi_r, const double* theta_dev, double* s2_dev, double* vn_dev,
                               int32_t* choice_dev, double tie_tol, void* cuda_stream) {
  if ((d != 2 && d != 3) || !theta_dev || !s2_dev || !vn_dev || !choice_dev || chi_l < 1 || chi_r < 1 ||
      !(tie_tol >= 0.0))
    return GCAMPS_EINVAL;
  // chi d <= the limit, compared without forming chi d (which could wrap for chi near INT_MAX)
  if (chi_l > GCAMPS_NOALLOC_MAX_SIDE / d || chi_r > GCAMPS_NOALLOC_MAX_SIDE / d) return GCAMPS_ESIZE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return GCAMPS_ECUDA;
  if (dev < 0 || dev >= gcx::kStaticMaxDevices) return GCAMPS_ECUDA;
  {
    // Once per device, with that device current: the device addresses of the library's static
    // arrays and the class tables of d = 2 and 3.
    static std::mutex mu;
    static bool ready[gcx::kStaticMaxDevices] = {};
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[dev]) {
      const Tables& t2 = tables(2);
      const Tables& t3 = tables(3);
      if (t2.u.size() != (size_t)gcx::kStaticK2 * 16 * 2 || t3.u.size() != (size_t)gcx::kStaticK3 * 81 * 2 ||
          t2.img.size() != (size_t)gcx::kStaticK2 * 20 || t3.img.size() != (size_t)gcx::kStaticK3 * 20)
        return GCAMPS_EINVAL;
      if (gcx::static_setup(dev, t2.u.data(), t2.img.data(), t3.u.data(), t3.img.data()) != cudaSuccess)
        return GCAMPS_ECUDA;
      ready[dev] = true;
    }
  }
  const cudaError_t ce = gcx::launch_score_theta_static(dev, d, tie_tol, reinterpret_cast<const double2*>(theta_dev),
                                                        chi_l, chi_r, s2_dev, vn_dev, choice_dev,
                                                        static_cast<cudaStream_t>(cuda_stream));
  return ce == cudaSuccess ? GCAMPS_OK : GCAMPS_ECUDA;
}

int gcamps_get_last_theta(gcamps_t* h, int circuit, double* theta, int32_t* shape) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  std::vector<double> buf(3 * gcx::kMaxK + 2 + 2 * gcx::kSmall);
  GC_CUDA(h, cudaMemcpyAsync(buf.data(), h->e.lastsc + (long long)circuit * buf.size(), buf.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  const int cl = (int)buf[3 * gcx::kMaxK], cr = (int)buf[3 * gcx::kMaxK + 1], d = h->e.d;
  if (shape) {
    shape[0] = cl;
    shape[1] = cr;
  }
  const long long nel = (long long)cl * d * d * cr;
  if (theta && nel <= gcx::kSmall) std::memcpy(theta, &buf[3 * gcx::kMaxK + 2], (size_t)nel * 2 * sizeof(double));
  return device_status(h);
}

int gcamps_get_last_scores(gcamps_t* h, int circuit, double* s2, double* vn, uint8_t* evaluated) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  std::vector<double> buf(3 * gcx::kMaxK + 2 + 2 * gcx::kSmall);
  GC_CUDA(h, cudaMemcpyAsync(buf.data(), h->e.lastsc + (long long)circuit * buf.size(), buf.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < h->e.K; ++k) {
    if (s2) s2[k] = buf[k];
    if (vn) vn[k] = buf[gcx::kMaxK + k];
    if (evaluated) evaluated[k] = (uint8_t)(buf[2 * gcx::kMaxK + k] != 0.0);
  }
  return device_status(h);
}

int gcamps_get_decisions(gcamps_t* h, int circuit, int32_t* pairs, int32_t cap, int32_t* count) {
  int rc = check_circuit(h, circuit);
  if (rc) return rc;
  if (!count || cap < 0 || (cap > 0 && !pairs)) return fail(h, GCAMPS_EINVAL, "bad output");
  int meta[gcx::M_COUNT];
  GC_CUDA(h, cudaMemcpyAsync(meta, h->e.meta + (long long)circuit * gcx::M_COUNT, sizeof meta, cudaMemcpyDeviceToHost,
                             h->stream));
  GC_CUDA(h, cudaStreamSynchronize(h->stream));
  const int nd = meta[gcx::M_NDEC];
  *count = nd;
  const int ncopy = std::min(std::min(nd, (int)cap), gcx::kDecCap);
  if (ncopy > 0)
    GC_CUDA(h, cudaMemcpy(pairs, h->e.dec + (long long)circuit * gcx::kDecCap * 2, (size_t)ncopy * 2 * sizeof(int),
                          cudaMemcpyDeviceToHost));
  return device_status(h);
}

}  // extern "C"
