"""Error bound of the FP32 von Neumann estimate the disentangler prunes with at big bonds.

With the Renyi-2 lower bound alone, about 37 of 90 classes still needed an exact (FP64) entropy at
81 x 81 Grams, because S_vN - S2 is large there.  The engine estimates S_vN itself in FP32 with an error
bound dv and evaluates exactly only the identity and the classes with  S^_k - dv <= min_j (S^_j + dv) +
tie_tol.  This file pins that bound (the same formula as the library's vn_est_bound) on the CPU; the GPU
estimates are checked against it in test_gpu_estimate.py:

* theta' = Q theta and its Gram in FP32: |G^ - G|_F <= eta tr G with eta as for the Renyi-2 screen,
  eta = 2 e1 + e1^2 + (2M + 4) u (1 + e1)^2, e1 = d (d^2 + 6) u, u = 2^-24;
* scaling G^ to unit trace before the reduction (which keeps every square inside FP32's range) adds
  one rounding per entry, at most u tr G in Frobenius norm;
* an FP32 Hermitian eigensolver is backward stable: its eigenvalues are those of G^ + E, with
  |E|_F <= 2 m^2 u |G^|_F for a Householder reduction (m - 2 reflectors applied on both sides, each
  within about m u of the matrix norm), and |G^|_F <= (1 + eta) tr G; a bisection finish adds at most
  9 u tr G per eigenvalue;
* Hoffman-Wielandt and Cauchy-Schwarz: sum_i |lambda^_i - lambda_i| <= sqrt(m) |G^ + E - G|_F, so
  the l1 distance of the spectra is at most D = (sqrt(m) (eta + u + 2 m^2 u (1 + eta)) + 9 m u) tr G;
* normalising by the estimated trace (and clipping negative estimates) at most doubles the l1
  distance of the normalised spectra, so their trace distance is T <= D / tr G;
* Fannes-Audenaert: |S^ - S| <= T ln(m - 1) + H2(T); the bound used is twice that with ln m
  (dv = 2 (T ln m + H2(T)), T <= 1/2), which leaves room for the rounding of S^ itself.

The checks use numpy complex64 (another summation order than a GPU kernel's, which the bound does not
depend on) on random, rank-deficient, spiky and geometrically decaying tensors, with the FP64 SVD
entropy as reference, and check that the pruning rule keeps every exact minimiser.
"""
import numpy as np
import pytest

from oracle import clifford
from oracle.gcamps import entropy_from_singular_values

U = 2.0 ** -24
TIE = 1e-10


def _h2(t):
    return 0.0 if t <= 0 else float(-t * np.log(t) - (1 - t) * np.log(1 - t))


def _dv(d, rows, cols):
    m, M = min(rows, cols), max(rows, cols)
    e1 = d * (d * d + 6) * U
    eta = 2 * e1 + e1 * e1 + (2 * M + 4) * U * (1 + e1) ** 2
    t = np.sqrt(m) * (eta + U + 2 * m * m * U * (1 + eta)) + 9 * m * U
    assert t <= 0.5
    return 2 * (t * np.log(m) + _h2(t))


def _fp32_entropy(x):
    x32 = x.astype(np.complex64)
    g = x32 @ x32.conj().T if x.shape[0] <= x.shape[1] else x32.conj().T @ x32
    g = (g * np.float32(1.0 / np.trace(g).real)).astype(np.complex64)
    lam = np.clip(np.linalg.eigvalsh(g).astype(np.float64), 0.0, None)
    p = lam / lam.sum()
    p = p[p > 0]
    return float(-np.sum(p * np.log(p)))


def _thetas(rng, d, cl, cr):
    shape = (cl * d, d * cr)
    yield rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    r = max(1, min(shape) // 3)
    a = rng.standard_normal((shape[0], r)) + 1j * rng.standard_normal((shape[0], r))
    yield a @ (rng.standard_normal((r, shape[1])) + 1j * rng.standard_normal((r, shape[1])))
    spiky = rng.standard_normal(shape) * 1e-6 + 0j
    spiky[0, 0] = 1.0
    yield spiky
    m = min(shape)
    qa, _ = np.linalg.qr(rng.standard_normal((shape[0], m)) + 1j * rng.standard_normal((shape[0], m)))
    qb, _ = np.linalg.qr(rng.standard_normal((shape[1], m)) + 1j * rng.standard_normal((shape[1], m)))
    yield (qa * np.exp(-np.arange(m) / 6.0)) @ qb.conj().T        # Schmidt values decaying like an MPS bond


@pytest.mark.parametrize("d,cl,cr", [(2, 8, 16), (3, 9, 9), (3, 27, 27), (3, 27, 9)])
def test_fp32_entropy_estimate_stays_inside_the_bound(d, cl, cr):
    rng = np.random.default_rng(500 + 100 * d + cl + cr)
    cands = clifford.candidates(d)
    rows, cols = cl * d, d * cr
    dv = _dv(d, rows, cols)
    worst = 0.0
    for th in _thetas(rng, d, cl, cr):
        t = th.reshape(cl, d * d, cr)
        exact, est = [], []
        for _s, _i, q in cands:
            x = np.einsum("uv,avb->aub", q, t).reshape(rows, cols)
            exact.append(entropy_from_singular_values(np.linalg.svd(x, compute_uv=False)))
            est.append(_fp32_entropy(x))
        exact, est = np.array(exact), np.array(est)
        worst = max(worst, float(np.max(np.abs(est - exact))) / dv)
        # pruning with the bound keeps every class within tie_tol of the exact minimum
        keep = est - dv <= np.min(est + dv) + TIE
        assert np.all(keep[exact <= exact.min() + TIE])
    assert 0.0 < worst <= 1.0


def test_bound_size_at_the_largest_benchmark_bond():
    """At m = 81 (qutrits, theta 81 x 81) the bound is about 0.15 nats: much tighter than the Renyi-2
    bound's gap S_vN - S2 at such bonds (median 0.70 nats), which is what makes the estimate worth a
    kernel.  At m = 28 it is about a hundredth of a nat."""
    assert 0.1 < _dv(3, 81, 81) < 0.2
    assert 0.005 < _dv(3, 28, 28) < 0.02
