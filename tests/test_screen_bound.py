"""The FP32 Renyi-2 screen's error bound (the engine keeps S2_fp32 - margin as a lower bound of
S2 <= S_vN, which is what makes its class pruning exact).  The bound, retyped here from its derivation:
theta' = Q theta and its Gram in FP32 satisfy |G^ - G|_F <= eta tr G with
eta = 2 e1 + e1^2 + (2M + 4) u (1 + e1)^2, e1 = d (d^2 + 6) u, u = 2^-24 (M the longer side of theta'),
hence |S2^ - S2| <= 2 eta sqrt(m) + 2 eta.  Checked against FP32 computations (numpy complex64:
another summation order than the GPU's, which the bound does not depend on) of every class on random,
rank-deficient and spiky tensors, with the exact FP64 value as reference.  The engine uses the bound
only for 1e-12 < tr G < 1e12; far outside that range FP32 squares of the Gram entries underflow and the
bound fails, which the last test shows (the engine then evaluates every class exactly)."""
import numpy as np
import pytest

from oracle import clifford

U = 2.0 ** -24


def _bound(d, rows, cols):
    m, M = min(rows, cols), max(rows, cols)
    e1 = d * (d * d + 6) * U
    eta = 2 * e1 + e1 * e1 + (2 * M + 4) * U * (1 + e1) ** 2
    return 2 * eta * np.sqrt(m) + 2 * eta


def _s2(x):
    g = x @ x.conj().T if x.shape[0] <= x.shape[1] else x.conj().T @ x
    tr = np.trace(g).real
    return -np.log(np.sum(np.abs(g) ** 2) / tr ** 2)


def _thetas(rng, d, cl, cr):
    shape = (cl * d, d * cr)
    yield rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    r = max(1, min(shape) // 3)
    a = rng.standard_normal((shape[0], r)) + 1j * rng.standard_normal((shape[0], r))
    yield a @ (rng.standard_normal((r, shape[1])) + 1j * rng.standard_normal((r, shape[1])))
    spiky = rng.standard_normal(shape) * 1e-6 + 0j
    spiky[0, 0] = 1.0
    yield spiky
    yield (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * 1e-5   # tr ~ 1e-10 * size


@pytest.mark.parametrize("d,cl,cr", [(2, 4, 8), (3, 3, 3), (3, 9, 27), (3, 27, 27)])
def test_fp32_screen_error_stays_inside_the_bound(d, cl, cr):
    rng = np.random.default_rng(100 * d + cl + cr)
    cands = clifford.candidates(d)
    bound = _bound(d, cl * d, d * cr)
    worst = 0.0
    for th in _thetas(rng, d, cl, cr):
        t = th.reshape(cl, d * d, cr)
        t32 = t.astype(np.complex64)
        for _s, _i, q in cands[:: max(1, len(cands) // 12)]:
            exact = _s2(np.einsum("uv,avb->aub", q, t).reshape(cl * d, d * cr))
            x32 = np.einsum("uv,avb->aub", q.astype(np.complex64), t32).reshape(cl * d, d * cr)
            approx = float(_s2(x32.astype(np.complex64)))
            worst = max(worst, abs(approx - exact) / bound)
    assert worst <= 1.0
    assert worst > 0.0


def test_bound_fails_far_below_the_guarded_range():
    d, cl, cr = 3, 9, 27
    rng = np.random.default_rng(7)
    th = (rng.standard_normal((cl * d, d * cr)) + 1j * rng.standard_normal((cl * d, d * cr))) * 1e-12
    assert np.sum(np.abs(th) ** 2) < 1e-12                     # outside the guarded range
    exact = _s2(th)
    approx = float(_s2(th.astype(np.complex64)))
    assert abs(approx - exact) > _bound(d, cl * d, d * cr)
