"""The FP32 von Neumann estimates the disentangler prunes with (gcamps_estimate_theta) against the oracle's
FP64 SVD entropies of every class: |estimate - S_vN| <= bound for every class, on random, rank-deficient,
spiky and geometrically decaying two-site tensors of the CTA-level sizes where the engine uses them
(28 <= m <= 81 for qutrits, the big bonds of the n = 32 benchmark circuits), and the bound small enough
there to prune (a few tenths of a nat at most).  The decision the pruned search takes is checked against
the oracle's by the scoring and full-circuit parity tests."""
import numpy as np
import pytest

from oracle.gcamps import GCAMPS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import paper_2511_06672_gb300 as G
    return G


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
    yield (qa * np.exp(-np.arange(m) / 6.0)) @ qb.conj().T


@pytest.mark.parametrize("d,cl,cr", [(3, 27, 27), (3, 10, 27), (3, 27, 12), (3, 27, 81), (2, 16, 20)])
def test_estimates_stay_inside_their_bound(G, d, cl, cr):
    rng = np.random.default_rng(7000 + 100 * d + cl + cr)
    sim = G.Simulator(12, d, chi_max=81, cluster_size=8)
    ref = GCAMPS(2, d, chi_max=81)
    worst = 0.0
    try:
        for th in _thetas(rng, d, cl, cr):
            th = (th / np.linalg.norm(th)).reshape(cl, d, d, cr)
            est, bd = sim.estimate_theta(th)
            exact = ref.score_bond(th)
            m = min(cl * d, d * cr)
            assert np.all(bd < 0.5), (m, bd.max())
            err = np.abs(est - exact)
            assert np.all(err <= bd), (m, float(np.max(err / bd)))
            worst = max(worst, float(np.max(err / bd)))
    finally:
        sim.close()
    assert worst < 1.0
