"""gcamps_score_theta_noalloc: the disentangler scoring for callers that cannot allocate device memory.

Some callers may not call cudaMalloc: their GPU memory belongs to another allocator (a framework's
pool that has reserved the device) or they cannot take the device-wide synchronisation an
allocation may cause.  This entry point works in a fixed static device array of the library
instead.  The test checks its outputs against gcamps_score_theta (the handle-based entry point)
on the same tensors, two calls in a row, so that contents left in the shared array by the first
call cannot leak into the second.  It sits in a file of its own, collected last, and passes both
alone in a fresh process and after the other GPU tests.
"""
import numpy as np
import pytest

from oracle.gcamps import GCAMPS

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_06672_gb300.build import build_library
    build_library()
    import paper_2511_06672_gb300 as G
    return G


def _theta(rng, cl, d, cr, rank=None):
    """Seeded random normalised two-site tensor; `rank` < full makes the Gram rank-deficient."""
    shape = (cl * d, d * cr)
    if rank is None:
        m = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    else:
        a = rng.standard_normal((shape[0], rank)) + 1j * rng.standard_normal((shape[0], rank))
        b = rng.standard_normal((rank, shape[1])) + 1j * rng.standard_normal((rank, shape[1]))
        m = a @ b
    m /= np.linalg.norm(m)
    return m.reshape(cl, d, d, cr)


def _noalloc(G, torch, theta, d, stream):
    cl, cr = theta.shape[0], theta.shape[3]
    K = G.num_candidates(d)
    dev = torch.device("cuda", 0)
    th = torch.from_numpy(np.ascontiguousarray(theta)).to(dev)
    s2 = torch.full((K,), float("nan"), dtype=torch.float64, device=dev)
    vn = torch.full((K,), float("nan"), dtype=torch.float64, device=dev)
    ch = torch.full((3,), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    G.score_theta_noalloc(d, cl, cr, th, s2, vn, ch, tie_tol=1e-10, stream=stream)
    stream.synchronize()
    return s2.cpu().numpy(), vn.cpu().numpy(), ch.cpu().numpy()


# (d, chi_l, chi_r): warp-level classes (Gram <= 27 x 27), a CTA-level one with the Renyi-2 pruning
# (27 x 81), and the largest accepted shape for each d.
CASES = [(3, 3, 3), (3, 9, 27), (3, 27, 27), (2, 4, 8), (2, 40, 40)]


@pytest.mark.parametrize("d,cl,cr", CASES)
def test_noalloc_matches_handle_scoring_twice(G, d, cl, cr):
    import torch
    rng = np.random.default_rng(1000 * d + 10 * cl + cr)
    # Same cluster size as the static variant (4 CTAs), so that the pruning evaluates the same classes;
    # this handle's scoring accepts chi up to 64 (d = 2) / 81 (d = 3).
    sim = G.Simulator(12, d, chi_max=81, cluster_size=4)
    stream = torch.cuda.Stream(device=0)
    try:
        # Two different tensors in a row: the second call runs on the array the first one left.
        for theta in (_theta(rng, cl, d, cr), _theta(rng, cl, d, cr, rank=max(1, min(cl, cr) // 2))):
            s2_ref, vn_ref, choice_ref, nev_ref = sim.score_theta(theta)
            s2, vn, ch = _noalloc(G, torch, theta, d, stream)
            assert np.all(np.isfinite(s2)) and np.all(np.isfinite(vn))
            assert np.max(np.abs(s2 - s2_ref)) <= TOL
            assert np.max(np.abs(vn - vn_ref)) <= TOL
            assert int(ch[0]) == choice_ref and int(ch[1]) == nev_ref
            assert int(ch[2]) == 0
            # and directly against the oracle's SVD entropies of every class
            vn_oracle = GCAMPS(2, d, chi_max=81).score_bond(theta)
            assert np.max(np.abs(vn - vn_oracle)) <= TOL
    finally:
        sim.close()


def test_noalloc_rejects_shapes_above_the_static_limit(G):
    import torch
    from paper_2511_06672_gb300 import _native as N
    dev = torch.device("cuda", 0)
    th = torch.zeros(4, dtype=torch.complex128, device=dev)
    out = torch.zeros(90, dtype=torch.float64, device=dev)
    ch = torch.zeros(3, dtype=torch.int32, device=dev)
    for d, cl, cr in [(3, 28, 3), (3, 3, 28), (2, 41, 1), (3, 715827883, 1)]:
        with pytest.raises(G.GcampsError) as ei:
            G.score_theta_noalloc(d, cl, cr, th, out, out, ch)
        assert ei.value.code == N.ESIZE
    with pytest.raises(G.GcampsError) as ei:
        G.score_theta_noalloc(5, 1, 1, th, out, out, ch)
    assert ei.value.code == N.EINVAL
