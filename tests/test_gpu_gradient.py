"""Adjoint phase gradient of the library (gcamps_expect_gradient, the differentiation form) against the
oracle's dense gradient, against central differences of the library's own forward runs, and through
the torch.autograd binding (weyl_expectation).  Truncation is inactive in every case (the gradient is
exact there), with disentangling on (so the backward pass undoes real disentanglers)."""
import math

import numpy as np
import pytest

from oracle import statevector as sv
from oracle.weyl import Weyl
from synth import Diag, param_phase_circuit

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


def _sim(G, n, d, chi=81, gates=64):
    return G.Simulator(n, d, chi_max=chi, cutoff=1e-14, snapshot_entries=1 << 22, snapshot_max_gates=gates)


def _run(G, sim, gates, d):
    sim.reset()
    sim.run(G.ops_from_gates(gates, d))
    sim.sync()


def _obs(n, sites_z):
    x = np.zeros(n, dtype=np.int32)
    z = np.zeros(n, dtype=np.int32)
    for s_ in sites_z:
        z[s_] = 1
    return x, z


@pytest.mark.parametrize("d,n,layers,ngates,seed", [(3, 5, 6, 8, 1), (2, 6, 6, 8, 2), (3, 6, 8, 10, 3)])
def test_gradient_matches_dense_oracle(G, d, n, layers, ngates, seed):
    gates, _ = param_phase_circuit(n, d, layers, ngates, seed)
    x, z = _obs(n, [0, n - 1])
    sim = _sim(G, n, d)
    _run(G, sim, gates, d)
    assert sum(1 for _b, k in sim.decisions() if k) > 0      # disentanglers were applied
    val, grad = sim.expect_gradient(x, z)
    rval, rgrad = sv.observable_and_phase_gradient(gates, n, d, Weyl(0, x, z, d))
    assert abs(val - rval) < 1e-10
    assert grad.shape == (ngates, d)
    assert np.max(np.abs(grad - np.array(rgrad))) < 1e-9
    sim.close()


def test_gradient_n12_matches_dense_oracle_and_central_differences(G):
    """n = 12 qutrits with chi_max = 729 (the full Schmidt bound, so neither pass truncates)."""
    d, n = 3, 12
    gates, _ = param_phase_circuit(n, d, 10, 16, 5)
    x, z = _obs(n, [0, 6])
    sim = _sim(G, n, d, chi=729)
    _run(G, sim, gates, d)
    val, grad = sim.expect_gradient(x, z)
    rval, rgrad = sv.observable_and_phase_gradient(gates, n, d, Weyl(0, x, z, d))
    assert abs(val - rval) < 1e-10
    assert np.max(np.abs(grad - np.array(rgrad))) < 1e-9
    diag = [i for i, g in enumerate(gates) if not hasattr(g, "sp_index")]
    h = 1e-4
    for k, j in ((0, 1), (15, 2)):
        vals = []
        for sgn in (1, -1):
            gl = list(gates)
            g = gl[diag[k]]
            ph = list(g.phases)
            ph[j] += sgn * h
            gl[diag[k]] = Diag(g.site, tuple(ph), g.param)
            _run(G, sim, gl, d)
            vals.append(sim.expect_gradient(x, z)[0])
        assert abs(grad[k, j] - (vals[0] - vals[1]) / (2 * h)) < 1e-6
    sim.close()


def test_truncated_backward_pass_is_reported(G):
    """With chi_max too small for the backward state the call fails (GCAMPS_ECHI) instead of returning
    an inexact gradient; a gradient it does return is exact."""
    d, n = 3, 12
    gates, _ = param_phase_circuit(n, d, 10, 16, 5)
    x, z = _obs(n, [0, 6])
    sim = _sim(G, n, d, chi=9)
    _run(G, sim, gates, d)
    try:
        _val, grad = sim.expect_gradient(x, z)
    except G.GcampsError as ex:
        assert ex.code == 5            # GCAMPS_ECHI
    else:                              # accepted: then it is exact (if the forward kept everything)
        if sim.stats()["discarded_weight"] < 1e-20:
            rgrad = sv.observable_and_phase_gradient(gates, n, d, Weyl(0, x, z, d))[1]
            assert np.max(np.abs(grad - np.array(rgrad))) < 1e-9
    sim.close()


def test_autograd_binding_and_theta_chain_rule(G):
    import torch
    d, n = 3, 6
    gates, th = param_phase_circuit(n, d, 6, 6, 9)
    x, z = _obs(n, [1, 4])
    sim = _sim(G, n, d)
    theta = torch.tensor(th, dtype=torch.float64, requires_grad=True)
    zero = torch.zeros_like(theta)
    phases = torch.stack([zero, theta, -theta], dim=1)
    val = G.weyl_expectation(phases, sim, gates, x, z)
    val.backward()
    rval, rgrad = sv.observable_and_phase_gradient(gates, n, d, Weyl(0, x, z, d))
    assert abs(val.item() - rval) < 1e-10
    want = np.array([g[1] - g[2] for g in rgrad])
    assert np.max(np.abs(theta.grad.numpy() - want)) < 1e-9
    # theta = 2 pi / 9 everywhere is the benchmark T3 circuit
    t3 = torch.full((len(th),), 2 * math.pi / 9, dtype=torch.float64)
    v3 = G.weyl_expectation(torch.stack([torch.zeros_like(t3), t3, -t3], dim=1), sim, gates, x, z)
    gl = [Diag(g.site, (0.0, 2 * math.pi / 9, -2 * math.pi / 9), g.param) if not hasattr(g, "sp_index") else g
          for g in gates]
    assert abs(v3.item() - sv.observable_and_phase_gradient(gl, n, d, Weyl(0, x, z, d))[0]) < 1e-10
    sim.close()


def test_gradient_requires_snapshots_and_reports_a_full_arena(G):
    d, n = 3, 5
    gates, _ = param_phase_circuit(n, d, 5, 6, 4)
    x, z = _obs(n, [0])
    plain = G.Simulator(n, d, chi_max=27)
    _run(G, plain, gates, d)
    with pytest.raises(G.GcampsError):
        plain.expect_gradient(x, z)
    plain.close()
    small = G.Simulator(n, d, chi_max=27, cutoff=1e-14, snapshot_entries=1 << 16, snapshot_max_gates=3)
    small.reset()
    small.run(G.ops_from_gates(gates, d))
    with pytest.raises(G.GcampsError) as ei:
        small.sync()
    assert ei.value.code == 7      # GCAMPS_ESNAP: more gates than snapshot_max_gates
    small.close()
