"""Pins for the oracle's phase gradient (oracle/statevector.py: observable_and_phase_gradient),
the reference for the differentiation form: parametrised diagonal gates diag(1, e^{i th}, e^{-i th})
whose phases are the parameters (Sec. 2.3.2 writes the T gate through R_Z(theta)).

Pinned against central finite differences of the dense expectation (an independent computation:
only forward simulation), the chain rule for th (d/dth = d/dphi_1 - d/dphi_2), the T3 special case
th = 2 pi / 9 (same state as the benchmark T gate), and the Hermiticity of the observable."""
import math

import numpy as np
import pytest

from oracle import statevector as sv
from oracle.weyl import Weyl
from synth import Diag, param_phase_circuit, t_gate_phases


def _expect(gates, n, d, w):
    psi = sv.run(gates, n, d)
    return float(np.vdot(psi, sv.apply_weyl(psi, w, n, d)).real)


def _shift(gates, k, j, h):
    out = list(gates)
    g = out[k]
    ph = list(g.phases)
    ph[j] += h
    out[k] = Diag(g.site, tuple(ph), g.param)
    return out


@pytest.mark.parametrize("d,n,seed", [(3, 4, 1), (2, 5, 2), (3, 5, 3)])
def test_gradient_matches_central_differences(d, n, seed):
    gates, _ = param_phase_circuit(n, d, 4, 5, seed)
    x = np.zeros(n, dtype=np.int64)
    z = np.zeros(n, dtype=np.int64)
    z[0], z[n - 1] = 1, 1
    w = Weyl(0, x, z, d)
    val, grads = sv.observable_and_phase_gradient(gates, n, d, w)
    assert abs(val - _expect(gates, n, d, w)) < 1e-13
    diag_idx = [i for i, g in enumerate(gates) if not hasattr(g, "sp_index")]
    assert len(grads) == len(diag_idx) == 5
    h = 1e-5
    for gk, i in zip(grads, diag_idx):
        for j in range(d):
            fd = (_expect(_shift(gates, i, j, h), n, d, w) - _expect(_shift(gates, i, j, -h), n, d, w)) / (2 * h)
            assert abs(gk[j] - fd) < 1e-8
        assert abs(np.sum(gk)) < 1e-12      # a common phase of the gate changes nothing


def test_theta_chain_rule_and_t3_point():
    d, n = 3, 4
    gates, th = param_phase_circuit(n, d, 3, 3, 7)
    w = Weyl(0, [1, 0, 0, 0], [0, 0, 2, 0], d)
    _val, grads = sv.observable_and_phase_gradient(gates, n, d, w)
    i0 = next(i for i, g in enumerate(gates) if not hasattr(g, "sp_index"))
    dth = grads[0][1] - grads[0][2]
    h = 1e-5
    g = gates[i0]
    plus = list(gates)
    minus = list(gates)
    plus[i0] = Diag(g.site, (0.0, th[0] + h, -(th[0] + h)), g.param)
    minus[i0] = Diag(g.site, (0.0, th[0] - h, -(th[0] - h)), g.param)
    assert abs(dth - (_expect(plus, n, d, w) - _expect(minus, n, d, w)) / (2 * h)) < 1e-8
    # th = 2 pi / 9 is the benchmark T3 gate
    t3 = [Diag(g.site, t_gate_phases(3), g.param) if not hasattr(g, "sp_index") else g for g in gates]
    pt = [Diag(g.site, (0.0, 2 * math.pi / 9, -2 * math.pi / 9), g.param) if not hasattr(g, "sp_index") else g
          for g in gates]
    assert np.allclose(sv.run(t3, n, d), sv.run(pt, n, d), atol=1e-14)


def test_observable_is_real_part():
    d, n = 3, 3
    gates, _ = param_phase_circuit(n, d, 3, 2, 11)
    w = Weyl(0, [0, 1, 0], [1, 0, 0], d)
    psi = sv.run(gates, n, d)
    val, _ = sv.observable_and_phase_gradient(gates, n, d, w)
    assert abs(val - np.vdot(psi, sv.apply_weyl(psi, w, n, d)).real) < 1e-14
