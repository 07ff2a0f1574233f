"""Replay of recorded disentangler decisions and the MPS overlap between two handles (gcamps_set_replay,
gcamps_overlap), the GPU side of the oracle's replay mode: two runs of one circuit compared state to state.

* A run that replays another run's decisions reproduces its decisions and tableau bit for bit, and the two
  MPS overlap to 1 within 1e-12 (fidelity |<M1|M2>|^2 with equal tableaux).
* The overlap agrees with the dense state vectors: |<M1|M2>|^2 equals |<psi1|psi2>|^2 of the two dense states.
* The precision form replaying the FP64 run's decisions gives the same tableau, and its state has fidelity
  error below 1e-10 (its FP32 contractions feed only the scores; the MPS updates stay FP64).
* A replay list that does not match the visits invalidates the circuit (GCAMPS_EINVAL), with no fault.
"""
import numpy as np
import pytest

from oracle import statevector as sv
from synth import brickwork_circuit

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


def _run(G, gates, n, d, precision=0, replay=None):
    sim = G.Simulator(n, d, chi_max=d ** (n // 2), cutoff=1e-14, precision=precision)
    if replay is not None:
        sim.set_replay(replay)
    sim.run(G.ops_from_gates(gates, d))
    sim.sync()
    return sim


@pytest.mark.parametrize("d,n,layers,t,seed", [(3, 8, 8, 8, 1), (2, 10, 12, 12, 3)])
def test_replay_reproduces_a_run_and_overlap_is_one(G, d, n, layers, t, seed):
    gates = brickwork_circuit(n, d, layers, t, seed)
    a = _run(G, gates, n, d)
    dec = a.decisions()
    assert any(k != 0 for _, k in dec)
    b = _run(G, gates, n, d, replay=dec)
    c = _run(G, gates, n, d, precision=1, replay=dec)
    try:
        for other in (b, c):
            assert other.decisions() == dec
            ea, pa = a.tableau()
            eb, pb = other.tableau()
            assert np.array_equal(ea, eb) and np.array_equal(pa, pb)
        ov = a.overlap(b)
        assert abs(abs(ov) ** 2 - 1.0) < 1e-12
        assert abs(abs(a.overlap(c)) ** 2 - 1.0) < 1e-10
        # the overlap of the MPS equals the dense states' overlap (same Clifford frame)
        pa_, pb_ = a.statevector(), b.statevector()
        dense = abs(np.vdot(pa_, pb_)) ** 2 / (np.vdot(pa_, pa_).real * np.vdot(pb_, pb_).real)
        assert abs(abs(ov) ** 2 - dense) < 1e-10
        err, _ = sv.same_up_to_phase(pa_, sv.run(gates, n, d))
        assert err < 1e-10
    finally:
        for s in (a, b, c):
            s.close()


def test_replay_that_does_not_match_invalidates_the_circuit(G):
    from paper_2511_06672_gb300 import _native as N
    d, n = 3, 6
    gates = brickwork_circuit(n, d, 6, 6, 2)
    sim = G.Simulator(n, d, chi_max=27, cutoff=1e-14)
    try:
        sim.set_replay([(0, 0)])   # one pair where the run visits many bonds
        sim.run(G.ops_from_gates(gates, d))
        with pytest.raises(G.GcampsError) as ei:
            sim.sync()
        assert ei.value.code == N.EINVAL
        sim.set_replay([])
        sim.reset()
        sim.run(G.ops_from_gates(gates, d))
        sim.sync()
    finally:
        sim.close()
