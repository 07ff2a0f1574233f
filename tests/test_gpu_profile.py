"""Phase timers of the engine (gcamps_get_profile), a measurement aid with no counterpart in the paper.

* Every word is non-negative; the bucket visit counts add up to the bond visits of the statistics, and their
  exact evaluations to the exact von Neumann evaluations.
* The phase cycles recorded inside the visits of a size bucket add up to no more than that bucket's visit
  cycles and to most of them (the laps tile each visit but for a few instructions between them).
* The layout the header states (GCAMPS_PROF_WORDS words) is the one the binding reads.
"""
import ctypes as C

import numpy as np
import pytest

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


@pytest.mark.parametrize("d,n,layers,t,seed", [(3, 8, 10, 10, 2), (2, 12, 14, 14, 5)])
def test_profile_buckets_tile_the_visits(G, d, n, layers, t, seed):
    gates = brickwork_circuit(n, d, layers, t, seed)
    sim = G.Simulator(n, d, chi_max=d ** (n // 2), cutoff=1e-14)
    sim.run(G.ops_from_gates(gates, d))
    sim.sync()
    st = sim.stats()
    prof = sim.profile()
    raw = np.zeros(G._native.PROF_WORDS, dtype=np.int64)
    cnt = C.c_int32()
    lib = G._native.load()
    assert lib.gcamps_get_profile(sim._h, 0, raw.ctypes.data_as(C.POINTER(C.c_int64)), len(raw), C.byref(cnt)) == 0
    assert cnt.value == G._native.PROF_WORDS
    assert (raw >= 0).all()
    assert raw[-1] == 0   # no visit in progress once the launch has ended
    buckets = prof["buckets"].values()
    assert sum(b["visits"] for b in buckets) == st["bonds_visited"]
    assert sum(b["exact"] for b in buckets) <= st["vn_evaluations"]
    for b in buckets:
        inside = sum(b["phases"].values())
        assert inside <= b["cycles"]
        if b["visits"]:
            assert inside >= 0.8 * b["cycles"]
            assert b["phases"]["clifford"] == 0 and b["phases"]["mpo"] == 0
    lead = prof["leader_warp_exact"]
    assert lead["count"] >= 0 and (lead["count"] == 0) == (lead["cycles"] == 0)
