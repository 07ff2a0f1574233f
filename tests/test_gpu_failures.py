"""Failure paths of the library, exercised without faulting anything.

* An iteration cap that runs out: gcamps_set_jacobi_cap(1) makes the first Jacobi SVD that needs a second
  sweep give up; the engine records GCAMPS_ENOCONV in the circuit's status, stops the circuit's MPS work,
  and the next synchronising call returns it.  After gcamps_reset (and the default cap) the same handle
  runs the circuit again and matches the oracle.
* A device allocation that fails: a handle whose reservation exceeds the GPU's memory (n = 128 qutrits at
  chi_max = 5000, over a terabyte) is refused with GCAMPS_ENOMEM, and the device memory in use is the same
  before and after (nothing leaked).
"""
import numpy as np
import pytest

from oracle.gcamps import GCAMPS
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


def test_jacobi_cap_reports_enoconv_and_the_handle_recovers(G):
    from paper_2511_06672_gb300 import _native as N
    d, n, layers, t, seed = 3, 6, 6, 6, 3
    gates = brickwork_circuit(n, d, layers, t, seed)
    ops = G.ops_from_gates(gates, d)
    sim = G.Simulator(n, d, chi_max=64, cutoff=1e-14)
    try:
        sim.set_jacobi_cap(1)
        sim.run(ops)
        with pytest.raises(G.GcampsError) as ei:
            sim.sync()
        assert ei.value.code == N.ENOCONV
        assert "Jacobi" in str(ei.value)
        with pytest.raises(G.GcampsError):
            sim.set_jacobi_cap(0)   # refused, the cap stays 1
        sim.set_jacobi_cap(60)
        sim.reset()
        sim.run(ops)
        sim.sync()
        assert sim.stats()["status"] == 0
        ref = GCAMPS(n, d, chi_max=64, cutoff=1e-14)
        for g in gates:
            ref.apply_gate(g)
            if not hasattr(g, "sp_index"):
                ref.disentangle()
        assert sim.decisions() == ref.decisions
        err, _ = sv.same_up_to_phase(sim.statevector(), sv.run(gates, n, d))
        assert err < 1e-10
    finally:
        sim.close()


def test_oversized_handle_is_refused_with_enomem_and_leaks_nothing(G):
    import torch
    from paper_2511_06672_gb300 import _native as N
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    with pytest.raises(G.GcampsError) as ei:
        G.Simulator(128, 3, chi_max=5000)
    assert ei.value.code == N.ENOMEM
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < 64 << 20
