"""The bond-dimension-per-layer experiment (Fig. 5a) on the circuit family of Fig. 4: the seeded
generator, and the per-layer curve logic of bench.py run with the oracle as the simulator (CPU).

Pins: the generator's layout (a random Clifford on all qudits, then one T gate on qudit 0, per
layer); layer-by-layer runs are the whole circuit (dense state at the end); after one layer the bond
dimension is at most d (an MPO of bond dimension d applied to a product state); the scaled axis is
max chi / d^floor(n/2).
"""
import numpy as np
import pytest

import bench
from oracle import statevector as sv
from oracle.gcamps import GCAMPS
from synth import Clifford2, Diag, layered_t_circuit, t_gate_phases


@pytest.mark.parametrize("d,n,layers,depth", [(2, 5, 3, 0), (3, 4, 4, 2)])
def test_layered_generator_layout(d, n, layers, depth):
    gates, ends = layered_t_circuit(n, d, layers, seed=7, depth=depth)
    depth = depth or n
    assert len(ends) == layers and ends[-1] == len(gates)
    starts = [0] + ends[:-1]
    sub = 0
    for a, b in zip(starts, ends):
        layer = gates[a:b]
        assert isinstance(layer[-1], Diag) and layer[-1].site == 0
        assert layer[-1].phases == tuple(t_gate_phases(d))
        cliffs = layer[:-1]
        assert all(isinstance(g, Clifford2) and g.q1 == g.q0 + 1 for g in cliffs)
        want_pairs = []
        for _s in range(depth):
            want_pairs += [(i, i + 1) for i in range(sub % 2, n - 1, 2)]
            sub += 1
        assert [(g.q0, g.q1) for g in cliffs] == want_pairs
    again, _ = layered_t_circuit(n, d, layers, seed=7, depth=depth)
    other, _ = layered_t_circuit(n, d, layers, seed=8, depth=depth)
    assert again == gates and other != gates


def test_scaled_max_chi_axis():
    assert bench.scaled_max_chi([[1, 3, 1], [3, 9, 3]], 4, 3) == [3 / 9, 1.0]
    assert bench.scaled_max_chi([[2, 4, 2, 1]], 5, 2) == [1.0]


def _oracle_curve(n, d, layers, seed, budget_s=float("inf")):
    gates, ends = layered_t_circuit(n, d, layers, seed)
    starts = [0] + ends[:-1]
    ref = GCAMPS(n, d, chi_max=d ** (n // 2), cutoff=1e-12)

    def run_layer(gs):
        for gt in gs:
            ref.apply_gate(gt)
            if not hasattr(gt, "sp_index"):
                ref.disentangle()

    dims, secs = bench.bond_dims_per_layer([gates[a:b] for a, b in zip(starts, ends)], run_layer,
                                           ref.mps.bond_dims, budget_s)
    return gates, ref, dims, secs


@pytest.mark.parametrize("d,n,layers", [(3, 4, 6), (2, 6, 8)])
def test_layer_by_layer_oracle_run_is_the_whole_circuit(d, n, layers):
    gates, ref, dims, secs = _oracle_curve(n, d, layers, seed=3)
    assert len(dims) == layers and len(secs) == layers
    assert max(dims[0]) <= d
    for ds in dims:
        assert all(1 <= c <= d ** min(b + 1, n - 1 - b) for b, c in enumerate(ds))
    assert all(0 < v <= 1 for v in bench.scaled_max_chi(dims, n, d))
    assert dims[-1] == ref.mps.bond_dims()
    err, _ = sv.same_up_to_phase(ref.statevector(), sv.run(gates, n, d))
    assert err < 1e-9


def test_budget_stops_after_the_layer_that_exceeds_it():
    _g, _ref, dims, _secs = _oracle_curve(4, 2, 5, seed=1, budget_s=0.0)
    assert len(dims) == 1


def test_constant_regime_at_low_depth():
    """Fig. 5a's constant regime: with few T gates on a deep random Clifford the disentangled MPS
    stays a product state (seeded instances, qubits and qutrits)."""
    for d in (2, 3):
        _g, _ref, dims, _s = _oracle_curve(6, d, 3, seed=1)
        assert [max(ds) for ds in dims] == [1, 1, 1]


def test_reference_arm_prints_the_curves():
    """bench.py --impl reference --workload chi-layers: one JSON line with a curve per (d, n)."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                          "chi-layers", "--chi-layers-d", "2,3", "--chi-layers-n", "4", "--chi-layers-factor", "1",
                          "--chi-layers-score-kind", "2"],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "T-gates/s" and line["value"] > 0
    assert line["config"]["score_kind"] == 2
    assert [(c["d"], c["n"], c["layers_run"]) for c in line["curves"]] == [(2, 4, 4), (3, 4, 4)]
    for c in line["curves"]:
        assert len(c["scaled_max_chi"]) == len(c["max_chi"]) == 4
        assert c["scaled_layers"] == [0.25, 0.5, 0.75, 1.0]
