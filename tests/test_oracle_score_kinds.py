"""Pins for the disentangler score kinds of the oracle (the score readings of Sec. 3 / Sec. 4):
von Neumann entropy (kind 0), Renyi-2 entropy (kind 1) and the bond-dimension criterion read as the
number of Schmidt weights above max(1e-12, 4 cutoff^2) with the entropy as tie-break (kind 2).

Pinned against closed forms (maximally entangled and product spectra, two-level spectra written out
by hand), the ordering S2 <= S_vN, the rank of matrices built with a known rank, the Bell pair of
Sec. 3 (best class reaches zero under every kind), hand-made decision examples for the tie rules, and
exactness of whole runs against the dense state vector (the decision rule never changes the state).
"""
import numpy as np
import pytest

from oracle import clifford, statevector as sv
from oracle import gcamps as G
from synth import brickwork_circuit


def test_renyi2_closed_forms():
    for d in (2, 3, 5):
        assert abs(G.renyi2_from_singular_values(np.ones(d)) - np.log(d)) < 1e-14
    assert G.renyi2_from_singular_values(np.array([1.0, 0.0, 0.0])) == 0.0
    for a in (0.1, 0.25, 0.5, 0.9):
        s = np.sqrt(np.array([a, 1 - a])) * 3.0          # unnormalised on purpose
        want = -np.log(a * a + (1 - a) * (1 - a))
        assert abs(G.renyi2_from_singular_values(s) - want) < 1e-14


def test_renyi2_is_below_von_neumann():
    rng = np.random.default_rng(5)
    for _ in range(50):
        s = rng.random(rng.integers(1, 12)) ** 3
        assert G.renyi2_from_singular_values(s) <= G.entropy_from_singular_values(s) + 1e-14


def test_weight_rank_counts_known_rank_and_threshold():
    rng = np.random.default_rng(7)
    for r in (1, 2, 5, 9):
        a = rng.standard_normal((12, r)) + 1j * rng.standard_normal((12, r))
        b = rng.standard_normal((r, 15)) + 1j * rng.standard_normal((r, 15))
        assert G.weight_rank(np.linalg.svd(a @ b, compute_uv=False), 1e-12) == r
    s = np.array([1.0, 0.5, 1e-5, 1e-7])                 # weights ~ 1, 0.25, 1e-10, 1e-14
    assert G.weight_rank(s, 1e-12) == 3
    assert G.weight_rank(s, 1e-4) == 2                   # threshold 4e-8 drops the 1e-10 weight
    assert G.weight_rank(np.zeros(3), 1e-12) == 0


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("kind", [0, 1, 2])
def test_bell_pair_best_class_under_every_kind(d, kind):
    psi = np.zeros(d * d, dtype=complex)
    psi[0] = 1
    psi = clifford.SUM_gate(d) @ np.kron(clifford.H_gate(d), np.eye(d)) @ psi
    g = G.GCAMPS(2, d, chi_max=d, cutoff=1e-12, score_kind=kind)
    keys = g.score_keys(psi.reshape(1, d, d, 1))
    k = g.choose(keys)
    assert k != 0
    if kind == 2:
        rank, vn = keys
        assert rank[0] == d and rank[k] == 1 and vn[k] < 1e-12
    else:
        assert abs(keys[0] - np.log(d)) < 1e-12 and keys[k] < 1e-12


def test_choose_rules_by_hand():
    g = G.GCAMPS(2, 3, chi_max=9, cutoff=1e-12, score_kind=2)
    rank = np.array([3, 2, 2, 3])
    assert g.choose((rank, np.array([1.0, 0.5, 0.4, 0.1]))) == 2      # smallest rank, then entropy
    assert g.choose((rank, np.array([1.0, 0.4, 0.4 + 5e-11, 0.1]))) == 1   # tie -> lowest index
    assert g.choose((np.array([2, 2, 3]), np.array([0.5, 0.5 - 5e-11, 0.1]))) == 0   # no gain over I
    assert g.choose((np.array([3, 2, 3]), np.array([0.5, 0.9, 0.1]))) == 1   # rank beats entropy
    g1 = G.GCAMPS(2, 3, chi_max=9, cutoff=1e-12, score_kind=1)
    assert g1.choose(np.array([0.7, 0.3, 0.3 + 5e-11, 0.2])) == 3
    assert g1.choose(np.array([0.7, 0.7 - 5e-11])) == 0


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("d,n,seed", [(3, 6, 3), (2, 7, 4)])
def test_runs_stay_exact_under_every_kind(kind, d, n, seed):
    gates = brickwork_circuit(n, d, n, n, seed)
    psi = sv.run(gates, n, d)
    g = G.GCAMPS(n, d, chi_max=64, cutoff=1e-14, score_kind=kind)
    for gt in gates:
        g.apply_gate(gt)
        if not hasattr(gt, "sp_index"):
            g.disentangle()
    err, _ = sv.same_up_to_phase(g.statevector(), psi)
    assert err < 1e-10
    assert any(k for _b, k in g.decisions)


def test_score_kind_is_validated():
    with pytest.raises(ValueError):
        G.GCAMPS(4, 3, chi_max=9, score_kind=3)
