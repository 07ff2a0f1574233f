"""Pins for oracle/gcamps.py: exactness against dense simulation (Sec. 3: psi = C|MPS>),
the expansion of the diagonal gate, state invariance of the fold C~ = C Q^dag, and planted
mistakes that the pins must catch."""
import numpy as np
import pytest

from oracle import clifford, statevector as sv
from oracle import gcamps as G
from oracle.weyl import Weyl, Z, tau
from synth import brickwork_circuit, t_gate_phases


@pytest.mark.parametrize("d", [2, 3])
def test_expansion_coefficients(d):
    for phases in (t_gate_phases(d), tuple(np.random.default_rng(d).uniform(0, 6, d))):
        c = G.expansion_coefficients(phases, d)
        m = sum(c[k] * np.linalg.matrix_power(Z(d), k) for k in range(d))
        assert np.allclose(m, np.diag(np.exp(1j * np.array(phases))), atol=1e-15)
        assert np.isclose(np.sum(np.abs(c) ** 2), 1.0)     # Parseval


def run_both(d, n, layers, t, seed, **kw):
    gates = brickwork_circuit(n, d, layers, t, seed)
    psi = sv.run(gates, n, d)
    g = G.GCAMPS(n, d, **kw)
    for gt in gates:
        g.apply_gate(gt)
        if not hasattr(gt, "sp_index"):
            g.disentangle()
    return g, psi


@pytest.mark.parametrize("d,n,seed", [(3, 6, 1), (3, 6, 2), (2, 8, 1), (2, 7, 3)])
def test_gcamps_matches_dense(d, n, seed):
    g, psi = run_both(d, n, n, n, seed, chi_max=64, cutoff=1e-14)
    err, _ = sv.same_up_to_phase(g.statevector(), psi)
    assert err < 1e-10
    assert abs(g.mps.norm() - 1) < 1e-12
    rng = np.random.default_rng(seed)
    for _ in range(6):
        x, z = rng.integers(0, d, n), rng.integers(0, d, n)
        w = Weyl(0, x, z, d)
        assert abs(g.expect_weyl(x, z) - sv.expect_weyl(psi, w, n, d)) < 1e-10
    # a stabilizer of the final Clifford part (nonzero expectation on |0> part) is also right
    z0 = np.zeros(n, dtype=np.int64)
    z0[0] = 1
    assert abs(g.expect_weyl(np.zeros(n, dtype=np.int64), z0)
               - sv.expect_weyl(psi, Weyl(0, np.zeros(n), z0, d), n, d)) < 1e-10


def test_gcamps_without_disentangling_is_exact():
    d, n = 3, 5
    gates = brickwork_circuit(n, d, 5, 5, 4)
    psi = sv.run(gates, n, d)
    g = G.GCAMPS(n, d, chi_max=243, cutoff=1e-14, max_sweeps=0)
    for gt in gates:
        g.apply_gate(gt)
    assert sv.same_up_to_phase(g.statevector(), psi)[0] < 1e-10


def test_t_gate_on_product_state_keeps_chi_one():
    d, n = 3, 4
    g = G.GCAMPS(n, d, chi_max=16)
    g.apply_nonclifford(2, t_gate_phases(d))
    assert g.span == (2, 2)
    assert g.mps.bond_dims() == [1, 1, 1]


def test_disentangle_preserves_state():
    d, n = 3, 6
    gates = brickwork_circuit(n, d, 6, 6, 9)
    g = G.GCAMPS(n, d, chi_max=64, cutoff=1e-14)
    for gt in gates:
        g.apply_gate(gt)
        if not hasattr(gt, "sp_index"):
            before = g.statevector()
            st = g.disentangle()
            after = g.statevector()
            assert sv.same_up_to_phase(after, before)[0] < 1e-10
    assert g.decisions  # at least one bond was visited


def test_disentangle_reduces_entanglement_of_bell_pairs():
    d, n = 3, 4
    g = G.GCAMPS(n, d, chi_max=16)
    u = clifford.SUM_gate(d) @ np.kron(clifford.H_gate(d), np.eye(d))
    # put the MPS (not C) in two Bell pairs on bonds (0,1) and (2,3)
    psi = np.kron(u @ np.eye(d * d)[:, 0], u @ np.eye(d * d)[:, 0])
    t = psi.reshape(d, d, d, d)
    from oracle.mps import MPS
    m = MPS([np.ones((1, 1, 1))] * n, d)
    m.A = []
    rest = t.reshape(1, -1)
    for j in range(n - 1):
        cl = rest.shape[0]
        mat = rest.reshape(cl * d, -1)
        uu, s, vh = np.linalg.svd(mat, full_matrices=False)
        k = int(np.sum(s > 1e-12))
        m.A.append(uu[:, :k].reshape(cl, d, k))
        rest = s[:k, None] * vh[:k]
    m.A.append(rest.reshape(rest.shape[0], d, 1))
    m.oc = n - 1
    g.mps = m
    before = g.statevector()
    g.span = (0, 3)
    g.disentangle()
    assert g.mps.bond_dims() == [1, 1, 1]
    assert sv.same_up_to_phase(g.statevector(), before)[0] < 1e-10


def test_planted_phase_mistake_is_caught(monkeypatch):
    """Flip the commutation phase in the oracle's Weyl product: the dense comparison fails."""
    from oracle import weyl

    def wrong_mul(self, other):
        d = self.d
        r = self.r + other.r + 2 * int(np.sum(self.x * other.z))   # wrong: x.z' instead of z.x'
        return weyl.Weyl(r, self.x + other.x, self.z + other.z, d)

    monkeypatch.setattr(weyl.Weyl, "__mul__", wrong_mul)
    with pytest.raises(Exception):
        g, psi = run_both(3, 5, 5, 5, 1, chi_max=64, cutoff=1e-14)
        err, _ = sv.same_up_to_phase(g.statevector(), psi)
        assert err < 1e-10


def test_planted_transpose_mistake_is_caught(monkeypatch):
    """Fold the transposed candidate into the tableau (the MPS gets Q, C gets (Q^T)^dag):
    the state is no longer preserved and the dense comparison must fail."""
    from oracle.tableau import Tableau
    orig = Tableau.apply_gate_right_inverse

    def wrong_fold(self, u, sites):
        return orig(self, u.T, sites)

    monkeypatch.setattr(Tableau, "apply_gate_right_inverse", wrong_fold)
    g, psi = run_both(3, 6, 6, 6, 1, chi_max=64, cutoff=1e-14)
    err, _ = sv.same_up_to_phase(g.statevector(), psi)
    assert err > 1e-6


def test_replay_of_recorded_decisions_reproduces_the_run():
    """Replay mode (forced decisions, used to compare runs whose decisions could legitimately differ):
    feeding back the recorded decisions reproduces tableau, bond dimensions and state exactly; forcing
    'apply nothing' everywhere gives other decisions but the same physical state (Sec. 3: the fold
    C~ = C Q^dag never changes psi)."""
    d, n = 3, 6
    gates = brickwork_circuit(n, d, 6, 6, 13)
    a = G.GCAMPS(n, d, chi_max=64, cutoff=1e-14)
    per_gate = []
    for gt in gates:
        a.apply_gate(gt)
        if not hasattr(gt, "sp_index"):
            start = len(a.decisions)
            a.disentangle()
            per_gate.append([k for _b, k in a.decisions[start:]])
    assert any(any(x) for x in per_gate)
    b = G.GCAMPS(n, d, chi_max=64, cutoff=1e-14)
    c = G.GCAMPS(n, d, chi_max=64, cutoff=1e-14)
    it = iter(per_gate)
    for gt in gates:
        b.apply_gate(gt)
        c.apply_gate(gt)
        if not hasattr(gt, "sp_index"):
            b.disentangle(forced=next(it))
            c.disentangle(forced=[0] * 64)
    assert b.decisions == a.decisions
    ea, pa = a.tab.exps_phase()
    eb, pb = b.tab.exps_phase()
    assert np.array_equal(ea, eb) and np.array_equal(pa, pb)
    assert b.mps.bond_dims() == a.mps.bond_dims()
    assert np.array_equal(b.statevector(), a.statevector())
    assert all(k == 0 for _b, k in c.decisions)
    psi = sv.run(gates, n, d)
    assert sv.same_up_to_phase(c.statevector(), psi)[0] < 1e-10
    assert sv.same_up_to_phase(a.statevector(), psi)[0] < 1e-10
