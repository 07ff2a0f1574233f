"""Pins for oracle/tableau.py, oracle/statevector.py and oracle/mps.py.

* The initial tableau equals the |00> example of Sec. 2.2 (golden fixture).
* Row-by-row local updates equal full-matrix conjugation C Z_j C^dag with the dense C.
* Gaussian elimination + phase (Sec. 2.3.1) equals the dense C^dag P C.
* The fold C <- C Q^dag equals the dense conjugation with C Q^dag.
* MPS operations against dense linear algebra (Eckart-Young for the truncation).
"""
import os

import numpy as np
import pytest

from oracle import clifford, statevector as sv
from oracle.mps import MPS, truncation_rank
from oracle.tableau import Tableau
from oracle.weyl import Weyl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dense_gate(u, sites, n, d):
    """Full d^n x d^n matrix of a gate on ``sites``."""
    dim = d ** n
    m = np.zeros((dim, dim), dtype=complex)
    for col in range(dim):
        e = np.zeros(dim, dtype=complex)
        e[col] = 1
        m[:, col] = sv.apply_gate(e, u, sites, n, d)
    return m


def random_clifford_sequence(n, d, ngates, rng):
    gates = []
    for _ in range(ngates):
        q0 = int(rng.integers(0, n - 1))
        idx = int(rng.integers(0, len(clifford.sp_group(2, d))))
        shift = tuple(int(a) for a in rng.integers(0, d, 4))
        u = clifford.unitary_from_images(clifford.random_gate_images(idx, shift, d), 2, d)
        gates.append((u, [q0, q0 + 1]))
    return gates


def test_initial_tableau_golden():
    rows = []
    with open(os.path.join(GOLDEN, "tableau_00.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            rows.append(line.split())
    t = Tableau(2, 2)
    e, ph = t.exps_phase()
    for k, (a, b, sign) in enumerate(rows):
        assert sign == "+1" and ph[k] == 0
        for q, letter in enumerate((a, b)):
            assert e[k, q] == (letter == "X")
            assert e[k, 2 + q] == (letter == "Z")


@pytest.mark.parametrize("d,n", [(2, 3), (3, 3)])
def test_tableau_updates_match_dense_conjugation(d, n):
    rng = np.random.default_rng(3 + d)
    t = Tableau(n, d)
    c = np.eye(d ** n, dtype=complex)
    for u, sites in random_clifford_sequence(n, d, 6, rng):
        t.apply_gate(u, sites)
        c = dense_gate(u, sites, n, d) @ c
    for j in range(n):
        zj = Weyl.single(n, d, j, "Z").dense()
        xj = Weyl.single(n, d, j, "X").dense()
        assert t.rows[j] == clifford.snap(c @ zj @ c.conj().T, n, d)
        assert t.rows[n + j] == clifford.snap(c @ xj @ c.conj().T, n, d)
    # symplectic structure: stabilizers commute, Lambda(D_i, S_j) = Lambda(X_i, Z_j) = -delta_ij
    from oracle.weyl import symplectic_form
    for i in range(n):
        for j in range(n):
            si, sj, di = t.rows[i], t.rows[j], t.rows[n + i]
            assert symplectic_form(si.x, si.z, sj.x, sj.z, d) == 0
            assert symplectic_form(di.x, di.z, sj.x, sj.z, d) == ((d - 1) if i == j else 0)
    # decomposition: C^dag P C for random P, and the inverse rows
    for _ in range(8):
        p = Weyl(int(rng.integers(0, 2 * d)), rng.integers(0, d, n), rng.integers(0, d, n), d)
        got = t.conjugate_back(p)
        assert got == clifford.snap(c.conj().T @ p.dense() @ c, n, d)
        assert (got ** d) == (p ** d)          # conjugation preserves the scalar P^d
    inv = t.inverse_rows()
    for j in range(n):
        assert inv[j] == clifford.snap(c.conj().T @ Weyl.single(n, d, j, "Z").dense() @ c, n, d)


@pytest.mark.parametrize("d,n", [(2, 3), (3, 3)])
def test_fold_right_inverse(d, n):
    rng = np.random.default_rng(21 + d)
    t = Tableau(n, d)
    c = np.eye(d ** n, dtype=complex)
    for u, sites in random_clifford_sequence(n, d, 4, rng):
        t.apply_gate(u, sites)
        c = dense_gate(u, sites, n, d) @ c
    _s, _imgs, q = clifford.candidates(d)[int(rng.integers(1, 20))]
    t.apply_gate_right_inverse(q, [1, 2])
    c = c @ dense_gate(q, [1, 2], n, d).conj().T
    for j in range(n):
        assert t.rows[j] == clifford.snap(c @ Weyl.single(n, d, j, "Z").dense() @ c.conj().T, n, d)
        assert t.rows[n + j] == clifford.snap(c @ Weyl.single(n, d, j, "X").dense() @ c.conj().T, n, d)


def test_statevector_basics():
    d, n = 3, 3
    psi = sv.zero_state(n, d)
    psi = sv.apply_gate(psi, clifford.H_gate(d), [0], n, d)       # site 0 most significant
    assert np.allclose(psi[[0, 9, 18]], 1 / np.sqrt(3))
    psi = sv.apply_gate(psi, clifford.SUM_gate(d), [0, 2], n, d)  # |i,0,0> -> |i,0,i>
    assert np.allclose(psi[[0, 9 + 1, 18 + 2]], 1 / np.sqrt(3))
    assert np.isclose(np.linalg.norm(psi), 1)


def test_truncation_rank_rules():
    s = np.array([1.0, 0.5, 1e-13, 0.0])
    assert truncation_rank(s, 1e-12, 10) == 2
    assert truncation_rank(s, 1e-14, 10) == 3
    assert truncation_rank(s, 1e-14, 1) == 1
    assert truncation_rank(np.zeros(3), 1e-12, 5) == 1


def random_mps(n, d, chi, rng):
    ts = []
    dims = [1] + [min(chi, d ** min(j + 1, n - j - 1)) for j in range(n - 1)] + [1]
    for j in range(n):
        ts.append(rng.standard_normal((dims[j], d, dims[j + 1])) + 1j * rng.standard_normal((dims[j], d, dims[j + 1])))
    m = MPS(ts, d, 0)
    v = m.to_dense()
    m.A[0] /= np.linalg.norm(v)
    # bring into canonical form with the centre at 0
    m.oc = n - 1
    m.move_center(0)
    return m


def test_mps_moves_and_canonical_form():
    rng = np.random.default_rng(5)
    d, n = 3, 5
    m = random_mps(n, d, 4, rng)
    v0 = m.to_dense()
    for target in (3, 1, 4, 0, 2):
        m.move_center(target)
        assert np.allclose(m.to_dense(), v0)
        for j in range(target):
            a = m.A[j].reshape(-1, m.A[j].shape[2])
            assert np.allclose(a.conj().T @ a, np.eye(a.shape[1]))
        for j in range(target + 1, n):
            a = m.A[j].reshape(m.A[j].shape[0], -1)
            assert np.allclose(a @ a.conj().T, np.eye(a.shape[0]))
    for i in range(n - 1):
        dense_s = np.linalg.svd(v0.reshape(d ** (i + 1), -1), compute_uv=False)
        s = m.schmidt_values(i)
        assert np.allclose(s, dense_s[: len(s)])


def test_mpo_apply_vs_dense():
    rng = np.random.default_rng(9)
    d, n = 2, 5
    m = random_mps(n, d, 3, rng)
    v = m.to_dense()
    ws = []
    dense_op = np.array([[1.0 + 0j]])
    dl = 1
    for k in range(3):
        dr = 1 if k == 2 else 2
        w = rng.standard_normal((dl, dr, d, d)) + 1j * rng.standard_normal((dl, dr, d, d))
        ws.append(w)
        dl = dr
    # dense operator of the MPO on sites 1..3
    full = np.zeros((d ** 3, d ** 3), dtype=complex)
    for a in range(2):
        for b in range(2):
            full += np.kron(np.kron(ws[0][0, a], ws[1][a, b]), ws[2][b, 0])
    op = np.kron(np.kron(np.eye(d), full), np.eye(d))
    m.apply_mpo(ws, 1)
    assert np.allclose(m.to_dense(), op @ v)


def test_compress_eckart_young():
    rng = np.random.default_rng(13)
    d, n = 2, 6
    m = random_mps(n, d, 8, rng)
    v = m.to_dense()
    m.move_center(3)
    disc = m.compress(2, 3, 1e-14, 100)       # no truncation: exact
    assert disc < 1e-20 and np.allclose(m.to_dense(), v)
    m.move_center(2)
    s = m.schmidt_values(2)
    disc = m.compress(2, 3, 1e-14, 2)        # one bond truncated to 2: optimal error
    assert np.isclose(disc, np.sum(s[2:] ** 2))
    w = m.to_dense()
    kept = np.sqrt(1 - disc)
    assert np.isclose(np.linalg.norm(w), 1)
    assert np.isclose(abs(np.vdot(w, v)), kept, atol=1e-10)


def test_expect_local_vs_dense():
    rng = np.random.default_rng(17)
    d, n = 3, 4
    m = random_mps(n, d, 3, rng)
    v = m.to_dense()
    p = Weyl(0, rng.integers(0, d, n), rng.integers(0, d, n), d)
    ops = {j: p.local_matrix(j) for j in p.support()}
    assert np.isclose(m.expect_local(ops), sv.expect_weyl(v, p, n, d))
