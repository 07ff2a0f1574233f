"""Direct pins for the oracle's helper functions (the ones the end-to-end pins use but do not
name): the d-term MPO, the Gaussian elimination of Sec. 2.3.1, the symplectic representation,
the standard phase, the gate helpers of the dense simulator, the centre moves and the copies.

Each expected value comes from dense linear algebra or a closed form, not from the helper's own
arithmetic.
"""
import itertools

import numpy as np
import pytest

from oracle import clifford, statevector as sv
from oracle.gcamps import GCAMPS, expansion_coefficients
from oracle.mps import MPS
from oracle.tableau import Tableau
from oracle.weyl import Weyl, tau
from synth.circuits import Clifford2, Diag


def _contract_mpo(ws, d):
    """Dense operator of an MPO whose tensors are [left bond, right bond, out, in]."""
    cur = [ws[0][0, a] for a in range(ws[0].shape[1])]
    for w in ws[1:]:
        nxt = []
        for b in range(w.shape[1]):
            acc = 0
            for a in range(w.shape[0]):
                acc = acc + np.kron(cur[a], w[a, b])
            nxt.append(acc)
        cur = nxt
    assert len(cur) == 1
    return cur[0]


def _random_weyl_with_support(n, d, support, rng):
    x = np.zeros(n, dtype=np.int64)
    z = np.zeros(n, dtype=np.int64)
    for j in support:
        while x[j] == 0 and z[j] == 0:
            x[j], z[j] = rng.integers(0, d, 2)
    return Weyl(int(rng.integers(0, 2 * d)), x, z, d)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("support", [[2], [1, 2], [0, 3], [1, 2, 4]])
def test_mpo_tensors_equal_the_dense_weighted_power_sum(d, support):
    """Sec. 3: the MPO of sum_m c_m P^m over the span of P equals the dense sum, with P^m taken as
    dense matrix powers; sites of the span where P is the identity included."""
    n = 5
    rng = np.random.default_rng(40 + 7 * d + len(support))
    p = _random_weyl_with_support(n, d, support, rng)
    coeffs = rng.standard_normal(d) + 1j * rng.standard_normal(d)
    f, l, ws = GCAMPS(n, d, chi_max=8).mpo_tensors(p, coeffs)
    assert (f, l) == (support[0], support[-1])
    assert len(ws) == l - f + 1
    assert all(w.shape[1] <= d and w.shape[0] <= d for w in ws)
    op = np.kron(np.kron(np.eye(d ** f), _contract_mpo(ws, d)), np.eye(d ** (n - 1 - l)))
    pd = p.dense()
    want = sum(coeffs[m] * np.linalg.matrix_power(pd, m) for m in range(d))
    assert np.allclose(op, want, atol=1e-12)


@pytest.mark.parametrize("d,n", [(2, 3), (3, 2)])
def test_decompose_on_the_initial_tableau_is_the_closed_form(d, n):
    """With S_j = Z_j and D_j = X_j: prod_j Z_j^{z_j} X_j^{x_j} = omega^{sum z x} W(x, z), so the
    coefficients are (z | x) and the phase exponent is r - 2 sum_j x_j z_j (mod 2d)."""
    t = Tableau(n, d)
    for x in itertools.product(range(d), repeat=n):
        for z in itertools.product(range(d), repeat=n):
            r = (3 * sum(x) + sum(z)) % (2 * d)
            coeff, c0 = t.decompose(Weyl(r, x, z, d))
            assert list(coeff[:n]) == list(z) and list(coeff[n:]) == list(x)
            assert c0 == (r - 2 * int(np.dot(x, z))) % (2 * d)


@pytest.mark.parametrize("d,n", [(2, 2), (3, 2)])
def test_decompose_is_the_unique_row_product_by_brute_force(d, n):
    """Sec. 2.3.1 on a scrambled tableau: among all d^{2n} coefficient vectors exactly one gives
    prod_j S_j^{c_j} D_j^{c_{n+j}} proportional to P (dense matrices), and it is decompose's, with
    the phase tau^{c0}."""
    rng = np.random.default_rng(11 + d)
    t = Tableau(n, d)
    for _ in range(5):
        idx = int(rng.integers(0, len(clifford.sp_group(2, d))))
        shift = tuple(int(a) for a in rng.integers(0, d, 4))
        t.apply_gate(clifford.unitary_from_images(clifford.random_gate_images(idx, shift, d), 2, d), [0, 1])
    rows = [r.dense() for r in t.rows]
    dim = d ** n
    for _ in range(4):
        p = Weyl(int(rng.integers(0, 2 * d)), rng.integers(0, d, n), rng.integers(0, d, n), d)
        pd = p.dense()
        hits = []
        for c in itertools.product(range(d), repeat=2 * n):
            m = np.eye(dim, dtype=complex)
            for j in range(n):
                m = m @ np.linalg.matrix_power(rows[j], c[j]) @ np.linalg.matrix_power(rows[n + j], c[n + j])
            ov = np.vdot(m, pd) / dim
            if abs(abs(ov) - 1) < 1e-9:
                hits.append((c, m))
        assert len(hits) == 1
        c, m = hits[0]
        coeff, c0 = t.decompose(p)
        assert tuple(int(a) for a in coeff) == c
        assert np.allclose(tau(d) ** c0 * m, pd, atol=1e-12)


def test_symplectic_of_sum_gate_is_the_textbook_matrix():
    """SUM|i, j> = |i, i + j>: X_0 -> X_0 X_1, Z_0 -> Z_0, X_1 -> X_1, Z_1 -> Z_0^{-1} Z_1
    (columns in the coordinates x_0, z_0, x_1, z_1)."""
    for d in (2, 3):
        s = clifford.symplectic_of_images(clifford.images_by_conjugation(clifford.SUM_gate(d), 2, d), 2, d)
        want = np.array([[1, 0, 0, 0],
                         [0, 1, 0, d - 1],
                         [1, 0, 1, 0],
                         [0, 0, 0, 1]])
        assert np.array_equal(s, want)
        assert clifford.is_symplectic(s, d)


@pytest.mark.parametrize("d", [2, 3])
def test_symplectic_representation_is_a_homomorphism(d):
    """U V g V^dag U^dag: the symplectic matrix of a product is the product mod d."""
    rng = np.random.default_rng(70 + d)
    order = len(clifford.sp_group(2, d))
    for _ in range(4):
        us = []
        for _k in range(2):
            idx = int(rng.integers(0, order))
            shift = tuple(int(a) for a in rng.integers(0, d, 4))
            us.append(clifford.unitary_from_images(clifford.random_gate_images(idx, shift, d), 2, d))
        su, sv_ = (clifford.symplectic_of_images(clifford.images_by_conjugation(u, 2, d), 2, d) for u in us)
        suv = clifford.symplectic_of_images(clifford.images_by_conjugation(us[0] @ us[1], 2, d), 2, d)
        assert np.array_equal(suv, (su @ sv_) % d)


@pytest.mark.parametrize("d", [2, 3])
def test_standard_phase_gives_order_d_and_hermitian_qubit_paulis(d):
    """tau^{std} W(x, z) has W^d = I (odd d: already with phase 0); for d = 2 it is Hermitian
    (the Pauli strings with Y = i X Z)."""
    for x in itertools.product(range(d), repeat=2):
        for z in itertools.product(range(d), repeat=2):
            w = Weyl(clifford.std_phase(x, z, d), x, z, d).dense()
            assert np.allclose(np.linalg.matrix_power(w, d), np.eye(d * d))
            if d == 2:
                assert np.allclose(w, w.conj().T)
    assert clifford.std_phase([1], [1], 2) == 1 and clifford.std_phase([1], [1], 3) == 0


def test_generators_and_diag_gate():
    d = 3
    g = clifford.generators(2, d)
    assert [(list(w.x), list(w.z)) for w in g] == [([1, 0], [0, 0]), ([0, 0], [1, 0]),
                                                   ([0, 1], [0, 0]), ([0, 0], [0, 1])]
    ph = [0.3, -1.1, 2.0]
    u = clifford.diag_gate(ph)
    for j in range(d):
        e = np.zeros(d)
        e[j] = 1
        assert np.allclose(u @ e, np.exp(1j * ph[j]) * e)
    # the expansion of Sec. 3 rebuilds the same matrix from Z powers
    zm = np.diag(np.exp(2j * np.pi * np.arange(d) / d))
    c = expansion_coefficients(ph, d)
    assert np.allclose(sum(c[m] * np.linalg.matrix_power(zm, m) for m in range(d)), u)


@pytest.mark.parametrize("d", [2, 3])
def test_dense_simulator_gate_helpers(d):
    dg = Diag(site=2, phases=tuple(0.1 * (k + 1) for k in range(d)))
    assert sv.gate_sites(dg) == [2]
    assert np.allclose(sv.gate_unitary(dg, d), np.diag(np.exp(1j * np.array(dg.phases))))
    cg = Clifford2(q0=1, q1=2, sp_index=5, shift=(1, 0, 1, 1))
    assert sv.gate_sites(cg) == [1, 2]
    u = sv.gate_unitary(cg, d)
    assert np.allclose(u @ u.conj().T, np.eye(d * d))
    want = clifford.random_gate_images(5, (1, 0, 1, 1), d)
    assert clifford.images_by_conjugation(u, 2, d) == want


def test_single_centre_moves_keep_the_state_and_gauge():
    """One QR step right / left: same dense state, the site left behind is an isometry."""
    rng = np.random.default_rng(3)
    d, n, chi = 3, 4, 3
    dims = [1] + [min(chi, d ** min(b, n - b)) for b in range(1, n)] + [1]
    m = MPS([rng.standard_normal((dims[j], d, dims[j + 1])) + 1j * rng.standard_normal((dims[j], d, dims[j + 1]))
             for j in range(n)], d, oc=0)
    v0 = m.to_dense()
    m._move_right()
    assert m.oc == 1 and np.allclose(m.to_dense(), v0)
    a = m.A[0].reshape(-1, m.A[0].shape[2])
    assert np.allclose(a.conj().T @ a, np.eye(a.shape[1]))
    m._move_right()
    m._move_left()
    assert m.oc == 1 and np.allclose(m.to_dense(), v0)
    b = m.A[2].reshape(m.A[2].shape[0], -1)
    assert np.allclose(b @ b.conj().T, np.eye(b.shape[0]))


def test_copies_are_independent():
    d, n = 3, 3
    w = Weyl(1, [1, 0, 2], [0, 1, 1], d)
    wc = w.copy()
    wc.x[0] = 2
    assert w.x[0] == 1
    t = Tableau(n, d)
    tc = t.copy()
    tc.apply_gate(clifford.SUM_gate(d), [0, 1])
    assert all(r == Weyl.single(n, d, j, "Z") for j, r in enumerate(t.rows[:n]))
    assert any(a != b for a, b in zip(t.rows, tc.rows))
    m = MPS.zero_state(n, d)
    mc = m.copy()
    mc.A[0][...] = 0
    assert abs(m.norm() - 1) < 1e-12
