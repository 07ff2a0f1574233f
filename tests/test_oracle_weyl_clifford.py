"""Pins for oracle/weyl.py and oracle/clifford.py against the paper and the mathematics.

* Weyl products, powers and commutation phases vs explicit matrix algebra.
* H_d, S_d, SUM_d conjugation vs Table 1 (golden fixture).
* d = 2 reduces to the qubit Paulis of Eq. (paulis2) and the textbook H and sqrt(Z).
* |Sp(2n, F_d)| vs the closed-form group orders; 20 / 90 classes vs Sec. 3.
* Class invariance of the Schmidt spectrum and a brute-force minimum over every Clifford.
"""
import itertools
import os

import numpy as np
import pytest

from oracle import clifford
from oracle.weyl import Weyl, X, Z, omega, tau, symplectic_form, snap_to_weyl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(7)


def rand_weyl(n, d, rng=RNG):
    return Weyl(rng.integers(0, 2 * d), rng.integers(0, d, n), rng.integers(0, d, n), d)


@pytest.mark.parametrize("d", [2, 3])
def test_weyl_relations(d):
    x, z = X(d), Z(d)
    assert np.allclose(x @ z, omega(d) ** -1 * z @ x)          # XZ = omega^{-1} ZX
    assert np.allclose(np.linalg.matrix_power(x, d), np.eye(d))
    assert np.allclose(np.linalg.matrix_power(z, d), np.eye(d))
    y = (tau(d) if d % 2 == 0 else 1.0) * x @ z                 # Y = XZ, or tau XZ for even d
    assert np.allclose(np.linalg.matrix_power(y, d), np.eye(d))


def test_qubit_paulis_golden():
    mats = {}
    with open(os.path.join(GOLDEN, "qubit_paulis.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, rest = line.split(None, 1)
            rows = []
            for r in rest.split("/"):
                rows.append([complex(*map(float, c.split(","))) for c in r.split()])
            mats[name] = np.array(rows)
    assert np.allclose(X(2), mats["X"])
    assert np.allclose(Z(2), mats["Z"])
    assert np.allclose(Weyl(1, [1], [1], 2).dense(), mats["Y"])    # tau^1 X Z = i XZ


@pytest.mark.parametrize("d", [2, 3])
def test_weyl_product_and_power_vs_matrices(d):
    for n in (1, 2, 3):
        for _ in range(20):
            a, b = rand_weyl(n, d), rand_weyl(n, d)
            assert np.allclose((a * b).dense(), a.dense() @ b.dense())
            m = int(RNG.integers(0, 2 * d + 1))
            assert np.allclose((a ** m).dense(), np.linalg.matrix_power(a.dense(), m))


@pytest.mark.parametrize("d", [2, 3])
def test_symplectic_form_is_commutation_phase(d):
    for _ in range(30):
        a, b = rand_weyl(2, d), rand_weyl(2, d)
        lam = symplectic_form(a.x, a.z, b.x, b.z, d)
        assert np.allclose(a.dense() @ b.dense(), omega(d) ** lam * b.dense() @ a.dense())


@pytest.mark.parametrize("d", [2, 3])
def test_snap_roundtrip(d):
    for _ in range(10):
        w = rand_weyl(2, d)
        assert snap_to_weyl(w.dense(), 2, d) == w
        assert clifford.snap(w.dense(), 2, d) == w
    with pytest.raises(ValueError):
        clifford.snap(np.kron(clifford.H_gate(d), np.eye(d)), 2, d)


def _parse_site(tok, d):
    x = z = 0
    for f in tok.split():
        if f in ("I",):
            continue
        p = -1 if f.endswith("^-1") else 1
        if f.startswith("X"):
            x += p
        elif f.startswith("Z"):
            z += p
        else:
            raise ValueError(f)
    return x % d, z % d


def _table1(d):
    rules = []
    with open(os.path.join(GOLDEN, "table1_rules.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            tokens = line.split()
            gate, inp, out = tokens[0], tokens[1], " ".join(tokens[2:])
            r = 0
            if out.startswith("(tau)"):
                out = out[len("(tau)"):].strip()
                r = 1 if d % 2 == 0 else 0
            ins = [_parse_site(t, d) for t in inp.split("(x)")]
            outs = [_parse_site(t, d) for t in out.split("(x)")]
            rules.append((gate, ins, outs, r))
    return rules


@pytest.mark.parametrize("d", [2, 3])
def test_table1_rules(d):
    gates = {"H": clifford.H_gate(d), "S": clifford.S_gate(d), "SUM": clifford.SUM_gate(d)}
    rules = _table1(d)
    assert len(rules) == 8
    for gate, ins, outs, r in rules:
        u = gates[gate]
        nq = len(ins)
        w_in = Weyl(0, [a for a, _ in ins], [b for _, b in ins], d)
        w_out = Weyl(r, [a for a, _ in outs], [b for _, b in outs], d)
        got = clifford.snap(u @ w_in.dense() @ u.conj().T, nq, d)
        assert got == w_out, (gate, ins, got, w_out)
        assert np.allclose(u.conj().T @ u, np.eye(d ** nq))


def test_d2_gates_are_textbook():
    h = clifford.H_gate(2)
    assert np.allclose(h, np.array([[1, 1], [1, -1]]) / np.sqrt(2))
    s = clifford.S_gate(2)
    assert np.allclose(s @ s, Z(2))                  # S = sqrt(Z) (phase gate, Sec. 2.2)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]])
    assert np.allclose(clifford.SUM_gate(2), cnot)


@pytest.mark.parametrize("d", [2, 3])
def test_unitary_from_images_recovers_gates(d):
    for u, nq in ((clifford.H_gate(d), 1), (clifford.S_gate(d), 1), (clifford.SUM_gate(d), 2),
                  (np.kron(clifford.H_gate(d), clifford.S_gate(d)) @ clifford.SUM_gate(d), 2)):
        imgs = clifford.images_by_conjugation(u, nq, d)
        v = clifford.unitary_from_images(imgs, nq, d)
        ov = np.vdot(v.reshape(-1), u.reshape(-1))
        assert np.isclose(abs(ov), d ** nq)          # equal up to one global phase
        assert np.allclose(v * (ov / abs(ov)), u)


@pytest.mark.parametrize("d", [2, 3])
def test_group_orders(d):
    sp2 = clifford.sp_group(1, d)
    sp4 = clifford.sp_group(2, d)
    assert len(sp2) == d * (d * d - 1)                           # |SL(2, F_d)|
    assert len(sp4) == d ** 4 * (d ** 2 - 1) * (d ** 4 - 1)      # |Sp(4, F_d)|
    assert sp4 == sorted(set(sp4))
    for idx in RNG.integers(0, len(sp4), 50):
        assert clifford.is_symplectic(clifford.sp4_matrix(int(idx), d), d)


@pytest.mark.parametrize("d", [2, 3])
def test_random_gate_images_define_a_clifford(d):
    for _ in range(5):
        idx = int(RNG.integers(0, len(clifford.sp_group(2, d))))
        shift = tuple(int(a) for a in RNG.integers(0, d, 4))
        imgs = clifford.random_gate_images(idx, shift, d)
        u = clifford.unitary_from_images(imgs, 2, d)
        assert np.allclose(u.conj().T @ u, np.eye(d * d))
        assert clifford.images_by_conjugation(u, 2, d) == imgs
        # the shift is the Weyl operator applied after the standard-phase Clifford
        u0 = clifford.unitary_from_images(clifford.random_gate_images(idx, (0, 0, 0, 0), d), 2, d)
        w = Weyl(0, [shift[0], shift[2]], [shift[1], shift[3]], d).dense()
        ov = np.vdot((w @ u0).reshape(-1), u.reshape(-1))
        assert np.isclose(abs(ov), d * d)


def _entropy(psi_matrix):
    s = np.linalg.svd(psi_matrix, compute_uv=False)
    p = s ** 2 / np.sum(s ** 2)
    p = p[p > 1e-300]
    return float(-np.sum(p * np.log(p)))


def test_candidate_counts_golden():
    with open(os.path.join(GOLDEN, "candidate_counts.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    for d, k in rows:
        c = clifford.candidates(int(d))
        assert len(c) == int(k)
        assert np.array_equal(c[0][0], np.eye(4, dtype=np.int64))


@pytest.mark.parametrize("d", [2, 3])
def test_class_invariance_and_brute_force(d):
    cands = clifford.candidates(d)
    sp4 = clifford.sp_group(2, d)
    rng = np.random.default_rng(11)
    # theta with an environment on both sides: (chi_l, d*d, chi_r)
    chi = 2
    theta = rng.standard_normal((chi, d * d, chi)) + 1j * rng.standard_normal((chi, d * d, chi))
    theta /= np.linalg.norm(theta)

    def ent(u):
        t = np.einsum("uv,avb->aub", u, theta).reshape(chi * d, d * chi)
        return _entropy(t)

    rep_ent = {}
    for s, _imgs, u in cands:
        rep_ent[tuple(s.reshape(-1))] = ent(u)
    # every member of a class has the representative's entanglement
    sp2 = [np.array(t).reshape(2, 2) for t in clifford.sp_group(1, d)]
    for k in range(len(cands)):
        s, _imgs, _u = cands[k]
        for _ in range(3):
            b = np.zeros((4, 4), dtype=np.int64)
            b[:2, :2] = sp2[rng.integers(len(sp2))]
            b[2:, 2:] = sp2[rng.integers(len(sp2))]
            m = (b @ s) % d
            shift = rng.integers(0, d, 4)
            u = clifford.unitary_from_images(clifford.images_from_symplectic(m, shift, d), 2, d)
            assert abs(ent(u) - rep_ent[tuple(s.reshape(-1))]) < 1e-10
    # brute force: the minimum over the whole group equals the minimum over the classes
    idxs = range(len(sp4)) if d == 2 else rng.integers(0, len(sp4), 400)
    best = min(ent(clifford.unitary_from_images(
        clifford.images_from_symplectic(np.array(sp4[int(i)]).reshape(4, 4), (0, 0, 0, 0), d), 2, d))
        for i in idxs)
    assert min(rep_ent.values()) <= best + 1e-10
    if d == 2:
        assert abs(min(rep_ent.values()) - best) < 1e-10


@pytest.mark.parametrize("d", [2, 3])
def test_bell_pair_is_fully_disentangled(d):
    """SUM (H (x) I)|00> has entropy ln d; the best class brings it to 0."""
    psi = np.zeros(d * d, dtype=complex)
    psi[0] = 1
    u = clifford.SUM_gate(d) @ np.kron(clifford.H_gate(d), np.eye(d))
    psi = u @ psi
    assert abs(_entropy(psi.reshape(d, d)) - np.log(d)) < 1e-12
    ents = [_entropy((q @ psi).reshape(d, d)) for _s, _i, q in clifford.candidates(d)]
    assert abs(ents[0] - np.log(d)) < 1e-12
    assert min(ents) < 1e-12
