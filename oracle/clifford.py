"""Qudit Clifford gates, Cliffords from generator images, Sp(4, F_d) and the disentangler set.

Paper: gate definitions and Table 1 (Sec. 2.3); the exhaustive two-qudit disentangler search
over 20 (d = 2) / 90 (d = 3) entangling classes (Sec. 3); the class construction by reducing
every two-qudit Clifford to a canonical form under single-qudit gates (Sec. 3.1).

Conventions of this oracle (each one a reading; the CUDA library implements the same ones in
its own code):

* A Clifford on ``nq`` qudits is given by the images of the generators in the order
  X_0, Z_0, X_1, Z_1, ... as Weyl operators with phase (``weyl.Weyl``).
* Its symplectic matrix ``S`` has column k = exponent vector of image k in the coordinates
  (x_0, z_0, x_1, z_1, ...); the symplectic form is Lambda of ``weyl.symplectic_form``.
* "Standard phase" of an exponent vector: tau^0 for odd d; tau^{sum_q x_q z_q} for d = 2, which
  makes every local factor Hermitian (Y = tau XZ, Sec. 2.3).
* The random circuit gate (sp_index, shift) is  W(shift) U_S  where U_S maps each generator to
  the standard-phase Weyl operator of its column of S (the sp_index-th matrix of Sp(4, F_d) in
  lexicographic order of the row-major flattening of S).
* The unitary of a Clifford given by images: U|0..0> = the common +1 eigenvector v of the images
  of Z_q, with its first non-negligible entry made real and positive; U|y> = prod_q Ximg_q^{y_q} v.
"""
from __future__ import annotations

import functools
import itertools

import numpy as np

from .weyl import Weyl, X, Z, omega, tau, symplectic_form


# --------------------------------------------------------------------------- gates (Sec. 2.3)

def H_gate(d: int) -> np.ndarray:
    """H_d = d^{-1/2} sum_{i,j} omega^{ij} |j><i|."""
    w = omega(d)
    m = np.zeros((d, d), dtype=complex)
    for i in range(d):
        for j in range(d):
            m[j, i] += w ** (i * j)
    return m / np.sqrt(d)


def S_gate(d: int) -> np.ndarray:
    """S_d = sum_j omega^{j(j-1)/2}|j><j| for odd d; sum_j tau^{j^2}|j><j| for even d."""
    if d % 2:
        return np.diag([omega(d) ** (j * (j - 1) // 2) for j in range(d)]).astype(complex)
    return np.diag([tau(d) ** (j * j) for j in range(d)]).astype(complex)


def SUM_gate(d: int) -> np.ndarray:
    """SUM_d |i, j> = |i, i + j mod d>, first factor the control (most significant)."""
    m = np.zeros((d * d, d * d), dtype=complex)
    for i in range(d):
        for j in range(d):
            m[i * d + (i + j) % d, i * d + j] = 1.0
    return m


def diag_gate(phases) -> np.ndarray:
    return np.diag(np.exp(1j * np.asarray(phases, dtype=float)))


# ------------------------------------------------------------- Weyl basis and conjugation

@functools.lru_cache(maxsize=None)
def _weyl_basis(nq: int, d: int):
    """All d^{2 nq} phase-free strings: (stack of dense matrices, list of (x, z))."""
    mats, labels = [], []
    for digits in itertools.product(range(d), repeat=2 * nq):
        x = np.array(digits[0::2], dtype=np.int64)
        z = np.array(digits[1::2], dtype=np.int64)
        mats.append(Weyl(0, x, z, d).dense())
        labels.append((x, z))
    return np.array(mats), labels


def snap(m: np.ndarray, nq: int, d: int, tol: float = 1e-10) -> Weyl:
    """Write a dense matrix as tau^r W(x, z) (the strings are orthogonal under
    tr(A^dag B)/d^nq, so one overlap has modulus one).  Raises if m is no such operator."""
    mats, labels = _weyl_basis(nq, d)
    ov = np.einsum("kij,ij->k", mats.conj(), m) / (d ** nq)
    k = int(np.argmax(np.abs(ov)))
    if abs(abs(ov[k]) - 1.0) > 1e-8:
        raise ValueError("not a Weyl operator with phase")
    r = int(round(np.angle(ov[k]) / (np.pi / d))) % (2 * d)
    x, z = labels[k]
    w = Weyl(r, x, z, d)
    if np.max(np.abs(w.dense() - m)) > tol:
        raise ValueError("phase is not a power of tau")
    return w


def generators(nq: int, d: int):
    """X_0, Z_0, X_1, Z_1, ... as Weyl operators."""
    out = []
    for q in range(nq):
        out.append(Weyl.single(nq, d, q, "X"))
        out.append(Weyl.single(nq, d, q, "Z"))
    return out


def images_by_conjugation(u: np.ndarray, nq: int, d: int):
    """Images U g U^dag of the generators, found numerically and snapped (conjugation
    principle S' = U S U^dag, Sec. 2.2)."""
    return [snap(u @ g.dense() @ u.conj().T, nq, d) for g in generators(nq, d)]


def unitary_from_images(images, nq: int, d: int) -> np.ndarray:
    """The Clifford whose generator images are ``images`` (X_0, Z_0, X_1, Z_1, ...).

    U|0..0> = v, the common +1 eigenvector of the Z-images (phase: first entry with modulus
    above 1e-8 made real positive); U|y> = prod_q Ximg_q^{y_q} v, site 0 most significant.
    """
    dim = d ** nq
    proj = np.eye(dim, dtype=complex)
    for q in range(nq):
        zq = images[2 * q + 1].dense()
        acc = np.zeros((dim, dim), dtype=complex)
        p = np.eye(dim, dtype=complex)
        for _m in range(d):
            acc += p
            p = p @ zq
        proj = proj @ (acc / d)
    norms = np.linalg.norm(proj, axis=0)
    v = proj[:, int(np.argmax(norms))]
    v = v / np.linalg.norm(v)
    i0 = int(np.nonzero(np.abs(v) > 1e-8)[0][0])
    v = v * (abs(v[i0]) / v[i0])
    u = np.zeros((dim, dim), dtype=complex)
    xs = [images[2 * q].dense() for q in range(nq)]
    for y in range(dim):
        digits = [(y // d ** (nq - 1 - q)) % d for q in range(nq)]
        col = v.copy()
        for q in range(nq):
            for _ in range(digits[q]):
                col = xs[q] @ col
        u[:, y] = col
    return u


# --------------------------------------------------------------------- symplectic matrices

def std_phase(x, z, d: int) -> int:
    """tau exponent making tau^r W(x, z) the standard representative: 0 for odd d,
    sum_q x_q z_q for d = 2 (each factor then Hermitian)."""
    if d % 2:
        return 0
    return int(np.sum(np.asarray(x) * np.asarray(z))) % (2 * d)


def symplectic_of_images(images, nq: int, d: int) -> np.ndarray:
    s = np.zeros((2 * nq, 2 * nq), dtype=np.int64)
    for k, w in enumerate(images):
        s[0::2, k] = w.x
        s[1::2, k] = w.z
    return s


def _lam_vec(u, v, d):
    """Lambda on interleaved coordinates (x_0, z_0, x_1, z_1, ...)."""
    u = np.asarray(u)
    v = np.asarray(v)
    return symplectic_form(u[0::2], u[1::2], v[0::2], v[1::2], d)


def is_symplectic(s: np.ndarray, d: int) -> bool:
    m = s.shape[0]
    e = np.eye(m, dtype=np.int64)
    for i in range(m):
        for j in range(m):
            if _lam_vec(s[:, i], s[:, j], d) != _lam_vec(e[:, i], e[:, j], d):
                return False
    return True


@functools.lru_cache(maxsize=None)
def sp_group(nq: int, d: int):
    """All symplectic (2nq x 2nq) matrices over F_d as row-major tuples, sorted
    lexicographically.  Built column by column: each new column must be non-zero and have the
    generator commutation phases Lambda(e_i, e_k) with every earlier column."""
    m = 2 * nq
    vecs = [np.array(v, dtype=np.int64) for v in itertools.product(range(d), repeat=m)]
    nv = len(vecs)
    lam = np.array([[_lam_vec(u, v, d) for v in vecs] for u in vecs], dtype=np.int64)
    e = np.eye(m, dtype=np.int64)
    target = [[_lam_vec(e[:, i], e[:, j], d) for j in range(m)] for i in range(m)]
    out = []

    def extend(cols):
        k = len(cols)
        if k == m:
            s = np.stack([vecs[c] for c in cols], axis=1)
            out.append(tuple(int(a) for a in s.reshape(-1)))
            return
        ok = np.ones(nv, dtype=bool)
        ok[0] = False  # the zero vector
        for i, c in enumerate(cols):
            ok &= lam[c] == target[i][k]
        for v in np.nonzero(ok)[0]:
            extend(cols + [int(v)])

    extend([])
    out.sort()
    return out


def sp4_matrix(index: int, d: int) -> np.ndarray:
    return np.array(sp_group(2, d)[index], dtype=np.int64).reshape(4, 4)


def images_from_symplectic(s: np.ndarray, shift, d: int):
    """Images of X_0, Z_0, X_1, Z_1 for the gate W(shift) U_S (see module docstring):
    image k = tau^{std(v_k) + 2 Lambda(shift, v_k)} W(v_k), v_k = column k of S."""
    shift = np.asarray(shift, dtype=np.int64)
    nq = s.shape[0] // 2
    out = []
    for k in range(2 * nq):
        v = s[:, k]
        r = std_phase(v[0::2], v[1::2], d) + 2 * _lam_vec(shift, v, d)
        out.append(Weyl(r, v[0::2], v[1::2], d))
    return out


def random_gate_images(sp_index: int, shift, d: int):
    return images_from_symplectic(sp4_matrix(sp_index, d), shift, d)


# ------------------------------------------------------------ disentangler classes (Sec. 3.1)

@functools.lru_cache(maxsize=None)
def candidates(d: int):
    """The two-qudit Clifford classes modulo single-qudit Cliffords applied after them.

    Classes are {(L_0 (+) L_1) S : L_q in Sp(2, F_d)} (local gates after the entangler leave the
    bond entanglement unchanged).  Representative: the lexicographically smallest member,
    except that the class of the identity is represented by the identity and listed first;
    the rest follow in representative order.  Each entry: (S, images with standard phases,
    9x9 or 4x4 unitary).  Count: d^2 (d^2 + 1) = 20 (d = 2), 90 (d = 3), as Sec. 3 states.
    """
    sp4 = sp_group(2, d)
    sp2 = [np.array(t, dtype=np.int64).reshape(2, 2) for t in sp_group(1, d)]
    blocks = []
    for a in sp2:
        for b in sp2:
            m = np.zeros((4, 4), dtype=np.int64)
            m[0:2, 0:2] = a
            m[2:4, 2:4] = b
            blocks.append(m)
    blocks = np.array(blocks)
    assigned = {}
    reps = []
    for t in sp4:
        if t in assigned:
            continue
        s = np.array(t, dtype=np.int64).reshape(4, 4)
        members = (blocks @ s) % d
        cid = len(reps)
        for mm in members:
            assigned[tuple(int(a) for a in mm.reshape(-1))] = cid
        reps.append(s)
    ident = tuple(int(a) for a in np.eye(4, dtype=np.int64).reshape(-1))
    id_class = assigned[ident]
    order = [id_class] + [c for c in range(len(reps)) if c != id_class]
    out = []
    for c in order:
        s = np.eye(4, dtype=np.int64) if c == id_class else reps[c]
        imgs = images_from_symplectic(s, (0, 0, 0, 0), d)
        out.append((s, imgs, unitary_from_images(imgs, 2, d)))
    return out
