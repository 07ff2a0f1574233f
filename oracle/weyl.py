"""Generalised Pauli (Weyl) operators over Z_d (paper Sec. 2.3).

Definitions (Sec. 2.3): omega = exp(2 pi i / d), X|j> = |j+1 mod d>, Z|j> = omega^j |j>,
XZ = omega^{-1} ZX; for even d the Y operator carries tau = omega^{1/2}.

Representation used throughout the oracle: a Weyl operator with phase is a triple
(r, x, z) meaning  tau^r  (x)_j X_j^{x_j} Z_j^{z_j}  with tau = exp(i pi / d), r taken mod 2d,
x_j, z_j in Z_d.  Keeping the phase in units of tau (not omega) is needed for d = 2 (Y = tau XZ)
and costs nothing for odd d, where only even r occur.

Products are computed the slow, obvious way: by commuting Z^{z} past X^{x'} on each site,
Z^z X^x' = omega^{z x'} X^x' Z^z.
"""
from __future__ import annotations

import numpy as np


def omega(d: int) -> complex:
    return np.exp(2j * np.pi / d)


def tau(d: int) -> complex:
    return np.exp(1j * np.pi / d)


def X(d: int) -> np.ndarray:
    """X|j> = |j+1 mod d>  (column j has a 1 in row j+1)."""
    m = np.zeros((d, d), dtype=complex)
    for j in range(d):
        m[(j + 1) % d, j] = 1.0
    return m


def Z(d: int) -> np.ndarray:
    """Z|j> = omega^j |j>."""
    return np.diag([omega(d) ** j for j in range(d)]).astype(complex)


class Weyl:
    """tau^r (x)_j X_j^{x_j} Z_j^{z_j} on len(x) qudits."""

    __slots__ = ("r", "x", "z", "d")

    def __init__(self, r, x, z, d):
        self.d = d
        self.r = int(r) % (2 * d)
        self.x = np.asarray(x, dtype=np.int64) % d
        self.z = np.asarray(z, dtype=np.int64) % d

    @property
    def n(self) -> int:
        return len(self.x)

    @staticmethod
    def identity(n: int, d: int) -> "Weyl":
        return Weyl(0, np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.int64), d)

    @staticmethod
    def single(n: int, d: int, site: int, kind: str, power: int = 1) -> "Weyl":
        x = np.zeros(n, dtype=np.int64)
        z = np.zeros(n, dtype=np.int64)
        if kind == "X":
            x[site] = power
        elif kind == "Z":
            z[site] = power
        else:
            raise ValueError(kind)
        return Weyl(0, x, z, d)

    def copy(self) -> "Weyl":
        return Weyl(self.r, self.x.copy(), self.z.copy(), self.d)

    def __mul__(self, other: "Weyl") -> "Weyl":
        """(tau^r W(x,z)) (tau^r' W(x',z')): on each site X^x Z^z X^x' Z^z' =
        omega^{z x'} X^{x+x'} Z^{z+z'}, and omega = tau^2."""
        d = self.d
        assert other.d == d and other.n == self.n
        r = self.r + other.r + 2 * int(np.sum(self.z * other.x))
        return Weyl(r, self.x + other.x, self.z + other.z, d)

    def __pow__(self, m: int) -> "Weyl":
        out = Weyl.identity(self.n, self.d)
        for _ in range(m):
            out = out * self
        return out

    def __eq__(self, other) -> bool:
        return (self.d == other.d and self.r == other.r
                and np.array_equal(self.x, other.x) and np.array_equal(self.z, other.z))

    def __repr__(self) -> str:
        return f"Weyl(r={self.r}, x={self.x.tolist()}, z={self.z.tolist()}, d={self.d})"

    def support(self):
        """Sites where the operator is not the identity."""
        return [j for j in range(self.n) if self.x[j] or self.z[j]]

    def local_matrix(self, j: int) -> np.ndarray:
        """X^{x_j} Z^{z_j} as a d x d matrix (no phase)."""
        d = self.d
        return np.linalg.matrix_power(X(d), int(self.x[j])) @ np.linalg.matrix_power(Z(d), int(self.z[j]))

    def dense(self) -> np.ndarray:
        """Full d^n x d^n matrix, site 0 the most significant tensor factor."""
        m = np.array([[1.0 + 0j]])
        for j in range(self.n):
            m = np.kron(m, self.local_matrix(j))
        return tau(self.d) ** self.r * m


def symplectic_form(u_x, u_z, v_x, v_z, d: int) -> int:
    """Lambda(u, v) with W(u) W(v) = omega^{Lambda(u, v)} W(v) W(u):
    Lambda = sum_j z_j(u) x_j(v) - x_j(u) z_j(v)  (mod d)."""
    u_x, u_z, v_x, v_z = (np.asarray(a, dtype=np.int64) for a in (u_x, u_z, v_x, v_z))
    return int(np.sum(u_z * v_x) - np.sum(u_x * v_z)) % d


def snap_to_weyl(m: np.ndarray, n: int, d: int, tol: float = 1e-10) -> Weyl:
    """Identify a dense matrix as tau^r W(x, z) by its overlaps with every Weyl string.

    The d^{2n} strings W(v) are orthogonal under <A, B> = tr(A^dag B) / d^n, so exactly one
    overlap has modulus 1 when m is a Weyl operator with phase.  Raises if it is not.
    """
    dim = d ** n
    best = None
    for code in range(d ** (2 * n)):
        digits = []
        c = code
        for _ in range(2 * n):
            digits.append(c % d)
            c //= d
        x = np.array(digits[:n], dtype=np.int64)
        z = np.array(digits[n:], dtype=np.int64)
        w = Weyl(0, x, z, d).dense()
        ov = np.trace(w.conj().T @ m) / dim
        if abs(ov) > 0.5:
            best = (ov, x, z)
            break
    if best is None:
        raise ValueError("matrix is not a Weyl operator")
    ov, x, z = best
    r = int(round(np.angle(ov) / (np.pi / d))) % (2 * d)
    cand = Weyl(r, x, z, d)
    err = np.max(np.abs(cand.dense() - m))
    if err > tol:
        raise ValueError(f"matrix is not tau^r W(v): residual {err}")
    return cand
