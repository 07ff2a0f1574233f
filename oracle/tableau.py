"""Mod-d stabilizer tableau of the Clifford C (paper Sec. 2.2, Sec. 2.3, Sec. 2.3.1).

Layout (the qubit tableau of Sec. 2.2 with entries in Z_d, Sec. 2.3): 2n rows, each a Weyl
operator with phase.  Rows 0..n-1 are the stabilizers S_j = C Z_j C^dag, rows n..2n-1 the
destabilizers D_j = C X_j C^dag.  Exponent columns x_0..x_{n-1} | z_0..z_{n-1}; the phase is
kept mod 2d in units of tau = exp(i pi/d) (Sec. 2.3 puts it in Z_d; even d needs tau).

* ``apply_gate``: the conjugation principle S' = U S U^dag (Sec. 2.2) row by row.  The local
  part of each row on the gate's sites is conjugated as a dense matrix and snapped back to a
  Weyl operator; nothing here composes the update rules of Table 1 symbolically.
* ``decompose``: P = c prod_j S_j^{s_j} D_j^{d_j} by Gaussian elimination over F_d, then the
  phase c by explicitly multiplying the rows (Sec. 2.3.1).
* ``conjugate_back``: C^dag P C = c prod_j Z_j^{s_j} X_j^{d_j}, the operator the non-Clifford
  step applies to the MPS (Sec. 3).
"""
from __future__ import annotations

import numpy as np

from . import clifford
from .weyl import Weyl


def _inv_mod(a: int, d: int) -> int:
    """Inverse in F_d (d prime): a^{d-2}."""
    return pow(int(a) % d, d - 2, d)


class Tableau:
    def __init__(self, n: int, d: int):
        self.n = n
        self.d = d
        self.rows = [Weyl.single(n, d, j, "Z") for j in range(n)] + \
                    [Weyl.single(n, d, j, "X") for j in range(n)]

    def copy(self) -> "Tableau":
        t = Tableau.__new__(Tableau)
        t.n, t.d = self.n, self.d
        t.rows = [r.copy() for r in self.rows]
        return t

    # -- Clifford update (conjugation principle)
    def apply_gate(self, u: np.ndarray, sites) -> None:
        """C <- U C: every row R becomes U R U^dag; only the factors on ``sites`` change."""
        d = self.d
        k = len(sites)
        cache = {}
        for row in self.rows:
            key = tuple(int(row.x[s]) for s in sites) + tuple(int(row.z[s]) for s in sites)
            if key not in cache:
                loc = Weyl(0, key[:k], key[k:], d)
                cache[key] = clifford.snap(u @ loc.dense() @ u.conj().T, k, d)
            img = cache[key]
            row.r = (row.r + img.r) % (2 * d)
            for i, s in enumerate(sites):
                row.x[s] = img.x[i]
                row.z[s] = img.z[i]

    def apply_gate_right_inverse(self, u: np.ndarray, sites) -> None:
        """C <- C U^dag (the fold C~ = C Q^dag of Sec. 3).

        Row j is C W_j C^dag with W_j = Z_j or X_j.  It becomes C (U^dag W_j U) C^dag.  For W_j
        off ``sites`` this is unchanged; on ``sites``, U^dag W_j U (found by dense conjugation)
        is tau^r prod_q X_q^{a_q} Z_q^{b_q}, so the new row is tau^r prod_q D_q^{a_q} S_q^{b_q},
        a product of old rows (X_q -> D_q, Z_q -> S_q)."""
        d, n = self.d, self.n
        k = len(sites)
        old = [r.copy() for r in self.rows]
        for i, s in enumerate(sites):
            for kind, row_index in (("Z", s), ("X", n + s)):
                loc = Weyl.single(k, d, i, kind)
                img = clifford.snap(u.conj().T @ loc.dense() @ u, k, d)
                acc = Weyl(img.r, np.zeros(n), np.zeros(n), d)
                for q, sq in enumerate(sites):
                    acc = acc * (old[n + sq] ** int(img.x[q]))
                    acc = acc * (old[sq] ** int(img.z[q]))
                self.rows[row_index] = acc

    # -- Sec. 2.3.1
    def decompose(self, p: Weyl):
        """Return (coefficients c of length 2n, phase exponent c0) with
        P = tau^{c0} prod_{j=0}^{n-1} S_j^{c_j} D_j^{c_{n+j}}, product taken in increasing j,
        S_j before D_j.  Gaussian elimination over F_d on  sum_k c_k v_k = v_P."""
        n, d = self.n, self.d
        m = 2 * n
        a = np.zeros((m, m + 1), dtype=np.int64)
        for k, row in enumerate(self.rows):
            a[:n, k] = row.x
            a[n:, k] = row.z
        a[:n, m] = p.x
        a[n:, m] = p.z
        a %= d
        piv_row = 0
        pivots = []
        for col in range(m):
            pr = None
            for r in range(piv_row, m):
                if a[r, col] % d:
                    pr = r
                    break
            if pr is None:
                continue
            a[[piv_row, pr]] = a[[pr, piv_row]]
            a[piv_row] = (a[piv_row] * _inv_mod(a[piv_row, col], d)) % d
            for r in range(m):
                if r != piv_row and a[r, col]:
                    a[r] = (a[r] - a[r, col] * a[piv_row]) % d
            pivots.append(col)
            piv_row += 1
        if len(pivots) != m:
            raise ValueError("tableau rows are not independent")
        coeff = np.zeros(m, dtype=np.int64)
        for r, col in enumerate(pivots):
            coeff[col] = a[r, m]
        prod = Weyl.identity(n, d)
        for j in range(n):
            prod = prod * (self.rows[j] ** int(coeff[j]))
            prod = prod * (self.rows[n + j] ** int(coeff[n + j]))
        if not (np.array_equal(prod.x, p.x) and np.array_equal(prod.z, p.z)):
            raise AssertionError("elimination produced a wrong product")
        c0 = (p.r - prod.r) % (2 * d)
        return coeff, c0

    def conjugate_back(self, p: Weyl) -> Weyl:
        """C^dag P C = tau^{c0} prod_j Z_j^{c_j} X_j^{c_{n+j}} (same product order as
        ``decompose``), since C^dag S_j C = Z_j and C^dag D_j C = X_j."""
        n, d = self.n, self.d
        coeff, c0 = self.decompose(p)
        out = Weyl(c0, np.zeros(n), np.zeros(n), d)
        for j in range(n):
            out = out * (Weyl.single(n, d, j, "Z") ** int(coeff[j]))
            out = out * (Weyl.single(n, d, j, "X") ** int(coeff[n + j]))
        return out

    # -- views
    def exps_phase(self):
        """(uint8 [2n][2n] exponents x|z, uint8 [2n] phase mod 2d)."""
        n = self.n
        e = np.zeros((2 * n, 2 * n), dtype=np.uint8)
        ph = np.zeros(2 * n, dtype=np.uint8)
        for k, row in enumerate(self.rows):
            e[k, :n] = row.x
            e[k, n:] = row.z
            ph[k] = row.r
        return e, ph

    def inverse_rows(self):
        """C^dag Z_j C (rows 0..n-1) and C^dag X_j C (rows n..2n-1)."""
        n, d = self.n, self.d
        out = [self.conjugate_back(Weyl.single(n, d, j, "Z")) for j in range(n)]
        out += [self.conjugate_back(Weyl.single(n, d, j, "X")) for j in range(n)]
        return out
