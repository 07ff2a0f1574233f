"""Matrix product states (paper Sec. 2.4, Eq. mps) with an explicit orthogonality centre.

Site tensors A[j] have shape (chi_{j-1}, d, chi_j), chi_{-1} = chi_{n-1} = 1; the state is
sum_s A[0]_{s_0} ... A[n-1]_{s_{n-1}} |s_0 ... s_{n-1}>, site 0 most significant.

``oc`` is the orthogonality centre: sites left of it are left-orthonormal, sites right of it
right-orthonormal, so the singular values of a bond next to the centre are its Schmidt values.

Truncation (Sec. 2.4 keeps "a fixed number of singular values"; the reading used here): keep the
singular values s_i > cutoff * s_0, at most chi_max of them and at least one, and renormalise
the kept ones to unit norm.  The discarded weight is sum of the dropped s_i^2.

Library steps used as primitives: numpy.linalg.qr (reduced) and numpy.linalg.svd.
"""
from __future__ import annotations

import numpy as np


def truncation_rank(s: np.ndarray, cutoff: float, chi_max: int) -> int:
    if len(s) == 0 or s[0] <= 0:
        return 1
    keep = int(np.count_nonzero(s > cutoff * s[0]))
    return max(1, min(keep, chi_max))


class MPS:
    def __init__(self, tensors, d: int, oc: int = 0):
        self.A = [np.asarray(t, dtype=complex) for t in tensors]
        self.d = d
        self.oc = oc

    @staticmethod
    def zero_state(n: int, d: int) -> "MPS":
        ts = []
        for _ in range(n):
            t = np.zeros((1, d, 1), dtype=complex)
            t[0, 0, 0] = 1.0
            ts.append(t)
        return MPS(ts, d, 0)

    @property
    def n(self) -> int:
        return len(self.A)

    def bond_dims(self):
        return [self.A[j].shape[2] for j in range(self.n - 1)]

    def copy(self) -> "MPS":
        return MPS([a.copy() for a in self.A], self.d, self.oc)

    # -- centre moves (no truncation; reduced QR keeps min(rows, cols) directions)
    def _move_right(self):
        j = self.oc
        a = self.A[j]
        cl, d, cr = a.shape
        q, r = np.linalg.qr(a.reshape(cl * d, cr))
        k = q.shape[1]
        self.A[j] = q.reshape(cl, d, k)
        self.A[j + 1] = np.einsum("ab,bsc->asc", r, self.A[j + 1])
        self.oc = j + 1

    def _move_left(self):
        j = self.oc
        a = self.A[j]
        cl, d, cr = a.shape
        q, r = np.linalg.qr(a.reshape(cl, d * cr).conj().T)
        k = q.shape[1]
        self.A[j] = q.conj().T.reshape(k, d, cr)
        self.A[j - 1] = np.einsum("asb,bc->asc", self.A[j - 1], r.conj().T)
        self.oc = j - 1

    def move_center(self, target: int) -> None:
        while self.oc < target:
            self._move_right()
        while self.oc > target:
            self._move_left()

    # -- operators
    def apply_mpo(self, ws, f: int) -> None:
        """Contract MPO tensors W[k] (shape (D_l, D_r, d_out, d_in)) onto sites f, f+1, ...
        A'[(a, mu), s, (b, nu)] = sum_{s'} W[mu, nu, s, s'] A[a, s', b]."""
        for k, w in enumerate(ws):
            j = f + k
            a = self.A[j]
            cl, d, cr = a.shape
            dl, dr = w.shape[0], w.shape[1]
            t = np.einsum("mnst,atb->amsbn", w, a)
            self.A[j] = t.reshape(cl * dl, d, cr * dr)

    def compress(self, f: int, l: int, cutoff: float, chi_max: int) -> float:
        """Canonicalise [f, l] left to right with QR starting at f (centre ends at l), then
        truncate every bond l-1..f right to left with SVD (centre ends at f).  Requires
        f <= oc <= l on entry with everything outside [f, l] canonical; the tensors inside
        [f, l] may be anything (an MPO has just been applied there).  Returns the discarded
        weight."""
        assert f <= self.oc <= l
        self.oc = f
        self.move_center(l)
        disc = 0.0
        for j in range(l, f, -1):
            a = self.A[j]
            cl, d, cr = a.shape
            u, s, vh = np.linalg.svd(a.reshape(cl, d * cr), full_matrices=False)
            k = truncation_rank(s, cutoff, chi_max)
            disc += float(np.sum(s[k:] ** 2))
            sk = s[:k] / np.linalg.norm(s[:k])
            self.A[j] = vh[:k].reshape(k, d, cr)
            self.A[j - 1] = np.einsum("asb,bc->asc", self.A[j - 1], u[:, :k] * sk[None, :])
            self.oc = j - 1
        return disc

    def theta(self, i: int) -> np.ndarray:
        """Two-site tensor of bond i: (chi_{i-1}, d, d, chi_{i+1})."""
        return np.einsum("asb,btc->astc", self.A[i], self.A[i + 1])

    def split(self, i: int, theta: np.ndarray, centre_right: bool, cutoff: float, chi_max: int) -> float:
        """Replace sites i, i+1 by the truncated SVD of theta[(a,s),(t,b)].  centre_right: the
        left factor is U (left-orthonormal) and the centre moves to i+1; else the right factor
        is V^dag and the centre moves to i."""
        cl, d, _, cr = theta.shape
        u, s, vh = np.linalg.svd(theta.reshape(cl * d, d * cr), full_matrices=False)
        k = truncation_rank(s, cutoff, chi_max)
        disc = float(np.sum(s[k:] ** 2))
        sk = s[:k] / np.linalg.norm(s[:k])
        if centre_right:
            self.A[i] = u[:, :k].reshape(cl, d, k)
            self.A[i + 1] = (sk[:, None] * vh[:k]).reshape(k, d, cr)
            self.oc = i + 1
        else:
            self.A[i] = (u[:, :k] * sk[None, :]).reshape(cl, d, k)
            self.A[i + 1] = vh[:k].reshape(k, d, cr)
            self.oc = i
        return disc

    # -- readouts
    def to_dense(self) -> np.ndarray:
        v = self.A[0].reshape(self.d, -1)
        for j in range(1, self.n):
            a = self.A[j]
            v = np.einsum("xa,asb->xsb", v, a).reshape(-1, a.shape[2])
        return v.reshape(-1)

    def expect_local(self, ops) -> complex:
        """<M| (x)_j ops[j] |M> by transfer matrices (ops: dict site -> d x d)."""
        e = np.ones((1, 1), dtype=complex)
        for j, a in enumerate(self.A):
            op = ops.get(j)
            b = a if op is None else np.einsum("st,atb->asb", op, a)
            e = np.einsum("xy,xsa,ysb->ab", e, a.conj(), b)
        return complex(e[0, 0])

    def norm(self) -> float:
        return float(np.sqrt(abs(self.expect_local({}))))

    def schmidt_values(self, i: int) -> np.ndarray:
        """Schmidt values across bond i (computed on a canonicalised copy)."""
        m = self.copy()
        m.move_center(i)
        a = m.A[i]
        cl, d, cr = a.shape
        return np.linalg.svd(a.reshape(cl * d, cr), compute_uv=False)
