"""GCAMPS: psi = C|MPS> with C a mod-d stabilizer tableau (paper Sec. 3, Fig. 3).

* Clifford gate G: C <- G C, tableau only (Sec. 3, top loop of Fig. 3).
* Non-Clifford diagonal gate D on site k (Sec. 3, bottom loop of Fig. 3):
    1. expand D = sum_m c_m Z_k^m (the linear solve of Sec. 3; for a diagonal gate it is the
       discrete Fourier transform c_m = (1/d) sum_j t_j omega^{-m j});
    2. commute through C: C^dag D C = sum_m c_m P^m with P = C^dag Z_k C (Sec. 2.3.1);
    3. apply the d-term MPO sum_m c_m P^m to the MPS over the support span [f, l] of P
       (multi-site operators grow chi by up to a factor d, Sec. 2.4);
    4. compress with QR + truncated SVD over [f, l] (Sec. 2.4).
* Disentangling (Sec. 3): over the bonds of [f, l], try every two-qudit Clifford class Q
  (20 for d = 2, 90 for d = 3), score the entanglement of Q theta, apply the best one to the MPS
  and fold it into the tableau as C~ = C Q^dag.

Readings where the paper is silent (shared with the CUDA library, which implements them in its
own code):
* score: von Neumann entropy (natural log) of the normalised Schmidt spectrum of Q theta
  (score_kind 0); the Renyi-2 entropy -ln sum p^2 (score_kind 1); or the bond-dimension
  criterion of Sec. 4 read as the number of Schmidt weights p above max(1e-12, 4 cutoff^2), ties
  broken by the von Neumann entropy (score_kind 2);
* accept: best score < score of the identity - tie_tol; ties within tie_tol of the minimum go to
  the lowest class index;
* sweeps alternate direction (left to right first, centre starting at f), a split is done at
  every visited bond (with Q = I when nothing is accepted), and the loop stops after a sweep that
  accepts nothing or after max_sweeps sweeps;
* the centre is moved (QR, no truncation) to the nearest site of [f, l] before the MPO.
"""
from __future__ import annotations

import numpy as np

from . import clifford
from .mps import MPS
from .tableau import Tableau
from .weyl import Weyl, omega, tau


def entropy_from_singular_values(s: np.ndarray) -> float:
    p = s.astype(float) ** 2
    tot = p.sum()
    if tot <= 0:
        return 0.0
    p = p / tot
    p = p[p > 0]
    return float(-np.sum(p * np.log(p)))


def renyi2_from_singular_values(s: np.ndarray) -> float:
    """-ln sum p^2 with p = s^2 / sum s^2 (Renyi entropy of order 2)."""
    p = s.astype(float) ** 2
    tot = p.sum()
    if tot <= 0:
        return 0.0
    p = p / tot
    return float(-np.log(np.sum(p * p)))


def weight_rank(s: np.ndarray, cutoff: float) -> int:
    """Number of Schmidt weights p = s^2 / sum s^2 above max(1e-12, 4 cutoff^2)."""
    p = s.astype(float) ** 2
    tot = p.sum()
    if tot <= 0:
        return 0
    return int(np.sum(p / tot > max(1e-12, 4.0 * cutoff * cutoff)))


def expansion_coefficients(phases, d: int) -> np.ndarray:
    """c_m with diag(e^{i phases}) = sum_m c_m Z^m: c_m = (1/d) sum_j e^{i phase_j} omega^{-m j}."""
    t = np.exp(1j * np.asarray(phases, dtype=float))
    w = omega(d)
    return np.array([sum(t[j] * w ** (-m * j) for j in range(d)) / d for m in range(d)])


class GCAMPS:
    def __init__(self, n: int, d: int, chi_max: int, cutoff: float = 1e-14,
                 max_sweeps: int = 8, tie_tol: float = 1e-10, score_kind: int = 0):
        if d not in (2, 3):
            raise ValueError("d must be 2 or 3")
        self.n, self.d = n, d
        self.chi_max, self.cutoff = chi_max, cutoff
        self.max_sweeps, self.tie_tol = max_sweeps, tie_tol
        if score_kind not in (0, 1, 2):
            raise ValueError("score_kind must be 0, 1 or 2")
        self.score_kind = score_kind
        self.tab = Tableau(n, d)
        self.mps = MPS.zero_state(n, d)
        self.span = None
        self.cands = clifford.candidates(d)
        self.decisions = []      # (bond, class index) for every visited bond, in order
        self.discarded = 0.0
        self.last_weyl = None
        self.candidates_scored = 0

    # ---------------------------------------------------------------- Clifford loop
    def apply_clifford(self, sites, images) -> None:
        u = clifford.unitary_from_images(images, len(sites), self.d)
        self.tab.apply_gate(u, sites)

    def apply_gate(self, gate) -> None:
        if hasattr(gate, "sp_index"):
            self.apply_clifford([gate.q0, gate.q1],
                                clifford.random_gate_images(gate.sp_index, gate.shift, self.d))
        else:
            self.apply_nonclifford(gate.site, gate.phases)

    # ------------------------------------------------------------ non-Clifford loop
    def weyl_of_z(self, k: int) -> Weyl:
        return self.tab.conjugate_back(Weyl.single(self.n, self.d, k, "Z"))

    def mpo_tensors(self, p: Weyl, coeffs):
        """MPO of sum_m c_m P^m on the span [f, l] of P, bond dimension d, diagonal in m."""
        d = self.d
        sup = p.support()
        f, l = sup[0], sup[-1]
        powers = [p ** m for m in range(d)]
        ws = []
        if f == l:
            w = np.zeros((1, 1, d, d), dtype=complex)
            for m in range(d):
                w[0, 0] += coeffs[m] * tau(d) ** powers[m].r * powers[m].local_matrix(f)
            return f, l, [w]
        for j in range(f, l + 1):
            if j == f:
                w = np.zeros((1, d, d, d), dtype=complex)
                for m in range(d):
                    w[0, m] = coeffs[m] * tau(d) ** powers[m].r * powers[m].local_matrix(j)
            elif j == l:
                w = np.zeros((d, 1, d, d), dtype=complex)
                for m in range(d):
                    w[m, 0] = powers[m].local_matrix(j)
            else:
                w = np.zeros((d, d, d, d), dtype=complex)
                for m in range(d):
                    w[m, m] = powers[m].local_matrix(j)
            ws.append(w)
        return f, l, ws

    def apply_nonclifford(self, site: int, phases) -> float:
        p = self.weyl_of_z(site)
        self.last_weyl = p
        coeffs = expansion_coefficients(phases, self.d)
        f, l, ws = self.mpo_tensors(p, coeffs)
        self.mps.move_center(min(max(self.mps.oc, f), l))
        self.mps.apply_mpo(ws, f)
        disc = 0.0
        if l > f:
            disc = self.mps.compress(f, l, self.cutoff, self.chi_max)
        self.discarded += disc
        self.span = (f, l)
        return disc

    # ---------------------------------------------------------------- disentangling
    def schmidt_values(self, theta: np.ndarray):
        """Schmidt values of Q theta across (a, s) | (t, b) for every class Q (SVD)."""
        cl, d, _, cr = theta.shape
        t = theta.reshape(cl, d * d, cr)
        out = []
        for _s, _imgs, u in self.cands:
            tq = np.einsum("uv,avb->aub", u, t).reshape(cl * d, d * cr)
            out.append(np.linalg.svd(tq, compute_uv=False))
        return out

    def score_bond(self, theta: np.ndarray) -> np.ndarray:
        """Von Neumann entropy of Q theta for every class Q (Schmidt values by SVD)."""
        self.candidates_scored += len(self.cands)
        return np.array([entropy_from_singular_values(sv_) for sv_ in self.schmidt_values(theta)])

    def score_keys(self, theta: np.ndarray):
        """Scores of every class under score_kind: an array of entropies (kinds 0 and 1), or
        (rank, entropy) pairs (kind 2)."""
        svs = self.schmidt_values(theta)
        self.candidates_scored += len(self.cands)
        if self.score_kind == 1:
            return np.array([renyi2_from_singular_values(x) for x in svs])
        vn = np.array([entropy_from_singular_values(x) for x in svs])
        if self.score_kind == 0:
            return vn
        return np.array([weight_rank(x, self.cutoff) for x in svs]), vn

    def choose(self, scores) -> int:
        """Class to apply: the lowest index within tie_tol of the best score, if it beats the
        identity (class 0) by more than tie_tol.  Kind 2 compares ranks first; the entropies
        decide among the classes of the smallest rank and between equal ranks."""
        if isinstance(scores, tuple):
            rank, vn = scores
            rmin = int(np.min(rank))
            sel = rank == rmin
            best = float(np.min(vn[sel]))
            k = int(np.nonzero(sel & (vn <= best + self.tie_tol))[0][0])
            if rank[k] < rank[0] or vn[k] < vn[0] - self.tie_tol:
                return k
            return 0
        best = float(np.min(scores))
        k = int(np.nonzero(scores <= best + self.tie_tol)[0][0])
        if scores[k] < scores[0] - self.tie_tol:
            return k
        return 0

    def visit(self, i: int, left_to_right: bool, forced=None) -> int:
        theta = self.mps.theta(i)
        if forced is None:
            k = self.choose(self.score_keys(theta))
        else:
            k = forced
        if k:
            _s, imgs, u = self.cands[k]
            cl, d, _, cr = theta.shape
            theta = np.einsum("uv,avb->aub", u, theta.reshape(cl, d * d, cr)).reshape(cl, d, d, cr)
            self.tab.apply_gate_right_inverse(u, [i, i + 1])
        self.discarded += self.mps.split(i, theta, left_to_right, self.cutoff, self.chi_max)
        self.decisions.append((i, k))
        return k

    def disentangle(self, forced=None):
        """Alternating sweeps over the bonds of the last span.  ``forced``: optional list of
        class indices to use instead of scoring (replay), consumed in visit order."""
        if self.span is None:
            return {"sweeps": 0, "accepted": 0}
        f, l = self.span
        if l == f:
            return {"sweeps": 0, "accepted": 0}
        feed = None if forced is None else iter(forced)
        sweeps = accepted = 0
        while sweeps < self.max_sweeps:
            ltr = sweeps % 2 == 0
            self.mps.move_center(f if ltr else l)
            bonds = range(f, l) if ltr else range(l - 1, f - 1, -1)
            acc = 0
            for i in bonds:
                k = self.visit(i, ltr, None if feed is None else next(feed))
                acc += k != 0
            sweeps += 1
            accepted += acc
            if acc == 0:
                break
        return {"sweeps": sweeps, "accepted": accepted}

    # ---------------------------------------------------------------------- readouts
    def expect_weyl(self, x, z) -> complex:
        """<psi| W(x, z) |psi> = <M| C^dag W C |M> (Sec. 3)."""
        w = Weyl(0, x, z, self.d)
        p = self.tab.conjugate_back(w)
        ops = {j: p.local_matrix(j) for j in p.support()}
        return complex(tau(self.d) ** p.r * self.mps.expect_local(ops))

    def statevector(self, seed: int = 12345) -> np.ndarray:
        """Dense C|M> for small n, up to a global phase.

        C|x> = prod_j D_j^{x_j} C|0>, and C|0> is the common +1 eigenvector of the stabilizer
        rows S_j; it is found by projecting a fixed random vector with prod_j (1/d) sum_m S_j^m.
        """
        from . import statevector as sv
        n, d = self.n, self.d
        rng = np.random.default_rng(seed)
        v = rng.standard_normal(d ** n) + 1j * rng.standard_normal(d ** n)
        for j in range(n):
            acc = np.zeros_like(v)
            cur = v
            for _m in range(d):
                acc = acc + cur
                cur = sv.apply_weyl(cur, self.tab.rows[j], n, d)
            v = acc / d
        v = v / np.linalg.norm(v)
        m = self.mps.to_dense()
        out = np.zeros(d ** n, dtype=complex)
        for xi in range(d ** n):
            if m[xi] == 0:
                continue
            w = Weyl.identity(n, d)
            for j in range(n):
                xj = (xi // d ** (n - 1 - j)) % d
                w = w * (self.tab.rows[n + j] ** xj)
            out += m[xi] * sv.apply_weyl(v, w, n, d)
        return out
