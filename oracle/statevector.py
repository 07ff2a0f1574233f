"""Dense state-vector simulation of qudit circuits (paper Sec. 2.1).

The state of n qudits is a vector of d^n amplitudes; site 0 is the most significant digit of
the basis index (index = sum_j s_j d^{n-1-j}).  Gates act by contraction with the tensor axes
of the sites they touch.  This is the exactness anchor: with no truncation GCAMPS must
reproduce it (Sec. 3, psi = C|MPS>), up to the global phase that a Clifford given by its
generator images leaves undefined.
"""
from __future__ import annotations

import numpy as np

from . import clifford
from .weyl import Weyl, tau


def zero_state(n: int, d: int) -> np.ndarray:
    psi = np.zeros(d ** n, dtype=complex)
    psi[0] = 1.0
    return psi


def apply_gate(psi: np.ndarray, u: np.ndarray, sites, n: int, d: int) -> np.ndarray:
    """Apply a k-site gate (d^k x d^k, first listed site most significant) to psi."""
    k = len(sites)
    t = psi.reshape((d,) * n)
    g = u.reshape((d,) * (2 * k))
    t = np.tensordot(g, t, axes=(list(range(k, 2 * k)), list(sites)))
    t = np.moveaxis(t, list(range(k)), list(sites))
    return t.reshape(-1)


def apply_weyl(psi: np.ndarray, w: Weyl, n: int, d: int) -> np.ndarray:
    out = psi
    for j in range(n):
        if w.x[j] or w.z[j]:
            out = apply_gate(out, w.local_matrix(j), [j], n, d)
    return tau(d) ** w.r * out


def expect_weyl(psi: np.ndarray, w: Weyl, n: int, d: int) -> complex:
    return complex(np.vdot(psi, apply_weyl(psi, w, n, d)))


def gate_unitary(gate, d: int) -> np.ndarray:
    """Dense unitary of a generated gate (see ``synth.circuits``)."""
    if hasattr(gate, "sp_index"):
        imgs = clifford.random_gate_images(gate.sp_index, gate.shift, d)
        return clifford.unitary_from_images(imgs, 2, d)
    return clifford.diag_gate(gate.phases)


def gate_sites(gate):
    if hasattr(gate, "sp_index"):
        return [gate.q0, gate.q1]
    return [gate.site]


def run(gates, n: int, d: int) -> np.ndarray:
    psi = zero_state(n, d)
    for g in gates:
        psi = apply_gate(psi, gate_unitary(g, d), gate_sites(g), n, d)
    return psi


def same_up_to_phase(a: np.ndarray, b: np.ndarray):
    """(relative 2-norm distance after the best global phase, that phase)."""
    ov = np.vdot(a, b)
    ph = ov / abs(ov) if abs(ov) > 0 else 1.0
    return float(np.linalg.norm(a * ph - b) / np.linalg.norm(b)), ph
