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


def observable_and_phase_gradient(gates, n: int, d: int, w: Weyl):
    """<O> = Re <psi|W|psi> = <psi|(W + W^dag)/2|psi> for psi = U |0...0>, and its gradient with
    respect to the phases of every diagonal gate: gate k = diag(e^{i phi_{k,j}}) on site s_k has
    d phi_{k,j} derivatives.  d D / d phi_j = i Pi_j D (Pi_j the projector on level j of s_k), so with
    phi_k = the state right after gate k and lambda_k = (gates after k)^dag O psi,
    d<O>/d phi_{k,j} = 2 Re <psi| O A_k i Pi_j |phi_k> = -2 Im <lambda_k| Pi_j |phi_k>
    (the adjoint method on dense vectors; O is Hermitian).  Returns (<O>, list of d-vectors, one
    per diagonal gate in circuit order)."""
    psi = zero_state(n, d)
    states = []                      # state right after each gate
    for g in gates:
        psi = apply_gate(psi, gate_unitary(g, d), gate_sites(g), n, d)
        states.append(psi)
    wpsi = apply_weyl(psi, w, n, d)
    val = float(np.vdot(psi, wpsi).real)
    # W^dag = conj(tau^r) (x)_j L_j^dag for W = tau^r (x)_j L_j
    wdpsi = psi
    for j in range(n):
        if w.x[j] or w.z[j]:
            wdpsi = apply_gate(wdpsi, w.local_matrix(j).conj().T, [j], n, d)
    wdpsi = np.conj(tau(d) ** w.r) * wdpsi
    lam = 0.5 * (wpsi + wdpsi)       # O psi
    grads = []
    for idx in range(len(gates) - 1, -1, -1):
        g = gates[idx]
        if not hasattr(g, "sp_index"):
            t = states[idx].reshape((d,) * n)
            lt = lam.reshape((d,) * n)
            gk = np.zeros(d)
            for j in range(d):
                ov = np.vdot(np.take(lt, j, axis=g.site), np.take(t, j, axis=g.site))
                gk[j] = -2.0 * ov.imag
            grads.append(gk)
        u = gate_unitary(g, d)
        lam = apply_gate(lam, u.conj().T, gate_sites(g), n, d)
    grads.reverse()
    return val, grads
