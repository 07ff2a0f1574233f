"""Seeded T-doped random Clifford brickwork circuits (the paper's benchmark family, Sec. 4).

The paper's benchmark circuits interleave random Cliffords with T gates (Sec. 4, Fig. 4).
Here a circuit on ``n`` qudits has ``layers`` brickwork layers of random two-qudit Cliffords
and ``t`` diagonal non-Clifford gates placed between layers.

Layout (all deterministic in the seed):

* PRNG: SplitMix64, one stream per circuit, seeded with ``seed``.
* Layer ``l`` acts on the pairs ``(i, i+1)`` with ``i = l (mod 2)`` and ``i+1 < n``
  (open boundary), in increasing ``i``.  For each pair, in this order: one uniform index
  into the lexicographically sorted list of the |Sp(4, F_d)| symplectic 4x4 matrices, then
  four uniform shift exponents ``(a0, b0, a1, b1)`` in Z_d.  The gate these name is
  ``X^a0 Z^b0 (x) X^a1 Z^b1`` times the standard-phase Clifford of the symplectic matrix.
* Non-Clifford gate ``k = 0..t-1`` follows layer ``ceil((k+1) * layers / t) - 1``; its
  site is drawn uniformly right after that layer's gates, in increasing ``k``.

``layered_t_circuit`` gives the layout of the paper's Fig. 4 instead: per layer a random Clifford on all
qudits (a deep brickwork stand-in), then one T gate on qudit 0.

The module only draws integers and places gates.  It never interprets a symplectic index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Tuple, Union

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): 64-bit state, golden-ratio increment."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform_int(self, n: int) -> int:
        """Uniform integer in [0, n) by rejection (no modulo bias)."""
        if n <= 0:
            raise ValueError("n must be positive")
        limit = (1 << 64) - ((1 << 64) % n)
        while True:
            z = self.next_u64()
            if z < limit:
                return z % n

    def uniform_float(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def sp4_order(d: int) -> int:
    """|Sp(4, F_d)| = d^4 (d^2 - 1)(d^4 - 1): 720 for d = 2, 51840 for d = 3."""
    return d ** 4 * (d ** 2 - 1) * (d ** 4 - 1)


def t_gate_phases(d: int) -> Tuple[float, ...]:
    """Phases (radians) of the qudit T gate used by the benchmarks.

    d = 2: diag(1, e^{i pi/4}) (Sec. 2.3.2).  d = 3: diag(1, e^{2 pi i/9}, e^{-2 pi i/9}), the
    third-level-of-the-hierarchy qutrit T; the matrix printed in Sec. 2.3.2 is a different
    diagonal and can be passed explicitly instead.
    """
    if d == 2:
        return (0.0, math.pi / 4)
    if d == 3:
        return (0.0, 2 * math.pi / 9, -2 * math.pi / 9)
    raise ValueError("d must be 2 or 3")


@dataclass(frozen=True)
class Clifford2:
    """Random two-qudit Clifford on (q0, q0+1): symplectic index + Weyl shift (a0, b0, a1, b1)."""
    q0: int
    q1: int
    sp_index: int
    shift: Tuple[int, int, int, int]


@dataclass(frozen=True)
class Diag:
    """Diagonal non-Clifford gate diag(e^{i phases[j]}) on one site."""
    site: int
    phases: Tuple[float, ...]
    param: int = -1  # index of the parameter it carries, or -1


Gate = Union[Clifford2, Diag]


def _t_after_layer(k: int, layers: int, t: int) -> int:
    return ((k + 1) * layers + t - 1) // t - 1


def brickwork_circuit(n: int, d: int, layers: int, t: int, seed: int,
                      phases: Tuple[float, ...] = None) -> List[Gate]:
    """T-doped random Clifford brickwork circuit; see the module docstring for the layout."""
    if n < 2:
        raise ValueError("need n >= 2")
    if phases is None:
        phases = t_gate_phases(d)
    rng = SplitMix64(seed)
    order = sp4_order(d)
    after = [[] for _ in range(layers)]
    for k in range(t):
        after[_t_after_layer(k, layers, t)].append(k)
    out: List[Gate] = []
    for layer in range(layers):
        for i in range(layer % 2, n - 1, 2):
            idx = rng.uniform_int(order)
            shift = tuple(rng.uniform_int(d) for _ in range(4))
            out.append(Clifford2(i, i + 1, idx, shift))
        for _k in after[layer]:
            out.append(Diag(rng.uniform_int(n), tuple(phases)))
    return out


def param_phase_circuit(n: int, d: int, layers: int, ngates: int, seed: int) -> Tuple[List[Gate], List[float]]:
    """Brickwork circuit with ``ngates`` parametrised gates diag(1, e^{i th}, e^{-i th}) (d = 3)
    or diag(1, e^{i th}) (d = 2), th ~ U(0, 2 pi) drawn from the same stream.

    Returns the gate list and the parameter values; gate ``k`` carries ``param = k``.
    """
    rng = SplitMix64(seed)
    order = sp4_order(d)
    after = [[] for _ in range(layers)]
    for k in range(ngates):
        after[_t_after_layer(k, layers, ngates)].append(k)
    out: List[Gate] = []
    thetas: List[float] = []
    for layer in range(layers):
        for i in range(layer % 2, n - 1, 2):
            idx = rng.uniform_int(order)
            shift = tuple(rng.uniform_int(d) for _ in range(4))
            out.append(Clifford2(i, i + 1, idx, shift))
        for k in after[layer]:
            site = rng.uniform_int(n)
            th = 2 * math.pi * rng.uniform_float()
            thetas.append(th)
            ph = (0.0, th) if d == 2 else (0.0, th, -th)
            out.append(Diag(site, ph, k))
    return out, thetas


def layered_t_circuit(n: int, d: int, layers: int, seed: int, depth: int = 0,
                      phases: Tuple[float, ...] = None) -> Tuple[List[Gate], List[int]]:
    """The circuit family of the paper's Fig. 4: every layer is a random Clifford on all ``n`` qudits
    followed by one T gate on qudit 0, so the circuit has as many T gates as layers.

    The random n-qudit Clifford of a layer is ``depth`` (default ``n``) brickwork sublayers of random
    two-qudit Cliffords drawn as in ``brickwork_circuit`` (sublayer ``s`` of the whole circuit acts on
    the pairs ``(i, i+1)``, ``i = s (mod 2)``).  This is a stand-in: it is not the uniform distribution
    on the n-qudit Clifford group.  Returns the gate list and, for every layer, the index one past its
    last gate (the T gate)."""
    if n < 2:
        raise ValueError("need n >= 2")
    if phases is None:
        phases = t_gate_phases(d)
    depth = depth or n
    rng = SplitMix64(seed)
    order = sp4_order(d)
    out: List[Gate] = []
    ends: List[int] = []
    sub = 0
    for _layer in range(layers):
        for _s in range(depth):
            for i in range(sub % 2, n - 1, 2):
                idx = rng.uniform_int(order)
                shift = tuple(rng.uniform_int(d) for _ in range(4))
                out.append(Clifford2(i, i + 1, idx, shift))
            sub += 1
        out.append(Diag(0, tuple(phases)))
        ends.append(len(out))
    return out, ends


def batched_workload(count: int, seed0: int = 0, n_range=(16, 48), layer_range=(16, 48)):
    """Shapes of a batch of independent circuits: circuit ``i`` uses seed ``seed0 + i`` and draws,
    from a SplitMix64 stream seeded with ``seed0 + i`` xor a fixed tag (so that the shapes do not
    reuse the gate stream), its qudit count ``n`` and its layer count uniformly in the given
    inclusive ranges; it has ``t = n`` non-Clifford gates.  Returns a list of (n, layers, t, seed)."""
    out = []
    for i in range(count):
        rng = SplitMix64((seed0 + i) ^ 0x5EED5EED5EED5EED)
        n = n_range[0] + rng.uniform_int(n_range[1] - n_range[0] + 1)
        layers = layer_range[0] + rng.uniform_int(layer_range[1] - layer_range[0] + 1)
        out.append((n, layers, n, seed0 + i))
    return out
