"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random numbers and lays out circuits; it holds none of the
GCAMPS arithmetic (no Weyl algebra, no tableau, no symplectic group).  A
two-qudit Clifford is emitted as an integer index into the lexicographically
sorted list of 4x4 symplectic matrices over F_d plus a Weyl shift; each side
(oracle, CUDA library) turns that index into a gate with its own code.
"""
from .circuits import (  # noqa: F401
    SplitMix64,
    sp4_order,
    t_gate_phases,
    brickwork_circuit,
    Clifford2,
    Diag,
    param_phase_circuit,
    batched_workload,
    layered_t_circuit,
)
