"""FP64 CPU oracle for the GCAMPS non-Clifford step (arxiv 2511.06672).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or execute this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the CUDA library;
the only common input is the seeded circuit generator in ``synth/``.

It is written to be read against the paper, not to be fast:

* ``weyl``        generalised Pauli (Weyl) operators over Z_d, Sec. 2.3.
* ``clifford``    H_d, S_d, SUM_d (Sec. 2.3, Table 1), Cliffords from generator images,
                  Sp(4, F_d) and the two-qudit disentangler cosets (Sec. 3, Sec. 3.1).
* ``statevector`` dense d^n simulation (Sec. 2.1), the exactness anchor.
* ``tableau``     mod-d stabilizer tableau with dense-conjugation updates (Sec. 2.3) and
                  operator decomposition by Gaussian elimination (Sec. 2.3.1).
* ``mps``         matrix product states, MPO application, truncated SVD (Sec. 2.4, Eq. mps).
* ``gcamps``      psi = C|MPS>: Clifford loop, non-Clifford loop, disentangling (Sec. 3).

Every function of the package is pinned by ``tests/test_oracle_*.py`` against something
other than itself (paper tables, closed forms, dense simulation, brute force).  The two
readings that have no independent pin are flagged "parity unpinned" where they are defined.
"""
