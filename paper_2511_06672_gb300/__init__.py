"""GB300-native GCAMPS hot path (arxiv 2511.06672): Python binding of libgcamps.

The binding only marshals arguments; every step of the simulation runs in the CUDA kernels of
libgcamps (``csrc/``), behind the C ABI of ``include/gcamps.h``.  Importing the package does not
touch the GPU; creating a ``Simulator`` loads the library and fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes as C
from typing import Iterable, Optional, Sequence

import numpy as np

from . import _native as N
from ._native import OP_DTYPE, OP_CLIFFORD, OP_NONCLIFFORD, OP_DISENTANGLE
from ._native import GATE_H, GATE_S, GATE_SUM, GATE_X, GATE_Z

__all__ = ["Simulator", "GcampsError", "sp4_images", "named_images", "num_candidates", "candidate", "ops_from_gates",
           "score_theta_noalloc", "weyl_expectation",
           "OP_DTYPE", "OP_CLIFFORD", "OP_NONCLIFFORD", "OP_DISENTANGLE",
           "GATE_H", "GATE_S", "GATE_SUM", "GATE_X", "GATE_Z"]


class GcampsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"gcamps error {code}: {msg}")
        self.code = code


def _check(lib, h, rc):
    if rc != N.OK:
        msg = lib.gcamps_last_error(h).decode() if h else ""
        raise GcampsError(rc, msg)


def num_candidates(d: int) -> int:
    return N.load().gcamps_num_candidates(d)


def sp4_images(d: int, sp_index: int, shift=(0, 0, 0, 0)) -> np.ndarray:
    """Generator images (20 int32) of the seeded-circuit gate (sp_index, shift)."""
    lib = N.load()
    sh = np.ascontiguousarray(shift, dtype=np.int32)
    img = np.zeros(20, dtype=np.int32)
    rc = lib.gcamps_sp4_images(d, int(sp_index), N.ptr(sh, C.c_int32), N.ptr(img, C.c_int32))
    if rc:
        raise GcampsError(rc, "bad sp4 index or shift")
    return img


def named_images(d: int, gate: int) -> np.ndarray:
    """Generator images of a named gate (GATE_H, GATE_S, GATE_SUM, GATE_X, GATE_Z) in the layout of
    Simulator.apply_clifford: 6 int32 for a one-qudit gate, 20 for SUM."""
    lib = N.load()
    img = np.zeros(20, dtype=np.int32)
    nq = C.c_int32()
    rc = lib.gcamps_named_images(d, gate, N.ptr(img, C.c_int32), C.byref(nq))
    if rc:
        raise GcampsError(rc, "unknown named gate or unsupported d")
    return img[: 6 if nq.value == 1 else 20].copy()


def candidate(d: int, k: int):
    """(images[20], unitary d^2 x d^2) of disentangler class k, from the library's host tables."""
    lib = N.load()
    img = np.zeros(20, dtype=np.int32)
    u = np.zeros(2 * d ** 4)
    rc = lib.gcamps_candidate(d, k, N.ptr(img, C.c_int32), N.ptr(u, C.c_double))
    if rc:
        raise GcampsError(rc, "bad class index")
    return img, (u[0::2] + 1j * u[1::2]).reshape(d * d, d * d)


def _dev_ptr(x) -> int:
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


def score_theta_noalloc(d: int, chi_l: int, chi_r: int, theta_dev, s2_dev, vn_dev, choice_dev,
                        tie_tol: float = 1e-10, stream=None) -> None:
    """gcamps_score_theta_noalloc: class scores on caller-owned device buffers, with the library's
    static working memory (no device allocation).  Buffers are torch CUDA tensors or raw device
    addresses: theta (chi_l, d, d, chi_r) complex128, s2 and vn K float64, choice 3 int32.  stream:
    a torch.cuda.Stream, a raw cudaStream_t, or None (default stream).  Asynchronous."""
    lib = N.load()
    K = num_candidates(d)
    # shapes beyond the static limit are left to the library, which refuses them (ESIZE) before any launch
    if K > 0 and 1 <= chi_l <= N.NOALLOC_MAX_SIDE // d and 1 <= chi_r <= N.NOALLOC_MAX_SIDE // d:
        # torch tensors are checked against the shapes the call reads and writes (raw addresses are not)
        import torch
        for name, t, dtype, numel in (("theta", theta_dev, torch.complex128, chi_l * d * d * chi_r),
                                      ("s2", s2_dev, torch.float64, K), ("vn", vn_dev, torch.float64, K),
                                      ("choice", choice_dev, torch.int32, 3)):
            if isinstance(t, torch.Tensor):
                if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() < numel:
                    raise GcampsError(N.EINVAL, f"score_theta_noalloc: {name} must be a contiguous CUDA {dtype} "
                                                f"tensor of at least {numel} elements")
    st = getattr(stream, "cuda_stream", stream) or None
    rc = lib.gcamps_score_theta_noalloc(d, chi_l, chi_r, _dev_ptr(theta_dev), _dev_ptr(s2_dev), _dev_ptr(vn_dev),
                                        _dev_ptr(choice_dev), float(tie_tol), st)
    if rc:
        raise GcampsError(rc, "score_theta_noalloc: " + {N.EINVAL: "bad argument",
                                                          N.ESIZE: f"chi d above {N.NOALLOC_MAX_SIDE}",
                                                          N.ECUDA: "CUDA set-up or launch failed"}.get(rc, ""))


def ops_from_gates(gates: Iterable, d: int, disentangle_after_t: bool = True) -> np.ndarray:
    """Gate list (synth.circuits gates) -> array of gcamps_op records."""
    rows = []
    cache = {}
    for g in gates:
        if hasattr(g, "sp_index"):
            key = (g.sp_index, tuple(g.shift))
            if key not in cache:
                cache[key] = sp4_images(d, g.sp_index, g.shift)
            r = np.zeros((), dtype=OP_DTYPE)
            r["kind"], r["q0"], r["q1"] = OP_CLIFFORD, g.q0, g.q1
            r["img"] = cache[key]
            rows.append(r)
        else:
            r = np.zeros((), dtype=OP_DTYPE)
            r["kind"], r["q0"], r["q1"] = OP_NONCLIFFORD, g.site, -1
            ph = np.zeros(4)
            ph[: len(g.phases)] = g.phases
            r["phases"] = ph
            rows.append(r)
            if disentangle_after_t:
                r2 = np.zeros((), dtype=OP_DTYPE)
                r2["kind"] = OP_DISENTANGLE
                rows.append(r2)
    out = np.zeros(len(rows), dtype=OP_DTYPE)
    for i, r in enumerate(rows):
        out[i] = r
    return out


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Simulator:
    """psi = C|MPS> for ``batch`` independent circuits of n qudits (Sec. 3 of the paper).  ``n`` may
    be a sequence of per-circuit qudit counts (uneven batch; ``batch`` is then its length)."""

    def __init__(self, n, d: int, chi_max: int, cutoff: float = 1e-12, max_sweeps: int = 8,
                 tie_tol: float = 1e-10, batch: int = 1, stream=None, strict_weight: float = 0.0,
                 cluster_size: int = 8, score_kind: int = 0, snapshot_entries: int = 0,
                 snapshot_max_gates: int = 0, precision: int = 0):
        self._lib = N.load()
        o = N.Opts()
        self._lib.gcamps_default_opts(C.byref(o))
        o.cutoff, o.max_sweeps, o.tie_tol, o.strict_weight = cutoff, max_sweeps, tie_tol, strict_weight
        o.cluster_size = cluster_size
        o.score_kind = score_kind
        o.precision = precision
        o.snapshot_entries, o.snapshot_max_gates = snapshot_entries, snapshot_max_gates
        s = _stream_handle(stream)
        o.cuda_stream = C.c_void_p(s) if s else None
        h = C.c_void_p()
        if np.ndim(n) == 0:
            nq = [int(n)] * batch
            rc = self._lib.gcamps_create_batch(batch, int(n), d, chi_max, C.byref(o), C.byref(h))
        else:
            nq = [int(x) for x in n]
            batch = len(nq)
            na = np.ascontiguousarray(nq, dtype=np.int32)
            rc = self._lib.gcamps_create_batch_uneven(batch, N.ptr(na, C.c_int32), d, chi_max, C.byref(o),
                                                      C.byref(h))
        if rc:
            raise GcampsError(rc, "gcamps_create failed")
        self._h = h
        self.nq = nq
        self.n = max(nq)
        self.d, self.chi_max, self.batch = d, chi_max, batch
        self._snap_max = snapshot_max_gates

    def set_cluster_size(self, cluster_size: int):
        self._c(self._lib.gcamps_set_cluster_size(self._h, cluster_size))

    def set_exact_cta(self, min_m: int):
        """Exact class evaluations at warp-level sizes one per CTA from m = min_m on (gcamps_set_exact_cta)."""
        self._c(self._lib.gcamps_set_exact_cta(self._h, min_m))

    def set_jacobi_cap(self, sweeps: int):
        """Most sweeps of one Jacobi SVD before the engine reports GCAMPS_ENOCONV (default 60)."""
        self._c(self._lib.gcamps_set_jacobi_cap(self._h, sweeps))

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.gcamps_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, rc):
        _check(self._lib, self._h, rc)

    # -- gates
    def apply_clifford(self, q0: int, q1: int, img: Sequence[int]):
        a = np.ascontiguousarray(img, dtype=np.int32)
        self._c(self._lib.gcamps_apply_clifford(self._h, q0, q1, N.ptr(a, C.c_int32)))

    def apply_named(self, gate: int, q0: int, q1: int = -1):
        self._c(self._lib.gcamps_apply_named(self._h, gate, q0, q1))

    def apply_nonclifford(self, site: int, phases: Sequence[float]):
        p = np.zeros(4)
        p[: len(phases)] = phases
        self._c(self._lib.gcamps_apply_nonclifford(self._h, site, N.ptr(p, C.c_double)))

    def disentangle(self) -> dict:
        st = N.Stats()
        self._c(self._lib.gcamps_disentangle(self._h, C.byref(st)))
        return st.as_dict()

    def run(self, ops: np.ndarray, begin: Optional[Sequence[int]] = None):
        ops = np.ascontiguousarray(ops, dtype=OP_DTYPE)
        b = None if begin is None else np.ascontiguousarray(begin, dtype=np.int32)
        self._c(self._lib.gcamps_run(self._h, ops.ctypes.data_as(C.c_void_p), len(ops),
                                     None if b is None else N.ptr(b, C.c_int32)))

    def run_device(self, ops_dev_ptr: int, begin_dev_ptr: int):
        self._c(self._lib.gcamps_run_device(self._h, C.c_void_p(ops_dev_ptr), C.c_void_p(begin_dev_ptr)))

    def sync(self):
        self._c(self._lib.gcamps_sync(self._h))

    def reset(self):
        self._c(self._lib.gcamps_reset(self._h))

    # -- readouts
    def expect_weyl(self, x, z, circuit: int = 0) -> complex:
        xa = np.ascontiguousarray(x, dtype=np.int32)
        za = np.ascontiguousarray(z, dtype=np.int32)
        re, im = C.c_double(), C.c_double()
        self._c(self._lib.gcamps_batch_expect_weyl(self._h, circuit, N.ptr(xa, C.c_int32), N.ptr(za, C.c_int32),
                                             C.byref(re), C.byref(im)))
        return complex(re.value, im.value)

    def expect_gradient(self, x, z, circuit: int = 0):
        """(Re<W>, gradient [gates, d]) with respect to the phases of every non-Clifford gate since the
        last reset (adjoint pass of the library; needs a handle with snapshots)."""
        xa = np.ascontiguousarray(x, dtype=np.int32)
        za = np.ascontiguousarray(z, dtype=np.int32)
        cap = max(1, self._snap_max)
        g = np.zeros(cap * self.d)
        val, ng = C.c_double(), C.c_int32()
        self._c(self._lib.gcamps_expect_gradient(self._h, circuit, N.ptr(xa, C.c_int32), N.ptr(za, C.c_int32),
                                                 C.byref(val), N.ptr(g, C.c_double), cap, C.byref(ng)))
        return val.value, g[: ng.value * self.d].reshape(ng.value, self.d).copy()

    def statevector(self, circuit: int = 0) -> np.ndarray:
        dim = self.d ** self.nq[circuit]
        re, im = np.zeros(dim), np.zeros(dim)
        self._c(self._lib.gcamps_statevector(self._h, circuit, N.ptr(re, C.c_double), N.ptr(im, C.c_double)))
        return re + 1j * im

    def amplitude(self, digits, circuit: int = 0) -> complex:
        a = np.ascontiguousarray(digits, dtype=np.int32)
        re, im = C.c_double(), C.c_double()
        self._c(self._lib.gcamps_batch_amplitude(self._h, circuit, N.ptr(a, C.c_int32), C.byref(re), C.byref(im)))
        return complex(re.value, im.value)

    def tableau(self, circuit: int = 0):
        n = self.nq[circuit]
        e = np.zeros((2 * n, 2 * n), dtype=np.uint8)
        p = np.zeros(2 * n, dtype=np.uint8)
        self._c(self._lib.gcamps_batch_get_tableau(self._h, circuit, N.ptr(e, C.c_uint8), N.ptr(p, C.c_uint8)))
        return e, p

    def inverse_tableau(self, circuit: int = 0):
        n = self.nq[circuit]
        e = np.zeros((2 * n, 2 * n), dtype=np.uint8)
        p = np.zeros(2 * n, dtype=np.uint8)
        self._c(self._lib.gcamps_get_inverse_tableau(self._h, circuit, N.ptr(e, C.c_uint8), N.ptr(p, C.c_uint8)))
        return e, p

    def bond_dims(self, circuit: int = 0) -> list:
        a = np.zeros(self.nq[circuit] - 1, dtype=np.int32)
        self._c(self._lib.gcamps_batch_get_bond_dims(self._h, circuit, N.ptr(a, C.c_int32)))
        return a.tolist()

    def schmidt_values(self, bond: int, circuit: int = 0) -> np.ndarray:
        s = np.zeros(self.d * self.chi_max * self.d + 64)
        cnt = C.c_int32()
        self._c(self._lib.gcamps_get_schmidt(self._h, circuit, bond, N.ptr(s, C.c_double), C.byref(cnt)))
        return s[: cnt.value].copy()

    def site(self, j: int, circuit: int = 0) -> np.ndarray:
        """MPS tensor of site j, shape (chi_l, d, chi_r)."""
        dims = np.zeros(3, dtype=np.int32)
        self._c(self._lib.gcamps_get_site(self._h, circuit, j, None, 0, N.ptr(dims, C.c_int32)))
        t = np.zeros(int(np.prod(dims)), dtype=np.complex128)
        self._c(self._lib.gcamps_get_site(self._h, circuit, j, t.ctypes.data_as(C.POINTER(C.c_double)), t.size,
                                          N.ptr(dims, C.c_int32)))
        return t.reshape(tuple(int(x) for x in dims))

    def last_weyl(self, circuit: int = 0):
        x = np.zeros(self.nq[circuit], dtype=np.int32)
        z = np.zeros(self.nq[circuit], dtype=np.int32)
        r = C.c_int32()
        self._c(self._lib.gcamps_get_last_weyl(self._h, circuit, N.ptr(x, C.c_int32), N.ptr(z, C.c_int32),
                                               C.byref(r)))
        return r.value, x, z

    def stats(self, circuit: int = 0) -> dict:
        st = N.Stats()
        self._c(self._lib.gcamps_get_stats(self._h, circuit, C.byref(st)))
        return st.as_dict()

    def set_replay(self, pairs, circuit: int = 0):
        """Replay the (bond, class) decisions ``pairs`` (as from decisions()) at this circuit's bond visits from the
        next launch on; an empty list turns replay off."""
        a = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1))
        self._c(self._lib.gcamps_set_replay(self._h, circuit, N.ptr(a, C.c_int32) if a.size else None, a.size // 2))

    def overlap(self, other: "Simulator", circuit: int = 0, other_circuit: int = 0) -> complex:
        """<M|M'> of this circuit's MPS and another handle's (same n, d, chi_max)."""
        re, im = C.c_double(), C.c_double()
        self._c(self._lib.gcamps_overlap(self._h, circuit, other._h, other_circuit, C.byref(re), C.byref(im)))
        return complex(re.value, im.value)

    def profile(self, circuit: int = 0) -> dict:
        """Leader-CTA cycles per engine phase and per bond-visit size bucket since the last reset
        (gcamps_get_profile)."""
        p = np.zeros(N.PROF_WORDS, dtype=np.int64)
        cnt = C.c_int32()
        self._c(self._lib.gcamps_get_profile(self._h, circuit, p.ctypes.data_as(C.POINTER(C.c_int64)), N.PROF_WORDS,
                                             C.byref(cnt)))
        out = {"cycles": {k: int(p[i]) for i, k in enumerate(N.PROF_PHASES)}, "buckets": {},
               "leader_warp_exact": {"cycles": int(p[11]), "count": int(p[32])},
               "sm_ids": [int(v) - 1 for v in p[160:176] if v > 0]}
        nph = len(N.PROF_PHASES)
        for b, name in enumerate(N.PROF_BUCKETS):
            out["buckets"][name] = {"visits": int(p[12 + b]), "cycles": int(p[17 + b]), "exact": int(p[22 + b]),
                                    "estimates": int(p[27 + b]),
                                    "phases": {k: int(p[33 + nph * b + i]) for i, k in enumerate(N.PROF_PHASES)}}
            for g, level in enumerate(("warp", "cta")):
                w = 88 + 6 * (5 * g + b)
                out["buckets"][name]["exact_" + level] = {
                    "count": int(p[w]), "cycles": int(p[w + 1]), "gram": int(p[w + 2]), "householder": int(p[w + 3]),
                    "eigenvalues": int(p[w + 4]), "entropy": int(p[w + 5])}
        return out

    def score_theta(self, theta: np.ndarray):
        """(S2, S_vN, chosen class, exact evaluations) for theta of shape (chi_l, d, d, chi_r)."""
        t = np.ascontiguousarray(theta, dtype=np.complex128)
        cl, cr = t.shape[0], t.shape[3]
        s2 = np.zeros(self._lib.gcamps_num_candidates(self.d))
        vn = np.zeros_like(s2)
        ch = np.zeros(2, dtype=np.int32)
        self._c(self._lib.gcamps_score_theta(self._h, cl, cr, t.ctypes.data_as(C.POINTER(C.c_double)),
                                             N.ptr(s2, C.c_double), N.ptr(vn, C.c_double), N.ptr(ch, C.c_int32)))
        return s2, vn, int(ch[0]), int(ch[1])

    def estimate_theta(self, theta: np.ndarray):
        """(FP32 von Neumann estimate, its error bound) of every class for theta (chi_l, d, d, chi_r)."""
        t = np.ascontiguousarray(theta, dtype=np.complex128)
        cl, cr = t.shape[0], t.shape[3]
        est = np.zeros(self._lib.gcamps_num_candidates(self.d))
        bd = np.zeros_like(est)
        self._c(self._lib.gcamps_estimate_theta(self._h, cl, cr, t.ctypes.data_as(C.POINTER(C.c_double)),
                                                N.ptr(est, C.c_double), N.ptr(bd, C.c_double)))
        return est, bd

    def last_scores(self, circuit: int = 0):
        """(S2, S_vN, evaluated) of every class at the last disentangler bond visit."""
        K = self._lib.gcamps_num_candidates(self.d)
        s2, vn = np.zeros(K), np.zeros(K)
        ev = np.zeros(K, dtype=np.uint8)
        self._c(self._lib.gcamps_get_last_scores(self._h, circuit, N.ptr(s2, C.c_double), N.ptr(vn, C.c_double),
                                                 N.ptr(ev, C.c_uint8)))
        return s2, vn, ev.astype(bool)

    def last_theta(self, circuit: int = 0):
        """Two-site tensor of the last bond visit, shape (chi_l, d, d, chi_r), or None if too large."""
        shape = np.zeros(2, dtype=np.int32)
        buf = np.zeros(729, dtype=np.complex128)
        self._c(self._lib.gcamps_get_last_theta(self._h, circuit, buf.ctypes.data_as(C.POINTER(C.c_double)),
                                                N.ptr(shape, C.c_int32)))
        cl, cr = int(shape[0]), int(shape[1])
        nel = cl * self.d * self.d * cr
        return None if nel > 729 else buf[:nel].reshape(cl, self.d, self.d, cr).copy()

    def decisions(self, circuit: int = 0) -> list:
        cnt = C.c_int32()
        self._c(self._lib.gcamps_get_decisions(self._h, circuit, None, 0, C.byref(cnt)))
        a = np.zeros(2 * max(cnt.value, 1), dtype=np.int32)
        self._c(self._lib.gcamps_get_decisions(self._h, circuit, N.ptr(a, C.c_int32), cnt.value, C.byref(cnt)))
        return [(int(a[2 * i]), int(a[2 * i + 1])) for i in range(min(cnt.value, len(a) // 2))]


def weyl_expectation(phases, sim: "Simulator", gates, x, z, circuit: int = 0):
    """Re<W> of a parametrised circuit as a differentiable torch function of the phases of its
    non-Clifford gates.

    phases: tensor [gates, d] (row k = phases of the k-th diagonal gate of ``gates``, in order; the
    other fields of those gates are kept); gates: synth gate list; sim: a Simulator with snapshots
    (one circuit is run, ``circuit``).  The forward runs the circuit through the library and the
    backward returns the library's adjoint gradient (gcamps_expect_gradient).  Binding only: both
    directions run in the library's kernels."""
    import torch

    class _Expect(torch.autograd.Function):
        @staticmethod
        def forward(ctx, ph):
            import dataclasses
            p = ph.detach().cpu().numpy().astype(np.float64)
            k = 0
            gl = []
            for g in gates:
                if hasattr(g, "sp_index"):
                    gl.append(g)
                else:
                    gl.append(dataclasses.replace(g, phases=tuple(float(v) for v in p[k])))
                    k += 1
            sim.reset()
            ops = ops_from_gates(gl, sim.d)
            if sim.batch > 1:
                begin = [0] * (sim.batch + 1)
                for c in range(circuit + 1, sim.batch + 1):
                    begin[c] = len(ops)
                sim.run(ops, begin)
            else:
                sim.run(ops)
            val, grad = sim.expect_gradient(x, z, circuit)
            ctx.save_for_backward(torch.as_tensor(grad, dtype=ph.dtype, device=ph.device))
            return torch.as_tensor(val, dtype=ph.dtype, device=ph.device)

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout * grad

    return _Expect.apply(phases)
