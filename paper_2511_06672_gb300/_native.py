"""ctypes declarations for libgcamps (include/gcamps.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libgcamps.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ECHI, ESIZE, ESNAP = 0, 1, 2, 3, 4, 5, 6, 7
NOALLOC_MAX_SIDE = 81
PROF_WORDS = 192
PROF_PHASES = ("clifford", "mpo", "center", "theta", "screen", "vn_estimate", "exact", "decide", "apply_q", "split",
               "qr_move")
PROF_BUCKETS = ("m<=9", "m<=27", "m<=54", "m<=81", "m>81")
OP_CLIFFORD, OP_NONCLIFFORD, OP_DISENTANGLE = 1, 2, 3
GATE_H, GATE_S, GATE_SUM, GATE_X, GATE_Z = 1, 2, 3, 4, 5

OP_DTYPE = np.dtype([("kind", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("img", "<i4", (20,)),
                     ("pad", "<i4"), ("phases", "<f8", (4,))], align=True)
assert OP_DTYPE.itemsize == 128


class Opts(C.Structure):
    _fields_ = [("cutoff", C.c_double), ("max_sweeps", C.c_int), ("score_kind", C.c_int),
                ("precision", C.c_int), ("tie_tol", C.c_double), ("cuda_stream", C.c_void_p),
                ("strict_weight", C.c_double), ("cluster_size", C.c_int),
                ("snapshot_entries", C.c_int64), ("snapshot_max_gates", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("t_gates", C.c_int64), ("clifford_gates", C.c_int64), ("bonds_visited", C.c_int64),
                ("candidates_scored", C.c_int64), ("accepted", C.c_int64), ("sweeps", C.c_int64),
                ("vn_evaluations", C.c_int64), ("svd_calls", C.c_int64), ("jacobi_sweeps", C.c_int64),
                ("jacobi_max_sweeps", C.c_int64), ("qr_calls", C.c_int64),
                ("max_chi", C.c_int32), ("status", C.c_int32), ("discarded_weight", C.c_double),
                ("scoring_flops", C.c_double), ("screen_flops", C.c_double), ("tensor_flops", C.c_double),
                ("algorithmic_flops", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = [
    "gcamps_default_opts", "gcamps_num_candidates", "gcamps_sp4_images", "gcamps_candidate",
    "gcamps_named_images", "gcamps_apply_named", "gcamps_create", "gcamps_create_batch",
    "gcamps_create_batch_uneven", "gcamps_batch_create", "gcamps_batch_expect_weyl", "gcamps_batch_amplitude",
    "gcamps_batch_get_tableau", "gcamps_batch_get_bond_dims", "gcamps_destroy", "gcamps_num_qudits",
    "gcamps_set_cluster_size", "gcamps_set_jacobi_cap", "gcamps_set_exact_cta", "gcamps_apply_clifford",
    "gcamps_apply_nonclifford", "gcamps_disentangle", "gcamps_run", "gcamps_run_device", "gcamps_expect_weyl",
    "gcamps_expect_gradient", "gcamps_statevector", "gcamps_amplitude", "gcamps_get_tableau",
    "gcamps_get_inverse_tableau", "gcamps_get_bond_dims", "gcamps_get_schmidt", "gcamps_get_site",
    "gcamps_get_last_weyl", "gcamps_get_stats", "gcamps_get_profile", "gcamps_set_replay", "gcamps_overlap",
    "gcamps_get_decisions", "gcamps_get_last_scores", "gcamps_get_last_theta", "gcamps_score_theta",
    "gcamps_estimate_theta", "gcamps_score_theta_noalloc", "gcamps_sync", "gcamps_reset", "gcamps_last_error",
    "gcamps_measure_peaks",
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libgcamps; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgcamps not built ({path} missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, i32p, u8p, dp = C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_uint8), C.POINTER(C.c_double)
    sig = {
        "gcamps_default_opts": (None, [C.POINTER(Opts)]),
        "gcamps_num_candidates": (C.c_int, [C.c_int]),
        "gcamps_sp4_images": (C.c_int, [C.c_int, C.c_int64, i32p, i32p]),
        "gcamps_candidate": (C.c_int, [C.c_int, C.c_int, i32p, dp]),
        "gcamps_named_images": (C.c_int, [C.c_int, C.c_int, i32p, i32p]),
        "gcamps_apply_named": (C.c_int, [vp, C.c_int, C.c_int, C.c_int]),
        "gcamps_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(Opts), C.POINTER(vp)]),
        "gcamps_create_batch": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(Opts), C.POINTER(vp)]),
        "gcamps_create_batch_uneven": (C.c_int, [C.c_int, i32p, C.c_int, C.c_int, C.POINTER(Opts), C.POINTER(vp)]),
        "gcamps_destroy": (None, [vp]),
        "gcamps_num_qudits": (C.c_int, [vp, C.c_int]),
        "gcamps_set_cluster_size": (C.c_int, [vp, C.c_int]),
        "gcamps_set_jacobi_cap": (C.c_int, [vp, C.c_int]),
        "gcamps_set_exact_cta": (C.c_int, [vp, C.c_int]),
        "gcamps_apply_clifford": (C.c_int, [vp, C.c_int, C.c_int, i32p]),
        "gcamps_apply_nonclifford": (C.c_int, [vp, C.c_int, dp]),
        "gcamps_disentangle": (C.c_int, [vp, C.POINTER(Stats)]),
        "gcamps_run": (C.c_int, [vp, vp, C.c_int, i32p]),
        "gcamps_run_device": (C.c_int, [vp, vp, vp]),
        "gcamps_expect_weyl": (C.c_int, [vp, i32p, i32p, dp, dp]),
        "gcamps_batch_expect_weyl": (C.c_int, [vp, C.c_int, i32p, i32p, dp, dp]),
        "gcamps_batch_create": (C.c_int, [C.c_int, i32p, C.c_int, C.c_int, C.POINTER(Opts), C.POINTER(vp)]),
        "gcamps_expect_gradient": (C.c_int, [vp, C.c_int, i32p, i32p, dp, dp, C.c_int32, i32p]),
        "gcamps_statevector": (C.c_int, [vp, C.c_int, dp, dp]),
        "gcamps_amplitude": (C.c_int, [vp, i32p, dp, dp]),
        "gcamps_batch_amplitude": (C.c_int, [vp, C.c_int, i32p, dp, dp]),
        "gcamps_get_tableau": (C.c_int, [vp, u8p, u8p]),
        "gcamps_batch_get_tableau": (C.c_int, [vp, C.c_int, u8p, u8p]),
        "gcamps_get_inverse_tableau": (C.c_int, [vp, C.c_int, u8p, u8p]),
        "gcamps_get_bond_dims": (C.c_int, [vp, i32p]),
        "gcamps_batch_get_bond_dims": (C.c_int, [vp, C.c_int, i32p]),
        "gcamps_get_schmidt": (C.c_int, [vp, C.c_int, C.c_int, dp, i32p]),
        "gcamps_get_site": (C.c_int, [vp, C.c_int, C.c_int, dp, C.c_int64, i32p]),
        "gcamps_get_last_weyl": (C.c_int, [vp, C.c_int, i32p, i32p, i32p]),
        "gcamps_get_stats": (C.c_int, [vp, C.c_int, C.POINTER(Stats)]),
        "gcamps_get_profile": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int64), C.c_int32, i32p]),
        "gcamps_set_replay": (C.c_int, [vp, C.c_int, i32p, C.c_int32]),
        "gcamps_overlap": (C.c_int, [vp, C.c_int, vp, C.c_int, dp, dp]),
        "gcamps_get_decisions": (C.c_int, [vp, C.c_int, i32p, C.c_int32, i32p]),
        "gcamps_score_theta": (C.c_int, [vp, C.c_int, C.c_int, dp, dp, dp, i32p]),
        "gcamps_estimate_theta": (C.c_int, [vp, C.c_int, C.c_int, dp, dp, dp]),
        "gcamps_score_theta_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, vp, vp, vp, vp, C.c_double, vp]),
        "gcamps_get_last_scores": (C.c_int, [vp, C.c_int, dp, dp, u8p]),
        "gcamps_get_last_theta": (C.c_int, [vp, C.c_int, dp, i32p]),
        "gcamps_sync": (C.c_int, [vp]),
        "gcamps_measure_peaks": (C.c_int, [dp, C.c_int]),
        "gcamps_reset": (C.c_int, [vp]),
        "gcamps_last_error": (C.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))
