"""CPU checks of libgcamps: it builds for sm_103a, exports every symbol include/gcamps.h
declares, and its host-only tables (no GPU call) agree bit-exactly with the oracle:

* gcamps_sp4_images: the seeded-circuit gate (index into lexicographic Sp(4, F_d), Weyl shift)
  -> generator images, vs oracle.clifford.random_gate_images;
* gcamps_candidate: the 20 / 90 disentangler classes (order, images, unitaries) vs
  oracle.clifford.candidates.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_06672_gb300.build import build_library
    from paper_2511_06672_gb300 import _native
    build_library()
    return _native.load()


def declared_functions():
    with open(os.path.join(ROOT, "include", "gcamps.h")) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gcamps_[a-z0-9_]+)\s*\(", src)))


def test_exports_match_header(lib):
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    from paper_2511_06672_gb300._native import EXPORTS
    assert sorted(EXPORTS) == names


def test_every_entry_point_cites_its_passage():
    """Each declaration's comment names the passage of the paper it implements (Sec., Eq., Table, Fig.)
    or says that the paper has no counterpart."""
    with open(os.path.join(ROOT, "include", "gcamps.h")) as fh:
        src = fh.read()
    decl = re.compile(r"^(?:int|void|const char\*|int64_t)\s+\**(gcamps_[a-z0-9_]+)\s*\([^;]*\);", re.M)
    prev, missing = 0, []
    for m in decl.finditer(src):
        block = src[prev:m.start()]
        prev = m.end()
        if not any(t in block for t in ("Sec.", "Eq.", "Table", "Fig.", "counterpart")):
            missing.append(m.group(1))
    assert not missing


def test_num_candidates(lib):
    assert lib.gcamps_num_candidates(2) == 20
    assert lib.gcamps_num_candidates(3) == 90
    assert lib.gcamps_num_candidates(5) == -1


def _imgs_to_array(imgs):
    out = []
    for w in imgs:
        out.extend([int(w.x[0]), int(w.z[0]), int(w.x[1]), int(w.z[1]), int(w.r)])
    return np.array(out, dtype=np.int32)


@pytest.mark.parametrize("d", [2, 3])
def test_sp4_images_match_oracle(lib, d):
    from oracle import clifford
    import paper_2511_06672_gb300 as G
    rng = np.random.default_rng(100 + d)
    order = len(clifford.sp_group(2, d))
    for idx in list(rng.integers(0, order, 60)) + [0, order - 1]:
        shift = tuple(int(a) for a in rng.integers(0, d, 4))
        got = G.sp4_images(d, int(idx), shift)
        want = _imgs_to_array(clifford.random_gate_images(int(idx), shift, d))
        assert np.array_equal(got, want), (idx, shift)
    with pytest.raises(G.GcampsError):
        G.sp4_images(d, order, (0, 0, 0, 0))


@pytest.mark.parametrize("d", [2, 3])
def test_candidates_match_oracle(lib, d):
    from oracle import clifford
    import paper_2511_06672_gb300 as G
    cands = clifford.candidates(d)
    assert G.num_candidates(d) == len(cands)
    for k, (_s, imgs, u) in enumerate(cands):
        img, ug = G.candidate(d, k)
        assert np.array_equal(img, _imgs_to_array(imgs)), k
        assert np.allclose(ug, u, atol=1e-12), k


def test_create_without_gpu_fails_cleanly(lib):
    """With no CUDA device the create call returns an error code instead of crashing."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    rc = lib.gcamps_create(4, 3, 8, None, C.byref(h))
    assert rc != 0 and not h.value


def test_create_rejects_bad_options_before_touching_the_gpu(lib):
    """Option validation (score_kind 0..2, cluster size 1..16) happens on the host first."""
    from paper_2511_06672_gb300 import _native as N
    for field, value in (("score_kind", 3), ("score_kind", -1), ("cluster_size", 17), ("cluster_size", -2),
                         ("max_sweeps", -1)):
        o = N.Opts()
        lib.gcamps_default_opts(C.byref(o))
        setattr(o, field, value)
        h = C.c_void_p()
        assert lib.gcamps_create(4, 3, 8, C.byref(o), C.byref(h)) == N.EINVAL
        assert not h.value


def test_create_rejects_shapes_beyond_32_bit_matrix_indices(lib):
    """A handle whose largest matrix (the two-site tensor after the MPO, or the Jacobi rotations) would
    exceed 2^31 - 1 entries is refused on the host, before any CUDA call; shapes below the limit get
    past the check (without a GPU they then fail at the first CUDA call instead)."""
    import torch
    from paper_2511_06672_gb300 import _native as N
    for n, d, chi in ((40, 3, 1 << 16), (64, 2, 1 << 16), (128, 3, 1 << 30), (128, 2, 1 << 30), (20, 3, 6000)):
        h = C.c_void_p()
        assert lib.gcamps_create(n, d, chi, None, C.byref(h)) == N.EINVAL, (n, d, chi)
        assert not h.value
    if torch.cuda.is_available():
        return
    for n, d, chi in ((64, 3, 1024), (32, 3, 256), (20, 3, 5000), (40, 2, 11000)):
        h = C.c_void_p()
        rc = lib.gcamps_create(n, d, chi, None, C.byref(h))
        assert rc not in (N.OK, N.EINVAL), (n, d, chi)
        assert not h.value


@pytest.mark.parametrize("d", [2, 3])
def test_named_images_match_dense_conjugation(lib, d):
    """gcamps_named_images vs the oracle's dense conjugation U g U^dag of the gates as defined in
    Sec. 2.3 (H, S, SUM as matrices; X, Z the Weyl generators), snapped to tau^r W."""
    from oracle import clifford
    from oracle.weyl import X, Z
    import paper_2511_06672_gb300 as G
    dense = {G.GATE_H: (clifford.H_gate(d), 1), G.GATE_S: (clifford.S_gate(d), 1),
             G.GATE_SUM: (clifford.SUM_gate(d), 2), G.GATE_X: (X(d), 1), G.GATE_Z: (Z(d), 1)}
    for gate, (u, nq) in dense.items():
        imgs = clifford.images_by_conjugation(u, nq, d)
        if nq == 1:
            want = []
            for w in imgs:
                want.extend([int(w.x[0]), int(w.z[0]), int(w.r)])
            want = np.array(want, dtype=np.int32)
        else:
            want = _imgs_to_array(imgs)
        got = G.named_images(d, gate)
        assert np.array_equal(got, want), gate
    with pytest.raises(G.GcampsError):
        G.named_images(d, 6)
    with pytest.raises(G.GcampsError):
        G.named_images(5, G.GATE_H)


def test_noalloc_size_check_cannot_wrap(lib):
    """gcamps_score_theta_noalloc rejects shapes above its static limit before any CUDA call, including
    chi values whose product with d would wrap a 32-bit int (715827883 * 3 = 2^31 + 1).  The pointers are
    never dereferenced on this path."""
    from paper_2511_06672_gb300 import _native as N
    fake = C.c_void_p(16)
    for d, cl, cr in [(3, 715827883, 1), (3, 1, 715827883), (2, 1073741825, 1), (3, 28, 1), (2, 1, 41)]:
        rc = lib.gcamps_score_theta_noalloc(d, cl, cr, fake, fake, fake, fake, 1e-10, None)
        assert rc == N.ESIZE, (d, cl, cr, rc)


def test_handle_setters_reject_a_null_handle(lib):
    """The launch-shape and iteration-cap setters refuse a null handle before any CUDA call."""
    from paper_2511_06672_gb300 import _native as N
    assert lib.gcamps_set_exact_cta(None, 10) == N.EINVAL
    assert lib.gcamps_set_exact_cta(None, -1) == N.EINVAL
    assert lib.gcamps_set_jacobi_cap(None, 60) == N.EINVAL
    assert lib.gcamps_set_cluster_size(None, 12) == N.EINVAL
    cnt = C.c_int32(-7)
    assert lib.gcamps_get_profile(None, 0, None, 0, C.byref(cnt)) == N.EINVAL


def test_create_accepts_every_cluster_size_up_to_16(lib):
    """Cluster sizes 1..16 (not only powers of two) pass the host's option check; 0 means the default.
    Without a GPU the call then fails at its first CUDA call, never with EINVAL."""
    import torch
    from paper_2511_06672_gb300 import _native as N
    if torch.cuda.is_available():
        pytest.skip("checks the host-side path only")
    for cs in (0, 1, 3, 12, 14, 16):
        o = N.Opts()
        lib.gcamps_default_opts(C.byref(o))
        o.cluster_size = cs
        h = C.c_void_p()
        rc = lib.gcamps_create(4, 3, 8, C.byref(o), C.byref(h))
        assert rc not in (N.OK, N.EINVAL), (cs, rc)
        assert not h.value
