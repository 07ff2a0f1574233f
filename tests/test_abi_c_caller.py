"""A C program written against the contract's boundary builds and runs against libgcamps.

The caller below uses the call signatures and option fields of the hot-path contract exactly: the
single-circuit readouts gcamps_amplitude(h, digits, re, im), gcamps_expect_weyl(h, x, z, re, im),
gcamps_get_tableau(h, exps, phase), gcamps_get_bond_dims(h, chi); gcamps_opts with cutoff, max_sweeps,
score_kind, precision, tie_tol, cuda_stream first, in that order (initialised positionally); the gate
names GCAMPS_H/S/SUM/X/Z; gcamps_batch_create(count, n[], d, chi_max, ...).  Each signature is checked by
assigning the function to a pointer of the exact type (gcc -Werror rejects a mismatch).  It then runs the
host-only paths that need no GPU: named-gate images, class counts and the argument checks of creation.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SRC = r"""
#include <stddef.h>
#include <stdio.h>
#include "gcamps.h"

static int (*p_create)(int, int, int, const gcamps_opts*, gcamps_t**) = gcamps_create;
static void (*p_destroy)(gcamps_t*) = gcamps_destroy;
static int (*p_apply_clifford)(gcamps_t*, int, int, const int32_t*) = gcamps_apply_clifford;
static int (*p_apply_named)(gcamps_t*, int, int, int) = gcamps_apply_named;
static int (*p_apply_nonclifford)(gcamps_t*, int, const double*) = gcamps_apply_nonclifford;
static int (*p_disentangle)(gcamps_t*, gcamps_stats*) = gcamps_disentangle;
static int (*p_amplitude)(gcamps_t*, const int32_t*, double*, double*) = gcamps_amplitude;
static int (*p_expect_weyl)(gcamps_t*, const int32_t*, const int32_t*, double*, double*) = gcamps_expect_weyl;
static int (*p_get_tableau)(gcamps_t*, uint8_t*, uint8_t*) = gcamps_get_tableau;
static int (*p_get_bond_dims)(gcamps_t*, int32_t*) = gcamps_get_bond_dims;
static const char* (*p_last_error)(gcamps_t*) = gcamps_last_error;
static int (*p_batch_create)(int, const int32_t*, int, int, const gcamps_opts*, gcamps_t**) = gcamps_batch_create;

_Static_assert(offsetof(gcamps_opts, cutoff) == 0, "cutoff first");
_Static_assert(offsetof(gcamps_opts, max_sweeps) == sizeof(double), "max_sweeps second");
_Static_assert(offsetof(gcamps_opts, score_kind) == offsetof(gcamps_opts, max_sweeps) + sizeof(int), "score_kind");
_Static_assert(offsetof(gcamps_opts, precision) == offsetof(gcamps_opts, score_kind) + sizeof(int), "precision");
_Static_assert(offsetof(gcamps_opts, tie_tol) > offsetof(gcamps_opts, precision), "tie_tol after precision");
_Static_assert(offsetof(gcamps_opts, cuda_stream) > offsetof(gcamps_opts, tie_tol), "cuda_stream after tie_tol");
_Static_assert(offsetof(gcamps_opts, strict_weight) > offsetof(gcamps_opts, cuda_stream), "extensions last");

int main(void) {
  int linked = (p_create != 0) + (p_destroy != 0) + (p_apply_clifford != 0) + (p_apply_named != 0) +
               (p_apply_nonclifford != 0) + (p_disentangle != 0) + (p_amplitude != 0) + (p_expect_weyl != 0) +
               (p_get_tableau != 0) + (p_get_bond_dims != 0) + (p_last_error != 0) + (p_batch_create != 0);
  if (linked != 12) return 1;
  gcamps_opts o = {1e-12, 8, 0, 0, 1e-10, NULL};   /* the contract's fields, in its order */
  int32_t img[20];
  int32_t nq = 0;
  if (gcamps_named_images(3, GCAMPS_H, img, &nq) != GCAMPS_OK || nq != 1) return 2;
  if (gcamps_named_images(3, GCAMPS_SUM, img, &nq) != GCAMPS_OK || nq != 2) return 3;
  if (gcamps_num_candidates(2) != 20 || gcamps_num_candidates(3) != 90) return 4;
  gcamps_t* h = (gcamps_t*)&o;
  if (p_create(1, 3, 16, &o, &h) != GCAMPS_EINVAL || h != NULL) return 5;   /* n < 2: refused before CUDA */
  o.precision = 9;
  if (p_create(4, 3, 16, &o, &h) != GCAMPS_EINVAL || h != NULL) return 6;   /* unknown precision */
  o.precision = 0;
  int32_t ns[2] = {4, 1};
  if (p_batch_create(2, ns, 3, 16, &o, &h) != GCAMPS_EINVAL || h != NULL) return 7;
  if (p_last_error(NULL) == NULL) return 8;
  p_destroy(NULL);
  printf("c caller ok\n");
  return 0;
}
"""


@pytest.fixture(scope="module")
def libpath():
    from paper_2511_06672_gb300.build import build_library
    return build_library()


def test_c_caller_builds_and_runs_against_the_contract(libpath, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(C_SRC)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(libpath)
    cmd = [cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           "-L", libdir, "-lgcamps", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and "c caller ok" in r.stdout, (r.returncode, r.stdout, r.stderr)
