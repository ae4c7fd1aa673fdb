"""The C ABI used from C: a C99 program compiled with gcc against
include/trbl.h and linked with libtrbl.so builds the 20Ne-sized basis of
the paper (sd shell, 2+2 particles, 2M = 0: D = 640, App. C) and the
48Cr-sized one (pf shell, 4+4: D = 1,963,461, Sec. IV A) through the host-only
entry points, and gets TRBL_ERR_ARG with a message for a null argument
and for a NaN coefficient.  No GPU is needed: these calls do no device work."""
import os
import shutil
import subprocess

import pytest

import paper_1902_02064_gb300 as trbl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include "trbl.h"
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

/* shells of 2j listed in order; 2m ascending inside a shell */
static int space(const int* twoj_shells, int nshell, int k, int* twoj, int* twom, int* orbit, trbl_space* s) {
  int n = 0;
  for (int o = 0; o < nshell; ++o)
    for (int m = -twoj_shells[o]; m <= twoj_shells[o]; m += 2) {
      twoj[n] = twoj_shells[o];
      twom[n] = m;
      orbit[n] = o;
      ++n;
    }
  s->n_states = n;
  s->twoj = twoj;
  s->twom = twom;
  s->orbit = orbit;
  s->n_particles = k;
  return n;
}

static long long dim(const int* shells, int nshell, int k) {
  int twoj[32], twom[32], orbit[32];
  trbl_space s;
  space(shells, nshell, k, twoj, twom, orbit, &s);
  trbl_basis* b = NULL;
  if (trbl_basis_create(&s, &s, 0, &b) != TRBL_OK) return -1;
  trbl_basis_sizes z;
  if (trbl_basis_info(b, &z) != TRBL_OK) return -2;
  trbl_basis_destroy(b);
  return (long long)z.dim;
}

int main(void) {
  const int sd[3] = {1, 3, 5}, pf[4] = {1, 3, 5, 7};
  printf("sd %lld\n", dim(sd, 3, 2));
  printf("pf %lld\n", dim(pf, 4, 4));
  trbl_basis* b = NULL;
  printf("null %d %s\n", trbl_basis_create(NULL, NULL, 0, &b), trbl_last_error());

  int twoj[32], twom[32], orbit[32];
  trbl_space s;
  const int n = space(sd, 3, 2, twoj, twom, orbit, &s);
  if (trbl_basis_create(&s, &s, 0, &b) != TRBL_OK) return 1;
  double* h1 = calloc((size_t)n * n, sizeof(double));
  double* v2 = calloc((size_t)n * n * n * n, sizeof(double));
  h1[0] = NAN;
  trbl_hamiltonian* h = NULL;
  printf("nan %d %s\n", trbl_hamiltonian_create(b, h1, h1, v2, v2, v2, &h), trbl_last_error());
  free(h1);
  free(v2);
  trbl_basis_destroy(b);
  return 0;
}
"""


def test_c_program_drives_the_host_entry_points(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    lib = trbl.library_path()
    trbl.lib()  # builds the library if it is missing or stale
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    lib, "-lm", "-Wl,-rpath," + os.path.dirname(lib), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout.split("\n")
    assert out[0] == "sd 640"
    assert out[1] == "pf 1963461"
    assert out[2].startswith("null %d " % trbl.TRBL_ERR_ARG)
    assert out[3].startswith("nan %d " % trbl.TRBL_ERR_ARG) and "h1A[0] is not finite" in out[3]


LAYOUT = r"""
#include "trbl.h"
#include <stddef.h>
#include <stdio.h>
#define F(S, m) printf(#S " " #m " %zu %zu\n", offsetof(S, m), sizeof(((S*)0)->m))
int main(void) {
  printf("trbl_params size %zu\n", sizeof(trbl_params));
  F(trbl_params, nev); F(trbl_params, q); F(trbl_params, max_basis); F(trbl_params, keep);
  F(trbl_params, tol); F(trbl_params, precision); F(trbl_params, max_iter); F(trbl_params, check_every);
  F(trbl_params, seed); F(trbl_params, normH); F(trbl_params, projections); F(trbl_params, reorth);
  F(trbl_params, refine);
  printf("trbl_stats size %zu\n", sizeof(trbl_stats));
  F(trbl_stats, iterations); F(trbl_stats, restarts); F(trbl_stats, converged); F(trbl_stats, status);
  F(trbl_stats, normH); F(trbl_stats, ms_total); F(trbl_stats, ms_apply); F(trbl_stats, ms_orth);
  F(trbl_stats, ms_qr); F(trbl_stats, ms_ritz); F(trbl_stats, ms_restart); F(trbl_stats, basis_size);
  F(trbl_stats, second_passes); F(trbl_stats, ms_copy_in); F(trbl_stats, ms_copy_out);
  return 0;
}
"""


def test_struct_layouts_match_the_python_binding(tmp_path):
    """trbl_params and trbl_stats as the C compiler lays them out (offset and
    size of every member, whole size) equal the ctypes structures the Python
    binding passes through the ABI."""
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    import ctypes
    from paper_1902_02064_gb300 import _lib
    src = tmp_path / "layout.c"
    src.write_text(LAYOUT)
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    lines = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = {"trbl_params": set(), "trbl_stats": set()}
    for ln in lines:
        parts = ln.split()
        if len(parts) == 3 and parts[1] == "size":
            assert int(parts[2]) == ctypes.sizeof(getattr(_lib, parts[0])), ln
        elif len(parts) == 4:
            cls = getattr(_lib, parts[0])
            fld = getattr(cls, parts[1])
            assert (fld.offset, fld.size) == (int(parts[2]), int(parts[3])), ln
            seen[parts[0]].add(parts[1])
    for name, got in seen.items():
        assert got == {f for f, _ in getattr(_lib, name)._fields_}, name


def test_header_constants_match_the_binding():
    """Every integer constant #defined in include/trbl.h that the Python
    binding also names has the same value there (status codes, dtypes,
    precisions, projection and reorthogonalisation modes, product kernels,
    the autotuner's candidate count, the allocation-free scratch size)."""
    import re
    text = open(os.path.join(ROOT, "include", "trbl.h")).read()
    found = 0
    for name, value in re.findall(r"^#define (TRBL_[A-Z0-9_]+) (\(?[0-9][0-9u <]*\)?)", text, re.M):
        if not hasattr(trbl, name):
            continue
        expr = value.replace("u", "").strip("()")
        assert getattr(trbl, name) == eval(expr, {}), name
        found += 1
    assert found >= 20
