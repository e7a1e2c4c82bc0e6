"""Host-side checks of the C ABI: the library builds, loads, exports every entry
point that include/rbo.h declares, and the Python mirrors of its structs have the
C layout.  No kernel is launched."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rbo.h")


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16717_gb300 as p
    return p


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rbo_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_north_star_calls():
    names = declared_functions()
    for req in ["rbo_sketch_create", "rbo_block_orth_one_stage", "rbo_block_orth_two_stage",
                "rbo_mpk_csr", "rbo_sstep_gmres"]:
        assert req in names


def test_library_exports_every_declared_symbol(pkg):
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rbo_\w+)", out))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    for f in declared_functions():
        assert hasattr(pkg.lib, f)
        assert f in pkg.SIGNATURES


def test_binding_names_match_the_abi(pkg):
    for f in ["sketch_create", "sketch_apply", "gram", "block_orth_one_stage",
              "block_orth_two_stage", "block_orth_cholqr2", "mpk_csr", "sstep_gmres"]:
        assert callable(getattr(pkg, f))


def test_struct_layouts_match_header(pkg, tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "rbo.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(rbo_opts), '
                    'sizeof(rbo_info), sizeof(rbo_csr), offsetof(rbo_info, history), '
                    'offsetof(rbo_info, relres)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [ctypes.sizeof(pkg.Opts), ctypes.sizeof(pkg.Info), ctypes.sizeof(pkg.Csr),
                    pkg.Info.history.offset, pkg.Info.relres.offset]


def test_host_only_calls(pkg):
    assert pkg.version().startswith("rbo")
    assert pkg.lib.rbo_status_string(-3).decode().startswith("Cholesky")
    sk = pkg.sketch_create(1000, 244, 8, 42)
    assert sk.d == 244
    with pytest.raises(pkg.RboError):
        pkg.sketch_create(1000, 4, 8, 42)   # zeta > d
    with pytest.raises(pkg.RboError):
        pkg.sketch_create(1000, 244, 17, 42)  # zeta too large


def test_c_program_links_and_calls_host_entry_points(pkg, tmp_path):
    # the header compiles as strict C99 and a C program links against the library
    # and runs its host-only entry points (no GPU needed)
    prog = tmp_path / "host.c"
    prog.write_text(r'''
#include <math.h>
#include <stdio.h>
#include <string.h>
#include "rbo.h"
int main(void) {
  double H[4] = {2.0, 3.0, -3.0, 2.0};  /* eigenvalues 2 +- 3i, column-major */
  double a[3], b[3];
  rbo_sketch sk = NULL;
  if (strncmp(rbo_version(), "rbo", 3) != 0) return 1;
  if (rbo_newton_shifts(H, 2, 2, 2, a, b) != RBO_OK) return 2;
  if (fabs(a[0] - 2.0) > 1e-12 || fabs(a[1] - 2.0) > 1e-12 || fabs(b[1] - 9.0) > 1e-10) return 3;
  if (rbo_chebyshev_shifts(H, 2, 2, 3, a, b) != RBO_OK) return 4;
  if (fabs(a[2] - 2.0) > 1e-12 || fabs(b[1] - 4.5) > 1e-10 || fabs(b[2] - 2.25) > 1e-10) return 5;
  if (rbo_newton_shifts(H, 2, 0, 2, a, b) != RBO_ERR_ARG) return 6;
  if (rbo_sketch_create(1000, 244, 8, 42, &sk) != RBO_OK || sk == NULL) return 7;
  if (rbo_sketch_destroy(sk) != RBO_OK) return 8;
  printf("ok\n");
  return 0;
}
''')
    exe = tmp_path / "host"
    libdir = os.path.dirname(pkg.LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe),
                    "-L", libdir, "-l:" + os.path.basename(pkg.LIB_PATH),
                    "-Wl,-rpath," + libdir, "-lm"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
