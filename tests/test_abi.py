"""The C ABI library loads on a machine without a GPU and exports every entry
point include/ilg.h declares; the ctypes mirror of ilg_params has the C layout.
No compute call is made here."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        names += re.findall(r"^\s*(?:ilg_status|const char\*|void|int)\s+(ilg_\w+)\s*\(", text, re.M)
    return names


@pytest.fixture(scope="module")
def binding():
    import __graft_entry__ as g
    from paper_2203_01380_gb300 import build as b
    b.build()
    from paper_2203_01380_gb300 import binding as B
    return B


def test_every_declared_symbol_is_exported(binding):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(binding.lib(), n), n


def test_params_layout_matches_c(binding):
    src = r"""
#include <stddef.h>
#include <stdio.h>
#include "ilg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(ilg_params), offsetof(ilg_params, n0),
         offsetof(ilg_params, omega_eff), offsetof(ilg_params, seed), offsetof(ilg_params, replica),
         offsetof(ilg_params, sampler));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    P = binding.Params
    assert got == [ctypes.sizeof(P), P.n0.offset, P.omega_eff.offset, P.seed.offset, P.replica.offset,
                   P.sampler.offset]


def test_binding_refuses_to_import_without_library(tmp_path):
    """The product path has no fallback: without libilg.so beside it the binding
    module raises at import time (checked on a copy in an empty directory)."""
    import shutil
    pkg = tmp_path / "pkg"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2203_01380_gb300", "binding.py"), pkg / "binding.py")
    r = subprocess.run(["python", "-c", "import sys; sys.path.insert(0, %r); import binding" % str(pkg)],
                       capture_output=True, text=True)
    assert r.returncode != 0 and "no CPU fallback" in r.stderr


def test_lb_params_layout_matches_c(binding):
    src = r"""
#include <stddef.h>
#include <stdio.h>
#include "ilg.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(ilg_lb_params), offsetof(ilg_lb_params, n0),
         offsetof(ilg_lb_params, omega_j), offsetof(ilg_lb_params, omega), offsetof(ilg_lb_params, theta));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        got = [int(v) for v in subprocess.check_output([exe]).split()]
    P = binding.LBParams
    assert got == [ctypes.sizeof(P), P.n0.offset, P.omega_j.offset, P.omega.offset, P.theta.offset]
