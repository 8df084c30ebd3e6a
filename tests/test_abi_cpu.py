"""Host-side checks of the C ABI library: it loads and exports every declared symbol.

No compute calls are made (no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "parareal.h")


@pytest.fixture(scope="module")
def lib_path():
    from paper_2110_10762_gb300 import _abi, build
    if not os.path.exists(_abi.LIB_PATH):
        build.build()
    return _abi.LIB_PATH


def declared():
    from paper_2110_10762_gb300._abi import header_declared_names
    return header_declared_names(HEADER)


def test_header_declares_the_boundary():
    names = set(declared())
    for must in ["parareal_create", "parareal_set_problem", "parareal_run_sync",
                 "parareal_run_async", "parareal_adjoint", "parareal_destroy"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (parareal_\w+)", out))
    missing = set(declared()) - exported
    assert not missing, missing
    lib = ctypes.CDLL(lib_path)
    for name in declared():
        assert hasattr(lib, name)


def test_binding_covers_every_symbol(lib_path):
    from paper_2110_10762_gb300 import _abi
    import paper_2110_10762_gb300 as pkg
    assert set(declared()) == set(_abi.EXPORTS)
    for name in declared():
        assert callable(getattr(pkg, name)), name


def test_version_string_without_gpu(lib_path):
    from paper_2110_10762_gb300 import _abi
    lib = _abi.load(lib_path)
    assert b"sm_103a" in lib.parareal_version()


def test_struct_layouts_match_header():
    """ctypes structs mirror the C structs (sizes computed by the host compiler)."""
    from paper_2110_10762_gb300 import _abi
    src = f"""
#include <stdio.h>
#include "{HEADER}"
int main() {{ printf("%zu %zu %zu %zu\\n", sizeof(pr_problem), sizeof(pr_stats),
  sizeof(pr_async_opts), sizeof(pr_event)); return 0; }}
"""
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        exe = os.path.join(d, "s")
        open(c, "w").write(src)
        subprocess.run(["gcc", c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert sizes == [ctypes.sizeof(_abi.pr_problem), ctypes.sizeof(_abi.pr_stats),
                     ctypes.sizeof(_abi.pr_async_opts), ctypes.sizeof(_abi.pr_event)]


def test_null_context_calls_are_rejected(lib_path):
    """Entry points validate their context before touching the GPU."""
    from paper_2110_10762_gb300 import _abi
    lib = _abi.load(lib_path)
    assert lib.parareal_set_problem(None, None) == _abi.PR_EINVAL
    assert lib.parareal_run_sync(None, None, None) == _abi.PR_EINVAL
    assert lib.parareal_create(None, 0, None) == _abi.PR_EINVAL
