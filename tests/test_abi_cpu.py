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


def test_python_struct_layouts_match_the_header(tmp_path):
    """Compile a probe against include/parareal.h and compare sizeof / offsetof of
    every field of the public structs with the ctypes view the binding uses."""
    from paper_2110_10762_gb300 import _abi
    structs = {"pr_problem": _abi.pr_problem, "pr_stats": _abi.pr_stats,
               "pr_async_opts": _abi.pr_async_opts, "pr_event": _abi.pr_event}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    exe = tmp_path / "probe"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        s, f, v = ln.split()
        got[(s, f)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_noalloc_size_check_rejects_large_axes_without_overflow(lib_path):
    """parareal_coarse_noalloc bounds each axis and the running product before
    multiplying: three axes whose product wraps a 64-bit integer (2^21 each:
    2^63) or lands back under the limit must be rejected, as must a single
    axis beyond it.  The size check precedes every CUDA call and never
    dereferences the (fake, aligned, non-null) pointers."""
    from paper_2110_10762_gb300 import _abi
    lib = _abi.load(lib_path)
    fake = ctypes.c_void_p(256)
    it = ctypes.c_int(0)
    for n in [(1 << 21, 1 << 21, 1 << 21), (1 << 31) - 1, (131073,), (65536, 65536, 4),
              (2, 65537), (3000000000 % (1 << 31), 1, 1)]:
        n = n if isinstance(n, tuple) else (n, n, n)
        nn = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
        code = lib.parareal_coarse_noalloc(len(n), nn, 1e-3, fake, None, fake, 1e-10, 0,
                                           ctypes.byref(it), None)
        assert code == _abi.PR_EINVAL, n
