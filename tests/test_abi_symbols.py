"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads
without a GPU and exports every entry point that include/mars.h declares, and
the Python binding declares the same set."""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mars.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(mars_[a-z_]+)\s*\(", txt)
    return sorted(set(n for n in names if not n.endswith("_t")))


@pytest.fixture(scope="module")
def lib():
    from paper_2410_20429_gb300 import build as B
    path = B.build()
    return ct.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mars_scene_create", "mars_cache_create", "mars_render_iteration", "mars_update_counts",
              "mars_submit", "mars_poll"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_2410_20429_gb300 import _abi
    assert sorted(_abi.SIGNATURES) == _declared()


def test_error_string_and_version_without_gpu(lib):
    from paper_2410_20429_gb300 import _abi
    L = _abi.load()
    assert L.mars_version().startswith(b"mars-gb300")
    assert isinstance(L.mars_last_error_string(), bytes)
    # argument validation happens before any CUDA call
    h = ct.c_void_p()
    assert L.mars_scene_create(None, None, ct.byref(h)) == _abi.MARS_ERR_INVALID_ARG
    assert b"null" in L.mars_last_error_string()


def test_struct_sizes_match_header(lib, tmp_path):
    """Layouts of the descriptor structs as the C compiler sees them: a C
    program built against include/mars.h prints every struct's size and every
    field's offset, and the Python binding's ctypes structures must agree."""
    import shutil
    import subprocess
    from paper_2410_20429_gb300 import _abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [getattr(_abi, n) for n in dir(_abi)
               if n.startswith("mars_") and isinstance(getattr(_abi, n), type)
               and issubclass(getattr(_abi, n), ct.Structure)]
    assert len(structs) >= 9
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mars.h"', 'int main(void) {']
    for S in structs:
        lines.append(f'  printf("{S.__name__} size %zu\\n", sizeof({S.__name__}));')
        for f, _ in S._fields_:
            lines.append(f'  printf("{S.__name__} {f} %zu\\n", offsetof({S.__name__}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        name, field, v = line.split()
        got[(name, field)] = int(v)
    for S in structs:
        assert ct.sizeof(S) == got[(S.__name__, "size")], S.__name__
        for f, _ in S._fields_:
            assert getattr(S, f).offset == got[(S.__name__, f)], (S.__name__, f)
    # the sizes the header documents
    assert ct.sizeof(_abi.mars_iter_params) == 68
    assert ct.sizeof(_abi.mars_launch_config) == 56