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


def test_struct_sizes_match_header(lib):
    """Layouts of the descriptor structs as the C compiler sees them."""
    from paper_2410_20429_gb300 import _abi
    assert ct.sizeof(_abi.mars_iter_params) == 60
    assert ct.sizeof(_abi.mars_cache_desc) == 32
    assert ct.sizeof(_abi.mars_iter_stats) == 152 + 4 * 16 * 4 + 8 * 16 + 8 * 8 + 8
    assert ct.sizeof(_abi.mars_scene_desc) == 16 + 7 * 8 + 80 + 16
