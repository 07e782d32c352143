"""The C-ABI library builds, loads, and exports every entry point its header declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(sdd_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1402_0266_gb300 import build
    build.build()
    import paper_1402_0266_gb300 as sdd
    return sdd.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("sdd.h")
    assert "sdd_interface_mc" in names and "sdd_step" in names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    import paper_1402_0266_gb300 as sdd
    assert set(sdd.EXPORTS) == _declared("sdd.h")
    for n in sdd.EXPORTS:
        assert callable(getattr(sdd, n)), n


def test_library_is_sm103a_build():
    # the build compiles for sm_103a only
    from paper_1402_0266_gb300 import build
    assert build.ARCH == "-gencode=arch=compute_103a,code=sm_103a"


def test_host_checks_reject_bad_grid(lib):
    import ctypes
    import paper_1402_0266_gb300 as sdd
    h = ctypes.c_void_p()
    g = sdd._Grid(2, 5, 1, 1)   # nx < 3: rejected before any CUDA call
    assert lib.sdd_init(ctypes.byref(h), ctypes.byref(g), None, None, None, None) == sdd.SDD_EINVAL
    g = sdd._Grid(9, 9, 9, 1)   # more subdomains than cells
    assert lib.sdd_init(ctypes.byref(h), ctypes.byref(g), None, None, None, None) == sdd.SDD_EINVAL


def test_interface_nodes_of_the_workloads():
    import workloads as W
    i, j = W.interface_nodes(257, 257, 2, 2)
    assert i.size == 509
    i, j = W.interface_nodes(2049, 2049, 8, 8)
    assert i.size == 28609
    assert len(set(zip(i.tolist(), j.tolist()))) == i.size
