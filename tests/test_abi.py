"""The C ABI library: builds, loads, exports every declared symbol, and its
host-side argument checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(gg_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2212_08200_b300 import build
    build.build()
    import paper_2212_08200_b300 as gg
    return gg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["gg_graph_create_csr", "gg_graph_destroy", "gg_sssp", "gg_sssp_ex", "gg_graph_check",
                     "gg_status_string", "gg_last_error"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    so = os.path.join(ROOT, "paper_2212_08200_b300", "libgg.so")
    out = subprocess.check_output(["nm", "-D", "--defined-only", so], text=True)
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    for n in declared_functions():
        getattr(lib, n)


def test_status_strings_and_abi(lib):
    import paper_2212_08200_b300 as gg
    assert gg.gg_abi_version() == 4
    for code, name in gg.STATUS.items():
        assert gg.gg_status_string(code) == name


def test_options_struct_layout(lib):
    import paper_2212_08200_b300 as gg
    o = gg.gg_options()
    lib.gg_options_default(ctypes.byref(o))
    assert o.struct_size == ctypes.sizeof(gg.gg_options)
    assert o.policy == gg.GG_POLICY_BSP_GRAPH and o.direction == gg.GG_DIR_PUSH


def _create(lib, n, m, ro, col, w, flags=0):
    h = ctypes.c_void_p()
    P = lambda a: None if a is None else a.ctypes.data  # noqa: E731
    rc = lib.gg_graph_create_csr(n, m, P(ro), P(col), P(w), flags, None, ctypes.byref(h))
    return rc, h.value


def test_argument_checks_before_any_device_call(lib):
    ro = np.array([0, 1, 2], np.uint32)
    col = np.array([1, 0], np.uint32)
    w = np.array([3, 3], np.uint32)
    rc, h = _create(lib, 0, 0, ro, col, w)
    assert rc == 1 and h is None                                   # n == 0
    rc, _ = _create(lib, 2, 2, None, col, w)
    assert rc == 1                                                 # null row_offsets
    rc, _ = _create(lib, 2, 2, ro, None, w)
    assert rc == 1                                                 # null col_indices
    rc, _ = _create(lib, 2, 2 ** 32, ro, col, w)
    assert rc == 1                                                 # m does not fit uint32 offsets
    rc, _ = _create(lib, 2, 2, ro, col, w, flags=0x80)
    assert rc == 1                                                 # unknown flag
    bad = np.array([1, 1, 2], np.uint32)
    rc, _ = _create(lib, 2, 2, bad, col, w)
    assert rc == 1                                                 # offsets not starting at 0
    bad = np.array([0, 1, 1], np.uint32)
    rc, _ = _create(lib, 2, 2, bad, col, w)
    assert rc == 1                                                 # offsets not ending at m
    assert b"row_offsets" in lib.gg_last_error()
    assert lib.gg_sssp(None, 0, None, None) == 1
    assert lib.gg_graph_check(None) == 1
    assert lib.gg_graph_destroy(None) == 1
