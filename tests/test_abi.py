"""The C-ABI library builds, loads and exports every symbol include/silh.h declares.

No GPU is needed: only host-side entry points and argument validation (which
returns before any CUDA call) are exercised.
"""
import ctypes
import os
import re

import pytest

import oracle
from paper_2607_01993_b300 import build as silh_build
from paper_2607_01993_b300 import silh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(silh_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    silh_build.build()
    return silh.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for want in ("silh_sample_pps", "silh_estimate", "silh_exact", "silh_global"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert names
    for name in names:
        assert hasattr(lib, name), name
    assert set(silh.EXPORTS) <= set(names)


def test_t_from_eps_matches_oracle(lib):
    for eps, delta, n, k in [(0.5, 0.01, 1000, 4), (0.1, 0.05, 10**6, 32)]:
        assert silh.silh_t_from_eps(eps, delta, n, k) == oracle.t_from_eps(eps, delta, n, k)


def test_argument_validation_without_device(lib):
    st = silh.SilhSample(2, None, None, None, None, 0, 0)
    rc = lib.silh_sample_pps(None, 0, 10, 2, 2, None, 2, 0, 4.0, -1.0, 0.01, 0, 0, 0,
                             ctypes.byref(st), None)
    assert rc == -1
    assert b"null" in lib.silh_last_error()
    rc = lib.silh_estimate(None, 0, 10, 2, 2, None, 2, 0, 0, None, None, 0, None, None, None,
                           None, None)
    assert rc == -1
    # k = 1 is not a clustering for the silhouette (b undefined)
    rc = lib.silh_exact(ctypes.c_void_p(16), 0, 10, 2, 2, ctypes.c_void_p(16), 1, 0, 0, None, 0,
                        None, None, None, None, None)
    assert rc == -1
    rc = lib.silh_global(None, 10, None, None)
    assert rc == -1
    # the wait self-test refuses a limit outside [1 us, 1 s] before launching
    lib.silh_wait_selftest.argtypes = [ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p]
    assert lib.silh_wait_selftest(0, 0, None) == -1
    assert lib.silh_wait_selftest(0, 2_000_000_000, None) == -1
    assert lib.silh_version().startswith(b"silh")
