"""The C ABI library: builds, loads, exports every symbol include/isg.h
declares, and answers without a GPU by an error status (no CPU fallback).
Host-side arithmetic of the ABI (xi_2) is compared with the oracle here,
since it runs on the CPU.
"""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"\b(isg_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def abi():
    from paper_2503_14688_b300 import build

    build.build()
    from paper_2503_14688_b300 import _abi

    return _abi


def test_every_declared_symbol_is_exported(abi):
    names = _declared_functions()
    assert len(names) >= 15
    lib = ctypes.CDLL(abi.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a prototype for each of them
    assert set(names) <= set(abi.PROTOTYPES), set(names) - set(abi.PROTOTYPES)


def test_library_links_no_cpu_fallback(abi):
    """The kernels are sm_103a device code; the library has no host sweep."""
    lib = abi.lib()
    assert lib.isg_lattice_bytes(abi.ISG_ISING, 1 << 20) == (1 << 40) // 8
    assert lib.isg_lattice_bytes(abi.ISG_BLUME_CAPEL, 1 << 19) == (1 << 38) // 4
    assert lib.isg_lattice_bytes(abi.ISG_ISING, 100) == 0       # not a multiple of 64
    assert lib.isg_lattice_bytes(abi.ISG_ISING, 1 << 21) == 0   # above the maximum
    assert lib.isg_lattice_bytes(7, 256) == 0                   # unknown model


def test_invalid_arguments_rejected_before_any_device_work(abi):
    lib = abi.lib()
    h = ctypes.c_void_p()
    d = abi.isg_lattice_desc(model=0, L=100, seed=1, record_capacity=4)
    assert lib.isg_lattice_create(ctypes.byref(d), ctypes.byref(h)) == abi.ISG_ERR_INVALID
    assert b"multiple of 64" in lib.isg_last_error()
    d = abi.isg_lattice_desc(model=0, L=256, seed=1, record_capacity=0)
    assert lib.isg_lattice_create(ctypes.byref(d), ctypes.byref(h)) == abi.ISG_ERR_INVALID
    assert lib.isg_lattice_create(None, ctypes.byref(h)) == abi.ISG_ERR_INVALID
    assert lib.isg_sweep(None, 1, None, 0.4, 0) == abi.ISG_ERR_INVALID
    assert lib.isg_sweep(None, 1, None, -1.0, 0) == abi.ISG_ERR_INVALID
    lib.isg_lattice_destroy(None)  # NULL-safe
    # row slabs: offsets and heights in multiples of 16, inside the lattice
    for y0, rows in [(8, 16), (0, 24), (0, 0), (112, 32), (-16, 32)]:
        d = abi.isg_slab_desc(model=0, L=128, y0=y0, rows=rows, seed=1)
        assert lib.isg_slab_create(ctypes.byref(d), ctypes.byref(h)) == abi.ISG_ERR_INVALID
        assert not h.value
    assert lib.isg_slab_edge_bytes(abi.ISG_ISING, 1024) == 1024 // 16
    assert lib.isg_slab_edge_bytes(abi.ISG_BLUME_CAPEL, 1024) == 1024 // 8
    assert lib.isg_slab_edge_bytes(abi.ISG_ISING, 100) == 0
    assert lib.isg_slab_half_sweep(None, 0, 0.4) == abi.ISG_ERR_INVALID
    lib.isg_slab_destroy(None)  # NULL-safe


def test_without_gpu_create_reports_unsupported(abi):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2503_14688_b300 import IsgError, Lattice

    with pytest.raises(IsgError) as e:
        Lattice(256)
    assert e.value.status == abi.ISG_ERR_UNSUPPORTED


def test_xi2_host_arithmetic_matches_oracle_bitwise(abi, orc):
    from paper_2503_14688_b300 import xi2

    rng = np.random.default_rng(3)
    for L in (64, 256, 1000, 4096):
        for n in (1, 3, 17):
            R = rng.integers(-L, L + 1, size=(n, L)).astype(np.int32) + L // 2
            C = rng.integers(-L, L + 1, size=(n, L)).astype(np.int32) + L // 2
            M = R.sum(axis=1).astype(np.int64)
            a, b = xi2(M, R, C), orc.xi2(M, R, C)
            assert (np.isnan(a) and np.isnan(b)) or a == b, (L, n, a, b)


def test_load_rejects_foreign_and_missing_files(abi, tmp_path):
    lib = abi.lib()
    h = ctypes.c_void_p()
    missing = str(tmp_path / "nope.isg").encode()
    assert lib.isg_load(missing, None, 4, ctypes.byref(h)) == abi.ISG_ERR_INVALID
    bad = tmp_path / "bad.isg"
    bad.write_bytes(b"NOTALATT" + bytes(56))
    assert lib.isg_load(str(bad).encode(), None, 4, ctypes.byref(h)) == abi.ISG_ERR_INVALID
    assert b"not a lattice checkpoint" in lib.isg_last_error()
    assert not h.value


def test_xi_integral_closed_forms(abi):
    """C(r) = exp(-r/a): I2/I1 -> 2a (continuum); C = const: I2/I1 = (2/3) r_cut."""
    import math

    from paper_2503_14688_b300 import xi_integral

    r = np.linspace(0.0, 400.0, 40001)
    for a in (3.0, 10.0, 25.0):
        assert abs(xi_integral(r, np.exp(-r / a), 400.0) - 2 * a) < 1e-4 * a
    rc = np.arange(0.0, 101.0)
    assert abs(xi_integral(rc, np.ones_like(rc), 100.0) - 2 / 3 * 100.0) < 0.01
    # points beyond r_cut are ignored; degenerate input gives NaN
    assert abs(xi_integral(rc, np.ones_like(rc), 50.0) - 2 / 3 * 50.0) < 0.01
    assert math.isnan(xi_integral([0.0], [1.0], 10.0))
    assert math.isnan(xi_integral(rc, -np.ones_like(rc), 100.0))
