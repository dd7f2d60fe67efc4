"""The C-ABI library loads and exports every entry point include/hbe.h
declares; host-only calls answer without a GPU."""
import ctypes
import os
import re

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)
from paper_1803_01291_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hbe_[a-z_0-9]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        __graft_entry__.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 30
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    assert names == set(_lib.EXPORTS)


def test_host_only_calls(lib):
    out = ctypes.c_size_t()
    assert lib.hbe_workspace_bytes(64, 0, 1, ctypes.byref(out)) == 0
    # FP32 + compensated state: 8 state fields + 3 G fields of (64+8)*(64+4)*64 floats
    assert out.value == 8 * 1253376 + 3 * 1253376
    assert lib.hbe_workspace_bytes(4, 0, 1, ctypes.byref(out)) == _lib.EINVAL
    assert lib.hbe_workspace_bytes(64, 2, 1, ctypes.byref(out)) == _lib.EINVAL
    assert lib.hbe_status_string(5) == b"HBE_STOPPED"
    for prec in (0, 1, 2, 3):
        n = lib.hbe_variant_count(prec)
        assert n >= 3
        v = _lib.HbeVariant()
        assert lib.hbe_variant_info(prec, 0, ctypes.byref(v)) == 0
        assert v.tile_x == 32 * v.vec and v.vec in (1, 2, 4)
        assert v.tile_y == v.rows_per_warp * v.consumer_warps
        assert v.threads == 32 * (v.consumer_warps + 1)
        assert all(s <= 227 * 1024 for s in v.smem_bytes) and all(r >= 4 for r in v.ring)
        assert lib.hbe_variant_info(prec, n, ctypes.byref(v)) == _lib.EINVAL
    # the radial solver's limits and argument checks run on the host
    assert lib.hbe_radial_max_n(0) == lib.hbe_radial_max_n(1) == 4096
    assert lib.hbe_radial_max_n(2) == 0
    nul = None
    assert lib.hbe_radial_run(1, 3, 1.0, nul, nul, nul, nul, 0.0, 0.01, 1, 0, 0, 0.0, 0.0,
                              nul, nul, nul, nul, nul, nul) == _lib.EINVAL
    assert lib.hbe_radial_run(1, 64, 1.0, nul, nul, nul, nul, 0.0, 0.01, 1, 0, 0, 0.0, 0.0,
                              nul, nul, nul, nul, nul, nul) == _lib.EINVAL  # null arrays


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1803_01291_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in text and "from oracle" not in text, fn
                assert "hbe_oracle" not in text, fn
