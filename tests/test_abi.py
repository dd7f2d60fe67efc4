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


def test_stage_rings_fit_and_keep_planes_in_flight(lib):
    """The variant table (static, readable without a GPU): every stage kernel
    fits the 227 KB of shared memory a block may use, and every fused stages
    3+4 kernel of the memory-bound FP32-math precisions keeps at least two
    planes in flight (a ring slot is held for three plane steps, so ring >= 5;
    the FP64 kernels are bound by the FP64 pipe instead and keep 4 slots in a
    110 KB budget).  The FP32 128 x 11 tile's stages 3+4
    kernel, whose 44 KB slots with the compensation tiles inside would allow
    only 5, holds six 32 KB slots (phi, psi, G1, G2 halo tiles of 15 x 136
    floats, 128-byte aligned) and a ring of three 11 KB slots of compensation
    tiles (11 x 128 floats each) after a 384-byte header."""
    from paper_1803_01291_gb300 import solver
    limit = 227 * 1024
    for prec in (_lib.FP64, _lib.FP32, _lib.BF16, _lib.FP32_PLAIN):
        for v in solver.variants(prec):
            assert max(v["smem"]) <= limit and max(v["pair_smem"]) <= limit
            assert v["pair_ring"][1] >= (4 if prec == _lib.FP64 else 5), (prec, v)
    v0 = solver.variants(_lib.FP32)[0]
    assert (v0["tile_x"], v0["pair_tile_y"][1]) == (128, 11)
    halo = (15 * 136 * 4 + 127) // 128 * 128
    comp = 2 * 11 * 128 * 4
    assert v0["pair_ring"][1] == 6
    assert v0["pair_smem"][1] == 384 + 6 * 4 * halo + 3 * comp
