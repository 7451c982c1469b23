"""The C-ABI library: it builds for sm_103a, loads, exports every entry point
include/bsgd.h declares, and rejects bad arguments on the host (CPU only; no
compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_1903_11874_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bsgd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bsgd_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = B.load()
    names = declared_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(B.EXPORTS)


def test_status_strings():
    lib = B.load()
    assert lib.bsgd_status_string(0) == b"ok"
    assert lib.bsgd_status_string(1) == b"invalid argument"


@pytest.mark.parametrize("bad", [
    dict(nx=0),
    dict(kind="par2d", nz=4),
    dict(dsd=400.0),                 # dsd <= dso
    dict(dso=40.0, dsd=300.0),       # volume (half-diagonal 45) reaches the source circle
    dict(du=0.0),
    dict(dz=float("inf")),
])
def test_geometry_validation_rejects_bad_input(bad):
    s = dict(kind="cone3d", nx=64, ny=64, nz=64, dx=1.0, dy=1.0, dz=1.0, n_views=8, nu=32,
             nv=32, du=2.0, dv=2.0, dso=500.0, dsd=1000.0, M=2, N=2)
    s.update(bad)
    with pytest.raises(B.BSGDError) as ei:
        B.Geometry(**s)
    assert ei.value.status == 1


def test_block_counts_validated():
    s = dict(kind="par2d", nx=16, ny=16, nz=1, dx=1.0, dy=1.0, dz=1.0, n_views=8, nu=20,
             nv=1, du=1.0, dv=1.0)
    for M, N in [(0, 1), (9, 1), (1, 17), (1, 0)]:
        with pytest.raises(B.BSGDError) as ei:
            B.Geometry(M=M, N=N, **s)
        assert ei.value.status == 1
    with pytest.raises(B.BSGDError):
        B.Geometry(M=2, N=1, view_block=[0] * 8, **s)     # block 1 has no view


def test_null_handles_rejected():
    lib = B.load()
    assert lib.bsgd_geometry_destroy(None) == 1
    assert lib.bsgd_state_destroy(None) == 1
    assert lib.bsgd_block_step(None, None, 1, None) == 1
    n = ctypes.c_int64(0)
    assert lib.bsgd_state_checkpoint_bytes(None, ctypes.byref(n)) == 1
    assert lib.bsgd_state_save(None, None, 0, None) == 1
    assert lib.bsgd_state_restore(None, None, 0, None) == 1
    assert lib.bsgd_state_set_split(None, 1) == 1
    assert lib.bsgd_state_set_sampling(None, 0, 0, 1, None) == 1
    assert "NULL" in B.load().bsgd_last_error().decode()
