"""The update count that allocates no memory (bsgd_count_updates_noalloc).

It serves callers that cannot let the library allocate device memory; its
counters sit in a fixed __device__ array shared by every call. This file is
collected last, so that a run stopping at the first failure has run every
other test already. It checks, through the C ABI, that two calls in a row give
the same counts as bsgd_count_updates (which allocates its own counters), so
the shared array is cleared between calls, and that too many views are refused.
"""
import ctypes

import numpy as np
import pytest

from helpers import gpu_geom, spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1903_11874_gb300 import binding as B  # noqa: E402


@pytest.mark.parametrize("name", ["config1", "cone_small"])
def test_noalloc_count_matches_allocating_count_twice(name):
    gg = gpu_geom(spec(name))
    lib = B.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for rb, cb in [(None, None), ([1, 2], [0, 1])]:
        ref = B.bsgd_count_updates(gg, row_blocks=rb, col_blocks=cb)
        assert ref > 0
        rp, nr, _ra = B._ids(rb)
        cp, nc, _ca = B._ids(cb)
        for _ in range(2):                  # two calls in a row share the array
            out = ctypes.c_int64(-1)
            st = lib.bsgd_count_updates_noalloc(gg.handle, rp, nr, cp, nc, ctypes.byref(out),
                                                stream)
            assert st == 0, lib.bsgd_last_error()
            assert out.value == ref


def test_noalloc_count_rejects_too_many_views():
    s = dict(kind="par2d", nx=8, ny=8, nz=1, dx=1.0, dy=1.0, dz=1.0, n_views=16385, nu=12, nv=1,
             du=1.0, dv=1.0, M=1, N=1)
    gg = B.Geometry(**s)
    with pytest.raises(B.BSGDError) as ei:
        B.bsgd_count_updates_noalloc(gg)
    assert ei.value.status == 1
    assert "16384" in str(ei.value)
