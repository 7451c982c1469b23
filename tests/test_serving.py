"""Serving: continuous batching of reconstructions (bsgd_server_*).

CPU: the admission model (bytes a request holds) and the host-side checks.
GPU: every result equals the same request run alone (and the plain solver),
requests of mixed geometry, size and storage type overlap on the device,
admission respects the byte budget and the slot count, and a bounded wait
returns TIMEOUT without disturbing the request.
"""
import math
import time

import numpy as np
import pytest

from paper_1903_11874_gb300 import binding as B
from paper_1903_11874_gb300 import synth


def cone(n, views, nd=None, vox=None):
    """n^3 volume of (256 / n) mm voxels, views over 360 deg, n x n detector of
    1.6 * 256 / n mm pixels, DSO 500 / DSD 1000 (the serving workload's shapes)."""
    nd = nd or n
    h = 256.0 / n if vox is None else vox
    return dict(kind="cone3d", nx=n, ny=n, nz=n, dx=h, dy=h, dz=h, n_views=views, nu=nd, nv=nd,
                du=1.6 * 256.0 / nd, dv=1.6 * 256.0 / nd, dso=500.0, dsd=1000.0)


def params(storage=B.F32, seed=1, epochs=2, mu=None):
    if mu is None:
        return B.SolveParams(alpha=1 / 4, gamma=1 / 4, epochs=epochs, rho=0.25, power_iters=10,
                             pair_sampling=B.PAIRS_RESIDUAL, storage=storage, seed=seed)
    return B.SolveParams(alpha=1 / 4, gamma=1 / 4, epochs=epochs, step_rule=B.STEP_FIXED, mu=mu,
                         pair_sampling=B.PAIRS_RESIDUAL, storage=storage, seed=seed)


# ---- CPU --------------------------------------------------------------------------

def test_request_bytes_model():
    g = cone(64, 90)
    f32 = B.bsgd_request_bytes(g, 4, 4, params())
    bf = B.bsgd_request_bytes(g, 4, 4, params(B.BF16))
    R = 90 * 64 * 64
    C = 64 ** 3
    # the state holds y, r (two sinograms), z^j and r~^j for each block's band
    # (compact storage: less than the 2 N full sinograms), the image, g, ...
    assert f32 >= 2 * R * 4 + 3 * C * 4
    assert bf < f32
    # compact storage: doubling the column blocks adds far less than the 2 x 4
    # extra full sinograms (one pair per iteration in both cases)
    one = dict(alpha=1 / 4, epochs=2, rho=0.25, power_iters=10)
    f4 = B.bsgd_request_bytes(g, 4, 4, B.SolveParams(gamma=1 / 4, **one))
    f8 = B.bsgd_request_bytes(g, 4, 8, B.SolveParams(gamma=1 / 8, **one))
    assert f8 - f4 < 0.5 * (2 * 4 * R * 4)
    # growing the problem grows the bill
    assert B.bsgd_request_bytes(cone(128, 180), 4, 4, params()) > 4 * f32 / 2


def test_request_bytes_rejects_bad_geometry():
    with pytest.raises(B.BSGDError):
        B.bsgd_request_bytes(dict(cone(64, 90), nx=0), 4, 4, params())


def test_server_rejects_an_unknown_round_policy():
    with pytest.raises(B.BSGDError) as e:
        B.Server(budget_bytes=1 << 30, max_slots=2, priority=7)
    assert e.value.status == 1


# ---- GPU --------------------------------------------------------------------------

def _data(geo, seed):
    from paper_1903_11874_gb300.binding import Geometry
    import torch
    gg = Geometry(M=4, N=4, **geo)
    n = geo["nx"]
    vol = synth.ellipsoid_phantom(n, n, n, 6, seed=seed) * 0.01
    p = torch.zeros(gg.n_rows, device="cuda:0")
    B.bsgd_forward_project(gg, torch.from_numpy(vol.reshape(-1)).cuda(), p)
    return p.cpu().numpy().astype(np.float32), gg


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.gpu
def test_results_alone_equal_results_in_the_mix():
    """The same request served alone and among other requests of different
    geometry, size and storage type gives the same image (to float atomics
    order), and both equal the plain solver."""
    geoA, geoB, geoC = cone(64, 90), cone(96, 120, nd=80), cone(48, 72)
    yA, ggA = _data(geoA, 1)
    yB, _ = _data(geoB, 2)
    yC, _ = _data(geoC, 3)
    pA = params(seed=5)
    srv = B.Server(budget_bytes=8 << 30, max_slots=8)
    try:
        ida = srv.submit(geoA, 4, 4, pA, yA)
        x_alone, rep_alone = srv.wait(ida)
        # B is resident before A and C are submitted, and runs long enough
        # (400 epochs) for both to be admitted while it still runs
        idb = srv.submit(geoB, 4, 4, params(seed=6, epochs=400), yB)
        t0 = time.time()
        while srv.stats()["resident"] < 1 and srv.stats()["completed"] < 2 and time.time() - t0 < 60:
            time.sleep(0.001)
        ids = [idb, srv.submit(geoA, 4, 4, pA, yA), srv.submit(geoC, 4, 4, params(B.BF16, seed=7), yC)]
        outs = [srv.wait(i) for i in ids]
        traces = {1: srv.read_trace(ids[1]), 2: srv.read_trace(ids[2])}
        trace_alone = srv.read_trace(ida)
        st = srv.stats()
    finally:
        srv.close()
    x_mix = outs[1][0]
    assert _rel(x_mix, x_alone) <= 1e-5
    assert outs[1][1]["iteration"] == rep_alone["iteration"] == 2 * 16
    assert np.array_equal(traces[1], trace_alone)   # same draws alone and in the mix
    assert st["completed"] == 4 and st["failed"] == 0
    assert st["peak_resident"] >= 2          # the requests overlapped on the GPU
    # the plain one-call solver, same parameters and seed
    import torch
    x_plain = np.zeros(ggA.n_cols, dtype=np.float32)
    B.bsgd_solve(ggA, pA, yA, x_plain)
    assert _rel(x_alone, x_plain) <= 1e-5
    # the served results against the FP64 oracle: Algorithm 1 with the served
    # request's own draws and step, FP32 request A within 1e-5, BF16-storage
    # request C within 1e-2
    for k, geo, yk, seed, tol in ((1, geoA, yA, 5, 1e-5), (2, geoC, yC, 7, 1e-2)):
        x_srv, rep = outs[k]
        x_o, rn_o = oracle_replay_served(geo, yk, seed, rep["mu"], traces[k])
        assert traces[k].shape[0] == rep["iteration"] == 2 * 16
        assert _rel(x_srv, x_o) <= tol, k
        assert abs(rep["residual_norm"] - rn_o) <= tol * rn_o, k


def oracle_replay_served(geo, y, seed, mu, trace, M=4, N=4):
    """Run the FP64 oracle on a served request's own draws (one pair per
    iteration: trace row = [1, i, j, ...]); returns (x, ||y - sum_j z^j||)."""
    from oracle import bsgd as OB
    from oracle import projector as OP
    og = OP.Geometry(**geo)
    prm = OB.Params(M, N, 1 / M, 1 / N, mu, seed=seed, pair_sampling="residual")
    sels = [OB.Selection([(int(t[1]), int(t[2]))], [None]) for t in trace]
    assert all(int(t[0]) == 1 for t in trace)
    ost = OB.bsgd(og, np.asarray(y, dtype=np.float64), prm, len(sels), replay=sels)
    return ost.x, ost.residual_norm()


@pytest.mark.gpu
def test_budget_and_slots_bound_admission():
    geo = cone(64, 90)
    y, _ = _data(geo, 4)
    p = params(epochs=3)
    need = B.bsgd_request_bytes(geo, 4, 4, p)
    srv = B.Server(budget_bytes=int(2.5 * need), max_slots=8)   # room for two at a time
    try:
        ids = [srv.submit(geo, 4, 4, params(epochs=3, seed=s), y) for s in range(5)]
        for i in ids:
            srv.wait(i)
        st = srv.stats()
        with pytest.raises(B.BSGDError) as ei:
            srv.submit(cone(128, 180), 4, 4, p, np.zeros(180 * 128 * 128, np.float32))
        assert ei.value.status == 5                              # over budget
    finally:
        srv.close()
    assert st["completed"] == 5
    assert st["peak_resident"] <= 2
    assert st["peak_bytes"] <= int(2.5 * need)


@pytest.mark.gpu
def test_bounded_wait_times_out_and_request_finishes():
    geo = cone(96, 180)
    y, _ = _data(geo, 8)
    srv = B.Server(budget_bytes=8 << 30, max_slots=4)
    try:
        rid = srv.submit(geo, 4, 4, params(epochs=6), y)
        with pytest.raises(B.BSGDError) as ei:
            srv.wait(rid, timeout_ms=1)
        assert ei.value.status == 4
        x, rep = srv.wait(rid)
        assert rep["iteration"] == 6 * 16 and np.isfinite(x).all() and np.abs(x).max() > 0
    finally:
        srv.close()


@pytest.mark.gpu
def test_several_column_blocks_per_iteration_served():
    """Requests drawing 2 or 4 column blocks per iteration (the paper's Sec. 5
    and Sec. 6 settings, here with and without detector cells) served among a
    one-block request: each equals the plain solver's result and, replayed
    from its own draws, the FP64 oracle's (1e-5 FP32, 1e-2 BF16). More than 4
    blocks, or residual pairs with several blocks, are rejected at submit."""
    geo = cone(64, 96)
    y, gg = _data(geo, 9)
    y1, _ = _data(cone(48, 72), 10)
    p2 = B.SolveParams(alpha=1 / 4, gamma=2 / 4, epochs=3, rho=0.25, power_iters=10,
                       pair_sampling=B.PAIRS_UNIFORM, seed=11)
    p4 = B.SolveParams(alpha=1 / 4, gamma=4 / 4, epochs=2, rho=0.25, power_iters=10,
                       pair_sampling=B.PAIRS_UNIFORM, cells=B.CELLS_GEOMETRIC, n_cells=4,
                       storage=B.BF16, seed=12)
    srv = B.Server(budget_bytes=8 << 30, max_slots=8)
    try:
        ids = [srv.submit(geo, 4, 4, p2, y), srv.submit(cone(48, 72), 4, 4, params(seed=13), y1),
               srv.submit(geo, 4, 4, p4, y)]
        outs = [srv.wait(i) for i in ids]
        traces = [srv.read_trace(ids[0]), srv.read_trace(ids[2])]
        with pytest.raises(B.BSGDError) as ei:
            srv.submit(geo, 4, 8, B.SolveParams(alpha=1 / 4, gamma=5 / 8, pair_sampling=B.PAIRS_UNIFORM), y)
        assert ei.value.status == 1
        with pytest.raises(B.BSGDError) as ei:
            srv.submit(geo, 4, 4, B.SolveParams(alpha=1 / 4, gamma=2 / 4, pair_sampling=B.PAIRS_RESIDUAL), y)
        assert ei.value.status == 1
        st = srv.stats()
    finally:
        srv.close()
    assert st["completed"] == 3 and st["failed"] == 0
    assert outs[0][1]["iteration"] == 3 * 8 and outs[2][1]["iteration"] == 2 * 4
    for (x_srv, rep), prm in ((outs[0], p2), (outs[2], p4)):
        x_plain = np.zeros(gg.n_cols, dtype=np.float32)
        rp = B.bsgd_solve(gg, prm, y, x_plain)
        assert rep["updates"] == rp["updates"]
        assert _rel(x_srv, x_plain) <= (2e-3 if prm.storage == B.BF16 else 1e-5)
    # and against the FP64 oracle on the served requests' own draws and step:
    # two column blocks per iteration (FP32), and all four blocks with one
    # geometric detector quadrant per view and pair (BF16 storage)
    from oracle import bsgd as OB
    from oracle import projector as OP
    og = OP.Geometry(**geo)
    mv = gg.info.max_views_per_block
    for (x_srv, rep), prm, tr, kw, tol in (
            (outs[0], p2, traces[0], {}, 1e-5),
            (outs[2], p4, traces[1], dict(cells="geometric", n_cells=4), 1e-2)):
        sels = []
        for t in tr:
            n_p = int(t[0])
            pairs = [(int(t[1 + 2 * q]), int(t[2 + 2 * q])) for q in range(n_p)]
            cells = []
            for q, (i, _) in enumerate(pairs):
                nv = OP.row_block_views(og, 4, i).size
                c = np.array(t[1 + 2 * n_p + q * mv:1 + 2 * n_p + q * mv + nv], dtype=np.int64)
                cells.append(c if kw else None)
            sels.append(OB.Selection(pairs, cells))
        po = OB.Params(4, 4, prm.alpha, prm.gamma, rep["mu"], seed=prm.seed, **kw)
        ost = OB.bsgd(og, y.astype(np.float64), po, len(sels), replay=sels)
        assert _rel(x_srv, ost.x) <= tol
        if not kw:   # uniform pairs: the oracle's own sampler draws the same blocks
            assert [sorted(sel.pairs) for sel in sels] == \
                [sorted(OB.sample(og, po, k, None, None, None).pairs) for k in range(len(sels))]


@pytest.mark.gpu
def test_two_servers_on_one_device():
    """The first server on a device reads its request table from constant
    memory, a second one (alive at the same time) from global memory: both
    give the plain solver's result."""
    geo = cone(48, 72)
    y, gg = _data(geo, 8)
    p = params(seed=9)
    a = B.Server(budget_bytes=4 << 30, max_slots=4)
    b = B.Server(budget_bytes=4 << 30, max_slots=4)
    try:
        ia, ib = a.submit(geo, 4, 4, p, y), b.submit(geo, 4, 4, p, y)
        xa, _ = a.wait(ia)
        xb, _ = b.wait(ib)
    finally:
        b.close()
        a.close()
    x_plain = np.zeros(gg.n_cols, dtype=np.float32)
    B.bsgd_solve(gg, p, y, x_plain)
    assert _rel(xa, x_plain) <= 1e-5 and _rel(xb, x_plain) <= 1e-5


@pytest.mark.gpu
def test_age_priority_favours_the_oldest_request():
    """Round policy AGE: while two requests are resident the one submitted
    first advances every round and the other every second round. A long
    request L is submitted, then a shorter S of the same set-up: S's latency
    grows (it advances in every second round only), L is not slowed (it
    advances every round, as under the shared policy, in rounds that carry
    less work), and S's image is the same under both policies."""
    geo = cone(64, 90)
    y, _ = _data(geo, 4)
    out = {}
    for pol in (B.SERVE_SHARED, B.SERVE_AGE):
        srv = B.Server(budget_bytes=8 << 30, max_slots=4, priority=pol)
        try:
            # the first request warms the geometry and step caches, so that
            # S is admitted within a few rounds of L
            srv.wait(srv.submit(geo, 4, 4, params(seed=1, epochs=1), y))
            t0 = time.perf_counter()
            il = srv.submit(geo, 4, 4, params(seed=2, epochs=120), y)
            t1 = time.perf_counter()
            is_ = srv.submit(geo, 4, 4, params(seed=3, epochs=60), y)
            xs, _ = srv.wait(is_)
            ts = time.perf_counter() - t1
            srv.wait(il)
            tl = time.perf_counter() - t0
        finally:
            srv.close()
        out[pol] = (ts, tl, xs)
    (ts_sh, tl_sh, xs_sh), (ts_age, tl_age, xs_age) = out[B.SERVE_SHARED], out[B.SERVE_AGE]
    assert ts_age > 1.2 * ts_sh, (ts_age, ts_sh)
    assert tl_age <= 1.1 * tl_sh, (tl_age, tl_sh)
    assert _rel(xs_age, xs_sh) <= 1e-5
