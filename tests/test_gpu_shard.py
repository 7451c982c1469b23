"""Owner-computes sharding on the GPU (bsgd_state_set_shard, bsgd_shard_begin /
_end), against the FP64 oracle.

One process owning every column block, and two processes on the one GPU each
owning half of them, exchanging their parts of sum_j z^j through gloo on the
host (the kernels of one process never wait on the other's). Uniform draws
are the same on both sides, so whole trajectories are compared: the gathered
image within 1e-5 of the oracle's.
"""
import os
import socket
import sys

import numpy as np
import pytest

from helpers import gpu_geom, oracle_geom, rel_l2, spec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ITERS = 24


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def setup():
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from oracle import bsgd as OB
    from oracle import projector as OP
    from paper_1903_11874_gb300 import synth
    s = spec("cone_small")
    og = oracle_geom(s)
    xt = synth.ellipsoid_phantom(og.nx, og.ny, og.nz, 6, seed=0).astype(np.float64).reshape(-1)
    y = OP.fp(og, xt).reshape(-1).astype(np.float32)
    mu = 0.25 * OB.step_strip(og, s["N"], 1.0, 30)
    return s, og, y, mu


def gpu_params(B, mu, cells):
    # two row blocks and two column blocks per iteration (4 pairs)
    return B.SolveParams(alpha=0.5, gamma=0.5, step_rule=B.STEP_FIXED, mu=mu, seed=21,
                         cells=B.CELLS_UNIFORM if cells else B.CELLS_NONE, n_cells=4 if cells else 1)


def oracle_run(og, y, mu, cells):
    from oracle import bsgd as OB
    prm = OB.Params(4, 4, 0.5, 0.5, mu, seed=21, cells="uniform" if cells else "none",
                    n_cells=4 if cells else 1)
    return OB.bsgd(og, y.astype(np.float64), prm, ITERS)


@pytest.mark.parametrize("cells", [False, True])
def test_one_process_owning_every_block(cells):
    from paper_1903_11874_gb300 import binding as B
    from paper_1903_11874_gb300 import shard
    s, og, y, mu = setup()
    gg = gpu_geom(s)
    st = B.State(gg, gpu_params(B, mu, cells), torch.from_numpy(y).cuda())
    solver = shard.ShardedSolver(st, shard.owned_blocks(gg.N, 0, 1), lambda b: b,
                                 torch.empty(0, device="cuda:0"))
    x = torch.zeros(gg.n_cols, device="cuda:0")
    solver.block_step(x, ITERS)
    torch.cuda.synchronize()
    ref = oracle_run(og, y, mu, cells)
    assert rel_l2(x.cpu().numpy(), ref.x) <= 1e-5
    assert abs(st.query()["residual_norm"] - ref.residual_norm()) <= 1e-5 * ref.residual_norm()
    with pytest.raises(B.BSGDError):          # a sharded state steps only through begin / end
        st.block_step(x, 1)


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    from paper_1903_11874_gb300 import binding as B
    from paper_1903_11874_gb300 import shard
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        s, og, y, mu = setup()
        gg = gpu_geom(s)
        solver = shard.sharded_state(gg, gpu_params(B, mu, False), torch.from_numpy(y).cuda(),
                                     rank, world)
        x = torch.zeros(gg.n_cols, device="cuda:0")
        solver.block_step(x, ITERS)
        full = shard.gather_image(x)
        torch.cuda.synchronize()
        out.put((rank, full.cpu().numpy(), solver.owned))
    finally:
        dist.destroy_process_group()


def test_two_processes_each_owning_half_the_blocks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=600) for _ in range(2)), key=lambda t: t[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert [r[2] for r in res] == [[0, 1], [2, 3]]
    _, og, y, mu = setup()
    ref = oracle_run(og, y, mu, False)
    for _, x, _ in res:
        assert rel_l2(x, ref.x) <= 1e-5


def _nccl_one(port, out):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    from paper_1903_11874_gb300 import binding as B
    from paper_1903_11874_gb300 import shard
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")   # no NVLink multicast objects
    torch.cuda.set_device(0)
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    try:
        s, og, y, mu = setup()
        gg = gpu_geom(s)
        solver = shard.sharded_state(gg, gpu_params(B, mu, False), torch.from_numpy(y).cuda(), 0, 1)
        assert solver.exchange.backend == "nccl"
        x = torch.zeros(gg.n_cols, device="cuda:0")
        solver.block_step(x, ITERS)
        torch.cuda.synchronize()
        out.put(x.cpu().numpy())
    finally:
        dist.destroy_process_group()


def test_nccl_exchange_on_the_device():
    """The exchange through NCCL (an in-place all-reduce of the device buffer),
    one process owning every block: the same trajectory as the oracle."""
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_nccl_one, args=(_free_port(), q))
    p.start()
    x = q.get(timeout=600)
    p.join(120)
    assert p.exitcode == 0
    _, og, y, mu = setup()
    assert rel_l2(x, oracle_run(og, y, mu, False).x) <= 1e-5


def test_sharded_state_refuses_a_warm_start_and_other_draws():
    """A sharded state starts from x = 0 (its memories would need every
    process's A^j x0) and draws uniform pairs only: a non-zero image at the
    first step, and a later switch to residual-weighted pairs or to a replayed
    trace, are refused with INVALID_ARG."""
    from paper_1903_11874_gb300 import binding as B
    from paper_1903_11874_gb300 import shard
    s, og, y, mu = setup()
    gg = gpu_geom(s)
    st = B.State(gg, gpu_params(B, mu, False), torch.from_numpy(y).cuda())
    solver = shard.ShardedSolver(st, shard.owned_blocks(gg.N, 0, 1), lambda b: b,
                                 torch.empty(0, device="cuda:0"))
    x = torch.zeros(gg.n_cols, device="cuda:0")
    x[gg.n_cols // 2] = 1.0
    with pytest.raises(B.BSGDError) as e:
        solver.block_step(x, 1)
    assert e.value.status == 1
    with pytest.raises(B.BSGDError):
        st.set_sampling(B.PAIRS_RESIDUAL)
    with pytest.raises(B.BSGDError):
        st.set_replay(np.full((1, st.trace_stride), -1, dtype=np.int32))
    x.zero_()
    solver.block_step(x, 2)              # from zero it steps
    torch.cuda.synchronize()
    assert st.query()["iteration"] == 2
