"""Owner-computes sharding (Sec. 2, Fig. 1): the host logic, on CPU gloo ranks.

Each rank owns a contiguous run of column blocks and computes, with the FP64
oracle's projector, only the FP, BP and update of its own drawn pairs; the
ranks sum their parts of sum_j z^j with one all-reduce per iteration
(paper_1903_11874_gb300.shard drives the steps and the exchange). With 2 and 4
ranks the image, gathered over the ranks, equals the single-process oracle
trajectory (oracle/bsgd.py) to 1e-12.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

ITERS = 24


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def problem():
    sys.path.insert(0, ROOT)
    from oracle import bsgd as OB
    from oracle import projector as OP
    from paper_1903_11874_gb300 import synth
    # the paper's 2D set-up (Sec. 3.1): fan beam, 16^2, 36 views, 30 elements
    og = OP.Geometry("fan2d", 16, 16, 1, 1.0, 1.0, 1.0, 36, 30, 1, 1.0, 1.0, dso=50.0, dsd=100.0)
    xt = synth.ellipse_phantom(16, 16, 6, 0).reshape(-1)
    y = OP.fp(og, xt).reshape(-1)
    mu = 0.25 * OB.step_strip(og, 4)
    return og, y, mu


def params(mu, cells):
    from oracle import bsgd as OB
    # two row blocks and two column blocks per iteration: pairs of different
    # owners meet in one iteration
    return OB.Params(4, 4, 0.5, 0.5, mu, seed=13, cells="uniform" if cells else "none",
                     n_cells=2 if cells else 1)


class OracleShard:
    """One rank's pieces of a sharded iteration, in FP64 with the oracle's
    projector (test side): z^J, r~^J of the owned blocks, replicated r, g."""

    def __init__(self, og, y, prm):
        from oracle import bsgd as OB
        self.OB, self.og, self.prm = OB, og, prm
        self.y = np.asarray(y, dtype=np.float64)
        self.r = self.y.copy()
        self.z = np.zeros((prm.N, og.n_rows))
        self.rt = np.zeros((prm.N, og.n_rows))
        self.g = np.zeros(og.n_cols)
        self.it = 0

    def set_shard(self, owned):
        self.owned = set(owned)
        return self.og.n_rows

    def shard_begin(self, x, buf):
        from oracle import projector as OP
        OB, og, prm = self.OB, self.og, self.prm
        self.sel = OB.sample(og, prm, self.it, None, None, None)
        self.rows = [OB.selection_rows(og, prm, i, c) for (i, _), c in zip(self.sel.pairs, self.sel.cells)]
        xv = x.numpy()
        for (i, j), R in zip(self.sel.pairs, self.rows):
            if j in self.owned:
                self.z[j, R] = OP.fp_rows(og, xv, R, OP.column_block(og, prm.N, j))
        self.U = np.unique(np.concatenate(self.rows))
        b = buf.numpy()
        b[:] = 0.0
        mine = sorted(self.owned)
        b[self.U] = self.z[mine][:, self.U].sum(axis=0) if mine else 0.0

    def shard_end(self, x, buf):
        from oracle import projector as OP
        og, prm = self.og, self.prm
        xv, b = x.numpy(), buf.numpy()
        self.r[self.U] = self.y[self.U] - b[self.U]
        for (i, j), R in zip(self.sel.pairs, self.rows):
            if j in self.owned:
                OP.bp_rows(og, self.r[R] - self.rt[j, R], R, OP.column_block(og, prm.N, j), out=self.g)
                self.rt[j, R] = self.r[R]
        for j in sorted({j for _, j in self.sel.pairs}):
            if j in self.owned:
                vox = OP.column_block_voxels(og, prm.N, j)
                xv[vox] += prm.mu * self.g[vox]
        self.it += 1


def _rank(rank, world, port, cells, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1903_11874_gb300 import shard
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        og, y, mu = problem()
        prm = params(mu, cells)
        work = OracleShard(og, y, prm)
        owned = shard.owned_blocks(prm.N, rank, world)
        solver = shard.ShardedSolver(work, owned, shard.Exchange(), torch.empty(0, dtype=torch.float64))
        x = torch.zeros(og.n_cols, dtype=torch.float64)
        solver.block_step(x, ITERS)
        from oracle import projector as OP
        mine = [OP.column_block_voxels(og, prm.N, j) for j in owned]
        others = np.setdiff1d(np.arange(og.n_cols), np.concatenate(mine) if mine else [])
        assert not x.numpy()[others].any()            # only the owned voxels moved
        dist.all_reduce(x)
        out.put((rank, x.numpy().copy(), float(np.linalg.norm(work.r))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,cells", [(2, False), (4, False), (2, True)])
def test_sharded_ranks_equal_the_single_process_oracle(world, cells):
    from oracle import bsgd as OB
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, cells, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    og, y, mu = problem()
    ref = OB.bsgd(og, y, params(mu, cells), ITERS)
    for _, x, rn in res:
        np.testing.assert_allclose(x, ref.x, rtol=0, atol=1e-12 * np.abs(ref.x).max())
        assert abs(rn - ref.residual_norm()) <= 1e-12 * ref.residual_norm()


def test_owned_blocks_partition_the_columns():
    sys.path.insert(0, ROOT)
    from paper_1903_11874_gb300 import shard
    for N in (1, 4, 7, 8, 16):
        for world in (1, 2, 3, 4, 8):
            parts = [shard.owned_blocks(N, r, world) for r in range(world)]
            assert sorted(sum(parts, [])) == list(range(N))
            assert all(b == a + 1 for p in parts for a, b in zip(p, p[1:]))
    with pytest.raises(ValueError):
        shard.owned_blocks(8, 2, 2)
