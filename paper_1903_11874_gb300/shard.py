"""Owner-computes sharding of BSGD across processes (one process per GPU).

Sec. 2 of the paper (Fig. 1) spreads the column blocks x_J over servant nodes
that compute A_I^J x_J, while a master node sums those parts into the residual
r_I of the selected rows. Here every process owns a contiguous run of column
blocks and keeps x_J, g_J, z^J and the snapshots r~^J of its own blocks; the
residual r is replicated. One iteration:

  1. every process draws the same pairs (uniform draws from the shared seed),
     forward projects the drawn pairs of its own blocks and writes its part
     sum_{J owned} z^J of the rows whose z changed into an exchange buffer;
  2. one all-reduce sums the buffers over the processes: the master's sum;
  3. every process forms r = y - sum_j z^j on those rows, back projects the
     change r - r~^J of its own drawn pairs into g_J and steps x_J.

The gradient needs no collective: g_J stays with the owner of J. The device
work runs in the library's kernels (bsgd_shard_begin / bsgd_shard_end); this
module only orchestrates the three steps and calls torch.distributed for the
sum. The per-process work is an object with set_shard / shard_begin /
shard_end (binding.State is the CUDA one).
"""


def owned_blocks(N, rank, world):
    """Column blocks of process `rank` of `world`: [rank N / W, (rank + 1) N / W)."""
    if not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    return list(range(rank * N // world, (rank + 1) * N // world))


class Exchange:
    """Sum of a buffer over a process group: in place for CPU tensors and for
    NCCL, through a pinned host copy for device tensors on gloo."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.backend = dist.get_backend(group)
        self.host = None

    def __call__(self, buf):
        if not buf.is_cuda or self.backend == "nccl":
            self.dist.all_reduce(buf, group=self.group)
            return buf
        import torch
        if self.host is None or self.host.numel() != buf.numel() or self.host.dtype != buf.dtype:
            self.host = torch.empty(buf.numel(), dtype=buf.dtype, pin_memory=True)
        self.host.copy_(buf)
        self.dist.all_reduce(self.host, group=self.group)
        buf.copy_(self.host)
        return buf


class ShardedSolver:
    """BSGD iterations of one process of an owner-computes group.

    work: the per-process state (binding.State, or any object with the same
    set_shard / shard_begin / shard_end methods); owned: its column blocks;
    exchange: callable summing a buffer over the group in place; buffer_like:
    a tensor whose device and dtype the exchange buffer takes."""

    def __init__(self, work, owned, exchange, buffer_like):
        import torch
        self.work, self.owned, self.exchange = work, list(owned), exchange
        n = work.set_shard(self.owned)
        self.buf = torch.zeros(n, dtype=buffer_like.dtype, device=buffer_like.device)

    def block_step(self, x, n_iters):
        for _ in range(int(n_iters)):
            self.work.shard_begin(x, self.buf)
            self.exchange(self.buf)
            self.work.shard_end(x, self.buf)
        return x


def sharded_state(geom, params, y, rank, world, group=None):
    """A ShardedSolver over the CUDA library for process `rank` of `world`
    (torch.distributed initialised): it owns owned_blocks(N, rank, world)."""
    import torch
    from . import binding as B
    st = B.State(geom, params, y)
    return ShardedSolver(st, owned_blocks(geom.N, rank, world), Exchange(group),
                         torch.empty(0, dtype=torch.float32, device=y.device))


def gather_image(x, group=None):
    """The whole image on every process: each process's x is zero outside its
    own blocks, so the sum over the group is the image."""
    import torch
    import torch.distributed as dist
    full = x.float().clone()
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        Exchange(group)(full)
    return full if full.dtype == torch.float32 else full.float()
