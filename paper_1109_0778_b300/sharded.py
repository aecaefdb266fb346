"""Lloyd k-means over several devices: one process per device, the points split
into contiguous shards, every device holding all k centroids.

This is the keyed reduce split into chunks whose partial results are merged by
a combine (Sec. 2.4, DeliteReduceElem's alloc / combine), with the runtime
spreading one loop over several devices (Sec. 2.4, the Delite runtime). One
step on every rank:

1. ``kmeans_step_partial`` on the rank's shard: its assignment and a partials
   buffer of k*d FP64 sums, k counts, the objective and the changed count;
2. one sum all-reduce of that buffer across the ranks (torch.distributed: NCCL
   reduces the device buffer in place; another backend, e.g. gloo, goes through
   a host copy);
3. ``kmeans_apply_partials`` on the reduced buffer: the FP64 divide, which gives
   every rank the same new centroids bit for bit.

The stop rule reads the reduced buffer (changed count) and the shift, which are
the same on every rank, so every rank stops after the same step. All arithmetic
runs in the library's kernels; this module only sequences the calls and the
collective.
"""
from __future__ import annotations

from . import kmeans as km


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """Rows [lo, hi) of rank ``rank``: contiguous, sizes differing by at most one."""
    return n * rank // world, n * (rank + 1) // world


class ShardedLloyd:
    """One rank's share of a sharded Lloyd run.

    X_shard: this rank's rows (contiguous CUDA float32, (n_r, d)); C: the
    centroids, identical on every rank on entry (CUDA float32 (k, d), updated in
    place). ``group``: the torch.distributed process group (None = default).
    After a step, ``assign`` holds the shard's labels and ``sums`` / ``counts``
    the whole data set's per-cluster sums and counts.
    """

    def __init__(self, X_shard, C, *, precision="bf16", recheck=True, deterministic=False, group=None,
                 stream=None):
        import torch
        import torch.distributed as dist

        k, d = C.shape
        dev = C.device
        self.X, self.C = X_shard, C
        self.assign = torch.zeros(X_shard.shape[0], dtype=torch.int32, device=dev)
        self.part = torch.zeros(km.partials_len(k, d), dtype=torch.float64, device=dev)
        self.sums = torch.empty(k, d, dtype=torch.float32, device=dev)
        self.counts = torch.empty(k, dtype=torch.int32, device=dev)
        self.opts = dict(precision=precision, recheck=recheck, deterministic=deterministic)
        self.group, self.stream, self.dist = group, stream, dist
        self.via_host = dist.get_backend(group) != "nccl"
        self.host = None
        if self.via_host:
            self.host = torch.empty(self.part.shape, dtype=torch.float64, pin_memory=self.part.is_cuda)
        self.steps_done = 0

    def partial(self) -> dict:
        """The shard's assignment and partials (the first step cold, later ones continuing from the
        previous step's labels and cached codes)."""
        later = self.steps_done > 0
        return km.step_partial(self.X, self.C, self.assign, self.part, warm_start=later, reuse_x=later,
                               stream=self.stream, **self.opts)

    def exchange(self) -> None:
        """Element-wise sum of every rank's partials buffer, left in ``part`` on every rank."""
        op = self.dist.ReduceOp.SUM
        if self.via_host:
            self.host.copy_(self.part)
            self.dist.all_reduce(self.host, op=op, group=self.group)
            self.part.copy_(self.host)
        else:
            self.dist.all_reduce(self.part, op=op, group=self.group)

    def apply(self) -> dict:
        return km.apply_partials(self.part, self.C, self.sums, self.counts, stream=self.stream)

    def step(self) -> dict:
        """One sharded Lloyd step; returns the whole data set's statistics (objective J(a^t, C^t),
        n_changed, shift, n_empty) and this shard's re-check counts."""
        ps = self.partial()
        self.exchange()
        st = self.apply()
        self.steps_done += 1
        st.update(n_flagged_shard=ps["n_flagged"], n_full_shard=ps["n_full"], ms_partial=ps["ms"])
        return st

    def run(self, iters: int, tol: float = 0.0) -> dict:
        """Up to ``iters`` steps; with tol > 0, stops after the first step whose assignment equals the
        previous step's or whose largest centroid shift is <= tol (the same step on every rank)."""
        st = None
        for _ in range(iters):
            st = self.step()
            if tol > 0 and (st["n_changed"] == 0 or st["shift"] <= tol):
                break
        st["iters_done"] = self.steps_done
        return st
