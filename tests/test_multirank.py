"""Host-side multi-rank logic on CPU (gloo, world size 2).

Covers the two things a multi-process run depends on without needing a GPU:

* the sharded Lloyd step's exchange (each rank assigns its contiguous range of
  points and forms partial sums and counts; one all-reduce of k*d + k + 1 values
  and the same divide on every rank give the full step, Sec. 2.4's keyed reduce
  split by rows and combined), checked against the oracle's full-data step;
* bench.py's rank helpers (max over ranks of the timed region, barrier, the
  whole-job aggregate of weak-scaling replicas);
* the sharded driver (paper_1109_0778_b300.sharded.ShardedLloyd): its exchange
  of the partials buffer and its stop rule, with the two library calls of a
  step replaced by an FP64 stand-in on CPU tensors (the library itself runs in
  tests/test_gpu_sharded.py, two ranks on the GPU).
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _sharded_step(rank, world, X, C):
    """One Lloyd step over rows [lo, hi) of X, combined across ranks."""
    import oracle

    ref = oracle.oracle()
    n = X.shape[0]
    lo, hi = rank * n // world, (rank + 1) * n // world
    a, _, _, _ = ref.assign(X[lo:hi], C)
    sums, counts, _ = ref.update(X[lo:hi], a, C)
    J = ref.objective(X[lo:hi], C, a)
    packed = torch.from_numpy(np.concatenate([sums.ravel(), counts.astype(np.float64), [J]]))
    dist.all_reduce(packed, op=dist.ReduceOp.SUM)
    k, d = C.shape
    S = packed[: k * d].numpy().reshape(k, d)
    cnt = packed[k * d: k * d + k].numpy()
    Jall = float(packed[-1])
    Cnew = np.where(cnt[:, None] > 0, S / np.maximum(cnt, 1)[:, None], C)
    # the assignment itself is gathered only to check it
    sizes = [(r + 1) * n // world - r * n // world for r in range(world)]
    gathered = [torch.zeros(sz, dtype=torch.int32) for sz in sizes]
    if len(set(sizes)) == 1:
        dist.all_gather(gathered, torch.from_numpy(a))
    else:  # gloo all_gather wants equal sizes: pad to the largest shard
        m = max(sizes)
        buf = torch.full((m,), -1, dtype=torch.int32)
        buf[: hi - lo] = torch.from_numpy(a)
        padded = [torch.zeros(m, dtype=torch.int32) for _ in range(world)]
        dist.all_gather(padded, buf)
        gathered = [p[:sz] for p, sz in zip(padded, sizes)]
    return np.concatenate([g.numpy() for g in gathered]), cnt, Cnew, Jall


def _worker(rank, world, port, n):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle
        import synth

        # --- sharded step == full step
        X = synth.mixture(11, n, 8, 6, 5.0, 1.0)
        C = X[:6].astype(np.float64)
        a, cnt, Cnew, J = _sharded_step(rank, world, X, C)
        full = oracle.oracle().step(X, C)
        assert np.array_equal(a, full["assign"])
        assert np.array_equal(cnt.astype(np.int64), full["counts"])
        scale = np.abs(X).max()
        assert np.max(np.abs(Cnew - full["C"])) <= 1e-12 * scale
        assert abs(J - full["objective"]) <= 1e-12 * abs(full["objective"])
        # every rank holds the same centroids after the exchange
        mine = torch.from_numpy(Cnew.copy())
        other = mine.clone()
        dist.broadcast(other, src=0)
        assert torch.equal(mine, other)

        # --- bench.py's rank helpers
        t = bench.max_over_ranks(dist, 1.0 + rank, None)
        assert t == float(world)
        bench.barrier(dist)
        assert bench.aggregate_rate(units_per_rank=10, world=world, t_max=t) == 10 * world / t
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n", [1000, 1001])
def test_two_rank_sharded_step_and_bench_helpers(n):
    mp.start_processes(_worker, args=(WORLD, _free_port(), n), nprocs=WORLD, join=True, start_method="spawn")


def _driver_worker(rank, world, port, n, tol):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import synth
        from paper_1109_0778_b300.sharded import ShardedLloyd, shard_bounds

        ref = oracle.oracle()

        class OracleShard(ShardedLloyd):
            """The driver with its two library calls replaced by FP64 CPU arithmetic that fills the
            same partials buffer layout (k*d sums, k counts, objective, changed count)."""

            def partial(self):
                Xs = self.X.numpy()
                C64 = self.C.numpy().astype(np.float64)
                a, _, _, _ = ref.assign(Xs, C64)
                sums, counts, _ = ref.update(Xs, a, C64)
                J = ref.objective(Xs, C64, a)
                changed = len(a) if self.steps_done == 0 else int((a != self.assign.numpy()).sum())
                k, d = self.C.shape
                self.part.copy_(torch.from_numpy(np.concatenate([sums.ravel(), counts.astype(np.float64),
                                                                 [J, float(changed)]])))
                self.assign.copy_(torch.from_numpy(a.astype(np.int32)))
                return {"n_flagged": 0, "n_full": 0, "ms": 0.0}

            def apply(self):
                k, d = self.C.shape
                p = self.part.numpy()
                S, cnt = p[: k * d].reshape(k, d), p[k * d: k * d + k]
                old = self.C.numpy().astype(np.float64)
                new = np.where(cnt[:, None] > 0, S / np.maximum(cnt, 1)[:, None], old).astype(np.float32)
                shift = float(np.sqrt(((new.astype(np.float64) - old) ** 2).sum(axis=1)).max())
                self.C.copy_(torch.from_numpy(new))
                return {"objective": float(p[k * d + k]), "n_changed": int(p[k * d + k + 1]), "shift": shift,
                        "n_empty": int((cnt == 0).sum())}

        X = synth.mixture(23, n, 6, 5, 6.0, 1.0)
        lo, hi = shard_bounds(n, rank, world)
        C = torch.from_numpy(X[:5].copy())
        sh = OracleShard(torch.from_numpy(X[lo:hi].copy()), C, precision="fp32")
        assert sh.via_host
        st = sh.run(30, tol=tol)
        # every rank stopped after the same step with the same centroids
        steps = torch.tensor([st["iters_done"]], dtype=torch.int64)
        both = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(both, steps)
        assert len({int(b) for b in both}) == 1
        other = C.clone()
        dist.broadcast(other, src=0)
        assert torch.equal(C, other)
        # the same run on the whole data set in one process, step by step
        Cf = X[:5].astype(np.float64)
        prev = None
        for it in range(30):
            out = ref.step(X, Cf)
            shift = float(np.sqrt(((out["C"].astype(np.float32).astype(np.float64) - Cf) ** 2).sum(axis=1)).max())
            changed = n if prev is None else int((out["assign"] != prev).sum())
            prev = out["assign"]
            Cf = out["C"].astype(np.float32).astype(np.float64)
            if tol > 0 and (changed == 0 or shift <= tol):
                break
        assert st["iters_done"] == it + 1, (st["iters_done"], it + 1)
        assert np.max(np.abs(C.numpy() - Cf)) <= 1e-6 * np.abs(X).max()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n,tol", [(2000, 1e-9), (2001, 0.0)])
def test_sharded_driver_exchange_and_stop_rule(n, tol):
    mp.start_processes(_driver_worker, args=(WORLD, _free_port(), n, tol), nprocs=WORLD, join=True,
                       start_method="spawn")


def test_shard_bounds_cover_rows_once():
    from paper_1109_0778_b300.sharded import shard_bounds

    for n in (1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            b = [shard_bounds(n, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[r][1] == b[r + 1][0] for r in range(world - 1))
            assert max(h - lo for lo, h in b) - min(h - lo for lo, h in b) <= 1


def test_single_rank_helpers_are_identity():
    import bench

    assert bench.max_over_ranks(None, 3.5) == 3.5
    bench.barrier(None)
    assert bench.aggregate_rate(units_per_rank=7, world=1, t_max=2.0) == 3.5
