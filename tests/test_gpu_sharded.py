"""The sharded Lloyd step through the library: two ranks sharing the one GPU.

Two processes (torch.distributed, gloo, world size 2) each hold a contiguous
shard of the points and all k centroids. Each step every rank calls
kmeans_step_partial on its shard, the two partials buffers are summed through
host memory (gloo), and every rank calls kmeans_apply_partials on the sum
(paper_1109_0778_b300.sharded.ShardedLloyd). The exchange happens on the host
between launches, so no kernel of one process ever waits for the other.

Per step (teacher forcing, as the single-device parity tests) the gathered
assignment, the counts, the new centroids and the objective are checked against
the FP64 oracle's full-data step for the same input centroids; both ranks must
hold identical centroids after every step, and the changed count must equal the
number of labels that differ from the previous step's.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WORLD = 2
TESTS = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(TESTS)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gather_labels(dist, a, n, world, rank):
    from paper_1109_0778_b300.sharded import shard_bounds

    sizes = [shard_bounds(n, r, world)[1] - shard_bounds(n, r, world)[0] for r in range(world)]
    m = max(sizes)
    buf = torch.full((m,), -1, dtype=torch.int32)
    buf[: sizes[rank]] = a.cpu()
    parts = [torch.zeros(m, dtype=torch.int32) for _ in range(world)]
    dist.all_gather(parts, buf)
    return np.concatenate([p[:sz].numpy() for p, sz in zip(parts, sizes)])


def _child(rank, world, port, case):
    for p in (ROOT, TESTS):
        if p not in sys.path:
            sys.path.insert(0, p)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import parity
        import synth
        from paper_1109_0778_b300.sharded import ShardedLloyd, shard_bounds

        torch.cuda.set_device(0)
        prec, det, n, d, k, steps = case
        X = synth.mixture(7000 + n + d + k, n, d, k, 8.0, 1.0)
        lo, hi = shard_bounds(n, rank, world)
        Xd = torch.from_numpy(X[lo:hi].copy()).cuda()
        Cd = torch.from_numpy(X[:k].copy()).cuda()
        sl = ShardedLloyd(Xd, Cd, precision=prec, deterministic=det)
        ref = oracle.oracle()
        prev = None
        for it in range(steps):
            C_in = Cd.cpu().numpy().astype(np.float64)
            st = sl.step()
            a = _gather_labels(dist, sl.assign, n, world, rank)
            parity.check_assign(ref, X, C_in, a)
            parity.check_update(ref, X, C_in, a, Cd.cpu().numpy(), sl.sums.cpu().numpy(), sl.counts.cpu().numpy())
            parity.check_objective(ref, X, C_in, a, st["objective"])
            want_changed = n if prev is None else int((a != prev).sum())
            assert st["n_changed"] == want_changed, (it, st["n_changed"], want_changed)
            mine = Cd.cpu()
            other = mine.clone()
            dist.broadcast(other, src=0)
            assert torch.equal(mine, other), "ranks hold different centroids"
            prev = a
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", [
    ("fp32", False, 20001, 40, 64, 4),
    ("bf16", False, 20000, 128, 200, 4),
    ("bf16", True, 20001, 33, 129, 4),
    ("fp8", False, 30001, 64, 300, 4),
])
def test_two_ranks_on_one_gpu_match_the_oracle(case):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp

    mp.start_processes(_child, args=(WORLD, _free_port(), case), nprocs=WORLD, join=True, start_method="spawn")
