"""A bounded device wait that runs out returns KM_ETIMEOUT and leaves the context usable.

KM_DEBUG_STALL makes the tensor-core epilogue wait (50 ms limit) on an mbarrier that
nothing arrives on; every role then gives up, drains what it issued, frees its
tensor memory and returns. In the one-launch path of small FP32 problems it makes the
first grid barrier wait for one CTA more than the grid holds; every CTA gives up after
its 1 s limit and returns. No GPU fault, trap or endless loop is involved.
"""
import os

import numpy as np
import pytest

import parity
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_cleanly(ref):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans as km

    X = synth.mixture(3, 4000, 32, 12, 6.0, 1.0)
    Xd = torch.from_numpy(X).to("cuda:0")
    C = torch.from_numpy(X[:12].copy()).to("cuda:0")
    C_before = C.clone()
    os.environ["KM_DEBUG_STALL"] = "1"
    try:
        with pytest.raises(km.KMeansError) as e:
            km.step(Xd, C, precision="bf16")
        assert e.value.status == km.KM_ETIMEOUT
    finally:
        del os.environ["KM_DEBUG_STALL"]
    assert torch.equal(C, C_before), "C must hold its value on entry after a timeout"
    # the context is still usable and the next call is correct
    out = km.step(Xd, C, precision="bf16")
    parity.check_assign(ref, X, C_before.cpu().numpy().astype(np.float64), out.assign.cpu().numpy())


def test_small_path_grid_barrier_times_out_cleanly(ref):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans as km

    X = synth.mixture(4, 5000, 16, 8, 6.0, 1.0)  # a small FP32 problem: one cooperative launch per call
    Xd = torch.from_numpy(X).to("cuda:0")
    C = torch.from_numpy(X[:8].copy()).to("cuda:0")
    C_before = C.clone()
    os.environ["KM_DEBUG_STALL"] = "1"
    try:
        with pytest.raises(km.KMeansError) as e:
            km.run(Xd, C, 5)
        assert e.value.status == km.KM_ETIMEOUT
    finally:
        del os.environ["KM_DEBUG_STALL"]
    assert torch.equal(C, C_before), "C must hold its value on entry after a timeout"
    out = km.run(Xd, C, 5)
    assert out.stats["launches"] == 1 and out.stats["iters_done"] == 5
    r = ref.run(X, C_before.cpu().numpy().astype(np.float64), 5)
    assert (out.assign.cpu().numpy() != r["assign"]).sum() <= 2
