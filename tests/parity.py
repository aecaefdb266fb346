"""Step-level parity of the GPU library against the FP64 oracle (teacher forcing).

The GPU and FP64 trajectories may part ways after one near-tie, so parity is
checked one step at a time: the oracle is given the GPU's own input centroids
C^t (FP32 -> FP64 exactly) and
  - every GPU assignment must equal the oracle's argmin, except at points whose
    FP64 relative top-2 gap (D2 - D1) / D2 is below 1e-6 (counted, reported);
  - counts must equal the oracle's counts for the GPU's assignment exactly;
  - each new centroid coordinate must be within 1e-5 of the FP64 member mean,
    relative to max_t of the mean |x_it| over the cluster (empty clusters keep
    C^t bit for bit);
  - sums within the same relative bound times the count, and the objective
    J(a^t, C^t) within 1e-6 relative of the oracle's value for the GPU's a^t.
"""
from __future__ import annotations

import numpy as np

GAP_TOL = 1e-6
CENTROID_TOL = 1e-5
OBJECTIVE_TOL = 1e-6


def member_scale(X, a, k, chunk=1 << 18):
    """max_t of mean |x_it| over the members of each cluster (0 for empty clusters)."""
    import torch

    d = X.shape[1]
    acc = torch.zeros((k, d), dtype=torch.float64)
    at = torch.from_numpy(np.ascontiguousarray(a, dtype=np.int64))
    for r0 in range(0, X.shape[0], chunk):  # FP64 sums of |x| in row chunks (bounded host memory)
        xs = torch.from_numpy(X[r0:r0 + chunk]).abs().double()
        acc.index_add_(0, at[r0:r0 + chunk], xs)
    acc = acc.numpy()
    cnt = np.bincount(a, minlength=k).astype(np.float64)
    scale = np.zeros(k)
    nz = cnt > 0
    scale[nz] = (acc[nz] / cnt[nz, None]).max(axis=1)
    return scale, cnt


def check_assign(orc, X, C_in, a_gpu, rows=None):
    """Compare assignments (optionally only at `rows`); returns (n_near_tie_mismatch, n_checked)."""
    Xs = X if rows is None else X[rows]
    ag = a_gpu if rows is None else a_gpu[rows]
    ra, _, gap, _ = orc.assign(Xs, C_in)
    mism = ag != ra
    hard = mism & (gap >= GAP_TOL)
    assert not hard.any(), (
        f"{int(hard.sum())} assignments differ outside near-ties; first rows "
        f"{(np.flatnonzero(hard) if rows is None else rows[np.flatnonzero(hard)])[:8]}, "
        f"gpu {ag[hard][:8]} ref {ra[hard][:8]} gap {gap[hard][:8]}")
    return int(mism.sum()), int(len(ag))


def check_update(orc, X, C_in, a_gpu, C_out, sums_gpu, counts_gpu, empty_rtol=0.0):
    """Counts, sums and the new centroids against the oracle's update for the GPU's assignment.

    empty_rtol: empty clusters keep their centroid exactly (0), or within this distance relative
    to the row's largest coordinate when C_in comes from another run (whose reduce order may
    differ in the last bits, and so may the trajectory at a near-tie)."""
    k = C_in.shape[0]
    assert a_gpu.min() >= 0 and a_gpu.max() < k
    sums_ref, counts_ref, C_ref = orc.update(X, a_gpu, C_in)
    assert np.array_equal(counts_gpu.astype(np.int64), counts_ref), "counts differ"
    assert counts_gpu.sum() == X.shape[0]
    scale, cnt = member_scale(X, a_gpu, k)
    err = np.abs(C_out.astype(np.float64) - C_ref).max(axis=1)
    nz = cnt > 0
    bad = nz & (err > CENTROID_TOL * np.maximum(scale, np.finfo(np.float64).tiny))
    assert not bad.any(), f"centroid tolerance exceeded for clusters {np.flatnonzero(bad)[:8]}: {err[bad][:8]} vs {scale[bad][:8]}"
    keep = C_in[~nz].astype(np.float32)
    if empty_rtol == 0.0:
        assert np.array_equal(C_out[~nz], keep), "empty clusters must keep their centroid"
    else:
        rowmax = np.abs(keep.astype(np.float64)).max(axis=1, keepdims=True)
        dev = np.abs(C_out[~nz].astype(np.float64) - keep) - empty_rtol * rowmax
        assert np.all(dev <= 0.0), f"empty clusters moved: {np.abs(C_out[~nz] - keep).max()}"
    serr = np.abs(sums_gpu.astype(np.float64) - sums_ref).max(axis=1)
    assert np.all(serr <= CENTROID_TOL * scale * np.maximum(cnt, 1) + 1e-30), "sums tolerance exceeded"
    return float(err[nz].max() / max(scale[nz].max(), 1e-300)) if nz.any() else 0.0


def check_objective(orc, X, C_in, a_gpu, J_gpu):
    J_ref = orc.objective(X, C_in, a_gpu)
    assert abs(J_gpu - J_ref) <= OBJECTIVE_TOL * max(abs(J_ref), 1e-300), (J_gpu, J_ref)
    return J_ref
