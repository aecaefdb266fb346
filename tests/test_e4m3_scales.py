"""E4M3 centroid codes: one power-of-two scale per step versus one per centroid row.

The E4M3 path codes every centroid of a step with one power-of-two scale s
(the smallest with max_{j,t} |c_jt| / s <= 448). Because the scale is a power
of two, a per-row scale s_j <= s changes a code only where the shared scale
puts an element below E4M3's smallest normal (2^-6 s): every other element is
the same binary fraction shifted in exponent. And the per-row grid contains the
shared grid there, so each element's error can only shrink. The assignment's
rigorous margin uses the step's largest residual DCmax = max_j ||c~_j - c_j||,
which the largest centroids set; so on centroid sets whose norms span 2^10 the
margin's step maxima are the ones per-row scales would give. The CPU test
pins that argument with torch's E4M3 conversion. The GPU test runs E4M3 steps
on such a mixture against the FP64 oracle: with the assignment's per-centroid
error terms (each candidate's own h_j, norms and residual instead of the step
maxima) rows near the small centroids stay unflagged.
"""
import math

import numpy as np
import pytest

import parity
import synth

torch = pytest.importorskip("torch")


def _pow2_scale(amax: float) -> float:
    """Smallest power of two s with amax / s <= 448 (the codes' scale rule)."""
    m, e = math.frexp(amax / 448.0)
    return math.ldexp(1.0, e - 1 if m == 0.5 else e)


def _codes(C: np.ndarray, scales: np.ndarray) -> np.ndarray:
    """RN E4M3 codes of C / s, dequantised (s: power-of-two row scales, so both scalings are exact)."""
    Ct = torch.from_numpy(C.astype(np.float32))
    st = torch.from_numpy(scales.astype(np.float32))[:, None]
    q = (Ct / st).to(torch.float8_e4m3fn).to(torch.float32) * st
    return q.numpy().astype(np.float64)


@pytest.mark.parametrize("span", [10, 20])
def test_shared_scale_keeps_the_margin_of_per_row_scales(span):
    k, d = 128, 64
    mu = synth.means(0xE4A3 + span, k, d, 20.0)
    C = (mu * np.exp2(-span * np.arange(k) / (k - 1))[:, None]).astype(np.float32)
    norms = np.linalg.norm(C.astype(np.float64), axis=1)
    assert norms.max() / norms.min() > 2.0 ** (span - 1)
    s_shared = _pow2_scale(float(np.abs(C).max()))
    s_row = np.array([_pow2_scale(float(np.abs(r).max())) for r in C])
    assert np.all(s_row <= s_shared)
    q_sh = _codes(C, np.full(k, s_shared))
    q_row = _codes(C, s_row)
    C64 = C.astype(np.float64)
    r_sh = np.linalg.norm(q_sh - C64, axis=1)
    r_row = np.linalg.norm(q_row - C64, axis=1)
    # per element: equal where the shared scale keeps the element normal, never worse with per-row scales
    normal = np.abs(C64) >= 2.0 ** -6 * s_shared
    assert np.array_equal(q_sh[normal], q_row[normal])
    assert np.all(np.abs(q_row - C64) <= np.abs(q_sh - C64))
    # the margin's residual term: identical maxima (set by the largest centroids)
    assert r_sh.max() == r_row.max()
    assert np.argmax(r_sh) < k // 8
    # the smallest centroids keep residuals far below that maximum either way
    assert r_sh[-k // 8:].max() < 1e-2 * r_sh.max()
    # and the maximum norm of the codes, the other centroid term of the margin, is shared too
    assert np.linalg.norm(q_sh, axis=1).max() == np.linalg.norm(q_row, axis=1).max()


@pytest.mark.gpu
def test_e4m3_parity_with_centroid_norms_spanning_2_10(ref):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans as km

    n, d, k = 200_000, 64, 64
    X = synth.multiscale_mixture(0xE4A4, n, d, k, 20.0, 0.5, 10.0)
    Xd = torch.from_numpy(X).to("cuda:0")
    # one centroid per component: the first point of each (their norms span 2^10)
    _, comp = synth.mixture(0xE4A4, n, d, k, 20.0, 0.5, with_comp=True)
    first = np.array([np.flatnonzero(comp == c)[0] for c in range(k)])
    C0 = X[first].copy()
    norms = np.linalg.norm(C0.astype(np.float64), axis=1)
    assert norms.max() / norms.min() > 2.0 ** 9
    Cd = torch.from_numpy(C0).to("cuda:0")
    a, s, c = km.alloc_outputs(Xd, Cd)
    # a BF16 step first (a warm start, so that every step below codes C in E4M3)
    bf16_rate = km.step(Xd, Cd, a, s, c, precision="bf16").stats["n_flagged"] / n
    rates = []
    for it in range(3):
        C_in = Cd.cpu().numpy().astype(np.float64)
        out = km.step(Xd, Cd, a, s, c, precision="fp8", warm_start=True)
        ag = out.assign.cpu().numpy()
        parity.check_assign(ref, X, C_in, ag)
        parity.check_update(ref, X, C_in, ag, Cd.cpu().numpy(), out.sums.cpu().numpy(), out.counts.cpu().numpy())
        parity.check_objective(ref, X, C_in, ag, out.stats["objective"])
        assert out.stats["iters_bf16"] == 0
        rates.append(out.stats["n_flagged"] / n)
    # the FP32 path on the same data and centroids (its own margin)
    C_in = Cd.cpu().numpy().astype(np.float64)
    out = km.step(Xd, Cd, a, s, c, precision="fp32", warm_start=True)
    parity.check_assign(ref, X, C_in, out.assign.cpu().numpy())
    fp32_rate = out.stats["n_flagged"] / n
    print(f"centroid norms spanning 2^10: BF16 flag rate {bf16_rate:.4f}; "
          f"E4M3 flag rate per step {', '.join(f'{r:.4f}' for r in rates)}; FP32 {fp32_rate:.4f}")
    # per-centroid error terms: rows near the small centroids are decided by their own centroids'
    # bounds, not by those of the largest ones (which flagged 39% (BF16) and 79% (E4M3) of the points)
    assert bf16_rate < 0.01 and max(rates) < 0.01
