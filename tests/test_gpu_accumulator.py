"""The tensor-core accumulator model behind the near-tie margin, pinned on the GPU.

The margin of the BF16 / E4M3 assignment (km_assign_tc.cu) bounds the error of
the tensor core's FP32 accumulation of K products by gamma'_K * sum_k |a_k b_k|
with gamma'_K = K 2^-23 / (1 - K 2^-23): every addition may lose up to one unit
in the 23rd bit (truncation), twice the loss of round-to-nearest. These tests
run one 128 x 128 tile through the same operand layout, descriptors and MMA
sequence as the distance kernel (kmeans_probe_mma) and check

* the layout: integer operands give A B^T exactly;
* the rounding on hand-built sums (1 + 1.5 2^-24 in FP32 lies between two
  representable numbers; truncation gives 1, round-to-nearest 1 + 2^-23;
  E4M3 products 256 + 2^-15, 256 + 2^-16, 256 + 1.5 2^-16);
* the bound on adversarial sums that make a truncating accumulator lose almost a
  whole unit per addition (a first product P followed by K - 1 products just
  under two units of P's 23rd bit): the error nearly reaches gamma'_K, and an
  accumulator that kept one bit fewer would drop those products whole and
  exceed it;
* the bound on random operands with mixed exponents and signs.

The last test is a parity case built so that the exact score gaps sit just above
the margin: those points are decided by the tensor-core scores alone (no
re-check), so an accumulator looser than the model would assign some of them
to the wrong centroid.
"""
import numpy as np
import pytest

import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans

    return kmeans


def gamma_k(K):
    return K * 2.0 ** -23 / (1.0 - K * 2.0 ** -23)


def to_codes(a64, precision):
    """FP64 values that are exactly representable -> device code tensor (asserting exactness)."""
    t = torch.from_numpy(np.ascontiguousarray(a64, dtype=np.float64))
    q = t.to(torch.bfloat16) if precision == "bf16" else t.to(torch.float8_e4m3fn)
    assert torch.equal(q.double(), t), "operand not exactly representable"
    return q.contiguous().to(DEV)


def probe(km, A, B, precision):
    return km.probe_mma(to_codes(A, precision), to_codes(B, precision), precision=precision).cpu().double().numpy()


KS = {"bf16": (64, 128, 192, 256), "fp8": (128, 256, 384, 512)}


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_layout_integer_products_exact(km, precision):
    """Small integers: every product and partial sum is exact in FP32, so D must equal A B^T
    exactly (checks the swizzled K-major layout, K-block advance and descriptors)."""
    rng = np.random.default_rng(11)
    for K in KS[precision]:
        A = rng.integers(-15, 16, (128, K)).astype(np.float64)
        B = rng.integers(-15, 16, (128, K)).astype(np.float64)
        D = probe(km, A, B, precision)
        assert np.array_equal(D, A @ B.T), f"K={K}: {np.argwhere(D != A @ B.T)[:4]}"


def test_bf16_rounding_pins(km):
    """1 + 1.5 2^-24 (not representable in FP32): truncation gives 1, round-to-nearest 1 + 2^-23.
    The small product sits in the same MMA instruction (k = 1), in the next instruction of the
    same K block (k = 16) and in the next K block (k = 64). Either result is inside the model;
    the value is recorded in the test output."""
    K = 128
    A = np.zeros((128, K))
    B = np.zeros((128, K))
    for m, pos in enumerate((1, 16, 64)):
        A[m, 0] = 1.0
        A[m, pos] = 1.5 * 2.0 ** -24
    B[:, :] = 1.0
    D = probe(km, A, B, "bf16")
    for m, pos in enumerate((1, 16, 64)):
        assert D[m, 0] in (1.0, 1.0 + 2.0 ** -23), (pos, D[m, 0])
        print(f"bf16 1 + 1.5*2^-24 with the small term at k={pos}: {D[m, 0]!r}"
              f" ({'truncated' if D[m, 0] == 1.0 else 'rounded to nearest'})")
    # a representable sum is kept exactly wherever the small term sits
    A2 = np.zeros((128, K))
    for m, pos in enumerate((1, 16, 64)):
        A2[m, 0] = 1.0
        A2[m, pos] = 2.0 ** -23
    D2 = probe(km, A2, B, "bf16")
    assert all(D2[m, 0] == 1.0 + 2.0 ** -23 for m in range(3))


def test_fp8_rounding_pins(km):
    """E4M3 products around 256 = 16 x 16 (unit of the 23rd bit there: 2^-15):
    256 + 2^-15 is representable and kept; 256 + 2^-16 is half a unit (both rounding modes give
    256); 256 + 1.5 2^-16 gives 256 when truncated, 256 + 2^-15 when rounded to nearest."""
    K = 128
    A = np.zeros((128, K))
    B = np.zeros((128, K))
    small = {0: (2.0 ** -6, 2.0 ** -9), 1: (2.0 ** -7, 2.0 ** -9), 2: (6 * 2.0 ** -9, 2.0 ** -9)}  # 2^-15, 2^-16, 1.5*2^-16
    for m, (a, b) in small.items():
        for r, pos in enumerate((1, 32)):  # same instruction, next instruction
            row = 3 * r + m
            A[row, 0], B[row, 0] = 16.0, 16.0
            A[row, pos], B[row, pos] = a, b
    D = probe(km, A, B, "fp8")
    for r in range(2):
        assert D[3 * r + 0, 3 * r + 0] == 256.0 + 2.0 ** -15
        assert D[3 * r + 1, 3 * r + 1] == 256.0
        v = D[3 * r + 2, 3 * r + 2]
        assert v in (256.0, 256.0 + 2.0 ** -15), v
        print(f"fp8 256 + 1.5*2^-16 (small term in {'the same' if r == 0 else 'the next'} instruction): {v!r}")


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_adversarial_sum_within_gamma_k(km, precision):
    """A first product P followed by K - 1 products just under two units of P's 23rd bit: a
    truncating accumulator keeps one unit of each and drops the rest, an error of almost
    (K - 1) units, which gamma'_K sum|ab| still covers (one bit fewer would drop every small
    product whole: twice the bound). Rows vary where the large product sits and mix in signs."""
    if precision == "bf16":
        big, v = (1.0, 1.0), (1.9921875 * 2.0 ** -23, 1.0)       # products 1 and (2 - 2^-7) 2^-23
    else:
        big, v = (16.0, 16.0), (7 * 2.0 ** -9, 2.0 ** -8)       # products 256 and 1.75 2^-15
    rng = np.random.default_rng(5)
    for K in KS[precision]:
        A = np.zeros((128, K))
        B = np.zeros((128, K))
        for m in range(128):
            A[m, :] = v[0]
            B[m, :] = v[1]
            pos = 0 if m < 64 else int(rng.integers(0, K))
            A[m, pos], B[m, pos] = big
            if m % 4 == 3:  # a cancelling pair in the middle
                q = int(rng.integers(1, K))
                if q != pos:
                    A[m, q], B[m, q] = -big[0], big[1]
        D = probe(km, A, B, precision)
        exact = A @ B.T
        absum = np.abs(A) @ np.abs(B).T
        err = np.abs(D - exact)
        assert np.all(err <= gamma_k(K) * absum), f"K={K}: worst {np.max(err / (gamma_k(K) * absum)):.3f} of gamma'_K"
        diag = np.array([err[m, m] / (gamma_k(K) * absum[m, m]) for m in range(64)])
        print(f"{precision} K={K}: truncation-adversarial rows reach {diag.max():.3f} of gamma'_K")


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_random_mixed_exponents_within_gamma_k(km, precision):
    rng = np.random.default_rng(7)
    for K in KS[precision]:
        for trial in range(3):
            mant = rng.uniform(-1, 1, (2, 128, K))
            expo = rng.integers(-6, 5, (2, 128, K)) if precision == "fp8" else rng.integers(-20, 20, (2, 128, K))
            vals = mant * np.exp2(expo)
            t = torch.from_numpy(vals)
            vals = (t.to(torch.bfloat16) if precision == "bf16" else t.to(torch.float8_e4m3fn)).double().numpy()
            A, B = vals
            D = probe(km, A, B, precision)
            err = np.abs(D - A @ B.T)
            bound = gamma_k(K) * (np.abs(A) @ np.abs(B).T)
            assert np.all(err <= bound + 1e-300), f"K={K} trial {trial}: {np.max(err / np.maximum(bound, 1e-300))}"


def test_near_margin_gaps_bf16_parity(km, ref):
    """Points whose exact score gap to the second centroid is 1.3-2 x the BF16 margin.

    Data and centroids are BF16 values and the centroid set is symmetric about 0 (each pair
    also appears negated, far from every point), so the codes' centring vector -- the mean of
    the centroids -- is exactly 0, the codes are exact and the margin reduces to
    2 (c_h H + (gamma'_K' + 2u) ||x|| C~max) (1 + 2^-10) with u = 2^-24, K' = 128 + 16 (the
    contraction also accumulates the -h_j slice: 1 x (-h1, -h2, -h3)) and
    c_h = u + 2^-27 + gamma'_K' (1 + 2^-7) (the library's formula for BF16 with -h_j folded into
    the contraction, zero quantisation residuals). Such points are not flagged, their argmin
    comes from the tensor-core scores alone, and it must be the exact one."""
    rng = np.random.default_rng(2024)
    d, pairs, per = 128, 48, 64
    u = 2.0 ** -24

    def bf(a):
        return torch.from_numpy(np.asarray(a, dtype=np.float64)).to(torch.bfloat16).double().numpy()

    ya = bf(rng.uniform(-20, 20, (pairs, d)))
    yb = bf(ya + rng.normal(0, 0.25, (pairs, d)))
    C = np.empty((4 * pairs, d))
    C[0:2 * pairs:2], C[1:2 * pairs:2] = ya, yb
    C[2 * pairs:] = -C[:2 * pairs]  # the mirrored half: the centroids' mean is exactly 0
    h = 0.5 * np.sum(C * C, axis=1)
    H, Cmax = h.max(), np.sqrt(np.sum(C * C, axis=1)).max()
    gam = gamma_k(128 + 16)
    ch = u + 2.0 ** -27 + gam * (1 + 2.0 ** -7)
    pts, wanted = [], []
    for p in range(pairs):
        ca, cb = C[2 * p], C[2 * p + 1]
        w = cb - ca
        t = int(np.argmax(np.abs(w)))
        for q in range(per):
            x = bf((ca + cb) / 2 + rng.normal(0, 1.0, d))
            sign = 1.0 if q % 2 == 0 else -1.0
            for _ in range(4):  # move coordinate t so that the gap hits the target, then re-round
                margin = 2 * (ch * H + (gam + 2 * u) * np.linalg.norm(x) * Cmax) * (1 + 2.0 ** -10)
                target = sign * rng.uniform(1.45, 1.85) * margin
                g = 0.5 * (cb @ cb - ca @ ca) - x @ w  # s_b - s_a
                x[t] = bf(x[t] + (g - target) / w[t])
            margin = 2 * (ch * H + (gam + 2 * u) * np.linalg.norm(x) * Cmax) * (1 + 2.0 ** -10)
            g = 0.5 * (cb @ cb - ca @ ca) - x @ w
            if 1.3 * margin <= abs(g) <= 2.0 * margin:
                pts.append(x)
                wanted.append(abs(g) / margin)
    X = np.ascontiguousarray(np.array(pts), dtype=np.float32)
    assert len(X) >= pairs * per // 2, f"only {len(X)} points hit the gap window"
    perm = rng.permutation(len(X))
    X = X[perm]
    C32 = C.astype(np.float32)
    Xd = torch.from_numpy(X).to(DEV)
    Cd = torch.from_numpy(C32).to(DEV)
    out = km.step(Xd, Cd, precision="bf16")
    a = out.assign.cpu().numpy()
    ra, _, gap, _ = ref.assign(X, C)
    assert np.array_equal(a, ra), f"{int((a != ra).sum())} of {len(X)} near-margin points assigned differently"
    assert out.stats["n_flagged"] <= len(X) // 100, out.stats
    parity.check_update(ref, X, C, a, Cd.cpu().numpy(), out.sums.cpu().numpy(), out.counts.cpu().numpy())
    print(f"{len(X)} points with gaps {min(wanted):.2f}-{max(wanted):.2f} x margin; "
          f"flagged {out.stats['n_flagged']}; min relative FP64 gap {gap.min():.2e}")
