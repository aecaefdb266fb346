"""Keyed-reduce training on the GPU (kmeans_gda_train, kmeans_nb_train) against the FP64 oracle.

Tolerances (derived from the arithmetic, as for the k-means sums):
  - phi / prior: n_c / n rounded to FP32 -> within one FP32 ulp of the FP64 value;
  - mu: the class sums are FP32 Kahan runs combined in FP64 (error ~1e-7 of the sum
    of |x|), so |mu - mu_ref| <= 1e-5 * max_t mean_{y_i = c} |x_it| (the k-means
    centroid tolerance);
  - sigma: each entry is a sum of FP32 partials over 64 rows (<= 65u of the partial's
    sum of |terms|) accumulated in FP64, from rows centred with the FP32 class mean
    (a second-order change), so |sigma_ab - ref_ab| <= 1e-5 * S_ab with
    S_ab = (1/n) sum_i |c_ia| |c_ib|, c the rows centred with the FP64 means;
  - theta: (S + 1) / (T + d) from sums with relative error ~1e-7: 1e-6 relative.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def km():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1109_0778_b300 import kmeans

    return kmeans


def labelled(seed, n, d, ncls, R=6.0, sigma=1.5):
    X, comp = synth.mixture(seed, n, d, max(ncls, 1), R, sigma, with_comp=True)
    return X, comp.astype(np.int32)


def check_gda(ref, X, y, ncls, phi, mu, sigma):
    n, d = X.shape
    phi_r, mu_r, sig_r = ref.gda(X, y, ncls)
    phi, mu, sigma = (t.cpu().numpy().astype(np.float64) for t in (phi, mu, sigma))
    assert np.all(np.abs(phi - phi_r) <= np.spacing(np.float32(np.maximum(phi_r, 1e-30))).astype(np.float64))
    cnt = np.bincount(y, minlength=ncls)
    absmean = np.zeros((ncls, d))
    np.add.at(absmean, y, np.abs(X.astype(np.float64)))
    scale = np.where(cnt > 0, (absmean / np.maximum(cnt, 1)[:, None]).max(axis=1), 0.0)
    err = np.abs(mu - mu_r).max(axis=1)
    assert np.all(err <= 1e-5 * scale + 1e-30), (err / np.maximum(scale, 1e-30)).max()
    assert np.all(mu[cnt == 0] == 0.0)
    c = np.abs(X.astype(np.float64) - mu_r[y])
    S = c.T @ c / n
    serr = np.abs(sigma - sig_r)
    assert np.all(serr <= 1e-5 * S + 1e-30), (serr / np.maximum(S, 1e-30)).max()
    assert np.array_equal(sigma, sigma.T)


def check_nb(ref, X, y, ncls, prior, theta):
    prior_r, theta_r = ref.nb(X, y, ncls)
    prior, theta = prior.cpu().numpy().astype(np.float64), theta.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(prior - prior_r) <= np.spacing(np.float32(np.maximum(prior_r, 1e-30))).astype(np.float64))
    assert np.all(np.abs(theta - theta_r) <= 1e-6 * theta_r), (np.abs(theta - theta_r) / theta_r).max()


@pytest.mark.parametrize("n,d,ncls", [(1, 1, 1), (5, 3, 7), (1000, 17, 4), (20000, 64, 16), (7777, 200, 3),
                                      (3000, 256, 40), (50000, 65, 2), (4099, 128, 1)])
def test_gda_matches_oracle(km, ref, n, d, ncls):
    X, y = labelled(300 + n + d, n, d, ncls)
    Xd, yd = torch.from_numpy(X).to(DEV), torch.from_numpy(y).to(DEV)
    phi, mu, sigma = km.gda_train(Xd, yd, ncls)
    check_gda(ref, X, y, ncls, phi, mu, sigma)


def test_gda_rows_not_16_byte_aligned(km, ref):
    """X one float into a buffer (4-byte but not 16-byte aligned): the gathers and the covariance
    staging must fall back to 4-byte loads."""
    n, d, ncls = 3000, 64, 6
    X, y = labelled(4242, n, d, ncls)
    buf = torch.zeros(n * d + 1, dtype=torch.float32, device=DEV)
    Xd = buf[1:].view(n, d)
    Xd.copy_(torch.from_numpy(X))
    assert Xd.is_contiguous() and Xd.data_ptr() % 16 == 4
    phi, mu, sigma = km.gda_train(Xd, torch.from_numpy(y).to(DEV), ncls)
    check_gda(ref, X, y, ncls, phi, mu, sigma)


@pytest.mark.parametrize("n,d,ncls", [(1, 1, 1), (6, 4, 9), (2000, 30, 5), (30000, 256, 20), (4097, 129, 2)])
def test_nb_matches_oracle(km, ref, n, d, ncls):
    rng = np.random.default_rng(n + d)
    y = rng.integers(0, ncls, n).astype(np.int32)
    rate = rng.uniform(0.2, 3.0, (ncls, d))
    X = rng.poisson(rate[y]).astype(np.float32)
    Xd, yd = torch.from_numpy(X).to(DEV), torch.from_numpy(y).to(DEV)
    prior, theta = km.nb_train(Xd, yd, ncls)
    check_nb(ref, X, y, ncls, prior, theta)


def test_training_rejects_bad_labels(km):
    X = torch.zeros(100, 8, device=DEV)
    y = torch.zeros(100, dtype=torch.int32, device=DEV)
    y[37] = 5
    with pytest.raises(km.KMeansError) as e:
        km.gda_train(X, y, 5)
    assert e.value.status == km.KM_EINVAL
    y[37] = -1
    with pytest.raises(km.KMeansError) as e:
        km.nb_train(X, y, 5)
    assert e.value.status == km.KM_EINVAL
    # the library is still usable
    y[37] = 0
    prior, theta = km.nb_train(X, y, 5)
    assert abs(float(prior[0]) - 1.0) < 1e-7


def test_training_interleaves_with_kmeans(km, ref):
    """The training entry points share the k-means workspace: a run, a training call and a
    second run give the same results as without the training call."""
    X, y = labelled(9, 30000, 32, 10)
    Xd, yd = torch.from_numpy(X).to(DEV), torch.from_numpy(y).to(DEV)
    C0 = torch.from_numpy(X[:10].copy()).to(DEV)
    C1 = C0.clone()
    a1 = km.run(Xd, C1, 3).assign.clone()
    km.gda_train(Xd, yd, 10)
    C2 = C0.clone()
    a2 = km.run(Xd, C2, 3).assign
    assert torch.equal(a1, a2)


@pytest.mark.slow
def test_full_size_training(km, ref):
    """1,048,576 labelled rows: GDA (d=64, 16 classes) and NB (d=256, 20 classes)."""
    X, y = labelled(44, 1 << 20, 64, 16)
    Xd, yd = torch.from_numpy(X).to(DEV), torch.from_numpy(y).to(DEV)
    phi, mu, sigma = km.gda_train(Xd, yd, 16)
    check_gda(ref, X, y, 16, phi, mu, sigma)
    rng = np.random.default_rng(45)
    yb = rng.integers(0, 20, 1 << 20).astype(np.int32)
    Xb = rng.poisson(rng.uniform(0.2, 3.0, (20, 256))[yb]).astype(np.float32)
    prior, theta = km.nb_train(torch.from_numpy(Xb).to(DEV), torch.from_numpy(yb).to(DEV), 20)
    check_nb(ref, Xb, yb, 20, prior, theta)
