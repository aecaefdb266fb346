"""Pins of the oracle's keyed-reduce training (GDA, naive Bayes) to facts that
do not come from the oracle itself: hand-worked examples in ``tests/golden/``,
the law of total covariance, library routines (numpy mean, cov, bincount) on
the cases that reduce to them, closed forms of the smoothing, and invariants
(translation, scaling, row permutation, class relabelling, independence of the
classes)."""
from __future__ import annotations

import glob
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def parse(path):
    out = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (s.strip() for s in line.split(":", 1))
            vals = val.split()
            out[key] = int(vals[0]) if key in ("d", "ncls") else [Fraction(v) for v in vals]
    return out


def _close(got, exp, rel=1e-14, abs_=1e-14):
    return all(abs(Fraction(float(g)) - e) <= max(abs_, rel * abs(e)) for g, e in zip(np.ravel(got), exp))


def _data(seed, n, d, ncls):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-5, 5, (ncls, d))
    y = rng.integers(0, ncls, n).astype(np.int32)
    X = (centres[y] + rng.normal(0, 1.5, (n, d))).astype(np.float32)
    return X, y


def pin_gda_golden(orc):
    files = sorted(glob.glob(os.path.join(GOLDEN, "gda_*.txt")))
    assert len(files) >= 3
    for path in files:
        g = parse(path)
        d = g["d"]
        X = np.array([float(v) for v in g["X"]], np.float32).reshape(-1, d)
        y = np.array([int(v) for v in g["y"]], np.int32)
        phi, mu, sigma = orc.gda(X, y, g["ncls"])
        assert _close(phi, g["phi"]), (path, "phi", phi)
        assert _close(mu, g["mu"]), (path, "mu", mu)
        assert _close(sigma, g["sigma"]), (path, "sigma", sigma)


def pin_nb_golden(orc):
    files = sorted(glob.glob(os.path.join(GOLDEN, "nb_*.txt")))
    assert files
    for path in files:
        g = parse(path)
        d = g["d"]
        X = np.array([float(v) for v in g["X"]], np.float32).reshape(-1, d)
        y = np.array([int(v) for v in g["y"]], np.int32)
        prior, theta = orc.nb(X, y, g["ncls"])
        assert _close(prior, g["prior"]), (path, "prior", prior)
        assert _close(theta, g["theta"]), (path, "theta", theta)


def pin_gda_single_class_is_population_covariance(orc):
    """One class: phi = 1, mu = the mean, Sigma = the population covariance (numpy)."""
    X, _ = _data(3, 500, 6, 1)
    phi, mu, sigma = orc.gda(X, np.zeros(500, np.int32), 1)
    X64 = X.astype(np.float64)
    assert np.allclose(phi, [1.0])
    assert np.allclose(mu[0], X64.mean(axis=0), rtol=1e-12, atol=1e-12)
    assert np.allclose(sigma, np.cov(X64.T, bias=True), rtol=1e-10, atol=1e-10)


def pin_gda_total_covariance(orc):
    """Law of total covariance: Cov(X) = Sigma_within + sum_c phi_c (mu_c - m)(mu_c - m)^T."""
    for seed, (n, d, ncls) in enumerate([(400, 5, 3), (1000, 8, 7), (60, 3, 9)]):
        X, y = _data(10 + seed, n, d, ncls)
        phi, mu, sigma = orc.gda(X, y, ncls)
        X64 = X.astype(np.float64)
        m = X64.mean(axis=0)
        between = sum(phi[c] * np.outer(mu[c] - m, mu[c] - m) for c in range(ncls) if phi[c] > 0)
        assert np.allclose(sigma + between, np.cov(X64.T, bias=True), rtol=1e-9, atol=1e-9), seed
        # priors are the label frequencies (numpy bincount)
        assert np.allclose(phi, np.bincount(y, minlength=ncls) / n, rtol=0, atol=1e-15)


def pin_gda_invariants(orc):
    X, y = _data(21, 300, 4, 4)
    X = np.round(X * 64) / 64  # dyadic values: the shifts and scalings below are exact in FP32
    phi, mu, sigma = orc.gda(X, y, 4)
    # symmetric positive semidefinite
    assert np.array_equal(sigma, sigma.T)
    assert np.linalg.eigvalsh(sigma).min() > -1e-9
    # translation: means move, Sigma does not
    v = np.array([4.0, -2.0, 0.5, 8.0], np.float32)
    phi2, mu2, sigma2 = orc.gda(X + v, y, 4)
    assert np.allclose(mu2[phi2 > 0], (mu + v)[phi > 0], rtol=1e-12, atol=1e-9)
    assert np.allclose(sigma2, sigma, rtol=1e-9, atol=1e-9)
    # scaling by 2: Sigma by 4 (exact in binary)
    _, mu3, sigma3 = orc.gda(X * 2, y, 4)
    assert np.allclose(sigma3, 4 * sigma, rtol=1e-12, atol=1e-12)
    # row permutation and class relabelling
    p = np.random.default_rng(5).permutation(300)
    relabel = np.array([2, 0, 3, 1], np.int32)
    phi4, mu4, sigma4 = orc.gda(X[p], relabel[y[p]], 4)
    assert np.allclose(phi4[relabel], phi) and np.allclose(mu4[relabel], mu, rtol=1e-12, atol=1e-12)
    assert np.allclose(sigma4, sigma, rtol=1e-10, atol=1e-10)


def pin_nb_closed_forms(orc):
    """Smoothing closed forms: a class of all-zero rows is uniform (1/d); a class whose rows
    only ever count feature 0 (total T) has theta = ((T+1), 1, ..., 1) / (T + d)."""
    d = 5
    X = np.zeros((7, d), np.float32)
    X[3:, 0] = [2, 1, 4, 3]               # class 1: feature 0 only, T = 10
    y = np.array([0, 0, 0, 1, 1, 1, 1], np.int32)
    prior, theta = orc.nb(X, y, 2)
    assert np.allclose(theta[0], np.full(d, 1.0 / d), rtol=0, atol=1e-15)
    assert np.allclose(theta[1], np.array([11, 1, 1, 1, 1]) / 15.0, rtol=0, atol=1e-15)
    assert np.allclose(prior, [3 / 7, 4 / 7], rtol=0, atol=1e-15)


def pin_nb_invariants(orc):
    rng = np.random.default_rng(8)
    n, d, ncls = 400, 12, 5
    X = rng.poisson(2.0, (n, d)).astype(np.float32)
    y = rng.integers(0, ncls, n).astype(np.int32)
    prior, theta = orc.nb(X, y, ncls)
    # distributions: every theta row and the priors sum to 1, all entries positive
    assert np.allclose(theta.sum(axis=1), 1.0, rtol=0, atol=1e-12) and theta.min() > 0
    assert np.allclose(prior.sum(), 1.0) and np.allclose(prior, np.bincount(y, minlength=ncls) / n)
    # row permutation
    p = rng.permutation(n)
    prior2, theta2 = orc.nb(X[p], y[p], ncls)
    assert np.allclose(theta2, theta, rtol=1e-13, atol=0) and np.allclose(prior2, prior)
    # classes are independent: the rows of other classes do not change a class's theta
    keep = y == 2
    _, theta3 = orc.nb(X[keep], np.zeros(int(keep.sum()), np.int32), 1)
    assert np.allclose(theta3[0], theta[2], rtol=1e-13, atol=0)
    # more evidence moves theta toward the empirical frequencies (duplicated rows)
    _, theta4 = orc.nb(np.concatenate([X, X]), np.concatenate([y, y]), ncls)
    S = np.zeros((ncls, d))
    np.add.at(S, y, X.astype(np.float64))
    emp = S / S.sum(axis=1, keepdims=True)
    assert np.all(np.abs(theta4 - emp) <= np.abs(theta - emp) + 1e-15)


ALL_PINS = [pin_gda_golden, pin_nb_golden, pin_gda_single_class_is_population_covariance,
            pin_gda_total_covariance, pin_gda_invariants, pin_nb_closed_forms, pin_nb_invariants]
