"""Pins for the oracle's exact E step (Eq. 6, Eq. 9 numerator).

Each test checks the oracle against something other than its own formula: the
one-component closed form, additivity over the observation set, and the
translation / scale equivariances the Gaussian sums must satisfy.
"""
import math

import numpy as np
import pytest


def _one(orc, x, y, n, sigma):
    X = np.array([[*x, 0]], np.float32)
    Y = np.array([[*y, 0]], np.float32)
    Yn = np.array([[*n, 0]], np.float32)
    M0, M1, Ns = orc.estep_exact(X, Y, Yn, sigma)
    return M0[0], M1[0], Ns[0]


def test_single_component_closed_form(orc):
    # One observation point: M0 = exp(-r^2 / (2 sigma^2)), M1 = M0 y, Ns = M0 n.
    x, y, n, s = (0.1, -0.2, 0.3), (0.13, -0.17, 0.26), (0.0, 0.6, 0.8), 0.05
    xs, ys = np.float32(x).astype(np.float64), np.float32(y).astype(np.float64)
    r2 = float(((xs - ys) ** 2).sum())
    m0, m1, ns = _one(orc, x, y, n, s)
    assert m0 == pytest.approx(math.exp(-r2 / (2 * s * s)), rel=1e-12)
    np.testing.assert_allclose(m1, m0 * ys, rtol=1e-12)
    np.testing.assert_allclose(ns, m0 * np.float32(n).astype(np.float64), rtol=1e-12)


def test_additive_over_observations(orc):
    rng = np.random.default_rng(1)
    X = rng.normal(size=(7, 4)).astype(np.float32)
    Y = rng.normal(size=(11, 4)).astype(np.float32)
    Yn = rng.normal(size=(11, 4)).astype(np.float32)
    full = orc.estep_exact(X, Y, Yn, 0.7)
    a = orc.estep_exact(X, Y[:4], Yn[:4], 0.7)
    b = orc.estep_exact(X, Y[4:], Yn[4:], 0.7)
    for f, u, v in zip(full, a, b):
        np.testing.assert_allclose(f, u + v, rtol=1e-12, atol=1e-300)
    # and each term of the sum is the one-component closed form
    terms = [orc.estep_exact(X, Y[k:k + 1], Yn[k:k + 1], 0.7) for k in range(11)]
    np.testing.assert_allclose(full[0], sum(t[0] for t in terms), rtol=1e-12)


def test_translation_and_scale_equivariance(orc):
    rng = np.random.default_rng(2)
    # coordinates on a 1/1024 grid so that the shifted and scaled inputs are exact floats
    X = (np.round(rng.uniform(-1, 1, size=(9, 4)) * 1024) / 1024).astype(np.float32)
    Y = (np.round(rng.uniform(-1, 1, size=(13, 4)) * 1024) / 1024).astype(np.float32)
    M0, M1, _ = orc.estep_exact(X, Y, None, 0.4)
    # shift by a power of two so the float inputs stay exact
    t = np.array([0.5, -0.25, 1.0, 0], np.float32)
    M0t, M1t, _ = orc.estep_exact(X + t, Y + t, None, 0.4)
    np.testing.assert_allclose(M0t, M0, rtol=1e-9)
    np.testing.assert_allclose(M1t, M1 + M0[:, None] * t[:3].astype(np.float64), rtol=1e-9, atol=1e-12)
    M0s, M1s, _ = orc.estep_exact(2 * X, 2 * Y, None, 0.8)
    np.testing.assert_allclose(M0s, M0, rtol=1e-12)
    np.testing.assert_allclose(M1s, 2 * M1, rtol=1e-12)


def test_symmetric_pair_target_is_midpoint(orc):
    X = np.array([[0.25, 0.5, -0.5, 0]], np.float32)
    d = np.array([0.125, -0.0625, 0.25, 0], np.float32)
    Y = np.stack([X[0] + d, X[0] - d])
    M0, M1, _ = orc.estep_exact(X, Y, None, 0.3)
    np.testing.assert_allclose(M1[0] / M0[0], X[0, :3], rtol=0, atol=1e-12)


def test_target_in_bounding_box(orc):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(50, 4)).astype(np.float32)
    Y = rng.normal(size=(40, 4)).astype(np.float32)
    M0, M1, _ = orc.estep_exact(X, Y, None, 0.5)
    t = M1 / M0[:, None]
    assert (t >= Y[:, :3].min(0) - 1e-9).all() and (t <= Y[:, :3].max(0) + 1e-9).all()
