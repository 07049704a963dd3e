"""Pins for the oracle's d-dimensional lattice and feature-space E step.

Section 3.3 (Eq. feature_estep) replaces the point positions in the E step by
feature vectors with a diagonal covariance; Section 4.2 filters them with the
permutohedral lattice.  The generic-d oracle (oracle/lattice_d.c) is pinned by

- hand-derived d = 6 embeddings (tests/golden/lattice_canonical_d6.txt),
- bit equality with the separately pinned d = 3 lattice at d = 3,
- the invariants that define the lattice and its simplices for every d,
- the elevation as a similarity onto sum(z) = 0,
- closed forms of splat + slice and the augmentation identity,
- a restatement of splat + slice as a dictionary over the embedded vertices,
- the kernel's integral against a Riemann sum and the lattice covolume,
- the exact backend's separability over feature channels.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_canonical_d6.txt")


def _alpha(d):
    return math.sqrt(2.0 / 3.0) * (d + 1)


def _elevate(G, d):
    """z_j = sum_{i > j} c_i - j c_j with c_i = g_i alpha / sqrt(i (i+1)) (double)."""
    G = np.asarray(G, np.float64)
    c = G * np.array([_alpha(d) / math.sqrt(i * (i + 1)) for i in range(1, d + 1)])
    z = np.zeros((G.shape[0], d + 1))
    for j in range(d + 1):
        z[:, j] = c[:, j:].sum(1) - (j * c[:, j - 1] if j >= 1 else 0.0)
    return z


def _golden_cases():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, z, exp = [s.strip() for s in line.split("|")]
        z = [float(v) for v in z.split()]
        verts = []
        for tok in exp.split():
            w, k = tok.split(":")
            verts.append((float(w), tuple(int(v) for v in k.split(","))))
        cases.append((name, z, verts))
    return cases


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_golden_embeddings_d6(orc, case):
    _, z, verts = case
    d = 6
    # back-substitute the elevated-basis coefficients, then the feature
    c = np.zeros(d + 1)
    for j in range(d, 0, -1):
        c[j] = (c[j + 1:].sum() - z[j]) / j
    assert c[1:].sum() == pytest.approx(z[0], abs=1e-12)
    g = c[1:] / np.array([_alpha(d) / math.sqrt(i * (i + 1)) for i in range(1, d + 1)])
    keys, bary, st = orc.feature_embed(g[None, :], np.ones(d))
    assert st == 0
    got = {tuple(int(v) for v in keys[0, k]): float(bary[0, k]) for k in range(d + 1)}
    for w, key in verts:
        assert key in got, (key, got)
        assert got[key] == pytest.approx(w, abs=5e-6)
    listed = {k for _, k in verts}
    for key, w in got.items():
        if key not in listed:
            assert abs(w) < 5e-6


def _pts(seed, n, spread, dim=3):
    rng = np.random.default_rng(seed)
    return rng.uniform(-spread, spread, size=(n, dim)).astype(np.float32)


@pytest.mark.parametrize("sigma", [1.0, 0.05, 0.0123])
def test_generic_d3_equals_the_d3_lattice(orc, sigma):
    P = _pts(1, 3000, 2.0)
    k3, b3, _, _, st3 = orc.lattice_embed(P, sigma)
    kd, bd, std = orc.feature_embed(P, [sigma] * 3)
    assert st3 == 0 and std == 0
    np.testing.assert_array_equal(orc.feature_scales([sigma] * 3), orc.feature_scale(sigma))
    np.testing.assert_array_equal(kd, k3)
    np.testing.assert_array_equal(bd, b3)
    V = np.random.default_rng(2).normal(size=(3000, 4))
    l3 = orc.Lattice(P, V, sigma)
    ld = orc.FeatureLattice(P, V, [sigma] * 3)
    (kv3, vv3), (kvd, vvd) = l3.vertices(), ld.vertices()
    np.testing.assert_array_equal(kvd, kv3)
    np.testing.assert_allclose(vvd, vv3, rtol=1e-12, atol=1e-12)
    Q = _pts(3, 500, 2.0)
    np.testing.assert_allclose(ld.slice(Q)[0], l3.slice(Q)[0], rtol=1e-12, atol=1e-12)


def test_generic_d3_estep_equals_the_geometric_estep(orc):
    # features = positions with sigma_f = (sigma, sigma, sigma): Eq. feature_estep
    # reduces to the geometric E step (Eq. 6, Eq. 9 numerators)
    rng = np.random.default_rng(4)
    X, Y = _pts(5, 400, 0.3), _pts(6, 700, 0.3)
    Yn = rng.normal(size=(700, 3)).astype(np.float32)
    sigma = 0.046875  # a float32 value, so that both sides use the same sigma
    for backend in (orc.EXACT, orc.LATTICE):
        got = orc.estep_features(X, Y, [sigma] * 3, Y, Yn, backend=backend)
        ref = orc.estep(X, Y, Yn, sigma=sigma, backend=backend)
        np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("d", [1, 2, 4, 5, 6, 7])
def test_simplex_invariants(orc, d):
    D = d + 1
    rng = np.random.default_rng(10 + d)
    sigma_f = rng.uniform(0.2, 2.0, size=d).astype(np.float32)
    F = rng.uniform(-3, 3, size=(3000, d)).astype(np.float32)
    keys, bary, st = orc.feature_embed(F, sigma_f)
    assert st == 0
    assert np.allclose(bary.astype(np.float64).sum(1), 1.0, atol=4e-6)
    assert (bary >= -1e-6).all()
    assert (keys.sum(2) == 0).all()
    for k in range(D):
        assert (np.mod(keys[:, k, :], D) == k).all()
    # a lattice simplex: |v_l - v_k|^2 = D m (D - m), m = l - k, and vertex
    # l's coordinates below vertex k's are nested (the simplex is canonical
    # up to a permutation of coordinates and a lattice translation)
    for k in range(D):
        for l in range(k + 1, D):
            m = l - k
            diff = (keys[:, l, :] - keys[:, k, :]).astype(np.int64)
            assert ((diff == m) | (diff == m - D)).all()
            assert ((diff ** 2).sum(1) == D * m * (D - m)).all()
    # z (elevated in double from the normalised feature) is the barycentric
    # combination of the vertices: the point lies in its simplex
    G = F.astype(np.float64) / sigma_f.astype(np.float64)
    z = _elevate(G, d)
    rec = (bary[:, :, None].astype(np.float64) * keys.astype(np.float64)).sum(1)
    assert np.allclose(rec, z, atol=3e-5 * (1 + np.abs(z).max(1, keepdims=True)))


@pytest.mark.parametrize("d", [2, 6, 7])
def test_elevation_is_a_similarity(orc, d):
    # |z(f) - z(f')| = alpha |(f - f') / sigma_f|, and sum(z) = 0, measured on
    # the oracle's own simplices (z = sum_k b_k v_k)
    rng = np.random.default_rng(20 + d)
    sigma_f = rng.uniform(0.3, 1.5, size=d).astype(np.float32)
    F = rng.uniform(-2, 2, size=(200, d)).astype(np.float32)
    keys, bary, _ = orc.feature_embed(F, sigma_f)
    z = (bary[:, :, None].astype(np.float64) * keys.astype(np.float64)).sum(1)
    assert np.abs(z.sum(1)).max() < 1e-4
    G = F.astype(np.float64) / sigma_f
    dg = np.linalg.norm(G[:, None] - G[None], axis=-1)
    dz = np.linalg.norm(z[:, None] - z[None], axis=-1)
    np.testing.assert_allclose(dz, _alpha(d) * dg, rtol=1e-4, atol=1e-4)


def test_nonfinite_and_out_of_range_rejected(orc):
    F = np.zeros((2, 6), np.float32)
    F[0, 3] = np.nan
    F[1, 0] = 1e9
    *_, st = orc.feature_embed(F, np.ones(6))
    assert st != 0


def test_single_point_closed_forms(orc):
    # one observation splatted with [1, y]: at its own feature M0 = sum_k b_k^2,
    # M1 / M0 = y; far away nothing is sliced
    d = 6
    f = np.array([[0.31, -0.72, 0.05, 0.4, -0.15, 0.9]], np.float32)
    y = np.array([[0.5, -1.25, 2.0]], np.float32)
    sf = np.full(d, 0.3, np.float32)
    lat = orc.FeatureLattice(f, np.array([[1.0, *y[0].astype(np.float64)]]), sf)
    assert len(lat) == d + 1
    out, st = lat.slice(f)
    assert st == 0
    _, bary, _ = orc.feature_embed(f, sf)
    b = bary[0].astype(np.float64)
    assert out[0, 0] == pytest.approx((b * b).sum(), rel=1e-12)
    np.testing.assert_allclose(out[0, 1:] / out[0, 0], y[0], rtol=1e-12)
    far, _ = lat.slice(f + np.float32(10.0))
    assert (far == 0).all()


@pytest.mark.parametrize("d", [5, 6])
def test_slice_matches_a_vertex_dictionary(orc, d):
    # splat + slice restated: a dictionary from vertex key to sum b * v over
    # the observations, read back at the queries' vertices
    rng = np.random.default_rng(30 + d)
    sf = rng.uniform(0.3, 0.8, size=d).astype(np.float32)
    FY = rng.uniform(-1, 1, size=(400, d)).astype(np.float32)
    FX = rng.uniform(-1, 1, size=(150, d)).astype(np.float32)
    V = rng.normal(size=(400, 3))
    ky, by, _ = orc.feature_embed(FY, sf)
    table = {}
    for i in range(400):
        for k in range(d + 1):
            key = tuple(ky[i, k])
            table[key] = table.get(key, 0.0) + float(by[i, k]) * V[i]
    kx, bx, _ = orc.feature_embed(FX, sf)
    want = np.zeros((150, 3))
    for i in range(150):
        for k in range(d + 1):
            want[i] += float(bx[i, k]) * table.get(tuple(kx[i, k]), 0.0)
    lat = orc.FeatureLattice(FY, V, sf)
    assert len(lat) == len(table)
    got, _ = lat.slice(FX)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
    keys, vals = lat.vertices()
    for key, val in zip(keys[:50], vals[:50]):
        np.testing.assert_allclose(val, table[tuple(key)], rtol=1e-12, atol=1e-12)


def test_augmentation_identity(orc):
    # Eq. 13-14 in feature space: filtering [F_X, F_Y] with values [0, V_Y]
    # and reading at F_X equals the sum over F_Y alone (no blur)
    d = 6
    rng = np.random.default_rng(40)
    sf = np.full(d, 0.5, np.float32)
    FX = rng.uniform(-1, 1, size=(200, d)).astype(np.float32)
    FY = rng.uniform(-1, 1, size=(300, d)).astype(np.float32)
    VY = np.concatenate([np.ones((300, 1)), rng.normal(size=(300, 3))], 1)
    only_y, _ = orc.FeatureLattice(FY, VY, sf).slice(FX)
    both = orc.FeatureLattice(np.concatenate([FX, FY]), np.concatenate([np.zeros((200, 4)), VY]), sf)
    np.testing.assert_array_equal(both.slice(FX)[0], only_y)


def _lattice_basis_covolume(d):
    # the lattice is D * P(Z^D), P the projection onto sum(z) = 0; its first d
    # projected unit vectors are a basis.  In normalised feature units
    # g = E^T z / alpha with E's columns u_i / |u_i|.
    D = d + 1
    E = np.zeros((D, d))
    for i in range(1, d + 1):
        E[:i, i - 1] = 1.0
        E[i, i - 1] = -i
        E[:, i - 1] /= math.sqrt(i * (i + 1))
    P = np.eye(D) - np.ones((D, D)) / D
    B = E.T @ (D * P[:, :d]) / _alpha(d)
    return abs(np.linalg.det(B))


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7])
def test_kernel_mass_is_the_lattice_covolume(orc, d):
    # sum_v b_v(q) = 1 everywhere and every vertex's hat has the same
    # integral, so that integral is the volume per lattice point
    assert orc.feature_kernel_mass(d) == pytest.approx(_lattice_basis_covolume(d), rel=1e-12)
    if d == 3:
        assert orc.feature_kernel_mass(3) == pytest.approx(orc.kernel_mass(orc.LATTICE, False), rel=1e-12)


@pytest.mark.parametrize("d", [1, 2])
def test_kernel_mass_matches_a_riemann_sum(orc, d):
    # splat one observation with value 1; the sliced M0 integrated over a grid
    # of queries is the kernel mass (the integrand is continuous, piecewise
    # polynomial; a fine grid converges quickly)
    h = 0.01 if d == 1 else 0.02
    ax = np.arange(-4, 4, h) + h / 2
    Q = np.stack(np.meshgrid(*([ax] * d), indexing="ij"), -1).reshape(-1, d).astype(np.float32)
    f = np.array([[0.137, -0.291][:d]], np.float32)
    lat = orc.FeatureLattice(f, np.ones(1), np.ones(d, np.float32))
    m0, _ = lat.slice(Q)
    assert m0[:, 0].sum() * h ** d == pytest.approx(orc.feature_kernel_mass(d), rel=2e-3)


def test_exact_backend_is_separable_over_channels(orc):
    # K(f, f') = prod_c exp(-(f_c - f'_c)^2 / (2 sigma_c^2)): one observation,
    # the d = 6 sums equal the product of six d = 1 sums
    d = 6
    rng = np.random.default_rng(50)
    sf = rng.uniform(0.2, 1.0, size=d).astype(np.float32)
    FX = rng.uniform(-1, 1, size=(64, d)).astype(np.float32)
    FY = rng.uniform(-1, 1, size=(1, d)).astype(np.float32)
    Y = np.array([[0.25, -0.5, 2.0]], np.float32)
    got = orc.estep_features(FX, FY, sf, Y, backend=orc.EXACT)
    prod = np.ones(64)
    for c in range(d):
        one = orc.estep_features(FX[:, c:c + 1], FY[:, c:c + 1], sf[c:c + 1], Y, backend=orc.EXACT)
        prod *= one[:, 0]
    np.testing.assert_allclose(got[:, 0], prod, rtol=1e-12)
    np.testing.assert_allclose(got[:, 1:], prod[:, None] * Y.astype(np.float64), rtol=1e-12)
    # at its own feature the kernel is 1
    assert orc.estep_features(FY, FY, sf, Y, backend=orc.EXACT)[0, 0] == 1.0


def test_lattice_target_close_to_exact_target(orc):
    # the weighted mean M1 / M0 is a smoothed target: on dense smooth data the
    # lattice kernel's target stays near the Gaussian's (d = 6: xyz + a 3-d
    # attribute that varies smoothly with position)
    rng = np.random.default_rng(60)
    n = 20000
    P = rng.uniform(-1, 1, size=(n, 3)).astype(np.float32)
    A = np.stack([np.sin(2 * P[:, 0]), np.cos(2 * P[:, 1]), P[:, 2] ** 2], 1).astype(np.float32)
    FY = np.concatenate([P, A], 1)
    FX = FY[rng.choice(n, 300, replace=False)] + rng.normal(scale=0.01, size=(300, 6)).astype(np.float32)
    sf = np.array([0.15] * 3 + [0.3] * 3, np.float32)
    la = orc.estep_features(FX, FY, sf, P, backend=orc.LATTICE)
    ex = orc.estep_features(FX, FY, sf, P, backend=orc.EXACT)
    tl = la[:, 1:4] / la[:, :1]
    te = ex[:, 1:4] / ex[:, :1]
    err = np.linalg.norm(tl - te, axis=1)
    assert np.median(err) < 0.05
    assert (la[:, 0] > 0).all()
