"""Pins for the oracle's reference permutohedral lattice (Section 4.2).

The paper prints no worked example of the lattice, so the oracle is pinned by
hand-derived embeddings (tests/golden/lattice_canonical.txt), by the
invariants that define the lattice and its simplices, by the geometry of the
elevation (a similarity onto sum(z) = 0), by closed forms of splat+slice, by
the augmentation identity of Eq. 13-14, and by the kernel's integral measured
by Monte Carlo against the analytic volume per lattice point.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_canonical.txt")
ALPHA = math.sqrt(2.0 / 3.0) * 4.0


def _golden_cases():
    cases = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, c, exp = [s.strip() for s in line.split("|")]
        c = [float(v) for v in c.split()]
        verts = []
        for tok in exp.split():
            w, k = tok.split(":")
            verts.append((float(w), tuple(int(v) for v in k.split(","))))
        cases.append((name, c, verts))
    return cases


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c[0])
def test_golden_embeddings(orc, case):
    _, c, verts = case
    sigma = 1.0
    # point whose elevated-basis coefficients are c: p_i = c_i / scale_i
    scale = np.array([ALPHA / math.sqrt(i * (i + 1)) / sigma for i in (1, 2, 3)])
    p = np.array([[*(np.array(c) / scale), 0.0]], np.float32)
    keys, bary, z, rank, st = orc.lattice_embed(p, sigma)
    assert st == 0
    got = {tuple(keys[0, k]): float(bary[0, k]) for k in range(4)}
    for w, key in verts:
        assert key in got, (key, got)
        assert got[key] == pytest.approx(w, abs=2e-6)
    listed = {k for _, k in verts}
    for key, w in got.items():
        if key not in listed:
            assert abs(w) < 2e-6


def _random_points(seed, n, spread):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, 4), np.float32)
    P[:, :3] = rng.uniform(-spread, spread, size=(n, 3))
    return P


@pytest.mark.parametrize("sigma", [1.0, 0.05, 0.0123])
def test_simplex_invariants(orc, sigma):
    P = _random_points(4, 4000, 2.0)
    keys, bary, z, rank, st = orc.lattice_embed(P, sigma)
    assert st == 0
    zmax = np.abs(z).max(1)
    # elevated coordinates lie on sum(z) = 0 (up to float rounding)
    assert (np.abs(z.astype(np.float64).sum(1)) <= 4e-7 * (1 + zmax)).all()
    # barycentric weights are a partition of unity, non-negative
    assert np.allclose(bary.astype(np.float64).sum(1), 1.0, atol=2e-6)
    assert (bary >= -1e-6).all()
    # ranks form a permutation of 0..3
    assert (np.sort(rank, 1) == np.arange(4)).all()
    # vertex k is a remainder-k lattice point of the hyperplane
    assert (keys.sum(2) == 0).all()
    for k in range(4):
        assert (np.mod(keys[:, k, :], 4) == k).all()
    # the four vertices are a lattice simplex: |v_l - v_k|^2 = 4 m (4 - m), m = l - k
    for k in range(4):
        for l in range(k + 1, 4):
            m = l - k
            d2 = ((keys[:, l, :] - keys[:, k, :]).astype(np.int64) ** 2).sum(1)
            assert (d2 == 4 * m * (4 - m)).all()
    # and z is their barycentric combination (z lies in the simplex)
    rec = (bary[:, :, None].astype(np.float64) * keys.astype(np.float64)).sum(1)
    assert np.allclose(rec, z, atol=1e-5 * (1 + zmax[:, None]))


def test_elevation_is_a_similarity(orc):
    # |z(p) - z(q)| = alpha / sigma |p - q|, and z is orthogonal to (1,1,1,1)
    sigma = 0.25
    P = _random_points(5, 300, 1.0)
    _, _, z, _, _ = orc.lattice_embed(P, sigma)
    z = z.astype(np.float64)
    dp = np.linalg.norm(P[:, None, :3].astype(np.float64) - P[None, :, :3], axis=-1)
    dz = np.linalg.norm(z[:, None, :] - z[None, :, :], axis=-1)
    np.testing.assert_allclose(dz, ALPHA / sigma * dp, rtol=2e-5, atol=2e-5)


def test_nonfinite_and_out_of_range_rejected(orc):
    P = np.array([[np.nan, 0, 0, 0], [1e9, 0, 0, 0]], np.float32)
    *_, st = orc.lattice_embed(P, 0.01)
    assert st != 0


def test_splat_slice_single_point_closed_forms(orc):
    # One observation y splatted with values [1, y]; slicing at y itself gives
    # M0 = sum_k b_k^2 and M1 / M0 = y exactly.
    y = np.array([[0.31, -0.72, 0.05, 0]], np.float32)
    sigma = 0.1
    V = np.array([[1.0, *y[0, :3].astype(np.float64)]])
    lat = orc.Lattice(y, V, sigma)
    assert len(lat) == 4
    out, st = lat.slice(y)
    _, bary, _, _, _ = orc.lattice_embed(y, sigma)
    b = bary[0].astype(np.float64)
    assert out[0, 0] == pytest.approx((b * b).sum(), rel=1e-12)
    np.testing.assert_allclose(out[0, 1:] / out[0, 0], y[0, :3], rtol=1e-12)
    # far away there is nothing to slice
    far, _ = lat.slice(y + np.float32(10.0))
    assert (far == 0).all()


def test_slice_is_linear_in_values(orc):
    rng = np.random.default_rng(6)
    Y = _random_points(7, 500, 0.5)
    Q = _random_points(8, 200, 0.5)
    V1 = rng.normal(size=(500, 3))
    V2 = rng.normal(size=(500, 3))
    s1, _ = orc.Lattice(Y, V1, 0.07).slice(Q)
    s2, _ = orc.Lattice(Y, V2, 0.07).slice(Q)
    s12, _ = orc.Lattice(Y, 2 * V1 - V2, 0.07).slice(Q)
    np.testing.assert_allclose(s12, 2 * s1 - s2, rtol=1e-9, atol=1e-12)


def test_augmentation_identity(orc):
    # Eq. 13-14: filtering [F_X, F_Y] with values [0, V_Y] and reading the
    # result at X equals the sum over Y alone -- exactly, for splat+slice.
    # (With blur, X's zero-valued vertices could relay mass between Y's
    # vertices; the registration therefore never inserts X: slicing is a pure
    # query of the lattice built over Y.)
    X = _random_points(9, 300, 0.5)
    Y = _random_points(10, 400, 0.5)
    VY = np.concatenate([np.ones((400, 1)), Y[:, :3].astype(np.float64)], 1)
    only_y, _ = orc.Lattice(Y, VY, 0.06).slice(X)
    both = orc.Lattice(np.concatenate([X, Y]), np.concatenate([np.zeros((300, 4)), VY]), 0.06)
    aug, _ = both.slice(X)
    np.testing.assert_array_equal(aug, only_y)
    assert len(both) > len(orc.Lattice(Y, VY, 0.06))


@pytest.mark.parametrize("blur", [False, True])
def test_kernel_mass_matches_monte_carlo(orc, blur):
    # Uniform observations of density rho with value 1: far from the border
    # M0 ~ rho * integral(K), the kernel mass G (analytic volume per lattice
    # point in feature units, times 2^4 when blurred).
    rng = np.random.default_rng(11 + blur)
    n, half = 400_000, 6.0
    Y = np.zeros((n, 4), np.float32)
    Y[:, :3] = rng.uniform(-half, half, size=(n, 3))
    rho = n / (2 * half) ** 3
    lat = orc.Lattice(Y, np.ones(n), 1.0, blur=blur)
    Q = np.zeros((4000, 4), np.float32)
    Q[:, :3] = rng.uniform(-2, 2, size=(4000, 3))
    m0, _ = lat.slice(Q)
    est = m0[:, 0].mean() / rho
    G = orc.kernel_mass(orc.LATTICE, blur)
    assert est == pytest.approx(G, rel=0.01)
    assert G == pytest.approx((1.5 ** 1.5 / 2.0) * (16 if blur else 1), rel=1e-12)


def test_exact_kernel_mass(orc):
    # queries spread over many kernel widths so that their sampling errors
    # are nearly independent (relative error of the mean ~0.25%)
    rng = np.random.default_rng(13)
    n, half = 1_500_000, 7.0
    Y = np.zeros((n, 4), np.float32)
    Y[:, :3] = rng.uniform(-half, half, size=(n, 3))
    Q = np.zeros((200, 4), np.float32)
    Q[:, :3] = rng.uniform(-3, 3, size=(200, 3))
    M0, _, _ = orc.estep_exact(Q, Y, None, 1.0)
    est = M0.mean() / (n / (2 * half) ** 3)
    assert est == pytest.approx(orc.kernel_mass(orc.EXACT), rel=0.01)
    assert orc.kernel_mass(orc.EXACT) == pytest.approx((2 * math.pi) ** 1.5, rel=1e-12)


def test_blur_gain_on_complete_lattice(orc):
    # On a lattice whose every neighbour exists (dense uniform points), each
    # (1/2, 1, 1/2) pass doubles a locally constant field: blurred M0 at an
    # interior point is 16x the unblurred one up to sampling noise.
    rng = np.random.default_rng(14)
    n, half = 300_000, 5.0
    Y = np.zeros((n, 4), np.float32)
    Y[:, :3] = rng.uniform(-half, half, size=(n, 3))
    Q = np.zeros((2000, 4), np.float32)
    Q[:, :3] = rng.uniform(-1.5, 1.5, size=(2000, 3))
    a, _ = orc.Lattice(Y, np.ones(n), 1.0).slice(Q)
    b, _ = orc.Lattice(Y, np.ones(n), 1.0, blur=True).slice(Q)
    assert b[:, 0].mean() / a[:, 0].mean() == pytest.approx(16.0, rel=0.01)


def test_lattice_target_close_to_exact_target(orc):
    # The lattice approximates the Gaussian transform; on a dense smooth
    # surface the normalised targets M1/M0 agree to a fraction of sigma.  The
    # paper states no error bound, so this is a sanity bound, not parity.
    rng = np.random.default_rng(15)
    u = rng.normal(size=(20000, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    Y = np.zeros((20000, 4), np.float32)
    Y[:, :3] = u
    X = Y[:300].copy()
    X[:, :3] *= 1.01
    sigma = 0.05
    ex = orc.estep(X, Y, None, sigma, backend=orc.EXACT)
    la = orc.estep(X, Y, None, sigma, backend=orc.LATTICE, blur=True)
    te = ex[:, 1:4] / ex[:, :1]
    tl = la[:, 1:4] / la[:, :1]
    assert np.median(np.linalg.norm(te - tl, axis=1)) < 0.5 * sigma


def test_sigma_schedule(orc):
    s = orc.sigma_schedule(0.04, 0.01, 20)
    assert s[0] == np.float32(0.04) and s[-1] == np.float32(0.01)
    r = s[1:].astype(np.float64) / s[:-1]
    np.testing.assert_allclose(r, 0.25 ** (1 / 19), rtol=1e-6)
    assert (orc.sigma_schedule(0.02, 0.02, 5) == np.float32(0.02)).all()


def _blur_stencil():
    """The blur of Section 4.2 as one convolution: one (1/2, 1, 1/2) pass
    along each of the d + 1 = 4 lattice axes, the neighbour along axis j being
    offset by e_j = (1, 1, 1, 1) - 4 delta_j.  Offsets sum_j a_j e_j with
    a_j in {-1, 0, 1} and weights prod_j (1/2 if a_j != 0 else 1); because
    e_0 + ... + e_3 = 0, different a give the same offset and their weights
    add up."""
    import itertools
    e = [np.array([1, 1, 1, 1]) - 4 * np.eye(4, dtype=int)[j] for j in range(4)]
    out = {}
    for a in itertools.product((-1, 0, 1), repeat=4):
        off = tuple(int(x) for x in sum(aj * ej for aj, ej in zip(a, e)))
        out[off] = out.get(off, 0.0) + float(np.prod([0.5 if aj else 1.0 for aj in a]))
    return out


def test_blur_is_the_four_axis_stencil(orc):
    # A unit value at the lattice point 0 (a point at the origin sits on it
    # exactly: barycentric weight 1 there, 0 on the other three vertices),
    # inside a dense cloud of zero-valued points so that every vertex the
    # stencil reaches exists.  After the blur every vertex must hold exactly
    # the stencil weight of its offset from 0 (dyadic sums: exact in float64),
    # and every other vertex 0.  A pass along a repeated or wrong axis, a sign
    # error in the offset or a dropped pass changes some of these values.
    stencil = _blur_stencil()
    assert len(stencil) == 65 and sum(stencil.values()) == 16.0
    assert stencil[(0, 0, 0, 0)] == 1.0 + 2 * 0.5 ** 4   # a = 0 and a = +-(1, 1, 1, 1) fold onto 0
    rng = np.random.default_rng(16)
    n = 200_000
    P = np.zeros((n + 1, 4), np.float32)
    P[1:, :3] = rng.uniform(-5.0, 5.0, size=(n, 3))
    V = np.zeros((n + 1, 1))
    V[0, 0] = 1.0
    lat = orc.Lattice(P, V, 1.0, blur=True)
    keys, vals = lat.vertices()
    assert (keys.sum(1) == 0).all()
    expect = np.array([stencil.get(tuple(int(x) for x in k), 0.0) for k in keys])
    np.testing.assert_array_equal(vals[:, 0], expect)
    # every stencil offset is present (the neighbourhood was complete)
    present = {tuple(int(x) for x in k) for k in keys}
    assert set(stencil) <= present


def test_blur_second_moment_is_isotropic(orc):
    # The blurred unit impulse as a distribution over the lattice: mass 2^4,
    # mean 0 and, each pass adding variance 1/2 e_j e_j^T, second moment
    # 1/2 sum_j e_j e_j^T = 8 (I - 11^T / 4) -- isotropic within the hyperplane
    # sum z = 0, which the elevation maps feature space onto by a similarity.
    rng = np.random.default_rng(17)
    n = 200_000
    P = np.zeros((n + 1, 4), np.float32)
    P[1:, :3] = rng.uniform(-5.0, 5.0, size=(n, 3))
    V = np.zeros((n + 1, 1))
    V[0, 0] = 1.0
    keys, vals = orc.Lattice(P, V, 1.0, blur=True).vertices()
    w = vals[:, 0]
    z = keys.astype(np.float64)
    assert w.sum() == 16.0
    np.testing.assert_array_equal(w @ z, np.zeros(4))
    second = (z * w[:, None]).T @ z / w.sum()
    np.testing.assert_allclose(second, 8.0 * (np.eye(4) - np.ones((4, 4)) / 4.0), rtol=0, atol=1e-12)
