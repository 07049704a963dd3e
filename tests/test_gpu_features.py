"""GPU parity of the feature-space E step (Section 3.3, Eq. feature_estep) on
the d-dimensional permutohedral lattice against the CPU oracle.

Bar: vertex keys and barycentric weights bit-exact for every d (the same
float operations decide them on both sides); E-step sums within 1e-4 of the
oracle's float64 sums relative to |ref| + M0 max|v| (float32 atomics in
arbitrary order; a sum's rounding scales with its terms' magnitudes), and the
lattice's vertex count exact.  The exact feature sums are held to the same
bar as the geometric Gauss transform.
"""
import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_1811_10136_gb300 as fr
    assert torch.cuda.is_available()
    return fr.Context(0)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def pad4(P):
    out = np.zeros((P.shape[0], 4), np.float32)
    out[:, :3] = P[:, :3]
    return out


def clustered(seed, n, d, spread=1.0, clusters=40, scale=0.15):
    """Features around a few centres, so that vertices are shared."""
    rng = np.random.default_rng(seed)
    C = rng.uniform(-spread, spread, size=(clusters, d))
    lab = rng.integers(0, clusters, size=n)
    return (C[lab] + rng.normal(scale=scale, size=(n, d))).astype(np.float32)


def within(out, ref, Y, rel=1e-4):
    vmax = np.ones(ref.shape[1])
    vmax[1:4] = np.abs(Y[:, :3]).max(0)
    bound = rel * (np.abs(ref) + ref[:, :1] * vmax[None, :]) + 1e-7 * np.abs(ref).max(0, keepdims=True) + 1e-30
    return float((np.abs(out.astype(np.float64) - ref) / bound).max())


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("n", [1, 257, 3001])
def test_embed_bit_exact(ctx, orc, d, n):
    rng = np.random.default_rng(100 * d + n)
    F = rng.uniform(-3, 3, size=(n, d)).astype(np.float32)
    sf = rng.uniform(0.05, 1.5, size=d).astype(np.float32)
    k_ref, b_ref, st = orc.feature_embed(F, sf)
    assert st == 0
    keys, bary = ctx.feature_embed(dev(F), sf)
    np.testing.assert_array_equal(host(keys), k_ref)
    np.testing.assert_array_equal(host(bary) + 0.0, b_ref + 0.0)


def test_embed_ties_and_lattice_points(ctx, orc):
    # features on lattice points, edges and the canonical centroid (many equal
    # residuals, so the tie rule decides the ranks)
    d = 6
    alpha = np.sqrt(2.0 / 3.0) * 7
    sc = np.array([alpha / np.sqrt(i * (i + 1)) for i in range(1, 7)])
    rows = []
    for z in ([0] * 7, [1, 1, 1, 1, 1, 1, -6], [3, 2, 1, 0, -1, -2, -3], [7, -7, 0, 0, 0, 0, 0],
              [0.5] * 6 + [-3], [3.5, 0, 0, 0, 0, 0, -3.5]):
        c = np.zeros(7)
        for j in range(6, 0, -1):
            c[j] = (c[j + 1:].sum() - z[j]) / j
        rows.append(c[1:] / sc)
    F = np.array(rows, np.float32)
    F = np.concatenate([F, np.round(F * 4) / 4, np.zeros((3, 6), np.float32)]).astype(np.float32)
    k_ref, b_ref, _ = orc.feature_embed(F, np.ones(d))
    keys, bary = ctx.feature_embed(dev(F), np.ones(d, np.float32))
    np.testing.assert_array_equal(host(keys), k_ref)
    np.testing.assert_array_equal(host(bary) + 0.0, b_ref + 0.0)


def test_embed_rejects_bad_input(ctx):
    import paper_1811_10136_gb300 as fr
    F = np.zeros((4, 6), np.float32)
    F[1, 2] = np.nan
    with pytest.raises(fr.FilterRegError):
        ctx.feature_embed(dev(F), np.ones(6, np.float32))
    with pytest.raises(fr.FilterRegError):
        ctx.feature_embed(dev(np.zeros((4, 6), np.float32)), np.array([1, 1, 0, 1, 1, 1], np.float32))
    G = np.zeros((4, 8), np.float32)
    with pytest.raises(TypeError):
        ctx.feature_embed(dev(G), np.ones(8, np.float32))
    # d = 7 keys have 18-bit fields: |z| >= 131000 is refused there, accepted at d = 6
    big = np.zeros((1, 7), np.float32)
    big[0, 0] = 40000.0
    with pytest.raises(fr.FilterRegError):
        ctx.feature_embed(dev(big), np.ones(7, np.float32))
    ctx.feature_embed(dev(big[:, :6]), np.ones(6, np.float32))


@pytest.mark.parametrize("d", [2, 5, 6, 7])
@pytest.mark.parametrize("pt2pl", [False, True])
def test_estep_matches_oracle(ctx, orc, d, pt2pl):
    rng = np.random.default_rng(10 * d + pt2pl)
    N, M = 4099, 2051
    FY = clustered(d, N, d)
    FX = clustered(d, M, d) + np.float32(0.0)
    Y = pad4(rng.uniform(-1, 1, size=(N, 3)).astype(np.float32))
    Yn = pad4(rng.normal(size=(N, 3)).astype(np.float32)) if pt2pl else None
    sf = rng.uniform(0.1, 0.4, size=d).astype(np.float32)
    out, nv = ctx.estep_features(dev(FX), dev(FY), sf, dev(Y), dev(Yn) if pt2pl else None)
    ref = orc.estep_features(FX, FY, sf, Y, Yn, backend=orc.LATTICE)
    assert within(host(out), ref, Y) <= 1.0
    assert nv == len(orc.FeatureLattice(FY, np.ones(N), sf))
    assert ((host(out)[:, 0] > 0) == (ref[:, 0] > 0)).all()


def test_estep_d3_equals_the_geometric_estep(ctx):
    # features = positions, sigma_f = (s, s, s): the same lattice as fr_estep
    p = synth.depth_frame_pair(2, W=96, H=72)
    s = float(np.float32(0.03))
    feat, nv = ctx.estep_features(dev(p.X[:, :3]), dev(p.Y[:, :3]), [s] * 3, dev(p.Y), dev(p.Yn))
    geo = ctx.estep(dev(p.X), dev(p.Y), dev(p.Yn), sigma=s)
    a, b = host(feat).astype(np.float64), host(geo).astype(np.float64)
    scale = np.abs(b[:, :1]) * np.r_[1.0, [np.abs(p.Y[:, :3]).max()] * 3, [1.0] * 3][None, :]
    assert (np.abs(a - b) <= 1e-4 * (np.abs(b) + scale) + 1e-12).all()


def test_depth_frame_xyz_normal_full_size(ctx, orc):
    # the 320x240 frame pair with 6-d [position, normal] features: every row
    # on the GPU, 2000 sampled rows by the oracle, vertex count exact
    fp = synth.feature_frame_pair(0)
    sf = np.array([0.02] * 3 + [0.25] * 3, np.float32)
    out, nv = ctx.estep_features(dev(fp.FX), dev(fp.FY), sf, dev(fp.Y), dev(fp.Yn))
    rows = np.random.default_rng(1).choice(fp.FX.shape[0], 2000, replace=False)
    ref = orc.estep_features(fp.FX[rows], fp.FY, sf, fp.Y, fp.Yn, backend=orc.LATTICE)
    assert within(host(out)[rows], ref, fp.Y) <= 1.0
    assert nv == len(orc.FeatureLattice(fp.FY, np.ones(fp.FY.shape[0]), sf))


def test_repeated_calls_leave_the_table_empty(ctx, orc):
    # the context keeps one table: alternating shapes, d and residual must
    # give the same sums as the first call of each
    rng = np.random.default_rng(7)
    cases = []
    for d, pt2pl, N in ((6, True, 3000), (6, False, 3000), (3, False, 500), (7, True, 9000), (6, True, 3000)):
        FY = clustered(d + N, N, d)
        FX = clustered(d + N + 1, 700, d)
        Y = pad4(rng.uniform(-1, 1, size=(N, 3)).astype(np.float32))
        Yn = pad4(rng.normal(size=(N, 3)).astype(np.float32)) if pt2pl else None
        sf = np.full(d, 0.3, np.float32)
        cases.append((FX, FY, sf, Y, Yn))
    first = [host(ctx.estep_features(dev(a), dev(b), s, dev(y), dev(n) if n is not None else None)[0])
             for a, b, s, y, n in cases]
    again = [host(ctx.estep_features(dev(a), dev(b), s, dev(y), dev(n) if n is not None else None)[0])
             for a, b, s, y, n in reversed(cases)][::-1]
    for (FX, FY, sf, Y, Yn), f, g in zip(cases, first, again):
        ref = orc.estep_features(FX, FY, sf, Y, Yn, backend=orc.LATTICE)
        assert within(f, ref, Y) <= 1.0
        assert within(g, ref, Y) <= 1.0


def test_single_point_and_ragged_sizes(ctx, orc):
    d = 6
    sf = np.full(d, 0.5, np.float32)
    for N, M in ((1, 1), (1, 300), (255, 1), (257, 513)):
        FY = clustered(N, N, d)
        FX = clustered(N + 1, M, d)
        Y = pad4(np.random.default_rng(N).uniform(-1, 1, size=(N, 3)).astype(np.float32))
        out, nv = ctx.estep_features(dev(FX), dev(FY), sf, dev(Y))
        ref = orc.estep_features(FX, FY, sf, Y, backend=orc.LATTICE)
        assert within(host(out), ref, Y) <= 1.0
    # a model feature on the observation's own feature: M0 = sum_k b_k^2
    F = clustered(5, 1, d)
    out, nv = ctx.estep_features(dev(F), dev(F), sf, dev(pad4(np.ones((1, 3), np.float32))))
    _, b, _ = orc.feature_embed(F, sf)
    assert nv == d + 1
    assert host(out)[0, 0] == pytest.approx(float((b.astype(np.float64) ** 2).sum()), rel=1e-6)


def test_workspace_limit_refuses_then_recovers(ctx, orc):
    import paper_1811_10136_gb300 as fr
    d, N = 6, 20000
    FY = clustered(1, N, d)
    Y = pad4(np.zeros((N, 3), np.float32))
    sf = np.full(d, 0.2, np.float32)
    c2 = fr.Context(0)
    c2.set_workspace_limit(1 << 20)
    with pytest.raises(fr.FilterRegError):
        c2.estep_features(dev(FY[:100]), dev(FY), sf, dev(Y))
    c2.set_workspace_limit(0)
    out, _ = c2.estep_features(dev(FY[:100]), dev(FY), sf, dev(Y))
    ref = orc.estep_features(FY[:100], FY, sf, Y, backend=orc.LATTICE)
    assert within(host(out), ref, Y) <= 1.0


@pytest.mark.parametrize("d", [1, 6, 7])
@pytest.mark.parametrize("pt2pl", [False, True])
def test_exact_matches_oracle(ctx, orc, d, pt2pl):
    rng = np.random.default_rng(20 * d + pt2pl)
    N, M = 3001, 1027
    FY = clustered(d, N, d, scale=0.3)
    FX = clustered(d + 1, M, d, scale=0.3)
    Y = pad4(rng.uniform(-1, 1, size=(N, 3)).astype(np.float32))
    Yn = pad4(rng.normal(size=(N, 3)).astype(np.float32)) if pt2pl else None
    sf = rng.uniform(0.2, 0.6, size=d).astype(np.float32)
    out, _ = ctx.estep_features(dev(FX), dev(FY), sf, dev(Y), dev(Yn) if pt2pl else None, exact=True)
    ref = orc.estep_features(FX, FY, sf, Y, Yn, backend=orc.EXACT)
    assert within(host(out), ref, Y) <= 1.0


def test_profiling_times_the_three_kernels(ctx):
    d, N = 6, 5000
    FY = clustered(3, N, d)
    Y = pad4(np.zeros((N, 3), np.float32))
    sf = np.full(d, 0.3, np.float32)
    ctx.profile(reset=True)
    ctx.set_profiling(True)
    try:
        ctx.estep_features(dev(FY[:200]), dev(FY), sf, dev(Y))
    finally:
        ctx.set_profiling(False)
    prof = ctx.profile(reset=True)
    for name in ("build", "slice", "clear"):
        assert prof[name][0] == 1 and prof[name][1] > 0.0
