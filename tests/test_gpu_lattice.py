"""GPU parity of the lattice and E-step kernels against the CPU oracle.

Bar: lattice keys, simplex vertices and barycentric weights bit-exact (the
same float operations decide them on both sides); splat / blur / slice values
and E-step sums within 1e-4 relative of the oracle's float64 sums (the GPU
accumulates float32 atomics in arbitrary order).
"""
import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-4


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


def random_points(seed, n, spread=1.0):
    rng = np.random.default_rng(seed)
    P = np.zeros((n, 4), np.float32)
    P[:, :3] = rng.uniform(-spread, spread, size=(n, 3))
    return P


def close(gpu, ref, scale, rel=REL):
    """|gpu - ref| <= rel (|ref| + scale) elementwise, scale per row or scalar."""
    err = np.abs(gpu.astype(np.float64) - ref)
    bound = rel * (np.abs(ref) + scale)
    return bool((err <= bound).all()), float((err / bound).max()) if err.size else 0.0


@pytest.mark.parametrize("n", [1, 31, 257, 3001])
@pytest.mark.parametrize("sigma", [0.5, 0.02, 0.0123])
def test_embed_bit_exact(ctx, orc, n, sigma):
    P = random_points(n + int(sigma * 1e4), n, 1.5)
    k_ref, b_ref, _, _, st = orc.lattice_embed(P, sigma)
    assert st == 0
    keys, bary = ctx.lattice_embed(dev(P), sigma)
    np.testing.assert_array_equal(host(keys), k_ref)
    np.testing.assert_array_equal(host(bary) + 0.0, b_ref + 0.0)


def test_embed_ties_on_lattice_points(ctx, orc):
    # Points whose elevations hit lattice vertices, edges and faces exactly
    # exercise the rank tie-break (lower coordinate index first).
    alpha = np.sqrt(2.0 / 3.0) * 4.0
    scale = np.array([alpha / np.sqrt(i * (i + 1)) for i in (1, 2, 3)])
    cs = []
    for a in (-1, 0, 0.5, 1):
        for b in (-0.5, 0, 1):
            for c in (0, 0.25, 1, -1):
                cs.append([a, b, c])
    P = np.zeros((len(cs), 4), np.float32)
    P[:, :3] = np.array(cs) / scale
    k_ref, b_ref, *_ = orc.lattice_embed(P, 1.0)
    keys, bary = ctx.lattice_embed(dev(P), 1.0)
    np.testing.assert_array_equal(host(keys), k_ref)
    np.testing.assert_array_equal(host(bary) + 0.0, b_ref + 0.0)


def test_embed_depth_frame_full_size(ctx, orc):
    p = synth.depth_frame_pair(0)
    for sigma in (0.04, 0.01):
        k_ref, b_ref, *_ = orc.lattice_embed(p.Y, sigma)
        keys, bary = ctx.lattice_embed(dev(p.Y), sigma)
        np.testing.assert_array_equal(host(keys), k_ref)
        np.testing.assert_array_equal(host(bary) + 0.0, b_ref + 0.0)


def test_embed_rejects_bad_input(ctx):
    import paper_1811_10136_gb300 as fr
    P = np.zeros((3, 4), np.float32)
    P[1, 0] = np.nan
    with pytest.raises(fr.FilterRegError) as e:
        ctx.lattice_embed(dev(P), 0.1)
    assert e.value.status == fr.FR_EINVAL
    P[1, 0] = 1e8
    with pytest.raises(fr.FilterRegError):
        ctx.lattice_embed(dev(P), 0.1)


def _sorted_vertices(keys, vals):
    order = np.lexsort(keys.T[::-1])
    return keys[order], vals[order]


@pytest.mark.parametrize("n,vdim,sigma", [(1, 4, 0.1), (300, 4, 0.07), (5000, 7, 0.05), (4097, 8, 0.2)])
def test_build_splat_vertices_match(ctx, orc, n, vdim, sigma):
    P = random_points(n, n, 0.7)
    rng = np.random.default_rng(n)
    V = rng.normal(size=(n, vdim)).astype(np.float32)
    lat = ctx.lattice_build(dev(P), sigma)
    lat.splat(dev(V))
    nv, cap, vd = lat.info()
    keys, vals = lat.vertices()
    keys, vals = _sorted_vertices(host(keys), host(vals))
    ref = orc.Lattice(P, V.astype(np.float64), sigma)
    rk, rv = ref.vertices()
    assert nv == len(ref) == keys.shape[0]
    np.testing.assert_array_equal(keys, rk)            # the same vertex set, bit for bit
    # per-vertex magnitude scale: sum of |b v| bounded by the count of splats * max|v|
    scale = np.abs(V).max() * 1.0
    ok, worst = close(vals, rv, scale)
    assert ok, worst


@pytest.mark.parametrize("blur", [False, True])
def test_slice_matches_oracle(ctx, orc, blur):
    Y = random_points(21, 6000, 0.5)
    Q = random_points(22, 2500, 0.55)
    V = np.concatenate([np.ones((6000, 1)), Y[:, :3]], 1).astype(np.float32)
    sigma = 0.03
    lat = ctx.lattice_build(dev(Y), sigma)
    lat.splat(dev(V))
    if blur:
        lat.blur()
    out = host(lat.slice(dev(Q)))
    ref, _ = orc.Lattice(Y, V.astype(np.float64), sigma, blur=blur).slice(Q)
    m0 = ref[:, :1]
    ok, worst = close(out, ref, m0 * 1.0 + 1e-6)
    assert ok, worst


def moved_like_kernel(X, T):
    """x = T x_ref in float32 with the kernel's operation order (each product and
    sum rounded): ((T_j0 x + T_j1 y) + T_j2 z) + T_j3."""
    P = T.astype(np.float32)
    out = np.zeros_like(X)
    for j in range(3):
        a = P[j, 0] * X[:, 0] + P[j, 1] * X[:, 1]
        out[:, j] = (a + P[j, 2] * X[:, 2]) + P[j, 3]
    return out


@pytest.mark.parametrize("pt2pl", [False, True])
@pytest.mark.parametrize("blur", [False, True])
def test_estep_matches_oracle_small(ctx, orc, pt2pl, blur):
    # The GPU moves the model by T itself; the oracle is given the same float
    # positions (bit-exact embedding) at the identity pose.
    p = synth.depth_frame_pair(1, W=96, H=72)
    T = synth.make_T(synth.random_rotation(np.random.default_rng(0), 0.02), [0.003, -0.002, 0.001])
    sigma = float(np.float32(0.03))
    Yn = p.Yn if pt2pl else None
    out = host(ctx.estep(dev(p.X), dev(p.Y), dev(Yn) if pt2pl else None, sigma=sigma, blur=blur, T=T))
    ref = orc.estep(moved_like_kernel(p.X, T), p.Y, Yn, sigma, backend=orc.LATTICE, blur=blur)
    ymax = np.abs(p.Y[:, :3]).max()
    scale = ref[:, :1] * np.r_[1.0, [ymax] * 3, [1.0] * (3 if pt2pl else 0)][None, :]
    ok, worst = close(out, ref, scale + 1e-6)
    assert ok, worst


def test_estep_full_size_depth_frames(ctx, orc):
    # The 320x240 workload at the first and last sigma of its schedule, at the
    # identity pose (both sides embed the same float positions).
    p = synth.depth_frame_pair(0)
    ymax = np.abs(p.Y[:, :3]).max()
    for sigma in (0.04, 0.01):
        out = host(ctx.estep(dev(p.X), dev(p.Y), dev(p.Yn), sigma=sigma))
        ref = orc.estep(p.X, p.Y, p.Yn, sigma, backend=orc.LATTICE)
        scale = ref[:, :1] * np.r_[1.0, [ymax] * 3, [1.0] * 3][None, :]
        ok, worst = close(out, ref, scale + 1e-6)
        assert ok, worst
        assert (out[:, 0] > 0).sum() == (ref[:, 0] > 0).sum()


def test_estep_max_size_sampled(ctx, orc):
    # 300k observation points (the largest request size): the GPU E step at a
    # random sample of 2000 model points against the oracle at the same points.
    p = synth.depth_frame_pair(5, W=632, H=474)
    assert p.Y.shape[0] >= 280_000
    out = host(ctx.estep(dev(p.X), dev(p.Y), dev(p.Yn), sigma=0.02))
    idx = np.random.default_rng(0).choice(p.X.shape[0], 2000, replace=False)
    ref = orc.estep(p.X[idx], p.Y, p.Yn, 0.02, backend=orc.LATTICE)
    ymax = np.abs(p.Y[:, :3]).max()
    scale = ref[:, :1] * np.r_[1.0, [ymax] * 3, [1.0] * 3][None, :]
    ok, worst = close(out[idx], ref, scale + 1e-6)
    assert ok, worst


def test_augmentation_queries_do_not_insert(ctx, orc):
    # Slicing is a pure query: the vertex count is unchanged by slicing.
    Y = random_points(31, 2000, 0.5)
    lat = ctx.lattice_build(dev(Y), 0.05)
    lat.splat(dev(np.ones((2000, 1), np.float32)))
    before = lat.info()[0]
    lat.slice(dev(random_points(32, 3000, 2.0)))
    keys, _ = lat.vertices()
    assert keys.shape[0] == before == len(orc.Lattice(Y, np.ones(2000), 0.05))
