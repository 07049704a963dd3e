"""16-bit lattice storage (bfloat16 / half records made from float32 sums)
against the float64 oracle, with error bounds derived from the rounding.

The slice reads, per simplex vertex k, W_k and r_k = V_k - W_k p_k (V_k the
vertex's sum of b y, p_k its position) rounded to 16 bits: relative error at
most u (2^-8 bfloat16, 2^-11 half) each.  The vertex centroid q_k = V_k / W_k
lies within the cell's diameter of p_k: in the elevated space every simplex
edge is at most 4 long (d = 3: vertices 0, (1,1,1,-3), (2,2,-2,-2),
(3,-1,-1,-1) and permutations) and the elevation scales world distances by
alpha / sigma (alpha = 4 sqrt(2/3)), so |q_k - p_k| <= R = sqrt(3/2) sigma.
Hence, to first order in u:
  M0:              |dM0| <= u M0
  target M1 / M0:  |d| <= 2 u R (each q_k) + 4 u R (the weights' shift,
                   every q_k within 2R of the query)  = 6 u R
  Nsum (pt2pl):    |dN_c| <= u sum_k b_k |N_k| <= u M0   (|n| = 1)
plus the float32 path's own error (the splat's float32 atomics).
"""
import math

import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

pytestmark = pytest.mark.gpu

U = {1: 2.0 ** -8, 2: 2.0 ** -11}          # FR_BF16, FR_FP16 unit roundoff
F32_REL = 1e-4                             # the float32 path's bound on the same sums
F32_TARGET = 2e-5                          # float32 splat error on M1 / M0, x max|y|


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
    return t.detach().cpu().numpy().astype(np.float64)


def f32(x):
    return float(np.float32(x))


def check_estep(out, ref, u, sigma, ymax, pt2pl):
    """The bounds of the module docstring; returns the worst error / bound per term."""
    R = math.sqrt(1.5) * sigma
    m0, m0r = out[:, 0], ref[:, 0]
    assert ((m0 > 0) == (m0r > 0)).all()
    b0 = (u * (1 + 1e-3) + F32_REL) * m0r + 1e-6
    worst = {"M0": float((np.abs(m0 - m0r) / b0).max())}
    live = m0r > 1e-3 * m0r.max()
    t, tr = out[live, 1:4] / m0[live, None], ref[live, 1:4] / m0r[live, None]
    bt = 6 * u * R * (1 + 1e-2) + F32_TARGET * ymax + 1e-6 * (m0r.max() / m0r[live])
    worst["target"] = float((np.abs(t - tr).max(1) / bt).max())
    if pt2pl:
        bn = (u * (1 + 1e-3) + F32_REL) * m0r[:, None] + 1e-6
        worst["Nsum"] = float((np.abs(out[:, 4:7] - ref[:, 4:7]) / bn).max())
    return worst


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("pt2pl", [False, True])
@pytest.mark.parametrize("sigma", [0.03, 0.01])
def test_estep_within_rounding_bound(ctx, orc, storage, pt2pl, sigma):
    p = synth.depth_frame_pair(1, W=96, H=72)
    sigma = f32(sigma)
    Yn = p.Yn if pt2pl else None
    out = host(ctx.estep(dev(p.X), dev(p.Y), dev(Yn) if pt2pl else None, sigma=sigma,
                         storage=storage))
    ref = orc.estep(p.X, p.Y, Yn, sigma, backend=orc.LATTICE)
    worst = check_estep(out, ref, U[storage], sigma, np.abs(p.Y[:, :3]).max(), pt2pl)
    assert max(worst.values()) <= 1.0, worst


def test_estep_fp32_storage_is_fr_estep(ctx):
    p = synth.depth_frame_pair(1, W=96, H=72)
    a = host(ctx.estep(dev(p.X), dev(p.Y), dev(p.Yn), sigma=0.02))
    b = host(ctx.estep(dev(p.X), dev(p.Y), dev(p.Yn), sigma=0.02, storage=0))
    np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("storage", [1, 2])
def test_estep_full_size_depth_frame(ctx, orc, storage):
    # 76,800 observation points: half precision is scaled by 2^-3 here.
    p = synth.depth_frame_pair(0)
    for sigma in (0.04, 0.01):
        sigma = f32(sigma)
        out = host(ctx.estep(dev(p.X), dev(p.Y), dev(p.Yn), sigma=sigma, storage=storage))
        ref = orc.estep(p.X, p.Y, p.Yn, sigma, backend=orc.LATTICE)
        worst = check_estep(out, ref, U[storage], sigma, np.abs(p.Y[:, :3]).max(), True)
        assert max(worst.values()) <= 1.0, (sigma, worst)


def test_half_storage_does_not_overflow(ctx, orc):
    # 100,000 observations within 1e-4 of one point: a vertex's weight sum is
    # ~25,000, above half's range / 4 without the 2^-e scaling (e = 3 here).
    rng = np.random.default_rng(3)
    Y = np.zeros((100_000, 4), np.float32)
    Y[:, :3] = 0.25 + rng.normal(0.0, 1e-4, size=(100_000, 3))
    X = np.zeros((64, 4), np.float32)
    X[:, :3] = 0.25 + rng.normal(0.0, 0.01, size=(64, 3))
    sigma = f32(0.05)
    out = host(ctx.estep(dev(X), dev(Y), None, sigma=sigma, storage=2))
    ref = orc.estep(X, Y, None, sigma, backend=orc.LATTICE)
    assert np.isfinite(out).all()
    worst = check_estep(out, ref, U[2], sigma, np.abs(Y[:, :3]).max(), False)
    assert max(worst.values()) <= 1.0, worst


def test_storage_rejects_blur(ctx):
    import paper_1811_10136_gb300 as fr
    p = synth.sphere_bumps_pair(0)
    with pytest.raises(fr.FilterRegError) as e:
        ctx.register_rigid(dev(p.X), dev(p.Y), None, storage=1, iters=2, blur=1)
    assert e.value.status == fr.FR_ENOTSUPPORTED
    with pytest.raises(fr.FilterRegError) as e:
        ctx.register_rigid(dev(p.X), dev(p.Y), None, storage=7, iters=2)
    assert e.value.status == fr.FR_EINVAL


def rms_radius(X):
    P = X[:, :3].astype(np.float64)
    return float(np.sqrt(((P - P.mean(0)) ** 2).sum(1).mean()))


@pytest.fixture(scope="module")
def depth_oracle(orc):
    # The benchmark's workload: 320 x 240 point-to-plane, sigma 0.04 -> 0.01, 20 iterations.
    p = synth.depth_frame_pair(0)
    To, ro = orc.register_rigid(p.X, p.Y, p.Yn, sigma=f32(0.04), sigma_end=f32(0.01), w=f32(0.1),
                                iters=20, residual=1, backend=orc.LATTICE)
    return p, To


@pytest.mark.parametrize("storage", [1, 2])
def test_registration_within_rounding_bound(ctx, depth_oracle, storage):
    # Each iteration's targets move by at most 6 u R (R at that sigma); the
    # Gauss-Newton fit of a pose to targets all moved by at most e moves the
    # translation by at most e and the rotation by at most e / r (r: the model's
    # rms radius), so the final pose stays within those of the oracle's
    # (allowing the float32 path's own tolerance on top).
    p, To = depth_oracle
    Tg, rg = ctx.register_rigid(dev(p.X), dev(p.Y), dev(p.Yn), residual=1, iters=20,
                                sigma_start=f32(0.04), sigma_end=f32(0.01), w=f32(0.1), storage=storage)
    e = 6 * U[storage] * math.sqrt(1.5) * 0.01
    dr = math.radians(synth.rotation_angle_deg(Tg, To))
    dt = float(np.linalg.norm(Tg[:3, 3] - To[:3, 3]))
    assert dr <= 1e-3 + e / rms_radius(p.X) and dt <= 1e-4 + e, (dr, dt, e)
    assert rg.iters_run == 20 and rg.degenerate_iters == 0


@pytest.mark.parametrize("storage", [1, 2])
def test_kahan_sums_with_16bit_storage(ctx, depth_oracle, storage):
    # 16-bit lattice records with Kahan-compensated float32 partial sums of
    # J^T W J: the same bound as plain 16-bit storage (compensation only
    # shrinks the float32 part of the error).
    p, To = depth_oracle
    Tg, rg = ctx.register_rigid(dev(p.X), dev(p.Y), dev(p.Yn), residual=1, iters=20, sigma_start=f32(0.04),
                                sigma_end=f32(0.01), w=f32(0.1), storage=storage, kahan=1)
    e = 6 * U[storage] * math.sqrt(1.5) * 0.01
    dr = math.radians(synth.rotation_angle_deg(Tg, To))
    dt = float(np.linalg.norm(Tg[:3, 3] - To[:3, 3]))
    assert dr <= 1e-3 + e / rms_radius(p.X) and dt <= 1e-4 + e, (dr, dt, e)
    res = ctx.register_rigid_batch([(dev(p.X), dev(p.Y), dev(p.Yn))], residual=1, iters=20, sigma_start=f32(0.04),
                                   sigma_end=f32(0.01), w=f32(0.1), storage=storage, kahan=1)
    dr = math.radians(synth.rotation_angle_deg(res[0][0], To))
    assert res[0][2] == 0 and dr <= 1e-3 + e / rms_radius(p.X)


@pytest.mark.parametrize("storage", [1, 2])
def test_nodegraph_16bit_storage(ctx, storage):
    # The height-field node graph (the benchmark's shape: ~250k points, 1,000
    # nodes, sigma 2 cm, 10 EM x 20 PCG, lambda 10) with 16-bit lattice
    # records against the float32 records.  Each target moves by at most
    # e = 6 u R; the regularised least-squares fit of the node poses to the
    # targets moves the warped surface by at most e (rms) -- plus the float32
    # path's own 1e-4 -- and its error along the true normals by at most e.
    import paper_1811_10136_gb300 as fr
    p = synth.nodegraph_pair(0)
    ng = fr.NodeGraph(ctx, dev(p.Xref), torch_int(p.knn), dev(p.skw), p.node_pos, p.edges)
    sigma = f32(0.02)
    kw = dict(lam=10.0, pcg_iters=20, residual=1, iters=10, sigma_start=sigma, sigma_end=sigma, w=f32(0.1))
    T32, r32 = ng.register(dev(p.Y), dev(p.Yn), **kw)
    T16, r16 = ng.register(dev(p.Y), dev(p.Yn), storage=storage, **kw)
    X32 = ng.warp(T32).cpu().numpy()[:, :3].astype(np.float64)
    X16 = ng.warp(T16).cpu().numpy()[:, :3].astype(np.float64)
    e = 6 * U[storage] * math.sqrt(1.5) * 0.02
    rms = float(np.sqrt(((X16 - X32) ** 2).sum(1).mean()))
    assert rms <= 1e-4 + e, (rms, e)
    en32 = np.abs(np.sum((X32 - p.X_true) * p.Xn_true, 1)).mean()
    en16 = np.abs(np.sum((X16 - p.X_true) * p.Xn_true, 1)).mean()
    assert en16 <= en32 + e, (en16, en32, e)
    assert r16.iters_run == 10 and r16.lattice_vertices == r32.lattice_vertices
    ng.close()


def torch_int(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


@pytest.mark.parametrize("storage", [1, 2])
def test_batch_matches_single_path(ctx, storage):
    # The batched launch runs the same kernels on the same data: each item's
    # pose equals the single-pair call's within the rounding bound of one
    # 16-bit ulp flip (float32 sums in another order may round to the other
    # neighbour).
    views = [(96, 72, 105), (160, 120, 103), (200, 150, 105)]
    pairs = [synth.depth_frame_pair(s, W=w, H=h) for (w, h, s) in views]
    sig = [(f32(0.04), f32(0.01))] * len(pairs)
    res = ctx.register_rigid_batch([(dev(q.X), dev(q.Y), dev(q.Yn)) for q in pairs], sig,
                                   [f32(0.1)] * len(pairs), residual=1, iters=12, storage=storage)
    e = 6 * U[storage] * math.sqrt(1.5) * 0.01
    for q, (Tb, rb, stb) in zip(pairs, res):
        assert stb == 0
        Ts, rs = ctx.register_rigid(dev(q.X), dev(q.Y), dev(q.Yn), residual=1, iters=12,
                                    sigma_start=f32(0.04), sigma_end=f32(0.01), w=f32(0.1),
                                    storage=storage)
        dr = math.radians(synth.rotation_angle_deg(Tb, Ts))
        dt = float(np.linalg.norm(Tb[:3, 3] - Ts[:3, 3]))
        assert dr <= 1e-4 + e / rms_radius(q.X) and dt <= 1e-5 + e, (dr, dt)


@pytest.mark.parametrize("storage", [1, 2])
def test_articulated_exact_correspondences(ctx, storage):
    # Algorithm 1 on 16-bit storage, observation = the model's own points at a
    # planted pose, points >= 8 mm apart, sigma 3 mm: each vertex holds one
    # observation, so every q_k is that point and a restored target is off by
    # at most 2 u R (the weights' shift cancels to first order).  The fixed
    # point is the least-squares fit to targets moved by at most e = 2 u R:
    # its model points lie within e (rms) of the planted ones, whatever the
    # conditioning of the 26 parameters (the normal matrix's eigenvalue ratio
    # is ~1e-5, so the parameters themselves may move much further).
    tree = synth.random_kintree(3)
    rng = np.random.default_rng(4)
    P, _, B = synth.sample_capsules(tree, 4000, rng)
    Tz = synth.pose_bodies(tree, np.eye(4), np.zeros(tree.nj))
    W = np.einsum("nij,nj->ni", Tz[B][:, :3, :3], P[:, :3]) + Tz[B][:, :3, 3]
    keep = []
    for i in range(len(W)):
        if all(np.linalg.norm(W[i] - W[j]) >= 0.008 for j in keep):
            keep.append(i)
    P, B = P[keep], B[keep]
    q_gt = rng.uniform(-1, 1, tree.nj) * np.radians(0.15)
    R_gt = synth.make_T(synth.random_rotation(rng, np.radians(0.1)), [0.0004, -0.0003, 0.0002])
    Tb = synth.pose_bodies(tree, R_gt, q_gt)
    Y = np.zeros_like(P)
    Y[:, :3] = np.einsum("nij,nj->ni", Tb[B][:, :3, :3], P[:, :3].astype(np.float64)) + Tb[B][:, :3, 3]
    import torch
    R, q, rep = ctx.register_articulated(dev(P), torch.from_numpy(B.astype(np.int32)).cuda(), tree, dev(Y),
                                         iters=25, sigma_start=f32(0.003), sigma_end=f32(0.003), w=0.0,
                                         storage=storage)
    e = 2 * U[storage] * math.sqrt(1.5) * 0.003
    Te = synth.pose_bodies(tree, R, q)
    Xe = np.einsum("nij,nj->ni", Te[B][:, :3, :3], P[:, :3].astype(np.float64)) + Te[B][:, :3, 3]
    rms = float(np.sqrt(((Xe - Y[:, :3]) ** 2).sum(1).mean()))
    assert rms <= 1e-6 + e, (rms, e, float(np.abs(q - q_gt).max()))
