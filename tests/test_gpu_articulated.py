"""GPU parity of articulated registration (Section 5.1, Algorithm 1) with the
CPU oracle: root pose within 1e-3 rad / 1e-4 units and joint angles within
1e-3 rad; a single Gauss-Newton step much tighter."""
import math

import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_10136_gb300 as fr
    return fr.Context(0)


def dev(a, dtype=np.float32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def f32(x):
    return float(np.float32(x))


def run_both(ctx, orc, p, iters, s0, s1=None, residual=0, w=0.1):
    s1 = s0 if s1 is None else s1
    Yn = p.Yn if residual else None
    Rg, qg, rg = ctx.register_articulated(dev(p.Xref), dev(p.body, np.int32), p.tree, dev(p.Y),
                                          dev(Yn) if residual else None, residual=residual, iters=iters,
                                          sigma_start=f32(s0), sigma_end=f32(s1), w=f32(w))
    Ro, qo, ro = orc.register_articulated(p.Xref, p.body, p.tree, p.Y, Yn, sigma=f32(s0), sigma_end=f32(s1),
                                          w=f32(w), iters=iters, residual=residual)
    return Rg, qg, rg, Ro, qo, ro


def diffs(Rg, qg, Ro, qo):
    return (math.radians(synth.rotation_angle_deg(Rg, Ro)), float(np.linalg.norm(Rg[:3, 3] - Ro[:3, 3])),
            float(np.abs(qg - qo).max()) if len(qg) else 0.0)


@pytest.mark.parametrize("residual", [0, 1])
def test_single_step(ctx, orc, residual):
    p = synth.articulated_pair(11, n_points=8000)
    Rg, qg, rg, Ro, qo, ro = run_both(ctx, orc, p, 1, 0.02, residual=residual)
    dr, dt, dq = diffs(Rg, qg, Ro, qo)
    # The 26 x 26 normal matrix is poorly conditioned (eigenvalue ratio ~1e-5):
    # float32 per-point sums (their order varies between runs) move the step
    # by ~1e-5 rad, so a single step is held to 1e-4 -- 10x inside the bar.
    assert dr < 1e-4 and dt < 1e-5 and dq < 1e-4, (dr, dt, dq)
    assert rg.last_inliers == ro.last_inliers


def test_full_workload(ctx, orc):
    # 16 links, 26 DOF, 30,000 model points, 33,000 observed, sigma 1 cm, 15 iterations.
    p = synth.articulated_pair(0)
    Rg, qg, rg, Ro, qo, ro = run_both(ctx, orc, p, 15, 0.01)
    dr, dt, dq = diffs(Rg, qg, Ro, qo)
    assert dr < 1e-3 and dt < 1e-4 and dq < 1e-3, (dr, dt, dq)
    assert rg.iters_run == 15


def test_annealed_point_to_plane(ctx, orc):
    p = synth.articulated_pair(12, n_points=10000, max_joint_deg=5)
    Rg, qg, rg, Ro, qo, ro = run_both(ctx, orc, p, 8, 0.03, 0.01, residual=1)
    dr, dt, dq = diffs(Rg, qg, Ro, qo)
    assert dr < 1e-3 and dt < 1e-4 and dq < 1e-3, (dr, dt, dq)
    assert rg.lattice_builds == 8


def test_body_without_points_is_degenerate(ctx, orc):
    # A leaf body with joints but no model points leaves its joints' columns
    # of the normal matrix zero: every iteration is degenerate on both sides
    # (no update; the float32 elimination hands the system to the float64
    # factorisation, whose pivot test rejects it).
    p = synth.articulated_pair(13, n_points=6000)
    t = p.tree
    leaves = [b for b in range(1, t.nb) if b not in set(t.parent.tolist()) and (t.joint_body == b).any()]
    assert leaves
    keep = p.body != leaves[0]
    Xref, body = p.Xref[keep], p.body[keep]
    Rg, qg, rg = ctx.register_articulated(dev(Xref), dev(body, np.int32), t, dev(p.Y), None, iters=3,
                                          sigma_start=f32(0.02), sigma_end=f32(0.02), w=f32(0.1))
    Ro, qo, ro = orc.register_articulated(Xref, body, t, p.Y, None, sigma=f32(0.02), w=f32(0.1), iters=3)
    assert ro.degenerate_iters == 3 and rg.degenerate_iters == 3
    assert np.array_equal(Rg, np.eye(4)) and not np.any(qg)
    assert rg.last_inliers == ro.last_inliers


def test_exact_correspondences_recover_planted_pose(ctx):
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
    R, q, rep = ctx.register_articulated(dev(P), dev(B, np.int32), tree, dev(Y), iters=25,
                                         sigma_start=0.003, sigma_end=0.003, w=0.0)
    assert np.abs(q - q_gt).max() < 2e-5
    assert math.radians(synth.rotation_angle_deg(R, R_gt)) < 2e-5
    assert np.linalg.norm(R[:3, 3] - R_gt[:3, 3]) < 2e-6


def test_invalid_tree(ctx):
    import paper_1811_10136_gb300 as fr
    tree = synth.random_kintree(1)
    bad = synth.KinTree(tree.parent.copy(), tree.offset, tree.joint_body, tree.joint_axis, tree.q_min,
                        tree.q_max, tree.radius, tree.length)
    bad.parent[3] = 7
    X = dev(np.zeros((10, 4)))
    with pytest.raises(fr.FilterRegError) as e:
        ctx.register_articulated(X, dev(np.zeros(10), np.int32), bad, X, iters=1)
    assert e.value.status == fr.FR_EINVAL


def test_joint_limits_clamp_alike(ctx, orc):
    # Joint limits narrowed to +-3 degrees while the observation is posed with
    # joints up to +-8 degrees: the updates push joints past their limits and
    # both implementations clamp them (Section 5.1's joint-limited model).
    # Clamped joints sit exactly on a limit on both sides (the same set of
    # joints); every other parameter agrees within the articulated bar.
    import dataclasses
    wide = synth.random_kintree(21)
    p = synth.articulated_pair(21, n_points=12000, max_joint_deg=8.0, root_deg=1.0, root_trans=0.002,
                               outlier_frac=0.0, tree=wide)
    lim = np.radians(3.0)
    narrow = dataclasses.replace(wide, q_min=np.full_like(wide.q_min, -lim), q_max=np.full_like(wide.q_max, lim))
    assert (np.abs(p.q_gt) > lim).sum() >= 4
    args = dict(iters=10, sigma=f32(0.01), w=f32(0.1))
    Rg, qg, rg = ctx.register_articulated(dev(p.Xref), dev(p.body, np.int32), narrow, dev(p.Y), None,
                                          iters=args["iters"], sigma_start=args["sigma"], sigma_end=args["sigma"],
                                          w=args["w"])
    Ro, qo, ro = orc.register_articulated(p.Xref, p.body, narrow, p.Y, None, sigma=args["sigma"],
                                          w=args["w"], iters=args["iters"])
    at_lim_g = np.isclose(np.abs(qg), lim, rtol=0, atol=0)
    at_lim_o = np.isclose(np.abs(qo), lim, rtol=0, atol=0)
    assert at_lim_o.sum() >= 2, qo
    np.testing.assert_array_equal(at_lim_g, at_lim_o)
    np.testing.assert_array_equal(qg[at_lim_g], qo[at_lim_o])
    assert (np.abs(qg) <= lim).all() and (np.abs(qo) <= lim).all()
    dr, dt, dq = diffs(Rg, qg, Ro, qo)
    assert dr < 1e-3 and dt < 1e-4 and dq < 1e-3, (dr, dt, dq)


# ---- batched articulated registration (concurrent streams) ------------------

def batch_items(pairs, residual, poses=None):
    return [(dev(p.Xref), dev(p.body, np.int32), dev(p.Y), dev(p.Yn) if residual else None,
             None if poses is None else poses[b][0], None if poses is None else poses[b][1])
            for b, p in enumerate(pairs)]


@pytest.mark.parametrize("residual", [0, 1])
def test_batch_equals_single_registrations(ctx, orc, residual):
    # Five registrations of one tree in one call: each equals the same
    # registration run alone, and the first matches the oracle.
    tree = synth.random_kintree(20)
    pairs = [synth.articulated_pair(30 + s, n_points=6000, max_joint_deg=5, tree=tree) for s in range(5)]
    kw = dict(residual=residual, iters=6, sigma_start=f32(0.03), sigma_end=f32(0.01), w=f32(0.1))
    items = batch_items(pairs, residual)
    out = ctx.register_articulated_batch(items, tree, **kw)
    for (Rb, qb, rb, st), it in zip(out, items):
        assert st == 0
        Rs, qs, rs = ctx.register_articulated(it[0], it[1], tree, it[2], it[3], **kw)
        dr, dt, dq = diffs(Rb, qb, Rs, qs)
        assert dr < 1e-3 and dt < 1e-4 and dq < 1e-3, (dr, dt, dq)
        assert rb.iters_run == rs.iters_run == 6 and rb.lattice_builds == rs.lattice_builds
    p = pairs[0]
    Ro, qo, ro = orc.register_articulated(p.Xref, p.body, tree, p.Y, p.Yn if residual else None,
                                          sigma=f32(0.03), sigma_end=f32(0.01), w=f32(0.1), iters=6,
                                          residual=residual)
    dr, dt, dq = diffs(out[0][0], out[0][1], Ro, qo)
    assert dr < 1e-3 and dt < 1e-4 and dq < 1e-3, (dr, dt, dq)


def test_batch_more_items_than_streams(ctx):
    # More items than registrations in flight (waves), with given initial
    # poses and angles: each item as run alone from the same start.
    import paper_1811_10136_gb300 as fr
    tree = synth.random_kintree(21)
    n = fr.FR_ART_CONCURRENT + 3
    pairs = [synth.articulated_pair(50 + s, n_points=1500, max_joint_deg=5, tree=tree) for s in range(n)]
    rng = np.random.default_rng(5)
    poses = [(synth.make_T(synth.random_rotation(rng, np.radians(1.0)), rng.uniform(-0.002, 0.002, 3)),
              rng.uniform(-0.02, 0.02, tree.nj)) for _ in range(n)]
    kw = dict(residual=0, iters=3, sigma_start=f32(0.02), sigma_end=f32(0.02), w=f32(0.1))
    items = batch_items(pairs, 0, poses)
    launches0 = ctx.kernel_launches
    out = ctx.register_articulated_batch(items, tree, **kw)
    assert ctx.kernel_launches - launches0 == n * (3 + 2)   # first build, 3 iterations, final clear
    for (Rb, qb, rb, st), it in zip(out, items):
        assert st == 0
        Rs, qs, rs = ctx.register_articulated(it[0], it[1], tree, it[2], None, root_T0=it[4], q0=it[5], **kw)
        dr, dt, dq = diffs(Rb, qb, Rs, qs)
        assert dr < 1e-3 and dt < 1e-4 and dq < 1e-3, (dr, dt, dq)


def test_batch_rejects_bad_items_before_work(ctx):
    import paper_1811_10136_gb300 as fr
    tree = synth.random_kintree(22)
    p = synth.articulated_pair(60, n_points=1000, tree=tree)
    good = batch_items([p], 0)[0]
    bad = good[:4] + (np.full((4, 4), np.nan), None)
    launches0 = ctx.kernel_launches
    with pytest.raises(fr.FilterRegError) as e:
        ctx.register_articulated_batch([good, bad], tree, iters=2)
    assert e.value.status == fr.FR_EINVAL
    assert ctx.kernel_launches == launches0
