"""GPU parity of the node-graph model (Section 5.2, Eq. 21) with the CPU
oracle: the dual-quaternion warp, the assembled Gauss-Newton system, and
whole registrations; a single node equals the rigid path.

Bars: warped points within 2e-6 (float32 blend of poses of size ~1);
A within 2e-4 and g within 1e-3 of their largest entries (float32 sums of
~10^3-10^5 terms against float64, E step at float32 positions); node poses
after a registration within the rigid tests' 1e-3 rad / 1e-4 units.
"""
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


def model(ctx, p):
    import paper_1811_10136_gb300 as fr
    return fr.NodeGraph(ctx, dev(p.Xref), dev(p.knn, np.int32), dev(p.skw), p.node_pos, p.edges)


def jitter_poses(K, seed, ang=0.02, trans=0.003):
    rng = np.random.default_rng(seed)
    return np.stack([synth.make_T(synth.random_rotation(rng, ang), rng.uniform(-trans, trans, 3))
                     for _ in range(K)])


@pytest.fixture(scope="module")
def small():
    return synth.nodegraph_pair(1, W=64, H=48, n_nodes=30)


def test_warp_matches_oracle(ctx, orc, small):
    ng = model(ctx, small)
    T = jitter_poses(30, 0, ang=0.3, trans=0.05)
    out = ng.warp(T).cpu().numpy()[:, :3]
    ref = orc.nodegraph_warp(small.Xref, small.knn, small.skw, T)
    assert np.abs(out - ref).max() < 2e-6


@pytest.mark.parametrize("residual", [0, 1])
def test_system_matches_oracle(ctx, orc, small, residual):
    ng = model(ctx, small)
    T = jitter_poses(30, 1)
    sigma = f32(0.02)
    Yn = small.Yn if residual else None
    A, g, rep = ng.system(dev(small.Y), dev(Yn) if residual else None, node_T=T, lam=10.0, residual=residual,
                          sigma_start=sigma, sigma_end=sigma, w=f32(0.1))
    Ao, go, ro = orc.nodegraph_normal_equations(small.Xref, small.knn, small.skw, small.node_pos, small.edges,
                                                small.Y, Yn, sigma=sigma, w=f32(0.1), lam=10.0,
                                                residual=residual, node_T=T)
    assert np.abs(A - Ao).max() <= 2e-4 * np.abs(Ao).max()
    assert np.abs(g - go).max() <= 1e-3 * np.abs(go).max()
    assert abs(rep.last_inliers - ro.last_inliers) <= 2
    assert rep.last_cost == pytest.approx(ro.last_cost, rel=1e-3)
    assert rep.last_sum_w == pytest.approx(ro.last_sum_w, rel=1e-4)


def pose_diffs(Ta, Tb):
    dr = max(math.radians(synth.rotation_angle_deg(a, b)) for a, b in zip(Ta, Tb))
    dt = max(float(np.linalg.norm(a[:3, 3] - b[:3, 3])) for a, b in zip(Ta, Tb))
    return dr, dt


@pytest.mark.parametrize("residual", [0, 1])
def test_registration_matches_oracle(ctx, orc, small, residual):
    ng = model(ctx, small)
    sigma = f32(0.02)
    Yn = small.Yn if residual else None
    Tg, rg = ng.register(dev(small.Y), dev(Yn) if residual else None, lam=10.0, pcg_iters=20, residual=residual,
                         iters=10, sigma_start=sigma, sigma_end=sigma, w=f32(0.1))
    To, ro = orc.register_nodegraph(small.Xref, small.knn, small.skw, small.node_pos, small.edges, small.Y, Yn,
                                    sigma=sigma, w=f32(0.1), lam=10.0, pcg_iters=20, iters=10, residual=residual)
    dr, dt = pose_diffs(Tg, To)
    assert dr < 1e-3 and dt < 1e-4, (dr, dt)
    assert rg.iters_run == 10
    assert rg.last_cost == pytest.approx(ro.last_cost, rel=1e-2)


def test_annealed_sigma_rebuilds(ctx, orc, small):
    ng = model(ctx, small)
    Tg, rg = ng.register(dev(small.Y), dev(small.Yn), lam=10.0, pcg_iters=10, residual=1, iters=6,
                         sigma_start=f32(0.04), sigma_end=f32(0.015), w=f32(0.1))
    To, ro = orc.register_nodegraph(small.Xref, small.knn, small.skw, small.node_pos, small.edges, small.Y,
                                    small.Yn, sigma=f32(0.04), sigma_end=f32(0.015), w=f32(0.1), lam=10.0,
                                    pcg_iters=10, iters=6, residual=1)
    dr, dt = pose_diffs(Tg, To)
    assert dr < 1e-3 and dt < 1e-4, (dr, dt)
    assert rg.lattice_builds == 6


def test_single_node_equals_rigid_path(ctx):
    import paper_1811_10136_gb300 as fr
    q = synth.depth_frame_pair(3, W=96, H=72)
    M = q.X.shape[0]
    knn = np.zeros((M, 4), np.int32)
    skw = np.zeros((M, 4), np.float32)
    skw[:, 0] = 1.0
    ng = fr.NodeGraph(ctx, dev(q.X), dev(knn, np.int32), dev(skw), np.zeros((1, 3)), np.zeros((0, 2), np.int32))
    Tn, rn = ng.register(dev(q.Y), dev(q.Yn), lam=0.0, pcg_iters=3, residual=1, iters=8,
                         sigma_start=f32(0.03), sigma_end=f32(0.015), w=f32(0.1))
    Tr, rr = ctx.register_rigid(dev(q.X), dev(q.Y), dev(q.Yn), residual=1, iters=8, sigma_start=f32(0.03),
                                sigma_end=f32(0.015), w=f32(0.1))
    dr, dt = pose_diffs(Tn, [Tr])
    assert dr < 1e-4 and dt < 1e-5, (dr, dt)
    assert rn.last_inliers == rr.last_inliers


def test_full_workload_matches_oracle(ctx, orc):
    # ~250k model points, 1,000 nodes, 8,000 edges, sigma 2 cm, 10 EM
    # iterations of 20 PCG iterations, point-to-plane, lambda 10.
    p = synth.nodegraph_pair(0)
    ng = model(ctx, p)
    sigma = f32(0.02)
    Tg, rg = ng.register(dev(p.Y), dev(p.Yn), lam=10.0, pcg_iters=20, residual=1, iters=10,
                         sigma_start=sigma, sigma_end=sigma, w=f32(0.1))
    To, ro = orc.register_nodegraph(p.Xref, p.knn, p.skw, p.node_pos, p.edges, p.Y, p.Yn, sigma=sigma,
                                    w=f32(0.1), lam=10.0, pcg_iters=20, iters=10, residual=1)
    dr, dt = pose_diffs(Tg, To)
    assert dr < 1e-3 and dt < 1e-4, (dr, dt)
    # the error along the true surface normal (tangential motion of a smooth
    # surface is not observable by point-to-plane residuals) falls ~20x
    Xg = ng.warp(Tg).cpu().numpy()[:, :3]
    err0 = np.abs(np.sum((p.Xref[:, :3] - p.X_true) * p.Xn_true, 1)).mean()
    err = np.abs(np.sum((Xg - p.X_true) * p.Xn_true, 1)).mean()
    assert err < 0.1 * err0, (err, err0)


def test_rejects_bad_models(ctx, small):
    import paper_1811_10136_gb300 as fr
    bad = small.knn.copy()
    bad[0, 0] = 30
    with pytest.raises(fr.FilterRegError) as e:
        fr.NodeGraph(ctx, dev(small.Xref), dev(bad, np.int32), dev(small.skw), small.node_pos, small.edges)
    assert e.value.status == fr.FR_EINVAL
    edges = small.edges.copy()
    edges[0] = (3, 3)
    with pytest.raises(fr.FilterRegError) as e:
        fr.NodeGraph(ctx, dev(small.Xref), dev(small.knn, np.int32), dev(small.skw), small.node_pos, edges)
    assert e.value.status == fr.FR_EINVAL
    ng = model(ctx, small)
    with pytest.raises(fr.FilterRegError) as e:
        ng.register(dev(small.Y), None, blur=1, iters=2)
    assert e.value.status == fr.FR_ENOTSUPPORTED


def test_launch_count_is_the_same_replayed_or_issued(ctx, small):
    # every kernel counted once, whether the registration is issued directly
    # or replayed from its captured graph
    ng = model(ctx, small)
    kw = dict(lam=10.0, pcg_iters=5, residual=1, iters=3, sigma_start=f32(0.02), sigma_end=f32(0.02), w=f32(0.1))
    counts = []
    for use_graph in (0, 1, 1):
        n0 = ctx.kernel_launches
        ng.register(dev(small.Y), dev(small.Yn), use_graph=use_graph, **kw)
        counts.append(ctx.kernel_launches - n0)
    assert counts[0] == counts[1] == counts[2], counts
    # per iteration: points + edges, preconditioner set-up, 2 per PCG iteration, node update
    assert counts[0] >= 3 * (2 + 1 + 2 * 5 + 1)
