"""GPU parity of the sharded single registration's pieces (one GPU: shards are
computed one after the other and summed on the host -- no rank waits on
another).

Bar: a shard's normal equations as the single-step parity of the rigid path
(the step they solve to within 2e-6 rad / 2e-6 of the oracle's, weights and
inliers as there), the summed shards equal to the whole model's within float32
summation order, and registrations within the rigid path's 1e-3 rad / 1e-4.
"""
import math

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


def f32(x):
    return float(np.float32(x))


def pose_diff(A, B):
    return math.radians(synth.rotation_angle_deg(A, B)), float(np.linalg.norm(A[:3, 3] - B[:3, 3]))


def upper_to_full(ne):
    A = np.zeros((6, 6))
    t = 0
    for p in range(6):
        for q in range(p, 6):
            A[p, q] = A[q, p] = ne[t]
            t += 1
    return A


@pytest.mark.parametrize("residual", [0, 1])
def test_shard_normal_equations_match_oracle(ctx, orc, residual):
    import paper_1811_10136_gb300 as fr
    p = synth.depth_frame_pair(2, W=160, H=120)
    M = p.X.shape[0]
    a, b = M // 3, 2 * M // 3 + 5  # a ragged middle shard
    s = f32(0.03)
    Yn = p.Yn if residual else None
    g = ctx.rigid_normal_equations(dev(p.X[a:b]), dev(p.Y), dev(Yn) if residual else None, sigma=s,
                                   M_total=M, residual=residual, w=f32(0.1))
    o = orc.rigid_normal_equations(p.X[a:b], p.Y, Yn, sigma=s, M_total=M, residual=residual, w=f32(0.1))
    assert g[29] == o[29]                                  # inliers
    assert g[27] == pytest.approx(o[27], rel=1e-5)         # sum of weights
    assert g[28] == pytest.approx(o[28], rel=1e-3)         # cost
    Ag, Ao = upper_to_full(g), upper_to_full(o)
    assert np.abs(Ag - Ao).max() <= 1e-4 * np.abs(Ao).max()
    Tg, _, okg = fr.rigid_solve_update(g, np.eye(4))
    To, _, oko = fr.rigid_solve_update(o, np.eye(4))
    assert okg and oko
    dr, dt = pose_diff(Tg, To)
    assert dr < 2e-6 and dt < 2e-6, (dr, dt)


def test_shards_sum_to_the_whole_model(ctx):
    p = synth.depth_frame_pair(4, W=160, H=120)
    M = p.X.shape[0]
    T = synth.make_T(synth.random_rotation(np.random.default_rng(3), 0.02), [0.003, 0.0, -0.002])
    kw = dict(sigma=f32(0.02), residual=1, w=f32(0.1), T=T)
    whole = ctx.rigid_normal_equations(dev(p.X), dev(p.Y), dev(p.Yn), M_total=M, **kw)
    cuts = [0, 4097, 11000, M]
    parts = [ctx.rigid_normal_equations(dev(p.X[a:b]), dev(p.Y), dev(p.Yn), M_total=M, **kw)
             for a, b in zip(cuts[:-1], cuts[1:])]
    tot = np.sum(parts, 0)
    assert tot[29] == whole[29]
    assert np.abs(tot[:21] - whole[:21]).max() <= 1e-5 * np.abs(whole[:21]).max()
    assert tot[27] == pytest.approx(whole[27], rel=1e-5)


def test_two_shards_register_like_the_whole_model(ctx, orc):
    # the sharded EM loop with two shards on this GPU, summed on the host in
    # place of the all-reduce, against fr_register_rigid and the oracle
    import paper_1811_10136_gb300 as fr
    p = synth.depth_frame_pair(0)
    M = p.X.shape[0]
    X0, X1, Y, Yn = dev(p.X[:M // 2]), dev(p.X[M // 2:]), dev(p.Y), dev(p.Yn)
    kw = dict(residual=1, w=f32(0.1))

    def provider(T, sigma):
        return sum(ctx.rigid_normal_equations(Xs, Y, Yn, sigma=sigma, M_total=M, T=T, **kw) for Xs in (X0, X1))

    Ts, rep, st = fr.em_sharded(provider, None, sigma_start=f32(0.04), sigma_end=f32(0.01), iters=20, **kw)
    assert st == 0 and rep.iters_run == 20 and rep.degenerate_iters == 0
    Tw, _ = ctx.register_rigid(dev(p.X), Y, Yn, sigma_start=f32(0.04), sigma_end=f32(0.01), iters=20, **kw)
    To, _ = orc.register_rigid(p.X, p.Y, p.Yn, sigma=f32(0.04), sigma_end=f32(0.01), iters=20, w=f32(0.1),
                               residual=1)
    for ref in (Tw, To):
        dr, dt = pose_diff(Ts, ref)
        assert dr < 1e-3 and dt < 1e-4, (dr, dt)
    gr, gt = pose_diff(Ts, p.T_gt)
    assert math.degrees(gr) < 0.1 and gt < 1e-3


def test_register_rigid_sharded_single_rank(ctx, orc):
    p = synth.depth_frame_pair(1, W=160, H=120)
    kw = dict(sigma_start=f32(0.03), sigma_end=f32(0.01), iters=12, residual=1, w=f32(0.1))
    T, rep = ctx.register_rigid_sharded(dev(p.X), dev(p.Y), dev(p.Yn), M_total=p.X.shape[0], **kw)
    assert rep.iters_run == 12
    To, ro = orc.register_rigid(p.X, p.Y, p.Yn, sigma=f32(0.03), sigma_end=f32(0.01), iters=12, w=f32(0.1),
                                residual=1)
    dr, dt = pose_diff(T, To)
    assert dr < 1e-3 and dt < 1e-4, (dr, dt)
    assert rep.last_inliers == pytest.approx(ro.last_inliers, rel=1e-3)


def test_sharded_arguments_refused(ctx):
    import paper_1811_10136_gb300 as fr
    p = synth.depth_frame_pair(1, W=32, H=24)
    with pytest.raises(fr.FilterRegError):
        ctx.rigid_normal_equations(dev(p.X), dev(p.Y), None, M_total=p.X.shape[0] - 1)
    with pytest.raises(fr.FilterRegError):
        ctx.rigid_normal_equations(dev(p.X), dev(p.Y), None, update_sigma=1)
