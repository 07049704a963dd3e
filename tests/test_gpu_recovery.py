"""The GPU path recovers what the oracle recovers (its recovery range,
tests/test_oracle_recovery.py): the pronounced-bump sphere rotated by 10
degrees and the articulated model with joints perturbed by up to 2 degrees.

Bar: the same success criteria as the oracle's (rotation error < 2 deg in at
least 7 of 8 seeds; posed-surface error below 1.5 mm), and the sphere poses
within 2e-3 rad of the oracle's.
"""
import math

import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))  # noqa: E731
SPHERE = dict(amp=0.5, width=0.35, max_trans=0.05, exact_angle=True)


@pytest.fixture(scope="module")
def ctx():
    import torch
    import paper_1811_10136_gb300 as fr
    assert torch.cuda.is_available()
    return fr.Context(0)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_sphere_ten_degrees_like_the_oracle(ctx, orc):
    import paper_1811_10136_gb300 as fr
    sp = [synth.sphere_bumps_pair(s, max_angle_deg=10.0, **SPHERE) for s in range(8)]
    res = ctx.register_rigid_batch([(dev(q.X), dev(q.Y), None) for q in sp], sigmas=[(F32(0.2), F32(0.02))] * 8,
                                   residual=fr.FR_PT2PT, iters=60, w=F32(0.1))
    errs = [synth.rotation_angle_deg(T, q.T_gt) for (T, _, _), q in zip(res, sp)]
    assert sum(e < 2.0 for e in errs) >= 7, errs
    for (T, _, st), q in list(zip(res, sp))[:4]:
        assert st == 0
        To, _ = orc.register_rigid(q.X, q.Y, None, sigma=F32(0.2), sigma_end=F32(0.02), iters=60, w=F32(0.1))
        assert math.radians(synth.rotation_angle_deg(T, To)) < 2e-3


def test_articulated_small_perturbation_recovered(ctx):
    import torch
    ap = synth.articulated_pair(1000, n_points=10000, max_joint_deg=2.0, root_deg=1.0)
    R, q, _ = ctx.register_articulated(dev(ap.Xref), torch.from_numpy(ap.body.astype(np.int32)).cuda(), ap.tree,
                                       dev(ap.Y), None, iters=30, sigma_start=F32(0.01), sigma_end=F32(0.005),
                                       w=F32(0.1))
    after, p99 = synth.posed_surface_error(ap, R, q)
    assert after < 1.5e-3 and p99 < 6e-3, (after, p99)
