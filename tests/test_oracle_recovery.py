"""The oracle's recovery range: perturbations its EM brings back to the truth.

Bumpy sphere: with the stand-in's default bumps (amplitude 0.1, width 0.2 on
a unit sphere of 2,000 points) the rotation is nearly unobservable -- the EM
started at the true pose drifts over a degree away with exact sums -- so a
success rate there says nothing.  With pronounced bumps (amplitude 0.5,
width 0.35) the oracle recovers rotations of 10 degrees (sigma annealed 0.2 ->
0.02 over 60 point-to-point iterations, w = 0.1).

Articulated: the largest joint error is dominated by joints that hardly move
the surface (a revolute axis along its capsule), so recovery is measured on
the posed surface: the mean distance between the model posed at the estimate
and at the truth.  Joint perturbations up to 2 degrees (root 1 degree) come
back to below the 2 mm observation noise.
"""
import numpy as np

from paper_1811_10136_gb300 import synth

F32 = lambda x: float(np.float32(x))  # noqa: E731
SPHERE = dict(amp=0.5, width=0.35, max_trans=0.05, exact_angle=True)


def test_default_bumpy_sphere_leaves_rotation_unobservable(orc):
    p = synth.sphere_bumps_pair(0, max_angle_deg=5.0, max_trans=0.05, exact_angle=True)
    T, _ = orc.register_rigid(p.X, p.Y, None, sigma=F32(0.05), iters=100, w=F32(0.1), backend=orc.EXACT,
                              T0=p.T_gt)
    assert synth.rotation_angle_deg(T, p.T_gt) > 0.5


def test_pronounced_sphere_recovers_ten_degrees(orc):
    errs = []
    for seed in range(8):
        p = synth.sphere_bumps_pair(seed, max_angle_deg=10.0, **SPHERE)
        T, _ = orc.register_rigid(p.X, p.Y, None, sigma=F32(0.2), sigma_end=F32(0.02), iters=60, w=F32(0.1))
        errs.append(synth.rotation_angle_deg(T, p.T_gt))
    assert sum(e < 2.0 for e in errs) >= 7, errs


def test_articulated_recovers_small_joint_perturbations(orc):
    ap = synth.articulated_pair(1000, n_points=10000, max_joint_deg=2.0, root_deg=1.0)
    before, _ = synth.posed_surface_error(ap, np.eye(4), np.zeros_like(ap.q_gt))
    R, q, _ = orc.register_articulated(ap.Xref, ap.body, ap.tree, ap.Y, None, sigma=F32(0.01),
                                       sigma_end=F32(0.005), w=F32(0.1), iters=30)
    after, p99 = synth.posed_surface_error(ap, R, q)
    assert before > 3e-3 and after < 1.5e-3 and p99 < 6e-3, (before, after, p99)
