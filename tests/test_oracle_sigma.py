"""The oracle's sigma update (Section 3.3: sigma as a decision variable; its
closed form, which the paper defers to a missing supplement, re-derived as
the maximiser over sigma of the expected complete-data log-likelihood with
the E step's posteriors), pinned against values fixed independently:
  - one model point and one observation at distance r: sigma^2 = r^2 / 3;
  - a numeric 1-D maximisation of Q(sigma) = sum_ij P_ij [-|x_i - y_j|^2 /
    (2 sigma^2) - 3 log sigma] with P_ij = K_ij / (sum_k K_ik + c) computed
    here in numpy from the definitions (exact back-end);
  - the lattice back-end's update equals the same formula evaluated from the
    lattice slice of the values [1, y, |y|^2], divided by the lattice kernel's
    per-axis variance in units of sigma^2 (1/4, a closed form checked here
    against the kernel's measured second moment): the sigma at which the
    kernel actually used matches the residuals;
  - so the lattice update settles where the exact one does (its sigma times
    the kernel's width ratio 1/2) instead of contracting to its floor;
  - on a clean planted motion the updated-sigma EM recovers the motion and
    needs fewer iterations than the fixed-sigma EM to reach the same stop."""
import math

import numpy as np
import pytest

from paper_1811_10136_gb300 import synth


def _cloud(rng, n, scale=0.2):
    P = np.zeros((n, 4), np.float32)
    P[:, :3] = rng.normal(scale=scale, size=(n, 3))
    return P


def test_single_pair_closed_form(orc):
    X = np.array([[0.0, 0.0, 0.0, 0.0]], np.float32)
    Y = np.array([[0.03, -0.02, 0.01, 0.0]], np.float32)
    r2 = float(np.sum(Y[0, :3].astype(np.float64) ** 2))
    _, rep = orc.register_rigid(X, Y, None, sigma=0.05, sigma_end=1e-6, w=0.0, iters=1, backend=orc.EXACT,
                                update_sigma=True)
    assert rep.sigma_next ** 2 == pytest.approx(r2 / 3.0, rel=1e-12)


@pytest.mark.parametrize("w", [0.0, 0.2])
def test_matches_numeric_maximisation(orc, w):
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(41)
    X, Y = _cloud(rng, 60), _cloud(rng, 80)
    sigma = 0.1
    _, rep = orc.register_rigid(X, Y, None, sigma=sigma, sigma_end=1e-6, w=w, iters=1, backend=orc.EXACT,
                                update_sigma=True)
    x = X[:, :3].astype(np.float64)
    y = Y[:, :3].astype(np.float64)
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    K = np.exp(-d2 / (2 * sigma * sigma))
    # the outlier constant of Eq. 7 in the unnormalised kernel's units
    c = w / (1 - w) * (len(y) / len(x)) * sigma ** 3 * (2 * math.pi) ** 1.5
    P = K / (K.sum(1, keepdims=True) + c)

    def negQ(log_s):
        s2 = math.exp(2 * log_s)
        return -float((P * (-d2 / (2 * s2) - 3 * log_s)).sum())

    res = scipy_opt.minimize_scalar(negQ, bounds=(math.log(1e-3), math.log(1.0)), method="bounded",
                                    options={"xatol": 1e-12})
    assert rep.sigma_next == pytest.approx(math.exp(res.x), rel=1e-6)


def test_lattice_update_from_its_own_slice(orc):
    rng = np.random.default_rng(42)
    p = synth.sphere_bumps_pair(42, n_model=400, n_obs=500, outlier_frac=0.0)
    sigma = float(np.float32(0.05))
    w = 0.1
    _, rep = orc.register_rigid(p.X, p.Y, None, sigma=sigma, sigma_end=1e-6, w=w, iters=1, backend=orc.LATTICE,
                                update_sigma=True)
    y = p.Y[:, :3].astype(np.float64)
    V = np.concatenate([np.ones((len(y), 1)), y, (y * y).sum(1, keepdims=True)], 1)
    s, _ = orc.Lattice(p.Y, V, sigma).slice(p.X)
    x = p.X[:, :3].astype(np.float32).astype(np.float64)   # the slice's float positions
    c = orc.outlier_constant(w, len(y), len(x), sigma, orc.LATTICE)
    live = s[:, 0] > 0
    m0, m1, m2 = s[live, 0], s[live, 1:4], s[live, 4]
    q = m0 * (x[live] ** 2).sum(1) - 2 * (x[live] * m1).sum(1) + m2
    s2 = (q / (m0 + c)).sum() / (3 * (m0 / (m0 + c)).sum()) / orc.lattice_kernel_variance()
    assert rep.sigma_next == pytest.approx(math.sqrt(s2), rel=1e-9)
    assert rng is not None


def test_recovers_planted_motion_in_fewer_iterations(orc):
    # 800 points in a unit cube observed after a 10 degree / 5 cm motion (the
    # same points: exact correspondences exist), no outliers.  EM with sigma
    # re-estimated from 0.1 reaches the planted motion; EM with sigma fixed
    # at 0.1 needs more iterations to the same stop and keeps a bias from the
    # wide kernel (Table 1's fixed vs updated sigma rows, as a property).
    rng = np.random.default_rng(7)
    X = np.zeros((800, 4), np.float32)
    X[:, :3] = rng.uniform(-0.5, 0.5, (800, 3))
    T_gt = synth.make_T(synth.random_rotation(rng, math.radians(10.0), exact=True), [0.03, -0.04, 0.02])
    Y = np.zeros_like(X)
    Y[:, :3] = X[:, :3].astype(np.float64) @ T_gt[:3, :3].T + T_gt[:3, 3]
    kw = dict(w=0.0, iters=300, backend=orc.EXACT, stop_twist=1e-7)
    Tu, ru = orc.register_rigid(X, Y, None, sigma=0.1, sigma_end=0.002, update_sigma=True, **kw)
    Tf, rf = orc.register_rigid(X, Y, None, sigma=0.1, **kw)
    assert math.radians(synth.rotation_angle_deg(Tu, T_gt)) < 1e-5
    assert np.linalg.norm(Tu[:3, 3] - T_gt[:3, 3]) < 1e-5
    assert ru.iters_run < rf.iters_run / 2, (ru.iters_run, rf.iters_run)
    assert math.radians(synth.rotation_angle_deg(Tf, T_gt)) > 1e-3   # the fixed wide kernel's bias
    assert ru.last_sigma == pytest.approx(0.002)                      # the floor


def test_lattice_kernel_variance_is_its_second_moment(orc):
    # one point splatted with value 1 and sliced on a grid around it: the
    # per-axis second moment of K(p, .) about p, averaged over positions p
    rng = np.random.default_rng(3)
    h = 0.1
    ax = np.arange(-3.0, 3.0, h) + h / 2
    Q = np.zeros((ax.size ** 3, 4), np.float32)
    Q[:, :3] = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    moments = []
    for _ in range(24):
        P = np.zeros((1, 4), np.float32)
        P[0, :3] = rng.uniform(-1.0, 1.0, 3)
        K, _ = orc.Lattice(P, np.ones(1), 1.0).slice(Q)
        d2 = ((Q[:, :3].astype(np.float64) - P[0, :3]) ** 2).sum(1)
        moments.append((K[:, 0] * d2).sum() / K[:, 0].sum() / 3.0)
    assert orc.lattice_kernel_variance() == 0.25
    assert np.mean(moments) == pytest.approx(0.25, abs=0.01)


def test_lattice_update_settles_where_the_exact_one_does(orc):
    # 600 points in a cube, observed after a small motion with 1 cm noise:
    # the exact update settles near the residual scale; the lattice update
    # at twice that (its kernel is half as wide), far above the floor
    rng = np.random.default_rng(11)
    X = np.zeros((600, 4), np.float32)
    X[:, :3] = rng.uniform(-0.5, 0.5, (600, 3))
    T_gt = synth.make_T(synth.random_rotation(rng, math.radians(3.0), exact=True), [0.01, -0.02, 0.01])
    Y = np.zeros_like(X)
    Y[:, :3] = X[:, :3].astype(np.float64) @ T_gt[:3, :3].T + T_gt[:3, 3] + rng.normal(scale=0.01, size=(600, 3))
    kw = dict(w=0.0, iters=60, sigma=0.1, sigma_end=0.001, update_sigma=True)
    Te, re = orc.register_rigid(X, Y, None, backend=orc.EXACT, **kw)
    Tl, rl = orc.register_rigid(X, Y, None, backend=orc.LATTICE, **kw)
    assert rl.last_sigma > 10 * 0.001
    assert rl.last_sigma * 0.5 == pytest.approx(re.last_sigma, rel=0.25), (rl.last_sigma, re.last_sigma)
    for T in (Te, Tl):
        assert synth.rotation_angle_deg(T, T_gt) < 0.3
