"""Pins for the oracle's M step (Section 5) and the whole rigid EM loop.

- SE(3) exponential against scipy's matrix exponential and rotation-vector
  routines, log(exp) = id, and the first-order twist matrix printed in Eq. 16.
- Residual Jacobians against central finite differences of the residual
  under exp(eps zeta) perturbations (pins the sign reading of dx/dzeta).
- The outlier weight against the normalised Gaussian PDF of Eq. 7
  (scipy.stats), which pins the kernel-mass conversion of the constant c.
- Cholesky against numpy's solver.
- Whole EM: with well-separated points the E-step target of each model point
  is its own partner, so the converged pose must be the least-squares pose,
  computed independently by Kabsch (SVD) for point-to-point and by
  scipy.optimize.least_squares for point-to-plane.  And on the depth-frame
  tracking workload the lattice EM recovers the planted motion.
"""
import math

import numpy as np
import pytest
import scipy.linalg
from scipy.optimize import least_squares
from scipy.spatial.transform import Rotation
from scipy.stats import multivariate_normal

from paper_1811_10136_gb300 import synth


def _hat(z):
    w, v = z[:3], z[3:]
    T = np.zeros((4, 4))
    T[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    T[:3, 3] = v
    return T


@pytest.mark.parametrize("scale", [1e-7, 1e-4, 5e-4, 2e-3, 0.1, 1.0, 2.5])
def test_se3_exp_matches_expm(orc, scale):
    rng = np.random.default_rng(int(scale * 1e7) % 1000)
    for _ in range(20):
        z = rng.normal(size=6)
        z[:3] *= scale / np.linalg.norm(z[:3])
        T = orc.se3_exp(z)
        np.testing.assert_allclose(T, scipy.linalg.expm(_hat(z)), rtol=0, atol=2e-14 * (1 + abs(z).max()))
        np.testing.assert_allclose(T[:3, :3], Rotation.from_rotvec(z[:3]).as_matrix(), atol=1e-14)
        assert np.linalg.det(T[:3, :3]) == pytest.approx(1.0, abs=1e-13)


@pytest.mark.parametrize("scale", [1e-9, 1e-5, 0.01, 0.5, 2.0, 3.1])
def test_se3_log_inverts_exp(orc, scale):
    rng = np.random.default_rng(7)
    for _ in range(20):
        z = rng.normal(size=6)
        z[:3] *= scale / np.linalg.norm(z[:3])
        np.testing.assert_allclose(orc.se3_log(orc.se3_exp(z)), z, rtol=1e-6, atol=1e-10)


def test_first_order_is_the_printed_twist_matrix(orc):
    # Eq. 16: T_new ~ [[1, -g, b, a], [g, 1, -al, b'], [-b, al, 1, c], [0 0 0 1]] T
    al, be, ga, a, b, c = 0.3, -0.2, 0.5, 0.7, -0.1, 0.4
    printed = np.array([[1, -ga, be, a], [ga, 1, -al, b], [-be, al, 1, c], [0, 0, 0, 1.0]])
    for eps in (1e-3, 1e-4):
        E = orc.se3_exp(eps * np.array([al, be, ga, a, b, c]))
        lin = np.eye(4) + eps * (printed - np.eye(4))
        assert np.abs(E - lin).max() < 2 * eps * eps


def _fd_jacobian(orc, x, M0, M1, Ns, c_eff, sigma, residual, h=1e-6):
    cols = []
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        xp = (orc.se3_exp(e) @ np.r_[x, 1])[:3]
        xm = (orc.se3_exp(-e) @ np.r_[x, 1])[:3]
        _, rp, _ = orc.point_terms(xp, M0, M1, Ns, c_eff, sigma, residual)
        _, rm, _ = orc.point_terms(xm, M0, M1, Ns, c_eff, sigma, residual)
        cols.append((rp - rm) / (2 * h))
    return np.stack(cols, 1)


@pytest.mark.parametrize("residual", [0, 1])
def test_jacobian_matches_finite_differences(orc, residual):
    rng = np.random.default_rng(8 + residual)
    for _ in range(10):
        x = rng.normal(size=3)
        M0 = rng.uniform(0.2, 3.0)
        M1 = M0 * (x + 0.1 * rng.normal(size=3))
        Ns = M0 * rng.normal(size=3)
        W, r, J = orc.point_terms(x, M0, M1, Ns, 0.3, 0.05, residual)
        Jfd = _fd_jacobian(orc, x, M0, M1, Ns, 0.3, 0.05, residual)
        np.testing.assert_allclose(J, Jfd, rtol=1e-6, atol=1e-6 * np.abs(J).max())
        assert W == pytest.approx(M0 / (M0 + 0.3), rel=1e-14)


def test_outlier_weight_is_normalised_gmm_posterior(orc):
    # Eq. 7 with normalised Gaussians and c = w/(1-w) N/M; for a single
    # observation point the inlier weight is pdf / (pdf + c).
    x = np.array([0.01, -0.02, 0.015])
    y = np.array([0.0, 0.0, 0.0], np.float32)
    sigma, w, N, M = 0.02, 0.1, 2200, 2000
    X = np.array([[*x, 0]], np.float32)
    M0, M1, _ = orc.estep_exact(X, np.array([[*y, 0]], np.float32), None, sigma)
    c_eff = orc.outlier_constant(w, N, M, sigma, orc.EXACT)
    W, _, _ = orc.point_terms(X[0, :3].astype(np.float64), M0[0], M1[0], None, c_eff, sigma, 0)
    pdf = multivariate_normal.pdf(X[0, :3].astype(np.float64), mean=y, cov=sigma * sigma * np.eye(3))
    c = w / (1 - w) * N / M
    assert W == pytest.approx(pdf / (pdf + c), rel=1e-12)


def test_cholesky_solve(orc):
    rng = np.random.default_rng(9)
    for n in (1, 6, 26):
        B = rng.normal(size=(n, n))
        A = B @ B.T + n * np.eye(n)
        b = rng.normal(size=n)
        np.testing.assert_allclose(orc.cholesky_solve(A, b), np.linalg.solve(A, b), rtol=1e-10)
    assert orc.cholesky_solve(np.diag([1.0, -1.0]), np.ones(2)) is None
    assert orc.cholesky_solve(np.zeros((6, 6)), np.ones(6)) is None


def _separated_points(rng, n, min_dist, half=1.0):
    pts = []
    while len(pts) < n:
        p = rng.uniform(-half, half, size=3)
        if all(np.linalg.norm(p - q) >= min_dist for q in pts):
            pts.append(p)
    return np.array(pts)


def _kabsch(P, Q):
    cp, cq = P.mean(0), Q.mean(0)
    H = (P - cp).T @ (Q - cq)
    U, _, Vt = np.linalg.svd(H)
    D = np.diag([1, 1, np.sign(np.linalg.det(Vt.T @ U.T))])
    R = Vt.T @ D @ U.T
    return synth.make_T(R, cq - R @ cp)


def test_em_pt2pt_converges_to_kabsch(orc):
    # Points 0.3 apart, sigma 0.02: each model point's E-step target is its own
    # (noisy) partner, so the EM fixed point is the least-squares rigid pose.
    rng = np.random.default_rng(10)
    P = _separated_points(rng, 120, 0.3)
    T_true = synth.make_T(synth.random_rotation(rng, math.radians(2.0), exact=True), [0.02, -0.01, 0.015])
    Q = P @ T_true[:3, :3].T + T_true[:3, 3] + rng.normal(scale=0.002, size=P.shape)
    X = np.c_[P, np.zeros(len(P))].astype(np.float32)
    Y = np.c_[Q, np.zeros(len(Q))].astype(np.float32)
    T, rep = orc.register_rigid(X, Y, sigma=0.02, w=0.0, iters=40, backend=orc.EXACT)
    T_ls = _kabsch(X[:, :3].astype(np.float64), Y[:, :3].astype(np.float64))
    np.testing.assert_allclose(T, T_ls, atol=1e-9)
    assert rep.degenerate_iters == 0 and rep.last_inliers == 120


def test_em_pt2pl_converges_to_least_squares(orc):
    rng = np.random.default_rng(11)
    P = _separated_points(rng, 150, 0.3)
    T_true = synth.make_T(synth.random_rotation(rng, math.radians(2.0), exact=True), [0.01, 0.02, -0.01])
    Q = P @ T_true[:3, :3].T + T_true[:3, 3] + rng.normal(scale=0.002, size=P.shape)
    Nq = rng.normal(size=P.shape)
    Nq /= np.linalg.norm(Nq, axis=1, keepdims=True)
    X = np.c_[P, np.zeros(len(P))].astype(np.float32)
    Y = np.c_[Q, np.zeros(len(Q))].astype(np.float32)
    Yn = np.c_[Nq, np.zeros(len(Q))].astype(np.float32)
    T, _ = orc.register_rigid(X, Y, Yn, sigma=0.02, w=0.0, iters=40, residual=orc.PT2PL,
                              backend=orc.EXACT)
    Xd, Yd, Nd = (a[:, :3].astype(np.float64) for a in (X, Y, Yn))

    def res(p):
        R = Rotation.from_rotvec(p[:3]).as_matrix()
        return ((Xd @ R.T + p[3:] - Yd) * Nd).sum(1)

    sol = least_squares(res, np.zeros(6), xtol=1e-15, ftol=1e-15, gtol=1e-15)
    T_ls = synth.make_T(Rotation.from_rotvec(sol.x[:3]).as_matrix(), sol.x[3:])
    np.testing.assert_allclose(T, T_ls, atol=1e-8)


def test_lattice_em_recovers_planted_motion(orc):
    # Depth-frame tracking (320x240, 2 deg / 2 cm motion, sigma 0.04 -> 0.01):
    # the oracle's lattice EM recovers the planted motion well inside
    # 0.1 deg / 1 mm.
    p = synth.depth_frame_pair(3)
    T, rep = orc.register_rigid(p.X, p.Y, p.Yn, sigma=0.04, sigma_end=0.01, w=0.1, iters=20,
                                residual=orc.PT2PL, backend=orc.LATTICE)
    assert synth.rotation_angle_deg(T, p.T_gt) < 0.1
    assert np.linalg.norm(T[:3, 3] - p.T_gt[:3, 3]) < 1e-3
    assert rep.degenerate_iters == 0


def test_degenerate_when_nothing_overlaps(orc):
    p = synth.sphere_bumps_pair(0, n_model=200, n_obs=200)
    Y = p.Y.copy()
    Y[:, :3] += 50.0
    T, rep = orc.register_rigid(p.X, Y, sigma=0.02, iters=3)
    np.testing.assert_array_equal(T, np.eye(4))
    assert rep.degenerate_iters == 3 and rep.last_inliers == 0


def test_align_error_closed_forms():
    # Eq. 22's mean distance between the estimated and the true placement of
    # the model: a pure translation t moves every point by |t|; a rotation by
    # theta about z moves a point at radius rho by 2 rho sin(theta / 2); equal
    # poses give 0 and the empty model 0.
    import math
    import numpy as np
    import oracle as orc
    rng = np.random.default_rng(3)
    X = np.zeros((500, 4), np.float32)
    X[:, :3] = rng.normal(size=(500, 3))
    Tt = np.eye(4)
    Tt[:3, 3] = [0.3, -0.4, 1.2]
    assert abs(orc.align_error(X, np.eye(4), Tt) - 1.3) < 1e-12
    th = 0.7
    Rz = np.eye(4)
    Rz[:2, :2] = [[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]]
    rho = np.hypot(X[:, 0].astype(np.float64), X[:, 1].astype(np.float64))
    assert abs(orc.align_error(X, Rz, np.eye(4)) - np.mean(2 * rho * math.sin(th / 2))) < 1e-12
    assert orc.align_error(X, Rz, Rz) == 0.0
    assert orc.align_error(X[:0], Rz, np.eye(4)) == 0.0
