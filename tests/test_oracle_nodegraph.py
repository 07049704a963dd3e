"""Pins for the oracle's node-graph model (Section 5.2, Eq. 21).

- Dual quaternions: round trip to the matrix; the blend of equal poses is
  that pose; sign invariance; two screws about one axis blend to the half
  screw (dual-quaternion blending interpolates along the screw).
- A single node carrying every point with no regulariser is the rigid model:
  the node-graph EM equals the rigid EM.
- The assembled A and g equal J^T J and J^T r with J from finite differences
  of the actual dual-quaternion warp and of the regulariser residuals, at
  node poses that agree (where the first-order DQB derivative is exact).
- Block-Jacobi PCG: finite termination on a small SPD system; one iteration
  on a block-diagonal one.
- With exact correspondences and a planted motion shared by every node, the
  EM recovers it.
"""
import math

import numpy as np
import pytest

from paper_1811_10136_gb300 import synth


def se3(rng, ang, trans):
    return synth.make_T(synth.random_rotation(rng, ang), rng.uniform(-trans, trans, 3))


def test_dual_quaternion_round_trip(orc):
    rng = np.random.default_rng(0)
    for _ in range(20):
        T = se3(rng, math.pi, 1.0)
        dq = orc.dq_from_T(T)
        assert abs(np.linalg.norm(dq[:4]) - 1.0) < 1e-12
        assert abs(dq[:4] @ dq[4:]) < 1e-12                  # a rigid transform: q_r . q_d = 0
        np.testing.assert_allclose(orc.T_from_dq(dq), T, atol=1e-12)
        np.testing.assert_allclose(orc.T_from_dq(-dq), T, atol=1e-12)


def test_blend_of_equal_poses_and_signs(orc):
    rng = np.random.default_rng(1)
    T = se3(rng, 2.0, 0.5)
    dq = orc.dq_from_T(T)
    node_dq = np.stack([dq, -dq, dq, -dq])                  # the same pose, both signs
    np.testing.assert_allclose(orc.dqb(node_dq, [0, 1, 2, 3], [0.4, 0.3, 0.2, 0.1]), T, atol=1e-12)
    other = np.stack([dq, orc.dq_from_T(se3(rng, 1.0, 0.3))])
    np.testing.assert_allclose(orc.dqb(other, [0, 1, 1, 1], [1.0, 0.0, 0.0, 0.0]), T, atol=1e-12)


def test_blend_interpolates_a_screw(orc):
    # Rotation theta about z plus translation h along z, against the
    # identity: weights (1/2, 1/2) give theta/2 and h/2.
    theta, h = 1.1, 0.3
    c, s = math.cos(theta), math.sin(theta)
    T1 = np.array([[c, -s, 0, 0], [s, c, 0, 0], [0, 0, 1, h], [0, 0, 0, 1.0]])
    node_dq = np.stack([orc.dq_from_T(np.eye(4)), orc.dq_from_T(T1)])
    B = orc.dqb(node_dq, [0, 1, 0, 1], [0.25, 0.25, 0.25, 0.25])
    c2, s2 = math.cos(theta / 2), math.sin(theta / 2)
    np.testing.assert_allclose(B, [[c2, -s2, 0, 0], [s2, c2, 0, 0], [0, 0, 1, h / 2], [0, 0, 0, 1]],
                               atol=1e-12)


def test_warp_with_common_pose_is_rigid(orc):
    p = synth.nodegraph_pair(1, W=48, H=36, n_nodes=20)
    T = se3(np.random.default_rng(2), 0.3, 0.1)
    X = orc.nodegraph_warp(p.Xref, p.knn, p.skw, np.tile(T, (20, 1, 1)))
    np.testing.assert_allclose(X, synth.apply_T(T, p.Xref[:, :3].astype(np.float64)), atol=1e-12)


@pytest.mark.parametrize("residual", [0, 1])
def test_single_node_is_the_rigid_model(orc, residual):
    q = synth.depth_frame_pair(3, W=64, H=48)
    M = q.X.shape[0]
    knn = np.zeros((M, 4), np.int32)
    skw = np.zeros((M, 4), np.float32)
    skw[:, 0] = 1.0
    Yn = q.Yn if residual else None
    Tn, rn = orc.register_nodegraph(q.X, knn, skw, np.zeros((1, 3)), np.zeros((0, 2), np.int32), q.Y, Yn,
                                    sigma=0.03, sigma_end=0.015, w=0.1, lam=0.0, pcg_iters=3, iters=8,
                                    residual=residual)
    Tr, rr = orc.register_rigid(q.X, q.Y, Yn, sigma=0.03, sigma_end=0.015, w=0.1, iters=8, residual=residual)
    np.testing.assert_allclose(Tn[0], Tr, atol=1e-10)
    assert rn.last_inliers == rr.last_inliers
    assert rn.last_cost == pytest.approx(rr.last_cost, rel=1e-9)


@pytest.mark.parametrize("residual", [0, 1])
def test_assembly_equals_finite_difference_gauss_newton(orc, residual):
    p = synth.nodegraph_pair(2, W=32, H=24, n_nodes=8)
    K = p.node_pos.shape[0]
    rng = np.random.default_rng(3)
    T0 = se3(rng, 0.05, 0.01)
    node_T = np.tile(T0, (K, 1, 1))
    sigma, w, lam = 0.03, 0.1, 10.0
    Yn = p.Yn if residual else None
    A, g, rep = orc.nodegraph_normal_equations(p.Xref, p.knn, p.skw, p.node_pos, p.edges, p.Y, Yn,
                                               sigma=sigma, w=w, lam=lam, residual=residual, node_T=node_T)
    # E-step sums at the current warped points, held fixed (the M step's E values)
    X0 = orc.nodegraph_warp(p.Xref, p.knn, p.skw, node_T)
    es = orc.estep(X0.astype(np.float32), p.Y, Yn, sigma, backend=orc.LATTICE)
    c_eff = orc.outlier_constant(w, p.Y.shape[0], p.Xref.shape[0], sigma, orc.LATTICE)
    s = math.sqrt(lam) / sigma

    def residuals(nT):
        X = orc.nodegraph_warp(p.Xref, p.knn, p.skw, nT)
        out = []
        for i in range(X.shape[0]):
            _, r, _ = orc.point_terms(X[i], es[i, 0], es[i, 1:4], es[i, 4:7] if residual else None,
                                      c_eff, sigma, residual)
            out.append(r if len(r) else np.zeros(3 if residual == 0 else 1))
        for j, k in p.edges:
            pk = np.r_[p.node_pos[k], 1.0]
            out.append(s * ((nT[j] @ pk)[:3] - (nT[k] @ pk)[:3]))
        return np.concatenate(out)

    h = 1e-7
    cols = []
    for k in range(K):
        for c in range(6):
            z = np.zeros(6)
            z[c] = h
            Tp, Tm = node_T.copy(), node_T.copy()
            Tp[k] = orc.se3_exp(z) @ node_T[k]
            Tm[k] = orc.se3_exp(-z) @ node_T[k]
            cols.append((residuals(Tp) - residuals(Tm)) / (2 * h))
    J = np.stack(cols, 1)
    r0 = residuals(node_T)
    np.testing.assert_allclose(A, J.T @ J, rtol=1e-5, atol=1e-6 * np.abs(A).max())
    np.testing.assert_allclose(g, J.T @ r0, rtol=1e-5, atol=1e-6 * np.abs(g).max())
    assert rep.last_cost == pytest.approx(float(r0 @ r0), rel=1e-9)


def test_pcg_finite_termination_and_block_jacobi(orc):
    rng = np.random.default_rng(4)
    B = rng.normal(size=(12, 12))
    A = B @ B.T + 0.5 * np.eye(12)
    b = rng.normal(size=12)
    np.testing.assert_allclose(orc.pcg_block_jacobi(A, b, 12), np.linalg.solve(A, b), rtol=1e-7, atol=1e-9)
    D = np.zeros((18, 18))
    for k in range(3):
        C = rng.normal(size=(6, 6))
        D[6 * k:6 * k + 6, 6 * k:6 * k + 6] = C @ C.T + np.eye(6)
    b = rng.normal(size=18)
    np.testing.assert_allclose(orc.pcg_block_jacobi(D, b, 1), np.linalg.solve(D, b), rtol=1e-10, atol=1e-12)


def test_exact_correspondences_recover_common_motion(orc):
    # Sparse model (points >= 12 mm apart) observed after a planted rigid
    # motion shared by every node, sigma 2 mm, exact E step: each point's
    # target is its own partner; the regulariser vanishes at the plant.
    p = synth.nodegraph_pair(5, W=48, H=36, n_nodes=12)
    X = p.Xref[::3]
    keep = []
    for i in range(X.shape[0]):
        if all(np.linalg.norm(X[i, :3] - X[j, :3]) >= 0.012 for j in keep):
            keep.append(i)
    X = np.ascontiguousarray(X[keep])
    knn, skw, _ = synth.skinning(X[:, :3].astype(np.float64), p.node_pos)
    rng = np.random.default_rng(6)
    Tg = se3(rng, math.radians(0.2), 0.0008)
    Y = X.copy()
    Y[:, :3] = synth.apply_T(Tg, X[:, :3].astype(np.float64))
    nT, rep = orc.register_nodegraph(X, knn, skw, p.node_pos, p.edges, Y, None, sigma=0.002, w=0.0, lam=10.0,
                                     pcg_iters=40, iters=15, backend=orc.EXACT)
    Xw = orc.nodegraph_warp(X, knn, skw, nT)
    assert np.abs(Xw - Y[:, :3]).max() < 1e-6
    for k in range(nT.shape[0]):
        np.testing.assert_allclose(nT[k], Tg, atol=1e-5)
