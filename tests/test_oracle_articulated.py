"""Pins for the oracle's articulated model (Section 5.1, Eq. 20, Algorithm 1).

- Forward kinematics against the generator's independent numpy kinematics.
- The spatial velocity Jacobian against central finite differences of the
  body poses (twists from se3_log).
- Algorithm 1's factored normal matrix against the direct assembly
  sum_i J_i^T J_i with every point's full Jacobian d r_i / d theta taken by
  finite differences of the kinematics (pins the factoring identity of Eq. 20
  and the parameterisation: root by exponential, joints additive).
- With exact correspondences (observation = the model's own points at the
  planted pose, sigma well below the point spacing) the EM converges to the
  planted pose.
"""
import numpy as np
import pytest

from paper_1811_10136_gb300 import synth


@pytest.fixture(scope="module")
def tree():
    return synth.random_kintree(3)


def test_fk_matches_independent_kinematics(orc, tree):
    rng = np.random.default_rng(0)
    for _ in range(5):
        q = rng.uniform(-1.5, 1.5, tree.nj)
        R = synth.make_T(synth.random_rotation(rng, 1.0), rng.normal(size=3))
        T, aw, pw = orc.fk(tree, R, q)
        np.testing.assert_allclose(T, synth.pose_bodies(tree, R, q), atol=1e-13)
        np.testing.assert_allclose(np.linalg.norm(aw, axis=1), 1.0, atol=1e-12)


def test_spatial_jacobian_matches_finite_differences(orc, tree):
    rng = np.random.default_rng(1)
    q = rng.uniform(-0.5, 0.5, tree.nj)
    R0 = synth.make_T(synth.random_rotation(rng, 0.3), [0.1, -0.2, 0.05])
    T, aw, pw = orc.fk(tree, R0, q)
    h = 1e-6
    for b in range(tree.nb):
        J = orc.spatial_jacobian(tree, aw, pw, b)
        for k in range(6 + tree.nj):
            if k < 6:
                e = np.zeros(6)
                e[k] = h
                Tp = orc.fk(tree, orc.se3_exp(e) @ R0, q)[0]
                Tm = orc.fk(tree, orc.se3_exp(-e) @ R0, q)[0]
            else:
                qp, qm = q.copy(), q.copy()
                qp[k - 6] += h
                qm[k - 6] -= h
                Tp, Tm = orc.fk(tree, R0, qp)[0], orc.fk(tree, R0, qm)[0]
            inv = np.linalg.inv(T[b])
            tw = (orc.se3_log(Tp[b] @ inv) - orc.se3_log(Tm[b] @ inv)) / (2 * h)
            np.testing.assert_allclose(tw, J[:, k], atol=2e-8)


@pytest.mark.parametrize("residual", [0, 1])
def test_algorithm1_equals_direct_assembly(orc, tree, residual):
    p = synth.articulated_pair(5, n_points=1500, tree=tree)
    rng = np.random.default_rng(2)
    q0 = rng.uniform(-0.2, 0.2, tree.nj)
    R0 = synth.make_T(synth.random_rotation(rng, 0.05), [0.003, 0.0, -0.002])
    sigma, w = 0.02, 0.1
    Yn = p.Yn if residual else None
    A, g = orc.articulated_normal_equations(p.Xref, p.body, tree, p.Y, Yn, sigma=sigma, w=w,
                                            residual=residual, root_T=R0, q=q0)
    # E-step values at theta0 (held fixed in the M step)
    Tb = synth.pose_bodies(tree, R0, q0)
    Xw = np.einsum("nij,nj->ni", Tb[p.body][:, :3, :3], p.Xref[:, :3].astype(np.float64)) + Tb[p.body][:, :3, 3]
    Xf = np.zeros((len(Xw), 4), np.float32)
    Xf[:, :3] = Xw
    es = orc.estep(Xf, p.Y, Yn, sigma, backend=orc.LATTICE)
    c_eff = orc.outlier_constant(w, p.Y.shape[0], p.Xref.shape[0], sigma, orc.LATTICE)

    def residuals(R, q):
        Tb = synth.pose_bodies(tree, R, q)
        X = np.einsum("nij,nj->ni", Tb[p.body][:, :3, :3], p.Xref[:, :3].astype(np.float64)) + Tb[p.body][:, :3, 3]
        out = []
        for i in range(len(X)):
            Ns = es[i, 4:7] if residual else None
            _, r, _ = orc.point_terms(X[i], es[i, 0], es[i, 1:4], Ns, c_eff, sigma, residual)
            out.append(r if len(r) else np.zeros(3 if residual == 0 else 1))
        return np.concatenate(out)

    nd = 6 + tree.nj
    h = 1e-7
    cols = []
    for k in range(nd):
        if k < 6:
            e = np.zeros(6)
            e[k] = h
            rp = residuals(orc.se3_exp(e) @ R0, q0)
            rm = residuals(orc.se3_exp(-e) @ R0, q0)
        else:
            qp, qm = q0.copy(), q0.copy()
            qp[k - 6] += h
            qm[k - 6] -= h
            rp, rm = residuals(R0, qp), residuals(R0, qm)
        cols.append((rp - rm) / (2 * h))
    Jfd = np.stack(cols, 1)
    r0 = residuals(R0, q0)
    np.testing.assert_allclose(A, Jfd.T @ Jfd, rtol=1e-5, atol=1e-6 * np.abs(A).max())
    np.testing.assert_allclose(g, Jfd.T @ r0, rtol=1e-5, atol=1e-6 * np.abs(g).max())


def test_exact_correspondences_recover_planted_pose(orc, tree):
    # The observation is the model's own points at the planted pose; points
    # are kept >= 8 mm apart and sigma = 1 mm, so each point's E-step target is
    # its own partner and the EM's fixed point is the planted pose.
    rng = np.random.default_rng(4)
    P, _, B = synth.sample_capsules(tree, 4000, rng)
    keep = []
    Tz = synth.pose_bodies(tree, np.eye(4), np.zeros(tree.nj))
    W = np.einsum("nij,nj->ni", Tz[B][:, :3, :3], P[:, :3]) + Tz[B][:, :3, 3]
    for i in range(len(W)):
        if all(np.linalg.norm(W[i] - W[j]) >= 0.008 for j in keep):
            keep.append(i)
    P, B = P[keep], B[keep]
    q_gt = rng.uniform(-1, 1, tree.nj) * np.radians(0.15)
    R_gt = synth.make_T(synth.random_rotation(rng, np.radians(0.1)), [0.0004, -0.0003, 0.0002])
    Tb = synth.pose_bodies(tree, R_gt, q_gt)
    Y = np.zeros_like(P)
    Y[:, :3] = np.einsum("nij,nj->ni", Tb[B][:, :3, :3], P[:, :3].astype(np.float64)) + Tb[B][:, :3, 3]
    R, q, rep = orc.register_articulated(P, B, tree, Y, sigma=0.001, w=0.0, iters=25, backend=orc.EXACT)
    assert np.abs(q - q_gt).max() < 1e-6
    np.testing.assert_allclose(R, R_gt, atol=1e-8)
