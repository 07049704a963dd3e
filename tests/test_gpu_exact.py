"""The exact Gauss transform on the GPU (Section 4.1: the sums the lattice
approximates) against the oracle's float64 exact back-end.

Bar: |GPU - oracle| <= 1e-4 (|oracle| + M0 max|v|) + 1e-7 max|oracle| per
output, v the summed value (1, a coordinate of y, a normal component):
float32 rounding of a sum scales with the sum of its terms' magnitudes,
sum_j K_ij |v_j| <= M0 max|v| -- not with the result, which cancels for the
coordinate and normal sums.  Each kernel value exp(-q / 2 sigma^2) is
evaluated in float32 (relative error a few ulp of its argument's size), and
each thread sums 256-term tiles before adding them to its totals, so the
rounding grows like (256 + N / 256) u ~ 2e-5 of the magnitude sum here."""
import math

import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_10136_gb300 as fr
    return fr.Context(0)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def close(out, ref, Y):
    err = np.abs(out - ref)
    vmax = np.ones(ref.shape[1])
    vmax[1:4] = np.abs(Y[:, :3]).max(0)
    bound = 1e-4 * (np.abs(ref) + ref[:, :1] * vmax[None, :]) + 1e-7 * np.abs(ref).max(0, keepdims=True)
    return float((err / bound).max())


@pytest.mark.parametrize("pt2pl", [False, True])
@pytest.mark.parametrize("sigma", [0.01, 0.05])
def test_matches_oracle_exact(ctx, orc, pt2pl, sigma):
    # 3,001 model x 5,003 observation points: several tiles, a ragged tail,
    # the observation range split across blocks; a small rigid motion.
    rng = np.random.default_rng(31)
    src = synth.sphere_bumps_pair(31, n_model=3001, n_obs=5003, outlier_frac=0.0)
    X, Y = src.X, src.Y
    nv = rng.normal(size=(Y.shape[0], 3))
    Yn = np.zeros_like(Y)
    Yn[:, :3] = nv / np.linalg.norm(nv, axis=1, keepdims=True)
    T = synth.make_T(synth.random_rotation(rng, math.radians(3.0)), rng.uniform(-0.02, 0.02, 3))
    sigma = float(np.float32(sigma))
    out = ctx.gauss_transform(dev(X), dev(Y), dev(Yn) if pt2pl else None, sigma=sigma, T=T).cpu().numpy()
    ref = orc.estep(X, Y, Yn if pt2pl else None, sigma, T=T, backend=orc.EXACT)
    assert out.shape == ref.shape
    assert close(out.astype(np.float64), ref, Y) <= 1.0


def test_single_pair_closed_form(ctx):
    X = np.array([[0.1, -0.2, 0.3, 0.0]], np.float32)
    Y = np.array([[0.11, -0.185, 0.32, 0.0]], np.float32)
    sigma = 0.02
    out = ctx.gauss_transform(dev(X), dev(Y), None, sigma=sigma).cpu().numpy()[0]
    d2 = float(np.sum((X[0, :3].astype(np.float64) - Y[0, :3]) ** 2))
    k = math.exp(-d2 / (2 * sigma * sigma))
    assert out[0] == pytest.approx(k, rel=1e-5)
    np.testing.assert_allclose(out[1:4], k * Y[0, :3].astype(np.float64), rtol=1e-5)


def test_full_frame_sampled(ctx, orc):
    # The depth-frame workload (76,800 model x ~73,000 observation points):
    # every output computed on the GPU, 300 sampled rows by the oracle.
    p = synth.depth_frame_pair(0)
    T = p.T_gt
    sigma = float(np.float32(0.01))
    out = ctx.gauss_transform(dev(p.X), dev(p.Y), dev(p.Yn), sigma=sigma, T=T).cpu().numpy()
    rows = np.random.default_rng(5).choice(p.X.shape[0], 300, replace=False)
    ref = orc.estep(p.X[rows], p.Y, p.Yn, sigma, T=T, backend=orc.EXACT)
    assert close(out[rows].astype(np.float64), ref, p.Y) <= 1.0
    assert np.isfinite(out).all()


def test_rejects_bad_arguments(ctx):
    import paper_1811_10136_gb300 as fr
    X = dev(np.zeros((10, 4)))
    with pytest.raises(fr.FilterRegError) as e:
        ctx.gauss_transform(X, X, None, sigma=0.0)
    assert e.value.status == fr.FR_EINVAL
