"""Serving (continuous batching): each request's result equals the same
registration run alone (fr_register_rigid) within the batched path's
tolerance, whatever else is in flight -- ragged sizes, mixed sigma
schedules, device and host clouds, requests queued behind a small memory
budget, and a request whose compact table overflows and is rerun."""
import math
import time

import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

pytestmark = pytest.mark.gpu

# alone vs in the mix: float32 sums in another order; 10x inside the
# method's 1e-3 rad / 1e-4 bar
SAME_ROT, SAME_TRANS = 1e-4, 1e-5


@pytest.fixture(scope="module")
def ctx():
    import paper_1811_10136_gb300 as fr
    return fr.Context(0)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def pose_diff(A, B):
    return math.radians(synth.rotation_angle_deg(A, B)), float(np.linalg.norm(A[:3, 3] - B[:3, 3]))


VIEWS = [(96, 72, 105), (320, 240, 101), (64, 48, 109), (160, 120, 103), (200, 150, 105)]
SIGMAS = [(0.04, 0.01), (0.02, 0.02), (0.03, 0.015), (0.05, 0.05), (0.04, 0.01)]


@pytest.fixture(scope="module")
def pairs():
    return [synth.depth_frame_pair(seed, W=w, H=h) for w, h, seed in VIEWS]


def alone(ctx, p, s0, s1, w, iters, pt2pl=True):
    return ctx.register_rigid(dev(p.X), dev(p.Y), dev(p.Yn) if pt2pl else None, residual=int(pt2pl),
                              iters=iters, sigma_start=s0, sigma_end=s1, w=w)


@pytest.mark.parametrize("host", [False, True])
def test_requests_equal_single_registrations(ctx, pairs, host):
    import paper_1811_10136_gb300 as fr
    iters = 12
    with fr.Server(ctx, budget_bytes=1 << 30, max_live=64, residual=fr.FR_PT2PL, iters=iters) as srv:
        reqs = []
        # three rounds of the five views, submitted back to back: requests
        # join while others are mid-registration
        for r in range(3):
            for i, p in enumerate(pairs):
                s0, s1 = SIGMAS[(i + r) % len(SIGMAS)]
                args = (p.X, p.Y, p.Yn) if host else (dev(p.X), dev(p.Y), dev(p.Yn))
                reqs.append((i, s0, s1, srv.submit(*args, sigma_start=s0, sigma_end=s1, w=0.1, host=host)))
        results = [(i, s0, s1, srv.wait(t, 60_000)) for i, s0, s1, t in reqs]
        st = srv.stats()
    assert st["completed"] == len(reqs)
    for i, s0, s1, res in results:
        assert res.status == 0
        Ts, rs = alone(ctx, pairs[i], s0, s1, 0.1, iters)
        dr, dt = pose_diff(res.T, Ts)
        assert dr < SAME_ROT and dt < SAME_TRANS, (i, s0, s1, dr, dt)
        assert res.report.iters_run == rs.iters_run == iters
        assert res.report.lattice_builds == rs.lattice_builds
        assert res.report.lattice_vertices == rs.lattice_vertices
        assert res.submit_ns <= res.admit_ns <= res.complete_ns


def test_small_budget_queues_requests(ctx, pairs):
    # 128 MiB: the 320x240 request's three tables alone take 3/4 of the table
    # arena (2^20 slots), so requests wait for memory and are admitted as
    # others finish.
    import paper_1811_10136_gb300 as fr
    iters = 8
    with fr.Server(ctx, budget_bytes=128 << 20, max_live=8, residual=fr.FR_PT2PL, iters=iters) as srv:
        ts = [srv.submit(dev(p.X), dev(p.Y), dev(p.Yn), sigma_start=0.04, sigma_end=0.01) for p in pairs * 2]
        res = [srv.wait(t, 60_000) for t in ts]
    for k, r in enumerate(res):
        p = pairs[k % len(pairs)]
        Ts, _ = alone(ctx, p, 0.04, 0.01, 0.1, iters)
        dr, dt = pose_diff(r.T, Ts)
        assert r.status == 0 and dr < SAME_ROT and dt < SAME_TRANS, (k, dr, dt)
    # first come, first served: admissions in submission order
    admits = [r.admit_ns for r in res]
    assert admits == sorted(admits)


def test_point_to_point_and_fixed_sigma(ctx, pairs):
    import paper_1811_10136_gb300 as fr
    with fr.Server(ctx, budget_bytes=1 << 29, max_live=16, residual=fr.FR_PT2PT, iters=10) as srv:
        ts = [srv.submit(dev(p.X), dev(p.Y), None, sigma_start=0.03) for p in pairs]
        res = [srv.wait(t, 60_000) for t in ts]
    for p, r in zip(pairs, res):
        Ts, rs = alone(ctx, p, 0.03, 0.03, 0.1, 10, pt2pl=False)
        dr, dt = pose_diff(r.T, Ts)
        assert r.status == 0 and dr < SAME_ROT and dt < SAME_TRANS
        assert r.report.lattice_builds == 1


def test_overflowing_request_is_rerun(ctx):
    # 5,000 scattered points at sigma 1 cm: 20,000 vertices overflow the
    # compact table (16,384 slots); the server reruns the request at the safe size.
    import paper_1811_10136_gb300 as fr
    rng = np.random.default_rng(77)
    X = np.zeros((5000, 4), np.float32)
    X[:, :3] = rng.uniform(-1, 1, size=(5000, 3))
    T = synth.make_T(synth.random_rotation(rng, 0.002), [0.001, 0.0, -0.001])
    Y = np.zeros_like(X)
    Y[:, :3] = synth.apply_T(T, X)
    Ts, rs = ctx.register_rigid(dev(X), dev(Y), None, iters=3, sigma_start=0.01, sigma_end=0.01)
    with fr.Server(ctx, budget_bytes=1 << 28, max_live=4, iters=3) as srv:
        r = srv.wait(srv.submit(dev(X), dev(Y), None, sigma_start=0.01), 60_000)
    assert r.status == 0
    assert r.report.lattice_vertices > 16384
    dr, dt = pose_diff(r.T, Ts)
    assert dr < SAME_ROT and dt < SAME_TRANS


def test_rejects_bad_requests(ctx, pairs):
    import paper_1811_10136_gb300 as fr
    p = pairs[0]
    with fr.Server(ctx, budget_bytes=1 << 24, max_live=2, residual=fr.FR_PT2PL, iters=2) as srv:
        with pytest.raises(fr.FilterRegError) as e:
            srv.submit(dev(p.X), dev(p.Y), dev(p.Yn), sigma_start=-1.0)
        assert e.value.status == fr.FR_EINVAL
        with pytest.raises(fr.FilterRegError) as e:   # normals missing for point-to-plane
            srv.submit(dev(p.X), dev(p.Y), None)
        assert e.value.status == fr.FR_EINVAL
        big = synth.depth_frame_pair(0)               # 3 tables of 262,144 slots exceed the arena
        with pytest.raises(fr.FilterRegError) as e:
            srv.submit(dev(big.X), dev(big.Y), dev(big.Yn), sigma_start=0.04, sigma_end=0.01)
        assert e.value.status == fr.FR_ENOMEM
    with pytest.raises(fr.FilterRegError) as e:
        fr.Server(ctx, budget_bytes=1 << 24, blur=1)
    assert e.value.status == fr.FR_ENOTSUPPORTED


def test_poll_and_stream(ctx, pairs):
    # A short stream: requests submitted at ~1 ms intervals, polled.
    import paper_1811_10136_gb300 as fr
    dp = [(dev(p.X), dev(p.Y), dev(p.Yn)) for p in pairs]
    with fr.Server(ctx, budget_bytes=1 << 30, max_live=32, residual=fr.FR_PT2PL, iters=20) as srv:
        ts = []
        for k in range(40):
            X, Y, Yn = dp[k % len(dp)]
            ts.append(srv.submit(X, Y, Yn, sigma_start=0.04, sigma_end=0.01))
            time.sleep(0.001)
        out = {}
        t_end = time.time() + 60
        while len(out) < len(ts) and time.time() < t_end:
            for t in ts:
                if t not in out:
                    r = srv.poll(t)
                    if r is not None:
                        out[t] = r
        st = srv.stats()
    assert len(out) == len(ts) and all(r.status == 0 for r in out.values())
    assert st["ticks"] >= 22 and st["kernel_launches"] == st["ticks"]


def test_stream_configuration_requests_equal_alone(ctx):
    # The serving stream's configuration: clouds log-uniform in 1k..300k
    # points (depth frames at 4:3), sigma fixed per request in {0.01, 0.02,
    # 0.04}, 20 iterations, point-to-plane, 40 requests submitted at once
    # (all live together), plus a sparse cloud whose compact table overflows
    # and is rerun at the safe size.
    #
    # Alone and in the mix the float32 sums run in other orders (other block
    # partitions, points per thread); a near-planar view leaves the
    # point-to-plane normal matrix poorly conditioned and amplifies that.  The
    # bar is therefore per request: 10x the difference between two float32
    # runs alone (plain and Kahan-compensated sums), at least 1e-4 rad /
    # 1e-5, and never more than the method's 1e-3 rad / 1e-4.
    import paper_1811_10136_gb300 as fr
    rng = np.random.default_rng(2025)
    pool = []
    for i in range(10):
        n = float(np.exp(rng.uniform(np.log(1000.0), np.log(300000.0))))
        W = max(8, int(round(np.sqrt(n / 0.95 * 4.0 / 3.0))))
        H = max(6, int(round(W * 3 / 4)))
        pool.append(synth.depth_frame_pair(7000 + i, W=W, H=H, fx=300.0 * W / 320, fy=300.0 * W / 320))
    assert max(p.Y.shape[0] for p in pool) > 100000 and min(p.Y.shape[0] for p in pool) < 10000
    sparse = np.zeros((20000, 4), np.float32)
    sparse[:, :3] = rng.uniform(-1, 1, size=(20000, 3))
    sp_Y = sparse.copy()
    sp_Y[:, 0] += 0.002
    sp_n = np.zeros_like(sparse)
    nv = rng.normal(size=(20000, 3))
    sp_n[:, :3] = nv / np.linalg.norm(nv, axis=1, keepdims=True)
    dpool = [(dev(p.X), dev(p.Y), dev(p.Yn)) for p in pool] + [(dev(sparse), dev(sp_Y), dev(sp_n))]
    sig = np.array([0.01, 0.02, 0.04], np.float32)
    reqs = [(k % len(pool), float(sig[rng.integers(0, 3)])) for k in range(39)] + [(len(pool), 0.01)]
    iters = 20
    with fr.Server(ctx, budget_bytes=16 << 30, max_live=64, residual=fr.FR_PT2PL, iters=iters) as srv:
        tickets = [srv.submit(*dpool[i], sigma_start=s, w=0.1) for i, s in reqs]
        results = [srv.wait(t, 120_000) for t in tickets]
        st = srv.stats()
    assert st["completed"] >= len(reqs)
    worst = 0.0
    for (i, s), res in zip(reqs, results):
        assert res.status == 0, (i, s)
        X, Y, Yn = dpool[i]
        Ta, ra = ctx.register_rigid(X, Y, Yn, residual=1, iters=iters, sigma_start=s, sigma_end=s, w=0.1)
        Tk, _ = ctx.register_rigid(X, Y, Yn, residual=1, iters=iters, sigma_start=s, sigma_end=s, w=0.1, kahan=1)
        kr, kt = pose_diff(Ta, Tk)
        bar_r, bar_t = min(1e-3, max(1e-4, 10 * kr)), min(1e-4, max(1e-5, 10 * kt))
        dr, dt = pose_diff(res.T, Ta)
        worst = max(worst, dr / bar_r)
        assert dr < bar_r and dt < bar_t, (i, s, dr, dt, kr, kt)
        assert res.report.iters_run == ra.iters_run == iters
        assert res.report.lattice_vertices == ra.lattice_vertices
    # the sparse request overflowed its compact table (more vertices than
    # 3 N slots hold) and was rerun at the safe size
    assert results[-1].report.lattice_vertices > 1.5 * 20000


@pytest.mark.parametrize("storage", [1, 2])
def test_16bit_storage_requests_equal_single_registrations(ctx, pairs, storage):
    # bfloat16 / half lattice records in the server (a build's records are
    # converted in the tick after it): each request equals the single path
    # with the same storage, within the batched path's bar plus one 16-bit
    # ulp flip of the targets (float32 sums in another order may round a
    # record to the other neighbour): e = 6 u R moves the pose by at most e
    # (translation) and e / r (rotation, r the model's rms radius).
    import paper_1811_10136_gb300 as fr
    U = {1: 2.0 ** -8, 2: 2.0 ** -11}
    iters = 12
    with fr.Server(ctx, budget_bytes=1 << 30, max_live=64, residual=fr.FR_PT2PL, iters=iters,
                   storage=storage) as srv:
        reqs = []
        for r in range(2):
            for i, p in enumerate(pairs):
                s0, s1 = SIGMAS[(i + r) % len(SIGMAS)]
                reqs.append((i, s0, s1, srv.submit(dev(p.X), dev(p.Y), dev(p.Yn), sigma_start=s0, sigma_end=s1,
                                                   w=0.1)))
        results = [(i, s0, s1, srv.wait(t, 60_000)) for i, s0, s1, t in reqs]
    for i, s0, s1, res in results:
        assert res.status == 0
        p = pairs[i]
        Ts, rs = ctx.register_rigid(dev(p.X), dev(p.Y), dev(p.Yn), residual=1, iters=iters, sigma_start=s0,
                                    sigma_end=s1, w=0.1, storage=storage)
        P = p.X[:, :3].astype(np.float64)
        rr = float(np.sqrt(((P - P.mean(0)) ** 2).sum(1).mean()))
        e = 6 * U[storage] * math.sqrt(1.5) * min(s0, s1)
        dr, dt = pose_diff(res.T, Ts)
        assert dr <= SAME_ROT + e / rr and dt <= SAME_TRANS + e, (i, s0, s1, dr, dt)
        assert res.report.iters_run == rs.iters_run == iters
        assert res.report.lattice_builds == rs.lattice_builds
