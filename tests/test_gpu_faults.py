"""Failure handling by host-side fault injection (no GPU fault): device
allocations made to fail one at a time (fr_debug_fail_allocations), at every
allocation a call makes in turn.  Each failed call must return FR_ENOMEM, and
the same context (or a new server / node graph) must then complete the call
correctly: whatever a failed call had already allocated is either kept
consistently or released.
"""
import math

import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

pytestmark = pytest.mark.gpu

MAX_ALLOCS = 64  # more than any of these calls makes
# Poses after a failure against a clean run: lattice sums are float atomics,
# so two clean runs differ too (up to ~1e-4 on these small frames); the bound
# is the one the parity tests hold against the oracle, far below what a
# table left dirty or a buffer left unset produces.
ROT_TOL, TRANS_TOL = 1e-3, 1e-4


@pytest.fixture(autouse=True)
def clear_faults():
    import paper_1811_10136_gb300 as fr
    fr.debug_fail_allocations(0, 0)
    yield
    fr.debug_fail_allocations(0, 0)


def dev(a, dtype=np.float32):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def f32(x):
    return float(np.float32(x))


def pose_diff(A, B):
    return math.radians(synth.rotation_angle_deg(A, B)), float(np.linalg.norm(A[:3, 3] - B[:3, 3]))


def sweep(make, call, check):
    """For after = 0, 1, ...: on a fresh object from make(), fail the
    allocation after `after` successful ones during call(obj); a failure must
    be FR_ENOMEM, after which call(obj) succeeds and passes check.  Stops at
    the first `after` the call completes without reaching."""
    import paper_1811_10136_gb300 as fr
    failed = 0
    for after in range(MAX_ALLOCS):
        obj = make()
        fr.debug_fail_allocations(after, 1)
        try:
            call(obj)
            done = True
        except fr.FilterRegError as e:
            assert e.status == fr.FR_ENOMEM, (after, e)
            done = False
        fr.debug_fail_allocations(0, 0)
        if done:
            check(call(obj))
            close = getattr(obj, "close", None)
            if close:
                close()
            assert failed >= 1  # the call allocates at least once
            return failed
        failed += 1
        check(call(obj))  # the same object after the failure
        close = getattr(obj, "close", None)
        if close:
            close()
    raise AssertionError("more allocations than expected")


def test_rigid_registration():
    import paper_1811_10136_gb300 as fr
    p = synth.depth_frame_pair(4, W=96, H=72)
    kw = dict(residual=1, iters=8, sigma_start=f32(0.03), sigma_end=f32(0.01), w=f32(0.1))
    T_ref, _ = fr.Context(0).register_rigid(dev(p.X), dev(p.Y), dev(p.Yn), **kw)

    def call(ctx):
        return ctx.register_rigid(dev(p.X), dev(p.Y), dev(p.Yn), **kw)[0]

    def check(T):
        dr, dt = pose_diff(T, T_ref)
        assert dr < ROT_TOL and dt < TRANS_TOL, (dr, dt)

    sweep(lambda: fr.Context(0), call, check)


def test_batched_registration():
    import paper_1811_10136_gb300 as fr
    pairs = [synth.depth_frame_pair(s, W=64, H=48) for s in (5, 6, 7)]
    kw = dict(residual=1, iters=6, sigma_start=f32(0.03), sigma_end=f32(0.01), w=f32(0.1))
    dpairs = [(dev(q.X), dev(q.Y), dev(q.Yn)) for q in pairs]
    ref = fr.Context(0).register_rigid_batch(dpairs, **kw)

    def call(ctx):
        out = ctx.register_rigid_batch(dpairs, **kw)
        bad = [st for _, _, st in out if st != 0]
        if bad:
            raise fr.FilterRegError(bad[0], "batch item")
        return out

    def check(out):
        for (T, _, st), (Tr, _, _) in zip(out, ref):
            assert st == 0
            dr, dt = pose_diff(T, Tr)
            assert dr < ROT_TOL and dt < TRANS_TOL, (dr, dt)

    sweep(lambda: fr.Context(0), call, check)


def test_feature_estep():
    import paper_1811_10136_gb300 as fr
    fp = synth.feature_frame_pair(2, W=64, H=48)
    sf = np.array([0.02] * 3 + [0.25] * 3, np.float32)
    ref = fr.Context(0).estep_features(dev(fp.FX), dev(fp.FY), sf, dev(fp.Y), dev(fp.Yn))[0].cpu().numpy()

    def call(ctx):
        return ctx.estep_features(dev(fp.FX), dev(fp.FY), sf, dev(fp.Y), dev(fp.Yn))[0].cpu().numpy()

    def check(out):
        scale = np.abs(ref[:, :1]) * 4 + 1e-6
        assert (np.abs(out - ref) <= 1e-4 * (np.abs(ref) + scale)).all()

    sweep(lambda: fr.Context(0), call, check)


def test_articulated_registration():
    import paper_1811_10136_gb300 as fr
    p = synth.articulated_pair(3, n_points=3000)
    kw = dict(residual=0, iters=4, sigma_start=f32(0.05), sigma_end=f32(0.02), w=f32(0.1))
    args = (dev(p.Xref), dev(p.body, np.int32), p.tree, dev(p.Y), None)
    R_ref, q_ref, _ = fr.Context(0).register_articulated(*args, **kw)

    def call(ctx):
        return ctx.register_articulated(*args, **kw)[:2]

    def check(out):
        R, q = out
        assert pose_diff(R, R_ref)[0] < ROT_TOL
        assert float(np.abs(q - q_ref).max(initial=0.0)) < ROT_TOL

    sweep(lambda: fr.Context(0), call, check)


def test_batched_articulated_registration():
    import paper_1811_10136_gb300 as fr
    tree = synth.random_kintree(23)
    pairs = [synth.articulated_pair(70 + s, n_points=2000, max_joint_deg=5, tree=tree) for s in range(3)]
    kw = dict(residual=0, iters=3, sigma_start=f32(0.03), sigma_end=f32(0.02), w=f32(0.1))
    items = [(dev(p.Xref), dev(p.body, np.int32), dev(p.Y), None, None, None) for p in pairs]
    ref = fr.Context(0).register_articulated_batch(items, tree, **kw)

    def call(ctx):
        out = ctx.register_articulated_batch(items, tree, **kw)
        bad = [r[3] for r in out if r[3] != 0]
        if bad:
            raise fr.FilterRegError(bad[0], "batch item")
        return out

    def check(out):
        for (R, q, _, st), (Rr, qr, _, _) in zip(out, ref):
            assert st == 0
            assert pose_diff(R, Rr)[0] < ROT_TOL
            assert float(np.abs(q - qr).max(initial=0.0)) < ROT_TOL

    sweep(lambda: fr.Context(0), call, check)


def test_node_graph_create_and_register():
    import paper_1811_10136_gb300 as fr
    ng_pair = synth.nodegraph_pair(1, W=64, H=48, n_nodes=30)
    ctx = fr.Context(0)
    kw = dict(lam=10.0, pcg_iters=10, residual=1, iters=3, sigma_start=f32(0.02), sigma_end=f32(0.02), w=f32(0.1))

    def make_graph():
        return fr.NodeGraph(ctx, dev(ng_pair.Xref), dev(ng_pair.knn, np.int32), dev(ng_pair.skw),
                            ng_pair.node_pos, ng_pair.edges)

    ref = make_graph().register(dev(ng_pair.Y), dev(ng_pair.Yn), **kw)[0]
    # creation: a failed create leaves nothing behind; the next create works
    for after in range(MAX_ALLOCS):
        fr.debug_fail_allocations(after, 1)
        try:
            g = make_graph()
        except fr.FilterRegError as e:
            assert e.status == fr.FR_ENOMEM
            fr.debug_fail_allocations(0, 0)
            continue
        fr.debug_fail_allocations(0, 0)
        T = g.register(dev(ng_pair.Y), dev(ng_pair.Yn), **kw)[0]
        assert max(pose_diff(a, b)[0] for a, b in zip(T, ref)) < ROT_TOL
        break
    else:
        raise AssertionError("more allocations than expected")
    assert after >= 1

    # registration on a fresh context (its tables and buffers come on first use)
    class Fresh:
        def __init__(self):
            self.ctx = fr.Context(0)
            self.g = fr.NodeGraph(self.ctx, dev(ng_pair.Xref), dev(ng_pair.knn, np.int32), dev(ng_pair.skw),
                                  ng_pair.node_pos, ng_pair.edges)

    def call(f):
        return f.g.register(dev(ng_pair.Y), dev(ng_pair.Yn), **kw)[0]

    def check(T):
        assert max(pose_diff(a, b)[0] for a, b in zip(T, ref)) < ROT_TOL

    sweep(Fresh, call, check)


def test_server_create():
    import paper_1811_10136_gb300 as fr
    p = synth.depth_frame_pair(8, W=64, H=48)
    ctx = fr.Context(0)
    kw = dict(residual=fr.FR_PT2PL, iters=6)
    T_ref, _ = ctx.register_rigid(dev(p.X), dev(p.Y), dev(p.Yn), residual=1, iters=6, sigma_start=f32(0.02),
                                  sigma_end=f32(0.02), w=f32(0.1))
    for after in range(MAX_ALLOCS):
        fr.debug_fail_allocations(after, 1)
        try:
            srv = fr.Server(ctx, budget_bytes=64 << 20, max_live=8, **kw)
        except fr.FilterRegError as e:
            assert e.status == fr.FR_ENOMEM
            fr.debug_fail_allocations(0, 0)
            continue
        fr.debug_fail_allocations(0, 0)
        with srv:
            t = srv.submit(dev(p.X), dev(p.Y), dev(p.Yn), sigma_start=f32(0.02), sigma_end=f32(0.02), w=f32(0.1))
            res = srv.wait(t, 60_000)
        assert res.status == 0
        dr, dt = pose_diff(res.T, T_ref)
        assert dr < ROT_TOL and dt < TRANS_TOL, (dr, dt)
        break
    else:
        raise AssertionError("more allocations than expected")
    assert after >= 1


def test_server_tick_allocation():
    """The first tick sizes the per-tick buffers; when that fails every
    request in the server ends with FR_ENOMEM and a new server works."""
    import paper_1811_10136_gb300 as fr
    p = synth.depth_frame_pair(9, W=64, H=48)
    ctx = fr.Context(0)
    srv = fr.Server(ctx, budget_bytes=64 << 20, max_live=8, residual=fr.FR_PT2PL, iters=6)
    fr.debug_fail_allocations(0, 1)
    with srv:
        t = srv.submit(dev(p.X), dev(p.Y), dev(p.Yn), sigma_start=f32(0.02), sigma_end=f32(0.02), w=f32(0.1))
        res = srv.wait(t, 60_000)
    fr.debug_fail_allocations(0, 0)
    assert res.status == fr.FR_ENOMEM
    with fr.Server(ctx, budget_bytes=64 << 20, max_live=8, residual=fr.FR_PT2PL, iters=6) as srv2:
        t = srv2.submit(dev(p.X), dev(p.Y), dev(p.Yn), sigma_start=f32(0.02), sigma_end=f32(0.02), w=f32(0.1))
        assert srv2.wait(t, 60_000).status == 0
