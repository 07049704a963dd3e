"""Sharded single registration (model points split across ranks) on CPU.

The E-step and Gauss-Newton sums of Eq. 17-18 are sums over model points, so
a shard's normal equations (with Eq. 7's outlier constant taken from the whole
model) add up to the whole model's.  Pinned here without a GPU:
- the oracle's shard normal equations are additive over 2 and 3 shards;
- the library's host solve and SE(3) update (fr_rigid_solve_update) against
  one step of the oracle's own EM driver (Cholesky, its exponential);
- the library's host EM loop (fr_em_sharded) with the oracle as provider
  against the oracle's registration (schedule, updates, stop test);
- two gloo ranks, each holding half of the model: both end at the same pose,
  the single-process registration's.
"""
import os
import socket

import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

F32 = lambda x: float(np.float32(x))  # noqa: E731 -- sigmas both sides read alike


def _pair():
    return synth.depth_frame_pair(3, W=64, H=48)


def _full_ne(orc, p, T, sigma, residual):
    return orc.rigid_normal_equations(p.X, p.Y, p.Yn, sigma=sigma, T=T, residual=residual)


@pytest.mark.parametrize("parts", [2, 3])
@pytest.mark.parametrize("residual", [0, 1])
def test_oracle_normal_equations_are_additive(orc, parts, residual):
    p = _pair()
    T = synth.make_T(synth.random_rotation(np.random.default_rng(1), 0.03), [0.004, -0.003, 0.002])
    sigma = F32(0.02)
    M = p.X.shape[0]
    whole = _full_ne(orc, p, T, sigma, residual)
    cuts = np.linspace(0, M, parts + 1).astype(int)
    shards = [orc.rigid_normal_equations(p.X[a:b], p.Y, p.Yn, sigma=sigma, T=T, residual=residual, M_total=M)
              for a, b in zip(cuts[:-1], cuts[1:])]
    np.testing.assert_allclose(np.sum(shards, 0), whole, rtol=1e-12, atol=1e-12 * np.abs(whole).max())
    assert whole[29] > 0.3 * M  # inliers counted
    # the outlier constant is the whole model's: a shard alone (M_total = its
    # own size) weighs its points differently
    a, b = cuts[0], cuts[1]
    alone = orc.rigid_normal_equations(p.X[a:b], p.Y, p.Yn, sigma=sigma, T=T, residual=residual)
    assert not np.allclose(alone[:27], shards[0][:27], rtol=1e-9)


def test_solve_update_matches_the_oracle_step(orc):
    import paper_1811_10136_gb300 as fr
    p = _pair()
    T0 = synth.make_T(synth.random_rotation(np.random.default_rng(2), 0.03), [0.01, 0.0, -0.005])
    sigma = F32(0.02)
    for residual in (0, 1):
        ne = _full_ne(orc, p, T0, sigma, residual)
        T1, tn, ok = fr.rigid_solve_update(ne, T0)
        assert ok and tn > 0
        Tref, rep = orc.register_rigid(p.X, p.Y, p.Yn, sigma=sigma, iters=1, residual=residual, T0=T0)
        np.testing.assert_allclose(T1, Tref, rtol=0, atol=1e-12)
        assert tn == pytest.approx(rep.last_twist_norm, rel=1e-10)


def test_solve_update_refuses_a_singular_system():
    import paper_1811_10136_gb300 as fr
    ne = np.zeros(30)
    T, tn, ok = fr.rigid_solve_update(ne, np.eye(4))
    assert not ok and (T == np.eye(4)).all()
    ne[:21] = [1, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 1, 0, 0]  # A[5][5] = 0
    assert not fr.rigid_solve_update(ne, np.eye(4))[2]


@pytest.mark.parametrize("residual", [0, 1])
def test_em_loop_with_the_oracle_provider_equals_the_oracle_driver(orc, residual):
    import paper_1811_10136_gb300 as fr
    p = _pair()
    s0, s1 = F32(0.04), F32(0.01)
    kw = dict(sigma_start=s0, sigma_end=s1, iters=8, w=F32(0.1), residual=residual)

    def provider(T, sigma):
        return orc.rigid_normal_equations(p.X, p.Y, p.Yn, sigma=sigma, T=T, residual=residual, w=F32(0.1))

    T, rep, st = fr.em_sharded(provider, None, **kw)
    assert st == 0 and rep.iters_run == 8
    Tref, rref = orc.register_rigid(p.X, p.Y, p.Yn, sigma=s0, sigma_end=s1, iters=8, w=F32(0.1),
                                    residual=residual)
    np.testing.assert_allclose(T, Tref, rtol=0, atol=1e-10)
    assert rep.last_sigma == pytest.approx(rref.last_sigma, rel=0)
    assert rep.last_inliers == rref.last_inliers


def test_em_loop_stops_and_reports_callback_failures(orc):
    import paper_1811_10136_gb300 as fr
    p = _pair()

    def provider(T, sigma):
        return orc.rigid_normal_equations(p.X, p.Y, p.Yn, sigma=sigma, T=T, residual=1)

    T, rep, st = fr.em_sharded(provider, None, sigma_start=F32(0.01), sigma_end=F32(0.01), iters=50,
                               residual=1, stop_twist=1e-5)
    assert st == 0 and rep.iters_run < 50 and rep.last_twist_norm < 1e-5

    def failing(v):
        raise RuntimeError("collective lost a rank")
    with pytest.raises(RuntimeError, match="lost a rank"):
        fr.em_sharded(provider, failing, sigma_start=F32(0.01), iters=3, residual=1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import oracle
    import paper_1811_10136_gb300 as fr
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _pair()
        M = p.X.shape[0]
        cuts = np.linspace(0, M, world + 1).astype(int)
        Xs = p.X[cuts[rank]:cuts[rank + 1]]

        def provider(T, sigma):
            return oracle.rigid_normal_equations(Xs, p.Y, p.Yn, sigma=sigma, T=T, residual=1, w=F32(0.1),
                                                 M_total=M)

        T, rep, st = fr.em_sharded(provider, fr.torch_allreduce(), sigma_start=F32(0.04), sigma_end=F32(0.01),
                                   iters=8, w=F32(0.1), residual=1)
        out.put((rank, T, rep.iters_run, st))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reach_the_single_process_pose(orc):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (_, T0, n0, s0), (_, T1, n1, s1) = res
    assert s0 == s1 == 0 and n0 == n1 == 8
    np.testing.assert_array_equal(T0, T1)  # the same summed system on every rank
    p = _pair()
    Tref, _ = orc.register_rigid(p.X, p.Y, p.Yn, sigma=F32(0.04), sigma_end=F32(0.01), iters=8, w=F32(0.1),
                                 residual=1)
    np.testing.assert_allclose(T0, Tref, rtol=0, atol=1e-9)
