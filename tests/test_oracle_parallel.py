"""The oracle's OpenMP build (the benchmark's all-core CPU baseline) returns
bit-identical results to its single-thread build: every sum keeps a fixed
order (fixed chunks reduced in chunk order; a total order for the splat
sort), so the number of threads changes nothing."""
import numpy as np
import pytest

from paper_1811_10136_gb300 import synth


@pytest.fixture(scope="module")
def both(orc):
    orc.build(openmp=True)
    yield orc
    orc.set_parallel(False)


def _register(orc, parallel, threads, pair, **kw):
    orc.set_parallel(parallel, threads)
    try:
        return orc.register_rigid(pair.X, pair.Y, pair.Yn, **kw)
    finally:
        orc.set_parallel(False)


@pytest.mark.parametrize("backend", ["lattice", "exact"])
def test_openmp_build_bit_identical(both, backend):
    orc = both
    if backend == "lattice":
        pair = synth.depth_frame_pair(7, W=160, H=120)
        kw = dict(sigma=0.04, sigma_end=0.015, w=0.1, iters=5, residual=orc.PT2PL, backend=orc.LATTICE)
    else:
        pair = synth.depth_frame_pair(8, W=48, H=36)
        kw = dict(sigma=0.03, sigma_end=0.03, w=0.1, iters=3, residual=orc.PT2PL, backend=orc.EXACT)
    T1, r1 = _register(orc, False, None, pair, **kw)
    for threads in (2, 3, 8):
        Tp, rp = _register(orc, True, threads, pair, **kw)
        np.testing.assert_array_equal(Tp, T1)
        assert rp.last_inliers == r1.last_inliers
        assert rp.last_cost == r1.last_cost and rp.last_sum_w == r1.last_sum_w


def test_openmp_lattice_vertices_bit_identical(both):
    orc = both
    pair = synth.depth_frame_pair(9, W=160, H=120)
    V = np.concatenate([np.ones((len(pair.Y), 1)), pair.Y[:, :3].astype(np.float64)], 1)
    k1, v1 = orc.Lattice(pair.Y, V, 0.02).vertices()
    orc.set_parallel(True, 4)
    try:
        k2, v2 = orc.Lattice(pair.Y, V, 0.02).vertices()
    finally:
        orc.set_parallel(False)
    np.testing.assert_array_equal(k1, k2)
    np.testing.assert_array_equal(v1, v2)


def test_thread_count_reported(both):
    orc = both
    assert orc.num_threads() == 1
    orc.set_parallel(True, 3)
    try:
        assert orc.num_threads() == 3
    finally:
        orc.set_parallel(False)
