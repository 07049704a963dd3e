"""fr_estep_noalloc against fr_estep.

fr_estep_noalloc serves callers that cannot call cudaMalloc (a framework
whose allocator owns the device memory, a real-time loop that must not stall
on allocation): it runs the E step on a fixed scratch array compiled into the
library.  Here it must give the same E-step sums as the context-based
fr_estep, within the tolerance of the other E-step tests, on two calls in a
row (the second call checks that the first left the shared table empty).
This file is collected last so that a failure here stops a run only after
every other test has run.
"""
import numpy as np
import pytest

from paper_1811_10136_gb300 import synth

pytestmark = pytest.mark.gpu

REL = 1e-4


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("normals", [True, False])
def test_noalloc_estep_matches_estep_two_calls(normals):
    import torch
    import paper_1811_10136_gb300 as fr
    ctx = fr.Context(0)
    for seed in (21, 22):
        p = synth.depth_frame_pair(seed, W=96, H=72)
        assert p.Y.shape[0] <= fr.FR_NOALLOC_MAX_OBS
        T = synth.make_T(synth.random_rotation(np.random.default_rng(seed), 0.01), [0.002, 0.001, -0.001])
        X, Y = _dev(p.X), _dev(p.Y)
        Yn = _dev(p.Yn) if normals else None
        ref = ctx.estep(X, Y, Yn, sigma=0.03, T=T).cpu().numpy().astype(np.float64)
        out = fr.estep_noalloc(X, Y, Yn, sigma=0.03, T=T)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.float64)
        ymax = float(np.abs(p.Y[:, :3]).max())
        cols = [1.0] + [ymax] * 3 + ([1.0] * 3 if normals else [])
        scale = ref[:, :1] * np.array(cols)[None, :] + 1e-6
        err = np.abs(got - ref)
        assert (err <= REL * (np.abs(ref) + scale)).all(), float((err / (REL * (np.abs(ref) + scale))).max())
        assert (got[:, 0] > 0).sum() == (ref[:, 0] > 0).sum()


def test_noalloc_rejects_too_many_points():
    import paper_1811_10136_gb300 as fr
    Y = _dev(np.zeros((fr.FR_NOALLOC_MAX_OBS + 1, 4)))
    X = _dev(np.zeros((4, 4)))
    with pytest.raises(fr.FilterRegError) as e:
        fr.estep_noalloc(X, Y, sigma=0.1)
    assert e.value.status == fr.FR_EINVAL
