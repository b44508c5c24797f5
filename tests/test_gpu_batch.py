"""Batched uneven problems in one graph launch (hfmm_plan_batch / hfmm_apply_batch).

Each problem's batched result must equal its own planned apply, the graph must replay
(second call) and re-capture for new buffers, and results stay within eps of the direct sum.
"""
import numpy as np
import pytest

from oracle import direct
from paper_0911_4114_gb300 import FmmBatch, workloads as wl
from gpu_util import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _problems(n, seed, nmin=800, nmax=5000):
    g = wl.rng(seed)
    sizes = np.exp(g.uniform(np.log(nmin), np.log(nmax), n)).astype(int)
    kappas = g.uniform(10.0, 30.0, n)
    return [(wl.cube(int(m), g), None, float(k)) for m, k in zip(sizes, kappas)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_single_applies_and_replays(precision):
    import torch
    probs = _problems(6, 60)
    eps, R = 1e-5, 2
    batch = FmmBatch([(x, x, k, eps) for x, _, k in probs], precision=precision, max_rhs=R, max_leaf=32)
    g = wl.rng(61)
    qs = [torch.as_tensor(wl.charges(len(x), R, g), device="cuda") for x, _, _ in probs]
    outs = batch.apply(qs)
    torch.cuda.synchronize()
    first = [o.cpu().numpy() for o in outs]
    for p, (x, _, k) in enumerate(probs):
        single = batch.plan(p).apply(qs[p])
        torch.cuda.synchronize()
        assert np.array_equal(single.cpu().numpy(), first[p]), p
    # replay of the cached graph into the same buffers
    for o in outs:
        o.zero_()
    batch.apply(qs, outs)
    torch.cuda.synchronize()
    for p in range(len(probs)):
        assert np.array_equal(outs[p].cpu().numpy(), first[p])
    # new output buffers: re-capture
    outs2 = batch.apply(qs)
    torch.cuda.synchronize()
    for p in range(len(probs)):
        assert np.array_equal(outs2[p].cpu().numpy(), first[p])
    x, _, k = probs[0]
    want = direct.direct(x, x, qs[0].cpu().numpy(), k)
    assert rel(first[0], want) <= eps
