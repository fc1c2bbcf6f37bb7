"""ofsc_objective_grad_noalloc: the objective and gradient with no device allocation.

Callers that must not allocate device memory while they run (a process whose memory is held by
another allocator, or a latency-bound loop) use this entry point; it takes its temporary storage
from a static array inside the library. Here it must give what ofsc_objective_grad gives, within
the tolerance of the other objective/gradient tests, on two calls in a row (the second call
reuses the array the first one left behind).
"""
import numpy as np
import pytest

from paper_2305_10356_gb300 import build, ofsc, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    ofsc.lib()
    return torch


def _graph(torch, e):
    src = torch.from_numpy(e.src).cuda()
    dst = torch.from_numpy(e.dst).cuda()
    w = None if e.w is None else torch.from_numpy(e.w).cuda()
    return ofsc.ofsc_graph_build(e.n, src, dst, w)


@pytest.mark.parametrize("which", [1, 2])
def test_noalloc_matches_objective_grad_twice(torch_cuda, which):
    """Two calls in a row (k = 29, then 32: different padding) against ofsc_objective_grad, element
    by element within 1e-5 of max|grad f| (the tolerance of the other gradient tests), and no change
    of the device's free memory across a call after the first (cudaMemGetInfo)."""
    torch = torch_cuda
    e, _ = synth.workload("wsbm_n20k_k32", n=3000)
    g = _graph(torch, e)
    for call in range(2):
        x = synth.initial_block(e.n, 29 + 3 * call, 100 + call)  # k = 29 then 32: padding differs
        X = torch.from_numpy(x).cuda()
        G_ref = torch.empty_like(X)
        f_ref = ofsc.ofsc_objective_grad(g, which, X, G_ref)
        G = torch.full_like(X, float("nan"))
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        f = ofsc.ofsc_objective_grad_noalloc(g, which, X, G)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        if call == 1:
            assert free1 == free0, (free0, free1)
        assert f == pytest.approx(f_ref, rel=1e-5)
        a = G.cpu().numpy().astype(np.float64)
        b = G_ref.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


def test_noalloc_rejects_sizes_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    n = (1 << 20) // 8 + 1  # n * kp just above 2^20 for k = 8
    e = synth.EdgeList(n=n, src=np.array([0], np.int32), dst=np.array([1], np.int32), w=None,
                       labels=np.zeros(n, np.int32), n_blocks=1)
    g = _graph(torch, e)
    X = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(ofsc.OfscError) as ei:
        ofsc.ofsc_objective_grad_noalloc(g, 1, X)
    assert ei.value.status == ofsc.ERR_INVALID_ARG
    assert "scratch" in str(ei.value)
