"""The seeded input recipes (CPU): the batch of uneven graphs and the edge-sampled stream."""
import numpy as np

from paper_2305_10356_gb300 import synth


def test_batch_recipe_sizes_and_determinism():
    """32 SBMs with N ~ U[2000, 100000] (scaled), k ~ U[8, 64], mean degree ~ U[16, 48]; the same
    graphs and X0 on every call."""
    scale = 0.05
    a = synth.batch("sbm_batch32", scale)
    b = synth.batch("sbm_batch32", scale)
    assert len(a) == 32
    ks = []
    for (e, x0), (e2, x2) in zip(a, b):
        k = e.n_blocks
        ks.append(k)
        assert 8 <= k <= 64
        assert max(4 * k, round(2000 * scale)) <= e.n <= round(100_000 * scale)
        assert x0.shape == (e.n, k) and x0.dtype == np.float32
        assert np.array_equal(e.src, e2.src) and np.array_equal(e.dst, e2.dst) and np.array_equal(x0, x2)
        assert e.src.min() >= 0 and e.dst.max() < e.n
        d = 2.0 * e.m / e.n
        assert 8.0 <= d <= 60.0  # mean degree ~ U[16, 48] before duplicates and loops are removed
    assert len(set(ks)) > 10  # the k's are spread out


def test_stream_snapshots_nest():
    """Each snapshot of the stream holds the previous one's edges and a tenth more of them."""
    snaps, x0 = synth.stream("sbm_stream_n200k_k71", n=2000)
    assert len(snaps) == 10
    prev = set()
    for s in snaps:
        cur = set(zip(s.src.tolist(), s.dst.tolist()))
        assert prev <= cur
        prev = cur
    assert x0.shape == (2000, 71)
