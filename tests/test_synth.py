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


def _pairs(e):
    src, dst = e.src.astype(np.int64), e.dst.astype(np.int64)
    keep = src != dst
    a, b = np.minimum(src[keep], dst[keep]), np.maximum(src[keep], dst[keep])
    u = np.unique(a * e.n + b)
    return u // e.n, u % e.n


def test_dcsbm_recipe_realises_its_parameters():
    """DC-SBM N = 50,000, 44 blocks, mean degree 40, within:between 3:1 in edge counts, Pareto
    2.5 degrees: after loops and repeats are removed the mean degree and the count ratio stay
    within 10% and 15% of the recipe, and the degrees are heavy-tailed (max about the structural
    cutoff sqrt(N d) = 1414)."""
    e, _ = synth.workload("dcsbm_n50k_k44")
    pa, pb = _pairs(e)
    deg = np.bincount(np.concatenate([pa, pb]), minlength=e.n)
    assert abs(deg.mean() - 40.0) <= 4.0
    within = int((e.labels[pa] == e.labels[pb]).sum())
    assert abs(within / (len(pa) - within) - 3.0) <= 0.45
    assert 700 <= deg.max() <= 3000 and deg.max() >= 20 * np.median(deg)
    assert deg.min() >= 1  # isolated nodes are joined to one random node
    assert len(np.unique(e.labels)) == 44


def test_sbm_probability_ratio_recipe():
    """SBM N = 1000, 11 blocks, mean degree 20, within:between edge probability 10:1."""
    e, _ = synth.workload("sbm_n1000_k11")
    pa, pb = _pairs(e)
    sizes = np.bincount(e.labels, minlength=11).astype(np.float64)
    same = e.labels[pa] == e.labels[pb]
    pairs_within = float((sizes * (sizes - 1) / 2).sum())
    pairs_between = e.n * (e.n - 1) / 2 - pairs_within
    ratio = (same.sum() / pairs_within) / ((~same).sum() / pairs_between)
    assert 7.0 <= ratio <= 13.0
    assert abs(2.0 * len(pa) / e.n - 20.0) <= 2.0
