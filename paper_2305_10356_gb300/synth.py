"""Seeded synthetic inputs: stochastic-block-model edge lists and initial feature blocks.

This module only draws inputs. It holds none of the method's arithmetic (no Laplacian, no
degrees, no deduplication), so both the CUDA path and the FP64 oracle can be fed from it
without sharing any computation.

The graphs stand in for the IEEE HPEC Graph Challenge stochastic-block-partition graphs that
Sec. 5 ("Dataset") uses: planted blocks with low/high block overlap and low/high block-size
variation. Node ids are randomly permuted, so block membership gives no memory locality.

Every generator returns an undirected edge list in which each sampled edge appears once as
(src, dst). The list may contain self-loops and repeated pairs; removing them is the graph
builder's job (Eq. (1) defines S as a 0/1 matrix with no self-loops).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    """Counter-based generator (Philox) seeded with `seed`."""
    return np.random.Generator(np.random.Philox(int(seed)))


@dataclasses.dataclass
class EdgeList:
    n: int
    src: np.ndarray  # int32 [m]
    dst: np.ndarray  # int32 [m]
    w: np.ndarray | None  # float32 [m] or None (binary S)
    labels: np.ndarray  # int32 [n], planted block of each node
    n_blocks: int

    @property
    def m(self) -> int:
        return int(self.src.shape[0])


def block_sizes_uniform(n: int, n_blocks: int, spread: float, rng) -> np.ndarray:
    """Block sizes drawn uniformly within +-spread of n/n_blocks, rescaled to sum to n."""
    base = n / n_blocks
    raw = rng.uniform(base * (1 - spread), base * (1 + spread), size=n_blocks)
    return _round_to_total(raw, n)


def block_sizes_lognormal(n: int, n_blocks: int, sigma: float, rng) -> np.ndarray:
    """Block sizes with lognormal(0, sigma) spread, rescaled to sum to n (each block >= 2)."""
    raw = rng.lognormal(0.0, sigma, size=n_blocks)
    return _round_to_total(raw, n)


def _round_to_total(raw: np.ndarray, n: int) -> np.ndarray:
    sizes = np.maximum(2, np.floor(raw / raw.sum() * n)).astype(np.int64)
    diff = n - int(sizes.sum())
    order = np.argsort(-raw)
    i = 0
    while diff != 0:
        j = order[i % len(order)]
        if diff > 0:
            sizes[j] += 1
            diff -= 1
        elif sizes[j] > 2:
            sizes[j] -= 1
            diff += 1
        i += 1
    return sizes


def truncated_pareto(n: int, gamma: float, cutoff: float, rng) -> np.ndarray:
    """Samples on [1, cutoff] with density proportional to x^(-gamma) (inverse CDF)."""
    a = gamma - 1.0
    u = rng.random(n)
    return (1.0 - u * (1.0 - cutoff ** (-a))) ** (-1.0 / a)


def pareto_cutoff(gamma: float, ratio: float) -> float:
    """Truncation point c of Pareto(gamma) on [1, c] with c / mean = ratio (bisection)."""
    a = gamma - 1.0

    def c_over_mean(c):
        if abs(a - 1.0) < 1e-12:
            mean = math.log(c) / (1.0 - 1.0 / c)
        else:
            mean = a / (a - 1.0) * (1.0 - c ** (1.0 - a)) / (1.0 - c ** (-a))
        return c / mean

    lo, hi = 1.0 + 1e-9, 1e12
    for _ in range(200):
        mid = math.sqrt(lo * hi)
        if c_over_mean(mid) < ratio:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def sbm(n: int, n_blocks: int, mean_degree: float, ratio: float, *, ratio_kind: str = "prob",
        sizes: str = "uniform", size_param: float = 0.2, gamma: float | None = None,
        weighted: bool = False, join_isolated: bool = True, seed: int = 0) -> EdgeList:
    """Stochastic block model (degree-corrected when `gamma` is given).

    ratio_kind="prob": within-block edge probability = ratio x between-block probability.
    ratio_kind="count": expected within-block edges = ratio x expected between-block edges.
    sizes="uniform": block sizes within +-size_param of n/n_blocks; "lognormal": sigma=size_param.
    gamma: node propensities theta ~ Pareto(gamma), truncated so that the largest expected
    degree is the structural cutoff sqrt(n * mean_degree), and normalised to mean 1 inside each
    block (Karrer-Newman degree correction); endpoints are drawn proportionally to theta.
    weighted: w ~ U(0.5, 1.5) in FP32 per sampled edge.
    """
    rng = rng_for(seed)
    if sizes == "uniform":
        bs = block_sizes_uniform(n, n_blocks, size_param, rng)
    elif sizes == "lognormal":
        bs = block_sizes_lognormal(n, n_blocks, size_param, rng)
    else:
        raise ValueError(sizes)
    off = np.concatenate([[0], np.cumsum(bs)])
    # propensities in block-position order
    if gamma is not None:
        cut = pareto_cutoff(gamma, math.sqrt(n * mean_degree) / mean_degree)
        theta = truncated_pareto(n, gamma, cut, rng)
        for r in range(n_blocks):
            seg = theta[off[r]:off[r + 1]]
            seg *= len(seg) / seg.sum()
    else:
        theta = np.ones(n)
    ctheta = np.concatenate([[0.0], np.cumsum(theta)])

    m_total = rng.poisson(n * mean_degree / 2.0)
    bsf = bs.astype(np.float64)
    if ratio_kind == "prob":
        pw = float(np.sum(bsf * (bsf - 1) / 2))
        pb = float((n * n - np.sum(bsf * bsf)) / 2)
        frac_in = ratio * pw / (ratio * pw + pb)
    elif ratio_kind == "count":
        frac_in = ratio / (ratio + 1.0)
    else:
        raise ValueError(ratio_kind)
    m_in = rng.binomial(m_total, frac_in)
    m_out = m_total - m_in

    def endpoints(blocks: np.ndarray) -> np.ndarray:
        lo = ctheta[off[blocks]]
        hi = ctheta[off[blocks + 1]]
        u = lo + rng.random(blocks.shape[0]) * (hi - lo)
        pos = np.searchsorted(ctheta, u, side="right") - 1
        return np.clip(pos, off[blocks], off[blocks + 1] - 1)

    # within-block edges: block chosen proportional to its number of node pairs
    wpair = bsf * (bsf - 1) if gamma is None else bsf * bsf
    cw = np.cumsum(wpair / wpair.sum())
    rb = np.minimum(np.searchsorted(cw, rng.random(m_in), side="right"), n_blocks - 1)
    a_in = endpoints(rb)
    b_in = endpoints(rb)
    # between-block edges: (r, s), r != s, proportional to n_r * n_s
    cb = np.cumsum(bsf / bsf.sum())
    r1 = np.minimum(np.searchsorted(cb, rng.random(m_out), side="right"), n_blocks - 1)
    r2 = np.minimum(np.searchsorted(cb, rng.random(m_out), side="right"), n_blocks - 1)
    same = r1 == r2
    while same.any():
        r2[same] = np.minimum(np.searchsorted(cb, rng.random(int(same.sum())), side="right"),
                              n_blocks - 1)
        same = r1 == r2
    a_out = endpoints(r1)
    b_out = endpoints(r2)
    a = np.concatenate([a_in, a_out])
    b = np.concatenate([b_in, b_out])
    block_of_pos = np.repeat(np.arange(n_blocks, dtype=np.int32), bs)

    if join_isolated:
        touched = np.zeros(n, dtype=bool)
        nl = a != b
        touched[a[nl]] = True
        touched[b[nl]] = True
        iso = np.nonzero(~touched)[0]
        if iso.size:
            other = rng.integers(0, n - 1, size=iso.size)
            other = other + (other >= iso)  # uniform over nodes != iso
            a = np.concatenate([a, iso])
            b = np.concatenate([b, other])

    perm = rng.permutation(n)  # block position -> node id
    src = perm[a].astype(np.int32)
    dst = perm[b].astype(np.int32)
    labels = np.empty(n, dtype=np.int32)
    labels[perm] = block_of_pos
    w = None
    if weighted:
        w = rng.uniform(0.5, 1.5, size=src.shape[0]).astype(np.float32)
    return EdgeList(n=n, src=src, dst=dst, w=w, labels=labels, n_blocks=n_blocks)


def initial_block(n: int, k: int, seed: int) -> np.ndarray:
    """X0 with i.i.d. N(0, 1/n) entries, stored in FP32 (row-major n x k)."""
    rng = rng_for(seed)
    return (rng.standard_normal((n, k)) / math.sqrt(n)).astype(np.float32)


# ---------------------------------------------------------------------------------------------
# Named workloads. Seeds: 2305*1000 + workload index for the graph, +1 for X0.
# ---------------------------------------------------------------------------------------------

WORKLOADS = {
    # tiny SBM: 1,000 nodes, 11 blocks (+-20%), mean degree 20, edge-probability ratio 10:1
    "sbm_n1000_k11": dict(n=1000, n_blocks=11, mean_degree=20.0, ratio=10.0, ratio_kind="prob",
                          sizes="uniform", size_param=0.2, gamma=None, idx=1),
    # DC-SBM: 50,000 nodes, 44 blocks (lognormal sigma 0.5), power-law 2.5, mean 40, 3:1
    "dcsbm_n50k_k44": dict(n=50_000, n_blocks=44, mean_degree=40.0, ratio=3.0, ratio_kind="count",
                           sizes="lognormal", size_param=0.5, gamma=2.5, idx=2),
    # DC-SBM: 2,000,000 nodes, 128 blocks, power-law 2.3, mean 32, 5:1
    "dcsbm_n2m_k128": dict(n=2_000_000, n_blocks=128, mean_degree=32.0, ratio=5.0,
                           ratio_kind="count", sizes="uniform", size_param=0.2, gamma=2.3, idx=3),
    # weighted SBM: 20,000 nodes, 32 blocks (+-20%), mean degree 32, 10:1, w ~ U(0.5, 1.5)
    "wsbm_n20k_k32": dict(n=20_000, n_blocks=32, mean_degree=32.0, ratio=10.0, ratio_kind="prob",
                          sizes="uniform", size_param=0.2, gamma=None, weighted=True, idx=5),
}


def edge_stream(edges: EdgeList, parts: int, seed: int) -> list[EdgeList]:
    """Cumulative snapshots of a graph revealed by uniform edge sampling: the edge list in a random
    order, snapshot s (s = 0..parts-1) holding its first round((s + 1) m / parts) edges, i.e.
    1/parts, 2/parts, ... of the edges. Nodes without an edge yet are isolated in that snapshot."""
    rng = rng_for(seed)
    order = rng.permutation(edges.m)
    out = []
    for s in range(parts):
        take = order[: int(round((s + 1) * edges.m / parts))]
        out.append(EdgeList(n=edges.n, src=edges.src[take], dst=edges.dst[take],
                            w=None if edges.w is None else edges.w[take], labels=edges.labels,
                            n_blocks=edges.n_blocks))
    return out


STREAMS = {
    # SBM, 200,000 nodes, 71 blocks (+-20%), mean degree 30 at 100%, within:between 5:1 (edge
    # counts), revealed in ten cumulative snapshots (10%, 20%, ..., 100% of the edges)
    "sbm_stream_n200k_k71": dict(n=200_000, n_blocks=71, mean_degree=30.0, ratio=5.0, ratio_kind="count",
                                 sizes="uniform", size_param=0.2, gamma=None, join_isolated=False, idx=4,
                                 parts=10),
}


def stream(name: str, n: int | None = None) -> tuple[list[EdgeList], np.ndarray]:
    """Snapshots and X0 of a named streaming workload; `n` shrinks the node count."""
    spec = dict(STREAMS[name])
    idx = spec.pop("idx")
    parts = spec.pop("parts")
    if n is not None:
        spec["n"] = n
    seed = 2305 * 1000 + idx
    full = sbm(seed=seed, **spec)
    return edge_stream(full, parts, seed + 2), initial_block(full.n, full.n_blocks, seed + 1)


BATCHES = {
    # 32 independent SBMs of uneven size: N ~ U[2000, 100000], blocks k ~ U[8, 64], mean degree
    # ~ U[16, 48], within:between 5:1 (edge counts), block sizes +-20%
    "sbm_batch32": dict(count=32, n=(2000, 100_000), k=(8, 64), mean_degree=(16.0, 48.0), ratio=5.0, idx=6),
}


def batch(name: str, scale: float = 1.0) -> list[tuple[EdgeList, np.ndarray]]:
    """Edge lists and X0 of a named batch of graphs; `scale` shrinks every node count (at least
    4 nodes per block). The sizes are drawn from one generator, each graph from its own seed."""
    spec = BATCHES[name]
    base = 2305 * 1000 + spec["idx"]
    rng = rng_for(base)
    count = spec["count"]
    ns = rng.integers(spec["n"][0], spec["n"][1] + 1, size=count)
    ks = rng.integers(spec["k"][0], spec["k"][1] + 1, size=count)
    ds = rng.uniform(spec["mean_degree"][0], spec["mean_degree"][1], size=count)
    out = []
    for i in range(count):
        k = int(ks[i])
        n = max(4 * k, int(round(int(ns[i]) * scale)))
        seed = base * 100 + 2 * i
        g = sbm(n, k, float(ds[i]), spec["ratio"], ratio_kind="count", sizes="uniform", size_param=0.2,
                gamma=None, seed=seed)
        out.append((g, initial_block(n, k, seed + 1)))
    return out


def workload(name: str, n: int | None = None, seed_offset: int = 0) -> tuple[EdgeList, np.ndarray]:
    """Edge list and X0 for a named workload; `n` shrinks the node count (same recipe)."""
    spec = dict(WORKLOADS[name])
    idx = spec.pop("idx")
    if n is not None:
        spec["n"] = n
    seed = 2305 * 1000 + idx + seed_offset
    g = sbm(seed=seed, **spec)
    x0 = initial_block(g.n, g.n_blocks, seed + 1)
    return g, x0
