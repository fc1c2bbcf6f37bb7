"""GPU path (through the C ABI) against the FP64 oracle on seeded inputs.

Tolerances: graph build, degrees and D^-1/2 are bit-exact; f and grad f match within 1e-5
relative (the gradient also element by element, against 1e-5 max|grad f|); iterates after a few
updates match element by element within 1e-4 (FP32 state; 2e-3 with BF16 gather storage, one BF16
unit roundoff); converged features match within a principal angle of 1e-4 rad; K-means labels
reach ARI >= 0.99.

Algorithm 2 is chaotic over long runs: an FP32 trajectory and the FP64 one part after a few tens
of updates, and runs can fall into long two-cycles of one column's beta (the FP64 oracle does too,
from perturbed starts). So converged results are compared where a run converges, and strictly
(stop counts included) with the optional restart on both sides.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import ofsc_oracle as o
from paper_2305_10356_gb300 import build, ofsc, synth

from .gpu_util import assert_elementwise, csr_host, gpu_graph, run_iterate, upload

pytestmark = pytest.mark.gpu
METHODS = [o.OFM_F1, o.TRI_F1, o.OFM_F2, o.TRI_F2]


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    ofsc.lib()
    return torch


def edge_case_graph(weighted):
    rng = np.random.default_rng(3)
    n = 50
    src = rng.integers(0, n - 5, 300).astype(np.int32)  # nodes n-5.. n-1 isolated
    dst = rng.integers(0, n - 5, 300).astype(np.int32)
    src[:7] = dst[:7]
    src = np.concatenate([src, [2, 5, 5]]).astype(np.int32)
    dst = np.concatenate([dst, [5, 2, 2]]).astype(np.int32)
    w = rng.uniform(0.5, 1.5, src.size).astype(np.float32) if weighted else None
    return synth.EdgeList(n=n, src=src, dst=dst, w=w, labels=np.zeros(n, np.int32), n_blocks=1)


GRAPH_CASES = {
    "edge_cases_binary": lambda: edge_case_graph(False),
    "edge_cases_weighted": lambda: edge_case_graph(True),
    "sbm_n1000_k11": lambda: synth.workload("sbm_n1000_k11")[0],
    "wsbm_n20k_k32": lambda: synth.workload("wsbm_n20k_k32")[0],
    "dcsbm_n50k_k44": lambda: synth.workload("dcsbm_n50k_k44")[0],
    "empty": lambda: synth.EdgeList(n=7, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32),
                                    w=None, labels=np.zeros(7, np.int32), n_blocks=1),
}


@pytest.mark.parametrize("case", list(GRAPH_CASES))
def test_graph_build_bit_exact(case):
    e = GRAPH_CASES[case]()
    og = o.build_graph(e.n, e.src, e.dst, e.w)
    g = gpu_graph(e)
    h = csr_host(g)
    inf = g.info()
    np.testing.assert_array_equal(h["row_ptr"], og.row_ptr)
    np.testing.assert_array_equal(h["col"], og.col)
    if e.w is not None:
        assert h["val"].tobytes() == og.val.tobytes()
    else:
        assert h["val"] is None
    assert h["deg"].tobytes() == og.deg.tobytes()
    assert h["dinv"].tobytes() == og.s32.tobytes()
    assert inf.nnz == og.nnz and inf.n_selfloops == og.n_selfloops
    assert inf.n_isolated == og.n_isolated
    assert inf.n_duplicates == 2 * (e.m - og.n_selfloops) - og.nnz
    assert inf.normA_fro2 == pytest.approx(o.normA_fro2(og), rel=1e-12)


def test_graph_build_rejects_bad_input(cuda_lib):
    torch = cuda_lib
    src = torch.tensor([0, 1, 7], dtype=torch.int32, device="cuda")
    dst = torch.tensor([1, 2, 0], dtype=torch.int32, device="cuda")
    with pytest.raises(ofsc.OfscError) as ei:
        ofsc.ofsc_graph_build(5, src, dst)
    assert ei.value.status == ofsc.ERR_INVALID_ARG
    src = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    dst = torch.tensor([1, 2], dtype=torch.int32, device="cuda")
    for bad in (float("nan"), -1.0, 0.0, float("inf")):
        w = torch.tensor([1.0, bad], dtype=torch.float32, device="cuda")
        with pytest.raises(ofsc.OfscError) as ei:
            ofsc.ofsc_graph_build(5, src, dst, w)
        assert ei.value.status == ofsc.ERR_INVALID_ARG


OBJ_CASES = [("sbm_n1000_k11", None, None), ("dcsbm_n50k_k44", 8000, None), ("dcsbm_n50k_k44", None, None),
             ("wsbm_n20k_k32", 4000, None), ("dcsbm_n2m_k128", 3001, 128)]


@pytest.mark.parametrize("name,n,k", OBJ_CASES)
@pytest.mark.parametrize("which", [1, 2])
def test_objective_and_gradient(cuda_lib, name, n, k, which):
    torch = cuda_lib
    e, x0 = synth.workload(name, n=n)
    if k is not None:
        x0 = synth.initial_block(e.n, k, 77)
    og = o.build_graph(e.n, e.src, e.dst, e.w)
    g = gpu_graph(e)
    X = torch.from_numpy(x0).cuda()
    G = torch.empty_like(X)
    f = ofsc.ofsc_objective_grad(g, which, X, G)
    x64 = x0.astype(np.float64)
    AX = o.apply_A(og, x64)
    f_ref = o.objective(which, x64, AX, o.normA_fro2(og))
    G_ref = o.gradient(which, x64, AX)
    assert f == pytest.approx(f_ref, rel=1e-5)
    Gh = G.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(Gh - G_ref) <= 1e-5 * np.linalg.norm(G_ref)
    assert np.abs(Gh - G_ref).max() <= 1e-5 * np.abs(G_ref).max()


@pytest.fixture(scope="module")
def c1():
    e, x0 = synth.workload("sbm_n1000_k11")
    return e, x0, o.build_graph(e.n, e.src, e.dst, e.w)


@pytest.mark.parametrize("restart", [False, True])
@pytest.mark.parametrize("method", METHODS)
def test_first_updates_match_oracle(c1, method, restart):
    """Five updates of Algorithm 2 (and, with restart=True, of the optional restart on both
    sides): X element by element, alpha and beta per update."""
    e, x0, og = c1
    g = gpu_graph(e)
    steps = 5
    X, r, tr = run_iterate(g, method, x0, 0.0, steps, trace_cap=steps + 2, cg_restart=restart)
    ref = o.iterate(og, method, x0, 0.0, steps, restart=restart)
    assert r.iterations == steps == ref.iterations
    assert_elementwise(X, ref.X, 1e-4, "X_5")
    k = x0.shape[1]
    for t in range(steps):
        np.testing.assert_allclose(tr[t, 3:3 + k], ref.alphas[t], rtol=1e-4)
        np.testing.assert_allclose(tr[t, 3 + k:3 + 2 * k], ref.betas[t], rtol=1e-3, atol=1e-5)
        assert tr[t, 0] == t


def test_full_size_c3_in_the_bench_configuration():
    """C3 at full size (DC-SBM, N = 2,000,000, k = 128, 60.6M stored entries) in the launch
    configuration bench.py times (tensor-core Grams and direction pass, merge-path product, BF16
    gathers), against the FP64 oracle on the whole block, not on samples:
      - the graph's degrees and D^-1/2 bit for bit, and f1 and grad f1 at X0 (FP32 path, element by
        element within 1e-5 of max|G|);
      - one update of Algorithm 2 (OFM-f1), element by element within 2e-3 of max|X| (one BF16 unit
        roundoff), its step within 1e-3;
      - the merge-path product against whole rows on the same update: the same X within FP32
        rounding (they differ only in how the diag(V^T AV) partials are grouped)."""
    import torch
    e, x0 = synth.workload("dcsbm_n2m_k128")
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    h = csr_host(g)
    assert h["deg"].tobytes() == og.deg.tobytes() and h["dinv"].tobytes() == og.s32.tobytes()
    assert g.info().nnz == og.nnz >= (1 << 23)  # large enough for the merge-path default
    X = torch.from_numpy(x0).cuda()
    G = torch.empty_like(X)
    f = ofsc.ofsc_objective_grad(g, 1, X, G)
    x64 = x0.astype(np.float64)
    AX = o.apply_A(og, x64)
    assert f == pytest.approx(o.objective(1, x64, AX, o.normA_fro2(og)), rel=1e-5)
    G_ref = o.gradient(1, x64, AX)
    assert np.abs(G.cpu().numpy() - G_ref).max() <= 1e-5 * np.abs(G_ref).max()
    del G, AX, G_ref
    ref = o.iterate(og, o.OFM_F1, x0, 0.0, 1)
    Xb, rb, tb = run_iterate(g, o.OFM_F1, x0, 0.0, 1, trace_cap=2, gather=ofsc.GATHER_BF16)
    assert rb.iterations == 1
    assert_elementwise(Xb, ref.X, 2e-3, "BF16 update")
    np.testing.assert_allclose(tb[0, 3:3 + 128], ref.alphas[0], rtol=1e-3)
    Xm, _, _ = run_iterate(g, o.OFM_F1, x0, 0.0, 1, gather=ofsc.GATHER_BF16, merge_path=1)
    Xr, _, _ = run_iterate(g, o.OFM_F1, x0, 0.0, 1, gather=ofsc.GATHER_BF16, merge_path=-1)
    assert np.array_equal(Xm, Xb)  # the default at this size is the merge-path form
    assert np.linalg.norm(Xm - Xr) <= 1e-5 * np.linalg.norm(Xr)
    g.free()


@pytest.mark.parametrize("k,method,gather", [(44, o.OFM_F1, 0), (44, o.OFM_F2, 1), (72, o.OFM_F1, 1),
                                             (72, o.OFM_F2, 0), (128, o.OFM_F1, 0), (128, o.OFM_F2, 1)])
def test_converged_features_at_larger_k(k, method, gather):
    """Converged features at k = 44 (CUDA-core passes), 72 and 128 (tensor-core Grams and
    direction pass), FP32 and BF16 gathers (BF16 with the FP32 refinement sweep), against the
    oracle run to 1e-7: the GPU reaches tol 1e-5 and its features lie within 1e-4 rad of the
    oracle's, and K-means on both sides gives the same clusters (ARI >= 0.99), which are the
    planted blocks. The graphs are SBMs with k blocks of about 83 nodes, mean degree 30 and ten
    times as many edges inside blocks as between them, so the bottom-k eigenspace is well
    separated (the C2 recipe's 3:1 overlap leaves the oracle itself short of 1e-7 after 4,000
    updates)."""
    import torch
    e = synth.sbm(83 * k, k, 30.0, 10.0, ratio_kind="count", seed=260 + k)
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, k, 261)
    ref = o.iterate(og, method, x0, 1e-7, 3000)
    assert ref.converged
    X = torch.from_numpy(x0).cuda()
    r = ofsc.ofsc_iterate(g, method, X, 1e-5, 3000, gather=gather, refine_tol=1e-2 if gather else 0.0)
    assert r.status == ofsc.OK and r.rel_dir_norm <= 1e-5
    Xg = X.cpu().numpy()
    assert math.asin(min(1.0, o.subspace_sin(Xg, ref.X))) <= 1e-4
    ofsc.ofsc_row_normalize(X)
    labels = torch.empty(e.n, dtype=torch.int32, device="cuda")
    ofsc.ofsc_kmeans(X, e.n_blocks, labels, seed=5, n_init=3)
    lab = labels.cpu().numpy()
    lab_ref, _ = o.kmeans(o.row_normalize(ref.X), e.n_blocks, seed=5, n_init=3)
    assert o.ari(lab, lab_ref) >= 0.99
    assert o.ari(lab, e.labels) >= 0.99


@pytest.mark.parametrize("method,gather", [(o.OFM_F1, 0), (o.TRI_F1, 0), (o.OFM_F2, 1), (o.TRI_F2, 0)])
def test_cg_state_resumes_algorithm_2(c1, method, gather):
    """Eight updates run as 5 + 3 with the CG state carried between the calls are Algorithm 2 as
    one run: element by element against the oracle's eight updates, and within rounding of one
    8-update call (the second call evaluates G_5 from an exact AX, the single call from the
    recurrence). Resuming from a host checkpoint of the state gives the same bits; without the
    state the second call restarts from steepest descent and departs from Algorithm 2."""
    import torch
    e, x0, og = c1
    g = gpu_graph(e)
    k = x0.shape[1]
    rtol = 2e-3 if gather else 1e-4
    ref = o.iterate(og, method, x0, 0.0, 8)
    X1, _, _ = run_iterate(g, method, x0, 0.0, 8, gather=gather)
    st = ofsc.State(g, k)
    assert st.info()[0] == 0
    X = torch.from_numpy(x0).cuda()
    ra = ofsc.ofsc_iterate(g, method, X, 0.0, 5, gather=gather, state=st)
    assert ra.iterations == 5 and st.info()[0] == 5
    image = st.save()
    Xmid = X.clone()
    rb = ofsc.ofsc_iterate(g, method, X, 0.0, 3, gather=gather, state=st)
    assert rb.iterations == 3 and st.info()[0] == 8
    Xr = X.cpu().numpy()
    assert_elementwise(Xr, ref.X, rtol, "resumed")
    assert np.linalg.norm(Xr - X1) <= rtol * np.linalg.norm(X1)
    # the same run from the host checkpoint, in a new state object
    st2 = ofsc.State(g, k)
    st2.load(image)
    assert st2.info()[0] == 5
    X2 = Xmid.clone()
    ofsc.ofsc_iterate(g, method, X2, 0.0, 3, gather=gather, state=st2)
    assert np.array_equal(X2.cpu().numpy(), Xr)
    # no state: the second call restarts from steepest descent
    X3 = Xmid.clone()
    ofsc.ofsc_iterate(g, method, X3, 0.0, 3, gather=gather)
    d_resumed = np.linalg.norm(Xr - ref.X)
    d_restart = np.linalg.norm(X3.cpu().numpy() - ref.X)
    assert d_restart > 10 * d_resumed, (d_restart, d_resumed)


def test_cg_state_rules(c1):
    """A state is for one n, k and method; a call that stops early leaves it empty; checkpoints
    are checked; ofsc_iterate_batched takes none."""
    import torch
    e, x0, og = c1
    g = gpu_graph(e)
    k = x0.shape[1]
    st = ofsc.State(g, k)
    X = torch.from_numpy(x0).cuda()
    ofsc.ofsc_iterate(g, o.OFM_F1, X, 0.0, 4, state=st)
    assert st.info()[0] == 4
    with pytest.raises(ofsc.OfscError) as ei:  # another method
        ofsc.ofsc_iterate(g, o.TRI_F1, X.clone(), 0.0, 2, state=st)
    assert ei.value.status == ofsc.ERR_INVALID_ARG
    with pytest.raises(ofsc.OfscError) as ei:  # another k
        ofsc.ofsc_iterate(g, o.OFM_F1, torch.from_numpy(x0[:, :k - 3].copy()).cuda(), 0.0, 2, state=st)
    assert ei.value.status == ofsc.ERR_INVALID_ARG
    with pytest.raises(ofsc.OfscError) as ei:
        ofsc.ofsc_iterate_batched([g], o.OFM_F1, [X.clone()], 0.0, 2, state=st)
    assert ei.value.status == ofsc.ERR_INVALID_ARG
    image = st.save()
    with pytest.raises(ofsc.OfscError) as ei:  # a damaged header
        st.load(b"x" * len(image))
    assert ei.value.status == ofsc.ERR_INVALID_ARG
    assert st.info()[0] == 4
    r = ofsc.ofsc_iterate(g, o.OFM_F1, X, 1e-1, 400, state=st)  # stops on tol: the state is emptied
    assert r.status == ofsc.OK and st.info()[0] == 0


def column_match(X, ref):
    """Columns equal up to sign (TriOFM fixed points are unique up to D = diag(+-1))."""
    s = np.sign(np.sum(X * ref, axis=0))
    return np.linalg.norm(X * s - ref) / np.linalg.norm(ref)


def check_features(e, method, X, ref, tol):
    """Converged GPU features against the oracle's: principal angle, TriOFM columns, Algorithm 1
    steps 3-4 on both sides (ARI against the oracle's labels and against the planted blocks)."""
    import torch
    sin = o.subspace_sin(X, ref.X)
    assert math.asin(min(1.0, sin)) <= 1e-4
    if method in (o.TRI_F1, o.TRI_F2):
        assert column_match(X.astype(np.float64), ref.X) <= 1e-4
    Xd = torch.from_numpy(X).cuda()
    ofsc.ofsc_row_normalize(Xd)
    labels = torch.empty(e.n, dtype=torch.int32, device="cuda")
    ofsc.ofsc_kmeans(Xd, e.n_blocks, labels, seed=5, n_init=3)
    lab_gpu = labels.cpu().numpy()
    lab_ref, _ = o.kmeans(o.row_normalize(ref.X), e.n_blocks, seed=5, n_init=3)
    assert o.ari(lab_gpu, lab_ref) >= 0.99
    assert o.ari(lab_gpu, e.labels) >= 0.9  # the planted blocks are recovered


@pytest.mark.parametrize("method", METHODS)
def test_converged_with_matching_restart(c1, method):
    """The 1,000-node case to tol 1e-6 (2,000 updates at most) with the optional restart on both
    sides: both converge, the GPU's returned relative direction norm meets tol (only exact updates
    stop a run), the stop counts agree within 50% (the FP32 and FP64 trajectories part after a few
    tens of updates), and the features and clusters agree."""
    e, x0, og = c1
    g = gpu_graph(e)
    X, r, _ = run_iterate(g, method, x0, 1e-6, 2000, cg_restart=True)
    ref = o.iterate(og, method, x0, 1e-6, 2000, restart=True)
    assert ref.converged
    assert r.status == ofsc.OK, (r.status, r.iterations, r.rel_dir_norm)
    assert r.rel_dir_norm <= 1e-6
    assert abs(r.iterations - ref.iterations) <= max(10, 0.5 * ref.iterations), (r.iterations, ref.iterations)
    check_features(e, method, X, ref, 1e-6)


PRECISIONS = {"fp32": {}, "bf16": {"gather": ofsc.GATHER_BF16},
              "bf16_refined": {"gather": ofsc.GATHER_BF16, "refine_tol": 1e-3}}


def test_converged_features_and_clusters(c1):
    """Algorithm 2 as printed (no restart) on the 1,000-node case, tol 1e-6, 2,000 updates at most,
    for every method in FP32, with BF16 gather storage, and BF16 with the FP32 refinement sweep. The
    oracle converges for every method. Every GPU run that reports convergence returns a relative
    direction norm <= tol and the oracle's features and clusters, within [1/2, 2] of its stop count
    (the trajectories part after a few tens of updates); a run that does not converge ends
    NOT_CONVERGED or NONFINITE. From this start OFM-f1 falls into a long two-cycle of one column's
    beta (the FP64 oracle does so too from perturbed starts, for up to 1,300 updates), so the test
    asks that at least 8 of the 12 runs converge."""
    e, x0, og = c1
    g = gpu_graph(e)
    converged = 0
    for method in METHODS:
        ref = o.iterate(og, method, x0, 1e-6, 2000)
        assert ref.converged
        for name, kw in PRECISIONS.items():
            try:
                X, r, _ = run_iterate(g, method, x0, 1e-6, 2000, **kw)
            except ofsc.OfscError as ex:
                assert ex.status == ofsc.ERR_NONFINITE, (method, name, ex)
                continue
            if r.status != ofsc.OK:
                assert r.status == ofsc.ERR_NOT_CONVERGED and r.iterations == 2000, (method, name, r.status)
                continue
            converged += 1
            assert r.rel_dir_norm <= 1e-6, (method, name)
            assert 0.5 * ref.iterations <= r.iterations <= 2 * ref.iterations, (method, name, r.iterations,
                                                                                ref.iterations)
            if name == "bf16_refined":
                assert 0 < r.refined_at <= r.iterations
            check_features(e, method, X, ref, 1e-6)
    assert converged >= 8, converged


@pytest.mark.parametrize("method", METHODS)
def test_single_call_replay_equals_direct_launches(c1, method):
    """ofsc_iterate replays its repeating updates from a captured CUDA graph by default; with
    direct_launch it launches every kernel itself. Both give the same bits of X, of the trace and of
    the result on the 1,000-node case run to tol 1e-6 (host checks, exact refreshes, the exact update
    scheduled once tol is met on a recurrence update)."""
    e, x0, _ = c1
    g = gpu_graph(e)
    Xa, ra, ta = run_iterate(g, method, x0, 1e-6, 600, trace_cap=601)
    Xb, rb, tb = run_iterate(g, method, x0, 1e-6, 600, trace_cap=601, direct_launch=True)
    assert np.array_equal(Xa, Xb) and np.array_equal(ta, tb)
    assert (ra.iterations, ra.status, ra.rel_dir_norm, ra.f) == (rb.iterations, rb.status, rb.rel_dir_norm, rb.f)


def test_allocator_hook_and_oom_injection():
    """ofsc_set_allocator: every device block of the library comes from the caller's allocator (here
    torch's caching allocator). One that refuses past a byte budget makes ofsc_graph_build and then
    ofsc_iterate return OFSC_ERR_OOM with every block they had taken given back; with room again the
    same calls run and give the bits they give on cudaMalloc; freeing the graph returns the rest."""
    import torch
    e = synth.sbm(3000, 6, 20.0, 6.0, ratio_kind="count", seed=161)
    x0 = synth.initial_block(e.n, 16, 162)
    X_ref, r_ref, _ = run_iterate(gpu_graph(e), o.OFM_F1, x0, 0.0, 8)
    live, budget = {}, [1 << 14]

    def alloc(nbytes):
        if sum(live.values()) + nbytes > budget[0]:
            return 0
        p = torch.cuda.caching_allocator_alloc(nbytes)
        live[p] = nbytes
        return p

    def free(p):
        del live[p]
        torch.cuda.caching_allocator_delete(p)

    try:
        ofsc.ofsc_set_allocator(alloc, free)
        with pytest.raises(ofsc.OfscError) as ei:
            gpu_graph(e)
        assert ei.value.status == ofsc.ERR_OOM and not live
        budget[0] = 1 << 30
        g = gpu_graph(e)
        held = sum(live.values())
        assert held > 0
        budget[0] = held + 4096  # too little for the iteration's workspace
        with pytest.raises(ofsc.OfscError) as ei:
            run_iterate(g, o.OFM_F1, x0, 0.0, 8)
        assert ei.value.status == ofsc.ERR_OOM and sum(live.values()) == held
        budget[0] = 1 << 30
        X, r, _ = run_iterate(g, o.OFM_F1, x0, 0.0, 8)
        assert np.array_equal(X, X_ref) and r.f == r_ref.f
        g.free()
        assert not live
    finally:
        ofsc.ofsc_set_allocator()


def test_bounded_wait_runs_out_and_the_next_call_succeeds():
    """Failure detection without a fault: with the test hook that makes the tensor-core direction
    pass's converter warps withhold their arrivals and a short spin limit, the MMA warp's first
    bounded wait runs out before any MMA is issued (the pass has no TMA copies), the kernel records
    OFSC_ERR_TIMEOUT, frees its tensor memory and returns, and the call reports the status. The next
    normal call on the same handle then runs and matches the oracle."""
    e = synth.sbm(3001, 9, 22.0, 6.0, seed=81, gamma=2.4, ratio_kind="count")
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, 128, 82)
    with pytest.raises(ofsc.OfscError) as ei:
        run_iterate(g, o.OFM_F1, x0, 0.0, 3, withhold_arrivals=True, spin_limit=1 << 12,
                    gram_engine=ofsc.GRAM_TC, direct_launch=True)
    assert ei.value.status == ofsc.ERR_TIMEOUT
    X, r, _ = run_iterate(g, o.OFM_F1, x0, 0.0, 3, gram_engine=ofsc.GRAM_TC)
    assert r.iterations == 3 and r.status == ofsc.ERR_NOT_CONVERGED
    ref = o.iterate(og, o.OFM_F1, x0, 0.0, 3)
    assert_elementwise(X, ref.X, 1e-4)


@pytest.mark.parametrize("method", METHODS)
def test_column_scales_leave_the_bits_unchanged(method):
    """The stored direction V diag(1/s) with power-of-two column scales s: forcing scales of about
    2^30 from the first update on (vscale_exp = -30) gives the same bits of X and of every alpha and
    beta as the default (scales 1 here), at k = 11 (CUDA-core Grams) and k = 128 (tensor cores)."""
    for n, k, seed in ((1000, 11, 3), (3001, 128, 4)):
        e = synth.sbm(n, 8, 20.0, 6.0, ratio_kind="count", seed=150 + seed)
        g = gpu_graph(e)
        x0 = synth.initial_block(e.n, k, 151 + seed)
        for gather in (ofsc.GATHER_FP32, ofsc.GATHER_BF16):
            Xa, ra, ta = run_iterate(g, method, x0, 0.0, 40, trace_cap=41, gather=gather)
            Xb, rb, tb = run_iterate(g, method, x0, 0.0, 40, trace_cap=41, gather=gather, vscale_exp=-30)
            assert np.array_equal(Xa, Xb) and np.array_equal(ta, tb), (n, k, gather)
            assert ra.rel_dir_norm == rb.rel_dir_norm


BF16_CASES = [("sbm_n1000_k11", None, None), ("dcsbm_n50k_k44", 8000, None), ("dcsbm_n50k_k44", None, None),
              ("dcsbm_n2m_k128", 4000, 128)]


@pytest.mark.parametrize("name,n,k", BF16_CASES)
@pytest.mark.parametrize("method", METHODS)
def test_bf16_first_updates_match_oracle(name, n, k, method):
    """BF16 gather storage of D^-1/2 V (FP32 master copy and accumulation; at k = 128 the bench's
    16-lane, 8-values-per-lane instantiation of the direction product) against the FP64 oracle,
    element by element after 5 updates, at k = 11, 44 and 128. Tolerance 2e-3 of max|X|, one BF16
    unit roundoff (2^-9): every gathered value carries one BF16 rounding, which enters A V and the
    line-search coefficients at that relative size; alpha within 1e-2 relative."""
    e, x0 = synth.workload(name, n=n)
    if k is not None:
        x0 = synth.initial_block(e.n, k, 77)
    og = o.build_graph(e.n, e.src, e.dst, e.w)
    g = gpu_graph(e)
    X, r, tr = run_iterate(g, method, x0, 0.0, 5, trace_cap=6, gather=ofsc.GATHER_BF16)
    ref = o.iterate(og, method, x0, 0.0, 5)
    assert r.iterations == 5 == ref.iterations
    assert_elementwise(X, ref.X, 2e-3, "X_5 with BF16 gathers")
    kk = x0.shape[1]
    np.testing.assert_allclose(tr[:5, 3:3 + kk], np.array(ref.alphas), rtol=1e-2)


@pytest.mark.parametrize("k", [1, 8, 128])
def test_widths(k):
    e = synth.sbm(700, 5, 14.0, 8.0, seed=40 + k)
    x0 = synth.initial_block(e.n, k, 41)
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    for method in (o.OFM_F2, o.TRI_F1):
        X, r, _ = run_iterate(g, method, x0, 0.0, 4)
        ref = o.iterate(og, method, x0, 0.0, 4)
        assert_elementwise(X, ref.X, 1e-4)


def test_degenerate_inputs(cuda_lib):
    torch = cuda_lib
    e = edge_case_graph(False)  # isolated nodes, loops, duplicates
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, 3, 2)
    X, r, _ = run_iterate(g, o.OFM_F1, x0, 0.0, 6)
    ref = o.iterate(og, o.OFM_F1, x0, 0.0, 6)
    assert_elementwise(X, ref.X, 1e-4)
    # X0 = 0 is stationary: no update, status OK
    Xz, r, _ = run_iterate(g, o.OFM_F1, np.zeros((e.n, 3), np.float32), 1e-6, 10)
    assert r.iterations == 0 and r.status == ofsc.OK and np.all(Xz == 0)
    # maxit = 0 leaves X0 untouched
    X0b, r, _ = run_iterate(g, o.TRI_F2, x0, 1e-6, 0)
    assert r.iterations == 0 and np.array_equal(X0b, x0)
    # non-finite start is rejected
    bad = x0.copy()
    bad[3, 1] = np.nan
    with pytest.raises(ofsc.OfscError) as ei:
        run_iterate(g, o.OFM_F1, bad, 1e-6, 5)
    assert ei.value.status == ofsc.ERR_NONFINITE
    # invalid arguments
    Xd = torch.from_numpy(x0).cuda()
    for method, maxit in ((7, 3), (-1, 3), (0, -1)):
        with pytest.raises(ofsc.OfscError) as ei:
            ofsc.ofsc_iterate(g, method, Xd, 0.0, maxit)
        assert ei.value.status == ofsc.ERR_INVALID_ARG
    with pytest.raises(ofsc.OfscError):
        ofsc.ofsc_iterate(g, 0, torch.zeros((e.n, 129), device="cuda"), 0.0, 1)
    # empty graph: every node isolated, A = -I
    ge = gpu_graph(GRAPH_CASES["empty"]())
    x7 = synth.initial_block(7, 2, 3)
    f = ofsc.ofsc_objective_grad(ge, 1, torch.from_numpy(x7).cuda())
    xx = x7.astype(np.float64)
    assert f == pytest.approx(o.objective_dense(1, -np.eye(7), xx), rel=1e-6)


def test_row_normalize_matches(cuda_lib):
    torch = cuda_lib
    x = synth.initial_block(1000, 11, 9)
    x[5] = 0.0
    X = torch.from_numpy(x).cuda()
    ofsc.ofsc_row_normalize(X)
    np.testing.assert_allclose(X.cpu().numpy(), o.row_normalize(x), rtol=2e-6, atol=1e-7)


def test_kmeans_matches_oracle(cuda_lib):
    torch = cuda_lib
    rng = np.random.default_rng(8)
    centers = rng.standard_normal((7, 5)) * 6
    truth = rng.integers(0, 7, 3000)
    x = (centers[truth] + rng.standard_normal((3000, 5)) * 0.5).astype(np.float32)
    X = torch.from_numpy(x).cuda()
    lab = torch.empty(3000, dtype=torch.int32, device="cuda")
    inertia = ofsc.ofsc_kmeans(X, 7, lab, seed=42, n_init=2)
    lg = lab.cpu().numpy()
    lr, ir = o.kmeans(x, 7, seed=42, n_init=2)
    assert o.ari(lg, lr) == 1.0 and o.ari(lg, truth) >= 0.99
    assert inertia == pytest.approx(ir, rel=1e-4)
    # a Lloyd fixed point checked in FP64 on the host
    xd = x.astype(np.float64)
    mu = np.stack([xd[lg == c].mean(axis=0) for c in range(7)])
    d = ((xd[:, None, :] - mu[None]) ** 2).sum(-1)
    assert np.mean(np.argmin(d, axis=1) == lg) >= 0.999
    lab2 = torch.empty_like(lab)
    ofsc.ofsc_kmeans(X, 7, lab2, seed=42, n_init=2)
    assert torch.equal(lab, lab2)  # deterministic given the seed


@pytest.mark.parametrize("n,k,ld,nr,lslot", [
    (100, 128, 128, 2, 1),        # warp-specialised TMA kernel: one CTA, ragged 32-row chunk
    (300_001, 128, 128, 2, 0),    # ... several accumulator segments per CTA
    (4_999, 100, 104, 1, 0),      # ... one block, features 100..127 zero-filled
    (150_001, 128, 128, 2, None), # ... two right blocks, the left block staged on its own
    (4_999, 100, 104, 2, None),   # ... the same with features 100..127 zero-filled
    (10_001, 128, 128, 4, 1),     # per-CTA kernel: four right blocks
    (3_333, 100, 104, 3, None),   # ... left block separate from the right blocks
    (777, 20, 24, 1, None)])
def test_tensor_core_gram_matches_fp64(cuda_lib, n, k, ld, nr, lslot):
    """ofsc_gram (tcgen05, 3-term TF32, FP32 tensor-memory accumulation) against FP64 numpy."""
    torch = cuda_lib
    rng = np.random.default_rng(n + k)
    L = (rng.standard_normal((n, ld)) / np.sqrt(n)).astype(np.float32)
    Rs = [L if b == lslot else (rng.standard_normal((n, ld)) / np.sqrt(n)).astype(np.float32)
          for b in range(nr)]
    Ld = torch.from_numpy(L).cuda()
    Rd = [Ld if b == lslot else torch.from_numpy(R).cuda() for b, R in enumerate(Rs)]
    out = torch.zeros((nr, k, k), dtype=torch.float64, device="cuda")
    ofsc.ofsc_gram(Ld, Rd, out, k=k)
    got = out.cpu().numpy()
    for b in range(nr):
        ref = L[:, :k].astype(np.float64).T @ Rs[b][:, :k].astype(np.float64)
        assert np.linalg.norm(got[b] - ref) <= 1e-5 * np.linalg.norm(ref)
        assert np.abs(got[b] - ref).max() <= 1e-5 * np.abs(ref).max()


def test_tensor_core_and_cuda_core_iterations_agree(cuda_lib):
    """k = 128: the iteration with tensor-core Grams tracks the FP32 CUDA-core one."""
    e = synth.sbm(4000, 8, 16.0, 8.0, seed=77)
    x0 = synth.initial_block(e.n, 128, 78)
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    for method in METHODS:
        Xs, rs, _ = run_iterate(g, method, x0, 0.0, 6, gram_engine=ofsc.GRAM_SIMT)
        Xt, rt, _ = run_iterate(g, method, x0, 0.0, 6, gram_engine=ofsc.GRAM_TC)
        ref = o.iterate(og, method, x0, 0.0, 6)
        # the TriOFM prefix cubics of the trailing columns sum over 120+ columns, which amplifies
        # FP32 rounding there to about 1e-3 of the block's scale after 6 updates
        for Xg in (Xt, Xs):
            assert np.linalg.norm(Xg - ref.X) <= 1e-4 * np.linalg.norm(ref.X)
            assert_elementwise(Xg, ref.X, 1e-3)


@pytest.mark.parametrize("k", [64, 128])
@pytest.mark.parametrize("gather", [0, 1])
def test_tma_gather_spmm_agrees(k, gather):
    """The TMA tile::gather4 sparse product gives the CUDA-core one's iterates (and the oracle's)."""
    e = synth.sbm(3000, 6, 24.0, 6.0, seed=90 + k, gamma=2.5, ratio_kind="count")
    x0 = synth.initial_block(e.n, k, 91)
    g = gpu_graph(e)
    Xs, _, trs = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, gather=gather, spmm_engine=ofsc.SPMM_SIMT)
    Xt, _, trt = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, gather=gather, spmm_engine=ofsc.SPMM_TMA)
    assert np.linalg.norm(Xt - Xs) <= 2e-5 * np.linalg.norm(Xs)
    np.testing.assert_allclose(trt[:5, 3], trs[:5, 3], rtol=1e-4)
    if gather == 0:
        og = o.build_graph(e.n, e.src, e.dst)
        ref = o.iterate(og, o.OFM_F1, x0, 0.0, 5)
        assert_elementwise(Xt, ref.X, 1e-4)



@pytest.mark.parametrize("k", [3, 12, 20, 44, 100])
def test_direction_product_all_lane_widths_weighted(k):
    """The warp-per-row direction product at every lane width (padded k 8 to 104: 2 to 32 lanes per
    nonzero, 16 to 1 nonzeros side by side), on a weighted graph with hub rows longer than a step
    and isolated (empty) rows, against the oracle's updates."""
    e = synth.sbm(2500, 5, 18.0, 5.0, seed=60 + k, gamma=2.2, ratio_kind="count", weighted=True)
    # 20 trailing nodes without edges: empty rows, also at the end of the last warp's range
    e = dataclasses.replace(e, n=e.n + 20, labels=np.concatenate([e.labels, np.zeros(20, np.int32)]))
    og = o.build_graph(e.n, e.src, e.dst, e.w)
    assert (og.deg[-20:] == 0).all() and np.diff(og.row_ptr).max() > 64
    x0 = synth.initial_block(e.n, k, 61)
    g = gpu_graph(e)
    X, r, tr = run_iterate(g, o.OFM_F2, x0, 0.0, 4, trace_cap=5)
    ref = o.iterate(og, o.OFM_F2, x0, 0.0, 4)
    assert_elementwise(X, ref.X, 1e-4)
    np.testing.assert_allclose(tr[:4, 3:3 + k], np.array(ref.alphas[:4]), rtol=1e-4, atol=1e-7)


def hub_graph(weighted, seed):
    """An SBM of 6,000 nodes with one hub joined to 4,000 random nodes: the hub's row holds about
    30 times a warp's share of the nonzeros (608 warps for about 80,000 stored entries)."""
    e = synth.sbm(6000, 6, 12.0, 6.0, ratio_kind="count", weighted=weighted, seed=seed)
    rng = np.random.default_rng(seed + 1)
    leaves = rng.choice(np.arange(1, e.n), 4000, replace=False).astype(np.int32)
    src = np.concatenate([e.src, np.zeros(4000, np.int32)])
    dst = np.concatenate([e.dst, leaves])
    w = None if e.w is None else np.concatenate([e.w, rng.uniform(0.5, 1.5, 4000).astype(np.float32)])
    return dataclasses.replace(e, src=src, dst=dst, w=w)


@pytest.mark.parametrize("k,gather,weighted", [(20, 0, True), (44, 0, False), (128, 1, False), (128, 0, True)])
def test_merge_path_splits_hub_rows(k, gather, weighted):
    """The direction product on merge-path shares (a long row spans several warps; their partial
    sums are added in warp order by the fixup): on a graph with a hub row of 4,000 nonzeros the first
    five updates match the oracle element by element (chosen automatically and forced), agree with
    the whole-row partition within FP32 rounding, repeat bit for bit, and the objective and gradient
    on the same graph match the oracle."""
    import torch
    e = hub_graph(weighted, 170 + k)
    og = o.build_graph(e.n, e.src, e.dst, e.w)
    assert og.row_ptr[1] - og.row_ptr[0] >= 4000
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, k, 171)
    ref = o.iterate(og, o.OFM_F1, x0, 0.0, 5)
    rtol = 2e-3 if gather else 1e-4
    # At k = 128 the default engines are the tensor cores' (3-term TF32 Grams and direction pass).
    # On this graph their rounding (the first step within 3e-6 of the oracle's, against 2e-8 on
    # the CUDA cores) grows to a few 1e-4 in one column's step by the fifth update, beyond the
    # 1e-4 element bound; so the three forms meet the oracle on the CUDA-core engines, and on the
    # default engines they agree with each other and with the oracle's first step.
    eng = dict(gram_engine=ofsc.GRAM_SIMT) if k > 64 and not gather else {}
    Xa, ra, ta = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, gather=gather, **eng)             # automatic
    Xm, rm, tm = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, gather=gather, merge_path=1, **eng)
    Xr, rr, tr = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, gather=gather, merge_path=-1, **eng)
    Xm2, _, tm2 = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, gather=gather, merge_path=1, **eng)
    for name, X in (("automatic", Xa), ("merge path", Xm), ("whole rows", Xr)):
        assert_elementwise(X, ref.X, rtol, name)
    assert np.array_equal(Xa, Xm) and np.array_equal(ta, tm)  # the hub makes the automatic choice merge path
    assert np.array_equal(Xm, Xm2) and np.array_equal(tm, tm2)
    assert np.linalg.norm(Xm - Xr) <= (1e-3 if gather else 1e-5) * np.linalg.norm(Xr)
    if eng:
        Xmt, _, tmt = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, merge_path=1)
        Xrt, _, _ = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, merge_path=-1)
        np.testing.assert_allclose(tmt[0, 3:3 + k], ref.alphas[0], rtol=1e-5)
        assert np.linalg.norm(Xmt - Xrt) <= 1e-5 * np.linalg.norm(Xrt)
        assert np.linalg.norm(Xmt - ref.X) <= 1e-4 * np.linalg.norm(ref.X)
    X = torch.from_numpy(x0).cuda()
    G = torch.empty_like(X)
    f = ofsc.ofsc_objective_grad(g, 1, X, G)
    x64 = x0.astype(np.float64)
    AX = o.apply_A(og, x64)
    assert f == pytest.approx(o.objective(1, x64, AX, o.normA_fro2(og)), rel=1e-5)
    G_ref = o.gradient(1, x64, AX)
    assert np.abs(G.cpu().numpy() - G_ref).max() <= 1e-5 * np.abs(G_ref).max()


@pytest.mark.parametrize("k", [20, 64])
def test_forced_tensor_core_grams_at_small_k(k):
    """gram_engine = OFSC_GRAM_TC below k = 64, where the workspace does not hold the tensor-core
    Gram partials until a call asks for them: five updates match the oracle element by element and
    the CUDA-core Grams within FP32 rounding, and a following default call is unaffected."""
    e = synth.sbm(5000, 6, 16.0, 5.0, ratio_kind="count", seed=200 + k)
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, k, 201)
    ref = o.iterate(og, o.OFM_F1, x0, 0.0, 5)
    Xs, rs, ts = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6)  # the default (CUDA-core) Grams
    Xt, rt, tt = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, gram_engine=ofsc.GRAM_TC)
    Xs2, rs2, ts2 = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6)
    assert rt.status == ofsc.ERR_NOT_CONVERGED and rt.iterations == 5
    assert_elementwise(Xt, ref.X, 1e-4, "tensor-core Grams")
    assert np.linalg.norm(Xt - Xs) <= 1e-5 * np.linalg.norm(Xs)
    assert np.array_equal(Xs, Xs2) and np.array_equal(ts, ts2)


@pytest.mark.parametrize("k,gather", [(32, 0), (128, 1)])
def test_autotune_times_the_merge_path_split(k, gather):
    """ofsc_autotune also times the merge-path split at every row partition (which reallocates and
    recomputes the warps' shares with the partition); later calls with merge_path = 0 take its
    choice: the result repeats bit for bit the run that forces that form, and matches the oracle
    element by element."""
    e = hub_graph(False, 190 + k)
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, k, 191)
    ref = o.iterate(og, o.OFM_F1, x0, 0.0, 5)
    w, u, mp, ms = ofsc.ofsc_autotune(g, k, gather, with_merge=True)
    assert w in [m * 152 for m in (4, 8, 16, 32)] and ms > 0.0
    Xa, _, ta = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, gather=gather)
    Xf, _, tf = run_iterate(g, o.OFM_F1, x0, 0.0, 5, trace_cap=6, gather=gather, merge_path=1 if mp else -1)
    assert np.array_equal(Xa, Xf) and np.array_equal(ta, tf)
    assert_elementwise(Xa, ref.X, 2e-3 if gather else 1e-4)
    # the other form on the tuned partition agrees within rounding
    Xo, _, _ = run_iterate(g, o.OFM_F1, x0, 0.0, 5, gather=gather, merge_path=-1 if mp else 1)
    assert np.linalg.norm(Xo - Xa) <= (1e-3 if gather else 1e-5) * np.linalg.norm(Xa)


@pytest.mark.parametrize("gather,k", [(0, 64), (1, 64), (0, 128)])
def test_iterations_are_bitwise_repeatable(gather, k):
    """Every reduction has a fixed shape (per-block partials summed in block order, no atomics), so
    two runs from the same X0 give the same bits (k = 128: tensor-core direction pass and Grams)."""
    e = synth.sbm(4000, 8, 24.0, 6.0, seed=71, gamma=2.4, ratio_kind="count")
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, k, 72)
    X1, r1, t1 = run_iterate(g, o.OFM_F1, x0, 0.0, 12, trace_cap=13, gather=gather)
    X2, r2, t2 = run_iterate(g, o.OFM_F1, x0, 0.0, 12, trace_cap=13, gather=gather)
    assert np.array_equal(X1, X2)
    assert np.array_equal(t1, t2)
    assert r1.rel_dir_norm == r2.rel_dir_norm


@pytest.mark.parametrize("method", METHODS)
def test_tensor_core_direction_pass(method):
    """k = 128: the direction pass on the tensor cores (3-term tf32; X_new R for the f1 methods,
    X_new B + AX_new R with the B operands streamed per K chunk for the f2 methods) against the
    CUDA-core pass and against the oracle, on 3001 rows (a ragged last 128-row tile)."""
    e = synth.sbm(3001, 9, 22.0, 6.0, seed=81, gamma=2.4, ratio_kind="count")
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, 128, 82)
    Xt, rt, tt = run_iterate(g, method, x0, 0.0, 6, trace_cap=7, gram_engine=ofsc.GRAM_TC)
    Xs, rs, ts = run_iterate(g, method, x0, 0.0, 6, trace_cap=7, gram_engine=ofsc.GRAM_SIMT)
    assert np.linalg.norm(Xt - Xs) <= 1e-5 * np.linalg.norm(Xs)
    # TriOFM's step for column i solves the prefix cubic over columns 1..i, which amplifies the
    # FP32-level difference of the two Gram engines to a few 1e-3 in some trailing columns' steps
    np.testing.assert_allclose(tt[:6, 3:3 + 128], ts[:6, 3:3 + 128], rtol=1e-4 if method == o.OFM_F1 else 5e-3,
                               atol=1e-7)
    ref = o.iterate(og, method, x0, 0.0, 6)
    assert np.linalg.norm(Xt - ref.X) <= 1e-4 * np.linalg.norm(ref.X)
    assert_elementwise(Xt, ref.X, 1e-3)
    assert abs(rt.rel_dir_norm - ref.rel_norms[-1]) <= 1e-4 * ref.rel_norms[-1] + 1e-7


def test_streaming_snapshots_warm_start_match_oracle():
    """The streaming form: five cumulative edge-sampled snapshots, a new graph per snapshot and X
    carried from one snapshot's iterations into the next (CG restarted from G of the new graph);
    every snapshot's X matches the oracle doing the same, and on the last snapshot the warm start
    reaches the tolerance in fewer updates than a cold start."""
    full = synth.sbm(3000, 6, 24.0, 5.0, ratio_kind="count", join_isolated=False, seed=91)
    snaps = synth.edge_stream(full, 5, seed=92)
    x0 = synth.initial_block(full.n, 6, 93)
    Xg, Xo = x0.copy(), x0.copy()
    for e in snaps:
        g = gpu_graph(e)
        Xg, r, _ = run_iterate(g, o.OFM_F1, Xg, 0.0, 8)
        ref = o.iterate(o.build_graph(e.n, e.src, e.dst), o.OFM_F1, Xo, 0.0, 8)
        Xo = ref.X
        assert_elementwise(Xg, Xo, 1e-4)
    g = gpu_graph(snaps[-1])
    # to tolerance with the optional restart: without it OFM-f1 can sit in a long two-cycle of one
    # column's beta, which says nothing about the warm start (the paper runs 2 updates a snapshot)
    _, warm, _ = run_iterate(g, o.OFM_F1, Xg, 1e-4, 2000, cg_restart=True)
    _, cold, _ = run_iterate(g, o.OFM_F1, x0, 1e-4, 2000, cg_restart=True)
    assert warm.status == ofsc.OK and cold.status == ofsc.OK
    assert warm.iterations < cold.iterations


@pytest.mark.parametrize("gather,rtol", [(ofsc.GATHER_FP32, 1e-4), (ofsc.GATHER_BF16, 5e-3)])
def test_streaming_full_size_in_the_bench_configuration(gather, rtol):
    """The stream of bench.py --workload sbm_stream_n200k_k71 at full size (200,000 nodes, k = 71,
    cumulative edge-sampled snapshots; the bench's BF16 gathers, and FP32), its first three
    snapshots with X carried from each into the next, five updates each: every snapshot against the
    oracle started from the same X (the GPU's X after the previous snapshot), element by element.
    FP32 within 1e-4. BF16 within 5e-3 of max|X|: the first snapshot holds 10% of the edges, about
    three neighbours a node, so a row's A V carries its few gathered values' BF16 rounding (2^-9)
    unaveraged, and five line-searched updates compound it to about two units (measured 1.9e-4
    against max|X| = 0.048 in 51 of 14.2M entries)."""
    import torch
    snaps, x0 = synth.stream("sbm_stream_n200k_k71")
    X = torch.from_numpy(x0).cuda()
    for e in snaps[:3]:
        g = gpu_graph(e)
        x_in = X.cpu().numpy()
        r = ofsc.ofsc_iterate(g, o.OFM_F1, X, 0.0, 5, gather=gather)
        assert r.iterations == 5
        ref = o.iterate(o.build_graph(e.n, e.src, e.dst), o.OFM_F1, x_in, 0.0, 5)
        assert_elementwise(X.cpu().numpy(), ref.X, rtol, f"snapshot with {e.src.size} listed edges")
        g.free()


def test_unrolled_grad_full_size():
    """The unrolled gradient on C5 at full size (weighted SBM, 20,000 nodes, k = 32, the graph of
    bench.py --workload wsbm_n20k_k32 --unrolled 20), through T = 5 updates with checkpoints every
    5 (the launches of every update are those of T = 20; five line-searched updates keep the
    gradient well conditioned): f1(X_T) within 1e-5, d/dX_0 and d/dw within 1e-3 (norm) of the
    oracle's reverse sweep, and every weight-gradient entry within 1e-3 of the largest."""
    import torch
    e, x0 = synth.workload("wsbm_n20k_k32")
    og = o.build_graph(e.n, e.src, e.dst, e.w.astype(np.float64), exact=True)
    g = gpu_graph(e)
    T = 5
    f_ref, g_ref, w_ref = o.unrolled_grad(og, x0.astype(np.float64), T, edges=(e.src, e.dst, e.w.astype(np.float64)))
    X0 = torch.from_numpy(x0).cuda()
    src, dst, _ = upload(e)
    grad = torch.empty_like(X0)
    gw = torch.full((e.src.size,), float("nan"), dtype=torch.float32, device="cuda")
    f = ofsc.ofsc_unrolled_grad(g, X0, T, grad, ckpt=5, src=src, dst=dst, grad_w=gw)
    G, W = grad.cpu().numpy(), gw.cpu().numpy()
    assert abs(f - f_ref) <= 1e-5 * abs(f_ref)
    assert np.linalg.norm(G - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
    assert np.linalg.norm(W - w_ref) <= 1e-3 * np.linalg.norm(w_ref)
    assert np.abs(W - w_ref).max() <= 1e-3 * np.abs(w_ref).max()


@pytest.mark.parametrize("k,n", [(8, 2500), (128, 2500), (8, 12000)])
def test_rayleigh_ritz_matches_oracle(k, n):
    """Ritz values of B = -A on span(X) and relerr (Sec. 5) from the device's Grams and FP64 k x k
    algebra, against the oracle's QR + dense eigendecomposition, for a raw random block (large
    relerr) and for a block after 300 oracle updates (small relerr). n = 12,000 with k = 8 takes
    more row groups for its one-pair Gram than the workspace's two-pair sizing holds, so the
    launch uses fewer, larger groups."""
    import torch
    e = synth.sbm(n, 8, 24.0, 6.0, ratio_kind="count", seed=101)
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, k, 102)
    x_conv = o.iterate(og, o.OFM_F1, x0, 0.0, 300).X.astype(np.float32)
    for X in (x0, x_conv):
        lam_ref, rel_ref = o.rayleigh_ritz_relerr(og, X.astype(np.float64))
        Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        ritz = torch.zeros(k, dtype=torch.float64, device="cuda")
        rel = ofsc.ofsc_rayleigh_ritz(g, Xd, ritz)
        lam = ritz.cpu().numpy()
        assert np.max(np.abs(lam - lam_ref)) <= 2e-6 * np.max(np.abs(lam_ref))
        assert abs(rel - rel_ref) <= 0.02 * rel_ref + 2e-6, (rel, rel_ref)
    # a rank-deficient block is refused
    Xbad = np.array(x0)
    Xbad[:, 1] = Xbad[:, 0]
    with pytest.raises(ofsc.OfscError):
        ofsc.ofsc_rayleigh_ritz(g, torch.from_numpy(Xbad).cuda(), torch.zeros(k, dtype=torch.float64, device="cuda"))


@pytest.mark.parametrize("which,k", [(1, 8), (2, 8), (1, 32), (2, 32)])
def test_weight_grad_matches_oracle(which, k):
    """df/dw for every listed edge of a weighted SBM (repeated pairs and self-loops included) against
    the oracle's FP64 gradient."""
    import torch
    e = synth.sbm(3000, 6, 20.0, 6.0, ratio_kind="count", weighted=True, seed=111)
    x = synth.initial_block(e.n, k, 112) * 3.0
    g = gpu_graph(e)
    src, dst, w = upload(e)
    Xd = torch.from_numpy(x).cuda()
    grad = torch.empty(e.m, dtype=torch.float32, device="cuda")
    ofsc.ofsc_weight_grad(g, which, Xd, src, dst, grad)
    ref = o.weight_grad(e.n, e.src, e.dst, e.w, x, which)
    got = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)
    loops = e.src == e.dst
    assert loops.any() and np.all(got[loops] == 0.0)


@pytest.mark.parametrize("which", [1, 2])
def test_autograd_objective_matches_central_differences(which):
    """The differentiable objective (weighted SBM, 20,000 nodes, k = 32, w ~ U(0.5, 1.5)): the
    directional derivatives of its hand-written backward in X and in the edge weights against FP64
    oracle central differences (step 1e-3, 64 random directions)."""
    import torch
    e, x0 = synth.workload("wsbm_n20k_k32")
    X = torch.from_numpy(x0 * 4.0).cuda().requires_grad_(True)
    src, dst, w = upload(e)
    w = w.clone().requires_grad_(True)
    f = ofsc.objective(X, w, src, dst, e.n, which)
    f.backward()
    gX = X.grad.cpu().numpy().astype(np.float64)
    gw = w.grad.cpu().numpy().astype(np.float64)
    f64 = o.objective_of_weights(e.n, e.src, e.dst, e.w, x0 * 4.0, which)
    assert abs(float(f.detach()) - f64) <= 1e-5 * max(1.0, abs(f64))
    rng = np.random.default_rng(113)
    eps = 1e-3
    xb, wb = (x0 * 4.0).astype(np.float64), e.w.astype(np.float64)
    for _ in range(64):
        dX = rng.standard_normal(xb.shape) * 1e-2
        dw = rng.standard_normal(wb.shape) * 1e-1
        fp = o.objective_of_weights(e.n, e.src, e.dst, wb + eps * dw, xb + eps * dX, which)
        fm = o.objective_of_weights(e.n, e.src, e.dst, wb - eps * dw, xb - eps * dX, which)
        fd = (fp - fm) / (2 * eps)
        an = float(np.sum(gX * dX) + np.sum(gw * dw))
        assert abs(an - fd) <= 1e-3 * abs(fd) + 1e-6, (an, fd)


def batch_problems(scale, count):
    """The first `count` graphs of the 32-graph batch recipe, node counts scaled by `scale`, plus:
    a graph with no nodes (skipped by the batch); one with k = 128 (tensor-core Grams and
    direction pass) to mix engines in one batch; and the first graph again from X0 = 0, where every
    direction vanishes, so that problem stops at t = 0 while the others go on."""
    probs = synth.batch("sbm_batch32", scale)[:count]
    probs.append((synth.EdgeList(n=0, src=np.zeros(0, np.int32), dst=np.zeros(0, np.int32), w=None,
                                 labels=np.zeros(0, np.int32), n_blocks=3), np.zeros((0, 3), np.float32)))
    e = synth.sbm(3000, 128, 20.0, 5.0, ratio_kind="count", seed=121)
    probs.append((e, synth.initial_block(e.n, 128, 122)))
    probs.append((probs[0][0], np.zeros_like(probs[0][1])))
    return probs


@pytest.mark.parametrize("method", METHODS)
def test_batched_equals_single_bit_for_bit(method):
    """ofsc_iterate_batched gives every problem the arithmetic ofsc_iterate gives it: same X, same
    result fields, bit for bit, with the replayed updates launched per graph on the graphs' streams
    (the default), grouped (one launch per kernel over the blocks of the graphs of a lane; two
    lanes here), and launched directly. maxit = 40 spans two host flag reads and one exact refresh
    of AX; tol = 1e-3 lets some problems stop early. Grouping takes fewer launches."""
    import torch
    probs = batch_problems(0.02, 6)
    graphs = [gpu_graph(e) for e, _ in probs]
    singles = []
    for g, (e, x0) in zip(graphs, probs):
        X = torch.from_numpy(x0).cuda()
        r = ofsc.ofsc_iterate(g, method, X, 1e-3, 40) if e.n > 0 else None
        singles.append((X.cpu().numpy(), r))
    totals = {}
    for direct, group in ((False, 0), (False, 2), (True, 0)):
        Xs = [torch.from_numpy(x0).cuda() for _, x0 in probs]
        rs = ofsc.ofsc_iterate_batched(graphs, method, Xs, 1e-3, 40, direct_launch=direct, group_launches=group)
        assert len(rs) == len(probs)
        stopped_early = 0
        for (Xr, r), X, rb, (e, _) in zip(singles, Xs, rs, probs):
            assert np.array_equal(X.cpu().numpy(), Xr), (direct, group)
            if e.n == 0:
                assert rb.iterations == 0
                continue
            assert (rb.iterations, rb.status, rb.rel_dir_norm, rb.f, rb.g0_norm) == \
                   (r.iterations, r.status, r.rel_dir_norm, r.f, r.g0_norm)
            if group == 0:
                assert rb.kernel_launches >= r.kernel_launches
            stopped_early += rb.iterations < 40
        assert stopped_early >= 1
        totals[(direct, group)] = sum(r.kernel_launches for r in rs)
    assert totals[(False, 2)] < totals[(False, 0)]


@pytest.mark.parametrize("gather", [0, 1])
def test_grouped_launches_match_per_graph_launches(gather):
    """The grouped form of a batch's replayed updates on graphs that take every variant of the
    direction product the grouping covers: weighted and binary S, hub rows split by merge path
    (with its fixup launch), k from 3 to 64, FP32 and BF16 gathers; the same bits as one launch per
    graph and kernel, for every method, and a single graph grouped on its own (group_launches = 1)
    as well. Lanes change only which graphs share a launch, never the bits."""
    import torch
    probs = synth.batch("sbm_batch32", 0.02)[:4]
    probs.append((hub_graph(True, 230), synth.initial_block(6000, 20, 231)))
    probs.append((hub_graph(False, 232), synth.initial_block(6000, 3, 233)))
    e = synth.sbm(2500, 7, 14.0, 4.0, ratio_kind="count", weighted=True, seed=234)
    probs.append((e, synth.initial_block(e.n, 64, 235)))
    graphs = [gpu_graph(e) for e, _ in probs]
    for method in METHODS:
        out = {}
        for group in (0, 1, 3, 7):  # per graph; one lane; three lanes; one graph per lane
            Xs = [torch.from_numpy(x0).cuda() for _, x0 in probs]
            rs = ofsc.ofsc_iterate_batched(graphs, method, Xs, 0.0, 37, gather=gather, group_launches=group)
            out[group] = ([X.cpu().numpy() for X in Xs], [(r.iterations, r.status, r.rel_dir_norm, r.f) for r in rs])
            for a, b in zip(out[group][0], out[0][0]):
                assert np.array_equal(a, b), (method, group)
            assert out[group][1] == out[0][1]
    X1 = torch.from_numpy(probs[4][1]).cuda()
    X2 = X1.clone()
    r1 = ofsc.ofsc_iterate(graphs[4], o.OFM_F1, X1, 0.0, 20, gather=gather, group_launches=1)
    r2 = ofsc.ofsc_iterate(graphs[4], o.OFM_F1, X2, 0.0, 20, gather=gather)
    assert torch.equal(X1, X2) and r1.rel_dir_norm == r2.rel_dir_norm


@pytest.mark.parametrize("gather", [0, 1])
def test_overlapped_grams_match_serial(gather):
    """opts.overlap_gram = 1 runs V^T X and V^T V on a second stream beside the direction product
    (the default for one graph of n kp <= 2^23, as here): the same kernels on the same inputs, so
    the same bits as the serial order (overlap_gram = -1), for every method,
    with the tensor-core Grams (k = 128) and the CUDA-core ones (k = 20), on whole rows and on
    merge-path shares, replayed and launched directly, and in a batched call."""
    import torch
    e = synth.sbm(6000, 8, 18.0, 5.0, ratio_kind="count", seed=250)
    cases = [(gpu_graph(e), synth.initial_block(e.n, 128, 251), 0),
             (gpu_graph(e), synth.initial_block(e.n, 20, 252), 0),
             (gpu_graph(hub_graph(False, 253)), synth.initial_block(6000, 128, 254), 1)]
    for method in METHODS:
        for g, x0, mp in cases:
            for direct in (False, True):
                out = []
                for ov in (-1, 0, 1):  # serial; the default (overlapped at these sizes); overlapped
                    X = torch.from_numpy(x0).cuda()
                    r = ofsc.ofsc_iterate(g, method, X, 0.0, 40, gather=gather, merge_path=mp,
                                          direct_launch=direct, overlap_gram=ov)
                    out.append((X.cpu().numpy(), (r.iterations, r.status, r.rel_dir_norm, r.f)))
                for x, res in out[1:]:
                    assert np.array_equal(out[0][0], x), (method, x0.shape, mp, direct)
                    assert out[0][1] == res
        graphs = [c[0] for c in cases]
        outs = []
        for ov in (-1, 1):
            Xs = [torch.from_numpy(c[1]).cuda() for c in cases]
            rs = ofsc.ofsc_iterate_batched(graphs, method, Xs, 0.0, 37, gather=gather, overlap_gram=ov)
            outs.append(([X.cpu().numpy() for X in Xs], [(r.iterations, r.status, r.rel_dir_norm) for r in rs]))
        for a, b in zip(outs[0][0], outs[1][0]):
            assert np.array_equal(a, b), method
        assert outs[0][1] == outs[1][1]
    for bad in (-2, 2):
        with pytest.raises(ofsc.OfscError) as ei:
            ofsc.ofsc_iterate(cases[1][0], o.OFM_F1, torch.from_numpy(cases[1][1]).cuda(), 0.0, 2, overlap_gram=bad)
        assert ei.value.status == ofsc.ERR_INVALID_ARG and "overlap_gram" in str(ei.value)


def test_batched_full_size_in_the_bench_configuration():
    """The 32-graph batch at full size (N from 3.5K to 99K, k from 8 to 64, sum N = 1.53M) as
    bench.py --workload sbm_batch32 runs it (one batched call, BF16 gathers, the product's shape
    autotuned per graph), five updates of OFM-f1; the smallest, the median and the largest graph
    against the oracle element by element (2e-3 of max|X|, one BF16 unit roundoff)."""
    import torch
    probs = synth.batch("sbm_batch32", 1.0)
    graphs = [gpu_graph(e) for e, _ in probs]
    for g, (e, x0) in zip(graphs, probs):
        ofsc.ofsc_autotune(g, x0.shape[1], ofsc.GATHER_BF16)
    Xs = [torch.from_numpy(x0).cuda() for _, x0 in probs]
    rs = ofsc.ofsc_iterate_batched(graphs, o.OFM_F1, Xs, 0.0, 5, gather=ofsc.GATHER_BF16)
    assert all(r.iterations == 5 for r in rs)
    order = np.argsort([e.n for e, _ in probs])
    for i in (order[0], order[len(order) // 2], order[-1]):
        e, x0 = probs[i]
        ref = o.iterate(o.build_graph(e.n, e.src, e.dst), o.OFM_F1, x0, 0.0, 5)
        assert_elementwise(Xs[i].cpu().numpy(), ref.X, 2e-3, f"graph {i} (N = {e.n}, k = {x0.shape[1]})")


def test_batched_matches_oracle():
    """Five updates of OFM-f1 on each of four problems of the batch recipe (k from 8 to 64) in one
    batched call, against the oracle run problem by problem."""
    import torch
    probs = synth.batch("sbm_batch32", 0.01)[:4]
    graphs = [gpu_graph(e) for e, _ in probs]
    Xs = [torch.from_numpy(x0).cuda() for _, x0 in probs]
    rs = ofsc.ofsc_iterate_batched(graphs, o.OFM_F1, Xs, 0.0, 5)
    for (e, x0), X, r in zip(probs, Xs, rs):
        ref = o.iterate(o.build_graph(e.n, e.src, e.dst), o.OFM_F1, x0, 0.0, 5)
        assert r.iterations == 5 == ref.iterations
        Xg = X.cpu().numpy()
        assert_elementwise(Xg, ref.X, 1e-4)


def test_batched_rejects_bad_arguments():
    import torch
    e, x0 = synth.batch("sbm_batch32", 0.01)[0]
    g = gpu_graph(e)
    X = torch.from_numpy(x0).cuda()
    with pytest.raises(ofsc.OfscError):
        ofsc.ofsc_iterate_batched([g, g], o.OFM_F1, [X, X.clone()], 0.0, 3)
    with pytest.raises(ofsc.OfscError):
        ofsc.ofsc_iterate_batched([g], 7, [X], 0.0, 3)
    assert ofsc.ofsc_iterate_batched([], o.OFM_F1, [], 0.0, 3) == []


def test_objective_reuses_its_graph_until_the_edges_change():
    """ofsc.objective builds the graph of (src, dst, w) once and reuses it while the same tensors
    come back unchanged; an in-place change of w (an optimiser step) builds it again, and f follows
    the new weights (against the oracle)."""
    import torch
    e = synth.sbm(2000, 8, 16.0, 6.0, weighted=True, seed=270)
    x0 = synth.initial_block(e.n, 8, 271) * 4.0
    src, dst, w = upload(e)
    w = w.clone().requires_grad_(True)
    X = torch.from_numpy(x0).cuda().requires_grad_(True)
    ofsc._OBJ_GRAPHS.clear()
    f1 = ofsc.objective(X, w, src, dst, e.n, 1)
    g_first = next(iter(ofsc._OBJ_GRAPHS.values()))[0]
    f1b = ofsc.objective(X, w, src, dst, e.n, 1)
    assert len(ofsc._OBJ_GRAPHS) == 1 and next(iter(ofsc._OBJ_GRAPHS.values()))[0] is g_first
    assert float(f1.detach()) == float(f1b.detach())
    with torch.no_grad():
        w.mul_(1.25)
    f2 = ofsc.objective(X, w, src, dst, e.n, 1)
    assert len(ofsc._OBJ_GRAPHS) == 2
    f_ref = o.objective_of_weights(e.n, e.src, e.dst, e.w.astype(np.float64) * 1.25, x0.astype(np.float64), 1)
    assert abs(float(f2.detach()) - f_ref) <= 1e-5 * max(1.0, abs(f_ref))
    f2.backward()
    assert w.grad is not None and torch.isfinite(w.grad).all()


@pytest.mark.parametrize("case", ["sbm_k8", "wsbm_k32"])
def test_unrolled_grad_matches_oracle(case):
    """d f1(X_20) / d X_0 (and d/dw on the weighted graph) through 20 updates of OFM-f1,
    checkpointed every 5 updates, against the oracle's reverse accumulation in FP64 (itself pinned
    by central differences); the same bits for every checkpoint interval, and T = 0 gives
    grad f1(X_0).

    Tolerance: after 20 line-searched updates the gradient is ill-conditioned: the oracle's own
    result moves by ~1e-3 (relative) when every entry of X_0 moves up by one FP32 ulp. The GPU
    result, computed in FP32, is allowed twice that measured sensitivity (at least 1e-3)."""
    import torch
    if case == "sbm_k8":
        e = synth.sbm(1500, 8, 16.0, 5.0, ratio_kind="count", seed=131)
        k = 8
    else:
        e = synth.sbm(2000, 32, 32.0, 10.0, seed=132, weighted=True)
        k = 32
    weighted = e.w is not None
    og = o.build_graph(e.n, e.src, e.dst, None if not weighted else e.w.astype(np.float64), exact=weighted)
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, k, 133)
    T = 20
    if weighted:
        f_ref, g_ref, w_ref = o.unrolled_grad(og, x0.astype(np.float64), T,
                                              edges=(e.src, e.dst, e.w.astype(np.float64)))
    else:
        f_ref, g_ref = o.unrolled_grad(og, x0.astype(np.float64), T)
    # every entry of X_0 one FP32 ulp up: the GPU's FP32 arithmetic perturbs each update by about
    # that much, and such a shift moves the oracle's gradient by ~1e-3 on the binary graph
    xp = np.nextafter(x0, np.float32(np.inf)).astype(np.float64)
    if weighted:
        _, gp, wp = o.unrolled_grad(og, xp, T, edges=(e.src, e.dst, e.w.astype(np.float64)))
        wtol = max(1e-3, 2.0 * np.linalg.norm(wp - w_ref) / np.linalg.norm(w_ref))
    else:
        _, gp = o.unrolled_grad(og, xp, T)
    tol = max(1e-3, 2.0 * np.linalg.norm(gp - g_ref) / np.linalg.norm(g_ref))
    X0 = torch.from_numpy(x0).cuda()
    src, dst, _ = upload(e)
    outs = {}
    for ckpt in (5, 1, 7, 20):
        grad = torch.empty_like(X0)
        gw = torch.full((e.src.size,), float("nan"), dtype=torch.float32, device="cuda") if weighted else None
        f = ofsc.ofsc_unrolled_grad(g, X0, T, grad, ckpt=ckpt, src=src if weighted else None,
                                    dst=dst if weighted else None, grad_w=gw)
        outs[ckpt] = (f, grad.cpu().numpy(), None if gw is None else gw.cpu().numpy())
    f, G, W = outs[5]
    assert abs(f - f_ref) <= 1e-5 * abs(f_ref)
    err = np.linalg.norm(G - g_ref) / np.linalg.norm(g_ref)
    assert err <= tol, (err, tol)
    if weighted:
        werr = np.linalg.norm(W - w_ref) / np.linalg.norm(w_ref)
        assert werr <= wtol, (werr, wtol)
    for ckpt in (1, 7, 20):
        assert outs[ckpt][0] == f and np.array_equal(outs[ckpt][1], G)
        if weighted:
            assert np.array_equal(outs[ckpt][2], W)
    grad0 = torch.empty_like(X0)
    f0 = ofsc.ofsc_unrolled_grad(g, X0, 0, grad0)
    Gd = torch.empty_like(X0)
    fo = ofsc.ofsc_objective_grad(g, 1, X0, Gd)
    assert abs(f0 - fo) <= 1e-6 * abs(fo)
    # the two paths form X^T X on different engines (tensor cores vs. CUDA cores): FP32 rounding apart
    G0, Gr = grad0.cpu().numpy(), Gd.cpu().numpy()
    assert np.linalg.norm(G0 - Gr) <= 1e-5 * np.linalg.norm(Gr)


def test_autotune_keeps_results_within_rounding():
    """ofsc_autotune picks a row partition (4..32 warps per SM) and the gathers in flight per lane
    by timing; the first five updates after it still match the oracle element by element, and
    every shape gives the same A V rows (only the fold of diag(V^T AV) changes its rounding). Then
    every slot count is forced in turn through the tuned shape and compared with the default."""
    e = synth.sbm(20000, 16, 24.0, 5.0, ratio_kind="count", seed=141)
    og = o.build_graph(e.n, e.src, e.dst)
    g = gpu_graph(e)
    x0 = synth.initial_block(e.n, 16, 142)
    Xa, ra, _ = run_iterate(g, o.OFM_F1, x0, 0.0, 5)
    w, u, ms = ofsc.ofsc_autotune(g, 16, ofsc.GATHER_FP32)
    assert w in [m * 152 for m in (4, 8, 16, 32)] and u in (2, 4, 6, 8) and ms > 0.0
    Xb, rb, _ = run_iterate(g, o.OFM_F1, x0, 0.0, 5)
    ref = o.iterate(og, o.OFM_F1, x0, 0.0, 5)
    for X in (Xa, Xb):
        assert_elementwise(X, ref.X, 1e-4)
    assert np.linalg.norm(Xa - Xb) <= 1e-5 * np.linalg.norm(Xa)
    # BF16 storage at k = 128 (16 lanes per nonzero: slots 2 to 8 are all valid shapes)
    e2 = synth.sbm(6000, 8, 24.0, 5.0, ratio_kind="count", seed=143, gamma=2.3)
    og2 = o.build_graph(e2.n, e2.src, e2.dst)
    g2 = gpu_graph(e2)
    x2 = synth.initial_block(e2.n, 128, 144)
    w2, u2, _ = ofsc.ofsc_autotune(g2, 128, ofsc.GATHER_BF16)
    assert u2 in (2, 4, 6, 8)
    X2, _, _ = run_iterate(g2, o.OFM_F1, x2, 0.0, 5, gather=ofsc.GATHER_BF16)
    assert_elementwise(X2, o.iterate(og2, o.OFM_F1, x2, 0.0, 5).X, 2e-3)


def cubic_cases(seed):
    """Seeded cubics {c3, c2, c1, c0} with three well-separated real roots or one real root,
    scales from 1e-6 to 1e6, whose antiderivative values at the roots differ by more than 1e-6
    (so that the root choice is not a near-tie that rounding may flip), and the edge cases."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < 6000:
        s = 10.0 ** rng.uniform(-6, 6) * rng.choice([-1.0, 1.0])
        if len(out) % 2 == 0:
            r = np.sort(rng.uniform(-10, 10, 3))
            if np.min(np.diff(r)) < 0.1:
                continue
            c = (s, -s * r.sum(), s * (r[0] * r[1] + r[0] * r[2] + r[1] * r[2]), -s * r.prod())
            qv = sorted(o.quartic_antiderivative(c, x) for x in r)
            if qv[1] - qv[0] <= 1e-6 * max(1.0, abs(qv[0])):
                continue
        else:  # (a - r)(a^2 + b a + d) with b^2 < 4 d
            r0, b = rng.uniform(-10, 10, 2)
            d = b * b / 4.0 + rng.uniform(0.5, 20.0)
            c = (s, s * (b - r0), s * (d - b * r0), -s * d * r0)
        out.append(c)
    edge = [(0.0, 1.0, -3.0, 2.0),    # quadratic, roots 1 and 2
            (0.0, 0.0, 2.0, -1.0),    # linear
            (0.0, 1.0, 0.0, 1.0),     # quadratic without a real root
            (0.0, 0.0, 0.0, 0.0),     # zero
            (1.0, 0.0, -3.0, 2.0),    # (a - 1)^2 (a + 2): a double root
            (1.0, -6.0, 12.0, -8.0),  # (a - 2)^3
            (2.0, 0.0, 0.0, 0.0)]     # 2 a^3
    return np.array(out + edge, dtype=np.float64), len(edge)


def test_line_search_step_matches_oracle():
    """The exact line search's root choice (Sec. 3.2) on its own: the one-thread and the one-warp
    device solvers give the same bits on every cubic, and match the oracle's Cardano roots and
    choice within 1e-10 relative on well-separated roots, one-root cubics and the edge cases
    (quadratic, linear, none, zero, double and triple roots); non-finite coefficients are flagged
    and give 0."""
    import torch
    c, n_edge = cubic_cases(260)
    bad_rows = np.array([[np.inf, 1.0, 1.0, 1.0], [1.0, np.nan, 0.0, 0.0]])
    coef = torch.from_numpy(np.vstack([c, bad_rows])).cuda()
    n = coef.shape[0]
    steps = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(2)]
    bads = [torch.full((n,), -1, dtype=torch.int32, device="cuda") for _ in range(2)]
    for solver in (0, 1):
        ofsc.ofsc_line_search_step(coef, steps[solver], bads[solver], solver=solver)
    s0, s1 = steps[0].cpu().numpy(), steps[1].cpu().numpy()
    b0, b1 = bads[0].cpu().numpy(), bads[1].cpu().numpy()
    assert np.array_equal(s0.view(np.int64), s1.view(np.int64)) and np.array_equal(b0, b1)
    assert b0[-2:].tolist() == [1, 1] and s0[-2:].tolist() == [0.0, 0.0] and not b0[:-2].any()
    ref = np.array([o.choose_root(tuple(row)) for row in c])
    np.testing.assert_allclose(s0[:len(c)], ref, rtol=1e-10, atol=1e-12)
    assert s0[len(c) - n_edge:len(c)].tolist() == pytest.approx([2.0, 0.5, 0.0, 0.0, -2.0, 2.0, 0.0])
    with pytest.raises(ofsc.OfscError) as ei:
        ofsc.ofsc_line_search_step(coef, steps[0], solver=2)
    assert ei.value.status == ofsc.ERR_INVALID_ARG
