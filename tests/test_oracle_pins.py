"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: brute force on tiny graphs,
closed-form spectra, finite differences, polynomial interpolation of the defining expression,
the fixed points stated by Theorems 1-4, published known-answer vectors, or a library routine.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import ofsc_oracle as o
from paper_2305_10356_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
METHODS = [o.OFM_F1, o.TRI_F1, o.OFM_F2, o.TRI_F2]


def small_graph(n=40, blocks=4, deg=6.0, seed=7, weighted=False):
    e = synth.sbm(n, blocks, deg, 8.0, seed=seed, weighted=weighted)
    return o.build_graph(n, e.src, e.dst, e.w), e


# ------------------------------------------------------------------------------------------
# Graph build (Eq. (1)): brute force on tiny edge lists
# ------------------------------------------------------------------------------------------

def brute_S(n, src, dst, w=None):
    S = {}
    for t, (a, b) in enumerate(zip(src, dst)):
        a, b = int(a), int(b)
        if a == b:
            continue
        val = 1.0 if w is None else float(w[t])
        for key in ((a, b), (b, a)):
            if w is None:
                S[key] = 1.0
            else:
                S[key] = S.get(key, 0.0) + val
    return S


@pytest.mark.parametrize("weighted", [False, True])
def test_graph_build_brute_force(weighted):
    rng = np.random.default_rng(3)
    n = 9
    src = rng.integers(0, n, 40)
    dst = rng.integers(0, n, 40)
    src[:3] = dst[:3]  # self-loops
    src = np.concatenate([src, [2, 5]])
    dst = np.concatenate([dst, [5, 2]])  # the same pair in both directions
    w = rng.uniform(0.5, 1.5, src.size).astype(np.float32) if weighted else None
    g = o.build_graph(n, src, dst, w)
    S = brute_S(n, src, dst, w)
    want_rows = [sorted(c for (r, c) in S if r == i) for i in range(n)]
    got_rows = [list(g.col[g.row_ptr[i]:g.row_ptr[i + 1]]) for i in range(n)]
    assert got_rows == want_rows
    if weighted:
        for i in range(n):
            for p in range(g.row_ptr[i], g.row_ptr[i + 1]):
                assert g.val[p] == np.float32(S[(i, int(g.col[p]))])
    assert g.n_selfloops == int(np.sum(src == dst))
    for i in range(n):
        d = sum(float(np.float32(S[(i, c)])) for c in want_rows[i])
        assert g.deg[i] == d
        assert g.s[i] == (1.0 / math.sqrt(d) if d > 0 else 0.0)
    assert g.n_isolated == sum(1 for i in range(n) if not want_rows[i])


def test_graph_build_rejects_bad_input():
    with pytest.raises(ValueError):
        o.build_graph(3, np.array([0]), np.array([3]))
    with pytest.raises(ValueError):
        o.build_graph(3, np.array([0]), np.array([1]), np.array([-1.0], np.float32))
    with pytest.raises(ValueError):
        o.build_graph(3, np.array([0]), np.array([1]), np.array([np.nan], np.float32))


def test_empty_graph():
    g = o.build_graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.nnz == 0 and g.n_isolated == 5
    X = np.arange(10.0).reshape(5, 2)
    np.testing.assert_array_equal(o.apply_A(g, X), -X)  # isolated nodes: L_ii = 1, A_ii = -1


# ------------------------------------------------------------------------------------------
# Spectrum of L (Eq. (1), Sec. 1): closed forms
# ------------------------------------------------------------------------------------------

def test_cycle_spectrum():
    n = 12
    src = np.arange(n)
    dst = (src + 1) % n
    g = o.build_graph(n, src, dst)
    lam = np.linalg.eigvalsh(o.dense_L(g))
    want = np.sort(1.0 - np.cos(2.0 * np.pi * np.arange(n) / n))
    np.testing.assert_allclose(lam, want, atol=1e-12)
    assert abs(lam[-1] - 2.0) < 1e-12  # even cycle is bipartite: largest eigenvalue is 2


def test_complete_graph_spectrum():
    n = 7
    src, dst = zip(*itertools.combinations(range(n), 2))
    g = o.build_graph(n, np.array(src), np.array(dst))
    lam = np.linalg.eigvalsh(o.dense_L(g))
    np.testing.assert_allclose(lam, [0.0] + [n / (n - 1)] * (n - 1), atol=1e-12)


def test_clique_union_null_space():
    sizes = [3, 4, 5, 2]
    src, dst, off = [], [], 0
    for s in sizes:
        for a, b in itertools.combinations(range(off, off + s), 2):
            src.append(a)
            dst.append(b)
        off += s
    g = o.build_graph(off, np.array(src), np.array(dst))
    lam = np.linalg.eigvalsh(o.dense_L(g))
    assert int(np.sum(np.abs(lam) < 1e-10)) == len(sizes)


def test_random_graph_spectrum_bounds_and_kernel():
    g, _ = small_graph(60, 3, 8.0, seed=11)
    L = o.dense_L(g)
    lam, U = np.linalg.eigh(L)
    assert lam[0] > -1e-12 and lam[-1] < 2.0 + 1e-12
    assert abs(lam[0]) < 1e-12
    v = np.sqrt(g.deg)
    v /= np.linalg.norm(v)
    assert abs(abs(U[:, 0] @ v) - 1.0) < 1e-10  # eigenvector of 0 is D^1/2 1 (connected)
    # A = L - 2I shares eigenvectors, eigenvalues in [-2, 0]
    lamA = np.linalg.eigvalsh(o.dense_A(g))
    np.testing.assert_allclose(lamA, lam - 2.0, atol=1e-12)


def test_apply_A_matches_dense():
    g, _ = small_graph(30, 3, 5.0, seed=5, weighted=True)
    X = np.random.default_rng(0).standard_normal((30, 4))
    np.testing.assert_allclose(o.apply_A(g, X), o.dense_A(g) @ X, atol=1e-13)


# ------------------------------------------------------------------------------------------
# Objectives and gradients (Eqs. (2), (3), (5), (10))
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("which", [1, 2])
def test_objective_matches_definition(which):
    g, _ = small_graph(25, 2, 5.0, seed=2, weighted=(which == 2))
    X = np.random.default_rng(1).standard_normal((25, 3)) * 0.3
    A = o.dense_A(g)
    f = o.objective(which, X, o.apply_A(g, X), o.normA_fro2(g))
    assert f == pytest.approx(o.objective_dense(which, A, X), rel=1e-12)


@pytest.mark.parametrize("which", [1, 2])
def test_gradient_finite_differences(which):
    g, _ = small_graph(20, 2, 4.0, seed=4)
    A = o.dense_A(g)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((20, 3)) * 0.4
    G = o.gradient(which, X, A @ X)
    h = 1e-5
    for _ in range(8):
        D = rng.standard_normal(X.shape)
        fd = (o.objective_dense(which, A, X + h * D) - o.objective_dense(which, A, X - h * D)) / (2 * h)
        assert np.sum(G * D) == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("method", [o.TRI_F1, o.TRI_F2])
def test_tri_direction_prefix_property(method):
    """triu makes column j of g depend only on columns 1..j (Eqs. (7), (12))."""
    g, _ = small_graph(20, 2, 4.0, seed=8)
    X = np.random.default_rng(3).standard_normal((20, 5))
    G = o.direction(method, X, o.apply_A(g, X))
    for i in range(1, 6):
        Xi = X[:, :i]
        np.testing.assert_allclose(o.direction(method, Xi, o.apply_A(g, Xi)), G[:, :i], atol=1e-12)


def test_ofm_f2_gradient_vanishes_at_eigenvectors():
    """Sec. 2.2: grad f2(U_k) = 0 while grad f1(U_k) != 0; grad f1(U_k sqrt(-Lam)) = 0."""
    g, _ = small_graph(30, 3, 6.0, seed=9)
    A = o.dense_A(g)
    lam, U = np.linalg.eigh(A)
    Uk = U[:, :3]
    assert np.abs(o.gradient(2, Uk, A @ Uk)).max() < 1e-12
    assert np.abs(o.gradient(1, Uk, A @ Uk)).max() > 1e-2
    W = Uk * np.sqrt(-lam[:3])[None, :]
    assert np.abs(o.gradient(1, W, A @ W)).max() < 1e-12


# ------------------------------------------------------------------------------------------
# Line search (Sec. 3.2, Eqs. (15)-(18)): interpolate the defining expression
# ------------------------------------------------------------------------------------------

def _fit_cubic(fun, scale):
    al = np.linspace(-2.0, 2.0, 9) * scale
    vals = np.array([fun(a) for a in al])
    return np.polyfit(al, vals, 3), al, vals


@pytest.mark.parametrize("method", METHODS)
def test_linesearch_coeffs_interpolate(method):
    g, _ = small_graph(24, 3, 5.0, seed=12, weighted=True)
    A = o.dense_A(g)
    rng = np.random.default_rng(5)
    k = 4
    X = rng.standard_normal((24, k)) * 0.3
    V = rng.standard_normal((24, k)) * 0.2
    coeffs = o.linesearch_coeffs(method, X, V, A @ X, A @ V)
    if method in (o.OFM_F1, o.OFM_F2):
        which = o.objective_of(method)
        scale = 0.25 if which == 1 else 1.0  # Eq. (15) as printed is d/dalpha f1 / 4

        def fun(a):
            Z = X + a * V
            return scale * np.sum(V * o.gradient(which, Z, A @ Z))

        fit, _, _ = _fit_cubic(fun, 1.0)
        np.testing.assert_allclose(coeffs[0], fit, rtol=1e-9, atol=1e-9 * np.abs(fit).max())
    else:
        for i in range(1, k + 1):
            Xi, Vi = X[:, :i], V[:, :i]

            def fun(a):
                Z = Xi + a * Vi
                return np.sum(Vi * o.direction(method, Z, A @ Z))

            fit, _, _ = _fit_cubic(fun, 1.0)
            np.testing.assert_allclose(coeffs[i - 1], fit, rtol=1e-9,
                                       atol=1e-9 * np.abs(fit).max())


def test_cubic_roots_known():
    for roots in ([1.0, -2.0, 3.5], [0.1, 0.2, 0.3], [-5.0, 1e-3, 7.0]):
        c = np.poly(roots) * 2.5
        got = sorted(r for r, _ in o.cubic_real_roots(*c))
        np.testing.assert_allclose(got, sorted(roots), rtol=1e-10, atol=1e-12)
    # one real root: (x - 2)(x^2 + x + 1)
    c = np.polymul([1.0, -2.0], [1.0, 1.0, 1.0])
    got = o.cubic_real_roots(*c)
    assert len(got) == 1 and abs(got[0][0] - 2.0) < 1e-12
    # exact double root: (x - 1)^2 (x + 2) -> simple root -2 chosen by the rule
    c = np.poly([1.0, 1.0, -2.0])
    assert o.choose_root(c) == pytest.approx(-2.0)
    # degenerate leading coefficient: quadratic, linear, all zero
    assert sorted(r for r, _ in o.cubic_real_roots(0.0, 1.0, -3.0, 2.0)) == pytest.approx([1.0, 2.0])
    assert o.cubic_real_roots(0.0, 0.0, 2.0, -1.0)[0][0] == pytest.approx(0.5)
    assert o.choose_root([0.0, 0.0, 0.0, 0.0]) == 0.0


def test_cubic_roots_random_vs_numpy():
    rng = np.random.default_rng(9)
    for _ in range(300):
        c = rng.standard_normal(4) * 10.0 ** rng.uniform(-3, 3, 4)
        got = sorted(r for r, _ in o.cubic_real_roots(*c))
        ref = np.roots(c)
        ref = sorted(x.real for x in ref if abs(x.imag) <= 1e-7 * max(1.0, abs(x)))
        if len(ref) != len(got):
            continue  # near-double roots: classification is ill-posed
        for a, b in zip(got, ref):
            assert abs(np.polyval(c, a)) <= 1e-9 * np.sum(np.abs(c) * np.abs(a) ** np.arange(3, -1, -1)) + 1e-300
            assert a == pytest.approx(b, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("method", [o.OFM_F1, o.OFM_F2])
def test_chosen_step_is_global_minimiser_along_line(method):
    """OFM: the chosen root minimises f(X + alpha V) over alpha (brute-force grid + refine)."""
    g, _ = small_graph(24, 3, 5.0, seed=13)
    A = o.dense_A(g)
    rng = np.random.default_rng(6)
    which = o.objective_of(method)
    nA2 = o.normA_fro2(g)
    for trial in range(6):
        X = rng.standard_normal((24, 3)) * 0.5
        V = -o.gradient(which, X, A @ X) * (0.5 if trial % 2 else 1.0)
        alpha = o.step_sizes(g, method, X, V, A @ X, A @ V, nA2)[0]

        def f(a):
            return o.objective(which, X + a * V, A @ (X + a * V), nA2)

        span = 4.0 * max(abs(alpha), 1e-3)
        grid = np.linspace(-span, span, 4001)
        vals = np.array([f(a) for a in grid])
        a0 = grid[np.argmin(vals)]
        # golden-section refinement around the grid minimum
        lo, hi = a0 - 2 * (grid[1] - grid[0]), a0 + 2 * (grid[1] - grid[0])
        phi = (math.sqrt(5) - 1) / 2
        for _ in range(80):
            m1, m2 = hi - phi * (hi - lo), lo + phi * (hi - lo)
            if f(m1) < f(m2):
                hi = m2
            else:
                lo = m1
        assert alpha == pytest.approx(0.5 * (lo + hi), rel=1e-5, abs=1e-9)
        assert f(alpha) <= min(vals) + 1e-12 * abs(min(vals))


def test_tri_root_choice_is_argmin_of_antiderivative():
    c = np.poly([-1.0, 0.5, 2.0])  # c3 > 0: two local minima of q at -1 and 2
    q = [o.quartic_antiderivative(c, r) for r in (-1.0, 0.5, 2.0)]
    want = [-1.0, 0.5, 2.0][int(np.argmin(q))]
    assert o.choose_root(c) == pytest.approx(want)


# ------------------------------------------------------------------------------------------
# Algorithm 2 converges to the fixed points of Theorems 1-4
# ------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def thm_case():
    g, e = small_graph(60, 4, 8.0, seed=39)
    A = o.dense_A(g)
    lam, U = np.linalg.eigh(A)
    k = 4
    assert lam[k] - lam[k - 1] > 0.05  # gap so the bottom-k space is well defined
    X0 = synth.initial_block(60, k, 99).astype(np.float64)
    return g, lam, U, k, X0


@pytest.mark.parametrize("method", METHODS)
def test_theorem_fixed_points(thm_case, method):
    g, lam, U, k, X0 = thm_case
    res = o.iterate(g, method, X0, tol=1e-11, maxit=3000)
    assert res.converged, (res.iterations, res.rel_dir_norm)
    X = res.X
    Uk = U[:, :k]
    assert o.subspace_sin(X, Uk) < 1e-8
    XtX = X.T @ X
    if method == o.OFM_F1:  # Theorem 1: X = U_k sqrt(-Lam_k) Q
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(XtX)), np.sort(-lam[:k]), atol=1e-9)
    elif method == o.OFM_F2:  # Theorem 3: X = U_k Q
        np.testing.assert_allclose(XtX, np.eye(k), atol=1e-9)
    elif method == o.TRI_F1:  # Theorem 2: X = U_k sqrt(-Lam_k) D
        for i in range(k):
            want = U[:, i] * math.sqrt(-lam[i])
            s = np.sign(X[:, i] @ want)
            np.testing.assert_allclose(X[:, i], s * want, atol=1e-8)
    else:  # Theorem 4: X = U_k D
        for i in range(k):
            s = np.sign(X[:, i] @ U[:, i])
            np.testing.assert_allclose(X[:, i], s * U[:, i], atol=1e-8)


@pytest.mark.parametrize("method", METHODS)
def test_first_step_is_exact_linesearch_along_minus_g(method):
    """Algorithm 2: V0 = -G0 and X1 = X0 + V0 diag(alpha) with the Sec. 3.2 step."""
    g, _ = small_graph(30, 3, 6.0, seed=3)
    A = o.dense_A(g)
    X0 = synth.initial_block(30, 3, 5).astype(np.float64)
    res = o.iterate(g, method, X0, tol=0.0, maxit=1)
    G0 = o.direction(method, X0, A @ X0)
    a = res.alphas[0]
    np.testing.assert_allclose(res.X, X0 - G0 * a[None, :], atol=1e-14)
    if method in (o.OFM_F1, o.OFM_F2):  # tr(V0^T grad f(X1)) = 0 at an exact line search
        which = o.objective_of(method)
        G1 = o.gradient(which, res.X, A @ res.X)
        assert abs(np.sum(G0 * G1)) < 1e-9 * np.sum(G0 * G0)


def test_iterate_stationary_start_and_zero_iterations():
    g, _ = small_graph(20, 2, 4.0, seed=1)
    res = o.iterate(g, o.OFM_F1, np.zeros((20, 3)), tol=1e-6, maxit=10)
    assert res.iterations == 0 and res.converged and np.all(res.X == 0)
    X0 = synth.initial_block(20, 3, 1)
    res = o.iterate(g, o.OFM_F1, X0, tol=1e-6, maxit=0)
    np.testing.assert_array_equal(res.X, X0.astype(np.float64))


def test_iterate_node_permutation_equivariance():
    """Relabelling nodes permutes the rows of every iterate (no index mix-up in Algorithm 2)."""
    e = synth.sbm(40, 3, 6.0, 8.0, seed=31)
    g = o.build_graph(40, e.src, e.dst)
    perm = np.random.default_rng(0).permutation(40)
    inv = np.argsort(perm)
    gp = o.build_graph(40, inv[e.src], inv[e.dst])
    X0 = synth.initial_block(40, 3, 7).astype(np.float64)
    for method in METHODS:
        r1 = o.iterate(g, method, X0, 0.0, 6)
        r2 = o.iterate(gp, method, X0[perm], 0.0, 6)
        np.testing.assert_allclose(r2.X, r1.X[perm], atol=1e-10)


def test_zero_padded_columns_are_inert():
    """Zero columns appended after the real ones stay zero and change nothing else."""
    g, _ = small_graph(30, 3, 6.0, seed=6)
    X0 = synth.initial_block(30, 3, 2).astype(np.float64)
    Xp = np.concatenate([X0, np.zeros((30, 2))], axis=1)
    for method in METHODS:
        a = o.iterate(g, method, X0, 0.0, 8)
        b = o.iterate(g, method, Xp, 0.0, 8)
        np.testing.assert_allclose(b.X[:, :3], a.X, atol=1e-12)
        assert np.all(b.X[:, 3:] == 0.0)


# ------------------------------------------------------------------------------------------
# Algorithm 1 steps 3-4, evaluation metrics, Philox
# ------------------------------------------------------------------------------------------

def test_row_normalize():
    X = np.array([[3.0, 4.0], [0.0, 0.0], [1.0, 0.0]])
    np.testing.assert_allclose(o.row_normalize(X), [[0.6, 0.8], [0.0, 0.0], [1.0, 0.0]])


def test_philox_known_answers():
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        rows = [line.split() for line in fh if line.strip() and not line.startswith("#")]
    assert rows
    for r in rows:
        v = [int(x, 16) for x in r]
        assert o.philox4x32_10(v[:4], v[4:6]) == tuple(v[6:])


def test_ari_matches_library():
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(4)
    for _ in range(10):
        a = rng.integers(0, 5, 200)
        b = np.where(rng.random(200) < 0.7, a, rng.integers(0, 6, 200))
        assert o.ari(a, b) == pytest.approx(sk.adjusted_rand_score(a, b), abs=1e-12)
    assert o.ari(a, a) == 1.0


def test_kmeans_blobs_and_fixed_point():
    rng = np.random.default_rng(8)
    centers = rng.standard_normal((5, 3)) * 10
    truth = rng.integers(0, 5, 500)
    X = centers[truth] + rng.standard_normal((500, 3)) * 0.3
    lab, inertia = o.kmeans(X, 5, seed=123, n_init=2)
    assert o.ari(lab, truth) == 1.0
    mu = np.stack([X[lab == c].mean(axis=0) for c in range(5)])
    d = ((X[:, None, :] - mu[None]) ** 2).sum(-1)
    np.testing.assert_array_equal(np.argmin(d, axis=1), lab)  # Lloyd fixed point
    assert inertia == pytest.approx(d[np.arange(500), lab].sum())
    lab2, _ = o.kmeans(X, 5, seed=123, n_init=2)
    np.testing.assert_array_equal(lab, lab2)


def test_lloyd_iterations_match_library():
    """From the same initial centres the oracle's Lloyd iterations reach scikit-learn's Lloyd
    result: the same labels and the same inertia."""
    sk = pytest.importorskip("sklearn.cluster")
    rng = np.random.default_rng(3)
    centers = rng.standard_normal((6, 4)) * 3
    X = centers[rng.integers(0, 6, 2000)] + rng.standard_normal((2000, 4))
    for seed in (1, 2, 3):
        idx = o.kmeans_pp_seeds(X, 6, seed, 0)
        lab, inertia = o.kmeans(X, 6, seed=seed, n_init=1)
        km = sk.KMeans(n_clusters=6, init=X[idx], n_init=1, max_iter=300, tol=0.0, algorithm="lloyd").fit(X)
        np.testing.assert_array_equal(lab, km.labels_)
        assert inertia == pytest.approx(km.inertia_, rel=1e-12)


def test_kmeanspp_seeding_follows_d_squared():
    """k-means++ (Arthur and Vassilvitskii): the first centre is uniform over the points and the
    next is point j with probability D(j)^2 / sum D^2 (D the distance to the chosen centre). Over
    4000 seeds the empirical frequencies of the second centre, given the first, pass a
    chi-square test at the 0.1% level for every first centre."""
    X = np.array([[0.0], [1.0], [3.0], [6.0], [10.0]])
    n = len(X)
    firsts = np.zeros(n)
    counts = np.zeros((n, n))
    for seed in range(4000):
        idx = o.kmeans_pp_seeds(X, 2, seed, 0)
        firsts[idx[0]] += 1
        counts[idx[0], idx[1]] += 1
    expect = 4000 / n
    assert np.sum((firsts - expect) ** 2 / expect) < 18.47  # chi-square, 4 dof, p = 0.001
    for c in range(n):
        d2 = (X[:, 0] - X[c, 0]) ** 2
        p = d2 / d2.sum()
        tot = counts[c].sum()
        assert counts[c, c] == 0
        keep = p > 0
        chi = np.sum((counts[c, keep] - tot * p[keep]) ** 2 / (tot * p[keep]))
        assert chi < 18.47, (c, counts[c], tot * p)


def test_subspace_sin_known_angle():
    th = 0.3
    assert o.subspace_sin(np.array([[1.0], [0.0]]), np.array([[math.cos(th)], [math.sin(th)]])) \
        == pytest.approx(math.sin(th), rel=1e-12)


def test_rayleigh_ritz_on_eigenvectors():
    g, _ = small_graph(30, 3, 6.0, seed=10)
    lam, U = np.linalg.eigh(o.dense_L(g))
    R = np.linalg.qr(np.random.default_rng(1).standard_normal((3, 3)))[0]
    ritz, rel = o.rayleigh_ritz_relerr(g, U[:, :3] @ R * 2.0)
    assert rel < 1e-12
    np.testing.assert_allclose(np.sort(ritz), np.sort(2.0 - lam[:3]), atol=1e-12)


def test_rayleigh_ritz_matches_generalised_eigenproblem():
    """For a random block, the Ritz values are the eigenvalues of the pencil (X^T B X, X^T X)
    (scipy's generalised symmetric solver, no orthonormalisation), and relerr is the residual of
    the Ritz vectors U = X z written out with the dense B, relative to ||U Lam||_F."""
    import scipy.linalg as sla
    g, _ = small_graph(60, 4, 8.0, seed=12)
    B = -o.dense_A(g)
    X = np.random.default_rng(5).standard_normal((60, 4))
    lam, Z = sla.eigh(X.T @ B @ X, X.T @ X)
    U = X @ Z
    rel = np.linalg.norm(B @ U - U * lam[None, :]) / np.linalg.norm(U * lam[None, :])
    ritz, rel_o = o.rayleigh_ritz_relerr(g, X)
    np.testing.assert_allclose(np.sort(ritz), lam, rtol=1e-10, atol=1e-12)
    assert rel_o == pytest.approx(rel, rel=1e-9)
    assert rel > 1e-3  # a random block is far from invariant


@pytest.mark.parametrize("method", [o.TRI_F1, o.OFM_F1])
def test_optional_restart_gives_descent_directions(method):
    """The optional restart (not in Algorithm 2; restart=True) gives every column a descent
    direction, v_j^T g_j < 0, while its gradient is above rounding level."""
    g, _ = small_graph(40, 3, 7.0, seed=17)
    A = o.dense_A(g)
    X0 = synth.initial_block(40, 3, 4).astype(np.float64)
    X = X0.copy()
    # replay the recurrences step by step and check the sign of v_j^T g_j
    res = o.iterate(g, method, X0, 0.0, 400, restart=True)
    assert np.all(np.isfinite(res.X))
    G_prev = o.direction(method, X0, A @ X0)
    g0 = np.linalg.norm(G_prev, axis=0)
    V = -G_prev
    for t in range(1, len(res.betas)):
        X = X + V * res.alphas[t - 1][None, :]
        G = o.direction(method, X, A @ X)
        V = -G + V * res.betas[t][None, :]
        vg = np.sum(V * G, axis=0)
        live = np.linalg.norm(G, axis=0) > 1e-8 * g0
        assert np.all(vg[live] < 0), (t, vg)
    assert res.rel_norms[-1] < 1e-9


@pytest.mark.parametrize("method", METHODS)
def test_long_run_past_convergence_stays_finite(method):
    """Algorithm 2 as printed (no restart), in FP64: 1500 updates on a 40-node graph, far past the
    rounding floor, keep X finite and the relative direction norm at that floor."""
    g, _ = small_graph(40, 3, 7.0, seed=17)
    X0 = synth.initial_block(40, 3, 4).astype(np.float64)
    res = o.iterate(g, method, X0, 0.0, 1500)
    assert np.all(np.isfinite(res.X))
    assert min(res.rel_norms) < 1e-14 and res.rel_norms[-1] < 1e-13


# ------------------------------------------------------------------------------------------
# The Polak-Ribiere coefficient of Algorithm 2, pinned by what it implies: n-step termination of
# CG near a minimiser, the column-wise (per-column) form, and acceleration over steepest descent
# (Sec. 3.1). A planted mistake in cg_beta fails at least one of the three.
# ------------------------------------------------------------------------------------------

def _pin_local_termination() -> bool:
    """One column of OFM-f1 started 1e-6 from the minimiser x* = u_1 sqrt(-lambda_1) (Theorem 1).
    There f1 is a quadratic (Hessian 4(A - lambda_1 I) + 8 (-lambda_1) u_1 u_1^T, positive definite
    when lambda_1 < lambda_2) plus O(|e|^3). Nonlinear CG with an exact line search then repeats
    linear CG up to O(|e|), and linear CG ends in at most n steps on an n-dimensional quadratic, so
    after n updates the relative gradient is O(|e_0|). Steepest descent (beta = 0) only gains
    ((kappa - 1)/(kappa + 1))^n, about 1e-2 on these graphs."""
    for n_nodes, seed in ((10, 3), (12, 5), (16, 7)):
        g, _ = small_graph(n_nodes, 2, 4.0, seed=seed)
        lam, U = np.linalg.eigh(o.dense_A(g))
        assert lam[1] - lam[0] > 0.1
        x_star = U[:, :1] * math.sqrt(-lam[0])
        X0 = x_star + 1e-6 * np.random.default_rng(1).standard_normal(x_star.shape)
        r = o.iterate(g, o.OFM_F1, X0, 0.0, n_nodes)
        if not r.rel_norms[-1] <= 1e-4:
            return False
    return True


def _pin_columnwise() -> bool:
    """TriOFM's first i columns evolve on their own: g(X)[:, :i] = g(X[:, :i]), the prefix-i cubic
    involves only the first i columns, and Algorithm 2 sums beta's quotient column by column. So
    the first i columns of a run equal a run from X_0[:, :i]."""
    g, _ = small_graph(40, 3, 7.0, seed=17)
    X0 = synth.initial_block(40, 3, 4).astype(np.float64)
    for method in (o.TRI_F1, o.TRI_F2):
        full = o.iterate(g, method, X0, 0.0, 30).X
        for i in (1, 2):
            if not np.allclose(full[:, :i], o.iterate(g, method, X0[:, :i], 0.0, 30).X, rtol=0, atol=1e-12):
                return False
    return True


def _pin_accelerates(monkeypatch) -> bool:
    """Sec. 3.1 adopts CG to accelerate gradient descent: on the 60-node, 4-block graph of the
    Theorem pins, Algorithm 2 reaches 1e-10 in fewer updates than the same iteration with beta = 0
    (steepest descent with the same exact line search), for OFM-f1 and TriOFM-f1."""
    g, _ = small_graph(60, 4, 8.0, seed=39)
    X0 = synth.initial_block(60, 4, 99).astype(np.float64)
    for method in (o.OFM_F1, o.TRI_F1):
        cg = o.iterate(g, method, X0, 1e-10, 2000).iterations
        with monkeypatch.context() as m:
            m.setattr(o, "cg_beta", lambda Gn, G: (np.zeros(Gn.shape[1]), np.sum(G * G, axis=0)))
            sd = o.iterate(g, method, X0, 1e-10, 2000).iterations
        if not cg < sd:
            return False
    return True


def test_beta_n_step_termination_near_a_minimiser():
    assert _pin_local_termination()


def test_beta_is_columnwise():
    assert _pin_columnwise()


def test_beta_accelerates_steepest_descent(monkeypatch):
    assert _pin_accelerates(monkeypatch)


def _q(num, den):
    return np.where(den != 0.0, num / np.where(den != 0.0, den, 1.0), 0.0)


BETA_MISTAKES = {
    "fletcher_reeves": lambda Gn, G: (_q(np.sum(Gn * Gn, 0), np.sum(G * G, 0)), np.sum(G * G, 0)),
    "zero": lambda Gn, G: (np.zeros(Gn.shape[1]), np.sum(G * G, 0)),
    "swapped_t_and_t_minus_1": lambda Gn, G: (_q(np.sum((G - Gn) * G, 0), np.sum(Gn * Gn, 0)), np.sum(Gn * Gn, 0)),
    "sign": lambda Gn, G: (-_q(np.sum((Gn - G) * Gn, 0), np.sum(G * G, 0)), np.sum(G * G, 0)),
    "dropped_minus_in_numerator": lambda Gn, G: (_q(np.sum((Gn + G) * Gn, 0), np.sum(G * G, 0)), np.sum(G * G, 0)),
    "denominator_of_G_t": lambda Gn, G: (_q(np.sum((Gn - G) * Gn, 0), np.sum(Gn * Gn, 0)), np.sum(G * G, 0)),
    "one_beta_for_all_columns": lambda Gn, G: (np.full(Gn.shape[1], _q(np.sum((Gn - G) * Gn), np.sum(G * G))),
                                               np.sum(G * G, 0)),
}


@pytest.mark.parametrize("mistake", list(BETA_MISTAKES))
def test_beta_pins_catch_planted_mistakes(monkeypatch, mistake):
    """Each plausible mistake in the Polak-Ribiere coefficient, planted in the oracle, fails at
    least one of the three beta pins."""
    monkeypatch.setattr(o, "cg_beta", BETA_MISTAKES[mistake])
    assert not (_pin_local_termination() and _pin_columnwise() and _pin_accelerates(monkeypatch))


def test_edge_stream_snapshots_are_cumulative_uniform_samples():
    """Streaming snapshots: each holds a prefix of one random order of the full edge list, so they
    are nested, the last one is the whole graph, and the sizes step by m / parts."""
    full = synth.sbm(500, 4, 12.0, 5.0, ratio_kind="count", join_isolated=False, seed=3)
    snaps = synth.edge_stream(full, 5, seed=4)
    prev = None
    for s, e in enumerate(snaps):
        assert e.m == int(round((s + 1) * full.m / 5))
        pairs = list(zip(e.src.tolist(), e.dst.tolist()))
        if prev is not None:
            assert pairs[: len(prev)] == prev
        prev = pairs
    assert sorted(prev) == sorted(zip(full.src.tolist(), full.dst.tolist()))
    # the early snapshots leave nodes isolated; the builder gives them D = 0 (Eq. (1) reading)
    og = o.build_graph(snaps[0].n, snaps[0].src, snaps[0].dst)
    assert (og.deg == 0).any()


def _objective_of_weights(n, src, dst, w, X, which):
    """Eqs. (2)/(3) written out densely in FP64 as a function of the listed edge weights."""
    S = np.zeros((n, n))
    for a, b, x in zip(src, dst, w):
        if a != b:
            S[a, b] += x
            S[b, a] += x
    d = S.sum(axis=1)
    sd = np.where(d > 0, 1.0 / np.sqrt(np.where(d > 0, d, 1.0)), 0.0)
    A = -np.eye(n) - sd[:, None] * S * sd[None, :]
    return o.objective_dense(which, A, X)


@pytest.mark.parametrize("which", [1, 2])
def test_weight_grad_matches_central_differences(which):
    """d f / d w for every listed edge against central differences of the dense FP64 objective, on
    a graph with a pair listed twice (in both directions), a self-loop and an isolated node."""
    rng = np.random.default_rng(11 + which)
    n, k = 10, 3
    src = np.array([0, 1, 2, 3, 4, 5, 6, 1, 7, 2, 8, 3], dtype=np.int64)
    dst = np.array([1, 2, 3, 4, 5, 6, 0, 0, 7, 5, 2, 0], dtype=np.int64)  # (1, 0) repeats (0, 1); (7, 7) a loop; 9 isolated
    w = rng.uniform(0.5, 1.5, src.size)
    X = rng.standard_normal((n, k)) * 0.4
    got = o.weight_grad(n, src, dst, w, X, which)
    eps = 1e-5
    for e in range(src.size):
        wp, wm = w.copy(), w.copy()
        wp[e] += eps
        wm[e] -= eps
        fd = (_objective_of_weights(n, src, dst, wp, X, which) - _objective_of_weights(n, src, dst, wm, X, which)) / (2 * eps)
        assert abs(got[e] - fd) <= 1e-6 * max(1.0, abs(fd)), (e, got[e], fd)
    assert got[8] == 0.0  # the self-loop
    assert got[0] == got[7]  # both listings of {0, 1}


@pytest.mark.parametrize("which", [1, 2])
def test_sparse_objective_of_weights_matches_dense(which):
    """The sparse FP64 objective of the listed weights equals Eqs. (2)/(3) written out densely."""
    rng = np.random.default_rng(31 + which)
    n, k = 14, 4
    src = rng.integers(0, n, 40)
    dst = rng.integers(0, n, 40)
    w = rng.uniform(0.5, 1.5, 40)
    X = rng.standard_normal((n, k)) * 0.3
    got = o.objective_of_weights(n, src, dst, w, X, which)
    ref = _objective_of_weights(n, src, dst, w, X, which)
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


# ------------------------------------------------------------------------------------------
# Differentiating through unrolled updates of OFM-f1: central differences in random directions
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed,T,restart,eps", [(5, 1, False, 1e-6), (5, 12, False, 1e-6), (12, 20, False, 1e-6),
                                                (24, 20, False, 1e-8), (12, 20, True, 1e-6), (24, 20, True, 1e-6)])
def test_unrolled_grad_matches_central_differences(seed, T, restart, eps):
    """d f1(X_T) / d X_0 through T updates of Algorithm 2 (line search by the implicit-function
    theorem, beta's quotient, the Hessian-vector products of the direction) against central
    differences of the FP64 iteration itself; with the optional restart, seeds 12 and 24 have
    columns restarted (beta held at 0) in several updates. Without the restart, seed 24's
    20-update map bends so sharply that central differences settle only below a step of 1e-7
    (1e-6 is off by 2%, 1e-8 agrees to 3e-7), hence its smaller step."""
    e = synth.sbm(80 if seed == 5 else 60, 3, 10.0 if seed == 5 else 8.0, 5.0, ratio_kind="count", seed=seed)
    g = o.build_graph(e.n, e.src, e.dst)
    x0 = synth.initial_block(e.n, 3, seed + 1).astype(np.float64)
    rec = []
    o.iterate(g, o.OFM_F1, x0, 0.0, T, record=rec, restart=restart)
    assert len(rec) == T
    if restart:
        assert sum(int(r["restart"].sum()) for r in rec) >= 6
    f, grad = o.unrolled_grad(g, x0, T, restart=restart)
    assert f == o.unrolled_objective(g, x0, T, restart=restart)
    rng = np.random.default_rng(seed * 100 + T)
    for _ in range(3):
        D = rng.standard_normal(x0.shape)
        fd = (o.unrolled_objective(g, x0 + eps * D, T, restart)
              - o.unrolled_objective(g, x0 - eps * D, T, restart)) / (2 * eps)
        assert abs(float(np.sum(grad * D)) - fd) <= 2e-6 * abs(fd), (float(np.sum(grad * D)), fd)


def test_unrolled_grad_without_updates_is_the_gradient():
    """T = 0 leaves L = f1(X_0), whose gradient is Eq. (5)."""
    g, _ = small_graph()
    x0 = synth.initial_block(g.n, 4, 3).astype(np.float64)
    f, grad = o.unrolled_grad(g, x0, 0)
    A = o.dense_A(g)
    np.testing.assert_allclose(grad, 4.0 * (A @ x0 + x0 @ (x0.T @ x0)), rtol=1e-12, atol=1e-14)
    assert abs(f - o.objective_dense(1, A, x0)) <= 1e-10 * abs(f)


@pytest.mark.parametrize("T", [1, 6, 20])
def test_unrolled_weight_grad_matches_central_differences(T):
    """d f1(X_T) / d w for every listed weight, through T updates of OFM-f1 (A enters every G_t,
    every line-search cubic and f1 itself), against central differences of the FP64 iteration on
    the graph rebuilt from the perturbed weights (FP64 throughout, no FP32 rounding of S)."""
    e = synth.sbm(60, 3, 8.0, 5.0, ratio_kind="count", seed=12, weighted=True)
    src, dst, w = e.src, e.dst, e.w.astype(np.float64)
    x0 = synth.initial_block(e.n, 3, 13).astype(np.float64)
    g = o.build_graph(e.n, src, dst, w, exact=True)
    f, gx, gw = o.unrolled_grad(g, x0, T, edges=(src, dst, w))
    f2, gx2 = o.unrolled_grad(g, x0, T)
    assert f == f2 and np.array_equal(gx, gx2)
    rng = np.random.default_rng(T)
    eps = 1e-6
    for _ in range(3):
        D = rng.standard_normal(w.shape)
        fp = o.unrolled_objective(o.build_graph(e.n, src, dst, w + eps * D, exact=True), x0, T)
        fm = o.unrolled_objective(o.build_graph(e.n, src, dst, w - eps * D, exact=True), x0, T)
        fd = (fp - fm) / (2 * eps)
        assert abs(float(np.sum(gw * D)) - fd) <= 2e-5 * abs(fd), (float(np.sum(gw * D)), fd)
    # T = 0: the same as the plain weight gradient of f1
    if T == 1:
        _, _, gw0 = o.unrolled_grad(g, x0, 0, edges=(src, dst, w))
        np.testing.assert_allclose(gw0, o.weight_grad(e.n, src, dst, w, x0, 1), rtol=1e-12, atol=1e-14)
