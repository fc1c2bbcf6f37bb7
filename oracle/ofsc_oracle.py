"""FP64 CPU oracle for spectral clustering via orthogonalization-free methods (arXiv 2305.10356).

TEST INFRASTRUCTURE ONLY. This module is the slow, plain statement of what the GPU path
computes. Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the product path never routes through it. It shares no code with
the CUDA library: it takes the same seeded inputs (edge lists, FP32 X0) and nothing else.

Arithmetic is FP64 throughout. Library primitives (scipy sparse product, numpy matmul, sort,
eigh, svd) serve as single steps; there is no blocking, fusion or reordering beyond what the
paper's formulas state.

Paper map:
  Eq. (1)           normalized Laplacian L = I - D^-1/2 S D^-1/2          -> build_graph, apply_A
  Eqs. (2), (3)     objectives f1, f2 on A = L - 2I                        -> objective
  Eqs. (5),(7),(10),(12)  directions grad f1, g1, grad f2, g2              -> direction
  Sec. 3.2, Eqs. (15)-(18)  exact line-search cubics                       -> linesearch_coeffs
  Sec. 3.2          Cardano roots and the three-case root choice           -> cubic_real_roots, choose_root
  Algorithm 2       column-wise nonlinear CG framework                     -> iterate
  Algorithm 1       row normalisation + K-means                            -> row_normalize, kmeans
  Sec. 5            ARI, relerr via Rayleigh-Ritz                          -> ari, rayleigh_ritz_relerr
  Eqs. (2), (5), (15), Algorithm 2   f1 after T updates, differentiated     -> unrolled_grad
                    in reverse through the updates (X_0 and edge weights)

Readings of the paper taken where it is silent or ambiguous (each one is pinned by a test):
  * X_i, V_i in Eqs. (16), (18) are the first i columns; alpha_i moves the whole prefix.
  * Eq. (15) as printed is one quarter of d/dalpha f1 (the roots are the same).
  * TriOFM has no objective, so "minimal function value" becomes the minimal value of the
    antiderivative q(alpha) of the printed cubic. For OFM the objective itself is evaluated.
  * The paper's momentum coefficient is Polak-Ribiere as Algorithm 2 writes it; 0/0 -> 0.
  * Algorithm 2 has no restart, and neither does `iterate` by default. An optional restart
    (restart=True: a column whose new direction would not descend, v_j^T g_j >= 0, takes
    beta_j = 0) exists only to check the library's matching opt-in option; it is not the paper's.
  * Step 0 of Algorithm 2 uses the same exact line search unless a fixed alpha0 > 0 is given.
  * Stop when ||G_t||_F / ||G_0||_F <= tol, or after maxit updates (Algorithm 2's t_max).
  * Isolated nodes (degree 0) get D^-1/2 = 0, i.e. L_ii = 1.
  * Repeated undirected pairs collapse (binary S) or have their weights summed (weighted S).

K-means is pinned in parts: its Lloyd iterations reach scikit-learn's Lloyd result from the same
initial centres, its seeding follows the D^2 rule of k-means++ in a chi-square test, and its
uniforms are Philox-4x32-10 known-answer vectors. The choice of seeding rule itself (which index
a uniform selects) is a reading; the GPU's agreement with the oracle is then judged by ARI.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

OFM_F1, TRI_F1, OFM_F2, TRI_F2 = 0, 1, 2, 3
METHOD_NAMES = {OFM_F1: "OFM-f1", TRI_F1: "TriOFM-f1", OFM_F2: "OFM-f2", TRI_F2: "TriOFM-f2"}


def objective_of(method: int) -> int:
    """1 for the f1 methods, 2 for the f2 methods."""
    return 1 if method in (OFM_F1, TRI_F1) else 2


# =============================================================================================
# Graph and operator, Eq. (1) and A = L - 2I (Sec. 1)
# =============================================================================================

@dataclasses.dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray  # int32 [nnz], ascending inside each row
    val: np.ndarray | None  # float32 [nnz] (weighted S) or None (binary S)
    deg: np.ndarray  # float64 [n], D_ii = sum_j S_ij
    s: np.ndarray  # float64 [n], D_ii^-1/2 (0 for isolated nodes)
    s32: np.ndarray  # float32 [n], FP32 rounding of s
    n_selfloops: int
    n_isolated: int

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def S(self) -> sp.csr_matrix:
        """S as an FP64 scipy CSR matrix."""
        data = np.ones(self.nnz) if self.val is None else self.val.astype(np.float64)
        return sp.csr_matrix((data, self.col, self.row_ptr), shape=(self.n, self.n))

    def A_hat(self) -> sp.csr_matrix:
        """D^-1/2 S D^-1/2 in FP64."""
        d = sp.diags(self.s)
        return (d @ self.S() @ d).tocsr()


def build_graph(n: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray | None = None,
                exact: bool = False) -> Graph:
    """S from an undirected edge list (Eq. (1)): symmetric, no self-loops, one entry per pair.

    Binary S: a pair listed several times (in either direction) is one edge of weight 1.
    Weighted S: the FP32 weights of all listings of a pair are summed in FP64, then rounded
    once to FP32. Degrees: D_ii = sum_j S_ij (an integer count, or an FP64 sum of the FP32
    entries). D^-1/2 is 1/sqrt(D_ii) in FP64, and 0 when D_ii = 0.
    exact=True keeps the weights and their sums in FP64 (no FP32 rounding anywhere), so that S is
    a smooth function of the listed weights (for derivatives by finite differences).
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    if n < 0 or src.shape != dst.shape:
        raise ValueError("bad sizes")
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= n or dst.max() >= n):
        raise ValueError("node id out of range")
    if w is not None:
        w = np.asarray(w, dtype=np.float64 if exact else np.float32)
        if w.shape != src.shape or not np.all(np.isfinite(w)) or np.any(w <= 0):
            raise ValueError("weights must be finite and > 0")
    loop = src == dst
    n_selfloops = int(loop.sum())
    keep = ~loop
    rows = np.concatenate([src[keep], dst[keep]])
    cols = np.concatenate([dst[keep], src[keep]])
    key = rows * max(n, 1) + cols
    # sort the (row, col) keys; the first entry of each run of equal keys is a distinct pair
    order = np.argsort(key, kind="stable")
    key_s = key[order]
    head = np.ones(key_s.size, dtype=bool)
    head[1:] = key_s[1:] != key_s[:-1]
    ukey = key_s[head]
    if w is None:
        val = None
    else:
        ww = np.concatenate([w[keep], w[keep]]).astype(np.float64)
        start = np.nonzero(head)[0]
        sums = np.add.reduceat(ww[order], start) if key_s.size else np.zeros(0)
        val = sums if exact else sums.astype(np.float32)
    r = (ukey // max(n, 1)).astype(np.int64)
    c = (ukey % max(n, 1)).astype(np.int32)
    counts = np.bincount(r, minlength=n)
    row_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    if val is None:
        deg = counts.astype(np.float64)
    else:
        deg = np.zeros(n)
        np.add.at(deg, r, val.astype(np.float64))
    s = np.zeros(n)
    nz = deg > 0
    s[nz] = 1.0 / np.sqrt(deg[nz])
    return Graph(n=n, row_ptr=row_ptr, col=c, val=val, deg=deg, s=s, s32=s.astype(np.float32),
                 n_selfloops=n_selfloops, n_isolated=int((~nz).sum()))


def apply_A(g: Graph, X: np.ndarray) -> np.ndarray:
    """A X with A = L - 2I = -I - D^-1/2 S D^-1/2 (Eq. (1), Sec. 1), in FP64."""
    X = np.asarray(X, dtype=np.float64)
    sx = g.s[:, None] * X
    return -X - g.s[:, None] * (g.S() @ sx)


def dense_A(g: Graph) -> np.ndarray:
    """A as a dense FP64 matrix (small graphs only)."""
    return -np.eye(g.n) - g.A_hat().toarray()


def dense_L(g: Graph) -> np.ndarray:
    """L = I - D^-1/2 S D^-1/2 as a dense FP64 matrix (small graphs only)."""
    return np.eye(g.n) - g.A_hat().toarray()


def normA_fro2(g: Graph) -> float:
    """||A||_F^2 = N + sum_ij (D^-1/2 S D^-1/2)_ij^2 (diagonal of A is -1, S has no loops)."""
    ah = g.A_hat()
    return float(g.n + np.sum(ah.data ** 2))


# =============================================================================================
# Objectives and directions, Eqs. (2), (3), (5), (7), (10), (12)
# =============================================================================================

def direction(method: int, X: np.ndarray, AX: np.ndarray) -> np.ndarray:
    """G = g(X) for the method: grad f1 (Eq. (5)), g1 (Eq. (7)), grad f2 (Eq. (10)), g2 (Eq. (12))."""
    XtX = X.T @ X
    if method == OFM_F1:
        return 4.0 * AX + 4.0 * X @ XtX
    if method == TRI_F1:
        return AX + X @ np.triu(XtX)
    XtAX = X.T @ AX
    if method == OFM_F2:
        return 4.0 * AX - 2.0 * X @ XtAX - 2.0 * AX @ XtX
    if method == TRI_F2:
        return 2.0 * AX - AX @ np.triu(XtX) - X @ np.triu(XtAX)
    raise ValueError(method)


def objective(which: int, X: np.ndarray, AX: np.ndarray, normA2: float) -> float:
    """f1 = ||A + X X^T||_F^2 (Eq. (2)) or f2 = tr((2I - X^T X) X^T A X) (Eq. (3)).

    f1 uses ||A + XX^T||^2 = ||A||^2 + 2 tr(X^T A X) + ||X^T X||^2 (A symmetric); the tests
    check it against the dense definition.
    """
    XtX = X.T @ X
    XtAX = X.T @ AX
    if which == 1:
        return float(normA2 + 2.0 * np.trace(XtAX) + np.sum(XtX * XtX))
    return float(np.trace((2.0 * np.eye(X.shape[1]) - XtX) @ XtAX))


def objective_dense(which: int, A: np.ndarray, X: np.ndarray) -> float:
    """Eqs. (2)/(3) evaluated literally with a dense A (small graphs only)."""
    if which == 1:
        M = A + X @ X.T
        return float(np.sum(M * M))
    return float(np.trace((2.0 * np.eye(X.shape[1]) - X.T @ X) @ X.T @ A @ X))


def gradient(which: int, X: np.ndarray, AX: np.ndarray) -> np.ndarray:
    """True gradient of f1 (Eq. (5)) or f2 (Eq. (10))."""
    return direction(OFM_F1 if which == 1 else OFM_F2, X, AX)


def objective_of_weights(n: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray, X: np.ndarray, which: int) -> float:
    """f1 (Eq. (2)) or f2 (Eq. (3)) in FP64 straight from the listed edge weights (pairs summed,
    self-loops dropped, no FP32 rounding of S), sparse: with A = -I - A_hat and tr(A_hat) = 0,
    ||A||_F^2 = n + ||A_hat||_F^2."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    a = np.minimum(src, dst)
    b = np.maximum(src, dst)
    keep = a != b
    keys, inv = np.unique(a[keep] * n + b[keep], return_inverse=True)
    pa, pb = keys // n, keys % n
    S = np.zeros(keys.size)
    np.add.at(S, inv, w[keep])
    d = np.zeros(n)
    np.add.at(d, pa, S)
    np.add.at(d, pb, S)
    sd = np.where(d > 0, 1.0 / np.sqrt(np.where(d > 0, d, 1.0)), 0.0)
    ah = S * sd[pa] * sd[pb]
    AX = -X.copy()
    np.add.at(AX, pa, -ah[:, None] * X[pb])
    np.add.at(AX, pb, -ah[:, None] * X[pa])
    normA2 = n + 2.0 * float(np.sum(ah * ah))
    return objective(which, X, AX, normA2)


def _pairs(n: int, src, dst, w):
    """The distinct undirected pairs {a < b} of an edge list with their FP64 summed weights:
    (kept listings, listing -> pair index, a, b, D^-1/2 per node, A_hat per pair)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    a = np.minimum(src, dst)
    b = np.maximum(src, dst)
    keep = a != b
    keys, inv = np.unique(a[keep] * n + b[keep], return_inverse=True)
    pa, pb = keys // n, keys % n
    S = np.zeros(keys.size)
    np.add.at(S, inv, w[keep])
    d = np.zeros(n)
    np.add.at(d, pa, S)
    np.add.at(d, pb, S)
    sd = np.where(d > 0, 1.0 / np.sqrt(np.where(d > 0, d, 1.0)), 0.0)
    return keep, inv, pa, pb, sd, S * sd[pa] * sd[pb]


def _weight_chain(n: int, keep, inv, pa, pb, sd, ah, gam) -> np.ndarray:
    """d/dw per listing from Gamma = d/dA_hat on the pairs (symmetric): a listing of {a, b}
    moves S_ab = S_ba and both degrees, 2 Gamma_ab / sqrt(d_a d_b) - r_a / d_a - r_b / d_b with
    r_a = sum_j Gamma_aj A_hat_aj."""
    r = np.zeros(n)
    np.add.at(r, pa, gam * ah)
    np.add.at(r, pb, gam * ah)
    gp = 2.0 * gam * sd[pa] * sd[pb] - r[pa] * sd[pa] ** 2 - r[pb] * sd[pb] ** 2
    out = np.zeros(keep.size)
    out[keep] = gp[inv]
    return out


def weight_grad(n: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray, X: np.ndarray, which: int) -> np.ndarray:
    """d f / d w_e for every listed edge e of a weighted graph, f = f1 (Eq. (2)) or f2 (Eq. (3)).

    Everything in FP64 from the listed weights (no FP32 rounding of S). With
    A_hat = D^-1/2 S D^-1/2, A = -I - A_hat and Gamma = df/dA_hat (symmetric),
        Gamma = 2 (I + A_hat - X X^T)          for f1,
        Gamma = -X (2I - X^T X) X^T            for f2,
    a listing of the pair {a, b} (a != b) changes S_ab = S_ba and the degrees d_a, d_b, so
        df/dw = 2 Gamma_ab / sqrt(d_a d_b) - r_a / d_a - r_b / d_b,   r_a = sum_j Gamma_aj A_hat_aj.
    Listings of the same pair share one value; self-loops (dropped from S) get 0.
    """
    X = np.asarray(X, dtype=np.float64)
    keep, inv, pa, pb, sd, ah = _pairs(n, src, dst, w)
    AhX = np.zeros_like(X)
    np.add.at(AhX, pa, ah[:, None] * X[pb])
    np.add.at(AhX, pb, ah[:, None] * X[pa])
    if which == 1:
        gam = 2.0 * (ah - np.sum(X[pa] * X[pb], axis=1))
        sq = np.zeros(n)
        np.add.at(sq, pa, ah * ah)
        np.add.at(sq, pb, ah * ah)
        r = 2.0 * (sq - np.sum(X * AhX, axis=1))
    else:
        Z = X @ (2.0 * np.eye(X.shape[1]) - X.T @ X)
        gam = -np.sum(X[pa] * Z[pb], axis=1)
        r = -np.sum(Z * AhX, axis=1)
    gp = 2.0 * gam * sd[pa] * sd[pb] - r[pa] * sd[pa] ** 2 - r[pb] * sd[pb] ** 2
    out = np.zeros(src.size)
    out[keep] = gp[inv]
    return out


# =============================================================================================
# Exact line search, Sec. 3.2, Eqs. (15)-(18)
# =============================================================================================

def _tr(M):
    return float(np.trace(M))


def linesearch_coeffs(method: int, X, V, AX, AV) -> np.ndarray:
    """Cubic coefficients [c3, c2, c1, c0] as printed in Eqs. (15)-(18).

    OFM methods: one cubic (shape [1, 4]). TriOFM methods: one cubic per prefix i = 1..k
    (shape [k, 4]), with X_i, V_i the first i columns of X, V.
    """
    VtV = V.T @ V
    VtX = V.T @ X
    XtV = X.T @ V
    XtX = X.T @ X
    VtAV = V.T @ AV
    VtAX = V.T @ AX
    XtAV = X.T @ AV
    XtAX = X.T @ AX
    tu = np.triu
    if method == OFM_F1:  # Eq. (15)
        c3 = _tr(VtV @ VtV)
        c2 = 3.0 * _tr(VtV @ XtV)
        c1 = _tr(VtAV + VtX @ VtX + VtX @ XtV + VtV @ XtX)
        c0 = _tr(VtAX + VtX @ XtX)
        return np.array([[c3, c2, c1, c0]])
    if method == OFM_F2:  # Eq. (17)
        c3 = -4.0 * _tr(VtV @ VtAV)
        c2 = -6.0 * _tr(VtX @ VtAV + VtV @ VtAX)
        c1 = 2.0 * _tr(2.0 * VtAV - 2.0 * VtX @ XtAV - 2.0 * VtX @ VtAX - VtV @ XtAX - XtX @ VtAV)
        c0 = 2.0 * _tr(2.0 * VtAX - VtX @ XtAX - XtX @ VtAX)
        return np.array([[c3, c2, c1, c0]])
    k = X.shape[1]
    out = np.zeros((k, 4))
    for i in range(1, k + 1):
        s = slice(0, i)
        Qi, Pi, Pti, Ri = VtV[s, s], VtX[s, s], XtV[s, s], XtX[s, s]
        Ci, Ei, Eti, Bi = VtAV[s, s], VtAX[s, s], XtAV[s, s], XtAX[s, s]
        if method == TRI_F1:  # Eq. (16)
            c3 = _tr(Qi @ tu(Qi))
            c2 = _tr(Qi @ tu(Pti) + Qi @ tu(Pi) + Pi @ tu(Qi))
            c1 = _tr(Ci + Pi @ tu(Pi) + Pi @ tu(Pti) + Qi @ tu(Ri))
            c0 = _tr(Ei + Pi @ tu(Ri))
        elif method == TRI_F2:  # Eq. (18)
            c3 = -_tr(Ci @ tu(Qi) + Qi @ tu(Ci))
            c2 = -_tr(Ei @ tu(Qi) + Ci @ tu(Pti) + Ci @ tu(Pi) + Pi @ tu(Ci) + Qi @ tu(Eti)
                      + Qi @ tu(Ei))
            c1 = _tr(2.0 * Ci - Ei @ tu(Pti) - Ei @ tu(Pi) - Ci @ tu(Ri) - Pi @ tu(Eti)
                     - Pi @ tu(Ei) - Qi @ tu(Bi))
            c0 = _tr(2.0 * Ei - Ei @ tu(Ri) - Pi @ tu(Bi))
        else:
            raise ValueError(method)
        out[i - 1] = [c3, c2, c1, c0]
    return out


def _polish(c, x, steps=2):
    c3, c2, c1, c0 = c
    for _ in range(steps):
        f = ((c3 * x + c2) * x + c1) * x + c0
        d = (3.0 * c3 * x + 2.0 * c2) * x + c1
        if d == 0.0 or not np.isfinite(d):
            break
        nx = x - f / d
        if not np.isfinite(nx):
            break
        x = nx
    return x


def cubic_real_roots(c3, c2, c1, c0):
    """Real roots of c3 a^3 + c2 a^2 + c1 a + c0 = 0 by Cardano's formula (Sec. 3.2).

    Returns a list of (root, multiplicity). Roots are polished by two FP64 Newton steps.
    When c3 == 0 the polynomial is solved as a quadratic or linear one; when every
    coefficient is zero the list is empty.
    """
    if c3 == 0.0:
        if c2 == 0.0:
            if c1 == 0.0:
                return []
            return [(-c0 / c1, 1)]
        disc = c1 * c1 - 4.0 * c2 * c0
        if disc < 0.0:
            return []
        if disc == 0.0:
            return [(-c1 / (2.0 * c2), 2)]
        sq = math.sqrt(disc)
        qq = -0.5 * (c1 + math.copysign(sq, c1))
        r1 = qq / c2
        r2 = c0 / qq if qq != 0.0 else -c1 / c2 - r1
        return [(r1, 1), (r2, 1)]
    a, b, c = c2 / c3, c1 / c3, c0 / c3
    p = b - a * a / 3.0
    q = 2.0 * a ** 3 / 27.0 - a * b / 3.0 + c
    shift = -a / 3.0
    disc = (q / 2.0) ** 2 + (p / 3.0) ** 3
    coeffs = (c3, c2, c1, c0)
    if disc > 0.0:
        # one real root; the sign choice avoids cancellation inside the cube root
        u = np.cbrt(-q / 2.0 - math.copysign(math.sqrt(disc), q))
        t = u - p / (3.0 * u) if u != 0.0 else 0.0
        return [(_polish(coeffs, t + shift), 1)]
    if disc == 0.0:
        if p == 0.0:
            return [(shift, 3)]
        return [(_polish(coeffs, 3.0 * q / p + shift), 1), (-3.0 * q / (2.0 * p) + shift, 2)]
    r = 2.0 * math.sqrt(-p / 3.0)
    phi = math.acos(max(-1.0, min(1.0, (3.0 * q / (2.0 * p)) * math.sqrt(-3.0 / p))))
    return [(_polish(coeffs, r * math.cos(phi / 3.0 - 2.0 * math.pi * j / 3.0) + shift), 1)
            for j in range(3)]


def quartic_antiderivative(c, a):
    """q(a) = c3 a^4/4 + c2 a^3/3 + c1 a^2/2 + c0 a, the antiderivative of the cubic."""
    c3, c2, c1, c0 = c
    return ((c3 / 4.0 * a + c2 / 3.0) * a + c1 / 2.0) * a * a + c0 * a


def choose_root(c, value_of=None) -> float:
    """The step size from the cubic's real roots, by the three cases of Sec. 3.2.

    One real root: that root. A double root and a simple root: the simple root. Three real
    roots: the one with the smallest function value, where `value_of(alpha)` gives the
    objective along the line (OFM) or, when None, the antiderivative q (TriOFM reading).
    Ties go to the smaller |alpha|, then the smaller alpha. No real root: 0.
    """
    roots = cubic_real_roots(*c)
    if not roots:
        return 0.0
    if len(roots) == 1:
        return float(roots[0][0])
    if len(roots) == 2 and any(m == 2 for _, m in roots):
        return float([r for r, m in roots if m == 1][0]) if any(m == 1 for _, m in roots) \
            else float(roots[0][0])
    vals = [(value_of(r) if value_of is not None else quartic_antiderivative(c, r), abs(r), r)
            for r, _ in roots]
    return float(min(vals)[2])


# =============================================================================================
# Algorithm 2 (column-wise nonlinear CG with exact line search)
# =============================================================================================

@dataclasses.dataclass
class IterResult:
    X: np.ndarray
    iterations: int
    rel_dir_norm: float
    g0_norm: float
    f: float
    converged: bool
    alphas: list
    betas: list
    rel_norms: list


def step_sizes(g: Graph, method: int, X, V, AX, AV, normA2: float) -> np.ndarray:
    """alpha (k-vector) by exact line search (Sec. 3.2); OFM uses one alpha for all columns."""
    k = X.shape[1]
    C = linesearch_coeffs(method, X, V, AX, AV)
    if method in (OFM_F1, OFM_F2):
        which = objective_of(method)

        def f_along(a):
            return objective(which, X + a * V, AX + a * AV, normA2)

        return np.full(k, choose_root(C[0], f_along))
    return np.array([choose_root(C[i]) for i in range(k)])


def cg_beta(G_new: np.ndarray, G_old: np.ndarray):
    """Column-wise Polak-Ribiere coefficient of Algorithm 2:
    beta_i = sum_l (G_new - G_old)_li G_new,li / sum_l G_old,li^2, with 0 where the denominator
    is 0 (a zero column of G_old, e.g. a padded column). Returns (beta, denominator)."""
    num = np.sum((G_new - G_old) * G_new, axis=0)
    den = np.sum(G_old * G_old, axis=0)
    beta = np.where(den != 0.0, num / np.where(den != 0.0, den, 1.0), 0.0)
    return beta, den


def iterate(g: Graph, method: int, X0: np.ndarray, tol: float, maxit: int,
            alpha0: float = 0.0, record: list | None = None, restart: bool = False) -> IterResult:
    """Algorithm 2 for one of the four methods, in FP64, from the FP32 (or FP64) start X0.

    G_0 = g(X_0); V_0 = -G_0; X_1 = X_0 + alpha V_0 (alpha0 > 0 given, else exact line
    search); then for t = 1, 2, ...: G_t = g(X_t); stop if ||G_t|| <= tol ||G_0|| or t = maxit;
    beta_t by cg_beta (Polak-Ribiere, 0 when the denominator is 0); V_t = -G_t + V_{t-1} diag(beta);
    alpha by exact line search; X_{t+1} = X_t + V_t diag(alpha).
    restart=True (not in the paper; off by default) also sets beta_i = 0 where the new column
    would not descend: -|g_i|^2 + beta_i v_i^T g_i >= 0.
    `record`, when given, receives one dict per update t: X_t, G_t, V_t, AV_t, alpha_t, beta_t,
    the denominators of beta_t and the columns whose beta the optional restart set to 0.
    """
    X = np.array(X0, dtype=np.float64)
    normA2 = normA_fro2(g)
    AX = apply_A(g, X)
    G = direction(method, X, AX)
    g0 = float(np.linalg.norm(G))
    alphas, betas, rels = [], [], []
    if maxit <= 0 or g0 == 0.0:
        f = objective(objective_of(method), X, AX, normA2)
        return IterResult(X, 0, 0.0, g0, f, g0 == 0.0, alphas, betas, rels)
    V = -G
    AV = apply_A(g, V)
    if alpha0 > 0.0:
        alpha = np.full(X.shape[1], alpha0)
    else:
        alpha = step_sizes(g, method, X, V, AX, AV, normA2)
    alphas.append(alpha.copy())
    betas.append(np.zeros(X.shape[1]))
    if record is not None:
        k = X.shape[1]
        record.append(dict(X=X, G=G, V=V, AV=AV, alpha=alpha.copy(), beta=np.zeros(k), den=np.zeros(k),
                           restart=np.zeros(k, dtype=bool)))
    X = X + V * alpha[None, :]
    t = 1
    rel = float("nan")
    converged = False
    while True:
        AX = apply_A(g, X)
        Gn = direction(method, X, AX)
        rel = float(np.linalg.norm(Gn)) / g0
        rels.append(rel)
        if rel <= tol:
            converged = True
            break
        if t >= maxit:
            break
        beta, den = cg_beta(Gn, G)
        restarted = np.zeros(X.shape[1], dtype=bool)
        if restart:
            restarted = -np.sum(Gn * Gn, axis=0) + beta * np.sum(V * Gn, axis=0) >= 0.0
            beta = np.where(restarted, 0.0, beta)
        V = -Gn + V * beta[None, :]
        AV = apply_A(g, V)
        alpha = step_sizes(g, method, X, V, AX, AV, normA2)
        alphas.append(alpha.copy())
        betas.append(beta.copy())
        if record is not None:
            record.append(dict(X=X, G=Gn, V=V, AV=AV, alpha=alpha.copy(), beta=beta.copy(), den=den,
                               restart=restarted))
        X = X + V * alpha[None, :]
        G = Gn
        t += 1
    f = objective(objective_of(method), X, AX, normA2)
    return IterResult(X, t, rel, g0, f, converged, alphas, betas, rels)


# =============================================================================================
# Differentiating through unrolled updates (OFM-f1)
# =============================================================================================

def hess_f1_quarter(g: Graph, Z: np.ndarray, U: np.ndarray) -> np.ndarray:
    """The Hessian of f1/4 at Z applied to U: the derivative of A Z + Z Z^T Z (= grad f1 / 4,
    Eq. (5)) along U, i.e. A U + U Z^T Z + Z U^T Z + Z Z^T U."""
    return apply_A(g, U) + U @ (Z.T @ Z) + Z @ (U.T @ Z) + Z @ (Z.T @ U)


def unrolled_objective(g: Graph, X0: np.ndarray, T: int, restart: bool = False) -> float:
    """L(X_0) = f1(X_T) after T updates of OFM-f1 (Algorithm 2, no stopping test)."""
    r = iterate(g, OFM_F1, X0, 0.0, T, restart=restart)
    return r.f


def unrolled_grad(g: Graph, X0: np.ndarray, T: int, edges=None, restart: bool = False):
    """dL/dX_0 for L = f1(X_T) after T updates of OFM-f1, by reverse accumulation through
    Algorithm 2 as `iterate` runs it. Per update t, X_{t+1} = X_t + alpha_t V_t with
      * alpha_t a root of p(a) = <V_t, grad f1(X_t + a V_t)> / 4 (the cubic of Eq. (15)); by the
        implicit-function theorem d alpha = -(dp at fixed a) / p'(alpha), where
        dp/dX = H(X_{t+1})[V_t], dp/dV = grad f1(X_{t+1})/4 + alpha H(X_{t+1})[V_t] and
        p'(alpha) = <V_t, H(X_{t+1})[V_t]>, H the Hessian of f1/4 (hess_f1_quarter);
      * V_t = -G_t + V_{t-1} diag(beta_t), beta_t,j = <G_t - G_{t-1}, G_t>_j / |G_{t-1},j|^2, with
        beta held at 0 (no derivative) where a zero denominator (or, with the optional restart,
        the restart) set it;
      * G_t = grad f1(X_t) = 4(A X_t + X_t X_t^T X_t), whose derivative along U is 4 H(X_t)[U].
    Returns (L, dL/dX_0), or with edges = (src, dst, w) of a weighted graph (g built from them
    with exact=True) also dL/dw per listing: A enters G_t (adjoint 4 Gbar_t X_t^T), the cubic of
    alpha_t (c V_t X_{t+1}^T, c the implicit-function factor) and f1(X_T) itself; with
    Gamma = dL/dA_hat = -dL/dA symmetrised, the weights follow as in weight_grad."""
    rec: list = []
    res = iterate(g, OFM_F1, X0, 0.0, T, record=rec, restart=restart)
    X = res.X
    pairs = _pairs(g.n, *edges) if edges is not None else None
    gam = None
    if pairs is not None:
        _, _, pa, pb, _, ah = pairs
        gam = 2.0 * (ah - np.sum(X[pa] * X[pb], axis=1))  # f1(X_T) directly

    def finish(f, dX):
        if pairs is None:
            return f, dX
        return f, dX, _weight_chain(g.n, *pairs, gam)

    if not rec:  # T = 0, or X_0 stationary: L = f1(X_0)
        return finish(res.f, gradient(1, X, apply_A(g, X)))
    Gnext = gradient(1, X, apply_A(g, X))  # grad f1(X_T)
    Xbar = Gnext.copy()
    Vbar = np.zeros_like(X)
    Gcarry = np.zeros_like(X)
    Xnext = X
    for t in range(len(rec) - 1, -1, -1):
        r = rec[t]
        V, a = r["V"], float(r["alpha"][0])
        H1 = hess_f1_quarter(g, Xnext, V)
        abar = float(np.sum(Xbar * V))
        c = -abar / float(np.sum(V * H1))
        Vbar = Vbar + a * Xbar + c * (0.25 * Gnext + a * H1)
        Xbar = Xbar + c * H1
        Gt = Gcarry - Vbar
        if t >= 1:
            Gp, Vp = rec[t - 1]["G"], rec[t - 1]["V"]
            bbar = np.sum(Vbar * Vp, axis=0)
            live = (~r["restart"]) & (r["den"] != 0.0)
            den = np.where(live, r["den"], 1.0)
            nbar = np.where(live, bbar / den, 0.0)
            dbar = np.where(live, -bbar * r["beta"] / den, 0.0)
            Gt = Gt + nbar * (2.0 * r["G"] - Gp)
            Gcarry = -nbar * r["G"] + 2.0 * dbar * Gp
            Vbar = Vbar * r["beta"]
        Xbar = Xbar + 4.0 * hess_f1_quarter(g, r["X"], Gt)
        if gam is not None:
            Xt = r["X"]
            gam = gam - 0.5 * (4.0 * (np.sum(Gt[pa] * Xt[pb], axis=1) + np.sum(Gt[pb] * Xt[pa], axis=1))
                               + c * (np.sum(V[pa] * Xnext[pb], axis=1) + np.sum(V[pb] * Xnext[pa], axis=1)))
        Gnext, Xnext = r["G"], r["X"]
    return finish(res.f, Xbar)


# =============================================================================================
# Algorithm 1, steps 3-4: row normalisation and K-means
# =============================================================================================

def row_normalize(X: np.ndarray) -> np.ndarray:
    """Each row divided by its Euclidean norm; zero rows stay zero (Algorithm 1, step 3)."""
    X = np.asarray(X, dtype=np.float64)
    nr = np.sqrt(np.sum(X * X, axis=1))
    out = np.zeros_like(X)
    nz = nr > 0
    out[nz] = X[nz] / nr[nz, None]
    return out


_PHILOX_M0, _PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
_PHILOX_W0, _PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
_M32 = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Philox-4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, SC'11), on Python ints."""
    c0, c1, c2, c3 = (int(x) & _M32 for x in ctr)
    k0, k1 = (int(x) & _M32 for x in key)
    for r in range(10):
        if r:
            k0 = (k0 + _PHILOX_W0) & _M32
            k1 = (k1 + _PHILOX_W1) & _M32
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0, p1 & _M32, (p0 >> 32) ^ c3 ^ k1, p0 & _M32)
    return c0, c1, c2, c3


def kmeans_uniform(seed: int, run: int, draw: int) -> float:
    """The draw-th uniform in [0, 1) of K-means run `run`: word 0 of Philox(ctr, key) / 2^32."""
    out = philox4x32_10((draw, run, 0, 0), (seed & _M32, (seed >> 32) & _M32))
    return out[0] / 4294967296.0


def kmeans_pp_seeds(X: np.ndarray, n_clusters: int, seed: int, run: int) -> np.ndarray:
    """K-means++ seeding (Arthur and Vassilvitskii 2007) with the Philox uniforms above.

    First centre: index floor(u_0 N). Centre c: the first index whose running sum of D^2
    (squared distance to the nearest chosen centre, FP64) exceeds u_c * sum D^2.
    """
    n = X.shape[0]
    idx = [min(int(kmeans_uniform(seed, run, 0) * n), n - 1)]
    d2 = np.sum((X - X[idx[0]]) ** 2, axis=1)
    for c in range(1, n_clusters):
        total = float(np.sum(d2))
        if total <= 0.0:
            j = min(int(kmeans_uniform(seed, run, c) * n), n - 1)
        else:
            target = kmeans_uniform(seed, run, c) * total
            j = int(np.searchsorted(np.cumsum(d2), target, side="right"))
            j = min(j, n - 1)
        idx.append(j)
        d2 = np.minimum(d2, np.sum((X - X[j]) ** 2, axis=1))
    return np.array(idx)


def kmeans(X: np.ndarray, n_clusters: int, seed: int, n_init: int = 1, maxit: int = 300):
    """Euclidean K-means (Algorithm 1, step 4): K-means++ seeding, then Lloyd iterations.

    Lloyd: assign each point to the nearest centroid (ties: lowest index); stop when no label
    changes or after maxit assignments; centroid = mean of its points; an empty cluster takes
    the point farthest from its own centroid (ties: lowest index), each such point used once.
    Of n_init runs the lowest inertia wins (ties: the earlier run).
    Returns (labels int32, inertia float).
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    best = None
    for run in range(n_init):
        mu = X[kmeans_pp_seeds(X, n_clusters, seed, run)].copy()
        lab = None
        for _ in range(maxit):
            d = np.stack([np.sum((X - mu[c]) ** 2, axis=1) for c in range(n_clusters)], axis=1)
            new = np.argmin(d, axis=1)
            if lab is not None and np.array_equal(new, lab):
                break
            lab = new
            dist_own = d[np.arange(n), lab]
            taken = np.zeros(n, dtype=bool)
            for c in range(n_clusters):
                members = lab == c
                if members.any():
                    mu[c] = X[members].mean(axis=0)
                else:
                    cand = np.where(taken, -1.0, dist_own)
                    j = int(np.argmax(cand))
                    taken[j] = True
                    mu[c] = X[j]
        d = np.stack([np.sum((X - mu[c]) ** 2, axis=1) for c in range(n_clusters)], axis=1)
        lab = np.argmin(d, axis=1)
        inertia = float(np.sum(d[np.arange(n), lab]))
        if best is None or inertia < best[1]:
            best = (lab.astype(np.int32), inertia)
    return best


# =============================================================================================
# Evaluation (Sec. 5): ARI, principal angles, Rayleigh-Ritz relerr
# =============================================================================================

def _comb2(x):
    x = np.asarray(x, dtype=np.float64)
    return x * (x - 1.0) / 2.0


def ari(a: np.ndarray, b: np.ndarray) -> float:
    """Adjusted Rand index (Hubert and Arabie 1985) from the contingency table."""
    a = np.asarray(a)
    b = np.asarray(b)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    table = np.zeros((ai.max() + 1, bi.max() + 1))
    np.add.at(table, (ai, bi), 1.0)
    sum_ij = _comb2(table).sum()
    sum_a = _comb2(table.sum(axis=1)).sum()
    sum_b = _comb2(table.sum(axis=0)).sum()
    total = _comb2(len(a))
    expected = sum_a * sum_b / total if total > 0 else 0.0
    maxidx = 0.5 * (sum_a + sum_b)
    if maxidx == expected:
        return 1.0
    return float((sum_ij - expected) / (maxidx - expected))


def subspace_sin(X1: np.ndarray, X2: np.ndarray) -> float:
    """sin of the largest principal angle between span(X1) and span(X2): ||(I - Q1Q1^T)Q2||_2."""
    Q1, _ = np.linalg.qr(np.asarray(X1, dtype=np.float64))
    Q2, _ = np.linalg.qr(np.asarray(X2, dtype=np.float64))
    M = Q2 - Q1 @ (Q1.T @ Q2)
    return float(np.linalg.norm(M, 2))


def rayleigh_ritz_relerr(g: Graph, X: np.ndarray):
    """Ritz pairs of B = 2I - L = -A on span(X) and relerr = ||B U - U Lam||_F / ||U Lam||_F (Sec. 5).

    Orthonormalise X (QR), form the k x k projection U^T B U, diagonalise it, rotate.
    Returns (ritz values of B ascending, relerr).
    """
    Q, _ = np.linalg.qr(np.asarray(X, dtype=np.float64))
    BQ = -apply_A(g, Q)
    H = Q.T @ BQ
    lam, Z = np.linalg.eigh(0.5 * (H + H.T))
    U = Q @ Z
    BU = BQ @ Z
    res = BU - U * lam[None, :]
    return lam, float(np.linalg.norm(res) / np.linalg.norm(U * lam[None, :]))
