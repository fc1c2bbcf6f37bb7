"""Thin Python binding of the ofsc C ABI (include/ofsc.h): argument marshalling only.

Every computation runs in libofsc.so. Arrays are passed as device pointers taken from objects
with a ``data_ptr()`` method (torch CUDA tensors); streams as the raw cudaStream_t of a torch
stream. If the library has not been built, every call raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libofsc.so")
# OFSC_LIB (an absolute path) selects another build of the library, e.g. the checked build
# libofsc_debug.so; it is read when this module is imported.
if os.environ.get("OFSC_LIB"):
    LIB_PATH = os.environ["OFSC_LIB"]
HEADER = os.path.join(os.path.dirname(_PKG), "include", "ofsc.h")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_NONFINITE, ERR_TIMEOUT, ERR_NOT_CONVERGED, ERR_CUDA = range(7)
OFM_F1, TRI_F1, OFM_F2, TRI_F2 = 0, 1, 2, 3
F1, F2 = 1, 2
GATHER_FP32, GATHER_BF16 = 0, 1
GRAM_AUTO, GRAM_SIMT, GRAM_TC = 0, 1, 2
SPMM_AUTO, SPMM_SIMT, SPMM_TMA = 0, 1, 2
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "NONFINITE", 4: "TIMEOUT",
                5: "NOT_CONVERGED", 6: "CUDA"}


class OfscError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"ofsc status {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("m_in", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("n_selfloops", ctypes.c_int64), ("n_duplicates", ctypes.c_int64),
                ("n_isolated", ctypes.c_int64), ("weighted", ctypes.c_int32),
                ("normA_fro2", ctypes.c_double)]


PHASES = ["direction", "beta", "spmm", "gram", "gram_reduce", "linesearch", "refresh", "other"]


class Profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(PHASES)), ("launches", ctypes.c_int64 * len(PHASES))]

    def as_dict(self) -> dict:
        return {p: {"ms": self.ms[i], "launches": int(self.launches[i])} for i, p in enumerate(PHASES)}


class Opts(ctypes.Structure):
    _fields_ = [("gather", ctypes.c_int32), ("y_refresh", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("alpha0", ctypes.c_double),
                ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_int32),
                ("profile", ctypes.POINTER(Profile)), ("gram_engine", ctypes.c_int32),
                ("spmm_engine", ctypes.c_int32), ("direct_launch", ctypes.c_int32),
                ("cg_restart", ctypes.c_int32), ("refine_tol", ctypes.c_double),
                ("exact_tail", ctypes.c_double), ("vscale_exp", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("withhold_arrivals", ctypes.c_int32),
                ("merge_path", ctypes.c_int32), ("group_launches", ctypes.c_int32),
                ("state", ctypes.c_void_p), ("overlap_gram", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rel_dir_norm", ctypes.c_double), ("g0_norm", ctypes.c_double),
                ("f", ctypes.c_double), ("kernel_launches", ctypes.c_int64), ("refined_at", ctypes.c_int32),
                ("exact_at", ctypes.c_int32)]


_lib = None

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
_allocator = None  # the ctypes callbacks in use (kept alive while the library may call them)


def header_functions() -> list[str]:
    """Names of the functions that include/ofsc.h declares."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(ofsc_\w+)\s*\(", text, re.M)))


def lib() -> ctypes.CDLL:
    """The loaded libofsc.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OfscError(ERR_CUDA, f"{LIB_PATH} is missing: build it with "
                                      "paper_2305_10356_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double)
        sig = {
            "ofsc_graph_build": [i64, i64, vp, vp, vp, u32, vp, ctypes.POINTER(vp)],
            "ofsc_graph_free": [vp],
            "ofsc_graph_get_info": [vp, ctypes.POINTER(GraphInfo)],
            "ofsc_graph_csr": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                               ctypes.POINTER(vp), ctypes.POINTER(vp)],
            "ofsc_objective_grad": [vp, i32, i32, vp, ctypes.POINTER(dbl), vp, vp],
            "ofsc_objective_grad_noalloc": [vp, i32, i32, vp, ctypes.POINTER(dbl), vp, vp],
            "ofsc_iterate": [vp, i32, i32, vp, dbl, i32, ctypes.POINTER(Opts),
                             ctypes.POINTER(Result), vp],
            "ofsc_iterate_batched": [i32, ctypes.POINTER(vp), i32, ctypes.POINTER(i32), ctypes.POINTER(vp), dbl,
                                     i32, ctypes.POINTER(Opts), ctypes.POINTER(Result), vp],
            "ofsc_rayleigh_ritz": [vp, i32, vp, vp, ctypes.POINTER(dbl), vp],
            "ofsc_unrolled_grad": [vp, i32, vp, i32, i32, i64, vp, vp, ctypes.POINTER(dbl), vp, vp, vp],
            "ofsc_autotune": [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                              ctypes.POINTER(dbl), vp],
            "ofsc_weight_grad": [vp, i32, i32, vp, i64, vp, vp, vp, vp],
            "ofsc_row_normalize": [i64, i32, vp, vp],
            "ofsc_gram": [i64, i32, i32, vp, i32, ctypes.POINTER(vp), i64, vp, vp],
            "ofsc_kmeans": [i64, i32, vp, i32, u64, i32, i32, vp, ctypes.POINTER(dbl), vp],
            "ofsc_set_allocator": [ALLOC_FN, FREE_FN, vp],
            "ofsc_state_create": [vp, i32, ctypes.POINTER(vp)],
            "ofsc_state_free": [vp],
            "ofsc_state_info": [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)],
            "ofsc_state_save": [vp, vp, i64, vp],
            "ofsc_state_load": [vp, vp, i64, vp],
            "ofsc_line_search_step": [i64, vp, i32, vp, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = i32
        L.ofsc_last_error.argtypes = []
        L.ofsc_last_error.restype = ctypes.c_char_p
        L.ofsc_version.argtypes = []
        L.ofsc_version.restype = i32
        _lib = L
    return _lib


class _DeviceArray:
    """Exposes a raw device pointer through __cuda_array_interface__ (zero copy)."""

    def __init__(self, ptr: int, shape: tuple, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2}


def device_view(ptr: int, shape: tuple, typestr: str):
    """A torch CUDA tensor viewing device memory owned by the library (no copy)."""
    import torch
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device="cuda")


def _check(status: int, allow=(OK,)) -> int:
    if status not in allow:
        raise OfscError(status, lib().ofsc_last_error().decode())
    return status


def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def _arg(t, name: str, dtype: str, rows: int | None = None, numel: int | None = None, like=None) -> int | None:
    """Device pointer of a tensor argument after the checks the C ABI cannot make on a raw pointer:
    a contiguous CUDA tensor of the expected dtype and size (None passes through)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise OfscError(ERR_INVALID_ARG, f"{name}: a torch tensor is required")
    if t.dtype != getattr(torch, dtype):
        raise OfscError(ERR_INVALID_ARG, f"{name}: dtype {t.dtype}, expected torch.{dtype}")
    if not t.is_contiguous():
        raise OfscError(ERR_INVALID_ARG, f"{name}: must be contiguous")
    if not t.is_cuda:
        raise OfscError(ERR_INVALID_ARG, f"{name}: must be a CUDA tensor")
    if rows is not None and (t.dim() != 2 or t.shape[0] != rows):
        raise OfscError(ERR_INVALID_ARG, f"{name}: shape {tuple(t.shape)}, expected {rows} rows")
    if numel is not None and t.numel() != numel:
        raise OfscError(ERR_INVALID_ARG, f"{name}: {t.numel()} elements, expected {numel}")
    if like is not None and tuple(t.shape) != tuple(like.shape):
        raise OfscError(ERR_INVALID_ARG, f"{name}: shape {tuple(t.shape)}, expected {tuple(like.shape)}")
    return int(t.data_ptr())


def _rows(g) -> int:
    return int(g.info().n)


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    return int(getattr(stream, "cuda_stream", stream))


class Graph:
    """Owns an ofsc_graph handle (freed with the object)."""

    def __init__(self, handle: int):
        self.handle = ctypes.c_void_p(handle)

    def info(self) -> GraphInfo:
        inf = GraphInfo()
        _check(lib().ofsc_graph_get_info(self.handle, ctypes.byref(inf)))
        return inf

    def csr(self) -> dict:
        """Device pointers of the CSR arrays (owned by the handle)."""
        ptrs = [ctypes.c_void_p() for _ in range(5)]
        _check(lib().ofsc_graph_csr(self.handle, *[ctypes.byref(p) for p in ptrs]))
        return dict(zip(["row_ptr", "col", "val", "dinv", "deg"], [p.value for p in ptrs]))

    def free(self):
        if self.handle is not None and self.handle.value:
            lib().ofsc_graph_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ofsc_graph_build(n: int, src, dst, w=None, stream=None) -> Graph:
    """S, D and D^-1/2 (Eq. (1)) from device int32 edge arrays (and optional FP32 weights)."""
    h = ctypes.c_void_p()
    m = 0 if src is None else int(src.numel())
    ps, pd = _arg(src, "src", "int32"), _arg(dst, "dst", "int32", numel=m)
    pw = _arg(w, "w", "float32", numel=m)
    _check(lib().ofsc_graph_build(n, m, ps, pd, pw, 0, _stream(stream), ctypes.byref(h)))
    return Graph(h.value)


def ofsc_objective_grad(g: Graph, objective: int, X, G_out=None, stream=None) -> float:
    """f (Eq. (2)/(3)) at the device block X (n x k, FP32); the gradient goes to G_out if given."""
    f = ctypes.c_double()
    px = _arg(X, "X", "float32", rows=_rows(g))
    _check(lib().ofsc_objective_grad(g.handle, objective, int(X.shape[1]), px,
                                     ctypes.byref(f), _arg(G_out, "G_out", "float32", like=X), _stream(stream)))
    return f.value


def ofsc_objective_grad_noalloc(g: Graph, objective: int, X, G_out=None, stream=None) -> float:
    """As ofsc_objective_grad, with no device allocation (static scratch; n * kp <= 2^20)."""
    f = ctypes.c_double()
    px = _arg(X, "X", "float32", rows=_rows(g))
    _check(lib().ofsc_objective_grad_noalloc(g.handle, objective, int(X.shape[1]), px,
                                             ctypes.byref(f), _arg(G_out, "G_out", "float32", like=X),
                                             _stream(stream)))
    return f.value


def ofsc_iterate(g: Graph, method: int, X, tol: float, maxit: int, *, gather: int = GATHER_FP32,
                 y_refresh: int = 0, check_every: int = 0, alpha0: float = 0.0, trace=None,
                 profile: Profile | None = None, gram_engine: int = GRAM_AUTO,
                 spmm_engine: int = SPMM_AUTO, cg_restart: bool = False, refine_tol: float = 0.0,
                 exact_tail: float = 0.0, vscale_exp: int = 0, direct_launch: bool = False,
                 spin_limit: int = 0, withhold_arrivals: bool = False, merge_path: int = 0,
                 group_launches: int = 0, state: "State | None" = None, overlap_gram: int = 0,
                 stream=None) -> Result:
    """Algorithm 2 in place on the device block X (n x k, FP32). Returns the ofsc_result. With a
    State, the call continues the run the state holds and leaves its own state in it."""
    px = _arg(X, "X", "float32", rows=_rows(g))
    o = Opts(gather, y_refresh, check_every, alpha0, _arg(trace, "trace", "float64"),
             0 if trace is None else int(trace.shape[0]),
             ctypes.pointer(profile) if profile is not None else None, gram_engine, spmm_engine,
             1 if direct_launch else 0, 1 if cg_restart else 0, float(refine_tol), float(exact_tail),
             int(vscale_exp), int(spin_limit), 1 if withhold_arrivals else 0, int(merge_path),
             int(group_launches), None if state is None else state.handle, int(overlap_gram))
    r = Result()
    _check(lib().ofsc_iterate(g.handle, method, int(X.shape[1]), px, float(tol), int(maxit),
                              ctypes.byref(o), ctypes.byref(r), _stream(stream)),
           allow=(OK, ERR_NOT_CONVERGED))
    return r


def ofsc_iterate_batched(graphs: list[Graph], method: int, Xs: list, tol: float, maxit: int, *,
                         gather: int = GATHER_FP32, y_refresh: int = 0, check_every: int = 0,
                         alpha0: float = 0.0, gram_engine: int = GRAM_AUTO, spmm_engine: int = SPMM_AUTO,
                         direct_launch: bool = False, cg_restart: bool = False, refine_tol: float = 0.0,
                         exact_tail: float = 0.0, vscale_exp: int = 0, merge_path: int = 0,
                         group_launches: int = 0, state=None, overlap_gram: int = 0,
                         stream=None) -> list[Result]:
    """Algorithm 2 in place on every device block Xs[i] (n_i x k_i, FP32) of the graphs, in one
    call. Returns one ofsc_result per problem, in order."""
    count = len(graphs)
    if len(Xs) != count:
        raise ValueError("ofsc_iterate_batched: one X per graph")
    o = Opts(gather, y_refresh, check_every, alpha0, None, 0, None, gram_engine, spmm_engine,
             1 if direct_launch else 0, 1 if cg_restart else 0, float(refine_tol), float(exact_tail),
             int(vscale_exp), 0, 0, int(merge_path), int(group_launches),
             None if state is None else state.handle, int(overlap_gram))
    hs = (ctypes.c_void_p * count)(*[g.handle for g in graphs])
    ks = (ctypes.c_int32 * count)(*[int(X.shape[1]) for X in Xs])
    xs = (ctypes.c_void_p * count)(*[_arg(X, f"Xs[{i}]", "float32", rows=_rows(g))
                                     for i, (g, X) in enumerate(zip(graphs, Xs))])
    rs = (Result * count)()
    _check(lib().ofsc_iterate_batched(count, hs, method, ks, xs, float(tol), int(maxit), ctypes.byref(o), rs,
                                      _stream(stream)),
           allow=(OK, ERR_NOT_CONVERGED))
    return list(rs)


def ofsc_gram(L, Rs, out, k: int | None = None, rows_per_block: int = 0, stream=None) -> None:
    """out[b] = L^T Rs[b] (FP64 [nr, k, k]) on the tensor cores; L and Rs[b] are n x ld FP32."""
    n, ld = int(L.shape[0]), int(L.shape[1])
    arr = (ctypes.c_void_p * len(Rs))(*[_arg(r, f"Rs[{b}]", "float32", like=L) for b, r in enumerate(Rs)])
    _check(lib().ofsc_gram(n, ld if k is None else k, ld, _arg(L, "L", "float32"), len(Rs), arr, rows_per_block,
                           _arg(out, "out", "float64"), _stream(stream)))


def ofsc_autotune(g: Graph, k: int, gather: int = GATHER_FP32, stream=None,
                  with_merge: bool = False) -> tuple:
    """Times the direction product at several row partitions and gathers in flight per lane, and
    the merge-path split at each partition; keeps the fastest in the handle. Returns (warps, slots
    per lane, ms per product), or (warps, slots, merge path chosen, ms) with with_merge."""
    w = ctypes.c_int32(0)
    u = ctypes.c_int32(0)
    mp = ctypes.c_int32(0)
    ms = ctypes.c_double(0.0)
    _check(lib().ofsc_autotune(g.handle, int(k), int(gather), ctypes.byref(w), ctypes.byref(u), ctypes.byref(mp),
                               ctypes.byref(ms), _stream(stream)))
    if with_merge:
        return w.value, u.value, bool(mp.value), ms.value
    return w.value, u.value, ms.value


def ofsc_unrolled_grad(g: Graph, X0, T: int, grad=None, ckpt: int = 0, src=None, dst=None, grad_w=None,
                       stream=None) -> float:
    """d f1(X_T) / d X_0 through T updates of OFM-f1 into the device block grad (n x k, FP32), and
    d f1(X_T) / d w into grad_w (one FP32 per listed edge of src, dst) for a weighted graph;
    returns f1(X_T)."""
    f = ctypes.c_double(0.0)
    m = 0 if src is None else int(src.numel())
    px = _arg(X0, "X0", "float32", rows=_rows(g))
    _check(lib().ofsc_unrolled_grad(g.handle, int(X0.shape[1]), px, int(T), int(ckpt), m,
                                    _arg(src, "src", "int32"), _arg(dst, "dst", "int32", numel=m),
                                    ctypes.byref(f), _arg(grad, "grad", "float32", like=X0),
                                    _arg(grad_w, "grad_w", "float32", numel=m), _stream(stream)))
    return f.value


def ofsc_weight_grad(g: Graph, objective: int, X, src, dst, grad, stream=None) -> None:
    """d f / d w for every listed edge (device int32 src, dst; device float32 grad) of a weighted graph."""
    m = int(src.numel())
    _check(lib().ofsc_weight_grad(g.handle, objective, int(X.shape[1]), _arg(X, "X", "float32", rows=_rows(g)), m,
                                  _arg(src, "src", "int32"), _arg(dst, "dst", "int32", numel=m),
                                  _arg(grad, "grad", "float32", numel=m), _stream(stream)))


_OBJ_GRAPHS: dict = {}  # graphs of objective(): key -> (Graph, src, dst, w), most recent last
_OBJ_GRAPHS_MAX = 4


def _objective_graph(n: int, src, dst, w) -> "Graph":
    """The graph of (src, dst, w), built once and reused while the same tensors are passed again
    unchanged (same objects, same in-place version counters; the cache holds references to them,
    so their memory cannot be reused by other tensors meanwhile)."""
    key = (int(n), src.data_ptr(), src._version, dst.data_ptr(), dst._version,
           None if w is None else (w.data_ptr(), w._version))
    hit = _OBJ_GRAPHS.get(key)
    if hit is not None and hit[1] is src and hit[2] is dst and hit[3] is w:
        _OBJ_GRAPHS[key] = _OBJ_GRAPHS.pop(key)
        return hit[0]
    g = ofsc_graph_build(n, src, dst, w)
    _OBJ_GRAPHS[key] = (g, src, dst, w)
    while len(_OBJ_GRAPHS) > _OBJ_GRAPHS_MAX:
        _OBJ_GRAPHS.pop(next(iter(_OBJ_GRAPHS)))
    return g


def objective(X, w, src, dst, n: int, which: int = 1):
    """f1 (which=1) or f2 (which=2) of the graph with edge list (src, dst) and weights w at the
    feature block X, as a differentiable scalar (float64): backward gives df/dX (Eqs. (5), (10))
    and df/dw (ofsc_weight_grad). All tensors on one CUDA device; X float32 [n x k], w float32 [m]."""
    import torch

    class _Objective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, X, w):
            g = _objective_graph(n, src, dst, w)
            G = torch.empty_like(X)
            f = ofsc_objective_grad(g, which, X, G)
            ctx.g = g
            ctx.save_for_backward(X, G)
            return torch.tensor(f, dtype=torch.float64, device=X.device)

        @staticmethod
        def backward(ctx, gf):
            X, G = ctx.saved_tensors
            gX = gw = None
            if ctx.needs_input_grad[0]:
                gX = G * gf.to(G.dtype)
            if ctx.needs_input_grad[1]:
                gw = torch.empty(src.shape[0], dtype=torch.float32, device=X.device)
                ofsc_weight_grad(ctx.g, which, X, src, dst, gw)
                gw = gw * gf.to(gw.dtype)
            return gX, gw

    return _Objective.apply(X, w)


class State:
    """The CG state of Algorithm 2 between ofsc_iterate calls on one graph with k columns
    (ofsc_state_create): resume a run exactly, or checkpoint it to host memory."""

    def __init__(self, g: Graph, k: int):
        self.handle = ctypes.c_void_p()
        _check(lib().ofsc_state_create(g.handle, int(k), ctypes.byref(self.handle)))

    def info(self) -> tuple[int, int]:
        """(updates of the run it holds, 0 if empty; bytes of its host image)."""
        t, b = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(lib().ofsc_state_info(self.handle, ctypes.byref(t), ctypes.byref(b)))
        return t.value, b.value

    def save(self, stream=None) -> bytes:
        """The state's host image (a checkpoint)."""
        _, nbytes = self.info()
        buf = ctypes.create_string_buffer(nbytes)
        _check(lib().ofsc_state_save(self.handle, ctypes.cast(buf, ctypes.c_void_p), nbytes, _stream(stream)))
        return buf.raw

    def load(self, image: bytes, stream=None) -> None:
        """Replaces the state by a host image of a state of the same n and k."""
        buf = ctypes.create_string_buffer(bytes(image), len(image))
        _check(lib().ofsc_state_load(self.handle, ctypes.cast(buf, ctypes.c_void_p), len(image), _stream(stream)))

    def free(self):
        if self.handle is not None and self.handle.value:
            lib().ofsc_state_free(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def ofsc_rayleigh_ritz(g: Graph, X, ritz, stream=None) -> float:
    """Ritz values of B = 2I - L on span(X) into the device float64 vector `ritz` (ascending) and
    the relative residual relerr of Sec. 5, returned."""
    out = ctypes.c_double(0.0)
    _check(lib().ofsc_rayleigh_ritz(g.handle, int(X.shape[1]), _arg(X, "X", "float32", rows=_rows(g)),
                                    _arg(ritz, "ritz", "float64", numel=int(X.shape[1])), ctypes.byref(out),
                                    _stream(stream)))
    return float(out.value)


def ofsc_set_allocator(alloc=None, free=None) -> None:
    """Every device block the library allocates from now on comes from alloc(bytes) -> int device
    pointer (0 when it cannot) and goes back through free(ptr); both None: cudaMalloc again."""
    global _allocator
    if (alloc is None) != (free is None):
        raise OfscError(ERR_INVALID_ARG, "ofsc_set_allocator: give both functions or neither")
    if alloc is None:
        cb = (ALLOC_FN(), FREE_FN())
    else:
        cb = (ALLOC_FN(lambda nbytes, user: int(alloc(int(nbytes)) or 0)),
              FREE_FN(lambda ptr, user: free(int(ptr))))
    _check(lib().ofsc_set_allocator(cb[0], cb[1], None))
    # callbacks of blocks still owned by the library must outlive them: keep every pair set
    _allocator = (_allocator or ()) + (cb,)


def ofsc_line_search_step(coef, steps, bad=None, solver: int = 1, stream=None) -> None:
    """The exact line search's step (Sec. 3.2) of each cubic coef[i] = (c3, c2, c1, c0) (device
    FP64 [n, 4]) into steps (device FP64 [n]); bad (device int32 [n] or None) marks cubics with a
    coefficient that is not finite. solver 0: one thread per cubic; 1: one warp per cubic."""
    pc = _arg(coef, "coef", "float64")
    if coef.dim() != 2 or coef.shape[1] != 4:
        raise OfscError(ERR_INVALID_ARG, f"coef: shape {tuple(coef.shape)}, expected (n, 4)")
    n = int(coef.shape[0])
    _check(lib().ofsc_line_search_step(n, pc, int(solver),
                                       _arg(steps, "steps", "float64", numel=n),
                                       None if bad is None else _arg(bad, "bad", "int32", numel=n), _stream(stream)))


def ofsc_row_normalize(X, stream=None) -> None:
    """Row normalisation in place (Algorithm 1, step 3)."""
    _check(lib().ofsc_row_normalize(int(X.shape[0]), int(X.shape[1]), _arg(X, "X", "float32"), _stream(stream)))


def ofsc_kmeans(X, n_clusters: int, labels, seed: int = 0, n_init: int = 1, maxit: int = 300,
                stream=None) -> float:
    """K-means on the rows of X into the device int32 array `labels`; returns the inertia."""
    inertia = ctypes.c_double()
    _check(lib().ofsc_kmeans(int(X.shape[0]), int(X.shape[1]), _arg(X, "X", "float32"), n_clusters, seed, n_init,
                             maxit, _arg(labels, "labels", "int32", numel=int(X.shape[0])), ctypes.byref(inertia),
                             _stream(stream)))
    return inertia.value
