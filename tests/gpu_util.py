"""Helpers shared by the GPU parity tests: device uploads and host copies of library-owned arrays."""
import numpy as np

from paper_2305_10356_gb300 import ofsc


def upload(edges):
    import torch
    src = torch.from_numpy(np.ascontiguousarray(edges.src)).cuda()
    dst = torch.from_numpy(np.ascontiguousarray(edges.dst)).cuda()
    w = None if edges.w is None else torch.from_numpy(np.ascontiguousarray(edges.w)).cuda()
    return src, dst, w


def gpu_graph(edges):
    src, dst, w = upload(edges)
    return ofsc.ofsc_graph_build(edges.n, src, dst, w)


def csr_host(g):
    """Host numpy copies of the CSR, D^-1/2 and D held by a graph handle."""
    import torch
    inf = g.info()
    p = g.csr()
    n, nnz = int(inf.n), int(inf.nnz)
    out = {"row_ptr": ofsc.device_view(p["row_ptr"], (n + 1,), "<i8").cpu().numpy(),
           "dinv": ofsc.device_view(p["dinv"], (n,), "<f4").cpu().numpy() if n else np.zeros(0, np.float32),
           "deg": ofsc.device_view(p["deg"], (n,), "<f8").cpu().numpy() if n else np.zeros(0)}
    out["col"] = (ofsc.device_view(p["col"], (nnz,), "<i4").cpu().numpy() if nnz
                  else np.zeros(0, np.int32))
    out["val"] = (ofsc.device_view(p["val"], (nnz,), "<f4").cpu().numpy()
                  if (nnz and p["val"]) else None)
    torch.cuda.synchronize()
    return out


def run_iterate(g, method, x0, tol, maxit, trace_cap=0, **kw):
    """Runs ofsc_iterate on a copy of x0; returns (X numpy, result, trace numpy or None)."""
    import torch
    X = torch.from_numpy(np.ascontiguousarray(x0, dtype=np.float32)).cuda()
    tr = None
    if trace_cap:
        tr = torch.zeros((trace_cap, 3 + 2 * x0.shape[1]), dtype=torch.float64, device="cuda")
    r = ofsc.ofsc_iterate(g, method, X, tol, maxit, trace=tr, **kw)
    torch.cuda.synchronize()
    return X.cpu().numpy(), r, (None if tr is None else tr.cpu().numpy())


def assert_elementwise(got, ref, rtol, what=""):
    """Element by element: |got - ref| <= rtol (|ref| + max|ref|) for every entry (the absolute
    part keeps entries near zero to the block's own scale), so a few bad rows cannot hide inside a
    norm ratio."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = float(np.abs(ref).max()) if ref.size else 0.0
    np.testing.assert_allclose(got, ref, rtol=rtol, atol=rtol * scale, err_msg=what)
