"""The checked build (OFSC_DEBUG): the direction product checks every column index and row range
before it uses them, records the first violation instead of making the access, and the calls
that ran it return OFSC_ERR_INVALID_ARG naming it.

CPU: the checked units compile for sm_103a. GPU: the checked library, loaded in a child process
through OFSC_LIB, gives the release library's results bit for bit; a column index planted outside
[0, n) in its CSR makes ofsc_iterate fail with the bounds message (the access is skipped, so
nothing faults), and the same process then runs a fresh graph normally."""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest

from paper_2305_10356_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_units_compile():
    """The units that hold the checks (the direction product and the calls reporting it) compile
    with -DOFSC_DEBUG=1 (no link: a full checked build runs in the GPU test)."""
    with tempfile.TemporaryDirectory() as tmp:
        procs = []
        for src in ("spmm_dir.cu", "iterate.cu"):
            cmd = [build.nvcc(), *build.ARCH, *build.FLAGS, "-DOFSC_DEBUG=1", "-c",
                   os.path.join(build.CSRC, src), "-o", os.path.join(tmp, src + ".o")]
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)))
        for src, p in procs:
            out, err = p.communicate(timeout=600)
            assert p.returncode == 0, f"{src}:\n{out}\n{err}"


CHILD = r'''
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_2305_10356_gb300 import ofsc, synth

def graph(e):
    return ofsc.ofsc_graph_build(e.n, torch.from_numpy(e.src).cuda(), torch.from_numpy(e.dst).cuda())

out = {"lib": ofsc.LIB_PATH}
e = synth.sbm(3000, 6, 16.0, 5.0, ratio_kind="count", seed=240)
x0 = synth.initial_block(e.n, 24, 241)
g = graph(e)
X = torch.from_numpy(x0).cuda()
r = ofsc.ofsc_iterate(g, 0, X, 0.0, 5)
np.save(OUT_X, X.cpu().numpy())
out["iterations"] = r.iterations
# a column index outside [0, n) planted in the graph's CSR
nnz = int(g.info().nnz)
col = ofsc.device_view(g.csr()["col"], (nnz,), "<i4")
col[nnz // 2] = e.n + 5
torch.cuda.synchronize()
X = torch.from_numpy(x0).cuda()
try:
    ofsc.ofsc_iterate(g, 0, X, 0.0, 5)
    out["planted"] = "no error"
except ofsc.OfscError as err:
    out["planted"] = [err.status, str(err)]
# the process goes on: a fresh graph runs normally
g2 = graph(e)
X = torch.from_numpy(x0).cuda()
r = ofsc.ofsc_iterate(g2, 0, X, 0.0, 5)
out["after"] = [r.iterations, bool(np.isfinite(X.cpu().numpy()).all())]
print(json.dumps(out))
'''


@pytest.mark.gpu
def test_checked_build_matches_release_and_reports_bad_indices():
    import torch
    from paper_2305_10356_gb300 import ofsc, synth
    assert torch.cuda.is_available()
    build.build()
    dbg = build.build(debug=True)
    with tempfile.TemporaryDirectory() as tmp:
        out_x = os.path.join(tmp, "x_checked.npy")
        code = CHILD.replace("ROOT", repr(ROOT)).replace("OUT_X", repr(out_x))
        env = dict(os.environ, OFSC_LIB=dbg)
        p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
        assert p.returncode == 0, p.stdout + p.stderr
        res = json.loads(p.stdout.strip().splitlines()[-1])
        assert res["lib"] == dbg
        # release library, same run, in this process
        e = synth.sbm(3000, 6, 16.0, 5.0, ratio_kind="count", seed=240)
        x0 = synth.initial_block(e.n, 24, 241)
        g = ofsc.ofsc_graph_build(e.n, torch.from_numpy(e.src).cuda(), torch.from_numpy(e.dst).cuda())
        X = torch.from_numpy(x0).cuda()
        r = ofsc.ofsc_iterate(g, 0, X, 0.0, 5)
        assert res["iterations"] == r.iterations == 5
        assert np.array_equal(np.load(out_x), X.cpu().numpy())
    status, msg = res["planted"]
    assert status == ofsc.ERR_INVALID_ARG and "bounds check: column index" in msg and str(e.n + 5) in msg
    assert res["after"] == [5, True]
