"""Host-side pieces of bench.py (CPU): the direction product's byte model, the traffic lookup that
is keyed to the kernel sources, and the single-rank timing helper."""
import json
import os

import bench


def test_spmm_byte_model():
    """CSR (int64 row pointers, int32 columns, FP32 weights when weighted) + gathered rows that
    miss L2 + the epilogue read of V and D^-1/2 + the write of W."""
    n, kp, nnz = 1000, 128, 30_000
    b = bench.spmm_bytes(n, kp, nnz, 2, False, 0.25)
    assert b["csr"] == 8 * (n + 1) + 4 * nnz
    assert b["gather_all"] == nnz * kp * 2 and b["gather"] == int(0.75 * nnz * kp * 2)
    assert b["epilogue"] == 4 * n * kp + 4 * n and b["write"] == 4 * n * kp
    assert b["total"] == b["csr"] + b["gather"] + b["epilogue"] + b["write"]
    assert bench.spmm_bytes(n, kp, nnz, 2, True, 0.25)["csr"] == b["csr"] + 4 * nnz


def test_traffic_is_keyed_to_the_kernel_sources(tmp_path, monkeypatch):
    """An entry taken on other kernel sources is not this build's traffic (None), but is still
    returned on request for the cost model's L2 hit rate."""
    (tmp_path / "profiles").mkdir()
    entry = {"dram_read_bytes": 10, "dram_write_bytes": 2, "source_digest": "not-this-build"}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"entries": {"w/bf16": entry}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_digest", lambda names=None: "this-build")
    assert bench.measured_traffic("w", "bf16") is None
    assert bench.measured_traffic("w", "bf16", any_build=True)["dram_read_bytes"] == 10
    entry["source_digest"] = "this-build"
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"entries": {"w/bf16": entry}}))
    assert bench.measured_traffic("w", "bf16")["dram_write_bytes"] == 2
    assert bench.measured_traffic("w", "fp32") is None


def test_source_digest_covers_the_kernel_sources():
    d = bench.source_digest()
    assert len(d) == 16 and d == bench.source_digest()
    assert os.path.isdir(os.path.join(bench.ROOT, "paper_2305_10356_gb300", "csrc"))
    # the direction product's own digest covers its translation unit and the shared header only
    dp = bench.source_digest(bench.DIR_PRODUCT_SOURCES)
    assert len(dp) == 16 and dp != d


def test_max_over_ranks_single_rank():
    assert bench.max_over_ranks(3.25, 1) == 3.25
