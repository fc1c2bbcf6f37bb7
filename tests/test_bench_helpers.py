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


def test_l2_flush_rule_and_config_note():
    """The steps flush the L2 unless every N x kp block and the CSR are each more than twice its
    size: the 2M-node graph keeps its inputs larger than L2, the smaller workloads flush, and the
    config's note says which, for both arms."""
    import argparse

    def args(workload, nodes=None):
        return argparse.Namespace(workload=workload, nodes=nodes, method="ofm_f1", gather="bf16", iters=30)

    assert not bench.l2_flushed(args("dcsbm_n2m_k128"))
    for wl in ("sbm_n1000_k11", "dcsbm_n50k_k44", "wsbm_n20k_k32"):
        assert bench.l2_flushed(args(wl))
        assert bench.workload_config(args(wl))["l2"].startswith("L2 flushed")
    assert bench.l2_flushed(args("dcsbm_n2m_k128", nodes=100_000))
    assert bench.workload_config(args("dcsbm_n2m_k128"))["l2"].startswith("inputs larger than L2")


def test_whole_update_traffic_entry():
    """profiles/traffic.json holds the measured DRAM bytes of one whole update (keyed to the digest
    of every source, so bench.py reports them only for the build they were taken on), with its
    per-kernel breakdown adding up to the total."""
    e = bench.measured_traffic("dcsbm_n2m_k128/bf16", "update", any_build=True)
    assert e is not None
    assert sum(k["read"] for k in e["kernels"].values()) == e["dram_read_bytes"]
    assert sum(k["write"] for k in e["kernels"].values()) == e["dram_write_bytes"]
