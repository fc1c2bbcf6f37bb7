"""The C-ABI library builds, loads and exports every function that include/ofsc.h declares (CPU)."""
import os

import pytest

from paper_2305_10356_gb300 import build, ofsc


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ofsc.lib()


def test_exports_every_declared_symbol(lib):
    names = ofsc.header_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n


def test_version_and_error_string(lib):
    assert lib.ofsc_version() >= 100
    assert isinstance(lib.ofsc_last_error(), bytes)


def test_host_side_argument_checks(lib):
    """Argument validation happens on the host before any CUDA call."""
    import ctypes
    h = ctypes.c_void_p()
    assert lib.ofsc_graph_build(-1, 0, None, None, None, 0, None, ctypes.byref(h)) == ofsc.ERR_INVALID_ARG
    assert b"n=" in lib.ofsc_last_error()
    assert lib.ofsc_graph_build(4, 1, None, None, None, 0, None, ctypes.byref(h)) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_graph_build(4, 0, None, None, None, 7, None, ctypes.byref(h)) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_graph_build(4, 0, None, None, None, 0, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_iterate(None, 0, 4, None, 0.0, 1, None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_row_normalize(-1, 3, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_kmeans(10, 2, None, 11, 0, 1, 10, None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_graph_free(None) == ofsc.OK


def test_host_side_argument_checks_of_the_widened_entry_points(lib):
    """Batched iteration, the unrolled gradient, the autotuner, the weight gradient and
    Rayleigh-Ritz reject bad arguments on the host, before any CUDA call."""
    import ctypes
    i32 = ctypes.c_int32
    assert lib.ofsc_iterate_batched(-1, None, 0, None, None, 0.0, 1, None, None, None) == ofsc.ERR_INVALID_ARG
    assert b"count" in lib.ofsc_last_error()
    assert lib.ofsc_iterate_batched(2, None, 0, None, None, 0.0, 1, None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_iterate_batched(0, None, 0, None, None, 0.0, 1, None, None, None) == ofsc.OK
    assert lib.ofsc_unrolled_grad(None, 4, None, 3, 0, 0, None, None, None, None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_autotune(None, 4, 0, None, None, None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_weight_grad(None, 1, 4, None, 0, None, None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_rayleigh_ritz(None, 4, None, None, None, None) == ofsc.ERR_INVALID_ARG
    w = i32(0)
    assert lib.ofsc_autotune(None, 4, 0, ctypes.byref(w), None, None, None, None) == ofsc.ERR_INVALID_ARG


def test_state_api_argument_checks(lib):
    """The CG state calls reject NULL handles and bad sizes on the host; freeing NULL is a no-op."""
    import ctypes
    h = ctypes.c_void_p()
    assert lib.ofsc_state_create(None, 4, ctypes.byref(h)) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_state_create(None, 4, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_state_free(None) == ofsc.OK
    assert lib.ofsc_state_info(None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_state_save(None, None, 0, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_state_load(None, None, 0, None) == ofsc.ERR_INVALID_ARG


def test_line_search_step_argument_checks(lib):
    """The batch line-search step rejects a negative count, a solver other than 0 or 1 and NULL
    arrays on the host, and returns at once for n = 0 (no GPU needed)."""
    assert lib.ofsc_line_search_step(-1, None, 0, None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_line_search_step(0, None, 2, None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_line_search_step(3, None, 1, None, None, None) == ofsc.ERR_INVALID_ARG
    assert lib.ofsc_line_search_step(0, None, 1, None, None, None) == ofsc.OK


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(ofsc, "_lib", None)
    monkeypatch.setattr(ofsc, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ofsc.OfscError):
        ofsc.lib()


def test_set_allocator_argument_checks():
    """ofsc_set_allocator takes both functions or neither (host state only, no GPU needed)."""
    lib = ofsc.lib()
    alloc = ofsc.ALLOC_FN(lambda nbytes, user: 0)
    assert lib.ofsc_set_allocator(alloc, ofsc.FREE_FN(), None) == ofsc.ERR_INVALID_ARG
    assert b"both" in lib.ofsc_last_error()
    assert lib.ofsc_set_allocator(ofsc.ALLOC_FN(), ofsc.FREE_FN(), None) == ofsc.OK
