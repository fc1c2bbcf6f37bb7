"""The Python binding's argument checks (CPU): tensors reach the C ABI only as contiguous CUDA
tensors of the expected dtype and size, which a raw device pointer cannot show."""
import pytest
import torch

from paper_2305_10356_gb300 import build, ofsc


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return ofsc.lib()


def _raises(fn, text):
    with pytest.raises(ofsc.OfscError) as ei:
        fn()
    assert ei.value.status == ofsc.ERR_INVALID_ARG
    assert text in str(ei.value)


def test_dtype_layout_and_device_are_checked_before_the_call():
    x = torch.zeros((16, 8), dtype=torch.float32)
    _raises(lambda: ofsc.ofsc_row_normalize(x.double()), "dtype")
    _raises(lambda: ofsc.ofsc_row_normalize(x.t()), "contiguous")
    _raises(lambda: ofsc.ofsc_row_normalize(x), "CUDA")
    _raises(lambda: ofsc.ofsc_row_normalize(x.numpy()), "torch tensor")
    _raises(lambda: ofsc.ofsc_kmeans(x, 2, torch.zeros(16, dtype=torch.int64)), "CUDA")
    src = torch.tensor([0, 1], dtype=torch.int64)
    _raises(lambda: ofsc.ofsc_graph_build(4, src, src), "dtype")
    s32 = src.int()
    _raises(lambda: ofsc.ofsc_graph_build(4, s32, s32), "CUDA")
    _raises(lambda: ofsc.ofsc_gram(x, [x], torch.zeros((1, 8, 8), dtype=torch.float32)), "CUDA")
    c = torch.zeros((5, 4), dtype=torch.float64)
    _raises(lambda: ofsc.ofsc_line_search_step(c.float(), torch.zeros(5, dtype=torch.float64)), "dtype")
    _raises(lambda: ofsc.ofsc_line_search_step(c, torch.zeros(5, dtype=torch.float64)), "CUDA")
    _raises(lambda: ofsc.ofsc_line_search_step(c.numpy(), None), "torch tensor")
