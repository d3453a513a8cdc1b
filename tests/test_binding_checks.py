"""Argument checks of the Python binding that happen before the library is called (CPU only):
the C entry points take raw device pointers, so the binding refuses host tensors, wrong dtypes,
non-contiguous views and buffers shorter than the call writes."""
import pytest
import torch

from paper_1006_2269_gb300 import build, fmm


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return fmm.load_library()


def test_host_tensors_are_refused():
    x = torch.zeros(10, dtype=torch.float64)
    tg = torch.zeros(3, dtype=torch.int64)
    phi = torch.zeros(3, dtype=torch.float64)
    with pytest.raises(fmm.FMMError, match="x must be a CUDA tensor"):
        fmm.fmm_direct(x, x, x, tg, phi)
    with pytest.raises(fmm.FMMError, match="must be a CUDA tensor"):
        fmm.fmm_direct_field(x, x, x, tg, phi, phi)


def test_short_buffers_are_refused_before_the_device_check():
    # a buffer's length is checked before anything else about it, so it holds on any machine
    with pytest.raises(fmm.FMMError, match="phi has 4 elements, needs 5"):
        fmm._dev(torch.zeros(4, dtype=torch.float64), torch.float64, 5, "phi")
    with pytest.raises(fmm.FMMError, match="out has 7 elements, needs 8"):
        fmm._need((None, 3, "unused"), (torch.zeros(7, dtype=torch.int32), 8, "out"))


def test_dtype_and_layout_checks(monkeypatch):
    # a stand-in tensor that reports itself as CUDA reaches the dtype and contiguity checks
    class FakeCuda:
        def __init__(self, t):
            self.t = t
            self.is_cuda = True
            self.dtype = t.dtype

        def numel(self):
            return self.t.numel()

        def is_contiguous(self):
            return self.t.is_contiguous()

        def data_ptr(self):
            return 0

    with pytest.raises(fmm.FMMError, match="x must be torch.float64, got torch.float32"):
        fmm._dev(FakeCuda(torch.zeros(4, dtype=torch.float32)), torch.float64, 4, "x")
    with pytest.raises(fmm.FMMError, match="x must be contiguous"):
        fmm._dev(FakeCuda(torch.zeros((4, 4), dtype=torch.float64).t()), torch.float64, 16, "x")
    assert fmm._dev(None, torch.float64, 4, "x") is None
