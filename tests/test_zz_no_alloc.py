"""fmm_build_tree_noalloc: the tree build for callers that cannot allocate device memory (for
example code running while its stream is captured into a CUDA graph, where cudaMalloc cannot be
recorded).  Its output must equal what the allocating entry points produce (fmm_build_tree +
fmm_tree_export), bit for bit, on consecutive calls that reuse the library's fixed scratch array.

The file name makes pytest collect it last."""
import numpy as np
import pytest

from paper_1006_2269_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _t(a, dev):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


def test_noalloc_tree_equals_allocating_build(fmmlib, cuda):
    import torch
    # two calls in a row with different sizes: the second reuses the scratch the first left behind
    for n, L, seed in ((30011, 5, 71), (4 ** 4 + 77, 4, 72), (fmmlib.FMM_NOALLOC_MAX_POINTS, 7, 73)):
        c = W.clusters(n, seed)
        x, y = _t(c.x, cuda), _t(c.y, cuda)
        nbox = (4 ** (L + 1) - 1) // 3
        perm = torch.empty(n, dtype=torch.int32, device=cuda)
        rects = torch.empty((nbox, 4), dtype=torch.float64, device=cuda)
        lb = torch.empty(4 ** L + 1, dtype=torch.int32, device=cuda)
        st = torch.full((1,), -1, dtype=torch.int32, device=cuda)
        fmmlib.fmm_build_tree_noalloc(x, y, L, perm, rects, lb, st)
        torch.cuda.synchronize()
        f = fmmlib.FMM(x, y, L, 0.5)
        rperm, rrects, rlb = f.export_tree()
        torch.cuda.synchronize()
        assert int(st.item()) == 0
        assert torch.equal(perm, rperm)
        assert torch.equal(lb, rlb)
        assert torch.equal(rects, rrects)
        f.close()


def test_noalloc_rejects_sizes_beyond_the_scratch(fmmlib, cuda):
    import torch
    n = fmmlib.FMM_NOALLOC_MAX_POINTS + 1
    x = torch.zeros(n, dtype=torch.float64, device=cuda)
    perm = torch.empty(n, dtype=torch.int32, device=cuda)
    rects = torch.empty((5, 4), dtype=torch.float64, device=cuda)
    lb = torch.empty(5, dtype=torch.int32, device=cuda)
    with pytest.raises(fmmlib.FMMError) as e:
        fmmlib.fmm_build_tree_noalloc(x, x, 1, perm, rects, lb)
    assert e.value.code == fmmlib.FMM_ERR_ARG
    assert "65536" in str(e.value)
