"""fmm_build_tree_noalloc: the tree build for callers that cannot allocate device memory (for
example code inside an application whose own memory manager owns the device, or a loop that
cannot take the synchronisation cudaMalloc may cause).  Its output must equal what the
allocating entry points produce (fmm_build_tree + fmm_tree_export), bit for bit, on
consecutive calls that reuse the library's fixed scratch array, and it must leave the free
device memory unchanged.

The file name makes pytest collect it last."""
import os
import subprocess
import sys

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


_FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_1006_2269_gb300 import fmm, workloads as W
fmm.load_library()
n, L = 65536, 5  # boxes of level 2 hold 4096 points: levels 2-4 split inside blocks
c = W.clusters(n, 74)
dev = torch.device("cuda", 0)
x, y = (torch.as_tensor(v, device=dev) for v in (c.x, c.y))
perm = torch.empty(n, dtype=torch.int32, device=dev)
rects = torch.empty(((4 ** (L + 1) - 1) // 3, 4), dtype=torch.float64, device=dev)
lb = torch.empty(4 ** L + 1, dtype=torch.int32, device=dev)
fmm.fmm_build_tree_noalloc(x, y, L, perm, rects, lb)
torch.cuda.synchronize()
np.savez(sys.argv[2], perm=perm.cpu().numpy(), rects=rects.cpu().numpy(), lb=lb.cpu().numpy())
"""


def test_noalloc_first_in_a_fresh_process(fmmlib, cuda, orc, tmp_path):
    # no tree handle exists in that process: the first no-allocation call itself must prepare
    # the block-local split (its shared memory is above the default launch limit)
    out = str(tmp_path / "tree.npz")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root, out], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    got = np.load(out)
    c = W.clusters(65536, 74)
    operm, orects, olb = orc.tree(c.x, c.y, 5)
    assert np.array_equal(got["perm"], operm)
    assert np.array_equal(got["rects"], orects)
    assert np.array_equal(got["lb"].astype(np.int64), olb)


def test_noalloc_allocates_no_device_memory(fmmlib, cuda):
    # the free device memory is the same before and after a call (after a first call has done
    # the once-per-device set-up), and the caller's buffers are the only outputs
    import torch
    n, L = 20000, 4
    c = W.clusters(n, 75)
    x, y = _t(c.x, cuda), _t(c.y, cuda)
    perm = torch.empty(n, dtype=torch.int32, device=cuda)
    rects = torch.empty(((4 ** (L + 1) - 1) // 3, 4), dtype=torch.float64, device=cuda)
    lb = torch.empty(4 ** L + 1, dtype=torch.int32, device=cuda)
    fmmlib.fmm_build_tree_noalloc(x, y, L, perm, rects, lb)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        fmmlib.fmm_build_tree_noalloc(x, y, L, perm, rects, lb)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0

