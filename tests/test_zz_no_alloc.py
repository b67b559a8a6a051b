"""The allocation-free 1-norm entry point (bbc_norm1_noalloc), for callers that
must not allocate device memory at call time, gives the oracle's ||A||_1 and the
same result as the handle-based bbc_norm1 -- on two calls in a row, which share
the library's fixed scratch array -- and rejects sizes beyond its fixed capacity."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1710_10989_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10989_gb300 import api as A
    return A


def test_noalloc_norm_matches_handle_norm_twice(api):
    import torch
    h = api.Handle(0)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # a larger matrix first, then a smaller one: the second call must not see
    # anything the first left in the shared scratch
    for n, seed in ((1500, 61), (257, 62)):
        Ah = W.gaussian(n, seed, None)
        A = torch.from_numpy(Ah).cuda()
        api.norm1_noalloc(A, out)
        torch.cuda.synchronize()
        got = out.item()
        # the oracle's column sums (its own loop, independent of the slab kernels)
        assert got == pytest.approx(O.norm1(Ah), rel=1e-14)
        assert got == pytest.approx(h.norm1(A), rel=1e-14)
    h.close()


def test_noalloc_norm_rejects_oversize(api):
    # rejected on the host before any pointer is used
    with pytest.raises(api.BBCError) as e:
        api.norm1_noalloc_raw(0, 65537, 0)
    assert e.value.code == api.INVALID_ARG and "65536" in str(e.value)
