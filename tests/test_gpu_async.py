"""GPU parity, graph-captured single-matrix calls (bbc_expm_fixed_async).

The three methods of the 64 x 64 single-matrix case -- the paper's scheme
(Section 3, T18 with s = 0), Paterson-Stockmeyer (eq. poli9, T16 with s = 1) and
diagonal Pade r_26 (eq. pade26, s = 0) -- captured once in a CUDA graph and
replayed, against the oracle at the same (m, s): 1e-13 relative Frobenius. The
status word is stream-ordered device memory, read after the replay.
"""
import numpy as np
import pytest

from gpu_util import rel_fro
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


@pytest.fixture(scope="module")
def h(api):
    hh = api.Handle(0)
    yield hh
    hh.close()


def _capture_and_replay(h, api, A, m, s, flags, replays=3):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    y = torch.zeros_like(x)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        h.expm_fixed_async(x, y, m, s, flags, stream=stream, status=st)  # sizes the workspace
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            h.expm_fixed_async(x, y, m, s, flags, stream=stream, status=st)
    for _ in range(replays):
        y.zero_()
        st.fill_(7)
        g.replay()
    torch.cuda.synchronize()
    return y.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("scheme,m,s", [("new", 18, 0), ("ps", 16, 1), ("pade26", 26, 0)])
def test_small_case_three_methods(h, api, scheme, m, s):
    flag = {"new": api.SCHEME_NEW, "ps": api.SCHEME_PS, "pade26": api.SCHEME_PADE26}[scheme]
    A = W.small_case()
    _, oi = O.expm(A, scheme)
    assert (oi.m, oi.s) == (m, s)            # the (m, s) each method selects for this matrix
    E, status = _capture_and_replay(h, api, A, m, s, flag)
    want, _ = O.expm(A, scheme, m=m, s=s)
    assert status == 0
    assert rel_fro(E, want) < 1e-13, rel_fro(E, want)


@pytest.mark.parametrize("n,norm", [(5, 3.0), (130, 20.0), (300, 0.2)])
def test_other_sizes_and_split_products(h, api, n, norm):
    A = W.gaussian(n, 40 + n, norm)
    _, oi = O.expm(A, "new")
    E, status = _capture_and_replay(h, api, A, oi.m, oi.s, api.SCHEME_NEW)
    want, _ = O.expm(A, "new", m=oi.m, s=oi.s)
    assert status == 0 and rel_fro(E, want) < 1e-12
    E2, status = _capture_and_replay(h, api, A, oi.m, oi.s, api.SCHEME_NEW | api.PREC_OZAKI)
    assert status == 0 and rel_fro(E2, want) < 1e-12


def test_upper_flag_matches_triangular_oracle(h, api):
    A = W.nonnormal_upper(96, 101, 5.0)
    _, oi = O.expm_upper(A, "new")
    E, status = _capture_and_replay(h, api, A, oi.m, oi.s, api.SCHEME_NEW | api.UPPER)
    want, _ = O.expm_upper(A, "new", m=oi.m, s=oi.s)
    assert status == 0
    assert np.all(np.tril(E, -1) == 0.0)
    assert rel_fro(E, want) < 1e-12


def test_status_word_reports_overflow(h, api):
    A = np.eye(32) * 900.0                   # e^900 overflows binary64
    _, oi = O.expm(A, "new")
    _, status = _capture_and_replay(h, api, A, oi.m, oi.s, api.SCHEME_NEW | api.DENSE, replays=1)
    assert status & 1


def test_capture_without_workspace_is_refused(api):
    import torch
    hh = api.Handle(0)
    x = torch.from_numpy(W.gaussian(48, 3, 1.0)).cuda()
    y = torch.zeros_like(x)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            with pytest.raises(api.BBCError):
                hh.expm_fixed_async(x, y, 12, 0, stream=stream)
            y.add_(1.0)                      # the capture itself stays valid
    g.replay()
    torch.cuda.synchronize()
    assert float(y[0, 0]) == 1.0
    hh.close()


def test_bounded_wait_reports_timeout_and_context_survives(h, api):
    """Failure detection without a fault: a device wait that nothing completes
    gives up after its bound (about 2 s), the status word says TIMEOUT, and the
    next exp(A) on the same handle still matches the oracle."""
    import time
    t0 = time.perf_counter()
    assert h.selftest_wait() == api.TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    A = W.small_case()
    E, status = _capture_and_replay(h, api, A, 18, 0, api.SCHEME_NEW, replays=1)
    want, _ = O.expm(A, "new", m=18, s=0)
    assert status == 0 and rel_fro(E, want) < 1e-13
