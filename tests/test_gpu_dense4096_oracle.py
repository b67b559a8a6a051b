"""GPU parity at the dense workload's full size: all twelve 4096 x 4096 matrices
(six Gaussian, six upper triangular; 1-norms 0.01 .. 100) through bbc_expm in the
form the benchmark times (split products from 6 BF16 slices), in the library's
default form (7 slices) and with FP64 products, each against the oracle's exp(A)
at the same (m, s): relative Frobenius error below the workload's 1e-12
(Section 1, eq. eses; Table 2 at u = 2^-53). The oracle's result for each matrix
is computed once (2 N^3 triple loops: about two seconds per product on 16 cores)
and shared by the three forms."""
import numpy as np
import pytest

from gpu_util import empty_like_dev, rel_fro, to_dev, to_host
from oracle import oracle as O
from paper_1710_10989_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12
CASES = [(i, nn) for nn in (False, True) for i in range(len(W.DENSE_NORMS))]


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


@pytest.mark.parametrize("idx,nonnormal", CASES)
def test_dense4096_forms_match_oracle(h, api, idx, nonnormal):
    A = W.dense_case(idx, nonnormal=nonnormal)
    want, oi = O.expm_upper(A, "new") if nonnormal else O.expm(A, "new")
    dA = to_dev(A)
    out = empty_like_dev(A.shape[0])
    forms = {"split6 (benchmarked)": api.PREC_OZAKI | api.ozaki_slices(6),
             "split7 (library default)": api.PREC_OZAKI,
             "fp64": api.PREC_FP64}
    errs = {}
    for name, prec in forms.items():
        info = h.expm(dA, out, 0.0, api.SCHEME_NEW | prec)
        assert info.structure == (1 if nonnormal else 0), name
        assert (info.m, info.s, info.products) == (oi.m, oi.s, oi.products), (name, info.as_dict(), oi)
        errs[name] = rel_fro(to_host(out), want)
    print(f"dense4096 norm {W.DENSE_NORMS[idx]} {'upper' if nonnormal else 'gaussian'} (m, s) = "
          f"({oi.m}, {oi.s}): " + ", ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    assert max(errs.values()) < TOL, errs
