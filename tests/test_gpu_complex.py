"""GPU parity, complex A (bbc_expm_complex: the real form [[Re A, -Im A],
[Im A, Re A]] through the real path, (m, s) from the complex 1-norm by the theta
rule of Section 2) against the complex oracle at the same (m, s): 1e-12
relative Frobenius, FP64 and exact-split products."""
import numpy as np
import pytest

from gpu_util import rel_fro
from oracle import complex_oracle as C
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


def _complex(n, seed, norm):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return A * (norm / C.norm1(A))


def _run(h, A, flags=0):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(A, dtype=np.complex128)).cuda()
    y = torch.full_like(x, complex("nan"))
    info = h.expm_complex(x, y, 0.0, flags)
    torch.cuda.synchronize()
    return y.cpu().numpy(), info


@pytest.mark.parametrize("n,norm", [(1, 0.7), (7, 0.01), (64, 1.0), (130, 30.0), (300, 5.0)])
def test_matches_complex_oracle(h, api, n, norm):
    A = _complex(n, 60 + n, norm)
    E, info = _run(h, A)
    want, (m, s, products, nrm) = C.expm(A)
    assert (info.m, info.s, info.products) == (m, s, products)
    assert abs(info.norm1 - nrm) <= 1e-14 * nrm
    assert rel_fro(E, want) < 1e-12, rel_fro(E, want)


@pytest.mark.parametrize("n,norm", [(96, 2.0), (257, 40.0)])
def test_split_products_match_complex_oracle(h, api, n, norm):
    A = _complex(n, 80 + n, norm)
    E, info = _run(h, A, api.PREC_OZAKI)
    want, _ = C.expm(A, m=info.m, s=info.s)
    assert rel_fro(E, want) < 1e-12, rel_fro(E, want)


def test_skew_hermitian_gives_unitary(h, api):
    rng = np.random.default_rng(3)
    G = rng.standard_normal((200, 200)) + 1j * rng.standard_normal((200, 200))
    H = (G + G.conj().T) / 2
    A = 1j * H * (20.0 / C.norm1(1j * H))
    E, _ = _run(h, A)
    assert np.linalg.norm(E.conj().T @ E - np.eye(200)) < 1e-11


def test_real_input_is_the_real_path_bit_for_bit(h, api):
    """For real A the real form is [[A, 0], [0, A]]: every product sums the same
    terms in the same order plus exact zeros, so the FP64 result equals bbc_expm's."""
    import torch
    A = W.gaussian(80, 21, 6.0)
    E, info = _run(h, A.astype(np.complex128))
    x = torch.from_numpy(A).cuda()
    y = torch.empty_like(x)
    ri = h.expm(x, y, 0.0, api.DENSE)
    torch.cuda.synchronize()
    assert (info.m, info.s) == (ri.m, ri.s)
    assert np.array_equal(E.real, y.cpu().numpy())
    assert np.all(E.imag == 0.0)


def test_errors(h, api):
    import torch
    bad = _complex(16, 1, 1.0)
    bad[3, 4] = complex(np.nan, 0.0)
    with pytest.raises(api.BBCError) as ei:
        _run(h, bad)
    assert ei.value.code == api.NONFINITE_INPUT
    x = torch.from_numpy(_complex(16, 2, 1.0)).cuda()
    with pytest.raises(api.BBCError) as ei:
        h.expm_complex(x, x)
    assert ei.value.code == api.INVALID_ARG
    with pytest.raises(api.BBCError) as ei:
        h.expm_complex(x, torch.empty_like(x), 0.0, api.UPPER)
    assert ei.value.code == api.INVALID_ARG
