"""The C-ABI library loads on a machine without a GPU and exports every symbol
that include/*.h declares; host-only entry points (theta, selection) agree with
the oracle. No GPU compute is called here."""
import ctypes
import glob
import os
import re

import pytest

from oracle import theta as TH

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(bbc_\w+)\s*\(", text, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1710_10989_gb300 import build
    return ctypes.CDLL(build.build())


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_1710_10989_gb300 import api
    assert set(declared_symbols()) <= set(api.exported_symbols())


@pytest.mark.parametrize("u", [2.0 ** -53, 2.0 ** -24])
def test_library_theta_matches_oracle(u):
    from paper_1710_10989_gb300 import api
    for m in (1, 2, 4, 6, 8, 9, 12, 16, 18):
        assert api.theta(m, u) == pytest.approx(TH.theta_taylor(m, u), rel=1e-13)


def test_library_selection_matches_oracle():
    from oracle import oracle as O
    from paper_1710_10989_gb300 import api
    import numpy as np
    norms = np.concatenate([[0.0, 1e-30, 1e-10], np.logspace(-6, 3, 400)])
    for scheme, name in ((api.SCHEME_NEW, "new"), (api.SCHEME_PS, "ps")):
        for u, uu in ((api.U_DOUBLE, 2.0 ** -53), (api.U_SINGLE, 2.0 ** -24)):
            for nrm in norms:
                assert api.select(float(nrm), u, scheme) == O.select(float(nrm), name, uu), (nrm, name)


def test_host_argument_errors():
    from paper_1710_10989_gb300 import api
    with pytest.raises(api.BBCError) as e:
        api.theta(0)
    assert e.value.code == api.INVALID_ARG
    with pytest.raises(api.BBCError) as e:
        api.select(float("nan"))
    assert e.value.code == api.NONFINITE_INPUT
    with pytest.raises(api.BBCError):
        api.select(1.0, u=0.5)


@pytest.mark.parametrize("u", [2.0 ** -53, 2.0 ** -24])
def test_library_pade_theta_matches_oracle(u):
    # double-double series in the library, exact rationals in the oracle
    from paper_1710_10989_gb300 import api
    for two_m in (2, 6, 10, 14, 18, 26):
        assert api.theta_pade(two_m, u) == pytest.approx(TH.theta_pade(two_m, u), rel=1e-13)


def test_library_pade_selection_matches_oracle():
    from oracle import oracle as O
    from paper_1710_10989_gb300 import api
    import numpy as np
    for nrm in np.logspace(-3, 3, 200):
        assert api.select(float(nrm), scheme=api.SCHEME_PADE26) == O.select(float(nrm), "pade26")


def declared_arities():
    """{name: parameter count} of every bbc_ prototype in include/*.h."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", " ", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(bbc_\w+)\s*\(([^;{]*?)\)\s*;", text, re.S):
            params = " ".join(m.group(2).split())
            out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_the_header():
    """Each ctypes prototype of the binding takes as many arguments as the C
    declaration, so no call marshals a shifted or missing argument."""
    from paper_1710_10989_gb300 import api
    arities = declared_arities()
    assert len(arities) >= 10
    for name, argtypes in api._SIGS.items():
        assert name in arities, name
        assert len(argtypes) == arities[name], (name, len(argtypes), arities[name])


def test_selection_at_extreme_norms():
    """Norms where norm / theta_m overflows binary64 (above ~4e292), up to the
    largest double, and the smallest ones: the library's (m, s) equal the oracle's."""
    from oracle import oracle as O
    from paper_1710_10989_gb300 import api
    for nrm in (1e200, 4e292, 1e300, 1.7976931348623157e308, 1e-300, 5e-324, 0.0):
        for scheme, name in ((api.SCHEME_NEW, "new"), (api.SCHEME_PS, "ps"), (api.SCHEME_PADE26, "pade26")):
            assert api.select(nrm, scheme=scheme) == O.select(nrm, name), (nrm, name)


def test_certified_selection_at_extreme_norms():
    """The alpha_2 certificate with power norms up to the largest double (where the
    device's overflowed power norms would otherwise reach it) agrees with the oracle."""
    from oracle import oracle as O
    from paper_1710_10989_gb300 import api
    big = 1.7976931348623157e308
    for norms in ((1e200, 1e300, big), (4e292, big, big), (big, big, big), (1e100, 0.0, 0.0), (5.0, 1e-300, 0.0)):
        for scheme, name in ((api.SCHEME_NEW, "new"), (api.SCHEME_PS, "ps")):
            assert api.select_certified(norms, scheme=scheme) == O.select_certified(norms, name), (norms, name)
    with pytest.raises(api.BBCError) as e:
        api.select_certified((1.0, float("inf"), 1.0))
    assert e.value.code == api.NONFINITE_INPUT
