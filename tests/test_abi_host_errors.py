"""The C ABI's error behaviour before any device work, run without a GPU: a null
handle, N <= 0, sizes out of range, null pointers and negative counts come back
as BBC_INVALID_ARG with a message; the host-only calls handle empty input. Every
call here returns before its first CUDA call."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from oracle import mlp as MLP

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# arguments after the (null) handle: pointers null, sizes and flags otherwise valid
HANDLE_CALLS = {
    "bbc_workspace_size": None,  # takes the handle only nominally: checked separately
    "bbc_norm1": (None, 4, None, None),
    "bbc_solve": (None, None, 4, None),
    "bbc_gemm": (None, None, 4, None, 0, None),
    "bbc_taylor": (None, 4, 18, 0, None, 0, None, None),
    "bbc_expm": (None, 4, None, 0.0, 0, None, None),
    "bbc_selftest_wait": (None, None),
    "bbc_expm_complex": (None, 4, None, 0.0, 0, None, None),
    "bbc_expm_fixed_async": (None, 4, None, 18, 0, 0, None, None),
    "bbc_expm_fixed": (None, 4, None, 18, 0, 0, None, None),
    "bbc_expm_host": (None, 4, None, 0.0, 0, None, None),
    "bbc_expm_host_many": (None, None, 0, None, 0.0, 0, None, None),
    "bbc_batch_reserve": (64, 0),
    "bbc_expm_batched": (None, None, 0, None, 0, 0.0, 0, None, None),
    "bbc_expm_apply_batched": (None, None, None, 0, None, 0, 0.0, 0, None, None),
    "bbc_batch_tune": (64, 0.0, None, None, None),
    "bbc_batch_set_tuning": (0, 0),
    "bbc_batch_get_shapes": (None,),
    "bbc_batch_set_shapes": (None,),
    "bbc_batch_launch_shape": (1, None, None),
    "bbc_batch_set_selector": (None, 64, 60, 10, None, None),
    "bbc_selector_data_batched": (None, None, 0, 0, None, None, None, None),
    "bbc_profile_enable": (1,),
    "bbc_profile_read": (-1, None, None),
    "bbc_profile_flops": (-1, None),
}


@pytest.fixture(scope="module")
def api():
    from paper_1710_10989_gb300 import api as A
    return A


def handle_functions():
    """Prototypes of include/*.h whose first parameter is a bbc_handle."""
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", " ", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(bbc_\w+)\s*\(\s*bbc_handle\s+\w+", text):
            names.add(m.group(1))
    return names


def test_every_handle_call_rejects_a_null_handle(api):
    assert handle_functions() - {"bbc_destroy"} == set(HANDLE_CALLS)
    for name, args in HANDLE_CALLS.items():
        if args is None:
            continue
        assert getattr(api._lib, name)(None, *args) == api.INVALID_ARG, name
        assert b"null handle" in api._lib.bbc_last_error(), name
    assert api._lib.bbc_destroy(None) == api.OK
    assert api._lib.bbc_create(None, 0) == api.INVALID_ARG


def test_workspace_query_is_host_arithmetic(api):
    L, nb = api._lib, ctypes.c_size_t()
    assert L.bbc_workspace_size(None, 0, 0, 0, ctypes.byref(nb)) == api.INVALID_ARG
    assert L.bbc_workspace_size(None, 64, 1, 0, ctypes.byref(nb)) == api.INVALID_ARG  # FP64 storage only
    assert L.bbc_workspace_size(None, 64, 0, 0x7, ctypes.byref(nb)) == api.INVALID_ARG  # no such scheme
    n = 4096
    assert L.bbc_workspace_size(None, n, 0, api.PREC_FP64, ctypes.byref(nb)) == api.OK
    fp64 = nb.value
    assert fp64 >= 10 * n * n * 8                      # the scheme's work matrices
    assert L.bbc_workspace_size(None, n, 0, api.PREC_OZAKI | api.ozaki_slices(6), ctypes.byref(nb)) == api.OK
    assert nb.value >= fp64 + 2 * 6 * n * n * 2        # plus 6 BF16 planes per operand


def test_norm1_noalloc_bounds_before_any_launch(api):
    L, buf = api._lib, ctypes.c_void_p(16)
    assert L.bbc_norm1_noalloc(buf, 0, buf, None) == api.INVALID_ARG
    assert L.bbc_norm1_noalloc(buf, -3, buf, None) == api.INVALID_ARG
    assert L.bbc_norm1_noalloc(buf, 65537, buf, None) == api.INVALID_ARG
    assert L.bbc_norm1_noalloc(None, 4, buf, None) == api.INVALID_ARG
    assert L.bbc_norm1_noalloc(buf, 4, None, None) == api.INVALID_ARG


def test_batch_order_empty_negative_and_stable(api):
    assert api.batch_order([]) == []
    L = api._lib
    assert L.bbc_batch_order(None, 0, None) == api.OK
    assert L.bbc_batch_order(None, -1, None) == api.INVALID_ARG
    assert L.bbc_batch_order(None, 2, None) == api.INVALID_ARG
    # largest first, equal sizes in input order
    assert api.batch_order([3, 9, 3, 12, 9]) == [3, 1, 4, 0, 2]


def test_mlp_sizes_follow_the_parameter_layout(api):
    L = api._lib
    n_p, ws = ctypes.c_int64(), ctypes.c_int64()
    for n_in, hid, n_out in ((5, 64, 60), (3, 7, 2), (1, 1, 1)):
        assert L.bbc_mlp_sizes(n_in, hid, n_out, 0, ctypes.byref(n_p), ctypes.byref(ws)) == api.OK
        assert n_p.value == sum(int(np.prod(s)) for s in MLP.shapes(n_in, hid, n_out))
        assert ws.value == 0
    assert L.bbc_mlp_sizes(0, 64, 60, 8, ctypes.byref(n_p), ctypes.byref(ws)) == api.INVALID_ARG
    assert L.bbc_mlp_sizes(5, 64, 60, -1, ctypes.byref(n_p), ctypes.byref(ws)) == api.INVALID_ARG
    assert L.bbc_mlp_forward(None, 5, 64, 60, None, 8, None, None, None) == api.INVALID_ARG
    assert L.bbc_mlp_grad(None, 5, 64, 60, None, None, 8, None, None, None, None) == api.INVALID_ARG
    assert L.bbc_mlp_adam(None, None, None, None, 8, 1e-3, 0.9, 0.999, 1e-8, 1, None) == api.INVALID_ARG


def test_certified_selection_checks_its_arguments(api):
    L = api._lib
    m, s = ctypes.c_int(), ctypes.c_int()
    norms = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    assert L.bbc_select_certified(None, 2.0 ** -53, 0, ctypes.byref(m), ctypes.byref(s)) == api.INVALID_ARG
    assert L.bbc_select_certified(norms, 0.5, 0, ctypes.byref(m), ctypes.byref(s)) == api.INVALID_ARG
    assert L.bbc_select_certified(norms, 2.0 ** -53, 2, ctypes.byref(m), ctypes.byref(s)) == api.INVALID_ARG
