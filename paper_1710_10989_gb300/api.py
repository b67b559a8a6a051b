"""Python binding of libbbcexpm.so (include/bbcexpm.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
converts torch CUDA tensors to device pointers and back. There is no CPU or
PyTorch fallback: importing fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libbbcexpm.so")

OK, INVALID_ARG, NONFINITE_INPUT, OVERFLOW, CUDA_ERROR, TIMEOUT, UNSUPPORTED = range(7)
SCHEME_NEW, SCHEME_PS, SCHEME_PADE26, SCHEME_PADE = 0x0, 0x1, 0x2, 0x3
PREC_FP64, PREC_OZAKI, PREC_SPLIT, PREC_SPLIT_TF32, PREC_FP32 = 0x00, 0x10, 0x20, 0x30, 0x40
SELECT_LEARNED, SELECT_ALPHA = 0x1000, 0x2000
DENSE, UPPER = 0x4000, 0x8000
DEGREES = (1, 2, 4, 8, 12, 18)
U_DOUBLE = 2.0 ** -53
U_SINGLE = 2.0 ** -24


def ozaki_slices(k: int) -> int:
    return (k & 0xF) << 8


def square_fp64_last(n: int) -> int:
    return (n & 0xF) << 16


class BBCError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bbc status {code}: {msg}")
        self.code = code


class Info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("s", ctypes.c_int), ("products", ctypes.c_int),
                ("selector", ctypes.c_int), ("norm1", ctypes.c_double), ("status", ctypes.c_int),
                ("structure", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1710_10989_gb300.build.build()")

_lib = ctypes.CDLL(LIB_PATH)
_vp, _i64, _int, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "bbc_create": [ctypes.POINTER(_vp), _int],
    "bbc_destroy": [_vp],
    "bbc_workspace_size": [_vp, _i64, _int, _int, ctypes.POINTER(ctypes.c_size_t)],
    "bbc_theta": [_int, _dbl, _dp],
    "bbc_theta_pade": [_int, _dbl, _dp],
    "bbc_select": [_dbl, _dbl, _int, _ip, _ip],
    "bbc_norm1": [_vp, _vp, _i64, _vp, _dp],
    "bbc_norm1_noalloc": [_vp, _i64, _vp, _vp],
    "bbc_gemm": [_vp, _vp, _vp, _i64, _vp, _int, _vp],
    "bbc_solve": [_vp, _vp, _vp, _i64, _vp],
    "bbc_taylor": [_vp, _vp, _i64, _int, _int, _vp, _int, _vp, _ip],
    "bbc_expm": [_vp, _vp, _i64, _vp, _dbl, _int, _vp, ctypes.POINTER(Info)],
    "bbc_expm_fixed": [_vp, _vp, _i64, _vp, _int, _int, _int, _vp, ctypes.POINTER(Info)],
    "bbc_expm_fixed_async": [_vp, _vp, _i64, _vp, _int, _int, _int, _vp, _vp],
    "bbc_expm_complex": [_vp, _vp, _i64, _vp, _dbl, _int, _vp, ctypes.POINTER(Info)],
    "bbc_selftest_wait": [_vp, _vp, ctypes.POINTER(_int)],
    "bbc_expm_host": [_vp, _vp, _i64, _vp, _dbl, _int, _vp, ctypes.POINTER(Info)],
    "bbc_expm_host_many": [_vp, _vp, _vp, _i64, _vp, _dbl, _int, _vp, _vp],
    "bbc_batch_reserve": [_vp, _i64, _int],
    "bbc_batch_order": [ctypes.POINTER(ctypes.c_int64), _i64, ctypes.POINTER(ctypes.c_int64)],
    "bbc_expm_batched": [_vp, _vp, _vp, _i64, _vp, _int, _dbl, _int, _vp, _vp],
    "bbc_expm_apply_batched": [_vp, _vp, _vp, _vp, _i64, _vp, _int, _dbl, _int, _vp, _vp],
    "bbc_mlp_sizes": [_int, _int, _int, _i64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "bbc_mlp_forward": [_vp, _int, _int, _int, _vp, _i64, _vp, _vp, _vp],
    "bbc_mlp_grad": [_vp, _int, _int, _int, _vp, _vp, _i64, _vp, _vp, _vp, _vp],
    "bbc_mlp_adam": [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                     _int, _vp],
    "bbc_select_certified": [_dp, _dbl, _int, _ip, _ip],
    "bbc_batch_set_selector": [_vp, _vp, _int, _int, _int, ctypes.POINTER(ctypes.c_float),
                               ctypes.POINTER(ctypes.c_float)],
    "bbc_selector_data_batched": [_vp, _vp, _vp, _i64, _int, _vp, _vp, _vp, _vp],
    "bbc_profile_enable": [_vp, _int],
    "bbc_profile_read": [_vp, _int, ctypes.POINTER(ctypes.c_int64), _dp],
    "bbc_profile_flops": [_vp, _int, _dp],
    "bbc_batch_tune": [_vp, _i64, _dbl, _vp, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int)],
    "bbc_batch_set_tuning": [_vp, ctypes.c_uint32, _int],
    "bbc_batch_get_shapes": [_vp, ctypes.POINTER(ctypes.c_uint32)],
    "bbc_batch_set_shapes": [_vp, ctypes.POINTER(ctypes.c_uint32)],
    "bbc_batch_launch_shape": [_vp, ctypes.c_int64, ctypes.POINTER(_int), ctypes.POINTER(_int)],
}
KERNEL_PRODUCT, KERNEL_NORM, KERNEL_LINCOMB, KERNEL_SPLIT, KERNEL_BATCHED, KERNEL_ALL = 0, 1, 2, 3, 4, -1
DTYPE_F64, DTYPE_F32 = 0, 1
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _int
_lib.bbc_last_error.argtypes = []
_lib.bbc_last_error.restype = ctypes.c_char_p


def exported_symbols() -> list[str]:
    return list(_SIGS) + ["bbc_last_error"]


def _check(rc: int) -> None:
    if rc != OK:
        raise BBCError(rc, _lib.bbc_last_error().decode())


def theta(m: int, u: float = U_DOUBLE) -> float:
    out = ctypes.c_double()
    _check(_lib.bbc_theta(m, u, ctypes.byref(out)))
    return out.value


def theta_pade(two_m: int, u: float = U_DOUBLE) -> float:
    out = ctypes.c_double()
    _check(_lib.bbc_theta_pade(two_m, u, ctypes.byref(out)))
    return out.value


def select(norm1: float, u: float = U_DOUBLE, scheme: int = SCHEME_NEW) -> tuple[int, int]:
    m, s = ctypes.c_int(), ctypes.c_int()
    _check(_lib.bbc_select(norm1, u, scheme, ctypes.byref(m), ctypes.byref(s)))
    return m.value, s.value


def norm1_noalloc(A, out, stream=None) -> None:
    """||A||_1 into the one-element float64 CUDA tensor `out`, allocating no
    device memory (no handle needed). For callers that must not allocate at
    call time; see bbc_norm1_noalloc in include/bbcexpm.h for the limits."""
    pa, n = _mat(A, "A")
    import torch
    if not (out.is_cuda and out.dtype == torch.float64 and out.numel() >= 1):
        raise ValueError("out: need a float64 CUDA tensor with at least one element")
    _check(_lib.bbc_norm1_noalloc(pa, n, out.data_ptr(), _stream(stream)))


def norm1_noalloc_raw(a_ptr: int, n: int, out_ptr: int, stream: int = 0) -> None:
    """Same entry point with raw device pointers (no tensor checks)."""
    _check(_lib.bbc_norm1_noalloc(a_ptr, n, out_ptr, stream))


def select_certified(norms3, u: float = U_DOUBLE, scheme: int = SCHEME_NEW) -> tuple[int, int]:
    """Cheapest (m, s) certified by ||A||_1 or alpha_2 from {||A||, ||A^2||, ||A^3||}."""
    arr = (ctypes.c_double * 3)(*[float(x) for x in list(norms3)[:3]])
    m, s = ctypes.c_int(), ctypes.c_int()
    _check(_lib.bbc_select_certified(arr, u, scheme, ctypes.byref(m), ctypes.byref(s)))
    return m.value, s.value


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


def _mat(t, name: str):
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 2 and t.shape[0] == t.shape[1]
            and t.is_contiguous()):
        raise ValueError(f"{name}: need a contiguous square float64 CUDA tensor")
    return t.data_ptr(), t.shape[0]


@dataclasses.dataclass
class Handle:
    device: int = 0

    def __post_init__(self):
        self._h = _vp()
        _check(_lib.bbc_create(ctypes.byref(self._h), self.device))

    def close(self) -> None:
        if self._h:
            _lib.bbc_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def profile_enable(self, enable: bool = True) -> None:
        _check(_lib.bbc_profile_enable(self._h, int(enable)))

    def profile_read(self, kind: int = KERNEL_ALL) -> tuple[int, float]:
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(_lib.bbc_profile_read(self._h, kind, ctypes.byref(n), ctypes.byref(ms)))
        return n.value, ms.value

    def batch_tune(self, max_n: int, tol: float = 0.0, stream=None) -> tuple[int, int]:
        """Time the batched path's choices on this GPU; returns (split_mask, ctas)."""
        mask = ctypes.c_uint32()
        ctas = ctypes.c_int()
        _check(_lib.bbc_batch_tune(self._h, max_n, tol, _stream(stream), ctypes.byref(mask), ctypes.byref(ctas)))
        return mask.value, ctas.value

    def batch_set_tuning(self, split_mask: int, ctas: int) -> None:
        _check(_lib.bbc_batch_set_tuning(self._h, split_mask & 0xFFFFFFFF, ctas))

    def batch_get_shapes(self) -> tuple[int, int, int]:
        """(FP64 16 x 16 tile mask, FP64 32 x 32 tile mask, split 16 x 16 task mask) per size bucket."""
        m = (ctypes.c_uint32 * 3)()
        _check(_lib.bbc_batch_get_shapes(self._h, m))
        return int(m[0]), int(m[1]), int(m[2])

    def batch_set_shapes(self, masks=None) -> None:
        if masks is None:
            _check(_lib.bbc_batch_set_shapes(self._h, None))
            return
        m = (ctypes.c_uint32 * 3)(*[int(x) & 0xFFFFFFFF for x in masks])
        _check(_lib.bbc_batch_set_shapes(self._h, m))

    def batch_launch_shape(self, count: int) -> tuple:
        """(CTAs per matrix, CTAs launched) of a batch of `count` matrices."""
        c, g = _int(), _int()
        _check(_lib.bbc_batch_launch_shape(self._h, count, ctypes.byref(c), ctypes.byref(g)))
        return c.value, g.value

    def profile_flops(self, kind: int = KERNEL_ALL) -> float:
        """Algorithmic flops of a kernel class since profile_enable (products: 2 N^3
        dense, N (N+1) (N+2) / 3 triangular)."""
        f = ctypes.c_double()
        _check(_lib.bbc_profile_flops(self._h, kind, ctypes.byref(f)))
        return f.value

    def batch_set_selector(self, net: "MLP", S: int, mu, sd) -> None:
        mu_a = (ctypes.c_float * 5)(*[float(x) for x in mu])
        sd_a = (ctypes.c_float * 5)(*[float(x) for x in sd])
        self._selector = net  # keep the parameters alive while installed
        _check(_lib.bbc_batch_set_selector(self._h, net.params.data_ptr(), net.hidden, net.n_out, S, mu_a, sd_a))

    def selector_data(self, batch: "Batch", stream=None):
        """(features [count, 5] float32, exact norms [count, 4] float64) as CUDA tensors."""
        import torch
        feat = torch.empty((batch.count, 5), dtype=torch.float32, device="cuda")
        norms = torch.empty((batch.count, 4), dtype=torch.float64, device="cuda")
        _check(_lib.bbc_selector_data_batched(self._h, batch.a_ptrs.data_ptr(), batch.ns.data_ptr(), batch.count,
                                              batch.dtype, feat.data_ptr(), norms.data_ptr(), _stream(stream),
                                              batch.info.data_ptr()))
        return feat, norms

    def batch_reserve(self, max_n: int, flags: int = 0) -> None:
        _check(_lib.bbc_batch_reserve(self._h, max_n, flags))

    def expm_batched(self, batch: "Batch", tol: float = 0.0, flags: int = 0, stream=None) -> None:
        _check(_lib.bbc_expm_batched(self._h, batch.a_ptrs.data_ptr(), batch.ns.data_ptr(), batch.count,
                                     batch.o_ptrs.data_ptr(), batch.dtype, tol, flags, _stream(stream),
                                     batch.info.data_ptr()))

    def expm_apply_batched(self, batch: "Batch", tol: float = 0.0, flags: int = 0, stream=None) -> None:
        """Out_i = exp(A_i) B_i for a Batch built with `rhs` (Out_i may be B_i)."""
        if batch.b_ptrs is None:
            raise ValueError("the batch has no right-hand sides (Batch(..., rhs=[...]))")
        _check(_lib.bbc_expm_apply_batched(self._h, batch.a_ptrs.data_ptr(), batch.b_ptrs.data_ptr(),
                                           batch.ns.data_ptr(), batch.count, batch.o_ptrs.data_ptr(),
                                           batch.dtype, tol, flags, _stream(stream), batch.info.data_ptr()))

    def workspace_size(self, n: int, flags: int = 0) -> int:
        b = ctypes.c_size_t()
        _check(_lib.bbc_workspace_size(self._h, n, 0, flags, ctypes.byref(b)))
        return b.value

    def norm1(self, A, stream=None) -> float:
        pa, n = _mat(A, "A")
        out = ctypes.c_double()
        _check(_lib.bbc_norm1(self._h, pa, n, _stream(stream), ctypes.byref(out)))
        return out.value

    def gemm(self, P, Q, C, flags: int = PREC_FP64, stream=None) -> None:
        pp, n = _mat(P, "P")
        pq, _ = _mat(Q, "Q")
        pc, _ = _mat(C, "C")
        _check(_lib.bbc_gemm(self._h, pp, pq, n, pc, flags, _stream(stream)))

    def solve(self, M, B, stream=None) -> None:
        """B <- M^-1 B in place (M is overwritten by its LU factors)."""
        pm, n = _mat(M, "M")
        pb, _ = _mat(B, "B")
        _check(_lib.bbc_solve(self._h, pm, pb, n, _stream(stream)))

    def taylor(self, A, m: int, s: int, T, flags: int = 0, stream=None) -> int:
        pa, n = _mat(A, "A")
        pt, _ = _mat(T, "T")
        prod = ctypes.c_int()
        _check(_lib.bbc_taylor(self._h, pa, n, m, s, pt, flags, _stream(stream), ctypes.byref(prod)))
        return prod.value

    def expm(self, A, out, tol: float = 0.0, flags: int = 0, stream=None) -> Info:
        pa, n = _mat(A, "A")
        po, _ = _mat(out, "out")
        info = Info()
        _check(_lib.bbc_expm(self._h, pa, n, po, tol, flags, _stream(stream), ctypes.byref(info)))
        return info

    def expm_fixed(self, A, out, m: int, s: int, flags: int = 0, stream=None) -> Info:
        pa, n = _mat(A, "A")
        po, _ = _mat(out, "out")
        info = Info()
        _check(_lib.bbc_expm_fixed(self._h, pa, n, po, m, s, flags, _stream(stream), ctypes.byref(info)))
        return info

    def selftest_wait(self, stream=None) -> int:
        """Status of a device wait that nothing completes (TIMEOUT when the bound works)."""
        st = _int()
        _check(_lib.bbc_selftest_wait(self._h, _stream(stream), ctypes.byref(st)))
        return st.value

    def expm_complex(self, A, out, tol: float = 0.0, flags: int = 0, stream=None) -> Info:
        """exp(A) for a square contiguous complex128 CUDA tensor A into `out` (same shape)."""
        import torch
        for t, name in ((A, "A"), (out, "out")):
            if (not t.is_cuda or t.dtype != torch.complex128 or t.dim() != 2 or t.shape[0] != t.shape[1]
                    or not t.is_contiguous()):
                raise ValueError(f"{name}: need a contiguous square complex128 CUDA tensor")
        if out.shape != A.shape:
            raise ValueError("out: shape differs from A")
        info = Info()
        _check(_lib.bbc_expm_complex(self._h, A.data_ptr(), A.shape[0], out.data_ptr(), tol, flags,
                                     _stream(stream), ctypes.byref(info)))
        return info

    def expm_fixed_async(self, A, out, m: int, s: int, flags: int = 0, stream=None, status=None) -> None:
        """Graph-capturable exp(A) at fixed (m, s); status: optional int32 CUDA tensor
        (one element) receiving the status bits, stream-ordered."""
        pa, n = _mat(A, "A")
        po, _ = _mat(out, "out")
        ps = None
        if status is not None:
            if not status.is_cuda or status.numel() < 1 or status.element_size() != 4:
                raise ValueError("status: need a 4-byte CUDA tensor")
            ps = status.data_ptr()
        _check(_lib.bbc_expm_fixed_async(self._h, pa, n, po, m, s, flags, _stream(stream), ps))

    def expm_host(self, A, out, tol: float = 0.0, flags: int = 0, stream=None) -> Info:
        """A, out: host tensors/arrays (float64, C-contiguous, square)."""
        pa, n = _host_ptr(A)
        po, _ = _host_ptr(out)
        info = Info()
        _check(_lib.bbc_expm_host(self._h, pa, n, po, tol, flags, _stream(stream), ctypes.byref(info)))
        return info


    def expm_host_many(self, As, outs, tol: float = 0.0, flags: int = 0, stream=None) -> list:
        """exp of each host matrix in `As` into `outs` (host tensors/arrays, float64,
        C-contiguous, square), with the copies pipelined behind the computation."""
        k = len(As)
        if len(outs) != k:
            raise ValueError("As and outs differ in length")
        pa = (ctypes.c_void_p * max(k, 1))()
        po = (ctypes.c_void_p * max(k, 1))()
        ns = (ctypes.c_int64 * max(k, 1))()
        for i, (a, o) in enumerate(zip(As, outs)):
            pa[i], ns[i] = _host_ptr(a)
            po[i], n2 = _host_ptr(o)
            if n2 != ns[i]:
                raise ValueError("output size differs from input size")
        infos = (Info * max(k, 1))()
        _check(_lib.bbc_expm_host_many(self._h, pa, ns, k, po, tol, flags, _stream(stream), infos))
        return [infos[i] for i in range(k)]


def batch_order(ns) -> list[int]:
    """Largest-first order of matrix sizes (host helper of the batched call)."""
    import numpy as np
    a = np.ascontiguousarray(ns, dtype=np.int64)
    out = np.empty_like(a)
    _check(_lib.bbc_batch_order(a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), len(a),
                                out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out.tolist()


class Batch:
    """Device-side descriptor arrays for bbc_expm_batched, built from lists of
    CUDA tensors (inputs and outputs stay owned by the caller)."""

    def __init__(self, inputs, outputs=None, rhs=None):
        import torch
        if outputs is None:  # feature / norm extraction only
            outputs = inputs
        if len(inputs) != len(outputs) or (rhs is not None and len(rhs) != len(inputs)):
            raise ValueError("inputs, outputs and right-hand sides differ in length")
        dt = inputs[0].dtype if inputs else torch.float32
        for a, o in zip(inputs, outputs):
            if not (a.is_cuda and o.is_cuda and a.dtype == dt and o.dtype == dt and a.is_contiguous()
                    and o.is_contiguous() and a.dim() == 2 and a.shape[0] == a.shape[1] and o.shape == a.shape):
                raise ValueError("need matching contiguous square CUDA tensors of one dtype")
        if dt not in (torch.float32, torch.float64):
            raise ValueError("float32 or float64 only")
        self.dtype = DTYPE_F32 if dt == torch.float32 else DTYPE_F64
        self.count = len(inputs)
        self.ns = torch.tensor([a.shape[0] for a in inputs], dtype=torch.int64, device="cuda")
        self.a_ptrs = torch.tensor([a.data_ptr() for a in inputs], dtype=torch.int64, device="cuda")
        self.o_ptrs = torch.tensor([o.data_ptr() for o in outputs], dtype=torch.int64, device="cuda")
        self.b_ptrs = None
        if rhs is not None:
            for a, b in zip(inputs, rhs):
                if not (b.is_cuda and b.dtype == dt and b.is_contiguous() and b.shape == a.shape):
                    raise ValueError("right-hand sides: need contiguous CUDA tensors shaped and typed as the inputs")
            self.b_ptrs = torch.tensor([b.data_ptr() for b in rhs], dtype=torch.int64, device="cuda")
        self.info = torch.zeros((max(1, self.count), ctypes.sizeof(Info) // 8), dtype=torch.float64,
                                device="cuda")

    def infos(self) -> list[dict]:
        raw = self.info.cpu().numpy().tobytes()
        n = ctypes.sizeof(Info)
        return [Info.from_buffer_copy(raw[i * n:(i + 1) * n]).as_dict() for i in range(self.count)]


class MLP:
    """Device-side (m, s)-proposing network: parameters, Adam state and an
    activation workspace as torch CUDA tensors; compute in the library's kernels."""

    def __init__(self, n_in: int, hidden: int, n_out: int, params=None, seed: int = 0):
        import torch
        self.n_in, self.hidden, self.n_out = n_in, hidden, n_out
        n, _ = self.sizes(0)
        if params is None:
            g = torch.Generator().manual_seed(seed)
            chunks = []
            for shp, fan_in in (((hidden, n_in), n_in), ((hidden,), 0), ((hidden, hidden), hidden), ((hidden,), 0),
                                ((n_out, hidden), hidden), ((n_out,), 0)):
                if fan_in:
                    chunks.append(torch.randn(shp, generator=g).flatten() * (2.0 / fan_in) ** 0.5)
                else:
                    chunks.append(torch.zeros(shp).flatten())
            params = torch.cat(chunks)
        self.params = torch.as_tensor(params, dtype=torch.float32).cuda().contiguous()
        assert self.params.numel() == n
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self._ws = None

    def sizes(self, B: int):
        n = ctypes.c_int64()
        w = ctypes.c_int64()
        _check(_lib.bbc_mlp_sizes(self.n_in, self.hidden, self.n_out, B, ctypes.byref(n), ctypes.byref(w)))
        return n.value, w.value

    def _workspace(self, B):
        import torch
        _, w = self.sizes(B)
        if self._ws is None or self._ws.numel() < w:
            self._ws = torch.empty(max(w, 1), dtype=torch.float32, device="cuda")
        return self._ws

    def forward(self, X, stream=None):
        import torch
        X = X.contiguous()
        B = X.shape[0]
        out = torch.empty((B, self.n_out), dtype=torch.float32, device="cuda")
        _check(_lib.bbc_mlp_forward(self.params.data_ptr(), self.n_in, self.hidden, self.n_out, X.data_ptr(), B,
                                    out.data_ptr(), self._workspace(B).data_ptr(), _stream(stream)))
        return out

    def grad(self, X, y, stream=None):
        import torch
        X = X.contiguous()
        y = y.to(torch.int32).contiguous()
        B = X.shape[0]
        g = torch.empty_like(self.params)
        loss = torch.empty(B, dtype=torch.float32, device="cuda")
        _check(_lib.bbc_mlp_grad(self.params.data_ptr(), self.n_in, self.hidden, self.n_out, X.data_ptr(),
                                 y.data_ptr(), B, g.data_ptr(), loss.data_ptr(), self._workspace(B).data_ptr(),
                                 _stream(stream)))
        return g, loss

    def train_step(self, X, y, lr=1e-3, stream=None):
        g, loss = self.grad(X, y, stream)
        self.step += 1
        _check(_lib.bbc_mlp_adam(self.params.data_ptr(), g.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                                 self.params.numel(), lr, 0.9, 0.999, 1e-8, self.step, _stream(stream)))
        return loss


def _host_ptr(x):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous() or x.dim() != 2:
                raise ValueError("need a contiguous float64 host tensor")
            return x.data_ptr(), x.shape[0]
    except ImportError:
        pass
    import numpy as np
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous and x.ndim == 2):
        raise ValueError("need a contiguous float64 host array")
    return x.ctypes.data, x.shape[0]
