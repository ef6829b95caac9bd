"""Python binding of libcmm (``include/cmm.h``): argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module passes
torch tensors' device pointers, sizes and the current CUDA stream through
ctypes.  There is no CPU fallback: if ``libcmm.so`` is missing the import of
this module fails.

Method: Pagh's compressed matrix multiplication in the Fast Walsh-Hadamard
Transform form (Andersson & Karppa, arXiv 2601.09477, Algorithm 1 and Sec. 4.2).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcmm.so")

OK = 0
ERR_ARG = -1
ERR_RANGE = -3
ERR_CAPACITY = -4
ERR_CUDA = -5
ERR_TIMEOUT = -6
ERR_WORKSPACE = -8

F64, F32, BF16 = 0, 1, 2
PREC_F64, PREC_F32, PREC_BF16TC, PREC_F16TC, PREC_FX64, PREC_TERNARY = 0, 1, 2, 3, 4, 5
MEDIAN, MEAN = 0, 1
MAX_D = 64
MAX_LOG2B = 24

_PREC = {"f64": PREC_F64, "f32": PREC_F32, "bf16tc": PREC_BF16TC, "f16tc": PREC_F16TC,
         "fx64": PREC_FX64, "ternary": PREC_TERNARY}
_REDUCE = {"median": MEDIAN, "mean": MEAN}
_DTYPE = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}


class CmmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("cmm error %d: %s" % (code, msg))
        self.code = code


class _Hashes(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("log2b", ctypes.c_int32),
                ("params", ctypes.POINTER(ctypes.c_uint64))]


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError("libcmm.so is not built (expected at %s); run "
                          "paper_2601_09477_gb300.build.build() first" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    i64, i32, u64, f64, sz = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                              ctypes.c_double, ctypes.c_size_t)
    H = ctypes.POINTER(_Hashes)
    sig = {
        "cmm_make_hashes": (ctypes.c_int, [u64, i32, P]),
        "cmm_sketch_workspace_bytes": (sz, [i64, i64, i64, i32, i32, i32, i32, i32]),
        "cmm_sketch": (ctypes.c_int, [P, i64, i32, P, i64, i32, i64, i64, i64, H, i32, P, P, sz, P]),
        "cmm_extract_workspace_bytes": (sz, [i64, i64, i32]),
        "cmm_extract": (ctypes.c_int, [P, H, i64, i64, i32, P, i64, P, sz, P]),
        "cmm_heavy_hitters": (ctypes.c_int, [P, H, i64, i64, i32, f64, P, P, P, i64,
                                             ctypes.POINTER(ctypes.c_int64), P, sz, P]),
        "cmm_threshold": (ctypes.c_int, [P, i64, i64, i64, f64, P, P, P, i64,
                                         ctypes.POINTER(ctypes.c_int64), P, sz, P]),
        "cmm_multiply_workspace_bytes": (sz, [i64, i64, i64, i32, i32, i32, i32, i32]),
        "cmm_multiply": (ctypes.c_int, [P, i64, i32, P, i64, i32, i64, i64, i64, H, i32, i32,
                                        P, i64, P, P, sz, P]),
        "cmm_multiply_threshold": (ctypes.c_int, [P, i64, i32, P, i64, i32, i64, i64, i64, H,
                                                  i32, i32, P, i64, P, f64, P, P, P, i64,
                                                  ctypes.POINTER(ctypes.c_int64), P, sz, P]),
        "cmm_multiply_host_workspace_bytes": (sz, [i64, i64, i64, i32, i32, i32, i32, i32, i64]),
        "cmm_multiply_host": (ctypes.c_int, [P, i64, i32, P, i64, i32, i64, i64, i64, H, i32, i32,
                                             P, i64, f64, i64, P, P, P,
                                             ctypes.POINTER(ctypes.c_int64), P, sz, P]),
        "cmm_sketch_cyclic_workspace_bytes": (sz, [i64, i64, i64, i32, i32, i32, i32, i32]),
        "cmm_sketch_cyclic": (ctypes.c_int, [P, i64, i32, P, i64, i32, i64, i64, i64, H, i32, P,
                                             P, sz, P]),
        "cmm_extract_cyclic": (ctypes.c_int, [P, H, i64, i64, i32, P, i64, P, sz, P]),
        "cmm_multiply_cyclic_workspace_bytes": (sz, [i64, i64, i64, i32, i32, i32, i32, i32]),
        "cmm_multiply_cyclic": (ctypes.c_int, [P, i64, i32, P, i64, i32, i64, i64, i64, H, i32,
                                               i32, P, i64, P, P, sz, P]),
        "cmm_mean_pairs": (ctypes.c_int, [P, H, i64, P, P, P, P]),
        "cmm_backward_workspace_bytes": (sz, [i64, i64, i64, i32, i32, i32, i32, i32]),
        "cmm_backward": (ctypes.c_int, [P, i64, i32, P, i64, i32, i64, i64, i64, H, i32, i64,
                                        P, P, P, P, i64, P, i64, P, sz, P]),
        "cmm_batched_workspace_bytes": (sz, [P, i32, i32, i32, i32]),
        "cmm_batched_prepare": (ctypes.c_int, [P, i32, i32, i32, i32, P, sz, P, P]),
        "cmm_batched_launch": (ctypes.c_int, [P, P]),
        "cmm_batched_launch_opts": (ctypes.c_int, [P, i64, i32, P]),
        "cmm_batched_status": (ctypes.c_int, [P, P]),
        "cmm_trace_enable": (ctypes.c_int, [i32]),
        "cmm_trace_read": (ctypes.c_int, [i32, P, P, P, P]),
        "cmm_last_error": (ctypes.c_char_p, []),
        "cmm_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def version() -> str:
    return lib.cmm_version().decode()


def trace_enable(on: bool = True):
    """Start (clearing earlier records) or stop the library's launch tracing."""
    _check(lib.cmm_trace_enable(int(bool(on))))


def trace_read(max_entries: int = 64) -> dict:
    """{kernel name: (launches, summed device ms)} of the launches traced so far."""
    names = ctypes.create_string_buffer(32 * max_entries)
    launches = (ctypes.c_int64 * max_entries)()
    total = (ctypes.c_double * max_entries)()
    n = ctypes.c_int32(0)
    _check(lib.cmm_trace_read(max_entries, names, launches, total, ctypes.byref(n)))
    out = {}
    for q in range(min(n.value, max_entries)):
        nm = names.raw[32 * q: 32 * (q + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[q]), float(total[q]))
    return out


def _check(rc: int):
    if rc != OK:
        raise CmmError(rc, lib.cmm_last_error().decode())


@dataclass
class Hashes:
    """Hash functions of all repetitions: ``params`` is (d, 8) uint64 with, per
    repetition, (a, c) of h1, h2, s1, s2 (Sec. 4.2)."""
    d: int
    log2b: int
    params: np.ndarray

    def __post_init__(self):
        self.params = np.ascontiguousarray(self.params, dtype=np.uint64).reshape(self.d, 8)
        self._c = _Hashes(self.d, self.log2b,
                          self.params.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))

    @property
    def ref(self):
        return ctypes.byref(self._c)

    @property
    def b(self) -> int:
        return 1 << self.log2b


def make_hashes(seed: int, d: int, log2b: int) -> Hashes:
    params = np.zeros((d, 8), dtype=np.uint64)
    _check(lib.cmm_make_hashes(seed & (2**64 - 1), d, params.ctypes.data))
    return Hashes(d, log2b, params)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def _operands(A: torch.Tensor, B: torch.Tensor, transA: bool):
    if A.dtype not in _DTYPE or B.dtype != A.dtype:
        raise TypeError("A and B must share a dtype among float64, float32, bfloat16")
    if A.dim() != 2 or B.dim() != 2:
        raise ValueError("A and B must be matrices")
    if A.stride(1) != 1 or B.stride(1) != 1:
        raise ValueError("A and B must be row-major (unit stride along rows)")
    if transA:
        k, m = A.shape
    else:
        m, k = A.shape
    k2, p = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ: %d vs %d" % (k, k2))
    return m, k, p, _DTYPE[A.dtype]


def sketch(A: torch.Tensor, B: torch.Tensor, h: Hashes, prec: str = "f32",
           transA: bool = False, stream=None) -> torch.Tensor:
    """Compress (Algorithm 1): R (d x b, float64, device), scaled by 1/b."""
    m, k, p, dt = _operands(A, B, transA)
    pr = _PREC[prec]
    ws = _workspace(lib.cmm_sketch_workspace_bytes(m, k, p, h.d, h.log2b, dt, pr, int(transA)),
                    A.device)
    R = torch.empty((h.d, h.b), dtype=torch.float64, device=A.device)
    _check(lib.cmm_sketch(A.data_ptr(), max(A.stride(0), 1), int(transA), B.data_ptr(),
                          max(B.stride(0), 1), dt, m, k, p, h.ref, pr, R.data_ptr(),
                          ws.data_ptr(), ws.numel(), _stream(stream)))
    return R


def extract(R: torch.Tensor, h: Hashes, m: int, p: int, reduce: str = "median",
            stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Decompress (Algorithm 1) every entry: the m x p float64 estimate."""
    _check_R(R, h)
    C = out if out is not None else torch.empty((m, p), dtype=torch.float64, device=R.device)
    ws = _workspace(lib.cmm_extract_workspace_bytes(m, p, h.d), R.device)
    _check(lib.cmm_extract(R.data_ptr(), h.ref, m, p, _REDUCE[reduce], C.data_ptr(),
                           max(C.stride(0), 1), ws.data_ptr(), ws.numel(), _stream(stream)))
    return C


def _check_R(R: torch.Tensor, h: Hashes):
    if R.dtype != torch.float64 or tuple(R.shape) != (h.d, h.b) or not R.is_contiguous():
        raise ValueError("R must be a contiguous float64 (d, b) tensor")


def heavy_hitters(R: torch.Tensor, h: Hashes, m: int, p: int, tau: float,
                  reduce: str = "median", capacity: int = 1 << 20, stream=None):
    """(I, J, V) of every |estimate| >= tau in (i, j) order, computed from R."""
    _check_R(R, h)
    dev = R.device
    I = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    J = torch.empty_like(I)
    V = torch.empty(max(capacity, 1), dtype=torch.float64, device=dev)
    cnt = ctypes.c_int64(0)
    ws = _workspace(lib.cmm_extract_workspace_bytes(m, p, h.d), dev)
    _check(lib.cmm_heavy_hitters(R.data_ptr(), h.ref, m, p, _REDUCE[reduce], float(tau),
                                 I.data_ptr(), J.data_ptr(), V.data_ptr(), capacity,
                                 ctypes.byref(cnt), ws.data_ptr(), ws.numel(), _stream(stream)))
    n = cnt.value
    return I[:n], J[:n], V[:n]


def threshold(C: torch.Tensor, tau: float, capacity: int = 1 << 20, stream=None):
    """(I, J, V) of every |C[i, j]| >= tau in (i, j) order, from a dense estimate."""
    if C.dtype != torch.float64 or C.dim() != 2 or C.stride(1) != 1:
        raise ValueError("C must be a row-major float64 matrix")
    m, p = C.shape
    dev = C.device
    I = torch.empty(max(capacity, 1), dtype=torch.int32, device=dev)
    J = torch.empty_like(I)
    V = torch.empty(max(capacity, 1), dtype=torch.float64, device=dev)
    cnt = ctypes.c_int64(0)
    ws = _workspace(lib.cmm_extract_workspace_bytes(m, p, 1), dev)
    _check(lib.cmm_threshold(C.data_ptr(), m, p, max(C.stride(0), 1), float(tau), I.data_ptr(),
                             J.data_ptr(), V.data_ptr(), capacity, ctypes.byref(cnt),
                             ws.data_ptr(), ws.numel(), _stream(stream)))
    n = cnt.value
    return I[:n], J[:n], V[:n]


def multiply_workspace_bytes(m, k, p, h: Hashes, dtype, prec: str = "f32", transA=False) -> int:
    return int(lib.cmm_multiply_workspace_bytes(m, k, p, h.d, h.log2b, _DTYPE[dtype],
                                                _PREC[prec], int(transA)))


def multiply(A: torch.Tensor, B: torch.Tensor, h: Hashes, prec: str = "f32",
             reduce: str = "median", transA: bool = False, R: torch.Tensor | None = None,
             out: torch.Tensor | None = None, ws: torch.Tensor | None = None, stream=None):
    """Compress then Decompress every entry: the m x p float64 estimate of A B.
    ``R`` (d x b float64) receives the sketch when given."""
    m, k, p, dt = _operands(A, B, transA)
    pr = _PREC[prec]
    need = lib.cmm_multiply_workspace_bytes(m, k, p, h.d, h.log2b, dt, pr, int(transA))
    if ws is None or ws.numel() < need:
        ws = _workspace(need, A.device)
    C = out if out is not None else torch.empty((m, p), dtype=torch.float64, device=A.device)
    if R is not None:
        _check_R(R, h)
    _check(lib.cmm_multiply(A.data_ptr(), max(A.stride(0), 1), int(transA), B.data_ptr(),
                            max(B.stride(0), 1), dt, m, k, p, h.ref, pr, _REDUCE[reduce],
                            C.data_ptr(), max(C.stride(0), 1),
                            R.data_ptr() if R is not None else None, ws.data_ptr(),
                            ws.numel(), _stream(stream)))
    return C


def multiply_threshold(A: torch.Tensor, B: torch.Tensor, h: Hashes, tau: float,
                       capacity: int = 1 << 20, prec: str = "f32", reduce: str = "median",
                       transA: bool = False, R: torch.Tensor | None = None,
                       out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                       hh=None, stream=None):
    """cmm_multiply and cmm_threshold in one call: the m x p float64 estimate
    and (I, J, V) of every |estimate| >= tau in (i, j) order.  ``hh`` may hold
    preallocated (I, J, V) device buffers of at least ``capacity`` entries."""
    m, k, p, dt = _operands(A, B, transA)
    pr = _PREC[prec]
    dev = A.device
    need = lib.cmm_multiply_workspace_bytes(m, k, p, h.d, h.log2b, dt, pr, int(transA))
    if ws is None or ws.numel() < need:
        ws = _workspace(need, dev)
    C = out if out is not None else torch.empty((m, p), dtype=torch.float64, device=dev)
    if R is not None:
        _check_R(R, h)
    if hh is None:
        hh = (torch.empty(max(capacity, 1), dtype=torch.int32, device=dev),
              torch.empty(max(capacity, 1), dtype=torch.int32, device=dev),
              torch.empty(max(capacity, 1), dtype=torch.float64, device=dev))
    I, J, V = hh
    if min(I.numel(), J.numel(), V.numel()) < capacity:
        raise ValueError("heavy-hitter buffers hold fewer than capacity entries")
    cnt = ctypes.c_int64(0)
    _check(lib.cmm_multiply_threshold(A.data_ptr(), max(A.stride(0), 1), int(transA),
                                      B.data_ptr(), max(B.stride(0), 1), dt, m, k, p, h.ref, pr,
                                      _REDUCE[reduce], C.data_ptr(), max(C.stride(0), 1),
                                      R.data_ptr() if R is not None else None, float(tau),
                                      I.data_ptr(), J.data_ptr(), V.data_ptr(), capacity,
                                      ctypes.byref(cnt), ws.data_ptr(), ws.numel(),
                                      _stream(stream)))
    n = cnt.value
    return C, (I[:n], J[:n], V[:n])


def sketch_cyclic(A: torch.Tensor, B: torch.Tensor, h: Hashes, transA: bool = False,
                  stream=None) -> torch.Tensor:
    """Compress of Pagh's cyclic form (Sec. 3.1, through the FFT, FP32
    butterflies): R (d x b, float64, device) with R_r = sum_t x_t * y_t."""
    m, k, p, dt = _operands(A, B, transA)
    pr = _PREC["f32"]
    ws = _workspace(lib.cmm_sketch_cyclic_workspace_bytes(m, k, p, h.d, h.log2b, dt, pr,
                                                          int(transA)), A.device)
    R = torch.empty((h.d, h.b), dtype=torch.float64, device=A.device)
    _check(lib.cmm_sketch_cyclic(A.data_ptr(), max(A.stride(0), 1), int(transA), B.data_ptr(),
                                 max(B.stride(0), 1), dt, m, k, p, h.ref, pr, R.data_ptr(),
                                 ws.data_ptr(), ws.numel(), _stream(stream)))
    return R


def extract_cyclic(R: torch.Tensor, h: Hashes, m: int, p: int, reduce: str = "median",
                   stream=None, out: torch.Tensor | None = None) -> torch.Tensor:
    """Decompress of the cyclic form: bucket (h1(i) + h2(j)) mod b."""
    _check_R(R, h)
    C = out if out is not None else torch.empty((m, p), dtype=torch.float64, device=R.device)
    ws = _workspace(lib.cmm_extract_workspace_bytes(m, p, h.d), R.device)
    _check(lib.cmm_extract_cyclic(R.data_ptr(), h.ref, m, p, _REDUCE[reduce], C.data_ptr(),
                                  max(C.stride(0), 1), ws.data_ptr(), ws.numel(),
                                  _stream(stream)))
    return C


def multiply_cyclic(A: torch.Tensor, B: torch.Tensor, h: Hashes, reduce: str = "median",
                    transA: bool = False, R: torch.Tensor | None = None,
                    out: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                    stream=None):
    """sketch_cyclic then extract_cyclic: the m x p float64 estimate of A B."""
    m, k, p, dt = _operands(A, B, transA)
    pr = _PREC["f32"]
    need = lib.cmm_multiply_cyclic_workspace_bytes(m, k, p, h.d, h.log2b, dt, pr, int(transA))
    if ws is None or ws.numel() < need:
        ws = _workspace(need, A.device)
    C = out if out is not None else torch.empty((m, p), dtype=torch.float64, device=A.device)
    if R is not None:
        _check_R(R, h)
    _check(lib.cmm_multiply_cyclic(A.data_ptr(), max(A.stride(0), 1), int(transA),
                                   B.data_ptr(), max(B.stride(0), 1), dt, m, k, p, h.ref, pr,
                                   _REDUCE[reduce], C.data_ptr(), max(C.stride(0), 1),
                                   R.data_ptr() if R is not None else None, ws.data_ptr(),
                                   ws.numel(), _stream(stream)))
    return C


def multiply_host_workspace_bytes(m, k, p, h: Hashes, dtype, prec: str = "f32",
                                  transA=False, capacity: int = 0) -> int:
    return int(lib.cmm_multiply_host_workspace_bytes(m, k, p, h.d, h.log2b, _DTYPE[dtype],
                                                     _PREC[prec], int(transA), int(capacity)))


def multiply_host(A: torch.Tensor, B: torch.Tensor, h: Hashes, prec: str = "f32",
                  reduce: str = "median", transA: bool = False, out: torch.Tensor | None = None,
                  tau: float | None = None, capacity: int = 0, hh_out=None,
                  ws: torch.Tensor | None = None, device="cuda", stream=None):
    """cmm_multiply on HOST tensors (pin them for full copy speed): returns the
    host estimate C and, when ``tau`` is given, the host heavy-hitter list
    (I, J, V) with |C| >= tau.  Synchronous."""
    if A.device.type != "cpu" or B.device.type != "cpu":
        raise ValueError("multiply_host takes host tensors")
    m, k, p, dt = _operands(A, B, transA)
    pr = _PREC[prec]
    cap = int(capacity) if tau is not None else 0
    need = lib.cmm_multiply_host_workspace_bytes(m, k, p, h.d, h.log2b, dt, pr, int(transA), cap)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, device)
    C = out if out is not None else torch.empty((m, p), dtype=torch.float64)
    cnt = ctypes.c_int64(0)
    if tau is not None:
        if hh_out is None:
            hh_out = (torch.empty(max(cap, 1), dtype=torch.int32),
                      torch.empty(max(cap, 1), dtype=torch.int32),
                      torch.empty(max(cap, 1), dtype=torch.float64))
        Ih, Jh, Vh = hh_out
        ptrs = (Ih.data_ptr(), Jh.data_ptr(), Vh.data_ptr(), ctypes.byref(cnt))
    else:
        ptrs = (None, None, None, None)
    _check(lib.cmm_multiply_host(A.data_ptr(), max(A.stride(0), 1), int(transA), B.data_ptr(),
                                 max(B.stride(0), 1), dt, m, k, p, h.ref, pr, _REDUCE[reduce],
                                 C.data_ptr(), max(C.stride(0), 1),
                                 float(tau) if tau is not None else 0.0, cap, *ptrs,
                                 ws.data_ptr(), ws.numel(), _stream(stream)))
    if tau is None:
        return C, None
    n = cnt.value
    return C, (hh_out[0][:n], hh_out[1][:n], hh_out[2][:n])


def backward(A: torch.Tensor, B: torch.Tensor, h: Hashes, I: torch.Tensor, J: torch.Tensor,
             W: torch.Tensor, prec: str = "f32", transA: bool = False, stream=None):
    """(dL/dA, dL/dB) of L = sum_q W[q] * mean-estimate[I[q], J[q]] (cmm_backward)."""
    m, k, p, dt = _operands(A, B, transA)
    pr = _PREC[prec]
    dev = A.device
    I = I.to(device=dev, dtype=torch.int32).contiguous()
    J = J.to(device=dev, dtype=torch.int32).contiguous()
    W = W.to(device=dev, dtype=torch.float64).contiguous()
    need = lib.cmm_backward_workspace_bytes(m, k, p, h.d, h.log2b, dt, pr, int(transA))
    if need == 0:
        raise CmmError(ERR_RANGE, "cmm_backward does not support these sizes / dtypes")
    ws = _workspace(need, dev)
    dA = torch.empty_like(A, memory_format=torch.contiguous_format)
    dB = torch.empty_like(B, memory_format=torch.contiguous_format)
    _check(lib.cmm_backward(A.data_ptr(), max(A.stride(0), 1), int(transA), B.data_ptr(),
                            max(B.stride(0), 1), dt, m, k, p, h.ref, pr, I.numel(), I.data_ptr(),
                            J.data_ptr(), W.data_ptr(), dA.data_ptr(), max(dA.stride(0), 1),
                            dB.data_ptr(), max(dB.stride(0), 1), ws.data_ptr(), ws.numel(),
                            _stream(stream)))
    return dA, dB


class _Problem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("transA", ctypes.c_int32),
                ("B", ctypes.c_void_p), ("ldb", ctypes.c_int64), ("m", ctypes.c_int64),
                ("k", ctypes.c_int64), ("p", ctypes.c_int64), ("log2b", ctypes.c_int32),
                ("hash_params", ctypes.POINTER(ctypes.c_uint64)), ("R", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("ldc", ctypes.c_int64), ("tile_log2", ctypes.c_int32),
                ("t_tile", ctypes.c_int64)]


class _BatchPlan(ctypes.Structure):
    _fields_ = [("opaque", ctypes.c_uint64 * 32)]


@dataclass
class Problem:
    """One problem of a batch: At holds A^T (k x m, float32), B (k x p, float32)."""
    At: torch.Tensor
    B: torch.Tensor
    hashes: Hashes
    R: torch.Tensor | None = None
    C: torch.Tensor | None = None
    tile_log2: int = 0
    t_tile: int = 0


class Batch:
    """A prepared batch: ``launch()`` runs every problem in one persistent
    kernel launch (capturable in a CUDA graph), ``status()`` checks it."""

    def __init__(self, problems, d: int, with_C: bool = True, ws: torch.Tensor | None = None,
                 stream=None):
        self.problems = list(problems)
        self.d = d
        arr = (_Problem * len(self.problems))()
        for q, pb in enumerate(self.problems):
            if pb.At.dtype != torch.float32 or pb.B.dtype != torch.float32:
                raise TypeError("batched problems take float32 operands")
            k, m = pb.At.shape
            k2, p = pb.B.shape
            if k != k2 or pb.hashes.d != d:
                raise ValueError("problem %d: shape or hash count mismatch" % q)
            if pb.R is None:
                pb.R = torch.empty((d, pb.hashes.b), dtype=torch.float64, device=pb.At.device)
            if with_C and pb.C is None:
                pb.C = torch.empty((m, p), dtype=torch.float64, device=pb.At.device)
            arr[q] = _Problem(pb.At.data_ptr(), max(pb.At.stride(0), 1), 1, pb.B.data_ptr(),
                              max(pb.B.stride(0), 1), m, k, p, pb.hashes.log2b,
                              pb.hashes.params.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                              pb.R.data_ptr(), pb.C.data_ptr() if pb.C is not None else None,
                              pb.C.stride(0) if pb.C is not None else 0, int(pb.tile_log2),
                              int(pb.t_tile))
        self._arr = arr
        need = lib.cmm_batched_workspace_bytes(arr, len(arr), d, F32, PREC_F32)
        if need == 0:
            raise CmmError(ERR_ARG, "invalid batch: " + lib.cmm_last_error().decode())
        dev = self.problems[0].At.device
        self.ws = ws if ws is not None and ws.numel() >= need else _workspace(need, dev)
        self.plan = _BatchPlan()
        _check(lib.cmm_batched_prepare(arr, len(arr), d, F32, PREC_F32, self.ws.data_ptr(),
                                       self.ws.numel(), ctypes.byref(self.plan), _stream(stream)))

    def launch(self, stream=None, wait_budget_us: int = 0, unmet_dependency: bool = False):
        _check(lib.cmm_batched_launch_opts(ctypes.byref(self.plan), int(wait_budget_us),
                                           int(bool(unmet_dependency)), _stream(stream)))

    def status(self, stream=None) -> int:
        return int(lib.cmm_batched_status(ctypes.byref(self.plan), _stream(stream)))


def mean_pairs(R: torch.Tensor, h: Hashes, I: torch.Tensor, J: torch.Tensor,
               stream=None) -> torch.Tensor:
    """Mean-over-d estimator at pairs (I[q], J[q])."""
    _check_R(R, h)
    I = I.to(device=R.device, dtype=torch.int32).contiguous()
    J = J.to(device=R.device, dtype=torch.int32).contiguous()
    out = torch.empty(I.numel(), dtype=torch.float64, device=R.device)
    _check(lib.cmm_mean_pairs(R.data_ptr(), h.ref, I.numel(), I.data_ptr(), J.data_ptr(),
                              out.data_ptr(), _stream(stream)))
    return out
