"""Python face of the FP64 CPU oracle (``cmm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use this module; the library never does.  It shares no code with
the CUDA library -- it compiles and loads its own C file with gcc.

The XOR (FWHT) form: every function is a thin ctypes wrapper; the arithmetic
lives in ``cmm_oracle.c`` and follows Algorithm 1 (Compress / Decompress) of
Andersson & Karppa, "Engineering Compressed Matrix Multiplication with the
Fast Walsh-Hadamard Transform" (arXiv 2601.09477), with the hash family of
Sec. 4.2.  See that file's header for the definitions and readings.  The
cyclic (FFT) form of Sec. 3.1 at the end of this file is plain numpy on the
same hash values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cmm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MEDIAN = 0
MEAN = 1


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64, i32, u64, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
        lib.orc_splitmix64_stream.argtypes = [u64, i64, P]
        lib.orc_draw_hashes.argtypes = [u64, i32, P]
        lib.orc_bucket.argtypes = [u64, u64, u64, i32]
        lib.orc_bucket.restype = ctypes.c_uint32
        lib.orc_sign.argtypes = [u64, u64, u64]
        lib.orc_sign.restype = i32
        lib.orc_bucket_array.argtypes = [u64, u64, i64, i32, P]
        lib.orc_sign_array.argtypes = [u64, u64, i64, P]
        lib.orc_fwht.argtypes = [P, i32]
        lib.orc_compress.argtypes = [P, i64, i32, P, i64, i64, i64, i64, i32, i32, P, P, i32]
        lib.orc_compress.restype = i32
        lib.orc_decompress.argtypes = [P, P, i32, i32, i64, i64, i32]
        lib.orc_decompress.restype = f64
        lib.orc_decompress_rows.argtypes = [P, P, i32, i32, i64, i64, i64, i32, P, i64, i32]
        lib.orc_heavy_hitters.argtypes = [P, P, i32, i32, i64, i64, i64, i32, f64, P, P, P, i64]
        lib.orc_heavy_hitters.restype = i64
        lib.orc_mean_at_pairs.argtypes = [P, P, i32, i32, i64, P, P, P]
        lib.orc_adjoint_G.argtypes = [P, i32, i32, i64, P, P, P, P]
        lib.orc_adjoint_M_rows.argtypes = [P, P, i32, i32, i64, i64, i64, P, i64]
        lib.orc_R_entry.argtypes = [P, i64, i32, P, i64, i64, i64, i64, i32, P, ctypes.c_uint32]
        lib.orc_R_entry.restype = f64
        lib.orc_openmp_max_threads.restype = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def max_threads() -> int:
    return int(_load().orc_openmp_max_threads())


def splitmix64_stream(seed: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint64)
    _load().orc_splitmix64_stream(seed & (2**64 - 1), n, _ptr(out))
    return out


def draw_hashes(seed: int, d: int) -> np.ndarray:
    """(d, 8) uint64: per repetition a_h1, c_h1, a_h2, c_h2, a_s1, c_s1, a_s2, c_s2."""
    hp = np.zeros((d, 8), dtype=np.uint64)
    _load().orc_draw_hashes(seed & (2**64 - 1), d, _ptr(hp))
    return hp


def bucket(a: int, c: int, x: int, log2b: int) -> int:
    return int(_load().orc_bucket(a, c, x, log2b))


def sign(a: int, c: int, x: int) -> int:
    return int(_load().orc_sign(a, c, x))


def buckets(a: int, c: int, n: int, log2b: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.uint32)
    _load().orc_bucket_array(int(a), int(c), n, log2b, _ptr(out))
    return out


def signs(a: int, c: int, n: int) -> np.ndarray:
    out = np.zeros(n, dtype=np.int32)
    _load().orc_sign_array(int(a), int(c), n, _ptr(out))
    return out


def fwht(x) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform (Sylvester order) of a length-2^L vector."""
    y = _f64(x).copy()
    L = int(y.shape[0]).bit_length() - 1
    assert y.ndim == 1 and y.shape[0] == 1 << L
    _load().orc_fwht(_ptr(y), L)
    return y


def compress(A, B, hp: np.ndarray, log2b: int, transA: bool = False,
             nthreads: int = 1) -> np.ndarray:
    """Algorithm 1 Compress in FP64; returns R (d x b), already scaled by 1/b.

    ``A`` is m x k (or, with ``transA``, the k x m array holding A^T); ``B`` is k x p.
    """
    A = _f64(A)
    B = _f64(B)
    if transA:
        k, m = A.shape
    else:
        m, k = A.shape
    k2, p = B.shape
    assert k == k2
    hp = np.ascontiguousarray(hp, dtype=np.uint64)
    d = hp.shape[0]
    R = np.zeros((d, 1 << log2b), dtype=np.float64)
    rc = _load().orc_compress(_ptr(A), A.shape[1], int(transA), _ptr(B), B.shape[1],
                              m, k, p, d, log2b, _ptr(hp), _ptr(R), int(nthreads))
    if rc != 0:
        raise MemoryError("oracle compress failed")
    return R


def R_entry(A, B, hp: np.ndarray, log2b: int, r: int, w: int, transA: bool = False) -> float:
    """R_r[w] from the bucket definition (every (i, j) visited; O(m p) + O(k) per pair)."""
    A = _f64(A)
    B = _f64(B)
    if transA:
        k, m = A.shape
    else:
        m, k = A.shape
    p = B.shape[1]
    hr = np.ascontiguousarray(hp[r], dtype=np.uint64)
    return float(_load().orc_R_entry(_ptr(A), A.shape[1], int(transA), _ptr(B), B.shape[1],
                                     m, k, p, log2b, _ptr(hr), w))


def decompress(R: np.ndarray, hp: np.ndarray, i: int, j: int, reduce: int = MEDIAN) -> float:
    R = _f64(R)
    hp = np.ascontiguousarray(hp, dtype=np.uint64)
    L = int(R.shape[1]).bit_length() - 1
    return float(_load().orc_decompress(_ptr(R), _ptr(hp), hp.shape[0], L, i, j, reduce))


def extract(R: np.ndarray, hp: np.ndarray, m: int, p: int, reduce: int = MEDIAN,
            rows=None, nthreads: int = 1) -> np.ndarray:
    """Estimate of rows ``rows=(i0, i1)`` (default: all m rows) of the m x p product."""
    R = _f64(R)
    hp = np.ascontiguousarray(hp, dtype=np.uint64)
    L = int(R.shape[1]).bit_length() - 1
    i0, i1 = rows if rows is not None else (0, m)
    C = np.zeros((i1 - i0, p), dtype=np.float64)
    _load().orc_decompress_rows(_ptr(R), _ptr(hp), hp.shape[0], L, i0, i1, p, reduce,
                                _ptr(C), p, int(nthreads))
    return C


def heavy_hitters(R: np.ndarray, hp: np.ndarray, m: int, p: int, tau: float,
                  reduce: int = MEDIAN, rows=None, capacity: int = 1 << 20,
                  nthreads: int = 1):
    """(I, J, V) of all |estimate| >= tau, sorted by (i, j).

    With ``nthreads`` > 1 the rows are split into contiguous ranges, each
    listed by the same C routine on its own host thread, and the lists are
    joined in row order (the per-entry arithmetic is unchanged)."""
    R = _f64(R)
    hp = np.ascontiguousarray(hp, dtype=np.uint64)
    L = int(R.shape[1]).bit_length() - 1
    i0, i1 = rows if rows is not None else (0, m)

    def one(a: int, b: int):
        I = np.zeros(capacity, dtype=np.int32)
        J = np.zeros(capacity, dtype=np.int32)
        V = np.zeros(capacity, dtype=np.float64)
        n = _load().orc_heavy_hitters(_ptr(R), _ptr(hp), hp.shape[0], L, a, b, p, reduce,
                                      float(tau), _ptr(I), _ptr(J), _ptr(V), capacity)
        if n > capacity:
            raise ValueError("heavy-hitter capacity %d too small for %d entries" % (capacity, n))
        return I[:n].copy(), J[:n].copy(), V[:n].copy()

    nthreads = max(1, min(int(nthreads), i1 - i0))
    if nthreads == 1:
        return one(i0, i1)
    from concurrent.futures import ThreadPoolExecutor
    cuts = [i0 + (i1 - i0) * q // nthreads for q in range(nthreads + 1)]
    with ThreadPoolExecutor(max_workers=nthreads) as ex:   # ctypes releases the GIL
        parts = list(ex.map(lambda q: one(cuts[q], cuts[q + 1]), range(nthreads)))
    return tuple(np.concatenate([pt[c] for pt in parts]) for c in range(3))


def mean_at_pairs(R: np.ndarray, hp: np.ndarray, I, J) -> np.ndarray:
    R = _f64(R)
    hp = np.ascontiguousarray(hp, dtype=np.uint64)
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    L = int(R.shape[1]).bit_length() - 1
    out = np.zeros(I.shape[0], dtype=np.float64)
    _load().orc_mean_at_pairs(_ptr(R), _ptr(hp), hp.shape[0], L, I.shape[0],
                              _ptr(I), _ptr(J), _ptr(out))
    return out


def adjoint_G(hp: np.ndarray, log2b: int, I, J, W) -> np.ndarray:
    hp = np.ascontiguousarray(hp, dtype=np.uint64)
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    W = _f64(W)
    G = np.zeros((hp.shape[0], 1 << log2b), dtype=np.float64)
    _load().orc_adjoint_G(_ptr(hp), hp.shape[0], log2b, I.shape[0], _ptr(I), _ptr(J),
                          _ptr(W), _ptr(G))
    return G


def adjoint_M(G: np.ndarray, hp: np.ndarray, m: int, p: int, rows=None) -> np.ndarray:
    G = _f64(G)
    hp = np.ascontiguousarray(hp, dtype=np.uint64)
    L = int(G.shape[1]).bit_length() - 1
    i0, i1 = rows if rows is not None else (0, m)
    M = np.zeros((i1 - i0, p), dtype=np.float64)
    _load().orc_adjoint_M_rows(_ptr(G), _ptr(hp), hp.shape[0], L, i0, i1, p, _ptr(M), p)
    return M


def adjoint(A, B, hp: np.ndarray, log2b: int, I, J, W, transA: bool = False):
    """(dL/dA, dL/dB) of L = sum_q W_q * Chat_mean[I_q, J_q]: dA = M B^T, dB = A^T M."""
    A = _f64(A)
    B = _f64(B)
    Am = A.T if transA else A
    m, _ = Am.shape
    p = B.shape[1]
    G = adjoint_G(hp, log2b, I, J, W)
    M = adjoint_M(G, hp, m, p)
    dA = M @ B.T
    dB = Am.T @ M
    return (dA.T.copy() if transA else dA), dB


# ---- Pagh's original (cyclic) form, Sec. 3.1 ----------------------------------
# Same sketches x_t, y_t as Algorithm 1 (hashes of Sec. 4.2), but the product
# polynomial is the cyclic convolution of Sec. 2, (x * y)[w] = sum over
# u + v = w mod b of x[u] y[v], taken here through numpy's FFT (FP64, a library
# step), and the estimate reads bucket (h1(i) + h2(j)) mod b.

def _hash_arrays(hp_r, m: int, p: int, log2b: int):
    h1 = buckets(int(hp_r[0]), int(hp_r[1]), m, log2b)
    h2 = buckets(int(hp_r[2]), int(hp_r[3]), p, log2b)
    s1 = signs(int(hp_r[4]), int(hp_r[5]), m).astype(np.float64)
    s2 = signs(int(hp_r[6]), int(hp_r[7]), p).astype(np.float64)
    return h1.astype(np.int64), h2.astype(np.int64), s1, s2


def compress_cyclic(A, B, hp: np.ndarray, log2b: int, transA: bool = False) -> np.ndarray:
    """R (d x b): R_r = sum_t x_{r,t} * y_{r,t} (cyclic convolution), FP64."""
    A = _f64(A)
    B = _f64(B)
    Am = A.T if transA else A            # m x k
    m, k = Am.shape
    p = B.shape[1]
    b = 1 << log2b
    hp = np.ascontiguousarray(hp, dtype=np.uint64)
    R = np.zeros((hp.shape[0], b), dtype=np.float64)
    for r in range(hp.shape[0]):
        h1, h2, s1, s2 = _hash_arrays(hp[r], m, p, log2b)
        X = np.zeros((b, k))
        np.add.at(X, h1, s1[:, None] * Am)          # column t of X is x_t
        Y = np.zeros((b, k))
        np.add.at(Y, h2, s2[:, None] * B.T)         # column t of Y is y_t
        P = (np.fft.fft(X, axis=0) * np.fft.fft(Y, axis=0)).sum(axis=1)
        R[r] = np.real(np.fft.ifft(P))
    return R


def R_entry_cyclic(A, B, hp: np.ndarray, log2b: int, r: int, w: int,
                   transA: bool = False) -> float:
    """R_r[w] from the bucket definition: sum of s1(i) s2(j) C[i, j] over every
    (i, j) with h1(i) + h2(j) = w (mod b), C = A B."""
    A = _f64(A)
    B = _f64(B)
    Am = A.T if transA else A
    m, p = Am.shape[0], B.shape[1]
    h1, h2, s1, s2 = _hash_arrays(np.ascontiguousarray(hp, dtype=np.uint64)[r], m, p, log2b)
    C = Am @ B
    sel = ((h1[:, None] + h2[None, :]) % (1 << log2b)) == w
    return float(np.sum((s1[:, None] * s2[None, :] * C)[sel]))


def extract_cyclic(R: np.ndarray, hp: np.ndarray, m: int, p: int, reduce: int = MEDIAN,
                   rows=None) -> np.ndarray:
    """Estimate rows ``rows=(i0, i1)``: median (or mean) over r of
    s1(i) s2(j) R_r[(h1(i) + h2(j)) mod b]; even d: mean of the two middle values."""
    R = _f64(R)
    hp = np.ascontiguousarray(hp, dtype=np.uint64)
    d, b = R.shape
    L = b.bit_length() - 1
    i0, i1 = rows if rows is not None else (0, m)
    vals = np.empty((d, i1 - i0, p))
    for r in range(d):
        h1, h2, s1, s2 = _hash_arrays(hp[r], m, p, L)
        w = (h1[i0:i1, None] + h2[None, :]) % b
        vals[r] = s1[i0:i1, None] * s2[None, :] * R[r][w]
    return vals.mean(axis=0) if reduce == MEAN else np.median(vals, axis=0)
