"""Seeded synthetic inputs for compressed matrix multiplication.

This module only draws input matrices (and evaluation pairs); it holds none of
the method's arithmetic, so both the library's tests and the CPU oracle's tests
can take their inputs from it.  Every generator is a pure function of its seed
(NumPy PCG64), so the same bytes reach the oracle and the GPU.

Workloads (shapes follow the paper's synthetic instances, Sec. 5.2, and the
product structures the method targets: a product dominated by a few large
entries):

* ``orthogonal_sparse``  A = Q (orthogonal factor of a Gaussian QR), B = Q^T S,
  so that A B = S exactly, S sparse with large entries (n=256, 64 nonzeros of
  N(0,1)*10 by default).
* ``planted_pm1``        A with i.i.d. uniform +-1 rows and ``pairs`` planted row
  pairs, row j copying row i entrywise with probability ``rho`` (else a fresh
  sign); B = A^T.  The product has large off-diagonal entries ~ rho*n at the
  planted pairs (a many-pair version of the paper's Lightbulb instance).
* ``orthogonal_precision`` A = Q, B = Q^T S + noise*N(0,1) (n=16384, 1024
  nonzeros N(0,1)*100 in the full size).
* ``batch_problems``     independent rectangular problems with i.i.d. N(0,1)
  entries plus planted rank-1 spikes A += alpha e_i e_t^T, B += alpha e_t e_j^T.
* ``diff_problem``       N(0,1)/sqrt(n) operands plus planted spikes and a list
  of (i, j, W) pairs for the differentiable mean estimator.
* the paper's four instance families (Sec. 5.2): ``logunit``, ``diagonal``,
  ``covariance``, ``lightbulb``.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _orthogonal(g: np.random.Generator, n: int, dtype=np.float64) -> np.ndarray:
    q, r = np.linalg.qr(g.standard_normal((n, n)))
    # fix the sign convention so Q is a deterministic function of the draw
    q *= np.sign(np.diag(r))[None, :]
    return np.ascontiguousarray(q.astype(dtype, copy=False))


def _sparse(g: np.random.Generator, m: int, p: int, nnz: int, scale: float) -> np.ndarray:
    S = np.zeros((m, p), dtype=np.float64)
    pos = g.choice(m * p, size=nnz, replace=False)
    S.flat[pos] = g.standard_normal(nnz) * scale
    return S


def orthogonal_sparse(n: int = 256, nnz: int = 64, scale: float = 10.0, seed: int = 1001):
    """A = Q, B = Q^T S with A B = S (up to FP64 rounding of Q^T Q = I)."""
    g = rng(seed)
    Q = _orthogonal(g, n)
    S = _sparse(g, n, n, nnz, scale)
    B = Q.T @ S
    return Q, np.ascontiguousarray(B), S


def planted_pm1(n: int = 8192, pairs: int = 64, rho: float = 0.9, seed: int = 1002,
                m: int | None = None, dtype=np.float64):
    """+-1 matrix A (m x n) with planted row pairs; returns (A, B=A^T, pair_list).

    pair_list is an int array (pairs, 2) of (i, j): row j copies row i entrywise
    with probability rho, otherwise draws a fresh uniform sign.
    """
    m = n if m is None else m
    g = rng(seed)
    A = (g.integers(0, 2, size=(m, n), dtype=np.int8) * 2 - 1)
    rows = g.choice(m, size=2 * pairs, replace=False)
    plist = rows.reshape(pairs, 2)
    for i, j in plist:
        keep = g.random(n) < rho
        fresh = g.integers(0, 2, size=n, dtype=np.int8) * 2 - 1
        A[j] = np.where(keep, A[i], fresh)
    A = A.astype(dtype)
    return A, np.ascontiguousarray(A.T), plist


def orthogonal_precision(n: int = 16384, nnz: int = 1024, scale: float = 100.0,
                         noise: float = 1e-3, seed: int = 1003, dtype=np.float32,
                         device=None):
    """A = Q, B = Q^T S + noise*N(0,1).  With ``device`` (a torch device) the QR
    runs there (torch.linalg.qr) and torch tensors are returned."""
    if device is None:
        g = rng(seed)
        Q = _orthogonal(g, n)
        S = _sparse(g, n, n, nnz, scale)
        B = Q.T @ S + noise * g.standard_normal((n, n))
        return Q.astype(dtype), np.ascontiguousarray(B.astype(dtype)), S
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    X = torch.randn(n, n, generator=gen, device=device, dtype=torch.float32)
    Q, Rq = torch.linalg.qr(X)
    Q = Q * torch.sign(torch.diagonal(Rq))[None, :]
    del X, Rq
    g = rng(seed)
    S = _sparse(g, n, n, nnz, scale)
    St = torch.from_numpy(S).to(device=device, dtype=torch.float32)
    B = Q.T @ St + noise * torch.randn(n, n, generator=gen, device=device)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    return Q.to(tdt).contiguous(), B.to(tdt).contiguous(), S


def planted_spikes(g: np.random.Generator, A: np.ndarray, B: np.ndarray, count: int,
                   value: float):
    """Add rank-1 spikes A += a e_i e_t^T, B += a e_t e_j^T with a = sqrt(value) and
    a distinct inner index t per spike, so (A B)[i, j] grows by ``value``."""
    m, k = A.shape
    p = B.shape[1]
    count = min(count, k)
    ts = g.choice(k, size=count, replace=False)
    ii = g.integers(0, m, size=count)
    jj = g.integers(0, p, size=count)
    a = math.sqrt(value)
    for i, t, j in zip(ii, ts, jj):
        A[i, t] += a
        B[t, j] += a
    return np.stack([ii, jj], axis=1)


def batch_problems(count: int = 256, lo: int = 512, hi: int = 4096, spikes: int = 16,
                   log2b_lo: int = 10, log2b_hi: int = 15, seed: int = 1004,
                   dtype=np.float32, uniform_log2b: int | None = None):
    """Independent problems (A_q, B_q, log2b_q, spike positions).

    m, k, p are uniform integers in [lo, hi]; entries N(0,1); ``spikes`` planted
    entries of magnitude 50*sqrt(k); log2 b uniform in [log2b_lo, log2b_hi]
    unless ``uniform_log2b`` fixes it."""
    g = rng(seed)
    out = []
    for _ in range(count):
        m, k, p = (int(v) for v in g.integers(lo, hi + 1, size=3))
        A = g.standard_normal((m, k))
        B = g.standard_normal((k, p))
        pos = planted_spikes(g, A, B, spikes, 50.0 * math.sqrt(k))
        L = uniform_log2b if uniform_log2b is not None else int(g.integers(log2b_lo, log2b_hi + 1))
        out.append((A.astype(dtype), B.astype(dtype), L, pos))
    return out


def batch_problems_device(count: int = 256, lo: int = 512, hi: int = 4096, spikes: int = 16,
                          log2b_lo: int = 10, log2b_hi: int = 15, seed: int = 1004,
                          device="cuda", uniform_log2b: int | None = None):
    """The distribution of ``batch_problems`` drawn on a torch device, with the
    left operand produced directly transposed (A^T, k x m, float32).  Sizes,
    sketch lengths and spike positions come from NumPy PCG64(seed); entries
    from a torch generator seeded with ``seed``.  Returns a list of
    (At, B, log2b, spike positions)."""
    import torch
    g = rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = []
    for _ in range(count):
        m, k, p = (int(v) for v in g.integers(lo, hi + 1, size=3))
        At = torch.randn(k, m, generator=gen, device=device, dtype=torch.float32)
        B = torch.randn(k, p, generator=gen, device=device, dtype=torch.float32)
        cnt = min(spikes, k)
        ts = g.choice(k, size=cnt, replace=False)
        ii = g.integers(0, m, size=cnt)
        jj = g.integers(0, p, size=cnt)
        a = math.sqrt(50.0 * math.sqrt(k))
        for i, t, j in zip(ii, ts, jj):
            At[int(t), int(i)] += a
            B[int(t), int(j)] += a
        L = uniform_log2b if uniform_log2b is not None else int(g.integers(log2b_lo, log2b_hi + 1))
        out.append((At, B, L, np.stack([ii, jj], axis=1)))
    return out


def diff_problem(n: int = 4096, spikes: int = 256, pairs: int = 4096, seed: int = 1005,
                 dtype=np.float32, spike_value: float = 1.0):
    """(A, B, I, J, W): N(0,1)/sqrt(n) operands with planted spikes, and a fixed
    list of (I, J) pairs (including the spikes) with weights W ~ N(0,1)."""
    g = rng(seed)
    A = g.standard_normal((n, n)) / math.sqrt(n)
    B = g.standard_normal((n, n)) / math.sqrt(n)
    pos = planted_spikes(g, A, B, spikes, spike_value)
    extra = pairs - pos.shape[0]
    I = np.concatenate([pos[:, 0], g.integers(0, n, size=max(extra, 0))])[:pairs]
    J = np.concatenate([pos[:, 1], g.integers(0, n, size=max(extra, 0))])[:pairs]
    W = g.standard_normal(pairs)
    return (A.astype(dtype), B.astype(dtype), I.astype(np.int32), J.astype(np.int32),
            W.astype(np.float64))


# ---- the paper's instance families (Sec. 5.2) ----------------------------------

def logunit(n: int, seed: int = 2001):
    """C = D P: log2 n entries equal to 1, the rest 0.01 * 0.01 = 1e-4, one per
    row/column.  A = D1 A~, B = A~^{-1} D2 P with floor(log2 n / 2) (resp. ceil)
    entries 100 and the rest 0.01 on D1 (resp. D2, on disjoint positions).  (The
    paper's text calls the small entries 0.001; its construction, followed here,
    makes them 1e-4.)  (The paper
    writes A = A~ D1 but derives A B = D1 A~ A~^{-1} D2 P = D1 D2 P, which needs
    D1 on the left.)"""
    g = rng(seed)
    L = int(math.log2(n))
    At = g.uniform(-1.0, 1.0, size=(n, n))
    idx = g.permutation(n)
    d1 = np.full(n, 0.01)
    d2 = np.full(n, 0.01)
    d1[idx[: L // 2]] = 100.0
    d2[idx[L // 2: L // 2 + (L + 1) // 2]] = 100.0
    perm = g.permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1.0
    A = d1[:, None] * At
    B = np.linalg.solve(At, np.diag(d2) @ P)
    C = (d1 * d2)[:, None] * P
    return np.ascontiguousarray(A), np.ascontiguousarray(B), C


def diagonal(n: int, seed: int = 2002):
    """C = P D with 0.5 <= |D_ii| <= 1; A ~ U(-1,1), B = A^{-1} P D."""
    g = rng(seed)
    A = g.uniform(-1.0, 1.0, size=(n, n))
    mag = g.uniform(0.5, 1.0, size=n)
    D = mag * np.where(g.random(n) < 0.5, -1.0, 1.0)
    perm = g.permutation(n)
    P = np.zeros((n, n))
    P[np.arange(n), perm] = 1.0
    PD = P * D[None, :]
    B = np.linalg.solve(A, PD)
    return A, np.ascontiguousarray(B), PD


def covariance(n: int, rho: float = 0.8, seed: int = 2003):
    """Gaussian A, B~ (scaled by 1/sqrt(n) so inner products are correlations),
    with column j* of B set to rho*a_{i*} + sqrt(1 - rho^2)*b~_{j*}."""
    g = rng(seed)
    A = g.standard_normal((n, n)) / math.sqrt(n)
    B = g.standard_normal((n, n)) / math.sqrt(n)
    i_s, j_s = int(g.integers(0, n)), int(g.integers(0, n))
    B[:, j_s] = rho * A[i_s, :] + math.sqrt(1.0 - rho * rho) * B[:, j_s]
    return A, B, (i_s, j_s)


def lightbulb(n: int, rho: float = 0.8, seed: int = 2004):
    """+-1 entries scaled by 1/n so inner products are correlations; column j* of
    B copies row i* of A with n(1-rho)/2 sign flips."""
    g = rng(seed)
    A = (g.integers(0, 2, size=(n, n)) * 2 - 1).astype(np.float64)
    B = (g.integers(0, 2, size=(n, n)) * 2 - 1).astype(np.float64)
    i_s, j_s = int(g.integers(0, n)), int(g.integers(0, n))
    col = A[i_s, :].copy()
    flips = g.choice(n, size=int(round(n * (1.0 - rho) / 2.0)), replace=False)
    col[flips] *= -1.0
    B[:, j_s] = col
    return A / math.sqrt(n), B / math.sqrt(n), (i_s, j_s)


def gpu_planted_pm1(n: int, pairs: int, rho: float, seed: int, device, dtype):
    """Same distribution as ``planted_pm1`` drawn on a torch device (for sizes
    where host generation and transfer dominate a benchmark's set-up).  Not
    bit-identical to the NumPy version; tests compare GPU and oracle on the same
    tensor, so only the distribution matters here."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    A = torch.randint(0, 2, (n, n), generator=gen, device=device, dtype=torch.int8)
    A = (A * 2 - 1)
    rows = torch.randperm(n, generator=gen, device=device)[: 2 * pairs].view(pairs, 2)
    keep = torch.rand(pairs, n, generator=gen, device=device) < rho
    fresh = torch.randint(0, 2, (pairs, n), generator=gen, device=device, dtype=torch.int8) * 2 - 1
    A[rows[:, 1]] = torch.where(keep, A[rows[:, 0]], fresh)
    A = A.to(dtype)
    return A, A.t().contiguous(), rows
