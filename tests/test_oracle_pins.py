"""Pins of the FP64 CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against something the paper or mathematics fixes:
published generator outputs, closed forms and special cases of the hash family
(Sec. 4.2), the explicit Sylvester Hadamard matrix (Sec. 3.2), brute-force XOR
convolution (Eq. 1), the bucket identity of Compress (Algorithm 1, with the
product computed by a plain matrix multiply), exact recovery of a sparse
product, unbiasedness and the variance bound (Sec. 3.1), and finite differences
of the bilinear mean estimator.  None of these re-types the oracle's own code.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2601_09477_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1


def _golden_hex(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [int(line.strip(), 16) for line in f
                if line.strip() and not line.startswith("#")]


# ---------------------------------------------------------------- hashes

def test_splitmix64_published_outputs():
    want = _golden_hex("splitmix64_seed0.txt")
    got = [int(v) for v in orc.splitmix64_stream(0, len(want))]
    assert got == want


def test_draw_hashes_order():
    # (a, c) of h1, h2, s1, s2 per repetition are consecutive generator outputs
    hp = orc.draw_hashes(0, 2)
    want = _golden_hex("splitmix64_seed0.txt")
    assert [int(v) for v in hp[0, :3]] == want


@pytest.mark.parametrize("L", [1, 2, 5, 12, 16, 18, 31])
def test_bucket_shift_special_case(L):
    # a = 2^(64-L), c = 0: (a x mod 2^64) >> (64-L) keeps the low L bits of x
    a = 1 << (64 - L)
    xs = [0, 1, 2, 3, (1 << L) - 1, 1 << L, (1 << L) + 5, 123456789, (1 << 32) - 1]
    for x in xs:
        assert orc.bucket(a, 0, x, L) == x % (1 << L)


@pytest.mark.parametrize("L", [1, 4, 16, 31])
def test_bucket_constant_and_wraparound(L):
    # a = 0: the bucket is the top L bits of c for every key
    c = 0xDEADBEEFCAFEF00D
    for x in [0, 7, 99999]:
        assert orc.bucket(0, c, x, L) == c >> (64 - L)
    # a = 1, c = 2^64 - 1: x = 0 gives all ones, x = 1 wraps to 0
    assert orc.bucket(1, M64, 0, L) == (1 << L) - 1
    assert orc.bucket(1, M64, 1, L) == 0
    # a = 2^63 + 1 wraps: a * 2 = 2 (mod 2^64)
    assert orc.bucket((1 << 63) + 1, 0, 2, L) == (2 >> (64 - L))


def test_sign_special_cases():
    assert orc.sign(0, 1 << 63, 5) == -1          # top bit set -> -1
    assert orc.sign(0, (1 << 63) - 1, 5) == 1     # top bit clear -> +1
    # a = 2^63: a x mod 2^64 = 2^63 (x mod 2): odd keys -> -1, even keys -> +1
    for x in range(10):
        assert orc.sign(1 << 63, 0, x) == (-1 if x % 2 else 1)


def test_bucket_arrays_match_scalar():
    hp = orc.draw_hashes(77, 1)
    a, c = int(hp[0, 0]), int(hp[0, 1])
    arr = orc.buckets(a, c, 1000, 10)
    assert [orc.bucket(a, c, x, 10) for x in range(0, 1000, 37)] == list(arr[::37])
    s = orc.signs(int(hp[0, 4]), int(hp[0, 5]), 1000)
    assert set(np.unique(s)) <= {-1, 1}


def test_bucket_uniformity():
    # 2-wise independent family: buckets of 2^16 keys into 2^8 buckets are
    # near-uniform for a random (a, c) -- chi-square well under its 1e-6 tail
    hp = orc.draw_hashes(5, 4)
    for r in range(4):
        h = orc.buckets(int(hp[r, 0]), int(hp[r, 1]), 1 << 16, 8)
        cnt = np.bincount(h, minlength=256)
        exp = (1 << 16) / 256
        chi2 = float(((cnt - exp) ** 2 / exp).sum())
        assert chi2 < 400.0  # df = 255; P(chi2 > 400) ~ 1e-8


# ---------------------------------------------------------------- FWHT

def _sylvester(L):
    H = np.array([[1.0]])
    for _ in range(L):
        H = np.block([[H, H], [H, -H]])
    return H


@pytest.mark.parametrize("L", list(range(0, 11)))
def test_fwht_matches_sylvester_matrix(L):
    b = 1 << L
    g = np.random.default_rng(L)
    x = g.standard_normal(b)
    np.testing.assert_allclose(orc.fwht(x), _sylvester(L) @ x, rtol=0, atol=1e-11 * b)


def test_fwht_closed_form_entries():
    L = 6
    b = 1 << L
    for v in range(b):
        e = np.zeros(b)
        e[v] = 1.0
        col = orc.fwht(e)
        want = np.array([(-1.0) ** bin(u & v).count("1") for u in range(b)])
        assert np.array_equal(col, want)


@pytest.mark.parametrize("L", [1, 3, 8, 12])
def test_fwht_involution_scale(L):
    # H H = b I for the unnormalised transform
    b = 1 << L
    x = np.random.default_rng(3).standard_normal(b)
    np.testing.assert_allclose(orc.fwht(orc.fwht(x)), b * x, rtol=1e-12, atol=1e-12 * b)


@pytest.mark.parametrize("L", [1, 2, 4, 6])
def test_xor_convolution_identity(L):
    # (1/b) H(Hx o Hy) equals the brute-force XOR convolution of Eq. 1
    b = 1 << L
    g = np.random.default_rng(L + 10)
    x = g.standard_normal(b)
    y = g.standard_normal(b)
    brute = np.zeros(b)
    for i in range(b):
        for j in range(b):
            brute[i ^ j] += x[i] * y[j]
    got = orc.fwht(orc.fwht(x) * orc.fwht(y)) / b
    np.testing.assert_allclose(got, brute, rtol=0, atol=1e-12 * b)


# ---------------------------------------------------------------- Compress

def _direct_R(C, hp, L):
    """R_r[w] = sum_{(i,j): h1(i) XOR h2(j) = w} s1(i) s2(j) C[i, j], with C given."""
    m, p = C.shape
    d = hp.shape[0]
    R = np.zeros((d, 1 << L))
    for r in range(d):
        a1, c1, a2, c2, as1, cs1, as2, cs2 = (int(v) for v in hp[r])
        h1 = orc.buckets(a1, c1, m, L).astype(np.int64)
        h2 = orc.buckets(a2, c2, p, L).astype(np.int64)
        s1 = orc.signs(as1, cs1, m).astype(np.float64)
        s2 = orc.signs(as2, cs2, p).astype(np.float64)
        w = h1[:, None] ^ h2[None, :]
        np.add.at(R[r], w.ravel(), (s1[:, None] * s2[None, :] * C).ravel())
    return R


@pytest.mark.parametrize("m,k,p,L,d", [(16, 8, 12, 4, 3), (64, 40, 50, 6, 5),
                                       (200, 33, 150, 9, 2), (7, 300, 9, 2, 4)])
def test_compress_equals_bucket_definition(m, k, p, L, d):
    g = np.random.default_rng(m * 1000 + p)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    hp = orc.draw_hashes(1234 + m, d)
    R = orc.compress(A, B, hp, L)
    Rd = _direct_R(A @ B, hp, L)
    scale = np.abs(A).sum() * np.abs(B).sum() / k
    np.testing.assert_allclose(R, Rd, rtol=0, atol=1e-12 * scale)


def test_compress_xor_convolution_per_inner_index():
    # R_r = sum_t x_t XOR-conv y_t with the sketches built by direct scatter
    m, k, p, L = 10, 5, 9, 3
    b = 1 << L
    g = np.random.default_rng(9)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    hp = orc.draw_hashes(99, 1)
    a1, c1, a2, c2, as1, cs1, as2, cs2 = (int(v) for v in hp[0])
    want = np.zeros(b)
    for t in range(k):
        x = np.zeros(b)
        y = np.zeros(b)
        for i in range(m):
            x[orc.bucket(a1, c1, i, L)] += orc.sign(as1, cs1, i) * A[i, t]
        for j in range(p):
            y[orc.bucket(a2, c2, j, L)] += orc.sign(as2, cs2, j) * B[t, j]
        for u in range(b):
            for v in range(b):
                want[u ^ v] += x[u] * y[v]
    np.testing.assert_allclose(orc.compress(A, B, hp, L)[0], want, rtol=0, atol=1e-12)


def test_compress_transposed_layout_and_threads():
    g = np.random.default_rng(4)
    A = g.standard_normal((30, 20))
    B = g.standard_normal((20, 25))
    hp = orc.draw_hashes(3, 3)
    R0 = orc.compress(A, B, hp, 5)
    R1 = orc.compress(np.ascontiguousarray(A.T), B, hp, 5, transA=True)
    R2 = orc.compress(A, B, hp, 5, nthreads=4)
    np.testing.assert_array_equal(R0, R1)
    np.testing.assert_allclose(R0, R2, rtol=0, atol=1e-12)


def test_compress_linear_in_each_operand():
    g = np.random.default_rng(8)
    A1, A2 = g.standard_normal((2, 24, 16))
    B = g.standard_normal((16, 20))
    hp = orc.draw_hashes(8, 2)
    lhs = orc.compress(2.0 * A1 - 3.0 * A2, B, hp, 5)
    rhs = 2.0 * orc.compress(A1, B, hp, 5) - 3.0 * orc.compress(A2, B, hp, 5)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-11)


def test_compress_pm1_inputs_are_exact_integers():
    A, B, _ = wl.planted_pm1(n=128, pairs=4, seed=5)
    hp = orc.draw_hashes(11, 3)
    R = orc.compress(A, B, hp, 7)
    assert np.array_equal(R, np.round(R))
    assert np.array_equal(R, _direct_R(A @ B, hp, 7))


# ---------------------------------------------------------------- Decompress

def test_decompress_median_and_mean_of_gathered_values():
    g = np.random.default_rng(21)
    for d in (1, 2, 3, 4, 5, 9):
        L = 6
        R = g.standard_normal((d, 1 << L))
        hp = orc.draw_hashes(100 + d, d)
        for (i, j) in [(0, 0), (3, 17), (41, 2)]:
            vals = []
            for r in range(d):
                a1, c1, a2, c2, as1, cs1, as2, cs2 = (int(v) for v in hp[r])
                w = orc.bucket(a1, c1, i, L) ^ orc.bucket(a2, c2, j, L)
                vals.append(orc.sign(as1, cs1, i) * orc.sign(as2, cs2, j) * R[r, w])
            assert orc.decompress(R, hp, i, j) == np.median(vals)
            assert abs(orc.decompress(R, hp, i, j, orc.MEAN) - np.mean(vals)) < 1e-15


def test_extract_rows_and_heavy_hitters_consistent():
    g = np.random.default_rng(5)
    R = g.standard_normal((5, 64)) * 3
    hp = orc.draw_hashes(6, 5)
    C = orc.extract(R, hp, 20, 30)
    part = orc.extract(R, hp, 20, 30, rows=(5, 9))
    np.testing.assert_array_equal(C[5:9], part)
    I, J, V = orc.heavy_hitters(R, hp, 20, 30, 2.5)
    ii, jj = np.nonzero(np.abs(C) >= 2.5)
    np.testing.assert_array_equal(I, ii)
    np.testing.assert_array_equal(J, jj)
    np.testing.assert_array_equal(V, C[ii, jj])


def test_exact_recovery_of_sparse_product():
    # n = 256, S with 64 nonzeros, b = 2^12 >= 8 nnz: the median recovers S
    # except where collisions hit a majority of repetitions (rare)
    A, B, S = wl.orthogonal_sparse(seed=1001)
    hp = orc.draw_hashes(2001, 5)
    R = orc.compress(A, B, hp, 12)
    C = orc.extract(R, hp, 256, 256)
    err = np.abs(C - S)
    assert np.mean(err < 1e-9) > 0.999
    # every wrong entry is explained by collisions with another nonzero of S in
    # a majority of the repetitions (Pagh's error identity, Sec. 6.4)
    nz = list(zip(*np.nonzero(S)))
    bad = list(zip(*np.nonzero(err >= 1e-9)))
    for (i, j) in bad:
        hits = 0
        for r in range(5):
            a1, c1, a2, c2 = (int(v) for v in hp[r, :4])
            w = orc.bucket(a1, c1, i, 12) ^ orc.bucket(a2, c2, j, 12)
            hits += any(orc.bucket(a1, c1, int(u), 12) ^ orc.bucket(a2, c2, int(v), 12) == w
                        for (u, v) in nz if (u, v) != (i, j))
        assert hits >= 3
    I, J, _ = orc.heavy_hitters(R, hp, 256, 256, 5.0)
    si, sj = np.nonzero(np.abs(S) >= 5.0)
    found = set(zip(I.tolist(), J.tolist()))
    assert set(zip(si.tolist(), sj.tolist())) <= found
    assert found - set(zip(si.tolist(), sj.tolist())) <= set(bad)


def test_unbiased_and_variance_bound():
    # d = 1: E[Chat_ij] = C_ij and Var <= ||C||_F^2 / b (Sec. 3.1, Theorem 1)
    g = np.random.default_rng(31)
    n, L, S = 24, 4, 3000
    A = g.standard_normal((n, n))
    B = g.standard_normal((n, n))
    C = A @ B
    est = np.empty((S, 3))
    pairs = [(0, 0), (5, 7), (23, 11)]
    for s in range(S):
        hp = orc.draw_hashes(10_000 + s, 1)
        R = orc.compress(A, B, hp, L)
        est[s] = [orc.decompress(R, hp, i, j) for (i, j) in pairs]
    bound = (C ** 2).sum() / (1 << L)
    for q, (i, j) in enumerate(pairs):
        assert abs(est[:, q].mean() - C[i, j]) < 5.0 * math.sqrt(bound / S)
        assert est[:, q].var() <= 1.1 * bound


# ---------------------------------------------------------------- cyclic form
# Pagh's original (Sec. 3.1): bucket h1(i) + h2(j) mod b, products through the
# cyclic convolution of Sec. 2.  The oracle takes it through numpy's FFT; these
# pins check it against loops that use neither the FFT nor the oracle's scatter.

def _sketch_loops(col, a, c, sa, sc, L):
    # x[u] = sum over i with h(i) = u of s(i) col[i], element by element
    x = [0.0] * (1 << L)
    for i, v in enumerate(col):
        x[orc.bucket(a, c, i, L)] += orc.sign(sa, sc, i) * v
    return x


def test_cyclic_matches_brute_force_convolution():
    g = np.random.default_rng(41)
    m, k, p, L, d = 37, 4, 29, 4, 2
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    hp = orc.draw_hashes(77, d)
    R = orc.compress_cyclic(A, B, hp, L)
    b = 1 << L
    for r in range(d):
        a1, c1, a2, c2, as1, cs1, as2, cs2 = (int(v) for v in hp[r])
        want = [0.0] * b
        for t in range(k):
            x = _sketch_loops(A[:, t], a1, c1, as1, cs1, L)
            y = _sketch_loops(B[t, :], a2, c2, as2, cs2, L)
            for u in range(b):
                for v in range(b):
                    want[(u + v) % b] += x[u] * y[v]
        np.testing.assert_allclose(R[r], want, rtol=0, atol=1e-12)


def test_cyclic_bucket_identity_and_pm1_integers():
    # R_r[w] = sum of s1(i) s2(j) C[i, j] over h1(i) + h2(j) = w (mod b); on +-1
    # inputs every R value is an integer
    g = np.random.default_rng(43)
    m, k, p, L = 9, 6, 8, 3
    A = np.where(g.random((m, k)) < 0.5, -1.0, 1.0)
    B = np.where(g.random((k, p)) < 0.5, -1.0, 1.0)
    hp = orc.draw_hashes(5, 2)
    R = orc.compress_cyclic(A, B, hp, L)
    b = 1 << L
    for r in range(2):
        a1, c1, a2, c2, as1, cs1, as2, cs2 = (int(v) for v in hp[r])
        want = [0] * b
        for i in range(m):
            for j in range(p):
                cij = sum(int(A[i, t]) * int(B[t, j]) for t in range(k))
                w = (orc.bucket(a1, c1, i, L) + orc.bucket(a2, c2, j, L)) % b
                want[w] += orc.sign(as1, cs1, i) * orc.sign(as2, cs2, j) * cij
        np.testing.assert_allclose(R[r], want, rtol=0, atol=1e-9)
        assert np.abs(R[r] - np.round(R[r])).max() < 1e-9


def test_cyclic_exact_recovery_of_sparse_product():
    # the n = 256 case with cyclic buckets: S recovered except where collisions
    # hit a majority of repetitions
    A, B, S = wl.orthogonal_sparse(seed=1001)
    hp = orc.draw_hashes(2001, 5)
    R = orc.compress_cyclic(A, B, hp, 12)
    C = orc.extract_cyclic(R, hp, 256, 256)
    err = np.abs(C - S)
    assert np.mean(err < 1e-9) > 0.999
    nz = list(zip(*np.nonzero(S)))
    for (i, j) in zip(*np.nonzero(err >= 1e-9)):
        hits = 0
        for r in range(5):
            a1, c1, a2, c2 = (int(v) for v in hp[r, :4])
            w = (orc.bucket(a1, c1, int(i), 12) + orc.bucket(a2, c2, int(j), 12)) % 4096
            hits += any((orc.bucket(a1, c1, int(u), 12) + orc.bucket(a2, c2, int(v), 12)) % 4096 == w
                        for (u, v) in nz if (u, v) != (i, j))
        assert hits >= 3


def test_cyclic_unbiased_and_variance_bound():
    # d = 1: E[Chat_ij] = C_ij and Var <= ||C||_F^2 / b hold for the cyclic form
    # too (Sec. 3.1; Pagh's Theorem 3.1)
    g = np.random.default_rng(37)
    n, L, S = 20, 4, 2000
    A = g.standard_normal((n, n))
    B = g.standard_normal((n, n))
    C = A @ B
    pairs = [(0, 0), (4, 9), (19, 2)]
    est = np.empty((S, len(pairs)))
    for s in range(S):
        hp = orc.draw_hashes(20_000 + s, 1)
        Cs = orc.extract_cyclic(orc.compress_cyclic(A, B, hp, L), hp, n, n)
        est[s] = [Cs[i, j] for (i, j) in pairs]
    bound = (C ** 2).sum() / (1 << L)
    for q, (i, j) in enumerate(pairs):
        assert abs(est[:, q].mean() - C[i, j]) < 5.0 * math.sqrt(bound / S)
        assert est[:, q].var() <= 1.1 * bound


# ---------------------------------------------------------------- adjoint

def _loss(A, B, hp, L, I, J, W):
    R = orc.compress(A, B, hp, L)
    return float(np.dot(W, orc.mean_at_pairs(R, hp, I, J)))


def test_adjoint_matches_finite_differences():
    g = np.random.default_rng(17)
    m, k, p, L, d = 12, 7, 10, 4, 3
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    hp = orc.draw_hashes(55, d)
    I = g.integers(0, m, 15).astype(np.int32)
    J = g.integers(0, p, 15).astype(np.int32)
    W = g.standard_normal(15)
    dA, dB = orc.adjoint(A, B, hp, L, I, J, W)
    # the loss is bilinear: a unit step in one entry gives the exact derivative
    for (i, t) in [(0, 0), (5, 3), (11, 6)]:
        E = np.zeros_like(A)
        E[i, t] = 1.0
        fd = (_loss(A + E, B, hp, L, I, J, W) - _loss(A - E, B, hp, L, I, J, W)) / 2
        assert abs(fd - dA[i, t]) < 1e-9 * (1 + abs(fd))
    for (t, j) in [(0, 0), (6, 9), (3, 4)]:
        E = np.zeros_like(B)
        E[t, j] = 1.0
        fd = (_loss(A, B + E, hp, L, I, J, W) - _loss(A, B - E, hp, L, I, J, W)) / 2
        assert abs(fd - dB[t, j]) < 1e-9 * (1 + abs(fd))


def test_adjoint_equals_dense_jacobian():
    # assemble dL/dA column by column from the forward map (the loss is linear in A)
    g = np.random.default_rng(23)
    m, k, p, L, d = 6, 4, 5, 3, 2
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    hp = orc.draw_hashes(8, d)
    I = np.array([0, 2, 5, 1], dtype=np.int32)
    J = np.array([4, 0, 3, 3], dtype=np.int32)
    W = np.array([1.5, -0.5, 2.0, 1.0])
    dA, dB = orc.adjoint(A, B, hp, L, I, J, W)
    Z = np.zeros_like(A)
    base = _loss(Z, B, hp, L, I, J, W)
    jac = np.zeros_like(A)
    for i in range(m):
        for t in range(k):
            E = np.zeros_like(A)
            E[i, t] = 1.0
            jac[i, t] = _loss(E, B, hp, L, I, J, W) - base
    np.testing.assert_allclose(dA, jac, rtol=0, atol=1e-12)
    assert dB.shape == B.shape


def test_R_entry_matches_compress():
    g = np.random.default_rng(41)
    A = g.standard_normal((40, 13))
    B = g.standard_normal((13, 35))
    hp = orc.draw_hashes(77, 2)
    R = orc.compress(A, B, hp, 6)
    for r, w in [(0, 0), (1, 17), (0, 63), (1, 5)]:
        assert abs(orc.R_entry(A, B, hp, 6, r, w) - R[r, w]) < 1e-12 * 40
    At = np.ascontiguousarray(A.T)
    assert abs(orc.R_entry(At, B, hp, 6, 1, 9, transA=True) - R[1, 9]) < 1e-12 * 40
