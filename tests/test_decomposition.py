"""The two identities the GPU design rests on, checked on the CPU in FP64
against the oracle's transform and hashes (no GPU code is involved).

1. Frequency split (the kernels' work decomposition): with b = C * N and an
   index u = u_hi * N + u_lo, the length-b transform of a bucketed column is,
   slice by slice, a length-N transform of the column scattered with an extra
   sign (-1)^popcount(u_hi & h_hi(i)) on the low bucket bits h_lo(i):
       (H_b x)[u_hi * N + u_lo] = (H_N f_{u_hi})[u_lo],
       f_{u_hi}[v] = sum_{i : h_lo(i) = v} s(i) (-1)^popcount(u_hi & h_hi(i)) a_i.
   So a CTA that owns slice u_hi needs no data from any other CTA.

2. Fixed-point scatter: values a_i scaled by a power of two 2^e with
   c_max * max|a| * 2^e < 2^29 (c_max: the most values sharing a bucket) round
   to integers whose bucket sums stay below 2^30 in magnitude, so 32-bit integer
   atomics add them exactly in any order; the sums scaled back by 2^-e differ
   from the exact ones by at most (number of values in the bucket) * 2^-e / 2.
"""
import math

import numpy as np

from oracle import oracle as orc


def _popc_parity(x):
    return np.array([bin(int(v)).count("1") & 1 for v in np.atleast_1d(x)])


def test_frequency_split_equals_full_transform():
    g = np.random.default_rng(1)
    hp = orc.draw_hashes(31, 3)
    m = 700
    for L, Llo in [(8, 5), (10, 4), (12, 12), (9, 1)]:
        N, C = 1 << Llo, 1 << (L - Llo)
        for r in range(3):
            a1, c1, as1, cs1 = (int(hp[r][q]) for q in (0, 1, 4, 5))
            h = orc.buckets(a1, c1, m, L).astype(np.int64)
            s = orc.signs(as1, cs1, m).astype(np.float64)
            col = g.standard_normal(m)
            x = np.zeros(1 << L)
            np.add.at(x, h, s * col)
            full = orc.fwht(x)
            h_lo, h_hi = h & (N - 1), h >> Llo
            for u_hi in range(C):
                sgn = 1.0 - 2.0 * _popc_parity(h_hi & u_hi)
                f = np.zeros(N)
                np.add.at(f, h_lo, s * sgn * col)
                part = orc.fwht(f)
                ref = full[u_hi * N:(u_hi + 1) * N]
                assert np.abs(part - ref).max() <= 1e-12 * np.abs(col).sum()


def test_fixed_point_bucket_sums_are_exact_integers_within_the_bound():
    g = np.random.default_rng(2)
    hp = orc.draw_hashes(32, 1)
    m, L = 5000, 10
    h = orc.buckets(int(hp[0][0]), int(hp[0][1]), m, L).astype(np.int64)
    s = orc.signs(int(hp[0][4]), int(hp[0][5]), m)
    cmax = int(np.bincount(h, minlength=1 << L).max())
    for scale in (1e-20, 1.0, 3.7e3, 1e15):
        col = g.standard_normal(m) * scale
        col[7] = 50.0 * scale                       # one dominant value
        amax = float(np.abs(col).max())
        e = 29 - math.ceil(math.log2(cmax * amax))  # c_max * max|a| * 2^e <= 2^29
        q = np.rint(col * s * 2.0 ** e).astype(np.int64)
        sums = np.zeros(1 << L, dtype=np.int64)
        np.add.at(sums, h, q)
        assert np.abs(sums).max() < 2 ** 30          # exact in 32-bit integers
        # any order of the additions gives the same integers; scaled back, each
        # bucket is within (its count) * 2^-e / 2 of the exact FP64 sum
        exact = np.zeros(1 << L)
        np.add.at(exact, h, col * s)
        count = np.bincount(h, minlength=1 << L)
        assert np.all(np.abs(sums * 2.0 ** -e - exact) <= count * 2.0 ** -e / 2 * (1 + 1e-12))
