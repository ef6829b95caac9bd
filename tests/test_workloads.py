"""The seeded input generators against the recipes they state (CPU): the
products they are built to have, their shapes, ranges and planted structure.
The generators hold none of the method's arithmetic; these checks only pin
that the synthetic inputs are what the benchmark and the tests say they are."""
import math

import numpy as np

from paper_2601_09477_gb300 import workloads as wl


def test_orthogonal_sparse_product_is_S():
    A, B, S = wl.orthogonal_sparse(n=128, nnz=40, scale=10.0, seed=3)
    assert np.count_nonzero(S) == 40
    assert np.abs(A.T @ A - np.eye(128)).max() < 1e-12
    assert np.abs(A @ B - S).max() < 1e-11 * np.abs(S).max()


def test_planted_pm1_pairs_agree_at_the_planted_rate():
    n, pairs, rho = 2048, 16, 0.9
    A, B, plist = wl.planted_pm1(n=n, pairs=pairs, rho=rho, seed=11)
    assert set(np.unique(A)) == {-1.0, 1.0}
    assert np.array_equal(B, A.T)
    assert len(set(plist.ravel().tolist())) == 2 * pairs          # disjoint rows
    # row j copies row i with probability rho, else a fresh sign that agrees
    # half the time: expected agreement rho + (1 - rho) / 2 = 0.95
    agree = np.mean([np.mean(A[i] == A[j]) for i, j in plist])
    sd = math.sqrt(0.95 * 0.05 / (n * pairs))
    assert abs(agree - 0.95) < 5 * sd
    # the planted products C[i, j] = <a_i, a_j> are about 0.9 n
    C = A @ B
    vals = np.array([C[i, j] for i, j in plist])
    assert np.all(np.abs(vals - rho * n) < 6 * math.sqrt(n))


def test_planted_spikes_add_the_rank_one_terms():
    g = np.random.default_rng(4)
    A = g.standard_normal((60, 50))
    B = g.standard_normal((50, 70))
    A0, B0 = A.copy(), B.copy()
    pos = wl.planted_spikes(np.random.default_rng(9), A, B, 5, 400.0)
    dA, dB = A - A0, B - B0
    # each spike adds a e_i e_t^T to A and a e_t e_j^T to B, a = sqrt(400), at
    # distinct t: the product gains exactly a^2 e_i e_j^T per spike plus the
    # cross terms a e_i (e_t^T B0) + a (A0 e_t) e_j^T
    assert np.count_nonzero(dA) == 5 and np.count_nonzero(dB) == 5
    ts = np.nonzero(dA)[1]
    assert len(set(ts.tolist())) == 5
    assert np.allclose(dA[dA != 0], 20.0) and np.allclose(dB[dB != 0], 20.0)
    assert np.array_equal(np.sort(np.nonzero(dA)[0]), np.sort(pos[:, 0]))
    assert np.allclose(A @ B - A0 @ B0, dA @ B0 + A0 @ dB + dA @ dB)
    assert np.allclose(np.diag(dA[pos[:, 0]] @ dB[:, pos[:, 1]]), 400.0)


def test_batch_problem_sizes_and_sketch_lengths():
    probs = wl.batch_problems(count=12, lo=64, hi=256, spikes=4, log2b_lo=10, log2b_hi=15,
                              seed=5)
    for A, B, L, pos in probs:
        m, k = A.shape
        assert B.shape[0] == k and 64 <= m <= 256 and 64 <= k <= 256 and 64 <= B.shape[1] <= 256
        assert 10 <= L <= 15 and A.dtype == np.float32 and pos.shape == (4, 2)


def test_diff_problem_pairs_start_with_the_spikes():
    A, B, I, J, W = wl.diff_problem(n=128, spikes=8, pairs=64, seed=2)
    assert A.shape == B.shape == (128, 128) and I.shape == J.shape == W.shape == (64,)
    assert I.min() >= 0 and I.max() < 128 and J.min() >= 0 and J.max() < 128
    C = A.astype(np.float64) @ B.astype(np.float64)
    # the first 8 pairs are the unit spikes, far above the N(0,1)/sqrt(n) background
    assert np.all(np.abs(C[I[:8], J[:8]]) > 0.5)


def test_logunit_product():
    n = 64
    A, B, C = wl.logunit(n, seed=3)
    assert np.abs(A @ B - C).max() < 1e-8
    nz = C[C != 0]
    assert nz.size == n                                            # one per row and column
    assert np.count_nonzero(C, axis=0).max() == 1 and np.count_nonzero(C, axis=1).max() == 1
    assert np.sum(np.isclose(nz, 1.0)) == int(math.log2(n))       # log2 n units
    assert np.sum(np.isclose(nz, 1e-4)) == n - int(math.log2(n))  # the construction's 0.01^2


def test_diagonal_product():
    n = 64
    A, B, PD = wl.diagonal(n, seed=4)
    assert np.abs(A @ B - PD).max() < 1e-9
    nz = np.abs(PD[PD != 0])
    assert nz.size == n and nz.min() >= 0.5 and nz.max() <= 1.0


def test_lightbulb_planted_entry_is_exact():
    # +-1 entries scaled by 1/sqrt(n); column j* of B is row i* of A with
    # round(n (1 - rho) / 2) signs flipped, so C[i*, j*] = 1 - 2 flips / n
    n, rho = 1000, 0.8
    A, B, (i, j) = wl.lightbulb(n, rho=rho, seed=6)
    assert abs((A @ B)[i, j] - (1.0 - 2.0 * round(n * (1 - rho) / 2) / n)) < 1e-12


def test_covariance_planted_correlation():
    n, rho = 2048, 0.8
    A, B, (i, j) = wl.covariance(n, rho=rho, seed=7)
    C = A @ B
    # rho ||a_i||^2 plus a noise term of order 1/sqrt(n); the background is O(1/sqrt(n))
    assert abs(C[i, j] - rho) < 0.15
    C[i, j] = 0.0
    assert np.abs(C).max() < 0.3


def test_correctness_counters_by_hand():
    # the counters of Sec. 5.3 on a 2 x 3 example counted by hand
    import torch
    from paper_2601_09477_gb300 import evaluate as ev
    C_true = torch.tensor([[1.0, 0.0, 0.001], [0.0, -0.8, 0.0]], dtype=torch.float64)
    big = C_true.abs() >= 0.5
    C_hat = torch.tensor([[0.95, 0.6, 0.0], [0.2, -0.45, 0.05]], dtype=torch.float64)
    c = ev.counters(C_hat, big, C_true)
    assert c == {"big": 2, "small": 4, "B_ge_0.5": 1, "S_le_0.5": 3,
                 "B_eps_le_0.1": 1, "S_eps_le_0.1": 2}
