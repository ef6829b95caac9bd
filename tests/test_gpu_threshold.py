"""Heavy-hitter lists (the goal of Sec. 1: every (i, j) with |Chat[i, j]| >= tau,
in (i, j) order) from a dense estimate, and the fused multiply + threshold
entry point, whose per-row counts are taken while Decompress writes C.

The test abs(e) >= tau runs on the magnitude bits of e; it must decide every
value exactly as the FP64 comparison does, including signed zeros,
subnormals, infinities and NaN (never a heavy hitter), for any tau (NaN tau:
no heavy hitters; tau <= 0: every non-NaN entry)."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2601_09477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cmm():
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2601_09477_gb300 import cmm as mod
    return mod


def _dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def _expected(C, tau):
    with np.errstate(invalid="ignore"):
        mask = np.abs(C) >= tau
    I, J = np.nonzero(mask)          # row-major order
    return I.astype(np.int32), J.astype(np.int32), C[I, J]


def _special_matrix(m, p, seed):
    g = np.random.default_rng(seed)
    C = g.standard_normal((m, p)) * 2
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 5e-324, -5e-324,
                         2.2250738585072014e-308, 1.5, -1.5, np.nextafter(1.5, 0),
                         np.nextafter(1.5, 2), 1e308, -1e308])
    idx = g.integers(0, m * p, 400)
    C.flat[idx] = specials[g.integers(0, len(specials), len(idx))]
    return C


@pytest.mark.parametrize("tau", [1.5, 0.0, -0.0, -1.0, np.inf, np.nan, 5e-324, 1e308, 3.0])
def test_threshold_matches_fp64_comparison(cmm, tau):
    # p = 1000 spans several 256-column chunks of a row plus a ragged tail
    C = _special_matrix(37, 1000, 5)
    I, J, V = cmm.threshold(_dev(C), tau, capacity=37 * 1000)
    Ie, Je, Ve = _expected(C, tau)
    assert np.array_equal(I.cpu().numpy(), Ie)
    assert np.array_equal(J.cpu().numpy(), Je)
    assert np.array_equal(V.cpu().numpy().view(np.int64), Ve.view(np.int64))


def test_threshold_padded_rows_and_capacity(cmm):
    C = _special_matrix(64, 300, 7)
    big = np.full((64, 311), 7.0)    # padding columns would all be hits
    big[:, :300] = C
    Ct = _dev(big)[:, :300]
    Ie, Je, Ve = _expected(C, 1.0)
    I, J, V = cmm.threshold(Ct, 1.0, capacity=len(Ie))
    assert np.array_equal(I.cpu().numpy(), Ie) and np.array_equal(J.cpu().numpy(), Je)
    with pytest.raises(cmm.CmmError) as e:
        cmm.threshold(Ct, 1.0, capacity=len(Ie) - 1)
    assert e.value.code == cmm.ERR_CAPACITY


@pytest.mark.parametrize("shape,prec,d,tau", [
    ((300, 77, 517, 10), "f32", 5, 2.0),
    ((129, 300, 1000, 12), "f64", 4, 1.0),
    ((1000, 64, 64, 9), "f32", 3, 0.0),      # every entry: rows of 64 hits
    ((8, 40, 4099, 13), "f32", 7, 3.0),
])
def test_multiply_threshold_equals_separate_calls(cmm, shape, prec, d, tau):
    m, k, p, L = shape
    g = np.random.default_rng(m + k + p)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    h = cmm.make_hashes(3 + L, d, L)
    Ad, Bd = _dev(A), _dev(B)
    R1 = torch.empty((d, 1 << L), dtype=torch.float64, device="cuda")
    C1, (I1, J1, V1) = cmm.multiply_threshold(Ad, Bd, h, tau, capacity=m * p, prec=prec, R=R1)
    C2 = cmm.multiply(Ad, Bd, h, prec=prec)
    I2, J2, V2 = cmm.threshold(C2, tau, capacity=m * p)
    assert torch.equal(C1, C2)
    assert torch.equal(I1, I2) and torch.equal(J1, J2) and torch.equal(V1, V2)
    # the list is the oracle's heavy-hitter list of the same sketch
    Io, Jo, Vo = orc.heavy_hitters(R1.cpu().numpy(), h.params, m, p, tau, capacity=m * p)
    assert np.array_equal(I1.cpu().numpy(), Io) and np.array_equal(J1.cpu().numpy(), Jo)
    assert np.array_equal(V1.cpu().numpy(), Vo)


def test_multiply_threshold_planted_pairs_and_capacity(cmm):
    # planted +-1 rows (the benchmark's structure at n = 1024, b = 2^16, d = 9):
    # the diagonal (n) and the planted pairs (~0.9 n) pass tau = n / 2
    A, B, plist = wl.planted_pm1(1024, pairs=8, seed=5)
    Ad, Bd = _dev(A), _dev(B)
    h = cmm.make_hashes(11, 9, 16)
    C, (I, J, V) = cmm.multiply_threshold(Ad, Bd, h, 512.0, capacity=1 << 16)
    I2, J2, V2 = cmm.threshold(C, 512.0, capacity=1 << 16)
    assert torch.equal(I, I2) and torch.equal(J, J2) and torch.equal(V, V2)
    pairs = set(zip(I.cpu().tolist(), J.cpu().tolist()))
    assert all((i, i) in pairs for i in range(1024))
    assert all((int(i), int(j)) in pairs and (int(j), int(i)) in pairs for i, j in plist)
    n = len(I)
    with pytest.raises(cmm.CmmError) as e:
        cmm.multiply_threshold(Ad, Bd, h, 512.0, capacity=n - 1)
    assert e.value.code == cmm.ERR_CAPACITY


def test_multiply_threshold_empty(cmm):
    h = cmm.make_hashes(1, 3, 8)
    A = torch.zeros((0, 5), dtype=torch.float64, device="cuda")
    B = torch.ones((5, 9), dtype=torch.float64, device="cuda")
    C, (I, J, V) = cmm.multiply_threshold(A, B, h, 0.0, capacity=4)
    assert C.shape == (0, 9) and I.numel() == 0


@pytest.mark.parametrize("m,p,L,d,tau", [
    (700, 1500, 11, 5, 1.0),     # candidates fit: one pass over the estimates
    (512, 600, 10, 5, 0.0),      # every entry a hit: 307,200 > 65,536 candidates, second pass
    (33, 4099, 9, 4, 1.5),       # ragged tiles, even d
])
def test_heavy_hitters_from_R_one_pass(cmm, m, p, L, d, tau):
    g = np.random.default_rng(m + p)
    R = g.standard_normal((d, 1 << L)) * 2
    h = cmm.make_hashes(50 + L, d, L)
    I, J, V = cmm.heavy_hitters(_dev(R), h, m, p, tau=tau, capacity=m * p)
    Io, Jo, Vo = orc.heavy_hitters(R, h.params, m, p, tau, capacity=m * p)
    assert np.array_equal(I.cpu().numpy(), Io)
    assert np.array_equal(J.cpu().numpy(), Jo)
    assert np.array_equal(V.cpu().numpy(), Vo)
    # and the same list as Decompress + threshold
    C = cmm.extract(_dev(R), h, m, p)
    I2, J2, V2 = cmm.threshold(C, tau, capacity=m * p)
    assert torch.equal(I, I2) and torch.equal(J, J2) and torch.equal(V, V2)
