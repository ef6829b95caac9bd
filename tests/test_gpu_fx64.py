"""The exact 64-bit fixed-point form (CMM_PREC_FX64) against the FP64 oracle:
R within the FP64 tolerance, 1e-12 of sum_t ||A[:, t]|| ||B[t, :]||, over
shapes that span one to many frequency slices, ragged tails, odd and even d,
every storage type and layout, extreme column scales, and the n = 256
recovery workload; Decompress of the same R equals the oracle's."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2601_09477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def cmm():
    assert torch.cuda.is_available()
    from paper_2601_09477_gb300 import cmm as mod
    return mod


def _scale(A, B):
    return float(np.sum(np.linalg.norm(A, axis=0) * np.linalg.norm(B, axis=1)))


def _dev(x, dtype, transA=False):
    x = x.T.copy() if transA else x
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


SHAPES = [
    # m, k, p, log2b, d
    (37, 19, 23, 1, 3),
    (64, 33, 50, 3, 5),
    (100, 70, 90, 4, 2),
    (256, 256, 256, 5, 5),
    (300, 517, 200, 8, 4),
    (513, 260, 700, 12, 5),
    (1000, 300, 1500, 13, 3),
    (2048, 600, 1024, 14, 5),
    (777, 1100, 901, 15, 6),
    (1500, 257, 1300, 17, 3),
]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype,transA", [(torch.float64, False), (torch.float64, True),
                                          (torch.float32, False), (torch.bfloat16, True)])
def test_fx64_matches_oracle(cmm, shape, dtype, transA):
    m, k, p, L, d = shape
    g = np.random.default_rng(m * 7 + k)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    Ad, Bd = _dev(A, dtype, transA), _dev(B, dtype)
    # the oracle runs on the values the library sees (rounded to the storage type)
    A64 = (Ad.t() if transA else Ad).double().cpu().numpy()
    B64 = Bd.double().cpu().numpy()
    h = cmm.make_hashes(4000 + L, d, L)
    R = cmm.sketch(Ad, Bd, h, prec="fx64", transA=transA).cpu().numpy()
    Ro = orc.compress(A64, B64, h.params, L, nthreads=orc.max_threads())
    err = np.abs(R - Ro).max() / _scale(A64, B64)
    assert err <= TOL, err


def test_fx64_extreme_column_scales(cmm):
    # columns spanning 1e-20 .. 1e15, a zero column, a column with one
    # dominant entry over tiny ones, a constant column
    m, k, p, L, d = 700, 64, 500, 14, 5
    g = np.random.default_rng(5)
    A = g.standard_normal((m, k)) * (10.0 ** g.uniform(-20, 15, size=k))[None, :]
    B = g.standard_normal((k, p)) * (10.0 ** g.uniform(-20, 15, size=k))[:, None]
    A[:, 3] = 0.0
    B[7, :] = 0.0
    A[:, 5] = 1e-12
    A[11, 5] = 1e6
    B[9, :] = 3.25
    h = cmm.make_hashes(77, d, L)
    R = cmm.sketch(_dev(A, torch.float64), _dev(B, torch.float64), h, prec="fx64").cpu().numpy()
    Ro = orc.compress(A, B, h.params, L, nthreads=orc.max_threads())
    err = np.abs(R - Ro).max() / _scale(A, B)
    assert err <= TOL, err


def _norm(x):
    # 2-norm without overflow or underflow of the squares
    s = np.abs(x).max()
    return 0.0 if s == 0 else float(s * np.linalg.norm(x / s))


def test_fx64_norms_at_powers_of_two_and_tiny_or_huge_columns(cmm):
    # the per-column scale comes from an integer upper bound of the column's l1
    # norm; each special column is checked alone (k = 1, so the tolerance is
    # relative to that column's own norm product): a norm exactly a power of
    # two, just below one (by 2^-40 and by one unit in the last place), just
    # above one, entries near the bottom of the normal range (norm below
    # 2^-962, where the scale 2^e leaves the FP64 range), one normal entry
    # among subnormal ones, and entries near the top of the range
    m, p, L, d = 640, 300, 14, 3
    g = np.random.default_rng(11)
    cols = {}
    c = np.zeros(m)
    c[:8] = 2.0 ** -3
    cols["pow2"] = c                              # l1 = 1
    c = np.full(m, 1.0 / 512.0)
    c[0] -= 2.0 ** -40
    cols["below_2^-40"] = c                       # l1 = 1.25 - 2^-40
    c = np.zeros(m)
    c[:2] = [0.5, np.nextafter(0.5, 0.0)]
    cols["below_ulp"] = c                         # l1 one ulp below 1
    c = np.zeros(m)
    c[:2] = [0.5, np.nextafter(0.5, 1.0)]
    cols["above_ulp"] = c                         # l1 one ulp above 1
    cols["tiny"] = 1e-300 * g.standard_normal(m)
    c = 1e-310 * g.integers(-3, 4, m).astype(np.float64)
    c[17] = 1e-300
    cols["normal_among_subnormal"] = c
    cols["huge"] = 1e300 * g.standard_normal(m) / m
    B = g.standard_normal((1, p))
    h = cmm.make_hashes(2024, d, L)
    for name, a in cols.items():
        A = a.reshape(m, 1).copy()
        R = cmm.sketch(_dev(A, torch.float64), _dev(B, torch.float64), h, prec="fx64").cpu().numpy()
        Ro = orc.compress(A, B, h.params, L)
        assert np.isfinite(R).all(), name
        err = np.abs(R - Ro).max() / (_norm(a) * _norm(B[0]))
        assert err <= TOL, (name, err)


def test_fx64_deterministic_and_exact_on_small_integers(cmm):
    # bitwise-identical reruns; +-1 inputs within the tolerance (the
    # multiply-accumulate is float-float, so integer R is not guaranteed bit
    # for bit)
    n, L, d = 512, 12, 5
    A, B, _ = wl.planted_pm1(n=n, pairs=8, rho=0.9, seed=3)
    h = cmm.make_hashes(99, d, L)
    Ad, Bd = _dev(A, torch.float64), _dev(B, torch.float64)
    R1 = cmm.sketch(Ad, Bd, h, prec="fx64")
    R2 = cmm.sketch(Ad, Bd, h, prec="fx64")
    assert torch.equal(R1, R2)
    Ro = orc.compress(A, B, h.params, L)
    assert np.abs(R1.cpu().numpy() - Ro).max() <= TOL * _scale(A, B)
    assert np.abs(R1.cpu().numpy() - Ro).max() < 1e-6   # integers to well below 1/2


def test_fx64_orthogonal_sparse_256(cmm):
    # A = Q orthogonal, B = Q^T S, S with 64 entries N(0,1)*10; b = 2^12, d = 5:
    # R at the FP64 tolerance and Decompress of the same R equal to the oracle's
    A, B, S = wl.orthogonal_sparse(n=256, nnz=64, scale=10.0, seed=1001)
    h = cmm.make_hashes(2001, 5, 12)
    R = torch.empty((5, 4096), dtype=torch.float64, device="cuda")
    C = cmm.multiply(_dev(A, torch.float64), _dev(B, torch.float64), h, prec="fx64", R=R)
    Rn = R.cpu().numpy()
    Ro = orc.compress(A, B, h.params, 12)
    assert np.abs(Rn - Ro).max() <= TOL * _scale(A, B)
    assert np.array_equal(C.cpu().numpy(), orc.extract(Rn, h.params, 256, 256))
    # the estimate moves by at most the largest change of R (the median is
    # 1-Lipschitz in the sup norm): against the plain FP64 form
    R64 = torch.empty_like(R)
    C64 = cmm.multiply(_dev(A, torch.float64), _dev(B, torch.float64), h, prec="f64", R=R64)
    dR = float((R - R64).abs().max().item())
    assert dR <= 2 * TOL * _scale(A, B)
    assert float((C - C64).abs().max().item()) <= dR


def test_fx64_empty_and_degenerate(cmm):
    h = cmm.make_hashes(5, 3, 6)
    for (m, k, p) in [(0, 5, 7), (5, 0, 7), (5, 7, 0), (1, 1, 1)]:
        A = torch.ones((m, k), dtype=torch.float64, device="cuda")
        B = torch.ones((k, p), dtype=torch.float64, device="cuda")
        R = cmm.sketch(A, B, h, prec="fx64").cpu().numpy()
        Ro = orc.compress(A.cpu().numpy(), B.cpu().numpy(), h.params, 6)
        assert np.abs(R - Ro).max() <= 1e-12 * max(1.0, m * k * p)
