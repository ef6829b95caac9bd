"""Full-size workloads on the GPU, checked on sampled outputs the oracle can
compute one by one (the bucket definition of a sketch entry, Decompress of a
row from the same R) and on properties that hold at any size."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2601_09477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cmm():
    assert torch.cuda.is_available()
    from paper_2601_09477_gb300 import cmm as mod
    return mod


def _scale_t(At, Bt):
    # sum_t ||A[:, t]|| ||B[t, :]|| on the device
    return float((torch.linalg.vector_norm(At.double(), dim=0) *
                  torch.linalg.vector_norm(Bt.double(), dim=1)).sum().item())


def test_planted_pm1_8192_exact(cmm):
    # n = 8192 +-1 rows, 64 planted pairs, B = A^T, b = 2^16, d = 9, FP64 storage:
    # FP32 and FP64 butterflies give the same R (every quantity an integer), R
    # entries equal the bucket definition, Decompress of rows equals the oracle
    # given R, and all planted off-diagonal pairs except collision victims reach n/2
    n, L, d = 8192, 16, 9
    A, B, pairs = wl.planted_pm1(n=n, pairs=64, rho=0.9, seed=1002)
    h = cmm.make_hashes(2002, d, L)
    Ad = torch.from_numpy(A).cuda()
    Bd = torch.from_numpy(B).cuda()
    R32 = torch.empty((d, 1 << L), dtype=torch.float64, device="cuda")
    C = cmm.multiply(Ad, Bd, h, prec="f32", R=R32)
    R64 = cmm.sketch(Ad, Bd, h, prec="f64")
    assert torch.equal(R32, R64)
    R = R32.cpu().numpy()
    assert np.array_equal(R, np.round(R))
    g = np.random.default_rng(7)
    for r, w in [(0, int(g.integers(1 << L))), (4, int(g.integers(1 << L))),
                 (8, int(g.integers(1 << L)))]:
        assert R[r, w] == orc.R_entry(A, B, h.params, L, r, w)
    rows = (4000, 4004)
    Co = orc.extract(R, h.params, n, n, rows=rows)
    assert np.array_equal(C[rows[0]:rows[1]].cpu().numpy(), Co)
    I, J, V = cmm.threshold(C, n / 2)
    found = set(zip(I.cpu().tolist(), J.cpu().tolist()))
    planted = {(int(i), int(j)) for i, j in pairs} | {(int(j), int(i)) for i, j in pairs}
    assert sum(q in found for q in planted) >= 0.95 * len(planted)
    # C_ii = n on the diagonal; one repetition's noise has sd about sqrt(||C||_F^2 / b)
    # ~ n/2 here, so a median below n/2 has probability ~0.4% per entry
    diag = sum(1 for (i, j) in found if i == j)
    assert diag >= 0.99 * n


@pytest.mark.parametrize("prec,tol", [("f32", 1e-5), ("bf16tc", 2e-2), ("f16tc", 2.5e-3)])
def test_precision_workload_16384(cmm, prec, tol):
    # n = 16384, A = Q (orthogonal), B = Q^T S + 1e-3 noise, S with 1024 entries
    # N(0,1)*100; b = 2^18 (slices of 2^14 / 2^15 with the frequency split), d = 7
    n, L, d = 16384, 18, 7
    A, B, S = wl.orthogonal_precision(n=n, seed=1003, device="cuda")
    h = cmm.make_hashes(2003, d, L)
    R = torch.empty((d, 1 << L), dtype=torch.float64, device="cuda")
    C = cmm.multiply(A, B, h, prec=prec, R=R)
    scale = _scale_t(A, B)
    Rn = R.cpu().numpy()
    A64 = A.double().cpu().numpy()
    B64 = B.double().cpu().numpy()
    g = np.random.default_rng(3)
    rms = float(np.sqrt(np.mean(Rn ** 2)))
    for r, w in [(0, int(g.integers(1 << L))), (6, int(g.integers(1 << L))),
                 (3, int(g.integers(1 << L)))]:
        want = orc.R_entry(A64, B64, h.params, L, r, w)
        assert abs(Rn[r, w] - want) <= tol * scale, (prec, r, w, Rn[r, w], want)
        # well inside the spread of R as well (catches a wrong transform that the
        # norm-relative tolerance alone would let through)
        assert abs(Rn[r, w] - want) <= 0.05 * rms, (prec, r, w, Rn[r, w], want, rms)
    # the 1024 planted entries (|S| up to a few hundred) are recovered within the noise
    si, sj = np.nonzero(S)
    est = C[torch.from_numpy(si).cuda(), torch.from_numpy(sj).cuda()].cpu().numpy()
    big = np.abs(S[si, sj]) > 50
    rel = np.abs(est[big] - S[si, sj][big]) / np.abs(S[si, sj][big])
    assert np.median(rel) < 0.1
