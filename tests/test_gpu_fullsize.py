"""Full-size workloads on the GPU, compared with the FP64 oracle element by
element (the whole sketch R, the whole heavy-hitter list, rows of the
estimate in every row block of the host-buffer path), plus sampled entries
from the bucket definition and properties that hold at any size."""
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


# ---------------------------------------------------------------- n = 8192
N8, L8, D8 = 8192, 16, 9
CAP8 = 1 << 22


@pytest.fixture(scope="module")
def planted(cmm):
    """The benchmark step: n = 8192 +-1 rows, 64 planted pairs, B = A^T, FP64
    storage, b = 2^16, d = 9, tau = n/2, run as the benchmark runs it (one
    cmm_multiply_threshold call with FP32 butterflies), and the oracle's R."""
    A, B, pairs = wl.planted_pm1(n=N8, pairs=64, rho=0.9, seed=1002)
    h = cmm.make_hashes(2002, D8, L8)
    Ad = torch.from_numpy(A).cuda()
    Bd = torch.from_numpy(B).cuda()
    R = torch.empty((D8, 1 << L8), dtype=torch.float64, device="cuda")
    C, (I, J, V) = cmm.multiply_threshold(Ad, Bd, h, N8 / 2, capacity=CAP8, prec="f32", R=R)
    torch.cuda.synchronize()
    Ro = orc.compress(A, B, h.params, L8, nthreads=orc.max_threads())
    return dict(A=A, B=B, pairs=pairs, h=h, Ad=Ad, Bd=Bd, R=R, C=C, I=I.cpu().numpy(),
                J=J.cpu().numpy(), V=V.cpu().numpy(), Ro=Ro)


def test_planted_8192_whole_R_bitexact(cmm, planted):
    # +-1 inputs: every quantity is an integer, so the whole R (9 x 2^16, all
    # four frequency slices, every block of the inner index) equals the
    # oracle's bit for bit, for FP32 and FP64 butterflies alike
    R = planted["R"].cpu().numpy()
    Ro = planted["Ro"]
    assert np.array_equal(R, Ro)
    assert np.array_equal(R, np.round(R)) and np.abs(R).max() < 2.0 ** 53
    R64 = cmm.sketch(planted["Ad"], planted["Bd"], planted["h"], prec="f64")
    assert np.array_equal(R64.cpu().numpy(), Ro)
    # three entries straight from the bucket definition as well
    g = np.random.default_rng(7)
    for r in (0, 4, 8):
        w = int(g.integers(1 << L8))
        assert R[r, w] == orc.R_entry(planted["A"], planted["B"], planted["h"].params, L8, r, w)


def test_planted_8192_whole_heavy_hitter_list(cmm, planted):
    # the complete list of |Chat| >= n/2 of the step (319k entries) against
    # the oracle's list from the same R: I, J, V and the count, bit for bit
    Io, Jo, Vo = orc.heavy_hitters(planted["Ro"], planted["h"].params, N8, N8, N8 / 2,
                                   capacity=1 << 21, nthreads=orc.max_threads())
    assert len(Io) == len(planted["I"])
    assert np.array_equal(planted["I"], Io)
    assert np.array_equal(planted["J"], Jo)
    assert np.array_equal(planted["V"], Vo)
    # and the list straight from R (cmm_heavy_hitters, no write of Chat)
    I2, J2, V2 = cmm.heavy_hitters(planted["R"], planted["h"], N8, N8, N8 / 2, capacity=CAP8)
    assert np.array_equal(I2.cpu().numpy(), Io) and np.array_equal(J2.cpu().numpy(), Jo)
    assert np.array_equal(V2.cpu().numpy(), Vo)


def _rows_every_block(n, blocks=8, per=32, seed=11):
    # `per` consecutive rows at a random offset inside each of `blocks` equal
    # row blocks, plus the first and last row of every block
    g = np.random.default_rng(seed)
    size = n // blocks
    ranges = []
    for q in range(blocks):
        off = int(g.integers(1, size - per - 1))
        ranges += [(q * size, q * size + 1), (q * size + off, q * size + off + per),
                   ((q + 1) * size - 1, (q + 1) * size)]
    return ranges


def test_planted_8192_rows_in_every_block(cmm, planted):
    # 8 x (32 + 2) rows of the 512 MiB estimate, spread over every 64 MiB row
    # block, against the oracle's Decompress from the same R
    C = planted["C"]
    for (i0, i1) in _rows_every_block(N8):
        Co = orc.extract(planted["Ro"], planted["h"].params, N8, N8, rows=(i0, i1), nthreads=8)
        assert np.array_equal(C[i0:i1].cpu().numpy(), Co), (i0, i1)


def test_planted_8192_host_path(cmm, planted):
    # cmm_multiply_host (pinned host buffers, the operands copied in parts
    # along the inner index, the estimate copied back in 64 MiB row blocks):
    # rows in every block and the whole heavy-hitter list against the oracle
    Ah = torch.from_numpy(planted["A"]).pin_memory()
    Bh = torch.from_numpy(planted["B"]).pin_memory()
    Ch = torch.empty((N8, N8), dtype=torch.float64).pin_memory()
    Ch.fill_(float("nan"))
    _, (Ih, Jh, Vh) = cmm.multiply_host(Ah, Bh, planted["h"], prec="f32", out=Ch, tau=N8 / 2,
                                        capacity=CAP8)
    Cn = Ch.numpy()
    for (i0, i1) in _rows_every_block(N8, seed=12):
        Co = orc.extract(planted["Ro"], planted["h"].params, N8, N8, rows=(i0, i1), nthreads=8)
        assert np.array_equal(Cn[i0:i1], Co), (i0, i1)
    assert not np.isnan(Cn).any()
    assert np.array_equal(Ih.numpy(), planted["I"]) and np.array_equal(Jh.numpy(), planted["J"])
    assert np.array_equal(Vh.numpy(), planted["V"])


def test_planted_8192_recovery(cmm, planted):
    # all planted off-diagonal pairs except collision victims reach n/2, and the
    # diagonal C_ii = n is recovered: one repetition's noise has sd about
    # sqrt(||C||_F^2 / b) ~ n/2 here, so a median below n/2 has probability
    # ~0.4% per entry
    found = set(zip(planted["I"].tolist(), planted["J"].tolist()))
    pairs = planted["pairs"]
    want = {(int(i), int(j)) for i, j in pairs} | {(int(j), int(i)) for i, j in pairs}
    assert sum(q in found for q in want) >= 0.95 * len(want)
    diag = sum(1 for (i, j) in found if i == j)
    assert diag >= 0.99 * N8


# ---------------------------------------------------------------- n = 16384
N16, L16, D16 = 16384, 18, 7


@pytest.fixture(scope="module")
def precision(cmm):
    """n = 16384, A = Q (orthogonal), B = Q^T S + 1e-3 noise, S with 1024
    entries N(0,1)*100, stored FP32; b = 2^18 (16 frequency slices of 2^14, 8
    of 2^15 for the 16-bit forms), d = 7; the oracle's R on the same FP32
    values widened to FP64 (one call, ~40 s on 16 host cores)."""
    A, B, S = wl.orthogonal_precision(n=N16, seed=1003, device="cuda")
    h = cmm.make_hashes(2003, D16, L16)
    A64 = A.double().cpu().numpy()
    B64 = B.double().cpu().numpy()
    Ro = orc.compress(A64, B64, h.params, L16, nthreads=orc.max_threads())
    return dict(A=A, B=B, S=S, h=h, A64=A64, B64=B64, Ro=Ro, scale=_scale_t(A, B))


@pytest.mark.parametrize("prec,tol,tol_max", [("f32", 1e-5, 1e-4), ("bf16tc", 2e-2, 5e-2),
                                              ("f16tc", 2.5e-3, 1e-2)])
def test_precision_16384_whole_R(cmm, precision, prec, tol, tol_max):
    A, B, h = precision["A"], precision["B"], precision["h"]
    R = torch.empty((D16, 1 << L16), dtype=torch.float64, device="cuda")
    C = cmm.multiply(A, B, h, prec=prec, R=R)
    Rn = R.cpu().numpy()
    Ro = precision["Ro"]
    err = np.abs(Rn - Ro)
    # the whole R, relative to sum_t ||A_t|| ||B_t||, and relative to max |R|
    # (catches a wrong transform that the norm-relative bound alone would pass)
    assert err.max() <= tol * precision["scale"], (prec, err.max() / precision["scale"])
    assert err.max() <= tol_max * np.abs(Ro).max(), (prec, err.max() / np.abs(Ro).max())
    # Decompress of rows from the same R equals the oracle's bit for bit
    for (i0, i1) in [(0, 4), (8190, 8194), (16380, 16384)]:
        Co = orc.extract(Rn, h.params, N16, N16, rows=(i0, i1), nthreads=8)
        assert np.array_equal(C[i0:i1].cpu().numpy(), Co), (prec, i0)
    # the planted entries (|S| up to a few hundred) are recovered within the noise
    S = precision["S"]
    si, sj = np.nonzero(S)
    est = C[torch.from_numpy(si).cuda(), torch.from_numpy(sj).cuda()].cpu().numpy()
    big = np.abs(S[si, sj]) > 50
    rel = np.abs(est[big] - S[si, sj][big]) / np.abs(S[si, sj][big])
    assert np.median(rel) < 0.1


def test_precision_16384_sampled_entries(cmm, precision):
    # three entries of the oracle's R straight from the bucket definition
    # (pins the oracle's Compress at this size, independently of its loops)
    g = np.random.default_rng(3)
    for r in (0, 3, 6):
        w = int(g.integers(1 << L16))
        want = orc.R_entry(precision["A64"], precision["B64"], precision["h"].params, L16, r, w)
        assert abs(precision["Ro"][r, w] - want) <= 1e-12 * precision["scale"]


def test_planted_8192_fx64_whole_R_and_list(cmm, planted):
    # the exact fixed-point form at the benchmark configuration: the whole R
    # within the FP64 tolerance of the oracle's, and its heavy-hitter list
    # equal to the oracle's outside a band of 1e-9 tau around the threshold
    A, B, h, Ro = planted["A"], planted["B"], planted["h"], planted["Ro"]
    R = torch.empty((D8, 1 << L8), dtype=torch.float64, device="cuda")
    C, (I, J, V) = cmm.multiply_threshold(planted["Ad"], planted["Bd"], h, N8 / 2, capacity=CAP8,
                                          prec="fx64", R=R)
    scale = float(np.sum(np.linalg.norm(A, axis=0) * np.linalg.norm(B, axis=1)))
    assert np.abs(R.cpu().numpy() - Ro).max() <= 1e-12 * scale
    got = set(zip(I.cpu().tolist(), J.cpu().tolist()))
    want = set(zip(planted["I"].tolist(), planted["J"].tolist()))   # the oracle's list
    tau = N8 / 2
    for (i, j) in got ^ want:
        e = orc.decompress(Ro, h.params, i, j)
        assert abs(abs(e) - tau) <= 1e-9 * tau, (i, j, e)


def test_precision_16384_fx64_whole_R(cmm, precision):
    # the precision workload's FP64 copy (the FP32 values widened) through the
    # exact fixed-point form: the whole R within 1e-12 of sum_t ||A_t|| ||B_t||
    A = torch.from_numpy(precision["A64"]).cuda()
    B = torch.from_numpy(precision["B64"]).cuda()
    R = cmm.sketch(A, B, precision["h"], prec="fx64")
    err = np.abs(R.cpu().numpy() - precision["Ro"]).max() / precision["scale"]
    assert err <= 1e-12, err
    del A, B, R
    torch.cuda.empty_cache()


def test_planted_8192_ternary_whole_R_and_list(cmm, planted):
    # the ternary (packed 16-bit integer) form at the benchmark configuration:
    # the whole R and the whole heavy-hitter list equal the oracle's bit for bit
    R = torch.empty((D8, 1 << L8), dtype=torch.float64, device="cuda")
    C, (I, J, V) = cmm.multiply_threshold(planted["Ad"], planted["Bd"], planted["h"], N8 / 2,
                                          capacity=CAP8, prec="ternary", R=R)
    assert np.array_equal(R.cpu().numpy(), planted["Ro"])
    assert np.array_equal(I.cpu().numpy(), planted["I"])
    assert np.array_equal(J.cpu().numpy(), planted["J"])
    assert np.array_equal(V.cpu().numpy(), planted["V"])


# ---------------------------------------------------------------- m = p = 2^16
def test_max_size_65536_squared(cmm):
    # 2^32 estimates (every linear index i p + j beyond 2^31 from row 32768 on,
    # a 32 GiB estimate): the whole R of the exact fixed-point form against the
    # oracle's (FP64 tolerance), rows of C at the start, the middle and the end
    # bit for bit against the oracle's Decompress of the same R, and the whole
    # heavy-hitter list straight from R against the oracle's list bit for bit.
    # A short inner dimension keeps the operands small; four planted products
    # (two beyond the 2^31-th entry) stand out of the sketch noise.
    n, k, L, d = 65536, 48, 14, 3
    g = np.random.default_rng(65536)
    A = g.standard_normal((n, k))
    B = g.standard_normal((k, n))
    spikes = [(5, 7, 0), (40000, 65535, 1), (65535, 40001, 2), (31000, 33000, 3)]
    for (i, j, t) in spikes:
        A[i, t] = 316.0
        B[t, j] = 316.0
    h = cmm.make_hashes(65536, d, L)
    Ad = torch.from_numpy(A).cuda()
    Bd = torch.from_numpy(B).cuda()
    R = torch.empty((d, 1 << L), dtype=torch.float64, device="cuda")
    C = cmm.multiply(Ad, Bd, h, prec="fx64", R=R)
    Rn = R.cpu().numpy()
    Ro = orc.compress(A, B, h.params, L, nthreads=orc.max_threads())
    scale = float(np.sum(np.linalg.norm(A, axis=0) * np.linalg.norm(B, axis=1)))
    assert np.abs(Rn - Ro).max() <= 1e-12 * scale
    for i0 in (0, 32767, 32768, 65534):
        rows = C[i0:i0 + 2].cpu().numpy()
        assert np.array_equal(rows, orc.extract(Rn, h.params, n, n, rows=(i0, i0 + 2)))
    del C
    torch.cuda.empty_cache()
    tau = 2.5e4
    I, J, V = cmm.heavy_hitters(R, h, n, n, tau, capacity=1 << 16)
    Io, Jo, Vo = orc.heavy_hitters(Rn, h.params, n, n, tau, capacity=1 << 16,
                                   nthreads=orc.max_threads())
    assert len(Io) >= len(spikes)
    assert np.array_equal(I.cpu().numpy(), Io)
    assert np.array_equal(J.cpu().numpy(), Jo)
    assert np.array_equal(V.cpu().numpy(), Vo)
    assert {(i, j) for (i, j, _) in spikes} <= set(zip(Io.tolist(), Jo.tolist()))
