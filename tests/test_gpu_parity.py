"""Parity of the CUDA path (called through the C ABI) with the FP64 oracle.

Sketch: R_gpu vs oracle Compress on the same input values (widened to FP64),
max |R_gpu - R_orc| / sum_t ||A[:,t]|| ||B[t,:]|| within 1e-12 (FP64
butterflies) or 1e-5 (FP32 butterflies); exactly equal on +-1 inputs.
Decompress / heavy hitters / mean at pairs: given the SAME R, the GPU result
is bit-identical to the oracle's (the median is a selection, the mean uses the
same operation order), and the heavy-hitter lists are identical.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2601_09477_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def cmm():
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2601_09477_gb300 import cmm as mod
    return mod


def _norm_scale(A64, B64):
    # sum_t ||A[:, t]||_2 ||B[t, :]||_2
    return float(np.sum(np.linalg.norm(A64, axis=0) * np.linalg.norm(B64, axis=1)))


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


SHAPES = [
    # (m, k, p, log2b, d)
    (100, 37, 90, 6, 3),
    (300, 129, 257, 12, 5),
    (513, 300, 411, 13, 3),
    (700, 260, 650, 14, 3),
    (1000, 200, 900, 15, 3),     # two FP32 slices (four FP64 slices)
    (300, 40, 9000, 14, 2),      # a B row longer than one scatter batch
    (517, 97, 333, 17, 2),       # 8 / 16 slices, even d
    (64, 1000, 50, 3, 1),        # tiny transform, many inner indices
    (1, 5, 1, 1, 1),             # b = 2
    (33, 70, 2, 5, 4),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_sketch_matches_oracle(cmm, prec, shape):
    m, k, p, L, d = shape
    g = np.random.default_rng(m * 7 + k * 3 + p + L)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    h = cmm.make_hashes(1000 + L, d, L)
    R = cmm.sketch(_dev(A, torch.float64), _dev(B, torch.float64), h, prec=prec).cpu().numpy()
    Ro = orc.compress(A, B, h.params, L, nthreads=8)
    err = np.abs(R - Ro).max() / _norm_scale(A, B)
    assert err <= TOL[prec], err


def _extreme_columns(m, k, p, seed):
    """Columns that stress the FP32 fixed-point scatter (one power-of-two scale
    per column from its max |value| and the bucket occupancy): a zero column,
    one dominant entry over tiny ones, constant columns, and column scales from
    1e-20 to 1e15 with B's row scaled by the inverse so products stay O(1)."""
    g = np.random.default_rng(seed)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    A[:, 0] = 0.0
    A[:, 1] = 1e-3 * g.standard_normal(m)
    A[m // 3, 1] = 1e3
    B[2, :] = 1e-3 * g.standard_normal(p)
    B[2, 5] = -7e2
    A[:, 3] = 1.0
    B[3, :] = -0.5
    scales = 10.0 ** g.uniform(-20, 15, size=k)
    scales[:5] = 1.0
    A *= scales[None, :]
    B /= scales[:, None]
    return A, B


@pytest.mark.parametrize("L", [12, 14, 15])
def test_fixed_point_scatter_extreme_columns(cmm, L):
    m, k, p, d = 1200, 40, 900, 3
    A, B = _extreme_columns(m, k, p, 7 + L)
    A32 = A.astype(np.float32).astype(np.float64)
    B32 = B.astype(np.float32).astype(np.float64)
    h = cmm.make_hashes(77 + L, d, L)
    R = cmm.sketch(_dev(A32, torch.float32), _dev(B32, torch.float32), h, prec="f32").cpu().numpy()
    Ro = orc.compress(A32, B32, h.params, L, nthreads=8)
    err = np.abs(R - Ro).max() / _norm_scale(A32, B32)
    assert err <= TOL["f32"], err


@pytest.mark.parametrize("L", [12, 16])
def test_fp32_sketch_is_deterministic(cmm, L):
    # integer bucket sums and fixed reduction orders: bitwise identical reruns
    g = np.random.default_rng(L)
    A = _dev(g.standard_normal((800, 300)), torch.float32)
    B = _dev(g.standard_normal((300, 700)), torch.float32)
    h = cmm.make_hashes(5, 3, L)
    R1 = cmm.sketch(A, B, h, prec="f32")
    R2 = cmm.sketch(A, B, h, prec="f32")
    assert torch.equal(R1, R2)


# tensor-core precisions: (max |R - R_orc| / sum_t ||A_t|| ||B_t||, max |R - R_orc| / max |R_orc|).
# BF16 keeps 8 significand bits, FP16 11: the FP16 bounds are the BF16 ones
# divided by 8 (the ratio of their unit roundoffs), the second rounded up to 1e-2.
TC_TOL = {"bf16tc": (2e-2, 0.05), "f16tc": (2.5e-3, 0.01)}


def _tc_error(cmm, A, B, h, L, prec):
    R = cmm.sketch(_dev(A, torch.float32), _dev(B, torch.float32), h, prec=prec).cpu().numpy()
    A32 = A.astype(np.float32).astype(np.float64)
    B32 = B.astype(np.float32).astype(np.float64)
    Ro = orc.compress(A32, B32, h.params, L, nthreads=8)
    dR = np.abs(R - Ro).max()
    return dR / _norm_scale(A32, B32), dR / np.abs(Ro).max()


@pytest.mark.parametrize("prec", ["bf16tc", "f16tc"])
@pytest.mark.parametrize("shape", [(1000, 200, 900, 15, 3), (517, 97, 333, 17, 2),
                                   (2048, 300, 1500, 16, 5), (64, 33, 70, 15, 1)])
def test_sketch_tensor_core(cmm, shape, prec):
    # 16-bit operands with exact +-1 Hadamard blocks, FP32 accumulation: the
    # error against the oracle on the same (FP32-rounded) inputs within TC_TOL,
    # and far below the signal
    m, k, p, L, d = shape
    g = np.random.default_rng(m + k + p)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    h = cmm.make_hashes(300 + L, d, L)
    err_norm, err_max = _tc_error(cmm, A, B, h, L, prec)
    assert err_norm <= TC_TOL[prec][0], err_norm
    assert err_max <= TC_TOL[prec][1], err_max


def test_sketch_f16_more_precise_than_bf16(cmm):
    # same input, same hashes: FP16 operands (3 more significand bits) give a
    # smaller error than BF16 ones
    m, k, p, L, d = 1500, 256, 1300, 16, 3
    g = np.random.default_rng(41)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    h = cmm.make_hashes(41, d, L)
    e16 = _tc_error(cmm, A, B, h, L, "f16tc")[1]
    ebf = _tc_error(cmm, A, B, h, L, "bf16tc")[1]
    assert e16 < 0.5 * ebf, (e16, ebf)


@pytest.mark.parametrize("prec", ["bf16tc", "f16tc"])
@pytest.mark.parametrize("L", [15, 16])
def test_tensor_core_extreme_columns(cmm, prec, L):
    # the fixed-point scale per column keeps the 16-bit operands in range for
    # column scales from 1e-20 to 1e15 (FP16: values scaled to below 2^15)
    m, k, p, d = 1200, 40, 900, 3
    A, B = _extreme_columns(m, k, p, 11 + L)
    h = cmm.make_hashes(88 + L, d, L)
    err_norm, _ = _tc_error(cmm, A, B, h, L, prec)
    assert err_norm <= TC_TOL[prec][0], err_norm


@pytest.mark.parametrize("prec", ["bf16tc", "f16tc"])
def test_sketch_tensor_core_needs_large_slices(cmm, prec):
    h = cmm.make_hashes(1, 3, 12)
    A = torch.zeros((20, 10), dtype=torch.float32, device="cuda")
    B = torch.zeros((10, 30), dtype=torch.float32, device="cuda")
    with pytest.raises(cmm.CmmError) as ei:
        cmm.sketch(A, B, h, prec=prec)
    assert ei.value.code == cmm.ERR_RANGE


_REGS_SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2601_09477_gb300 import cmm
m, k, p, L, d = (int(x) for x in sys.argv[2:7])
g = np.random.default_rng(m + k)
A = g.standard_normal((m, k)); B = g.standard_normal((k, p))
h = cmm.make_hashes(77 + L, d, L)
R = cmm.sketch(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), h, prec="f32")
np.savez(sys.argv[7], A=A, B=B, R=R.cpu().numpy(), hp=h.params)
"""


@pytest.mark.parametrize("kernel", ["regs"])
@pytest.mark.parametrize("shape", [(700, 260, 650, 14, 3), (300, 70, 500, 16, 2),
                                   (1024, 100, 2048, 16, 3)])
def test_alternative_sketch_kernels(cmm, shape, kernel, tmp_path):
    # the FP32 2^14-slice sketch has a TMEM kernel (default) and a register-only
    # kernel (CMM_SKETCH_KERNEL=regs); the second runs in a fresh process
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "alt.npz")
    env = dict(os.environ, CMM_SKETCH_KERNEL=kernel)
    subprocess.run([sys.executable, "-c", _REGS_SCRIPT, root] + [str(x) for x in shape] + [out],
                   check=True, env=env)
    z = np.load(out)
    m, k, p, L, d = shape
    Ro = orc.compress(z["A"], z["B"], z["hp"], L, nthreads=8)
    assert np.abs(z["R"] - Ro).max() / _norm_scale(z["A"], z["B"]) <= TOL["f32"]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.bfloat16])
@pytest.mark.parametrize("transA", [False, True])
def test_sketch_dtypes_and_layouts(cmm, prec, dtype, transA):
    m, k, p, L, d = 300, 150, 280, 11, 3
    g = np.random.default_rng(5)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    At = _dev(A.T if transA else A, dtype)
    Bt = _dev(B, dtype)
    # the oracle sees the same (rounded) values, widened to FP64
    A_in = At.double().cpu().numpy()
    B_in = Bt.double().cpu().numpy()
    h = cmm.make_hashes(77, d, L)
    R = cmm.sketch(At, Bt, h, prec=prec, transA=transA).cpu().numpy()
    Ro = orc.compress(A_in, B_in, h.params, L, transA=transA, nthreads=8)
    scale = _norm_scale(A_in.T if transA else A_in, B_in)
    assert np.abs(R - Ro).max() / scale <= TOL[prec]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sketch_pm1_exact(cmm, prec):
    A, B, _ = wl.planted_pm1(n=512, pairs=8, seed=3)
    h = cmm.make_hashes(5, 5, 13)
    R = cmm.sketch(_dev(A, torch.float64), _dev(B, torch.float64), h, prec=prec).cpu().numpy()
    Ro = orc.compress(A, B, h.params, 13, nthreads=8)
    assert np.array_equal(R, Ro)


def test_sketch_empty_inner_dimension(cmm):
    h = cmm.make_hashes(1, 3, 8)
    A = torch.zeros((20, 0), dtype=torch.float64, device="cuda")
    B = torch.zeros((0, 30), dtype=torch.float64, device="cuda")
    R = cmm.sketch(A, B, h, prec="f32")
    assert torch.count_nonzero(R).item() == 0


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 7, 9, 11, 16, 17, 25, 33, 35])
@pytest.mark.parametrize("reduce", ["median", "mean"])
def test_extract_bitwise_given_R(cmm, d, reduce):
    m, p, L = 67, 301, 9
    g = np.random.default_rng(d)
    R = g.standard_normal((d, 1 << L)) * 10
    R[0, :7] = 0.0   # exercise signed zeros
    h = cmm.make_hashes(40 + d, d, L)
    C = cmm.extract(_dev(R, torch.float64), h, m, p, reduce=reduce).cpu().numpy()
    Co = orc.extract(R, h.params, m, p, orc.MEDIAN if reduce == "median" else orc.MEAN)
    assert np.array_equal(C, Co)


@pytest.mark.parametrize("d", [3, 4, 9, 21])
def test_heavy_hitters_given_R(cmm, d):
    m, p, L = 150, 230, 8
    g = np.random.default_rng(100 + d)
    R = g.standard_normal((d, 1 << L)) * 3
    h = cmm.make_hashes(7 + d, d, L)
    Rt = _dev(R, torch.float64)
    I, J, V = cmm.heavy_hitters(Rt, h, m, p, tau=2.0)
    Io, Jo, Vo = orc.heavy_hitters(R, h.params, m, p, 2.0)
    assert np.array_equal(I.cpu().numpy(), Io)
    assert np.array_equal(J.cpu().numpy(), Jo)
    assert np.array_equal(V.cpu().numpy(), Vo)
    # from the dense estimate
    C = cmm.extract(Rt, h, m, p)
    I2, J2, V2 = cmm.threshold(C, 2.0)
    assert np.array_equal(I2.cpu().numpy(), Io) and np.array_equal(V2.cpu().numpy(), Vo)


def test_heavy_hitters_capacity(cmm):
    m, p, L, d = 40, 50, 6, 3
    R = np.random.default_rng(1).standard_normal((d, 1 << L)) * 3
    h = cmm.make_hashes(3, d, L)
    Rt = _dev(R, torch.float64)
    Io, Jo, Vo = orc.heavy_hitters(R, h.params, m, p, 1.0)
    assert len(Io) > 10
    with pytest.raises(cmm.CmmError) as ei:
        cmm.heavy_hitters(Rt, h, m, p, tau=1.0, capacity=10)
    assert ei.value.code == cmm.ERR_CAPACITY
    I, J, V = cmm.heavy_hitters(Rt, h, m, p, tau=1.0, capacity=len(Io))
    assert np.array_equal(I.cpu().numpy(), Io)
    I, J, V = cmm.heavy_hitters(Rt, h, m, p, tau=1e9)
    assert I.numel() == 0


def test_mean_pairs_bitwise(cmm):
    d, L = 5, 10
    g = np.random.default_rng(9)
    R = g.standard_normal((d, 1 << L))
    h = cmm.make_hashes(11, d, L)
    I = g.integers(0, 5000, 999).astype(np.int32)
    J = g.integers(0, 7000, 999).astype(np.int32)
    out = cmm.mean_pairs(_dev(R, torch.float64), h, torch.from_numpy(I), torch.from_numpy(J))
    assert np.array_equal(out.cpu().numpy(), orc.mean_at_pairs(R, h.params, I, J))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_multiply_orthogonal_sparse_256(cmm, prec):
    # n = 256, b = 2^12, d = 5, heavy-hitter threshold 5 (A B = S exactly)
    A, B, S = wl.orthogonal_sparse(seed=1001)
    h = cmm.make_hashes(2001, 5, 12)
    R = torch.empty((5, 4096), dtype=torch.float64, device="cuda")
    C = cmm.multiply(_dev(A, torch.float64), _dev(B, torch.float64), h, prec=prec, R=R)
    Rg = R.cpu().numpy()
    Ro = orc.compress(A, B, h.params, 12, nthreads=8)
    dR = np.abs(Rg - Ro).max()
    assert dR / _norm_scale(A, B) <= TOL[prec]
    Co = orc.extract(Ro, h.params, 256, 256)
    # the median is 1-Lipschitz in the sup norm of R
    assert np.abs(C.cpu().numpy() - Co).max() <= dR
    # heavy hitters: identical outside a band of |C| around tau
    I, J, V = cmm.threshold(C, 5.0)
    got = set(zip(I.cpu().tolist(), J.cpu().tolist()))
    Io, Jo, _ = orc.heavy_hitters(Ro, h.params, 256, 256, 5.0)
    want = set(zip(Io.tolist(), Jo.tolist()))
    band = {(i, j) for i in range(256) for j in range(256) if abs(abs(Co[i, j]) - 5.0) <= max(1e-9 * 5, 2 * dR)}
    assert got - band == want - band
    # and the planted entries are recovered
    si, sj = np.nonzero(np.abs(S) >= 5.0)
    assert set(zip(si.tolist(), sj.tolist())) <= got
