"""Pagh's original cyclic form (Sec. 3.1) on the GPU, against the FP64 oracle.

Sketch: R from the FFT kernel vs the oracle's cyclic Compress on the same input
values, max |R_gpu - R_orc| / sum_t ||A[:,t]|| ||B[t,:]|| within 1e-5 (FP32
butterflies), over shapes covering 1, 2, 4, 8 and 16 frequency classes and
ragged sizes.  Extraction: bit-identical to the oracle given the same R.
"""
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


def _norm_scale(A, B):
    return float(np.sum(np.linalg.norm(A, axis=0) * np.linalg.norm(B, axis=1)))


SHAPES = [
    # (m, k, p, log2b, d): classes C = 2^(log2b - 13)
    (300, 50, 280, 13, 3),
    (64, 33, 70, 14, 1),
    (1000, 120, 900, 15, 3),
    (517, 97, 333, 16, 2),
    (700, 40, 650, 17, 3),
    (1, 5, 1, 13, 1),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_cyclic_sketch_matches_oracle(cmm, shape):
    m, k, p, L, d = shape
    g = np.random.default_rng(m + 3 * k + p + L)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    h = cmm.make_hashes(900 + L, d, L)
    R = cmm.sketch_cyclic(_dev(A), _dev(B), h).cpu().numpy()
    A32 = A.astype(np.float32).astype(np.float64)
    B32 = B.astype(np.float32).astype(np.float64)
    Ro = orc.compress_cyclic(A32, B32, h.params, L)
    err = np.abs(R - Ro).max() / _norm_scale(A32, B32)
    assert err <= 1e-5, err


def test_cyclic_sketch_transposed_fp32_operands(cmm):
    m, k, p, L, d = 400, 64, 300, 15, 3
    g = np.random.default_rng(9)
    A = g.standard_normal((m, k)).astype(np.float32)
    B = g.standard_normal((k, p)).astype(np.float32)
    h = cmm.make_hashes(5, d, L)
    R = cmm.sketch_cyclic(_dev(A.T, torch.float32), _dev(B, torch.float32), h,
                          transA=True).cpu().numpy()
    Ro = orc.compress_cyclic(A.astype(np.float64), B.astype(np.float64), h.params, L)
    assert np.abs(R - Ro).max() / _norm_scale(A.astype(np.float64), B.astype(np.float64)) <= 1e-5


@pytest.mark.parametrize("d,reduce", [(3, "median"), (4, "median"), (5, "mean")])
def test_cyclic_extract_given_R(cmm, d, reduce):
    m, p, L = 130, 170, 13
    g = np.random.default_rng(d)
    Ro = g.standard_normal((d, 1 << L))
    h = cmm.make_hashes(31 + d, d, L)
    C = cmm.extract_cyclic(_dev(Ro), h, m, p, reduce=reduce).cpu().numpy()
    Co = orc.extract_cyclic(Ro, h.params, m, p, reduce=orc.MEAN if reduce == "mean" else orc.MEDIAN)
    if reduce == "median":
        assert np.array_equal(C, Co)
    else:
        np.testing.assert_allclose(C, Co, rtol=1e-15, atol=1e-15)


def test_cyclic_multiply_recovers_sparse_product(cmm):
    # n = 256, S with 64 nonzeros, b = 2^13 >= 8 nnz: the median recovers S
    # (up to the FP32 rounding of the inputs) except where collisions hit a
    # majority of repetitions; the GPU estimate is within max |R - R_orc| of
    # the oracle's (the median is 1-Lipschitz in the sup norm)
    A, B, S = wl.orthogonal_sparse(seed=1001)
    h = cmm.make_hashes(2001, 5, 13)
    R = torch.empty((5, 1 << 13), dtype=torch.float64, device="cuda")
    C = cmm.multiply_cyclic(_dev(A), _dev(B), h, R=R).cpu().numpy()
    A32 = A.astype(np.float32).astype(np.float64)
    B32 = B.astype(np.float32).astype(np.float64)
    Ro = orc.compress_cyclic(A32, B32, h.params, 13)
    Co = orc.extract_cyclic(Ro, h.params, 256, 256)
    assert np.mean(np.abs(Co - S) < 1e-4) > 0.999
    assert np.abs(C - Co).max() <= np.abs(R.cpu().numpy() - Ro).max() + 1e-15
    assert np.mean(np.abs(C - S) < 1e-4) > 0.999


def test_cyclic_argument_errors(cmm):
    A = _dev(np.ones((8, 4)))
    B = _dev(np.ones((4, 8)))
    with pytest.raises(cmm.CmmError) as e:
        cmm.sketch_cyclic(A, B, cmm.make_hashes(1, 3, 12))   # b below one 2^13 slice
    assert e.value.code == cmm.ERR_RANGE
