"""The exact form for ternary operands (CMM_PREC_TERNARY: every entry -1, 0 or
+1, the +-1 inputs of Sec. 5.2): R equal to the FP64 oracle's bit for bit
(every quantity is an integer), over one to several frequency slices, odd k
(a last pair with one row), every storage type and layout, zeros among the
signs, sizes that force the int32 running sums to be flushed after every
pair; the size limits and the entry check are reported as errors."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cmm():
    assert torch.cuda.is_available()
    from paper_2601_09477_gb300 import cmm as mod
    return mod


def _ternary(g, shape, zeros):
    x = np.where(g.random(shape) < 0.5, -1.0, 1.0)
    if zeros:
        x[g.random(shape) < 0.3] = 0.0
    return x


def _dev(x, dtype, transA=False):
    x = x.T.copy() if transA else x
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


@pytest.mark.parametrize("shape", [(512, 300, 700, 14, 5), (1000, 257, 900, 15, 3),
                                   (2048, 64, 2048, 16, 9), (301, 33, 4099, 17, 4)])
@pytest.mark.parametrize("dtype,transA,zeros", [(torch.float64, False, False),
                                                (torch.float64, True, True),
                                                (torch.float32, False, True),
                                                (torch.bfloat16, True, False)])
def test_ternary_bit_exact(cmm, shape, dtype, transA, zeros):
    m, k, p, L, d = shape
    g = np.random.default_rng(m + 3 * k + L)
    A = _ternary(g, (m, k), zeros)
    B = _ternary(g, (k, p), zeros)
    h = cmm.make_hashes(5000 + L, d, L)
    R = torch.empty((d, 1 << L), dtype=torch.float64, device="cuda")
    C = cmm.multiply(_dev(A, dtype, transA), _dev(B, dtype), h, prec="ternary", transA=transA, R=R)
    Ro = orc.compress(A, B, h.params, L, nthreads=orc.max_threads())
    Rn = R.cpu().numpy()
    assert np.array_equal(Rn, Ro)
    rows = (0, min(m, 64))
    Co = orc.extract(Rn, h.params, m, p, rows=rows)
    assert np.array_equal(C[rows[0]:rows[1]].cpu().numpy(), Co)


def test_ternary_flush_every_pair(cmm):
    # m = p = 24000: 2 m p > 2^30, so the int32 running sums are added into the
    # int64 accumulator after every pair of inner indices
    m = p = 24000
    k, L, d = 20, 14, 3
    g = np.random.default_rng(17)
    A = _ternary(g, (m, k), False)
    B = _ternary(g, (k, p), False)
    A[:, 1] = A[:, 0]   # correlated columns: large transformed values
    h = cmm.make_hashes(321, d, L)
    R = cmm.sketch(_dev(A, torch.float32), _dev(B, torch.float32), h, prec="ternary").cpu().numpy()
    Ro = orc.compress(A, B, h.params, L, nthreads=orc.max_threads())
    assert np.array_equal(R, Ro)


def test_ternary_rejects_other_entries_and_sizes(cmm):
    h = cmm.make_hashes(1, 3, 14)
    A = torch.ones((64, 16), dtype=torch.float64, device="cuda")
    B = torch.ones((16, 64), dtype=torch.float64, device="cuda")
    A[5, 3] = 2.0
    with pytest.raises(cmm.CmmError) as ei:
        cmm.sketch(A, B, h, prec="ternary")
    assert ei.value.code == cmm.ERR_ARG and "-1, 0 or 1" in str(ei.value)
    A[5, 3] = 0.5
    with pytest.raises(cmm.CmmError):
        cmm.sketch(A, B, h, prec="ternary")
    A[5, 3] = -1.0
    R = cmm.sketch(A, B, h, prec="ternary")   # valid again
    assert np.array_equal(R.cpu().numpy(), orc.compress(A.cpu().numpy(), B.cpu().numpy(),
                                                        h.params, 14))
    small = cmm.make_hashes(1, 3, 13)
    with pytest.raises(cmm.CmmError) as ei:
        cmm.sketch(A, B, small, prec="ternary")
    assert ei.value.code == cmm.ERR_RANGE
    Awide = torch.ones((32768, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(cmm.CmmError) as ei:
        cmm.sketch(Awide, torch.ones((2, 8), dtype=torch.float32, device="cuda"), h,
                   prec="ternary")
    assert ei.value.code == cmm.ERR_RANGE
