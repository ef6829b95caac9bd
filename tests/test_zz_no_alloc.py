"""cmm_sketch_noalloc: the sketch for callers that cannot allocate device memory.

Serving processes that fix their device-memory budget at start-up, plugins
whose host application owns every allocation, and latency-critical paths that
cannot pay for cudaMalloc's implicit synchronisation cannot pass a workspace.
This entry point keeps its scratch in a static device array inside libcmm.
These checks call it through the C ABI and compare it with cmm_sketch (the
workspace version) and with the FP64 oracle on two calls in a row, so the
second call runs on scratch that still holds the first call's data.  The file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "fx64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def cmm():
    assert torch.cuda.is_available(), "this test needs a CUDA GPU"
    from paper_2601_09477_gb300 import cmm as mod
    fn = mod.lib.cmm_sketch_noalloc
    fn.restype = ctypes.c_int
    i64, i32, P = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
    fn.argtypes = [P, i64, i32, P, i64, i32, i64, i64, i64, ctypes.POINTER(mod._Hashes), i32, P, P]
    return mod


def _noalloc(cmm, A, B, h, prec, transA=False):
    m, k, p, dt = cmm._operands(A, B, transA)
    R = torch.full((h.d, h.b), float("nan"), dtype=torch.float64, device=A.device)
    rc = cmm.lib.cmm_sketch_noalloc(A.data_ptr(), A.stride(0), int(transA), B.data_ptr(),
                                    B.stride(0), dt, m, k, p, h.ref, cmm._PREC[prec],
                                    R.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == cmm.OK, cmm.lib.cmm_last_error().decode()
    torch.cuda.synchronize()
    return R


def _scale(A, B):
    A = A.double().cpu().numpy()
    B = B.double().cpu().numpy()
    return float(np.sum(np.linalg.norm(A, axis=0) * np.linalg.norm(B, axis=1)))


@pytest.mark.parametrize("prec", ["f64", "fx64", "f32"])
def test_noalloc_matches_workspace_version_twice(cmm, prec):
    from oracle import oracle as orc
    g = np.random.default_rng(12)
    problems = [(256, 256, 256, 12, 5, torch.float64, False),
                (300, 517, 200, 13, 3, torch.float32, True)]
    for (m, k, p, L, d, dtype, transA) in problems:      # two calls in a row
        A = torch.from_numpy(g.standard_normal((k, m) if transA else (m, k))).to("cuda", dtype)
        B = torch.from_numpy(g.standard_normal((k, p))).to("cuda", dtype)
        h = cmm.make_hashes(900 + L, d, L)
        R_ws = cmm.sketch(A, B, h, prec=prec, transA=transA)
        R_na = _noalloc(cmm, A, B, h, prec, transA)
        assert not torch.isnan(R_na).any()
        At = A.t() if transA else A
        scale = _scale(At, B)
        err = (R_na - R_ws).abs().max().item() / scale
        assert err <= TOL[prec], err
        # and against the FP64 oracle on the same (widened) operand values
        Ro = orc.compress(A.double().cpu().numpy(), B.double().cpu().numpy(), h.params, L,
                          transA=transA)
        err_o = float(np.abs(R_na.cpu().numpy() - Ro).max()) / scale
        assert err_o <= TOL[prec], err_o


def test_noalloc_rejects_oversized_problem(cmm):
    # m = k = p = 64 with b = 2^20 and d = 9: the operands are small, but the
    # per-block partial sums and the reduced sums (d x b FP64 each) need more
    # scratch than the static array holds.  Every buffer is real and sized for
    # the problem, so even a call that got past the size check would only
    # compute a result.
    m = k = p = 64
    L, d = 20, 9
    h = cmm.make_hashes(1, d, L)
    need = cmm.lib.cmm_sketch_workspace_bytes(m, k, p, d, L, cmm.F64, cmm.PREC_F32, 0)
    assert need > (64 << 20)   # CMM_SKETCH_NOALLOC_SCRATCH_BYTES
    g = np.random.default_rng(5)
    A = torch.from_numpy(g.standard_normal((m, k))).cuda()
    B = torch.from_numpy(g.standard_normal((k, p))).cuda()
    R = torch.zeros((d, 1 << L), dtype=torch.float64, device="cuda")
    rc = cmm.lib.cmm_sketch_noalloc(A.data_ptr(), k, 0, B.data_ptr(), p, cmm.F64, m, k, p,
                                    h.ref, cmm.PREC_F32, R.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert rc == cmm.ERR_RANGE
    assert "static array" in cmm.lib.cmm_last_error().decode()
    torch.cuda.synchronize()
    assert not R.any()   # nothing ran
