"""cmm_sketch_noalloc: the sketch for callers that cannot allocate device memory.

Serving processes that fix their device-memory budget at start-up, plugins
whose host application owns every allocation, and latency-critical paths that
cannot pay for cudaMalloc's implicit synchronisation cannot pass a workspace.
This entry point keeps its scratch in a static device array inside libcmm.
These checks call it through the C ABI and compare it with cmm_sketch (the
workspace version) on two calls in a row, so the second call runs on scratch
that still holds the first call's data.  The file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


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


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_noalloc_matches_workspace_version_twice(cmm, prec):
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
        err = (R_na - R_ws).abs().max().item() / _scale(At, B)
        assert err <= TOL[prec], err


def test_noalloc_rejects_oversized_problem(cmm):
    # n = 8192, b = 2^16, d = 9 needs far more than the static array holds
    h = cmm.make_hashes(1, 9, 16)
    need = cmm.lib.cmm_sketch_workspace_bytes(8192, 8192, 8192, 9, 16, cmm.F64, cmm.PREC_F32, 0)
    assert need > (64 << 20)
    dummy = ctypes.c_void_p(256)   # never touched: the call fails its size check first
    rc = cmm.lib.cmm_sketch_noalloc(dummy, 8192, 0, dummy, 8192, cmm.F64, 8192, 8192, 8192,
                                    h.ref, cmm.PREC_F32, dummy, None)
    assert rc == cmm.ERR_RANGE
    assert "static array" in cmm.lib.cmm_last_error().decode()
