"""CPU-side checks of libcmm: the library loads, exports every entry point that
include/cmm.h declares, its host-side hash generation agrees bit for bit with
the oracle's, and argument errors come back before anything is launched (no
GPU is touched here)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cmm.h")


@pytest.fixture(scope="module")
def cmm():
    from paper_2601_09477_gb300 import build
    build.build()
    from paper_2601_09477_gb300 import cmm as mod
    return mod


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cmm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ["cmm_make_hashes", "cmm_sketch", "cmm_extract", "cmm_heavy_hitters",
              "cmm_threshold", "cmm_multiply", "cmm_mean_pairs", "cmm_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(cmm):
    lib = ctypes.CDLL(cmm.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert "sm_103a" in cmm.version()


@pytest.mark.parametrize("seed,d", [(0, 1), (1, 5), (2009, 9), (2**64 - 1, 64)])
def test_make_hashes_matches_oracle(cmm, seed, d):
    h = cmm.make_hashes(seed, d, 10)
    assert np.array_equal(h.params, orc.draw_hashes(seed, d))


def test_argument_errors_before_launch(cmm):
    lib = cmm.lib
    params = np.zeros((3, 8), dtype=np.uint64)
    hs = cmm.Hashes(3, 8, params)
    dummy = ctypes.c_void_p(256)   # never dereferenced: every call below fails its checks
    # bad d / log2b
    assert lib.cmm_make_hashes(1, 0, params.ctypes.data) == cmm.ERR_RANGE
    assert lib.cmm_make_hashes(1, 65, params.ctypes.data) == cmm.ERR_RANGE
    assert lib.cmm_make_hashes(1, 3, None) == cmm.ERR_ARG
    bad = cmm.Hashes(3, 25, params)
    assert lib.cmm_sketch(dummy, 4, 0, dummy, 4, cmm.F32, 4, 4, 4, bad.ref, cmm.PREC_F32,
                          dummy, dummy, 1 << 30, None) == cmm.ERR_RANGE
    # null operands, bad dtype, bad leading dimension, bad precision
    assert lib.cmm_sketch(None, 4, 0, dummy, 4, cmm.F32, 4, 4, 4, hs.ref, cmm.PREC_F32,
                          dummy, dummy, 1 << 30, None) == cmm.ERR_ARG
    assert lib.cmm_sketch(dummy, 4, 0, dummy, 4, 7, 4, 4, 4, hs.ref, cmm.PREC_F32,
                          dummy, dummy, 1 << 30, None) == cmm.ERR_ARG
    assert lib.cmm_sketch(dummy, 3, 0, dummy, 4, cmm.F32, 4, 4, 4, hs.ref, cmm.PREC_F32,
                          dummy, dummy, 1 << 30, None) == cmm.ERR_ARG
    assert lib.cmm_sketch(dummy, 4, 0, dummy, 4, cmm.F32, 4, 4, 4, hs.ref, 9,
                          dummy, dummy, 1 << 30, None) == cmm.ERR_ARG
    assert "precision" in lib.cmm_last_error().decode()
    # m, p must be < 2^31 (32-bit hash keys)
    assert lib.cmm_sketch(dummy, 1 << 31, 1, dummy, 4, cmm.F32, 1 << 31, 4, 4, hs.ref,
                          cmm.PREC_F32, dummy, dummy, 1 << 30, None) == cmm.ERR_RANGE
    # workspace: null, misaligned, too small
    need = lib.cmm_sketch_workspace_bytes(64, 64, 64, 3, 8, cmm.F64, cmm.PREC_F32, 0)
    assert need > 0
    assert lib.cmm_sketch(dummy, 64, 0, dummy, 64, cmm.F64, 64, 64, 64, hs.ref, cmm.PREC_F32,
                          dummy, None, 0, None) == cmm.ERR_WORKSPACE
    assert lib.cmm_sketch(dummy, 64, 0, dummy, 64, cmm.F64, 64, 64, 64, hs.ref, cmm.PREC_F32,
                          dummy, ctypes.c_void_p(257), need, None) == cmm.ERR_WORKSPACE
    assert lib.cmm_sketch(dummy, 64, 0, dummy, 64, cmm.F64, 64, 64, 64, hs.ref, cmm.PREC_F32,
                          dummy, dummy, need - 1, None) == cmm.ERR_WORKSPACE
    # extraction / heavy hitters
    assert lib.cmm_extract(dummy, hs.ref, 4, 4, 5, dummy, 4, dummy, 1 << 20, None) == cmm.ERR_ARG
    assert lib.cmm_extract(dummy, hs.ref, 4, 4, 0, dummy, 3, dummy, 1 << 20, None) == cmm.ERR_ARG
    cnt = ctypes.c_int64(0)
    assert lib.cmm_heavy_hitters(dummy, hs.ref, 4, 4, 0, 1.0, dummy, dummy, dummy, -1,
                                 ctypes.byref(cnt), dummy, 1 << 20, None) == cmm.ERR_ARG
    assert lib.cmm_heavy_hitters(dummy, hs.ref, 4, 4, 0, 1.0, dummy, dummy, dummy, 4,
                                 None, dummy, 1 << 20, None) == cmm.ERR_ARG
    assert lib.cmm_mean_pairs(dummy, hs.ref, -1, dummy, dummy, dummy, None) == cmm.ERR_ARG


def test_workspace_queries_scale(cmm):
    lib = cmm.lib
    small = lib.cmm_sketch_workspace_bytes(256, 256, 256, 5, 12, cmm.F64, cmm.PREC_F64, 0)
    big = lib.cmm_sketch_workspace_bytes(8192, 8192, 8192, 9, 16, cmm.F64, cmm.PREC_F32, 1)
    assert 0 < small < big
    assert small % 256 == 0 and big % 256 == 0
    assert lib.cmm_sketch_workspace_bytes(8, 8, 8, 0, 4, cmm.F32, cmm.PREC_F32, 0) == 0
    assert lib.cmm_extract_workspace_bytes(100, 100, 5) >= 5 * 200 * 4
    assert lib.cmm_multiply_workspace_bytes(256, 256, 256, 5, 12, cmm.F64, cmm.PREC_F64, 0) >= \
        5 * 4096 * 8


def test_parameter_rule_and_categories():
    # d = 2 floor(c_d log2 n / 2) + 1, b = c_b n (Sec. 5.6)
    import importlib
    ev = importlib.import_module("paper_2601_09477_gb300.evaluate")
    assert ev.params(1024, 1.0, 0.5) == (11, 9)
    assert ev.params(2 ** 15, 0.25, 0.25) == (3, 13)     # formula, not "next odd >= c_d log2 n"
    assert ev.params(2 ** 17, 2.0, 4.0) == (35, 19)
    n = 1024
    base = {"big": 10, "small": n * n - 10}
    perfect = dict(base, **{"B_ge_0.5": 10, "S_le_0.5": n * n - 10, "B_eps_le_0.1": 10,
                            "S_eps_le_0.1": n * n - 10})
    assert ev.category(perfect, n) == "perfect"
    good = dict(perfect, **{"S_eps_le_0.1": n * n - 10 - n})
    assert ev.category(good, n) == "good"
    decent = dict(good, **{"B_eps_le_0.1": 1, "S_eps_le_0.1": int(0.995 * (n * n - 10))})
    assert ev.category(decent, n) == "decent"
    sat = dict(decent, **{"B_eps_le_0.1": 0})
    assert ev.category(sat, n) == "satisfactory"
    none = dict(sat, **{"B_ge_0.5": 5})
    assert ev.category(none, n) == "none"


def test_tensor_core_precisions_checked_before_launch(cmm):
    # BF16TC and FP16TC share the 2^15-slice plan: the same workspace, and a
    # sketch length below one slice is refused before anything is launched
    lib = cmm.lib
    ws_bf = lib.cmm_sketch_workspace_bytes(512, 300, 400, 3, 16, cmm.F32, cmm.PREC_BF16TC, 0)
    ws_f16 = lib.cmm_sketch_workspace_bytes(512, 300, 400, 3, 16, cmm.F32, cmm.PREC_F16TC, 0)
    assert ws_bf > 0 and ws_bf == ws_f16
    params = np.zeros((3, 8), dtype=np.uint64)
    small = cmm.Hashes(3, 12, params)
    dummy = ctypes.c_void_p(256)   # never dereferenced: the calls fail their checks
    for prec in (cmm.PREC_BF16TC, cmm.PREC_F16TC):
        assert lib.cmm_sketch(dummy, 4, 0, dummy, 4, cmm.F32, 4, 4, 4, small.ref, prec,
                              dummy, dummy, 1 << 30, None) == cmm.ERR_RANGE
        assert "tensor-core" in lib.cmm_last_error().decode()
    assert lib.cmm_sketch(dummy, 4, 0, dummy, 4, cmm.F32, 4, 4, 4, small.ref, 6,
                          dummy, dummy, 1 << 30, None) == cmm.ERR_ARG   # no precision 6
