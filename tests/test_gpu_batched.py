"""Many independent problems in one persistent launch (cmm_batched_*).

Every problem's R is checked against the oracle's Compress (FP32 tolerance
relative to sum_t ||A_t|| ||B_t||) and its dense estimate against the oracle's
Decompress of the same R (bit-identical); the launch is replayed from a CUDA
graph; and the bounded dependency wait is made to run out on purpose (a
dependency target that nothing meets) to check that the timeout comes back as
CMM_ERR_TIMEOUT and the context stays usable.
"""
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


def _scale(A, B):
    return float(np.sum(np.linalg.norm(A, axis=0) * np.linalg.norm(B, axis=1)))


def _small_batch(cmm, d=5, seed=3):
    g = np.random.default_rng(seed)
    specs = [(20, 33, 41, 5), (100, 64, 90, 8), (257, 130, 200, 10), (300, 500, 120, 12),
             (64, 1000, 70, 13), (400, 77, 333, 14), (150, 260, 170, 15), (90, 40, 60, 16),
             (33, 300, 29, 11), (211, 211, 211, 9)]
    probs, host = [], []
    for q, (m, k, p, L) in enumerate(specs):
        A = g.standard_normal((m, k))
        B = g.standard_normal((k, p))
        At = torch.from_numpy(np.ascontiguousarray(A.T)).to("cuda", torch.float32)
        Bt = torch.from_numpy(B).to("cuda", torch.float32)
        h = cmm.make_hashes(5000 + q, d, L)
        tile = 0
        tt = 0
        if q == 7:
            tile, tt = 12, 17     # explicit b-tile / t-tile
        probs.append(cmm.Problem(At, Bt, h, tile_log2=tile, t_tile=tt))
        host.append((At.double().cpu().numpy().T.copy(), Bt.double().cpu().numpy(), h, L))
    return probs, host


def _check(cmm, probs, host):
    for pb, (A, B, h, L) in zip(probs, host):
        R = pb.R.cpu().numpy()
        Ro = orc.compress(A, B, h.params, L, nthreads=8)
        assert np.abs(R - Ro).max() <= 1e-5 * _scale(A, B)
        Co = orc.extract(R, h.params, A.shape[0], B.shape[1])
        assert np.array_equal(pb.C.cpu().numpy(), Co)


def test_batched_matches_oracle(cmm):
    probs, host = _small_batch(cmm)
    batch = cmm.Batch(probs, d=5)
    batch.launch()
    assert batch.status() == cmm.OK
    _check(cmm, probs, host)


def test_batched_graph_replay(cmm):
    probs, host = _small_batch(cmm, seed=8)
    batch = cmm.Batch(probs, d=5)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.launch(stream=s)          # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    first = [(pb.R.clone(), pb.C.clone()) for pb in probs]
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.launch()
    for pb in probs:
        pb.R.zero_()
        pb.C.zero_()
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert batch.status() == cmm.OK
        for pb, (R0, C0) in zip(probs, first):
            assert torch.equal(pb.R, R0) and torch.equal(pb.C, C0)
    _check(cmm, probs, host)


def test_batched_wait_timeout_is_reported(cmm):
    probs, host = _small_batch(cmm, seed=11)
    batch = cmm.Batch(probs, d=5)
    batch.launch(wait_budget_us=200_000, unmet_dependency=True)
    assert batch.status() == cmm.ERR_TIMEOUT
    assert "wait" in cmm.lib.cmm_last_error().decode()
    # the context is still usable and a normal launch is correct
    batch.launch()
    assert batch.status() == cmm.OK
    _check(cmm, probs, host)


def test_autotuner_choices_are_valid_and_correct(cmm, tmp_path):
    from paper_2601_09477_gb300 import autotune
    probs, host = _small_batch(cmm, seed=21)
    cache = str(tmp_path / "tune.json")
    tuner = autotune.tune_batch(probs, d=5, cache_path=cache, budget_s=60)
    assert len(tuner.table) >= 3
    for key, (tile, tt) in tuner.table.items():
        L = int(key.split("_")[0][1:])
        assert tt >= 0 and (tile == 0 or 5 <= tile <= min(14, L))
    # a fresh tuner reads the cache back; the tuned batch is still exact
    again = autotune.Tuner(cache)
    assert again.table == tuner.table
    batch = cmm.Batch(probs, d=5)
    batch.launch()
    assert batch.status() == cmm.OK
    _check(cmm, probs, host)


def test_batched_rejects_bad_problems(cmm):
    h = cmm.make_hashes(1, 5, 10)
    At = torch.zeros((10, 20), dtype=torch.float64, device="cuda")
    B = torch.zeros((10, 30), dtype=torch.float32, device="cuda")
    with pytest.raises(TypeError):
        cmm.Batch([cmm.Problem(At, B, h)], d=5)
    with pytest.raises(ValueError):
        cmm.Batch([cmm.Problem(At.float(), B[:5], h)], d=5)


def test_batched_256_uneven_problems(cmm):
    # 256 problems, m, k, p uniform in [512, 4096], b = 2^10 .. 2^15, d = 5, FP32,
    # 16 planted spikes each; one problem per sketch length checked in full
    d = 5
    raw = wl.batch_problems_device(count=256, seed=1004, device="cuda")
    probs = [cmm.Problem(At, B, cmm.make_hashes(7000 + q, d, L)) for q, (At, B, L, _) in enumerate(raw)]
    batch = cmm.Batch(probs, d=d)
    batch.launch()
    assert batch.status() == cmm.OK
    work = [pb.At.shape[0] * (1 << pb.hashes.log2b) * pb.hashes.log2b for pb in probs]
    # the cheapest problem of every sketch length b = 2^10 .. 2^15 in full: the
    # whole R against the oracle's Compress, the whole estimate against the
    # oracle's Decompress of the same R
    classes = sorted({pb.hashes.log2b for pb in probs})
    assert classes == list(range(10, 16))
    for L in classes:
        q = min((q for q in range(len(probs)) if probs[q].hashes.log2b == L), key=lambda q: work[q])
        pb = probs[q]
        A = pb.At.double().cpu().numpy().T.copy()
        B = pb.B.double().cpu().numpy()
        Ro = orc.compress(A, B, pb.hashes.params, L, nthreads=orc.max_threads())
        R = pb.R.cpu().numpy()
        assert np.abs(R - Ro).max() <= 1e-5 * _scale(A, B), (q, L)
        Co = orc.extract(R, pb.hashes.params, A.shape[0], B.shape[1], nthreads=8)
        assert np.array_equal(pb.C.cpu().numpy(), Co), (q, L)
    # the largest-b, largest-m problem on sampled entries and rows
    qb = int(np.argmax([pb.hashes.log2b * 10**8 + pb.At.shape[0] for pb in probs]))
    pb = probs[qb]
    A = pb.At.double().cpu().numpy().T.copy()
    B = pb.B.double().cpu().numpy()
    L = pb.hashes.log2b
    R = pb.R.cpu().numpy()
    scale = _scale(A, B)
    g = np.random.default_rng(0)
    for r, w in [(0, int(g.integers(0, 1 << L))), (d - 1, int(g.integers(0, 1 << L)))]:
        assert abs(R[r, w] - orc.R_entry(A, B, pb.hashes.params, L, r, w)) <= 1e-5 * scale
    rows = (5, 9)
    Co = orc.extract(R, pb.hashes.params, A.shape[0], B.shape[1], rows=rows)
    assert np.array_equal(pb.C[rows[0]:rows[1]].cpu().numpy(), Co)


def test_batched_256_problems_literal_b1024(cmm):
    # the literal sketch-length rule (every problem at b = 2^10) on the same 256
    # operand pairs: the smallest and the largest problem in full against the
    # oracle (whole R, whole estimate given the same R)
    d = 5
    raw = wl.batch_problems_device(count=256, seed=1004, device="cuda")
    probs = [cmm.Problem(At, B, cmm.make_hashes(7000 + q, d, 10)) for q, (At, B, _, _) in enumerate(raw)]
    batch = cmm.Batch(probs, d=d)
    batch.launch()
    assert batch.status() == cmm.OK
    size = [pb.At.shape[0] * pb.At.shape[1] * pb.B.shape[1] for pb in probs]
    for q in (int(np.argmin(size)), int(np.argmax(size))):
        pb = probs[q]
        A = pb.At.double().cpu().numpy().T.copy()
        B = pb.B.double().cpu().numpy()
        Ro = orc.compress(A, B, pb.hashes.params, 10, nthreads=orc.max_threads())
        R = pb.R.cpu().numpy()
        assert np.abs(R - Ro).max() <= 1e-5 * _scale(A, B), q
        Co = orc.extract(R, pb.hashes.params, A.shape[0], B.shape[1], nthreads=8)
        assert np.array_equal(pb.C.cpu().numpy(), Co), q
