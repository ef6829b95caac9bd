"""The host-buffer entry point (cmm_multiply_host): operands copied in parts on
an internal stream while earlier parts are sketched, the estimate extracted in
row blocks and copied back block by block.  Its results must equal those of
the device-buffer path (cmm_multiply + cmm_threshold): bit for bit on +-1
inputs, where every quantity is an integer and the order of additions cannot
matter, and bit for bit whenever the operands are too small to be split."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cmm():
    assert torch.cuda.is_available(), "these tests need a CUDA GPU"
    from paper_2601_09477_gb300 import cmm as mod
    return mod


def _pm1(shape, seed):
    g = np.random.default_rng(seed)
    return np.where(g.random(shape) < 0.5, -1.0, 1.0)


@pytest.mark.parametrize("transA", [False, True])
@pytest.mark.parametrize("n,prec", [(2048, "f32"), (2048, "f64"), (4096, "f32")])
def test_host_path_split_matches_device_path(cmm, transA, n, prec):
    # FP64 operands of 64 MiB or more: two parts along the inner index (three
    # from 256 MiB, n = 4096), growing geometrically; one row block per 16 MiB
    # of the estimate (2 at n = 2048, 8 at n = 4096)
    A = _pm1((n, n), 1)
    A[5] = A[9]            # a planted pair: C[5, 9] = n
    B = A.T.copy()
    h = cmm.make_hashes(17, 9, 16)
    Ah = torch.from_numpy(np.ascontiguousarray(A.T) if transA else A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    tau = 0.75 * n
    Ch, (I, J, V) = cmm.multiply_host(Ah, Bh, h, prec=prec, transA=transA, tau=tau,
                                      capacity=1 << 20)
    Cd = cmm.multiply(Ah.cuda(), Bh.cuda(), h, prec=prec, transA=transA)
    assert torch.equal(Ch, Cd.cpu())
    Id, Jd, Vd = cmm.threshold(Cd, tau, capacity=1 << 20)
    assert np.array_equal(I.numpy(), Id.cpu().numpy())
    assert np.array_equal(J.numpy(), Jd.cpu().numpy())
    assert np.array_equal(V.numpy(), Vd.cpu().numpy())
    assert (5, 9) in set(zip(I.tolist(), J.tolist()))


def test_host_path_four_parts_full_size(cmm):
    # the benchmark's size: 1 GiB of FP64 operands in four parts, 512 MiB of
    # estimate in eight row blocks; bit-identical to the device path on +-1
    n = 8192
    A = _pm1((n, n), 7)
    A[11] = A[3]
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()
    h = cmm.make_hashes(2002, 9, 16)
    Ch, (I, J, V) = cmm.multiply_host(Ah, Bh, h, prec="f32", tau=n / 2, capacity=1 << 22)
    Ad, Bd = Ah.cuda(), Bh.cuda()
    Cd, (Id, Jd, Vd) = cmm.multiply_threshold(Ad, Bd, h, n / 2, capacity=1 << 22, prec="f32")
    assert torch.equal(Ch, Cd.cpu())
    assert np.array_equal(I.numpy(), Id.cpu().numpy())
    assert np.array_equal(J.numpy(), Jd.cpu().numpy())
    assert np.array_equal(V.numpy(), Vd.cpu().numpy())
    assert (3, 11) in set(zip(I.tolist(), J.tolist()))


@pytest.mark.parametrize("prec,L", [("f32", 12), ("bf16tc", 15), ("f16tc", 15)])
def test_host_path_padded_small(cmm, prec, L):
    # below the split thresholds: one part, one row block; padded leading
    # dimensions on the host side; every butterfly precision
    m, k, p, d = 300, 200, 250, 3
    g = np.random.default_rng(3)
    Abig = torch.from_numpy(g.standard_normal((m, k + 7)).astype(np.float32)).pin_memory()
    Bbig = torch.from_numpy(g.standard_normal((k, p + 3)).astype(np.float32)).pin_memory()
    A, B = Abig[:, :k], Bbig[:, :p]
    h = cmm.make_hashes(5, d, L)
    Ch, _ = cmm.multiply_host(A, B, h, prec=prec, tau=1e30, capacity=4)
    Cd = cmm.multiply(A.cuda(), B.cuda(), h, prec=prec)
    assert torch.equal(Ch, Cd.cpu())
    if prec != "f32":
        return
    # and the estimate is the oracle's decompression of the oracle's sketch
    A64 = A.double().numpy()
    B64 = B.double().numpy()
    Ro = orc.compress(A64, B64, h.params, L, nthreads=8)
    R = cmm.sketch(A.cuda(), B.cuda(), h, prec="f32").cpu().numpy()
    scale = float(np.sum(np.linalg.norm(A64, axis=0) * np.linalg.norm(B64, axis=1)))
    assert np.abs(R - Ro).max() / scale <= 1e-5


@pytest.mark.parametrize("transA", [False, True])
def test_host_path_parts_fx64_and_ternary(cmm, transA):
    # the exact forms through the host path: FP64 operands of 64 MiB, split in
    # parts along the inner index (the fixed-point form reads its FP64 rows at
    # 8 bytes per element in every part); N(0,1) operands for the fixed-point
    # form (within the FP64 tolerance of the device path), +-1 operands for the
    # ternary form (one part, bit for bit)
    n = 2048
    g = np.random.default_rng(3)
    A = g.standard_normal((n, n))
    B = g.standard_normal((n, n))
    h = cmm.make_hashes(19, 5, 15)
    Ah = torch.from_numpy(np.ascontiguousarray(A.T) if transA else A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    Ch, _ = cmm.multiply_host(Ah, Bh, h, prec="fx64", transA=transA)
    Cd = cmm.multiply(Ah.cuda(), Bh.cuda(), h, prec="fx64", transA=transA)
    scale = float(np.sum(np.linalg.norm(A, axis=0) * np.linalg.norm(B, axis=1)))
    assert float((Ch - Cd.cpu()).abs().max()) <= 2e-12 * scale
    Ro = orc.compress(A, B, h.params, 15, nthreads=orc.max_threads())
    Co = orc.extract(Ro, h.params, n, n, rows=(100, 104))
    assert np.abs(Ch[100:104].numpy() - Co).max() <= 2e-12 * scale
    P = _pm1((n, n), 4)
    Ph = torch.from_numpy(P).pin_memory()
    Qh = torch.from_numpy(np.ascontiguousarray(P.T)).pin_memory()
    Ct, (I, J, V) = cmm.multiply_host(Ph, Qh, h, prec="ternary", tau=0.75 * n, capacity=1 << 20)
    Ctd = cmm.multiply(Ph.cuda(), Qh.cuda(), h, prec="ternary")
    assert torch.equal(Ct, Ctd.cpu())
    assert len(I) > 0 and bool((Ct[I.long(), J.long()] == V).all())
