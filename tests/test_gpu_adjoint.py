"""The differentiable estimator and its hand-written adjoint on the GPU.

Pins: the oracle's adjoint (dL/dA = M B^T, dL/dB = A^T M with the bucketed
weight matrix M, itself pinned by finite differences and the dense Jacobian in
test_oracle_pins), central finite differences of the GPU forward in FP64 (the
loss is bilinear, so a unit step is exact up to rounding), and torch.gradcheck.
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


def _dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype)


@pytest.mark.parametrize("shape", [(64, 50, 70, 8, 3), (200, 130, 90, 12, 5),
                                   (300, 64, 257, 15, 3), (33, 17, 40, 3, 2),
                                   (512, 96, 256, 14, 4), (1000, 40, 3000, 17, 2)])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("transA", [False, True])
def test_backward_matches_oracle(cmm, shape, prec, transA):
    m, k, p, L, d = shape
    g = np.random.default_rng(m + k + p + L)
    A = g.standard_normal((m, k))
    B = g.standard_normal((k, p))
    P = 300
    I = g.integers(0, m, P).astype(np.int32)
    J = g.integers(0, p, P).astype(np.int32)
    W = g.standard_normal(P)
    h = cmm.make_hashes(31 + L, d, L)
    dt = torch.float64 if prec == "f64" else torch.float32
    Ad = _dev(A.T if transA else A, dt)
    Bd = _dev(B, dt)
    A_in = Ad.double().cpu().numpy()
    B_in = Bd.double().cpu().numpy()
    dA, dB = cmm.backward(Ad, Bd, h, torch.from_numpy(I), torch.from_numpy(J),
                          torch.from_numpy(W), prec=prec, transA=transA)
    dAo, dBo = orc.adjoint(A_in, B_in, h.params, L, I, J, W, transA=transA)
    # tolerance relative to the norm product that bounds each XOR convolution,
    # sum_r ||G_r||_2 ||y_t||, as the sketch tolerance uses sum_t ||A_t|| ||B_t||:
    # column t of dA against ||B[t, :]||, row t of dB against ||A[:, t]||
    G = orc.adjoint_G(h.params, L, I, J, W)
    gn = np.linalg.norm(G, axis=1).sum()
    Am = A_in.T if transA else A_in
    sA = gn * np.linalg.norm(B_in, axis=1)          # per t
    sB = gn * np.linalg.norm(Am, axis=0)            # per t
    tol = 1e-12 if prec == "f64" else 1e-5
    eA = np.abs(dA.double().cpu().numpy() - dAo)
    eB = np.abs(dB.double().cpu().numpy() - dBo)
    eA_t = eA.max(axis=1) if transA else eA.max(axis=0)
    assert (eA_t <= tol * sA).all(), (eA_t / sA).max()
    assert (eB.max(axis=1) <= tol * sB).all(), (eB.max(axis=1) / sB).max()


def test_backward_finite_differences_fp64(cmm):
    # n = 64, b = 2^8: the GPU forward in FP64 differenced against the GPU adjoint
    m = k = p = 64
    L, d = 8, 5
    g = np.random.default_rng(2)
    A = _dev(g.standard_normal((m, k)) / 8)
    B = _dev(g.standard_normal((k, p)) / 8)
    P = 64
    I = torch.from_numpy(g.integers(0, m, P).astype(np.int32)).cuda()
    J = torch.from_numpy(g.integers(0, p, P).astype(np.int32)).cuda()
    W = torch.from_numpy(g.standard_normal(P)).cuda()
    h = cmm.make_hashes(8, d, L)

    def loss(Ax, Bx):
        R = cmm.sketch(Ax, Bx, h, prec="f64")
        return float((cmm.mean_pairs(R, h, I, J) * W).sum().item())

    dA, dB = cmm.backward(A, B, h, I, J, W, prec="f64")
    for (i, t) in [(0, 0), (5, 63), (40, 17), (63, 63)]:
        E = torch.zeros_like(A)
        E[i, t] = 1.0
        fd = (loss(A + E, B) - loss(A - E, B)) / 2
        assert abs(fd - dA[i, t].item()) <= 1e-10 * (1 + abs(fd))
    for (t, j) in [(0, 0), (3, 60), (63, 1)]:
        E = torch.zeros_like(B)
        E[t, j] = 1.0
        fd = (loss(A, B + E) - loss(A, B - E)) / 2
        assert abs(fd - dB[t, j].item()) <= 1e-10 * (1 + abs(fd))


def test_autograd_function_gradcheck(cmm):
    from paper_2601_09477_gb300.autograd_fn import compressed_mean_at_pairs
    m, k, p, L, d = 12, 9, 10, 4, 3
    g = np.random.default_rng(4)
    A = _dev(g.standard_normal((m, k))).requires_grad_()
    B = _dev(g.standard_normal((k, p))).requires_grad_()
    I = torch.from_numpy(g.integers(0, m, 20).astype(np.int32)).cuda()
    J = torch.from_numpy(g.integers(0, p, 20).astype(np.int32)).cuda()
    h = cmm.make_hashes(5, d, L)
    f = lambda A_, B_: compressed_mean_at_pairs(A_, B_, I, J, h, "f64")
    assert torch.autograd.gradcheck(f, (A, B), eps=1e-3, atol=1e-9, rtol=1e-7)


def test_differentiation_workload_4096(cmm):
    # n = 4096 FP32, b = 2^14, d = 5, 4096 weighted pairs (including planted spikes);
    # forward vs oracle on sampled pairs, backward vs the oracle's M B^T / A^T M on
    # sampled rows and columns
    from paper_2601_09477_gb300.autograd_fn import compressed_mean_at_pairs
    A, B, I, J, W = wl.diff_problem(n=4096, spikes=256, pairs=4096, seed=1005)
    L, d = 14, 5
    h = cmm.make_hashes(2005, d, L)
    Ad = _dev(A, torch.float32).requires_grad_()
    Bd = _dev(B, torch.float32).requires_grad_()
    It, Jt = torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()
    Wt = torch.from_numpy(W).cuda()
    est = compressed_mean_at_pairs(Ad, Bd, It, Jt, h, "f32")
    (est.double() * Wt).sum().backward()
    A64, B64 = A.astype(np.float64), B.astype(np.float64)
    # forward: the sketch against the oracle's Compress, and the estimate within
    # the sketch error (the mean is 1-Lipschitz in the sup norm of R)
    R = cmm.sketch(Ad.detach(), Bd.detach(), h, prec="f32").cpu().numpy()
    Ro = orc.compress(A64, B64, h.params, L, nthreads=16)
    dR = np.abs(R - Ro).max()
    scale = float(np.sum(np.linalg.norm(A64, axis=0) * np.linalg.norm(B64, axis=1)))
    assert dR <= 1e-5 * scale
    got = est.detach().double().cpu().numpy()
    assert np.abs(got - orc.mean_at_pairs(Ro, h.params, I, J)).max() <= dR * (1 + 1e-6)
    # backward: the oracle's bucketed weight matrix M, then dA = M B^T, dB = A^T M
    G = orc.adjoint_G(h.params, L, I, J, W)
    M = orc.adjoint_M(G, h.params, 4096, 4096)
    for got, want, scale in [(Ad.grad, M @ B64.T, np.abs(M) @ np.abs(B64).T),
                             (Bd.grad, A64.T @ M, np.abs(A64).T @ np.abs(M))]:
        err = np.abs(got.double().cpu().numpy() - want)
        assert (err <= 1e-4 * scale + 1e-12).all(), (err.max(), scale.max())
