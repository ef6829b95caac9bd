"""The paper's evaluation of an estimate (Sec. 5.3) and its parameter rule
(Sec. 5.6), on top of the library.

* ``params(n, c_d, c_b)``: d = 2 * floor(c_d * log2 n / 2) + 1 and b = c_b * n
  (rounded up to a power of two; the sketch length must be one).
* ``counters(C_hat, big_mask, C_true)``: the four counts of Sec. 5.3 --
  big entries with |estimate| >= 0.5, small entries with |estimate| <= 0.5,
  big / small entries within 0.1 of the true value.
* ``category(...)``: the Perfect / Good / Decent / Satisfactory classes of
  Sec. 5.6 for one run.
* ``run_instance(name, n, c_d, c_b, seed, hash_seed)``: draw one of the paper's
  instance families, estimate A B on the GPU and return the counters.

The counters are computed with torch on the device; no step of the method
itself runs here.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import cmm
from . import workloads as wl


def params(n: int, c_d: float, c_b: float):
    """(d, log2 b) of the paper's rule; b = c_b n rounded up to a power of two."""
    d = 2 * int(math.floor(c_d * math.log2(n) / 2.0)) + 1
    b = max(2, c_b * n)
    return d, int(math.ceil(math.log2(b)))


def counters(C_hat: torch.Tensor, big: torch.Tensor, C_true: torch.Tensor) -> dict:
    small = ~big
    err = (C_hat - C_true).abs()
    a = C_hat.abs()
    return {
        "big": int(big.sum().item()),
        "small": int(small.sum().item()),
        "B_ge_0.5": int((big & (a >= 0.5)).sum().item()),
        "S_le_0.5": int((small & (a <= 0.5)).sum().item()),
        "B_eps_le_0.1": int((big & (err <= 0.1)).sum().item()),
        "S_eps_le_0.1": int((small & (err <= 0.1)).sum().item()),
    }


def category(c: dict, n: int) -> str:
    """Best class of Sec. 5.6 that this single run satisfies."""
    B, S = c["big"], c["small"]
    if c["B_eps_le_0.1"] + c["S_eps_le_0.1"] == B + S:
        return "perfect"
    if c["B_eps_le_0.1"] == B and c["S_eps_le_0.1"] >= S - n:
        return "good"
    if (c["B_eps_le_0.1"] >= max(B - math.log2(n), 1) and c["S_eps_le_0.1"] >= 0.99 * S):
        return "decent"
    if c["B_ge_0.5"] >= 0.99 * B and c["S_le_0.5"] >= 0.99 * S:
        return "satisfactory"
    return "none"


def instance(name: str, n: int, seed: int):
    """(A, B, C_true, big_mask) as device float64 tensors for one instance family."""
    if name == "logunit":
        A, B, C = wl.logunit(n, seed=seed)
        big = np.abs(C) >= 0.5
    elif name == "diagonal":
        A, B, C = wl.diagonal(n, seed=seed)
        big = np.abs(C) >= 0.5
    elif name in ("covariance", "lightbulb"):
        gen = wl.covariance if name == "covariance" else wl.lightbulb
        A, B, (i, j) = gen(n, seed=seed)
        C = None
        big = np.zeros((n, n), dtype=bool)
        big[i, j] = True
    else:
        raise ValueError(name)
    dev = torch.device("cuda")
    At = torch.from_numpy(np.ascontiguousarray(A)).to(dev)
    Bt = torch.from_numpy(np.ascontiguousarray(B)).to(dev)
    Ct = At @ Bt if C is None else torch.from_numpy(np.ascontiguousarray(C)).to(dev)
    return At, Bt, Ct, torch.from_numpy(big).to(dev)


def variance_experiment(name: str, n: int, log2b: int, draws: int, seed: int = 1,
                        prec: str = "f64"):
    """Sec. 5.4: d = 1, ``draws`` independent hash draws, the estimate of the
    instance's largest entry each time.  Returns (mean, sample variance, true
    value, ||C||_F^2 / b)."""
    A, B, C, big = instance(name, n, seed)
    flat = int(torch.argmax(C.abs()).item())
    i, j = divmod(flat, n)
    I = torch.tensor([i], dtype=torch.int32, device=A.device)
    J = torch.tensor([j], dtype=torch.int32, device=A.device)
    est = torch.empty(draws, dtype=torch.float64, device=A.device)
    for s in range(draws):
        h = cmm.make_hashes(10_000 + s, 1, log2b)
        R = cmm.sketch(A, B, h, prec=prec)
        est[s] = cmm.mean_pairs(R, h, I, J)[0]
    bound = float((C ** 2).sum().item()) / (1 << log2b)
    return float(est.mean().item()), float(est.var().item()), float(C[i, j].item()), bound


def run_instance(name: str, n: int, c_d: float, c_b: float, seed: int = 1, hash_seed: int = 2,
                 prec: str = "f64") -> dict:
    d, L = params(n, c_d, c_b)
    A, B, C, big = instance(name, n, seed)
    h = cmm.make_hashes(hash_seed, d, L)
    C_hat = cmm.multiply(A, B, h, prec=prec)
    out = counters(C_hat, big, C)
    out.update({"instance": name, "n": n, "d": d, "log2b": L, "c_d": c_d, "c_b": c_b,
                "category": category(out, n)})
    return out
