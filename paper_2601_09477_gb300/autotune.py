"""Autotuner for the batched launch: per problem class, the b-tile (log2 of the
transform slice one CTA holds; the rest of log2 b is folded into the scatter)
and the t-tile (inner indices per sketch task).

A class is (log2 b, the power of two just above k, d): the sketch work per
task grows with k and b, while m and p only change the scatter length.  For each class
the tuner times one batched launch over copies of a representative problem
(enough copies to fill the GPU) for every candidate tile pair, and keeps the
fastest.  Results persist in a JSON cache so a later process (or a CUDA-graph
capture) reuses them without timing.  Timing uses CUDA events on the launch
stream after a warm-up launch.
"""
from __future__ import annotations

import json
import math
import os
import time

import torch

from . import cmm

DEFAULT_CACHE = os.environ.get(
    "CMM_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cmm_autotune.json"))


def _pow2_ceil(x: int) -> int:
    return 1 << max(0, int(math.ceil(math.log2(max(1, x)))))


def class_key(m: int, k: int, p: int, log2b: int, d: int) -> str:
    return "L%d_k%d_d%d" % (log2b, _pow2_ceil(k), d)


def candidates(log2b: int, k: int):
    """(tile_log2, t_tile) pairs; 0 means the library's default rule."""
    tiles = sorted({t for t in (log2b - 2, log2b - 1, log2b, 14, 13)
                    if 5 <= t <= min(14, log2b)}, reverse=True)
    tts = [0, 64, 256, 1024]
    return [(t, tt) for t in tiles for tt in tts if tt == 0 or tt < k]


class Tuner:
    def __init__(self, cache_path: str | None = DEFAULT_CACHE):
        self.cache_path = cache_path
        self.table: dict[str, list[int]] = {}
        if cache_path and os.path.exists(cache_path):
            try:
                with open(cache_path) as f:
                    self.table = {k: list(v) for k, v in json.load(f).items()}
            except (OSError, ValueError):
                self.table = {}

    def save(self):
        if not self.cache_path:
            return
        os.makedirs(os.path.dirname(self.cache_path) or ".", exist_ok=True)
        tmp = self.cache_path + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(self.table, f, indent=1, sort_keys=True)
        os.replace(tmp, self.cache_path)

    def lookup(self, m, k, p, log2b, d):
        return self.table.get(class_key(m, k, p, log2b, d))

    def _time(self, data, log2b, d, tile, tt) -> float:
        probs = [cmm.Problem(At, B, h, tile_log2=tile, t_tile=tt) for (At, B, h) in data]
        batch = cmm.Batch(probs, d=d)
        batch.launch()
        if batch.status() != cmm.OK:
            return float("inf")
        s = torch.cuda.current_stream()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        batch.launch()
        e1.record(s)
        torch.cuda.synchronize()
        if batch.status() != cmm.OK:
            return float("inf")
        return e0.elapsed_time(e1)

    def tune_class(self, m, k, p, log2b, d, device="cuda", copies: int | None = None) -> list[int]:
        key = class_key(m, k, p, log2b, d)
        if key in self.table:
            return self.table[key]
        if copies is None:
            # about two CTAs' worth of sketch tasks per SM at the default tiles
            work = d * max(1, 1 << (log2b - min(14, log2b))) * max(1, k // 256)
            copies = max(2, min(32, int(math.ceil(304 / max(1, work)))))
        gen = torch.Generator(device=device)
        gen.manual_seed(1234)
        data = [(torch.randn(k, m, generator=gen, device=device),
                 torch.randn(k, p, generator=gen, device=device),
                 cmm.make_hashes(77 + q, d, log2b)) for q in range(copies)]
        best, best_ms = [0, 0], float("inf")
        for tile, tt in candidates(log2b, k):
            ms = self._time(data, log2b, d, tile, tt)
            if ms < best_ms * 0.98:
                best, best_ms = [tile, tt], ms
        self.table[key] = best
        return best

    def apply(self, problems, d, tune_missing: bool = True):
        """Set tile_log2 / t_tile of every cmm.Problem from the table (tuning
        classes not yet in it when ``tune_missing``)."""
        for pb in problems:
            k, m = pb.At.shape
            p = pb.B.shape[1]
            hit = self.lookup(m, k, p, pb.hashes.log2b, d)
            if hit is None and tune_missing:
                hit = self.tune_class(m, k, p, pb.hashes.log2b, d, device=pb.At.device)
            if hit is not None:
                pb.tile_log2, pb.t_tile = int(hit[0]), int(hit[1])
        return problems


def tune_batch(problems, d, cache_path: str | None = DEFAULT_CACHE, budget_s: float = 300.0):
    """Tune every class present in ``problems`` (largest work first) within a
    time budget, save the cache, and apply the choices."""
    tuner = Tuner(cache_path)
    t0 = time.time()
    classes = {}
    for pb in problems:
        k, m = pb.At.shape
        p = pb.B.shape[1]
        classes.setdefault(class_key(m, k, p, pb.hashes.log2b, d), (m, k, p, pb.hashes.log2b))
    order = sorted(classes.values(), key=lambda s: -(s[1] * (1 << s[3]) * s[3]))
    for (m, k, p, L) in order:
        if time.time() - t0 > budget_s:
            break
        tuner.tune_class(m, k, p, L, d)
    tuner.save()
    tuner.apply(problems, d, tune_missing=False)
    return tuner
