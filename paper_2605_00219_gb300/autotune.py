"""Autotuner for the step's launch shape: tile size x raster-backward
implementation x threads per tile, chosen by Thompson sampling over measured
step latencies (the scheduler the paper uses to pick between its two
rasterization-backward implementations, Sec. 4.2).

A candidate is (tile, bwd_impl, threads_per_tile).  The pixel-parallel
backward (impl 0) runs with one, two or (16-wide tiles) four pixels per
thread; the other two backward implementations, and the raster forward, with
one thread per pixel.

Each candidate keeps a Normal-Inverse-Gamma posterior over its latency.  A
round samples one latency per candidate from its posterior, runs the
candidate with the smallest sample once, and updates that posterior with the
measured latency; fast candidates are tried more often, slow ones rarely.
After the budget the candidate with the lowest posterior mean wins.  The
tuner runs before graph capture; the chosen shape is then fixed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TILES = [(8, 8), (16, 16), (16, 32)]
BWD_IMPLS = [0, 1, 2]


def pixels_per_thread_options(tile) -> list:
    """Pixels per raster thread a tile shape supports (warps of 8 x 4, 8 x 8
    or 8 x 16 pixels; an 8x8 tile needs at least one full warp)."""
    return [1, 2] if tile[0] == 8 else [1, 2, 4]


def default_candidates(tiles=TILES, impls=BWD_IMPLS) -> list:
    """(tile, bwd_impl, threads_per_tile) for every supported combination."""
    out = []
    for t in tiles:
        for b in impls:
            ppts = pixels_per_thread_options(t) if b == 0 else [1]
            out += [(tuple(t), b, t[0] * t[1] // k) for k in ppts]
    return out


def describe(c) -> str:
    return f"{c[0][0]}x{c[0][1]}/impl{c[1]}/tpt{c[2]}"


@dataclass
class NIGPosterior:
    """Normal-Inverse-Gamma posterior of an unknown mean and variance."""
    mu: float = 0.0
    kappa: float = 0.0
    alpha: float = 1.0
    beta: float = 1.0
    n: int = 0
    xs: list = field(default_factory=list)

    def update(self, x: float):
        self.xs.append(float(x))
        if self.n == 0:
            # first observation fixes the location; scale prior from it
            self.mu, self.kappa, self.alpha, self.beta = float(x), 1.0, 1.0, (0.1 * abs(x)) ** 2 + 1e-12
        else:
            k1 = self.kappa + 1.0
            mu1 = (self.kappa * self.mu + x) / k1
            self.beta += 0.5 * self.kappa * (x - self.mu) ** 2 / k1
            self.alpha += 0.5
            self.mu, self.kappa = mu1, k1
        self.n += 1

    def sample(self, rng: np.random.Generator) -> float:
        if self.n == 0:
            return -math.inf          # untried candidates go first
        var = self.beta / rng.gamma(self.alpha)
        return rng.normal(self.mu, math.sqrt(var / self.kappa))

    @property
    def mean(self) -> float:
        return self.mu if self.n else math.inf


class ThompsonTuner:
    def __init__(self, candidates, seed: int = 0):
        self.candidates = list(candidates)
        self.post = [NIGPosterior() for _ in self.candidates]
        self.rng = np.random.default_rng(seed)
        self.pulls = [0] * len(self.candidates)

    def choose(self) -> int:
        draws = [p.sample(self.rng) for p in self.post]
        return int(np.argmin(draws))

    def observe(self, i: int, latency: float):
        self.post[i].update(latency)
        self.pulls[i] += 1

    def run(self, measure, rounds: int):
        """measure(candidate) -> latency; returns the best candidate."""
        for _ in range(rounds):
            i = self.choose()
            self.observe(i, measure(self.candidates[i]))
        return self.best()

    def best(self):
        return self.candidates[int(np.argmin([p.mean for p in self.post]))]


def tune_trainer(scenes, cameras, rounds: int = 24, steps_per_pull: int = 2, lr=None, sh_bf16=False,
                 mom_bf16=False, target=None, capacity: int = 0, candidates=None, seed: int = 0):
    """Pick (tile, bwd_impl, threads_per_tile) for a workload by Thompson
    sampling over eager training steps (CUDA events on the current stream).
    `scenes` are SceneBuffers shared by all candidates.  Returns (best,
    tuner, trainers)."""
    import torch
    from .step import DEFAULT_LR, Trainer

    cands = candidates or default_candidates()
    trainers = {}

    def get(c):
        if c not in trainers:
            tr = Trainer(scenes, cameras, capacity=capacity, tile=c[0], bwd_impl=c[1], lr=lr or DEFAULT_LR,
                         sh_bf16=sh_bf16, mom_bf16=mom_bf16, threads_per_tile=c[2])
            if target is not None:
                tr.target.copy_(target)
            tr.step(0)               # first call sets kernel attributes
            trainers[c] = tr
        return trainers[c]

    def measure(c):
        tr = get(c)
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps_per_pull):
            tr.step(0)
        e1.record(st)
        e1.synchronize()
        return e0.elapsed_time(e1) / steps_per_pull

    tuner = ThompsonTuner(cands, seed)
    best = tuner.run(measure, rounds)
    return best, tuner, trainers
