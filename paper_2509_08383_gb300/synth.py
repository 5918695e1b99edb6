"""Seeded synthetic inputs shaped like LLM next-token logits.

This module holds no CutMax or CKKS arithmetic; it only draws inputs.  The
paper measures on logits of Mistral-7B, Qwen2.5-0.5B and GPT-2 over arXiv
abstracts (Sect. 4); those models and that dataset are not available, so these
seeded generators stand in for them with the stated shapes and distributions.
"""
import numpy as np


def _raise_top(x, gap):
    i = int(np.argmax(x))
    s = np.sort(x)
    x[i] = s[-2] + gap
    return x


def logits_gaussian(seed, n=1024, sd=2.0, gap=0.5):
    """n entries from N(0, sd^2); the top entry is set to top-2 + gap."""
    rng = np.random.default_rng([0xC0FFEE, int(seed)])
    x = rng.normal(0.0, sd, size=n)
    return _raise_top(x, gap)


def logits_heavy_tail(seed, n=32000, sd=3.0, heavy=50, exp_scale=1.5, gap=0.2):
    """N(0, sd^2) base; `heavy` distinct indices get + Exp(scale); top-1 = top-2 + gap."""
    rng = np.random.default_rng([0xBEEF, int(seed)])
    x = rng.normal(0.0, sd, size=n)
    idx = rng.choice(n, size=heavy, replace=False)
    x[idx] += rng.exponential(exp_scale, size=heavy)
    return _raise_top(x, gap)


def uniforms(seed, n):
    """U(0,1) draws in the open interval, for nucleus cut-noise."""
    rng = np.random.default_rng([0x5A5A, int(seed)])
    u = rng.random(n)
    return np.clip(u, 2.0 ** -53, 1.0 - 2.0 ** -53)


class HeavyTail:
    """Picklable generator of the full-vocabulary workload: logits_heavy_tail
    with the top-1 gap cycling through `gaps` by seed."""

    def __init__(self, n=32000, gaps=(0.05, 0.2, 1.0), heavy=50):
        self.n, self.gaps, self.heavy = int(n), tuple(gaps), int(heavy)

    def __call__(self, seed):
        return logits_heavy_tail(seed, n=self.n, heavy=self.heavy, gap=self.gaps[int(seed) % len(self.gaps)])


class Gaussian:
    """Picklable generator: logits_gaussian with fixed n, sd and gap."""

    def __init__(self, n=1024, sd=2.0, gap=0.5):
        self.n, self.sd, self.gap = int(n), float(sd), float(gap)

    def __call__(self, seed):
        return logits_gaussian(seed, n=self.n, sd=self.sd, gap=self.gap)
