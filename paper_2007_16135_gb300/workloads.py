"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays them out; it holds none of the
TWED arithmetic, so both the CUDA path and the CPU oracle may use it.

Packed set layout (shared by the C ABI, the oracle and the tests):
``vals [sum(len), dim]`` row-major (the ``dim`` components of a point are
contiguous), ``ts [sum(len)]``, ``offs [nseries + 1]`` int64 with
``offs[0] = 0``; series ``s`` occupies rows ``offs[s]:offs[s+1]``.

Seeds follow one rule: ``PCG64(1000 * workload + stream)`` with stream 0 = set
A / queries, 1 = set B / database, 2 = pair sampling, 3 = training pairs.
Workload numbers:

1. one 1-D pair, n = m = 1000, random walks, t_i = i (nu = 1, lambda = 1).
2. one 3-D pair, n = m = 1e5 (or 1e6), random walks, times are cumulative
   Exp(1) gaps (nu = 0.001, lambda = 1).
3. 4096 series of dim 8, lengths U[64, 2048], three-sinusoid mixtures plus
   N(0, 0.1) noise, t_i = i (nu = 0.5, lambda = 0.5); all pairs.
4. 2048 x 2048 series of dim 64, lengths U[256, 1024], N(0,1) smoothed by a
   length-5 box filter, t_i = i (nu = 1, lambda = 1).
5. 1e5 database + 1000 query series of dim 4, lengths U[128, 512], random
   walks, t_i = i (nu = 1, lambda = 1).
6. stand-in with the shape of the paper's first validation set: 600 1-D
   series of 60 points in six pattern classes (level noise, cycles, rising
   and falling trends, upward and downward shifts), t_i = i.
7. stand-in with the shape of its second validation set: 10 1-D series of
   100,000 points (sinusoids whose periods drift, plus noise), t_i = i.
8. symbol sequences for the LCS program: 4096 sequences of i.i.d. uniform
   symbols over an alphabet of 4, lengths U[64, 2048] (the lengths of 3).
9. stand-in with the shape of the paper's third validation set (handwritten
   digit images): 28 x 28 images of one random cubic Bezier pen stroke each,
   read row by row as 28 points in R^28, t_i = i (nu = 1, lambda = 1).

All use p = 2.  The paper's own timing runs used random series of power-of-two
lengths (section "Basic Methodology and Results"); its UCI and MNIST data are
not available here and only their shapes are imitated.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

PARAMS = {
    1: dict(nu=1.0, lam=1.0, p=2),
    2: dict(nu=0.001, lam=1.0, p=2),
    3: dict(nu=0.5, lam=0.5, p=2),
    4: dict(nu=1.0, lam=1.0, p=2),
    5: dict(nu=1.0, lam=1.0, p=2),
    6: dict(nu=1.0, lam=1.0, p=2),
    7: dict(nu=1.0, lam=1.0, p=2),
}


def rng_for(workload: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(1000 * workload + stream))


@dataclass
class SeriesSet:
    vals: np.ndarray  # [sum_len, dim]
    ts: np.ndarray  # [sum_len]
    offs: np.ndarray  # [n + 1] int64

    @property
    def n(self) -> int:
        return int(self.offs.shape[0] - 1)

    @property
    def dim(self) -> int:
        return int(self.vals.shape[1])

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offs)

    def series(self, s: int):
        lo, hi = int(self.offs[s]), int(self.offs[s + 1])
        return self.vals[lo:hi], self.ts[lo:hi]

    def astype(self, dtype) -> "SeriesSet":
        return SeriesSet(np.ascontiguousarray(self.vals, dtype=dtype),
                         np.ascontiguousarray(self.ts, dtype=dtype), self.offs.copy())

    def subset(self, idx) -> "SeriesSet":
        return pack([self.series(int(i)) for i in idx], dtype=self.vals.dtype)

    def as_tuple(self):
        return self.vals, self.ts, self.offs


def pack(series, dtype=np.float64) -> SeriesSet:
    """Pack a list of ``(vals [len, dim], ts [len])`` into one set."""
    lens = [len(t) for _, t in series]
    offs = np.zeros(len(series) + 1, dtype=np.int64)
    offs[1:] = np.cumsum(lens)
    dim = np.asarray(series[0][0]).reshape(lens[0], -1).shape[1]
    vals = np.empty((int(offs[-1]), dim), dtype=dtype)
    ts = np.empty(int(offs[-1]), dtype=dtype)
    for s, (v, t) in enumerate(series):
        vals[offs[s]:offs[s + 1]] = np.asarray(v).reshape(lens[s], dim)
        ts[offs[s]:offs[s + 1]] = t
    return SeriesSet(vals, ts, offs)


def random_walk(rng: np.random.Generator, n: int, dim: int) -> np.ndarray:
    """x_i = sum_{k<=i} e_k, e_k ~ N(0, 1) per component, x_0 = 0."""
    return np.cumsum(rng.standard_normal((n, dim)), axis=0)


def unit_times(n: int) -> np.ndarray:
    return np.arange(1, n + 1, dtype=np.float64)


def exp_gap_times(rng: np.random.Generator, n: int) -> np.ndarray:
    """t_1 = g_1, t_i = t_{i-1} + g_i with g ~ Exp(1)."""
    return np.cumsum(rng.exponential(1.0, n))


def pair_w1(n: int = 1000, m: int = 1000):
    """Workload 1: one 1-D random-walk pair with unit time steps."""
    ra, rb = rng_for(1, 0), rng_for(1, 1)
    return (random_walk(ra, n, 1), unit_times(n), random_walk(rb, m, 1), unit_times(m))


def pair_w2(n: int = 100_000, m: int | None = None):
    """Workload 2: one 3-D random-walk pair, cumulative Exp(1) time gaps."""
    m = n if m is None else m
    ra, rb = rng_for(2, 0), rng_for(2, 1)
    a = random_walk(ra, n, 3)
    ta = exp_gap_times(ra, n)
    b = random_walk(rb, m, 3)
    tb = exp_gap_times(rb, m)
    return a, ta, b, tb


def _lengths(rng, nseries, lo, hi):
    return rng.integers(lo, hi + 1, size=nseries)


def set_w3(nseries: int = 4096, len_lo: int = 64, len_hi: int = 2048, dim: int = 8,
           stream: int = 0) -> SeriesSet:
    """Workload 3: sinusoid mixtures (3 frequencies in [0.01, 0.2] cycles per
    sample, amplitudes U[0.5, 2], phases U[0, 2 pi)) plus N(0, 0.1) noise."""
    rng = rng_for(3, stream)
    lens = _lengths(rng, nseries, len_lo, len_hi)
    out = []
    for n in lens:
        i = np.arange(1, n + 1, dtype=np.float64)[:, None, None]  # [n,1,1]
        f = rng.uniform(0.01, 0.2, size=(1, 3, dim))
        amp = rng.uniform(0.5, 2.0, size=(1, 3, dim))
        ph = rng.uniform(0.0, 2.0 * np.pi, size=(1, 3, dim))
        v = (amp * np.sin(2.0 * np.pi * f * i + ph)).sum(axis=1)
        v = v + rng.normal(0.0, 0.1, size=(n, dim))
        out.append((v, unit_times(n)))
    return pack(out)


def set_w4(nseries: int = 2048, len_lo: int = 256, len_hi: int = 1024, dim: int = 64,
           stream: int = 0) -> SeriesSet:
    """Workload 4: N(0,1) drawn at len+4 points, then a length-5 moving mean
    ('valid'), so each component has variance 1/5."""
    rng = rng_for(4, stream)
    lens = _lengths(rng, nseries, len_lo, len_hi)
    out = []
    for n in lens:
        raw = rng.standard_normal((n + 4, dim))
        c = np.cumsum(np.vstack([np.zeros((1, dim)), raw]), axis=0)
        v = (c[5:] - c[:-5]) / 5.0
        out.append((v, unit_times(n)))
    return pack(out)


def seqs_w8(nseries: int = 4096, len_lo: int = 64, len_hi: int = 2048, alphabet: int = 4,
            stream: int = 0) -> list:
    """Workload 8: i.i.d. uniform int32 symbols in [0, alphabet)."""
    rng = rng_for(8, stream)
    lens = _lengths(rng, nseries, len_lo, len_hi)
    return [rng.integers(0, alphabet, int(n)).astype(np.int32) for n in lens]


def set_w5(nseries: int = 100_000, len_lo: int = 128, len_hi: int = 512, dim: int = 4,
           stream: int = 1) -> SeriesSet:
    """Workload 5: random walks; stream 1 = database, stream 0 = queries."""
    rng = rng_for(5, stream)
    lens = _lengths(rng, nseries, len_lo, len_hi)
    out = [(random_walk(rng, int(n), dim), unit_times(int(n))) for n in lens]
    return pack(out)


def sample_upper_pairs(nseries: int, k: int, workload: int) -> np.ndarray:
    """k distinct (i < j) pairs drawn uniformly from the upper triangle."""
    rng = rng_for(workload, 2)
    total = nseries * (nseries - 1) // 2
    flat = rng.choice(total, size=min(k, total), replace=False)
    # invert the row-major upper-triangle enumeration
    i = (2 * nseries - 1 - np.sqrt((2 * nseries - 1) ** 2 - 8 * flat.astype(np.float64))) // 2
    i = i.astype(np.int64)
    row_start = i * (2 * nseries - i - 1) // 2
    # guard the floating-point inverse at row boundaries
    over = flat < row_start
    i[over] -= 1
    row_start = i * (2 * nseries - i - 1) // 2
    under = flat >= row_start + (nseries - 1 - i)
    i[under] += 1
    row_start = i * (2 * nseries - i - 1) // 2
    j = flat - row_start + i + 1
    return np.stack([i, j], axis=1).astype(np.int64)


def sample_block_pairs(na: int, nb: int, k: int, workload: int) -> np.ndarray:
    """k distinct (i, j) pairs drawn uniformly from an na x nb block."""
    rng = rng_for(workload, 2)
    flat = rng.choice(na * nb, size=min(k, na * nb), replace=False)
    return np.stack([flat // nb, flat % nb], axis=1).astype(np.int64)


def set_u1(nseries: int = 600, length: int = 60, stream: int = 0) -> SeriesSet:
    """Workload 6: six classes of 1-D pattern series, nseries / 6 each.

    Every series is a level 30 plus N(0, 2) noise; class 1 adds a sine of
    amplitude U[10, 15] and period U[10, 15]; classes 2 and 3 add a trend of
    slope +-U[0.2, 0.5]; classes 4 and 5 add a step of height +-U[7.5, 20]
    at a point U[length/3, 2 length/3].  Class 0 is the noise alone."""
    rng = rng_for(6, stream)
    out = []
    t = np.arange(1, length + 1, dtype=np.float64)
    for s_ in range(nseries):
        c = s_ % 6
        y = 30.0 + rng.normal(0.0, 2.0, length)
        if c == 1:
            y += rng.uniform(10, 15) * np.sin(2 * np.pi * t / rng.uniform(10, 15))
        elif c in (2, 3):
            y += (1 if c == 2 else -1) * rng.uniform(0.2, 0.5) * t
        elif c in (4, 5):
            t0 = rng.integers(length // 3, 2 * length // 3 + 1)
            y += (1 if c == 4 else -1) * rng.uniform(7.5, 20) * (t >= t0)
        out.append((y[:, None], t.copy()))
    return pack(out)


def set_u3(nseries: int = 60_000, stream: int = 0, samples: int = 48, pen: float = 1.0) -> SeriesSet:
    """Workload 9: one pen stroke per 28 x 28 image: a cubic Bezier curve with
    four control points U[4, 24]^2, sampled at `samples` points, each drawn as
    a Gaussian blob of width `pen` pixels; intensities clipped to [0, 1].
    Row r of the image is point r + 1 of the series (28 points in R^28)."""
    rng = rng_for(9, stream)
    ctrl = rng.uniform(4.0, 24.0, size=(nseries, 4, 2))
    u = np.linspace(0.0, 1.0, samples)
    basis = np.stack([(1 - u) ** 3, 3 * u * (1 - u) ** 2, 3 * u ** 2 * (1 - u), u ** 3], axis=1)  # [S, 4]
    pts = np.einsum("sk,nkd->nsd", basis, ctrl)  # [n, S, 2] (row, column)
    grid = np.arange(28, dtype=np.float64)
    out = np.empty((nseries, 28, 28), dtype=np.float64)
    for c0 in range(0, nseries, 4096):
        p = pts[c0:c0 + 4096]
        gr = np.exp(-0.5 * ((grid[None, None, :] - p[:, :, 0:1]) / pen) ** 2)  # [n, S, 28] rows
        gc = np.exp(-0.5 * ((grid[None, None, :] - p[:, :, 1:2]) / pen) ** 2)  # [n, S, 28] columns
        out[c0:c0 + 4096] = np.minimum(np.matmul(gr.transpose(0, 2, 1), gc), 1.0)
    ts = np.tile(unit_times(28), nseries)
    offs = np.arange(nseries + 1, dtype=np.int64) * 28
    return SeriesSet(out.reshape(nseries * 28, 28), ts, offs)


def set_u2(nseries: int = 10, length: int = 100_000, stream: int = 0) -> SeriesSet:
    """Workload 7: long 1-D pseudo-periodic series: sum over r = 1..3 of
    A_r sin(phi_r(i)) with A_r ~ U[0.5, 1.5], an instantaneous period drifting
    linearly from U[40, 200] to U[40, 200] samples, plus N(0, 0.05)."""
    rng = rng_for(7, stream)
    out = []
    i = np.arange(length, dtype=np.float64)
    for _ in range(nseries):
        y = rng.normal(0.0, 0.05, length)
        for _r in range(3):
            p0, p1 = rng.uniform(40, 200, 2)
            period = p0 + (p1 - p0) * i / max(length - 1, 1)
            phase = 2 * np.pi * np.cumsum(1.0 / period) + rng.uniform(0, 2 * np.pi)
            y += rng.uniform(0.5, 1.5) * np.sin(phase)
        out.append((y[:, None], i + 1.0))
    return pack(out)
