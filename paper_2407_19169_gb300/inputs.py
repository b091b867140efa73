"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only draws numbers. Every random choice goes
through SplitMix64 (Steele, Lea & Flood 2014), so a seed fixes the input on every machine.

Workloads (the synthetic stand-ins for the paper's test problems, Section 3):
  burgers1d   u0 = 0.5 + sin(pi x) on [0, 2], periodic, 200 cells, P2, to t = 1.5
  euler1d     N = 2^16, P3, seeded Riemann problem on [0, 1] (rho, p in [0.1, 5], |u| < 2), outflow
  euler2d     2048 x 2048 on [0, 1]^2, Q2, seeded four-quadrant Riemann data (rho, p in [0.1, 2],
              |u|, |v| < 1), outflow; the quadrant split sits on a cell face
  vortex2d    isentropic vortex of Example 3.4(a) on [0, 10] x [-5, 5], periodic
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64: state += 0x9E3779B97F4A7C15, then the two xor-shift-multiply mixing rounds."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float, hi: float) -> float:
        # 53 random bits -> [0, 1)
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def block_u64(self, n: int) -> np.ndarray:
        """The next n outputs at once: output k is the mix of state + k * gamma (counter form)."""
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + k * np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * 0x9E3779B97F4A7C15) & MASK64
        return z

    def array(self, n: int, lo: float, hi: float) -> np.ndarray:
        u = (self.block_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
        return lo + (hi - lo) * u


def riemann1d_params(seed: int, x_split: float = 0.5):
    """Left/right primitive states (rho, u, p), drawn in the order rho, u, p, left then right."""
    g = SplitMix64(seed)
    out = []
    for _ in range(2):
        rho = g.uniform(0.1, 5.0)
        u = g.uniform(-2.0, 2.0)
        p = g.uniform(0.1, 5.0)
        out += [rho, u, p]
    return out + [x_split]


def quadrant_params(seed: int, x_split: float = 0.5, y_split: float = 0.5):
    """(rho, u, v, p) for the quadrants Q1 (x>xs, y>ys), Q2, Q3, Q4, then the split point."""
    g = SplitMix64(seed)
    out = []
    for _ in range(4):
        rho = g.uniform(0.1, 2.0)
        u = g.uniform(-1.0, 1.0)
        v = g.uniform(-1.0, 1.0)
        p = g.uniform(0.1, 2.0)
        out += [rho, u, v, p]
    return out + [x_split, y_split]


def random_modal_state(shape, seed: int, avg_ranges, high_scale: float = 0.05, decay: float = 0.5):
    """Modal coefficients u[v][m][cell]: cell averages uniform in avg_ranges[v], higher modes uniform
    in +-high_scale * decay^(m-1) * (range width). Rough from cell to cell, so the filter is active."""
    nv, nm, nc = shape
    g = SplitMix64(seed)
    u = np.zeros(shape)
    for v in range(nv):
        lo, hi = avg_ranges[v]
        u[v, 0] = g.array(nc, lo, hi)
        for m in range(1, nm):
            amp = high_scale * decay ** (m - 1) * (hi - lo)
            u[v, m] = g.array(nc, -amp, amp)
    return u


random_modal_state_fast = random_modal_state  # vectorised draws: the same stream, any size

# averages that keep every Euler state physical: rho in [1, 2], |m| <= 0.5, E in [4, 6]
EULER1D_AVG = [(1.0, 2.0), (-0.5, 0.5), (4.0, 6.0)]
EULER2D_AVG = [(1.0, 2.0), (-0.5, 0.5), (-0.5, 0.5), (4.0, 6.0)]

WORKLOADS = {
    "burgers1d": dict(dim=1, nx=200, x0=0.0, x1=2.0, k=2, eq="burgers", bc="periodic", T=1.5,
                      ic=("sine", [0.5, 1.0, np.pi, 0.0])),
    "euler1d": dict(dim=1, nx=1 << 16, x0=0.0, x1=1.0, k=3, eq="euler", bc="outflow", T=0.2,
                    ic=("riemann1d", None)),
    "euler2d": dict(dim=2, nx=2048, ny=2048, x0=0.0, x1=1.0, y0=0.0, y1=1.0, k=2, eq="euler",
                    bc="outflow", T=0.25, ic=("quadrant2d", None)),
    "vortex2d": dict(dim=2, x0=0.0, x1=10.0, y0=-5.0, y1=5.0, k=2, eq="euler", bc="periodic", T=10.0,
                     ic=("vortex2d", [5.0, 0.0, 5.0, 0.0])),
}


def batched_specs(n=512, seed=4, riemann_seeds=(1, 2, 3, 4), quadrant_seeds=(1, 4, 7, 8)):
    """The batched workload: n uneven instances. Per instance: 1D or 2D with probability 1/2; 1D
    cells log-uniform in [1e3, 1e6], 2D side log-uniform in [64, 1024] (both rounded to even, so a
    Riemann split at 1/2 lies on a face); degree uniform in {1, 2, 3}; seeded Riemann data or the
    smooth problem of that dimension (1D entropy wave, 2D vortex) with probability 1/2."""
    g = SplitMix64(seed)
    out = []
    for i in range(n):
        dim = 1 if g.uniform(0, 1) < 0.5 else 2
        if dim == 1:
            size = 2 * int(round(10 ** g.uniform(3.0, 6.0) / 2))
        else:
            size = 2 * int(round(2 ** g.uniform(6.0, 10.0) / 2))
        k = 1 + min(int(g.uniform(0, 3)), 2)
        riemann = g.uniform(0, 1) < 0.5
        if dim == 1:
            kind, s = ("riemann1d", riemann_seeds[i % len(riemann_seeds)]) if riemann else ("entropy1d", 0)
        else:
            kind, s = ("quadrant2d", quadrant_seeds[i % len(quadrant_seeds)]) if riemann else ("vortex2d", 0)
        out.append(dict(dim=dim, n=size, k=k, kind=kind, seed=s))
    return out
