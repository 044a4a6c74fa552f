"""Seeded synthetic workload definitions shared by the oracle, the tests and bench.py.

This module holds problem *parameters* only (grid sizes, KL/PCE settings, sources,
time steps) and a counter-based random generator for the batched workload and for
Monte Carlo samples.  It contains none of the solver's arithmetic: no KL, no PCE,
no assembly, no solves.  Both the CUDA path and the oracle receive these plain
parameters and compute everything else independently.

Readings of the paper used for the parameters (Sec. 6 "Numerical Results"):
  * CFL number 0.65 for the time step when a config gives none (dt = 0.65 h / c_ref,
    c_ref = 1, the median wave speed of the log-normal field with g0 = 0).
  * Rayleigh damping alpha0 = 0.5445, alpha1 = 0.0174 (values printed in Sec. 6.2
    and the Rayleigh appendix).
  * Newmark gamma = 1/2, zeta = 1/4 (Sec. 2).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

ALPHA0 = 0.5445  # Rayleigh mass coefficient printed in Sec. 6.2
ALPHA1 = 0.0174  # Rayleigh stiffness coefficient printed in Sec. 6.2
CFL = 0.65       # Courant number used for every experiment (Sec. 6)

SOURCE_NONE = 0
SOURCE_PULSE = 1   # initial Gaussian pulse u0 = amp * exp(-r^2 / width^2)
SOURCE_RICKER = 2  # point source r(t) delta(x - x_s), Ricker wavelet of peak freq


@dataclasses.dataclass(frozen=True)
class Source:
    kind: int = SOURCE_NONE
    x0: float = 0.5
    y0: float = 0.5
    width: float = 0.05
    freq: float = 10.0
    amp: float = 1.0


@dataclasses.dataclass(frozen=True)
class Problem:
    """One stochastic-Galerkin wave problem on the unit square.

    N        cells per side of the structured grid (each cell split along (i,j)->(i+1,j+1))
    s        subdomains per side (s x s partition, N % s == 0)
    M        number of KL random variables
    p        output PCE total order; p_in the input (coefficient) order
    sigma    standard deviation of the Gaussian field g; bx, by correlation lengths
    g0       mean of g (so c^2 = exp(g) has median exp(g0))
    dt       time step; steps the number of steps of the run
    tol      relative PCG residual ||r||_2 / ||G_Gamma||_2 on the interface
    """
    name: str
    N: int
    s: int
    M: int
    p: int
    p_in: int
    sigma: float
    bx: float
    by: float
    g0: float
    dt: float
    steps: int
    tol: float
    source: Source
    alpha0: float = ALPHA0
    alpha1: float = ALPHA1
    max_iter: int = 500

    @property
    def h(self) -> float:
        return 1.0 / self.N

    @property
    def P(self) -> int:
        return math.comb(self.M + self.p, self.p)

    @property
    def P_in(self) -> int:
        return math.comb(self.M + self.p_in, self.p_in)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def cfl_dt(N: int) -> float:
    return CFL / N


def config(name: str) -> Problem:
    """The five workloads of the benchmark plus small test problems."""
    if name == "pulse32":  # 32x32 grid, 2x2 subdomains, M=2, p=2, 50 steps, tol 1e-10
        return Problem("pulse32", N=32, s=2, M=2, p=2, p_in=2, sigma=0.3, bx=0.5, by=0.5,
                       g0=0.0, dt=1e-3, steps=50, tol=1e-10,
                       source=Source(SOURCE_PULSE, 0.5, 0.5, 0.05, 0.0, 1.0))
    if name == "ricker128":  # 128x128 grid, 4x4 subdomains, M=3, p=3 (P=20), 200 steps
        return Problem("ricker128", N=128, s=4, M=3, p=3, p_in=3, sigma=0.3, bx=0.3, by=0.3,
                       g0=0.0, dt=cfl_dt(128), steps=200, tol=1e-8,
                       source=Source(SOURCE_RICKER, 0.3, 0.5, 0.0, 10.0, 1.0))
    if name == "ricker512":  # 512x512 grid, 8x8 subdomains, M=4, p=3 (P=35), 500 steps
        return Problem("ricker512", N=512, s=8, M=4, p=3, p_in=3, sigma=0.4, bx=0.2, by=0.2,
                       g0=0.0, dt=cfl_dt(512), steps=500, tol=1e-8,
                       source=Source(SOURCE_RICKER, 0.3, 0.5, 0.0, 10.0, 1.0))
    if name == "ricker1024":  # 1024x1024 grid, 16x16 subdomains, M=5, p=2 (P=21), 1000 steps
        return Problem("ricker1024", N=1024, s=16, M=5, p=2, p_in=2, sigma=0.3, bx=0.1, by=0.1,
                       g0=0.0, dt=cfl_dt(1024), steps=1000, tol=1e-8,
                       source=Source(SOURCE_RICKER, 0.3, 0.5, 0.0, 10.0, 1.0))
    if name == "ricker1024q":  # the 1024^2 workload's subdomains and PCE on a quarter of its grid
        # (512x512, 8x8 subdomains of 65x65 nodes, M=5, p=2): kernel profiles of a few GB
        return dataclasses.replace(config("ricker1024"), name="ricker1024q", N=512, s=8, dt=cfl_dt(512))
    if name == "tiny":  # smallest useful DD problem for exhaustive checks
        return Problem("tiny", N=8, s=2, M=1, p=2, p_in=2, sigma=0.3, bx=0.5, by=0.5,
                       g0=0.0, dt=0.02, steps=5, tol=1e-12,
                       source=Source(SOURCE_PULSE, 0.5, 0.5, 0.2, 0.0, 1.0))
    if name == "small":  # several subdomains, corners shared by four subdomains
        return Problem("small", N=24, s=3, M=2, p=2, p_in=2, sigma=0.3, bx=0.5, by=0.5,
                       g0=0.0, dt=cfl_dt(24), steps=10, tol=1e-12,
                       source=Source(SOURCE_RICKER, 0.3, 0.5, 0.0, 10.0, 1.0))
    raise KeyError(name)


# ---------------------------------------------------------------------------
# Counter-based generator (SplitMix64, Steele/Lea/Flood 2014) and Box-Muller.
# ---------------------------------------------------------------------------
_MASK = (1 << 64) - 1


def splitmix64(state: int):
    """One SplitMix64 step: returns (new_state, 64-bit output)."""
    state = (state + 0x9E3779B97F4A7C15) & _MASK
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return state, z ^ (z >> 31)


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state, z = splitmix64(self.state)
        return z

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (inclusive), by scaling a uniform draw."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)

    def normal_pair(self):
        u1 = 1.0 - self.uniform()  # (0, 1]
        u2 = self.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        return r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2)


BATCH_SEED = 20251227


def batch_problems(n: int = 256, seed: int = BATCH_SEED, steps: int = 100) -> List[Problem]:
    """The batched workload: n independent problems of uneven size.

    Per instance, drawn in this order: s in {2,4,8}; N uniform over multiples of 8
    in [64, 256] that s divides into whole cells; M in {2,3,4}; p in {2,3};
    sigma ~ U[0.1, 0.5].  Correlation length 0.3, Ricker source at (0.3, 0.5),
    dt from CFL 0.65, FP32 subdomain solves in the optimised mode.
    """
    g = SplitMix64(seed)
    out = []
    for k in range(n):
        s = (2, 4, 8)[g.randint(0, 2)]
        Ns = [N for N in range(64, 257, 8) if N % s == 0]
        N = Ns[g.randint(0, len(Ns) - 1)]
        M = g.randint(2, 4)
        p = g.randint(2, 3)
        sigma = 0.1 + 0.4 * g.uniform()
        out.append(Problem(f"batch{k}", N=N, s=s, M=M, p=p, p_in=p, sigma=sigma, bx=0.3, by=0.3,
                           g0=0.0, dt=cfl_dt(N), steps=steps, tol=1e-8,
                           source=Source(SOURCE_RICKER, 0.3, 0.5, 0.0, 10.0, 1.0)))
    return out


def normal_samples(n: int, dim: int, seed: int = 0):
    """n x dim standard normal draws (list of lists) from SplitMix64 + Box-Muller."""
    g = SplitMix64(seed)
    out = []
    buf = []
    for _ in range(n):
        row = []
        for _ in range(dim):
            if not buf:
                buf.extend(g.normal_pair())
            row.append(buf.pop(0))
        out.append(row)
    return out


@dataclasses.dataclass(frozen=True)
class MeshConfig:
    """A workload on a seeded unstructured mesh of the unit square (sg_workloads.meshes): the Delaunay
    mesh parameters, the number of recursive-coordinate-bisection subdomains, and the SG problem
    (its N and s are unused; dt, KL, PCE, source, tolerance as for the structured configs)."""
    name: str
    n: int
    jitter: float
    seed: int
    nparts: int
    prob: Problem

    def build(self):
        """(xy, dirichlet flags, triangles, subdomain ids) of the mesh and partition."""
        from . import meshes
        xy, tri, boundary = meshes.delaunay_square(self.n, self.jitter, self.seed)
        return xy, boundary, tri, meshes.rcb_partition(xy, tri, self.nparts)


def mesh_config(name: str) -> MeshConfig:
    """Mesh workloads sized after the paper's unstructured experiments (Sec. 6): the mesh sizes are the
    paper's (its meshes are not available; seeded Delaunay meshes of the same vertex count stand in),
    the KL / PCE sizes those of the experiment quoted.  The paper spreads its subdomains over CPU cores
    (up to 720); on one GPU fewer, larger subdomains keep the coarse problem small, so the 37k-vertex
    mesh comes with a 64-subdomain partition and, separately, with the paper's 720.
      umesh_small   24 cells per side (625 vertices), 6 subdomains, M = 3, order 2 (test size).
      umesh13k      117^2 = 13689 vertices (paper: 13472), 32 subdomains, M = 7, order 3 (P = 120):
                    the strong-scaling problem (Sec. 6.3, 1.6 million unknowns), dt 6.5e-3.
      umesh37k      193^2 = 37249 vertices (paper: 37267), 64 subdomains, M = 3, order 3 (P = 20):
                    the smallest case of the scaling-with-random-variables study (Sec. 6.4), dt 3.9e-3.
      umesh37k_rv9  the same mesh and partition with M = 9, order 3 (P = 220, 8.19 million unknowns),
                    the largest case of that study.
      umesh37k_720  umesh37k on the paper's 720 subdomains (1284 corners: a dense coarse matrix of
                    25680^2 values, 5.3 GB, whose inverse takes minutes of host set-up).
      umesh_e1      40^2 = 1600 vertices (paper: 1563), deterministic medium (M = 0, P = 1), dt 0.01:
                    the preconditioner comparison of Sec. 6.1 (its subdomain counts vary; 4 here)."""
    ricker = Source(SOURCE_RICKER, 0.3, 0.5, 0.0, 10.0, 1.0)
    base = Problem(name=name, N=0, s=0, M=3, p=2, p_in=2, sigma=0.3, bx=0.3, by=0.3, g0=0.0, dt=0.02,
                   steps=20, tol=1e-8, source=ricker)
    rv3 = base.replace(M=3, p=3, p_in=3, dt=3.9e-3, steps=128)
    if name == "umesh_small":
        return MeshConfig(name, 24, 0.3, 11, 6, base)
    if name == "umesh13k":
        return MeshConfig(name, 116, 0.3, 13, 32, base.replace(M=7, p=3, p_in=3, dt=6.5e-3, steps=77))
    if name == "umesh37k":
        return MeshConfig(name, 192, 0.3, 37, 64, rv3)
    if name == "umesh37k_rv9":
        return MeshConfig(name, 192, 0.3, 37, 64, rv3.replace(M=9))
    if name == "umesh37k_720":
        return MeshConfig(name, 192, 0.3, 37, 720, rv3)
    if name == "umesh_e1":
        return MeshConfig(name, 39, 0.3, 61, 4, base.replace(M=0, p=0, p_in=0, sigma=0.0, dt=0.01, steps=50))
    raise KeyError(name)


def uniform_samples(n: int, seed: int = 0) -> List[float]:
    """n uniform draws in [0, 1) from SplitMix64 (mesh jitter of the unstructured meshes)."""
    g = SplitMix64(seed)
    return [g.uniform() for _ in range(n)]
