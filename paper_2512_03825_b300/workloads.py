"""Seeded synthetic workloads: the only module both the CUDA path and the CPU oracle are fed
from. It holds problem descriptions (lattice size, temperature ladders, seeds, request
streams) and none of the method's arithmetic.

The paper (arXiv 2512.03825, Sec. 4.2) times a 300 x 300 lattice with J = 1, B = 0 and up to
1500 replicas; it publishes no dataset. The workloads below are synthetic stand-ins of the
same kind: periodic square lattices, uniform random +/-1 initial spins drawn from the seed,
inverse-temperature ladders spanning the critical point beta_c = ln(1 + sqrt 2) / 2.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np


@dataclasses.dataclass(frozen=True)
class Problem:
    """One parallel-tempering problem: lattice L x L, R temperatures, coupling J, field h,
    seed, and the run that is asked of it (sweeps, exchange every m sweeps; 0 = none)."""
    L: int
    betas: tuple
    J: float = 1.0
    h: float = 0.0
    seed: int = 0
    sweeps: int = 0
    every: int = 0

    @property
    def R(self) -> int:
        return len(self.betas)

    @property
    def attempts(self) -> int:
        """Spin-flip attempts of the whole run: L^2 sites x R replicas x sweeps."""
        return self.L * self.L * self.R * self.sweeps

    def with_run(self, sweeps: int, every: Optional[int] = None) -> "Problem":
        return dataclasses.replace(self, sweeps=int(sweeps),
                                   every=self.every if every is None else int(every))


def geometric_ladder(b0: float, b1: float, R: int) -> tuple:
    """beta_k = b0 (b1/b0)^(k/(R-1))."""
    if R == 1:
        return (float(b0),)
    return tuple(float(b0 * (b1 / b0) ** (k / (R - 1))) for k in range(R))


def linear_ladder(b0: float, b1: float, R: int) -> tuple:
    """beta_k = b0 + (b1 - b0) k/(R-1)."""
    if R == 1:
        return (float(b0),)
    return tuple(float(b0 + (b1 - b0) * k / (R - 1)) for k in range(R))


def paper_ladder(R: int) -> tuple:
    """The paper's temperature assignment T_i = 1 + 3 i / |R| (Sec. 3), as betas."""
    return tuple(1.0 / (1.0 + 3.0 * i / R) for i in range(R))


# The three single-problem workloads (seeds 0x5EED0000 + index).
SINGLE = {
    "L16_R8": Problem(L=16, betas=geometric_ladder(0.20, 0.60, 8), seed=0x5EED0001,
                      sweeps=1000, every=10),
    "L128_R32": Problem(L=128, betas=linear_ladder(0.30, 0.55, 32), seed=0x5EED0002,
                        sweeps=10_000, every=1),
    "L1024_R64": Problem(L=1024, betas=linear_ladder(0.35, 0.50, 64), seed=0x5EED0003,
                         sweeps=1000, every=5),
}


def paper_problem(R: int = 1500, sweeps: int = 300_000, every: int = 100) -> Problem:
    """The paper's own workload (Sec. 4): a 300 x 300 lattice, J = 1, B = 0, temperatures
    T_i = 1 + 3 i / |R| for up to 1500 replicas, 300,000 iterations per replica, swaps every
    0 / 100 / 1k / 10k iterations. Read with one iteration = one sweep of the lattice (our
    update unit), the run is 300,000 sweeps with a swap iteration every 100 sweeps. Seed
    0x5EED0006."""
    return Problem(L=300, betas=paper_ladder(R), seed=0x5EED0006, sweeps=sweeps, every=every)


BATCH_SIZES = (32, 48, 64, 96, 128, 256)


def batched_problems(n: int = 256, sweeps: int = 2000, every: int = 1,
                     draw_seed: int = 2025) -> List[Problem]:
    """The batched workload: n independent problems, L uniform over {32,48,64,96,128,256},
    R uniform in 8..48, betas linear 0.30 -> 0.60, J = 1, h = 0; problem j has seed
    0x5EED1000 + j. Sizes are drawn from numpy's PCG64(draw_seed)."""
    rng = np.random.Generator(np.random.PCG64(draw_seed))
    Ls = rng.choice(np.array(BATCH_SIZES), size=n)
    Rs = rng.integers(8, 49, size=n)
    return [Problem(L=int(Ls[j]), betas=linear_ladder(0.30, 0.60, int(Rs[j])),
                    seed=0x5EED1000 + j, sweeps=sweeps, every=every) for j in range(n)]


@dataclasses.dataclass(frozen=True)
class Request:
    """One serving request: a problem and its arrival time (seconds from stream start)."""
    rid: int
    arrival: float
    problem: Problem


def serving_requests(n: int = 2000, rate_per_s: float = 10.0, draw_seed: int = 2026,
                     L_max: int = 512, sweeps_exp=(2.0, 4.0)) -> List[Request]:
    """The serving workload: Poisson arrivals at ``rate_per_s``; L uniform in [16, L_max]
    rounded to a multiple of 32 (at least 32); R uniform in 8..64; sweeps log-uniform over
    10^2..10^4; J = 1; h uniform over {0, 0.1}; betas linear 0.30 -> 0.60; exchange every
    sweep; request j has seed 0x5EED2000 + j."""
    rng = np.random.Generator(np.random.PCG64(draw_seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=n)
    t = np.cumsum(gaps) - gaps[0]
    Lraw = rng.uniform(16, L_max, size=n)
    Ls = np.maximum(32, 32 * np.round(Lraw / 32)).astype(int)
    Rs = rng.integers(8, 65, size=n)
    sw = np.round(10.0 ** rng.uniform(sweeps_exp[0], sweeps_exp[1], size=n)).astype(int)
    hs = rng.choice(np.array([0.0, 0.1]), size=n)
    out = []
    for j in range(n):
        p = Problem(L=int(Ls[j]), betas=linear_ladder(0.30, 0.60, int(Rs[j])), J=1.0,
                    h=float(hs[j]), seed=0x5EED2000 + j, sweeps=int(sw[j]), every=1)
        out.append(Request(rid=j, arrival=float(t[j]), problem=p))
    return out


def random_spins(L: int, seed: int) -> np.ndarray:
    """A seeded random +/-1 int8 lattice (for set-spins tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, L))
