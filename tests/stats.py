"""Statistics helpers for the oracle's pins: exact enumeration of small lattices, Onsager's
closed forms, and blocking error bars for correlated Markov-chain time series.

These are written from textbook definitions and share nothing with the oracle.
"""
from __future__ import annotations

import math

import numpy as np


def enumerate_lattice(L, J, h):
    """All 2^(L*L) states of the periodic L x L lattice: (E, M) arrays, E from the Ising
    Hamiltonian E = h * sum sigma - J * sum_<ij> sigma_i sigma_j (each bond once)."""
    n = L * L
    assert n <= 20
    idx = np.arange(1 << n, dtype=np.int64)
    bits = ((idx[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)
    sig = (2 * bits - 1).reshape(-1, L, L)
    bonds = np.zeros(sig.shape[0], dtype=np.int64)
    for y in range(L):
        for x in range(L):
            bonds += sig[:, y, x] * sig[:, y, (x + 1) % L]
            bonds += sig[:, y, x] * sig[:, (y + 1) % L, x]
    M = sig.reshape(sig.shape[0], -1).sum(axis=1)
    E = h * M - J * bonds
    return E.astype(np.float64), M.astype(np.float64)


def boltzmann_weights(E, beta):
    w = -beta * E
    w = np.exp(w - w.max())
    return w / w.sum()


def exact_moments(E, M, beta):
    p = boltzmann_weights(E, beta)
    return dict(E=float((p * E).sum()), absM=float((p * np.abs(M)).sum()),
                M=float((p * M).sum()))


def blocked_mean_se(x, min_blocks=32):
    """Mean and standard error of a correlated series by the blocking method
    (Flyvbjerg and Petersen 1989): pair-average repeatedly and take the largest error
    estimate seen while at least ``min_blocks`` blocks remain."""
    x = np.asarray(x, dtype=np.float64)
    mean = float(x.mean())
    best = float(x.std(ddof=1) / math.sqrt(x.size)) if x.size > 1 else 0.0
    y = x.copy()
    while y.size // 2 >= min_blocks:
        y = 0.5 * (y[: 2 * (y.size // 2):2] + y[1: 2 * (y.size // 2):2])
        se = float(y.std(ddof=1) / math.sqrt(y.size))
        best = max(best, se)
    return mean, best


def _agm(a, b):
    for _ in range(60):
        a, b = 0.5 * (a + b), math.sqrt(a * b)
    return a


def ellipk(k):
    """Complete elliptic integral of the first kind K(k) (modulus k) by the
    arithmetic-geometric mean: K = pi / (2 AGM(1, sqrt(1 - k^2)))."""
    return math.pi / (2.0 * _agm(1.0, math.sqrt(max(1.0 - k * k, 1e-300))))


def onsager_energy_per_spin(beta, J=1.0):
    """Onsager's internal energy per spin of the infinite square-lattice Ising model, h = 0:
    u = -J coth(2 beta J) [1 + (2/pi)(2 tanh^2(2 beta J) - 1) K(kappa)],
    kappa = 2 sinh(2 beta J) / cosh^2(2 beta J)."""
    t = 2.0 * beta * J
    kappa = 2.0 * math.sinh(t) / math.cosh(t) ** 2
    return -J / math.tanh(t) * (1.0 + (2.0 / math.pi) * (2.0 * math.tanh(t) ** 2 - 1.0)
                                * ellipk(kappa))


def onsager_magnetisation(beta, J=1.0):
    """Spontaneous magnetisation per spin (Onsager / Yang): (1 - sinh^-4(2 beta J))^(1/8)
    above beta_c = ln(1 + sqrt 2) / 2, zero below."""
    s = math.sinh(2.0 * beta * J)
    v = 1.0 - s ** -4
    return v ** 0.125 if v > 0 else 0.0


BETA_C = 0.5 * math.log(1.0 + math.sqrt(2.0))
