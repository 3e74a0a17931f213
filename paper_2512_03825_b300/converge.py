"""Sweeps to convergence against lattice size (the benchmark of Sec. 4.1, Fig. 3b).

The paper plots the iterations its replicas need to reach the target distribution against L
and reports a quadratic growth; it does not state how convergence was detected. The reading
taken here is a two-start diagnostic that needs no estimate of the equilibrium values:

* a problem is run twice with the same seed, ladder and exchange interval: once from the
  random initial spins that pt_create draws ("hot"), once from every spin +1 at every
  temperature ("cold", set with pt_set_spins before the first sweep);
* both runs record the per-sweep trace (E_int of every temperature index, after the sweep
  and its swap iteration);
* temperature index k has converged at the first sweep count t at which the hot run's
  energy is at or below the cold run's, E_hot[t][k] <= E_cold[t][k]: the energy of the
  disordered start has come down to that of the ordered start, which approaches the same
  equilibrium value from below;
* the problem has converged at t* = the largest of these over its temperatures.

All inputs of the criterion are exact integers from the trace, so the GPU path and the
oracle give the same t* whenever their traces agree (a GPU test checks both). The sampler
runs in the CUDA library; this module only schedules runs and reads their traces.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import workloads as W

NOT_YET = -1


def first_crossing(E_hot: np.ndarray, E_cold: np.ndarray, first_sweep: int = 1) -> np.ndarray:
    """Per temperature index k (columns), the sweep count of the first row with
    E_hot <= E_cold (row j of the arrays was taken after first_sweep + j sweeps), or NOT_YET
    when no row has it. E_hot and E_cold: [rows][R] integer arrays."""
    E_hot = np.asarray(E_hot)
    E_cold = np.asarray(E_cold)
    if E_hot.shape != E_cold.shape or E_hot.ndim != 2:
        raise ValueError("traces must have the same [rows][R] shape")
    hit = E_hot <= E_cold
    any_hit = hit.any(axis=0)
    first = hit.argmax(axis=0) + int(first_sweep)
    return np.where(any_hit, first, NOT_YET).astype(np.int64)


def converged_at(per_temperature: np.ndarray) -> int:
    """t* = the last temperature to converge; NOT_YET if any has not."""
    per_temperature = np.asarray(per_temperature)
    if (per_temperature == NOT_YET).any():
        return NOT_YET
    return int(per_temperature.max())


def fit_exponent(Ls: Sequence[float], t: Sequence[float]) -> float:
    """Least-squares slope of log t against log L (t ~ L^slope)."""
    x = np.log(np.asarray(Ls, dtype=np.float64))
    y = np.log(np.asarray(t, dtype=np.float64))
    if x.size < 2:
        raise ValueError("need at least two sizes")
    A = np.vstack([x, np.ones_like(x)]).T
    slope, _ = np.linalg.lstsq(A, y, rcond=None)[0]
    return float(slope)


def paper_ladder_problem(L: int, R: int, seed: int, every: int) -> W.Problem:
    """A problem on the paper's temperature ladder T_i = 1 + 3i/|R| (Sec. 3), J = 1, B = 0."""
    return W.Problem(L=L, betas=W.paper_ladder(R), J=1.0, h=0.0, seed=seed, every=every)


def cold_start(handle, L: int, R: int) -> None:
    """Every spin +1 at every temperature index (the ordered start)."""
    up = np.ones((L, L), dtype=np.int8)
    for k in range(R):
        handle.set_spins(k, up)


@dataclasses.dataclass
class Run:
    """One (L, seed) measurement: the hot and cold problems and what is known so far."""
    L: int
    seed: int
    hot: object
    cold: object
    per_temperature: np.ndarray
    done: int = 0  # sweeps run so far

    @property
    def t_star(self) -> int:
        return converged_at(self.per_temperature)


def measure(api, Ls: Sequence[int], seeds: Sequence[int], R: int = 32, every: int = 1,
            cap_factor: float = 8.0, cap_min: int = 2000, stream=None,
            chunk_factor: float = 0.25, chunk_min: int = 200,
            details: Optional[dict] = None) -> Dict[int, List[int]]:
    """Sweeps to convergence t* for every L and seed, on the GPU. Every (L, seed) runs as a
    hot/cold pair; all pairs advance together through pt_sweep_batch in chunks of
    max(chunk_min, chunk_factor L^2) sweeps of their own size class, and a pair leaves the
    batch once every temperature has converged, or after max(cap_min, cap_factor L^2) sweeps
    (then its t* is NOT_YET: censored). Returns {L: [t* per seed]}; with `details`, also
    fills details[(L, seed)] with the per-temperature convergence sweeps."""
    runs: List[Run] = []
    cap = {L: int(max(cap_min, cap_factor * L * L)) for L in Ls}
    chunk = {L: int(max(chunk_min, chunk_factor * L * L)) for L in Ls}
    for L in Ls:
        for s in seeds:
            p = paper_ladder_problem(L, R, s, every)
            hot = api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=stream)
            cold = api.PTProblem(p.L, p.betas, J=p.J, h=p.h, seed=p.seed, stream=stream)
            cold_start(cold, L, R)
            for h in (hot, cold):
                h.trace_start(chunk[L])
            runs.append(Run(L=L, seed=s, hot=hot, cold=cold,
                            per_temperature=np.full(R, NOT_YET, dtype=np.int64)))
    active = list(runs)
    while active:
        n = [min(chunk[r.L], cap[r.L] - r.done) for r in active]
        handles, ns = [], []
        for r, k in zip(active, n):
            handles += [r.hot, r.cold]
            ns += [k, k]
        api.sweep_batch(handles, ns, [every] * len(handles))
        still = []
        for r, k in zip(active, n):
            f_h, E_h, _ = r.hot.trace(k)
            f_c, E_c, _ = r.cold.trace(k)
            assert f_h == f_c == r.done + 1 and len(E_h) == len(E_c) == k
            new = first_crossing(E_h, E_c, f_h)
            todo = r.per_temperature == NOT_YET
            r.per_temperature[todo] = new[todo]
            r.done += k
            if r.t_star == NOT_YET and r.done < cap[r.L]:
                still.append(r)
        active = still
    out: Dict[int, List[int]] = {L: [] for L in Ls}
    for r in runs:
        out[r.L].append(r.t_star)
        if details is not None:
            details[(r.L, r.seed)] = r.per_temperature.tolist()
        r.hot.close()
        r.cold.close()
    return out


def summarise(result: Dict[int, List[int]], caps: Optional[Dict[int, int]] = None) -> dict:
    """Median (and quartiles) of t* per L over the seeds, the fitted exponents of the median
    in sweeps and in single-spin-flip iterations (t* L^2 trials per replica), and how many runs
    were censored. A censored run counts as its cap in the median (a lower bound)."""
    Ls = sorted(result)
    rows = {}
    med = []
    for L in Ls:
        ts = np.array(result[L], dtype=np.float64)
        cens = int((ts == NOT_YET).sum())
        if caps is not None:
            ts = np.where(ts == NOT_YET, caps[L], ts)
        q1, q2, q3 = (float(np.percentile(ts, q)) for q in (25, 50, 75))
        rows[str(L)] = {"median_sweeps": q2, "q1": q1, "q3": q3, "censored": cens,
                        "runs": int(ts.size), "median_iterations": q2 * L * L,
                        "t_star": [int(x) for x in result[L]]}
        med.append(q2)
    out = {"per_L": rows}
    if len(Ls) >= 2 and all(m > 0 for m in med):
        e = fit_exponent(Ls, med)
        out["exponent_sweeps"] = e
        out["exponent_iterations"] = e + 2.0
    if len(Ls) >= 3 and all(m > 0 for m in med):
        out["exponent_sweeps_without_largest"] = fit_exponent(Ls[:-1], med[:-1])
    return out


def slowest_temperatures(details: dict) -> dict:
    """Per L: how often each temperature index was the last to converge, as
    {L: {index: runs}} (a run that has not converged at every temperature is left out)."""
    out: Dict[str, Dict[str, int]] = {}
    for (L, _), per_k in sorted(details.items()):
        per_k = np.asarray(per_k)
        if (per_k == NOT_YET).any():
            continue
        k = int(per_k.argmax())
        row = out.setdefault(str(L), {})
        row[str(k)] = row.get(str(k), 0) + 1
    return out


def default_caps(Ls: Sequence[int], cap_factor: float = 8.0, cap_min: int = 2000) -> dict:
    return {L: int(max(cap_min, cap_factor * L * L)) for L in Ls}
