"""Write tests/golden/oracle_regression.json from the CPU oracle alone.

The paper prints no worked numeric example (its Sec. 4 reports plots and speed-ups only),
so these fixtures are not the paper's numbers: they are the oracle's outputs on small seeded
cases, stored so that any later change to the oracle's arithmetic shows up as a diff that
has to be justified. Run: python tests/golden/make_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2512_03825_b300 import workloads as W  # noqa: E402

CASES = [
    ("L16_R8_1000sweeps_every10", W.SINGLE["L16_R8"]),
    ("L8_R5_field0.1_50sweeps_every3",
     W.Problem(L=8, betas=W.linear_ladder(0.2, 0.7, 5), J=1.0, h=0.1, seed=7, sweeps=50,
               every=3)),
    ("L6_R3_antiferro_40sweeps_every2",
     W.Problem(L=6, betas=(0.3, 0.5, 0.9), J=-1.0, h=0.25, seed=99, sweeps=40, every=2)),
]


def summarise(prob):
    p = oracle.OracleProblem(prob.L, prob.betas, J=prob.J, h=prob.h, seed=prob.seed)
    p.sweep(prob.sweeps, prob.every)
    att, acc = p.swap_stats()
    return {
        "L": prob.L, "betas": list(prob.betas), "J": prob.J, "h": prob.h, "seed": prob.seed,
        "sweeps": prob.sweeps, "every": prob.every,
        "E_int": p.energies_int().tolist(), "M": p.magnetisations().tolist(),
        "scale": p.scale, "attempted": att.tolist(), "accepted": acc.tolist(),
        "chain_map": p.chain_map().tolist(), "counters": list(p.counters()),
        "spins_sha256": hashlib.sha256(p.spins().tobytes()).hexdigest(),
    }


def main():
    out = {"source": "oracle/pt_oracle.c via tests/golden/make_golden.py; the paper prints "
                     "no worked example (Sec. 4 gives plots and speed-ups only)",
           "cases": {name: summarise(prob) for name, prob in CASES}}
    path = os.path.join(HERE, "oracle_regression.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(path)


if __name__ == "__main__":
    main()
