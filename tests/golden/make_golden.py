"""Writes the stored expected values under tests/golden/.

Calls only the FP64 oracle (``oracle/``) and the seeded input generator; no
value here comes from the CUDA library.  Re-run after a change to the
oracle's arithmetic that a cited passage justifies:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2009_11742_gb300 import inputs  # noqa: E402


def small_forward():
    """Rank-2 leapfrog (Sec. 3.1, Eq. (shwave_rom_ode_tensor)) with Ricker point
    forcing (Sec. 2.2, 3.2) and receiver traces (Sec. 4.5.2) on a tiny
    non-square problem: Kv = 8, Ks = 6, M = 3, R = 2, 200 steps, r = 10."""
    p = inputs.make_problem(8, 6, 3, 2, seed=0)
    V, S, tr = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, np.zeros((8, 3)),
                              np.zeros((6, 3)), 200, T=p.T, r=10)
    return {
        "source": "oracle/rom_oracle.c orc_forward; leapfrog of Sec. 3.1, model "
                  "Eq. (shwave_rom_ode_tensor), Ricker source Sec. 3.2, traces Sec. 4.5.2",
        "problem": {"Kv": 8, "Ks": 6, "M": 3, "R": 2, "seed": 0, "steps": 200, "r": 10,
                    "n0": 0, "X0": "zero"},
        "dt": p.dt,
        "V": V.tolist(), "S": S.tolist(), "traces": tr.tolist(),
    }


def main():
    out = os.path.join(HERE, "oracle_small_forward.json")
    with open(out, "w") as f:
        json.dump(small_forward(), f, indent=1)
    print("wrote", out)


if __name__ == "__main__":
    main()
