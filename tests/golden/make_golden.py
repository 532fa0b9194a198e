"""Writes the stored expected trajectories of tests/golden/ from the FP64 oracle only.

    python tests/golden/make_golden.py        (a few minutes on a multi-core host)

cfg2_line_search_50.json: the r = 24, N = 12, CAS(6e,6o) system (synthetic integrals, seed 0), 50 Euler
steps with the line search (initial trial step 1e-3), no stopping rule: per step the accepted eps,
||A||^2 before the step and E after it.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import acse_inputs as I  # noqa: E402
from oracle import acse_oracle as O  # noqa: E402


def cfg2_line_search(nsteps=50):
    p = I.config_problem(2)
    t0 = time.time()
    out = O.run_acse(p.h, p.V, p.N, O.so_from_blocks(p.Daa, p.Dab, p.Dbb), None, nsteps, line_search=True,
                     eps0=1e-3)
    return {"system": p.name, "seed": 0, "nsteps": nsteps, "eps0": 1e-3,
            "eps": [float(x) for x in out["eps"]], "norm2": [float(x) for x in out["norm2"]],
            "E": [float(x) for x in out["E"]], "oracle_seconds": time.time() - t0,
            "source": "oracle.acse_oracle.run_acse (FP64 numpy, spin-orbital basis)"}


if __name__ == "__main__":
    d = cfg2_line_search()
    json.dump(d, open(os.path.join(HERE, "cfg2_line_search_50.json"), "w"), indent=1)
    print("wrote cfg2_line_search_50.json", d["oracle_seconds"])
