"""Writes the stored expected trajectories of tests/golden/ from the FP64 oracle only.

    python tests/golden/make_golden.py [cfg2] [cfg3]     (all files when no name is given)

cfg2_line_search_50.json: the r = 24, N = 12, CAS(6e,6o) system (synthetic integrals, seed 0), 50 Euler
steps with the line search (initial trial step 1e-3), no stopping rule: per step the accepted eps,
||A||^2 before the step and E after it.  A few minutes on a multi-core host.

cfg3_fixed_eps_5.json: the r = 48, N = 20, CAS(8e,8o) system (synthetic integrals, seed 0), 5 Euler steps
with the fixed step eps = 1e-4: E and ||A||^2 at D_0 ... D_5, and 64 seeded entries of each spin block of
D_5 (indices drawn by a PCG64 generator of seed 48, stored beside the values).  About ten minutes of
numpy on eight cores (eleven contraction passes at 2r = 96 spin orbitals).
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


def cfg3_fixed_eps(nsteps=5, eps=1e-4, nsample=64):
    p = I.config_problem(3)
    t0 = time.time()
    out = O.run_acse(p.h, p.V, p.N, O.so_from_blocks(p.Daa, p.Dab, p.Dbb), eps, nsteps)
    blocks = O.blocks_from_so(out["D"])
    rng = I.rng_for(48)
    idx = rng.integers(0, p.r, size=(3, nsample, 4))
    samples = [[float(b[tuple(ix)]) for ix in idx[s]] for s, b in enumerate(blocks)]
    return {"system": p.name, "seed": 0, "nsteps": nsteps, "eps": eps,
            "E": [float(x) for x in out["E"]], "norm2": [float(x) for x in out["norm2"]],
            "D_final_index": idx.tolist(), "D_final_aa_ab_bb": samples,
            "oracle_seconds": time.time() - t0,
            "source": "oracle.acse_oracle.run_acse (FP64 numpy, spin-orbital basis)"}


if __name__ == "__main__":
    which = sys.argv[1:] or ["cfg2", "cfg3"]
    if "cfg2" in which:
        d = cfg2_line_search()
        json.dump(d, open(os.path.join(HERE, "cfg2_line_search_50.json"), "w"), indent=1)
        print("wrote cfg2_line_search_50.json", d["oracle_seconds"])
    if "cfg3" in which:
        d = cfg3_fixed_eps()
        json.dump(d, open(os.path.join(HERE, "cfg3_fixed_eps_5.json"), "w"), indent=1)
        print("wrote cfg3_fixed_eps_5.json", d["oracle_seconds"])
