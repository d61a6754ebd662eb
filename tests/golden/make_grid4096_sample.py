"""Writes grid4096_sample.json: oracle resistances of 3000 edges of the 4096 x 4096 grid
(log-uniform conductances 1e-3..1e3, seed 5, node 0 grounded): 2000 drawn uniformly with a
fixed seed, and the 1000 edges of largest conductance.  The latter have the smallest
resistances, R_e <= 1/w_e, where y = z_lo - z_hi cancels the most, so they are the edges most
exposed to rounding.

The oracle has to factor the whole 16.7M-node Laplacian before it can answer any query, which
takes tens of minutes on one core, so these values are computed once by this script (which
calls only the oracle and the seeded generators) and stored for the GPU parity test.

    python tests/golden/make_grid4096_sample.py
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2606_31535_b300 import inputs as I  # noqa: E402

SAMPLE = 2000
HEAVY = 1000
SEED = 4096


def main():
    t0 = time.time()
    g = I.grid4096()
    u, v = g.all_edges()
    uni = np.random.default_rng(SEED).choice(u.size, SAMPLE, replace=False)
    heavy = np.argsort(-g.edge_weights(), kind="stable")
    heavy = heavy[~np.isin(heavy, uni)][:HEAVY]
    idx = np.sort(np.concatenate([uni, heavy]))
    F = oracle.Factor.of(g)
    t1 = time.time()
    R = F.resistance(u[idx], v[idx])
    t2 = time.time()
    out = {
        "about": "oracle (oracle/oracle.c) effective resistances of edges of the 4096x4096 "
                 "grid, log-uniform conductances 1e-3..1e3, seed 5, ground 0: a seeded uniform "
                 "sample of 2000 edges and the 1000 other edges of largest conductance",
        "selection": {"uniform": SAMPLE, "uniform_seed": SEED, "largest_conductance": HEAVY},
        "script": "tests/golden/make_grid4096_sample.py",
        "sample_seed": SEED,
        "edge_index": idx.tolist(),
        "u": u[idx].tolist(),
        "v": v[idx].tolist(),
        "R": [float(x) for x in R],
        "oracle_nnz_l": F.nnz_l,
        "oracle_factor_s": round(t1 - t0, 1),
        "oracle_query_s": round(t2 - t1, 1),
    }
    with open(os.path.join(HERE, "grid4096_sample.json"), "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main()
