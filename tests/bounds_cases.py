"""Small parity cases run through every device route, for the bounds-checked library.

Run as a script (python tests/bounds_cases.py OUT.npz) in a process whose $PEERS_LIB names the
library to load; it writes every result array to OUT.npz.  Used by test_gpu_bounds.py, which
runs it once with libpeers_bounds.so and compares with the regular library and the oracle.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2606_31535_b300 import inputs as I  # noqa: E402


def cases():
    """(name, graph, qu, qv, front_smem): edges of grids, a 3-layer mesh with non-edge pairs
    (two-branch walks), a geometric graph, and fronts forced into global memory."""
    pdn = I.pdn3(side=21, seed=61)
    u, v = pdn.all_edges()
    pu, pv = I.random_pairs(pdn.n, 400, seed=62)
    return [
        ("grid32", I.grid32(), None, None, 0),
        ("pdn3-21-pairs", pdn, np.concatenate([u, pu]), np.concatenate([v, pv]), 0),
        ("rgg-3000", I.rgg(3000, seed=63), None, None, 0),
        ("grid-60-spill", I.grid2d(60, 61, seed=64), None, None, 1),
    ]


def run(out_path):
    import torch
    from paper_2606_31535_b300 import peers as P
    ctx = P.Context(0)
    out = {}
    for name, g, qu, qv, fs in cases():
        opt = P.Options()
        opt.front_smem = fs
        sym = P.Symbolic.of(g, 0, qu, qv, True, opt)
        num = P.Numeric(ctx, sym)
        out[name + "/walk"] = P.query(ctx, sym, num)
        out[name + "/blockinv"] = P.query_blockinv(ctx, sym, num)
        if sym.info()["nq_two_branch"] == 0:
            out[name + "/selinv"] = P.query_selinv(ctx, sym, num)
        if fs == 0:
            opt2 = P.Options()
            opt2.carry_budget = 1 << 20   # several waves inside the static scratch
            sym2 = P.Symbolic.of(g, 0, qu, qv, True, opt2)
            num2 = P.Numeric(ctx, sym2)
            d = torch.empty(sym2.nq, dtype=torch.float64, device="cuda:0")
            P.query_noalloc(ctx, sym2, num2, d)
            out[name + "/noalloc"] = d.cpu().numpy()
        out[name + "/diag"] = num.diag()
    np.savez(out_path, **out)


if __name__ == "__main__":
    run(sys.argv[1])
