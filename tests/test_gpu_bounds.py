"""The bounds-checked build (libpeers_bounds.so, compiled with PEERS_BOUNDS=1).

In that build every kernel access to a panel, front, carry slot, relative map, inverse block
or result is checked against the extent the analysis computed; a violation records the source
line in the call's error flag, skips the access, and the call fails with PEERS_ECUDA naming
the line.  (No device sanitizer is used.)  The small parity cases of tests/bounds_cases.py go
through every route -- the walk with one- and two-branch queries and fronts in global memory,
the block inverse, the selected inversion, the no-allocation sweep, the factorization -- in a
process that loads the checked library: every call must finish without a recorded violation,
with results bit-identical to the regular library's and within 1e-9 of the oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-9
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def libs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_31535_b300 import build
    return build.build(), build.build(bounds=True)


def run_cases(lib, out):
    env = dict(os.environ, PEERS_LIB=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "bounds_cases.py"), str(out)],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    return dict(np.load(out))


def test_bounds_checked_build_runs_clean_and_matches(libs, tmp_path, oracle_mod):
    regular, checked = libs
    got = run_cases(checked, tmp_path / "checked.npz")
    ref = run_cases(regular, tmp_path / "regular.npz")
    assert got.keys() == ref.keys()
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    sys.path.insert(0, HERE)
    import bounds_cases
    for name, g, qu, qv, _ in bounds_cases.cases():
        if qu is None:
            qu, qv = g.all_edges()
        Ro = oracle_mod.resistance(g, qu, qv)
        for route in ("walk", "blockinv", "selinv", "noalloc"):
            key = name + "/" + route
            if key in got:
                assert float(np.max(np.abs(got[key] - Ro) / Ro)) <= TOL, key
