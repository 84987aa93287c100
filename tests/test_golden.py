"""The oracle reproduces its recorded output on a tiny seeded case."""
import json
import os

import numpy as np

import oracle as O
from tests.golden.make_golden import case

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_oracle_matches_recorded_fixture():
    with open(os.path.join(HERE, "oracle_6x5x4.json")) as f:
        rec = json.load(f)
    g, u, v, w = case()
    uo, vo, wo, phi = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    for name, arr in (("u_out", uo), ("v_out", vo), ("w_out", wo), ("phi", phi)):
        ref = np.array(rec[name])
        assert np.max(np.abs(arr.ravel() - ref)) < 1e-12 * (1 + np.max(np.abs(ref)))
