"""Writes tests/golden/oracle_6x5x4.json from the FP64 oracle (oracle/ only).

The paper prints no worked example for the projection, so this fixture is a
regression record of the oracle itself on a tiny seeded case: it catches an
accidental change of the oracle's arithmetic.  Its values were checked, when
written, by the pins in tests/test_oracle_pins.py.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O  # noqa: E402
from paper_2009_12849_gb300 import workloads as W  # noqa: E402


def case():
    g = W.make_grid(6, 5, 4, 50.0, 40.0, W.geometric_dz(4, 10.0, 60.0))
    u, v, w = W.random_fields(g, 7, True)
    return g, u, v, w


def main():
    g, u, v, w = case()
    uo, vo, wo, phi = O.project(u, v, w, g.dx, g.dy, g.dz, g.rho_c, g.rho_f)
    rec = {"grid": {"nx": g.nx, "ny": g.ny, "nz": g.nz, "dx": g.dx, "dy": g.dy,
                    "dz": "geometric 10->60 m", "seed": 7, "large_scale_mode": True},
           "u_out": uo.ravel().tolist(), "v_out": vo.ravel().tolist(),
           "w_out": wo.ravel().tolist(), "phi": phi.ravel().tolist()}
    with open(os.path.join(HERE, "oracle_6x5x4.json"), "w") as f:
        json.dump(rec, f, indent=0)


if __name__ == "__main__":
    main()
