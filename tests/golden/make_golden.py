"""Write tests/golden/config1_4x4.json from the oracle alone.

Workload (the 4^4 case): random SU(3) links exp(i 0.3 H), seed 1; plain Wilson
kappa = 0.12; open time boundary; Gamma = t 0..1, Gamma* = t 2..3 (no overlap);
12 point sources at the origin.  Stored: the oracle's full propagator,
factorized part (Sec. 3, eqs. quark_prop_I / quark_prop_II) and correction at a
fixed set of sites, as text.  The oracle itself is pinned against a dense-LU
brute force of the same matrix in tests/test_oracle_dense.py.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1612_06424_gb300 import inputs  # noqa: E402

DIMS = (4, 4, 4, 4)
SITES = [0, 17, 63, 100, 150, 200, 255]
COLS = [0, 5, 11]


def main():
    U = inputs.random_su3_field(DIMS, 0.3, 1)
    op = oracle.Operator(DIMS, U, 0.12, 0.0)
    eta = inputs.point_sources(DIMS, (0, 0, 0, 0))
    split = oracle.Split((0, 1), (2, 3))
    fact = oracle.factorized_propagator(op, split, eta)
    full = oracle.full_propagator(op, eta)
    corr = full - fact

    def pick(a):
        v = a[COLS][:, SITES].reshape(-1)
        return [[float(z.real), float(z.imag)] for z in v]

    out = {"dims": list(DIMS), "eps": 0.3, "seed": 1, "kappa": 0.12, "csw": 0.0, "bc": "open",
           "gamma": [0, 1], "gamma_star": [2, 3], "x_src": [0, 0, 0, 0], "sites": SITES, "cols": COLS,
           "layout": "[col in cols][site in sites][spin 4][colour 3] flattened, (re, im)",
           "full": pick(full), "fact": pick(fact), "corr": pick(corr),
           "source": "oracle (tests/golden/make_golden.py); paper prints no numeric example"}
    with open(os.path.join(HERE, "config1_4x4.json"), "w") as fh:
        json.dump(out, fh, separators=(",", ":"))


if __name__ == "__main__":
    main()
