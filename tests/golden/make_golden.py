"""Write tests/golden/oracle_series.json from the oracle alone.

Regression fixtures: P(t) and norm(t) of small systems as computed by the
FP64 oracle (oracle/), so that an accidental change of the oracle's
arithmetic shows up.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_0710_3747_gb300 import workloads as W  # noqa: E402

CASES = [
    # name, J builder, htype, seed, dt, steps
    ("ladder_2x3", lambda: W.ladder(3, 1.0, 0.5), oracle.XY, 1, 0.05, 40),
    ("ladder_2x4_rung0.1", lambda: W.ladder(4, 1.0, 0.1), oracle.XY, 7, 0.1, 30),
    ("star_dipolar_m6", lambda: W.star_dipolar(6, 2), oracle.DIPOLAR, 1, 0.02, 50),
    ("star_isotropic_m5", lambda: W.star_gaussian(5, 3), oracle.ISOTROPIC, 3, 0.05, 30),
]


def main():
    out = {}
    for name, mk, htype, seed, dt, steps in CASES:
        J = mk()
        P, nrm, _ = oracle.run(J, htype, seed, dt, steps)
        out[name] = {"J": J.tolist(), "htype": htype, "seed": seed, "dt": dt, "steps": steps,
                     "P": P.tolist(), "norm": nrm.tolist()}
    with open(os.path.join(HERE, "oracle_series.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
