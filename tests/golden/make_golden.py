"""Writes oracle_small.json: regression values of the CPU oracle on a seeded case (10/27 mechanism, six
cells of the uniform random field, seed 11).  It calls only the oracle (and the seeded input generator);
the paper prints no worked example, so these values pin the oracle to itself over time: a change of the
oracle's arithmetic that moves them must come with a new file and the passage that justifies it.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.oracle import Oracle  # noqa: E402
from paper_2311_14941_gb300 import synth  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")


def golden():
    m = synth.mechanism_small()
    o = Oracle(m)
    F = synth.field_uniform_random(m, 6, seed=11)
    cells = []
    for c in range(F.n_cells):
        y0 = o.state(F.T[c], F.Y[:, c])
        rec = {"T": float(F.T[c]), "p": float(F.p[c]), "Y": F.Y[:, c].tolist(), "dt": float(F.dt[c]),
               "f": o.rhs(F.T[c], F.p[c], F.Y[:, c])["f"].tolist()}
        for method, name in ((0, "rodas3"), (1, "ros2"), (2, "rodas4")):
            yn, ye = o.step(y0, F.p[c], 1e-11, method=method)
            r = o.integrate(F.T[c], F.p[c], F.Y[:, c], F.dt[c], method=method)
            rec[name] = {"step_h": 1e-11, "step_ynew": yn.tolist(), "step_yerr": ye.tolist(), "T": float(r["T"]),
                         "Y": np.asarray(r["Y"]).tolist(), "nsub": int(r["nsub"]), "status": int(r["status"])}
        cells.append(rec)
    return {"source": "CPU oracle (oracle/chem_oracle.cpp), written by tests/golden/make_golden.py",
            "case": "synth.mechanism_small(), synth.field_uniform_random(m, 6, seed=11), rtol 1e-6, atol 1e-12",
            "cells": cells}


if __name__ == "__main__":
    with open(OUT, "w") as f:
        json.dump(golden(), f, indent=1)
    print(OUT)
