"""Writes si8_g48_oracle.txt: FP64 oracle values on the 8-atom Si workload (48^3 grid), sampled.

Calls only oracle/ and the seeded input generators.  The file guards the oracle against silent
changes (tests/test_golden.py recomputes it); the oracle itself is pinned by the closed forms,
identities and brute-force checks of tests/test_oracle_pins.py.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle.oracle import Oracle  # noqa: E402
from paper_2603_21835_gb300 import inputs  # noqa: E402

POINTS = [0, 1, 47, 2305, 11111, 27648, 55296, 60001, 77777, 99999, 110592 - 1]
ORBITALS = [(0, 0), (0, 13), (5, 77), (12, 12), (40, 103), (103, 103), (64, 3), (90, 51)]


def compute():
    w = inputs.config_workload("si8_g48")
    o = Oracle(w.system)
    rho = o.rho(w.D).reshape(-1)
    H = o.vlocal(w.V)
    F = o.force(w.D, w.V)
    W, _ = o.count_pairs()
    ne = o.weight() * float(rho.sum())
    return dict(rho=[(g, float(rho[g])) for g in POINTS], H=[(m, n, float(H[m, n])) for m, n in ORBITALS],
                F=np.asarray(F, dtype=np.float64), W=float(W), ne=float(ne))


def main():
    d = compute()
    path = os.path.join(HERE, "si8_g48_oracle.txt")
    with open(path, "w") as f:
        f.write("# FP64 oracle, si8_g48 (8-atom cubic Si, 48^3 grid, seed 0), written by make_golden.py\n")
        f.write(f"W {d['W']!r}\n")
        f.write(f"Ne {d['ne']!r}\n")
        for g, v in d["rho"]:
            f.write(f"rho {g} {v!r}\n")
        for m, n, v in d["H"]:
            f.write(f"H {m} {n} {v!r}\n")
        for a in range(d["F"].shape[0]):
            f.write("F {} {!r} {!r} {!r}\n".format(a, *(float(x) for x in d["F"][a])))
    print("wrote", path)


if __name__ == "__main__":
    main()
