"""The FP64 oracle reproduces its stored values on the 8-atom Si workload (tests/golden)."""
import os

import numpy as np

from tests.golden.make_golden import HERE, compute


def _load():
    out = dict(rho={}, H={}, F={})
    with open(os.path.join(HERE, "si8_g48_oracle.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            k, *v = line.split()
            if k in ("W", "Ne"):
                out[k] = float(v[0])
            elif k == "rho":
                out["rho"][int(v[0])] = float(v[1])
            elif k == "H":
                out["H"][(int(v[0]), int(v[1]))] = float(v[2])
            elif k == "F":
                out["F"][int(v[0])] = np.array([float(x) for x in v[1:]])
    return out


def test_oracle_matches_stored_values():
    ref, d = _load(), compute()
    assert d["W"] == ref["W"]
    assert abs(d["ne"] - ref["Ne"]) <= 1e-13 * abs(ref["Ne"])
    rmax = max(abs(v) for v in ref["rho"].values())
    for g, v in d["rho"]:
        assert abs(v - ref["rho"][g]) <= 1e-13 * rmax, g
    hmax = max(abs(v) for v in ref["H"].values())
    for m, n, v in d["H"]:
        assert abs(v - ref["H"][(m, n)]) <= 1e-13 * hmax, (m, n)
    fmax = max(np.abs(v).max() for v in ref["F"].values())
    for a in range(d["F"].shape[0]):
        assert np.abs(d["F"][a] - ref["F"][a]).max() <= 1e-12 * fmax, a
