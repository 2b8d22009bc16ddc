"""GPU parity of the velocity-gauge projector overlaps <beta_{I j}| e^{-i A.r} |Phi_{J mu}> (paper
Sec. 3.3.2) against the FP64 oracle.  Both sides integrate in float64 with the same rule (140 radial
Gauss-Legendre nodes, the degree-17 product angular rule; the library computes its nodes itself,
the oracle's come from numpy), so they agree to rounding: 1e-11 of max |P|."""
import itertools

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2603_21835_gb300 import inputs
from tests.test_oracle_psibeta import angular_rule, radial_rule

pytestmark = pytest.mark.gpu
TOL = 1e-11
A = np.array([0.12, -0.07, 0.05])


def _case(name):
    from paper_2603_21835_gb300 import gint as G

    w = inputs.config_workload(name)
    s = w.system
    g = G.Gint(s)
    g.set_projectors([inputs.si_projectors()])
    P = g.psibeta(A).cpu().numpy()
    g.sync()
    sysp = inputs.System(cell=s.cell, pos=s.pos, species=s.species, sp=[inputs.si_projectors()], grid=s.grid)
    return dict(s=s, g=g, P=P, o=Oracle(s), op=Oracle(sysp))


@pytest.fixture(scope="module")
def si64():
    return _case("si64_g96")


@pytest.fixture(scope="module")
def si8():
    return _case("si8_g48")


def _expected_pairs(s, reach):
    A_ = np.asarray(s.cell, float)
    pos = np.asarray(s.pos, float)
    n = range(-3, 4)
    shifts = np.array(list(itertools.product(n, n, n))) @ A_
    out = []
    for I in range(len(pos)):
        for J in range(len(pos)):
            d = pos[J] + shifts - pos[I]
            if (np.linalg.norm(d, axis=1) < reach).any():
                out.append((I, J))
    return out


def _block(c, q):
    I, J = c["g"].pb_pairs[q]
    nb, no = c["op"]._norb_atom(I), c["o"]._norb_atom(J)
    return c["P"][c["g"].pb_off[q]:c["g"].pb_off[q + 1]].reshape(nb, no)


def test_pair_list(si64):
    got = [tuple(p) for p in si64["g"].pb_pairs]
    assert got == _expected_pairs(si64["s"], 2.5 + 7.0)


@pytest.mark.parametrize("case", ["si64", "si8"])
def test_sampled_pairs_match_the_oracle(case, si64, si8):
    c = si64 if case == "si64" else si8
    pairs = [tuple(p) for p in c["g"].pb_pairs]
    pmax = np.abs(c["P"]).max()
    picks = [pairs[0], pairs[len(pairs) // 3], pairs[len(pairs) // 2], pairs[-1]]
    picks += [p for p in pairs if p[0] == p[1]][:1]
    for I, J in picks:
        q = pairs.index((I, J))
        ref = c["o"].psibeta(c["op"], A, I, J, radial_rule(), angular_rule())
        assert np.abs(_block(c, q) - ref).max() <= TOL * pmax, (case, I, J)


def test_zero_field_is_real(si8):
    P0 = si8["g"].psibeta(np.zeros(3)).cpu().numpy()
    assert np.all(P0.imag == 0.0)
    assert np.abs(P0.real).max() > 1e-3
