"""Pins of the Ewald oracle (O3, Eq. screening): textbook Madelung constant,
splitting-parameter independence, absolutely convergent image sums, finite
differences."""
import numpy as np
import pytest

from conftest import rel_rms
from oracle.ewald import ewald, image_sum
from paper_2606_06617_b300 import workloads as wl

MADELUNG_NACL = 1.747564594633182   # textbook rock-salt Madelung constant


def test_nacl_madelung():
    """NaCl 2x2x2 conventional cells, a = 5.64 A, nearest neighbour a/2:
    E = -N/2 * M / (a/2), phi_i = -q_i M / (a/2), zero forces by symmetry."""
    s = wl.nacl()
    r0 = 5.64 / 2
    e = ewald(s.pos, s.q[0], s.box, 1)
    assert abs(e["E"] / (-32 * MADELUNG_NACL / r0) - 1) < 1e-11
    np.testing.assert_allclose(e["phi"], -s.q[0] * MADELUNG_NACL / r0, rtol=1e-10)
    assert np.max(np.abs(e["F"])) < 1e-10


@pytest.mark.parametrize("p,neutral", [(1, True), (1, False), (2, True), (2, False), (3, True), (3, False),
                                       (4, False), (5, False), (6, True), (6, False)])
def test_alpha_independence(p, neutral):
    s = wl.random_system(12, (6.0, 7.0, 6.5), (p,), seed=p, neutral=neutral)
    a = ewald(s.pos, s.q[0], s.box, p, alpha=0.9)
    b = ewald(s.pos, s.q[0], s.box, p, alpha=1.4)
    assert abs(a["E"] - b["E"]) < 1e-10 * max(1.0, abs(a["E"]))
    assert rel_rms(a["phi"], b["phi"]) < 1e-10
    assert rel_rms(a["F"], b["F"]) < 1e-10


@pytest.mark.parametrize("p,neutral", [(4, True), (4, False), (6, True), (6, False)])
def test_image_sum(p, neutral):
    """p > 3: the lattice sum converges absolutely; a tapered explicit image
    sum must agree with the Ewald split."""
    s = wl.random_system(8, (5.0, 6.0, 5.5), (p,), seed=3, neutral=neutral)
    e = ewald(s.pos, s.q[0], s.box, p, alpha=0.8)
    Ei, Fi = image_sum(s.pos, s.q[0], s.box, p, 70.0, smooth=True)
    assert abs(Ei / e["E"] - 1) < 5e-8
    assert rel_rms(Fi, e["F"]) < 5e-8


@pytest.mark.parametrize("p", [1, 6])
def test_forces_are_minus_gradient(p):
    s = wl.random_system(10, (6.0, 6.0, 6.0), (p,), seed=9, neutral=True)
    e = ewald(s.pos, s.q[0], s.box, p)
    h = 1e-5
    for i, d in [(0, 0), (3, 1), (7, 2)]:
        pp = s.pos.copy(); pp[i, d] += h
        pm = s.pos.copy(); pm[i, d] -= h
        fd = -(ewald(pp, s.q[0], s.box, p)["E"] - ewald(pm, s.q[0], s.box, p)["E"]) / (2 * h)
        assert abs(fd - e["F"][i, d]) < 1e-7 * max(1.0, np.abs(e["F"]).max())
    assert np.abs(e["F"].sum(0)).max() < 1e-10 * np.abs(e["F"]).max()


@pytest.mark.parametrize("p", [1, 4])
def test_quadratic_form(p):
    """E = 1/2 sum_i q_i phi_i (every Ewald piece is a quadratic form in q)."""
    s = wl.random_system(10, (6.0, 6.0, 6.0), (p,), seed=1, neutral=False)
    e = ewald(s.pos, s.q[0], s.box, p)
    assert abs(0.5 * np.dot(s.q[0], e["phi"]) / e["E"] - 1) < 1e-12


def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    return [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]


def test_screening_special_cases_from_the_paper():
    """The oracle's real-space screening Gamma(p/2, x^2)/Gamma(p/2) (library
    incomplete gamma) against the paper's closed forms for p = 1 and p = 6
    (tests/golden/ewald_screening.txt)."""
    import math
    from oracle.ewald import screening
    for p_s, x_s in _golden("ewald_screening.txt"):
        p, x = int(p_s), float(x_s)
        got = float(screening(p, x))
        if p == 1:
            ref = math.erfc(x)
        else:
            ref = math.exp(-x * x) * (1 + x * x + x ** 4 / 2)
        assert abs(got - ref) <= 1e-13 * max(1.0, abs(ref)), (p, x, got, ref)


def test_madelung_constant_golden():
    """The stored Madelung constant is the one the NaCl pin uses."""
    (val,), = _golden("nacl_madelung.txt")
    assert abs(float(val) - 1.747564594633182) < 1e-15
