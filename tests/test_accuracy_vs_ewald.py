"""Accuracy of the benchmarked parameter sets against the physical lattice
sum (O3, Ewald): discrete PSWF-LR (O1) + real-space complement - self energy,
per channel, relative force RMS <= 1e-5 (the tolerance the parameters are
chosen for).  The large ionic melt is checked on a density-matched sub-box
with the same grid spacing, mollifier and stencil."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from oracle.ewald import ewald
from oracle.grid import DiscretePSWF, GridConfig
from oracle.realspace import pswf_total
from paper_2606_06617_b300 import workloads as wl


def _check(s, M, P, r_c, tol, bound):
    c = math.log(3.0 / tol)
    eta = max(L / m for L, m in zip(s.box, M)) * (c / r_c) / math.pi
    cw = P * math.pi * (1 - eta / 2)
    o1 = DiscretePSWF(GridConfig(s.box, M, P, c, r_c, s.ps, c_w=cw)).evaluate(s.pos, s.q)
    tot = pswf_total(dict(E_ch=o1["E_ch"].numpy(), phi=o1["phi"].numpy(), f=o1["f"].numpy()),
                     s.pos, s.q, s.box, s.ps, c, r_c)
    errs = []
    for ci, p in enumerate(s.ps):
        ew = ewald(s.pos, s.q[ci], s.box, p)
        errs.append(rel_rms(tot["F_ch"][ci], ew["F"]))
    assert max(errs) <= bound, errs
    return errs


@pytest.mark.slow
def test_ionic_melt_parameters_subbox():
    """384^3 grid over L = 350 A (h = 0.911 A), r_c = 7, c = log(3e5), P = 7:
    sub-box L = 21.875 A, 24^3, 1024 atoms at the same density."""
    L = 350.0 * 24 / 384
    n = int(round(4194304 * (L / 350.0) ** 3))
    s = wl.ionic_melt(n, L, seed=3)
    _check(s, (24, 24, 24), 7, 7.0, 1e-5, 1e-5)


@pytest.mark.slow
def test_water_parameters():
    """Water-like box at its benchmarked parameters (64^3 over 31 A, P = 8,
    r_c = 4, tol 5e-6 so that the band truncation leaves room under 1e-5 with
    the 0.96 A intramolecular pairs): same density, 648 atoms, 38^3."""
    s = wl.water_box(n_side=6, L=18.6, seed=4)
    _check(s, (38, 38, 38), 8, 4.0, 5e-6, 1e-5)
