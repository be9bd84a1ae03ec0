"""Host-side checks of the C-ABI library (no GPU): every declared symbol is
exported, and the planner ("Parameter selection") behaves as specified."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lr():
    from paper_2606_06617_b300 import build
    build.build()
    from paper_2606_06617_b300 import lr as _lr
    _lr.lib()
    return _lr


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pswf_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(lr):
    names = declared_functions()
    assert "pswf_execute" in names and len(names) >= 10
    L = lr.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(lr.SIGNATURES)


def test_default_parameters(lr):
    """c = log(3 / tol); h <= eta pi / k_c with eta = 0.5; grid sizes
    2^a 3^b 5^c 7^d; c_w = P pi (1 - eta/2); smallest P meeting tol / 3."""
    box = (31.0, 25.0, 40.0)
    info = lr.plan_params(box, (1, 6), r_c=4.0, tol=1e-5)
    assert info["c"] == pytest.approx(math.log(3e5), rel=1e-14)
    k_c = info["c"] / 4.0
    for L, M in zip(box, info["grid"]):
        assert L / M <= 0.5 * math.pi / k_c + 1e-12
        r = M
        for f in (2, 3, 5, 7):
            while r % f == 0:
                r //= f
        assert r == 1
    assert info["c_w"] == pytest.approx(info["P"] * math.pi * (1 - info["eta"] / 2), rel=1e-12)
    assert info["est_err_spread"] <= 1e-5 / 3
    smaller = lr.plan_params(box, (1, 6), r_c=4.0, tol=1e-5, P=info["P"] - 1)
    assert smaller["est_err_spread"] > 1e-5 / 3


def test_overrides_and_errors(lr):
    info = lr.plan_params((12, 12, 12), (1,), r_c=4.0, P=6, grid=24, c=12.0)
    assert info["P"] == 6 and info["grid"] == [24, 24, 24] and info["c"] == 12.0
    with pytest.raises(lr.PswfError) as e:
        lr.plan_params((12, 12, 12), (7,), r_c=4.0)
    assert e.value.status == -1
    with pytest.raises(lr.PswfError) as e:
        lr.plan_params((12, -1, 12), (1,), r_c=4.0)
    assert e.value.status == -1
    with pytest.raises(lr.PswfError) as e:
        lr.plan_params((12, 12, 12), (1,), r_c=0.0)
    assert e.value.status == -1
    with pytest.raises(lr.PswfError) as e:          # h k_c >= pi
        lr.plan_params((12, 12, 12), (1,), r_c=4.0, grid=10)
    assert e.value.status == -7
    assert lr.lib().pswf_strerror(-7).decode().startswith("tolerance")


@pytest.mark.parametrize("c", [1.0, 6.0, 12.611537753638338, 20.0])
def test_planner_pswf_agrees_with_oracle(lr, c):
    """The planner's psi_0 (Legendre expansion of the prolate operator) and the
    oracle's (Nystrom on the integral operator) are independent computations."""
    from oracle.pswf import PSWF
    info = lr.plan_params((10, 10, 10), (1,), r_c=4.0, c=c, grid=64, P=8)
    ps = PSWF(c)
    assert info["lambda0"] == pytest.approx(ps.lam0, rel=1e-12)
    assert info["C0"] == pytest.approx(ps.C0, rel=1e-12)
    # psi_0(1) is a cancellation of O(1) terms on both sides: absolute bound
    assert abs(info["est_err_band"] - float(ps(1.0))) < 1e-10
