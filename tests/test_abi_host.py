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


def _header_defines():
    src = open(os.path.join(ROOT, "include", "pswf_lr.h")).read()
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"#define\s+(PSWF_\w+)\s+\(?(-?\d+)\)?", src)}


def test_binding_constants_match_header(lr):
    """Flags, transforms, stage names and their count in the binding are the
    header's."""
    d = _header_defines()
    for name in ("PSWF_FLAG_BACKWARD", "PSWF_FLAG_VIRIAL", "PSWF_FLAG_REAL_SPACE", "PSWF_TRANSFORM_FULL",
                 "PSWF_TRANSFORM_PRUNED", "PSWF_TRANSFORM_PRUNED_X", "PSWF_TRANSFORM_OWN"):
        assert getattr(lr, name) == d[name], name
    assert lr.NSTAGE == d["PSWF_NSTAGE"] == len(lr.STAGES)
    for i, stage in enumerate(lr.STAGES):
        assert d["PSWF_STAGE_" + stage.upper()] == i, stage


def test_info_struct_layout_matches_header(lr, tmp_path):
    """sizeof(pswf_info) and the offsets of its last fields, from a C program
    compiled against the header, equal the ctypes structure's."""
    import ctypes
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    c = tmp_path / "layout.c"
    c.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "pswf_lr.h"\n'
                 'int main(void) { printf("%zu %zu %zu %zu\\n", sizeof(pswf_info), offsetof(pswf_info, cell), '
                 'offsetof(pswf_info, deg_real), offsetof(pswf_info, nkx)); return 0; }\n')
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    size, off_cell, off_deg, off_nkx = map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                                                check=True).stdout.split())
    assert ctypes.sizeof(lr.PswfInfo) == size
    assert lr.PswfInfo.cell.offset == off_cell
    assert lr.PswfInfo.deg_real.offset == off_deg
    assert lr.PswfInfo.nkx.offset == off_nkx


def test_status_strings(lr):
    L = lr.lib()
    d = _header_defines()
    import ctypes
    L.pswf_strerror.restype = ctypes.c_char_p
    assert b"2048" in L.pswf_strerror(d["PSWF_ECELL"])
    for name in ("PSWF_EINVAL", "PSWF_ESTATE", "PSWF_ENONFINITE"):
        assert L.pswf_strerror(d[name])


def test_source_digest_ignores_comments():
    """The digest that keys committed traffic records to a kernel's code does
    not change with comments or whitespace, and does change with code."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    a = "int f(int x) {\n  return x + 1;  // one\n}\n"
    b = "/* header */\nint f(int x) {\n    return x + 1;\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.code_only(a) == bench.code_only(b)
    assert bench.code_only(a) != bench.code_only(c)
