"""Own transform passes of single FP32 plans (PSWF_TRANSFORM_PRUNED_X: own x
passes, cuFFT (z, y); PSWF_TRANSFORM_OWN: every pass own).

When the band |k| < k_c reaches only the lowest x frequencies, the x passes
of the 3-D transform are this library's kernels (rows of Mx = 32 N1 points,
only kx < nkx written and read).  Every row-length class is covered (N1
even, odd, a power of two, 15 = 3 x 5) on a ragged (y, z) grid (37 x 19: a
partial 32-row chunk) at liquid density (0.1 atoms per cubic Angstrom), two
cases near the pruning limit nkx = 3/4 (Mx/2 + 1).

Reference: the O1 oracle.  In these long thin boxes the FP32 path's error
grows with Mx whichever transform runs (FP32 against the FP64 path: 0.8e-6
at Mx = 64, 5e-6 at Mx = 512), so each case also runs the same structure
through a batch plan (full 3-D cuFFT transform, FP32) and the pruned kernels
must be within 2e-6 of the oracle or no worse than 1.25 times that path's
own error (plus 2e-7)."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from gpu_helpers import TOL_FP32, run_gpu, run_oracle, window_cw
from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu

C_TOL = math.log(3.0 / 1e-5)
R_C = 4.0


def _full_transform(s, info, M):
    """The same structure through a 2-slot batch plan (cuFFT 3-D transform)."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    bp = lr.BatchPlan(tuple(s.box), 2, s.n, len(s.ps), s.ps, R_C, c=C_TOL, c_w=info["c_w"], P=info["P"], grid=M,
                      device=dev)
    assert bp.info["transform"] == lr.PSWF_TRANSFORM_FULL
    bp.set_points(np.array([s.box]), np.array([s.ps], dtype=np.int32), np.array([0, s.n], dtype=np.int64),
                  torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=torch.float32, device=dev))
    e, phi, f = bp.execute()
    bp.sync()
    return e.cpu().numpy()[0], phi.cpu().double().numpy()[:, :s.n], f.cpu().double().numpy()[:s.n]


def _bound(err_full):
    return max(TOL_FP32, 1.25 * err_full + 2e-7)


@pytest.mark.parametrize("n1,hx", [(2, 0.3), (3, 0.3), (3, 0.7), (5, 0.3), (7, 0.3), (8, 0.3), (12, 0.3),
                                   (12, 0.7), (15, 0.3), (16, 0.3)])
def test_pruned_x_matches_oracle(n1, hx):
    from paper_2606_06617_b300 import lr
    Mx = 32 * n1
    M = (Mx, 37, 19)
    box = (hx * Mx, 13.0, 6.6)
    nat = int(0.1 * box[0] * box[1] * box[2])
    s = wl.random_system(nat, box, (1, 6), seed=100 + n1, neutral=bool(n1 % 2))
    s.pos = s.pos + np.random.default_rng(n1).integers(-1, 2, size=s.pos.shape) * np.asarray(box)
    cw = window_cw(s.box, M, 6, C_TOL, R_C)
    g = run_gpu(s, R_C, 6, M, C_TOL, cw, precision=0)
    info = g["info"]
    assert info["transform"] == lr.PSWF_TRANSFORM_PRUNED_X, info
    assert 0 < info["nkx"] * 4 <= (Mx // 2 + 1) * 3
    o = run_oracle(s, R_C, 6, M, C_TOL, cw)
    e_f, phi_f, f_f = _full_transform(s, info, M)
    for c in range(2):
        ref = abs(o["E_ch"][c])
        bound = _bound(abs(e_f[c] - o["E_ch"][c]) / ref)
        assert abs(g["E_ch"][c] - o["E_ch"][c]) <= bound * ref, (c, g["E_ch"], o["E_ch"], e_f)
    err_phi, err_f = rel_rms(g["phi"], o["phi"]), rel_rms(g["F"], o["F"])
    assert err_phi <= _bound(rel_rms(phi_f, o["phi"])), (err_phi, rel_rms(phi_f, o["phi"]))
    assert err_f <= _bound(rel_rms(f_f, o["F"])), (err_f, rel_rms(f_f, o["F"]))
    if n1 <= 5:
        assert err_phi <= TOL_FP32 and err_f <= TOL_FP32


def test_own_transform_cubic_melt_box():
    """Cubic ionic-melt box (K = 4, P = 7, r_c = 7) on 96^3: every pass is
    this library's (x, z, multiplier fused with y); plain FP32 budget."""
    from paper_2606_06617_b300 import lr
    L = 350.0 * 96 / 384
    s = wl.ionic_melt(int(round(4194304 * (L / 350.0) ** 3)), L, seed=4)
    M = (96, 96, 96)
    c = math.log(3.0 / 1e-5)
    cw = window_cw(s.box, M, 7, c, 7.0)
    g = run_gpu(s, 7.0, 7, M, c, cw, precision=0)
    assert g["info"]["transform"] == lr.PSWF_TRANSFORM_OWN
    o = run_oracle(s, 7.0, 7, M, c, cw)
    for ch in range(4):
        assert abs(g["E_ch"][ch] - o["E_ch"][ch]) <= TOL_FP32 * abs(o["E_ch"][ch])
    assert rel_rms(g["phi"], o["phi"]) <= TOL_FP32
    assert rel_rms(g["F"], o["F"]) <= TOL_FP32


@pytest.mark.parametrize("n1", [(2, 2, 2), (3, 4, 5), (12, 2, 3), (5, 7, 2), (16, 3, 2), (7, 16, 2)])
def test_own_transform_matches_oracle(n1):
    """All passes own (PSWF_TRANSFORM_OWN) on grids 32 (N1x, N1y, N1z): the
    column z pass and the fused y multiplier for every length class, the
    bit-reversed kz order of the z pass decoded by the multiplier."""
    from paper_2606_06617_b300 import lr
    M = tuple(32 * k for k in n1)
    h = (0.3, 0.42, 0.45)
    box = tuple(hd * m for hd, m in zip(h, M))
    nat = int(0.1 * box[0] * box[1] * box[2])
    s = wl.random_system(nat, box, (1, 6), seed=200 + sum(n1), neutral=bool(n1[0] % 2))
    cw = window_cw(s.box, M, 6, C_TOL, R_C)
    g = run_gpu(s, R_C, 6, M, C_TOL, cw, precision=0)
    info = g["info"]
    assert info["transform"] == lr.PSWF_TRANSFORM_OWN, info
    o = run_oracle(s, R_C, 6, M, C_TOL, cw)
    e_f, phi_f, f_f = _full_transform(s, info, M)
    for c in range(2):
        ref = abs(o["E_ch"][c])
        bound = _bound(abs(e_f[c] - o["E_ch"][c]) / ref)
        assert abs(g["E_ch"][c] - o["E_ch"][c]) <= bound * ref, (c, g["E_ch"], o["E_ch"], e_f)
    err_phi, err_f = rel_rms(g["phi"], o["phi"]), rel_rms(g["F"], o["F"])
    assert err_phi <= _bound(rel_rms(phi_f, o["phi"])), (err_phi, rel_rms(phi_f, o["phi"]))
    assert err_f <= _bound(rel_rms(f_f, o["F"])), (err_f, rel_rms(f_f, o["F"]))


def test_pruned_x_and_cufft_x_agree():
    """The same structure on the FP64 plan (pruned, cuFFT x passes) and the
    FP32 plan (own x passes): FP32 rounding apart."""
    from paper_2606_06617_b300 import lr
    M = (128, 37, 19)
    box = (38.4, 13.0, 6.6)
    s = wl.random_system(320, box, (1, 6), seed=5, neutral=True)
    cw = window_cw(s.box, M, 6, C_TOL, R_C)
    g32 = run_gpu(s, R_C, 6, M, C_TOL, cw, precision=0)
    g64 = run_gpu(s, R_C, 6, M, C_TOL, cw, precision=1)
    assert g32["info"]["transform"] == lr.PSWF_TRANSFORM_PRUNED_X
    assert g64["info"]["transform"] == lr.PSWF_TRANSFORM_PRUNED
    assert g32["info"]["nkx"] == g64["info"]["nkx"]
    assert rel_rms(g32["phi"], g64["phi"]) <= TOL_FP32
    assert rel_rms(g32["F"], g64["F"]) <= TOL_FP32


@pytest.mark.parametrize("n1", [(2, 2, 3), (5, 2, 2), (7, 3, 2), (15, 2, 2), (16, 2, 3)])
def test_quadruple_inverse_x_matches_oracle(n1):
    """Four channels (p = 1, 2, 4, 6) on own-transform grids: FP32 plans
    with K a multiple of 4, P <= 8 and no backward end the inverse
    transform with the pass that writes Psi as channel quadruples (one y
    row per warp, two complex rows per warp), which the gather reads as
    16-byte words; every row-length class, ragged y rows included."""
    from paper_2606_06617_b300 import lr
    M = tuple(32 * k for k in n1)
    h = (0.3, 0.42, 0.45)
    box = tuple(hd * m for hd, m in zip(h, M))
    nat = int(0.1 * box[0] * box[1] * box[2])
    s = wl.random_system(nat, box, (1, 2, 4, 6), seed=300 + sum(n1), neutral=bool(n1[0] % 2))
    cw = window_cw(s.box, M, 6, C_TOL, R_C)
    g = run_gpu(s, R_C, 6, M, C_TOL, cw, precision=0)
    info = g["info"]
    assert info["transform"] == lr.PSWF_TRANSFORM_OWN, info
    o = run_oracle(s, R_C, 6, M, C_TOL, cw)
    e_f, phi_f, f_f = _full_transform(s, info, M)
    for c in range(4):
        ref = abs(o["E_ch"][c])
        bound = _bound(abs(e_f[c] - o["E_ch"][c]) / ref)
        assert abs(g["E_ch"][c] - o["E_ch"][c]) <= bound * ref, (c, g["E_ch"], o["E_ch"], e_f)
    err_phi, err_f = rel_rms(g["phi"], o["phi"]), rel_rms(g["F"], o["F"])
    assert err_phi <= _bound(rel_rms(phi_f, o["phi"])), (err_phi, rel_rms(phi_f, o["phi"]))
    assert err_f <= _bound(rel_rms(f_f, o["F"])), (err_f, rel_rms(f_f, o["F"]))
