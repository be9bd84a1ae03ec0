"""Parity of the CUDA path (through the C-ABI) with the O1 oracle.

Same seeded inputs and the same explicit parameters (c, c_w, P, grid) on both
sides; FP32 path within 2e-6 relative RMS on phi and forces (and relative
energy), FP64 path within 2e-9."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from gpu_helpers import TOL_FP32, TOL_FP64, run_gpu, run_oracle, window_cw
from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu

C_TOL = math.log(3.0 / 1e-5)


def _compare(g, o, tol, what=""):
    for c in range(len(o["E_ch"])):
        assert abs(g["E_ch"][c] - o["E_ch"][c]) <= tol * max(abs(o["E_ch"][c]), 1e-300) + 1e-13, \
            (what, c, g["E_ch"], o["E_ch"])
    assert rel_rms(g["phi"], o["phi"]) <= tol, (what, rel_rms(g["phi"], o["phi"]))
    assert rel_rms(g["F"], o["F"]) <= tol, (what, rel_rms(g["F"], o["F"]))


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP32), (1, TOL_FP64)])
def test_random_charges_24(precision, tol):
    """64 charges +-1 in L = 12, p = 1, P = 6, grid 24^3."""
    s = wl.random_charges()
    M = (24, 24, 24)
    cw = window_cw(s.box, M, 6, C_TOL, 4.0)
    g = run_gpu(s, 4.0, 6, M, C_TOL, cw, precision=precision)
    o = run_oracle(s, 4.0, 6, M, C_TOL, cw)
    _compare(g, o, tol, "random_charges")


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP32), (1, TOL_FP64)])
def test_water_3000(precision, tol):
    """1000 three-site molecules, L = 31, channels p = 1 and p = 6 (non-neutral),
    grid 64^3, P = 8."""
    s = wl.water_box()
    M = (64, 64, 64)
    cw = window_cw(s.box, M, 8, C_TOL, 4.0)
    g = run_gpu(s, 4.0, 8, M, C_TOL, cw, precision=precision)
    o = run_oracle(s, 4.0, 8, M, C_TOL, cw)
    _compare(g, o, tol, "water")


@pytest.mark.parametrize("P", [4, 5, 7])
def test_ragged_box_all_exponents(P):
    """Orthorhombic box with odd / mixed grid sizes (ragged tiles), six channels
    p = 1..6, atoms outside the primary cell (wrapped)."""
    rng = np.random.default_rng(7)
    box = (13.0, 17.5, 11.0)
    s = wl.random_system(300, box, (1, 2, 3, 4, 5, 6), seed=11, neutral=True)
    s.pos = s.pos + rng.integers(-3, 4, size=s.pos.shape) * np.asarray(box)   # far images
    M = (27, 35, 21)
    c = 11.0
    cw = window_cw(box, M, P, c, 4.5)
    g = run_gpu(s, 4.5, P, M, c, cw)
    o = run_oracle(s, 4.5, P, M, c, cw)
    _compare(g, o, TOL_FP32, f"ragged P={P}")


def test_float32_positions_small_grid():
    """float32 positions, grid smaller than the stencil tile (M = 6 < 8) and
    P = 4: the stencil wraps over the whole grid."""
    s = wl.random_system(40, (5.0, 5.0, 6.0), (1, 6), seed=3, neutral=False)
    s.pos = s.pos.astype(np.float32).astype(np.float64)
    M = (6, 6, 8)
    c = 6.0
    cw = window_cw(s.box, M, 4, c, 2.5)
    g = run_gpu(s, 2.5, 4, M, c, cw, pos_dtype="float32")
    o = run_oracle(s, 2.5, 4, M, c, cw)
    _compare(g, o, TOL_FP32, "small grid")


def test_single_atom_and_empty():
    """n = 1 (self-interaction through the periodic images only; its force is
    pure discretisation noise, so it is compared on an absolute scale) and n = 0."""
    import torch
    from paper_2606_06617_b300 import lr
    s = wl.random_system(1, (9.0, 9.0, 9.0), (1,), seed=5, neutral=False)
    M = (18, 18, 18)
    cw = window_cw(s.box, M, 6, 10.0, 3.0)
    g = run_gpu(s, 3.0, 6, M, 10.0, cw)
    o = run_oracle(s, 3.0, 6, M, 10.0, cw)
    assert abs(g["E"] - o["E"]) <= TOL_FP32 * abs(o["E"])
    assert rel_rms(g["phi"], o["phi"]) <= TOL_FP32
    scale = abs(s.q[0, 0] * o["phi"][0, 0]) / min(s.box)      # force scale q phi / L
    assert np.max(np.abs(g["F"] - o["F"])) <= TOL_FP32 * scale
    plan = lr.Plan(s.box, 16, s.ps, 3.0, grid=M, P=6)
    dev = torch.device("cuda", 0)
    plan.set_points(torch.zeros(0, 3, device=dev, dtype=torch.float64), torch.zeros(1, 0, device=dev))
    e, phi, f = plan.execute()
    plan.sync()
    assert float(e[-1]) == 0.0 and phi.numel() == 0 and f.numel() == 0


def test_energy_is_half_q_phi():
    """Quadratic form: E_k = 1/2 sum_i q_i phi_i for neutral channels (GPU only)."""
    s = wl.random_system(500, (14.0, 14.0, 14.0), (1, 2, 4, 6), seed=2, neutral=True)
    M = (28, 28, 28)
    cw = window_cw(s.box, M, 6, C_TOL, 4.0)
    g = run_gpu(s, 4.0, 6, M, C_TOL, cw)
    half = 0.5 * np.sum(s.q * g["phi"], axis=1)
    np.testing.assert_allclose(g["E_ch"], half, rtol=2e-6)


def test_nonfinite_positions_reported():
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    plan = lr.Plan((10.0, 10.0, 10.0), 8, (1,), 3.0, grid=16, P=4)
    pos = torch.rand(8, 3, device=dev, dtype=torch.float64) * 10
    pos[3, 1] = float("nan")
    plan.set_points(pos, torch.randn(1, 8, device=dev))
    with pytest.raises(lr.PswfError) as ei:
        plan.sync()
    assert ei.value.status == -6
    plan.set_points(torch.rand(8, 3, device=dev, dtype=torch.float64), torch.randn(1, 8, device=dev))
    plan.execute()
    plan.sync()


def test_compute_host_matches_device_path():
    """pswf_compute_host (host buffers, copies inside) equals the device path."""
    s = wl.water_box(n_side=6, L=18.6, seed=1)
    M = (36, 36, 36)
    cw = window_cw(s.box, M, 6, C_TOL, 4.0)
    g = run_gpu(s, 4.0, 6, M, C_TOL, cw)
    e, phi, f = g["plan"].compute_host(s.pos, s.q)
    np.testing.assert_allclose(e[:-1], g["E_ch"], rtol=1e-6)
    assert rel_rms(phi, g["phi"]) < 1e-6 and rel_rms(f, g["F"]) < 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_compute_host_chunked_matches_device_path(precision):
    """300,000 atoms: the host path splits copies and conversions into chunks
    over several threads; results equal the device path on the same plan up
    to the order of the flush's global atomics (float sums, ~1e-8)."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.random_system(300000, (60.0, 62.0, 64.0), (1, 6, 4), seed=13, neutral=True)
    plan = lr.Plan(s.box, s.n, s.ps, 6.0, P=6, grid=(64, 64, 64), precision=precision, device=dev)
    plan.set_points(torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=plan.dtype, device=dev))
    e0, phi0, f0 = plan.execute()
    plan.sync()
    e, phi, f = plan.compute_host(s.pos, s.q)
    np.testing.assert_allclose(e, e0.cpu().numpy(), rtol=1e-6)
    assert rel_rms(phi, phi0.cpu().double().numpy()) < 1e-6
    assert rel_rms(f, f0.cpu().double().numpy()) < 1e-6


def _pinned(a):
    """A numpy array in page-locked host memory holding a copy of a (same
    dtype, float32 or float64)."""
    import torch
    t = torch.empty(a.shape, dtype=torch.float32 if a.dtype == np.float32 else torch.float64).pin_memory()
    out = t.numpy()
    out[...] = a
    return out, t   # the caller keeps t alive while out is in use


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("pinned", ["all", "inputs", "outputs"])
def test_compute_host_pinned_matches_device_path(precision, pinned):
    """Page-locked caller arrays are copied directly (positions in; potentials
    and forces out, widened on the device in FP32 plans); mixed pinned and
    pageable arrays take each side's own route.  Results equal the device
    path on the same plan up to the flush order."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.random_system(300000, (60.0, 62.0, 64.0), (1, 6, 4, 2), seed=17, neutral=True)
    plan = lr.Plan(s.box, s.n, s.ps, 6.0, P=6, grid=(64, 64, 64), precision=precision, device=dev)
    plan.set_points(torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=plan.dtype, device=dev))
    e0, phi0, f0 = plan.execute()
    plan.sync()
    keep = []
    pos, q = s.pos, s.q
    if pinned in ("all", "inputs"):
        (pos, t1), (q, t2) = _pinned(s.pos), _pinned(s.q)
        keep += [t1, t2]
    out = (np.zeros(len(s.ps) + 1), np.zeros((len(s.ps), s.n)), np.zeros((s.n, 3)))
    if pinned in ("all", "outputs"):
        (ph, t3), (ff, t4) = _pinned(out[1]), _pinned(out[2])
        keep += [t3, t4]
        out = (out[0], ph, ff)
    for _ in range(2):   # a second call reuses the plan's buffers
        e, phi, f = plan.compute_host(pos, q, out=out)
        np.testing.assert_allclose(e, e0.cpu().numpy(), rtol=1e-6)
        assert rel_rms(phi, phi0.cpu().double().numpy()) < 1e-6
        assert rel_rms(f, f0.cpu().double().numpy()) < 1e-6



@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("pinned", [True, False])
def test_compute_host_real_matches_device_path(precision, pinned):
    """pswf_compute_host_real: charges, potentials and forces in the plan's
    precision, copied as they are when page-locked and through the staging
    buffers otherwise; equal to the device path on the same plan up to the
    flush order."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.random_system(300000, (60.0, 62.0, 64.0), (1, 6, 4, 2), seed=18, neutral=True)
    plan = lr.Plan(s.box, s.n, s.ps, 6.0, P=6, grid=(64, 64, 64), precision=precision, device=dev)
    rdt = np.float32 if precision == 0 else np.float64
    qr = s.q.astype(rdt)
    plan.set_points(torch.tensor(s.pos, device=dev), torch.tensor(qr, device=dev))
    e0, phi0, f0 = plan.execute()
    plan.sync()
    keep = []
    pos, q = s.pos, qr
    out = (np.zeros(len(s.ps) + 1), np.zeros((len(s.ps), s.n), dtype=rdt), np.zeros((s.n, 3), dtype=rdt))
    if pinned:
        (pos, t1), (q, t2), (ph, t3), (ff, t4) = _pinned(s.pos), _pinned(qr), _pinned(out[1]), _pinned(out[2])
        keep += [t1, t2, t3, t4]
        out = (out[0], ph, ff)
    for _ in range(2):
        e, phi, f = plan.compute_host(pos, q, out=out, real=True)
        assert phi.dtype == rdt and f.dtype == rdt
        np.testing.assert_allclose(e, e0.cpu().numpy(), rtol=1e-6)
        assert rel_rms(phi.astype(np.float64), phi0.cpu().double().numpy()) < 1e-6
        assert rel_rms(f.astype(np.float64), f0.cpu().double().numpy()) < 1e-6
    e, phi, f = plan.compute_host(pos, q, phi=False, forces=False, real=True)
    assert phi is None and f is None
    np.testing.assert_allclose(e, e0.cpu().numpy(), rtol=1e-6)

def test_self_energy_matches_oracle():
    """E_self from the device FP64 reduction of the (FP32-stored) charges."""
    s = wl.water_box(n_side=5, L=15.5, seed=2)
    M = (32, 32, 32)
    cw = window_cw(s.box, M, 6, C_TOL, 4.0)
    g = run_gpu(s, 4.0, 6, M, C_TOL, cw)
    o = run_oracle(s, 4.0, 6, M, C_TOL, cw)
    q32 = s.q.astype(np.float32).astype(np.float64)
    from oracle.mollifiers import Mollifier
    m = Mollifier(C_TOL, 4.0)
    ref32 = [m.self_coef(p) * float(np.sum(q32[c] ** 2)) for c, p in enumerate(s.ps)]
    # self_coef: planner (Legendre) vs oracle (Nystrom) derivatives of psi_0 at 0
    np.testing.assert_allclose(g["plan"].self_energy(), ref32, rtol=1e-9)
    np.testing.assert_allclose(g["plan"].self_energy(), o["self"], rtol=1e-7)


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP32), (1, TOL_FP64)])
def test_ionic_melt_subbox(precision, tol):
    """The ionic-melt workload shape (K = 4 channels p = 1, 2, 4, 6, P = 7,
    r_c = 7, tol 1e-5) on a density-matched 64^3 sub-box (19,418 atoms,
    L = 58.33): the same kernels and channel chunking as the 384^3 run."""
    L = 350.0 * 64 / 384
    n = int(round(4194304 * (L / 350.0) ** 3))
    s = wl.ionic_melt(n, L, seed=3)
    M = (64, 64, 64)
    c = math.log(3.0 / 1e-5)
    cw = window_cw(s.box, M, 7, c, 7.0)
    g = run_gpu(s, 7.0, 7, M, c, cw, precision=precision)
    o = run_oracle(s, 7.0, 7, M, c, cw)
    _compare(g, o, tol, "melt sub-box")


@pytest.mark.parametrize("precision,tol", [(0, 2e-5), (1, 1e-7)])
def test_virial_matches_oracle(precision, tol):
    """Diagonal virial W_cd = -L_d dE_c/dL_d (PSWF_FLAG_VIRIAL) against the
    oracle's central differences of E_c under box scaling, all six
    exponents, an orthorhombic box."""
    import torch
    from oracle.grid import DiscretePSWF, GridConfig
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    box = (12.0, 13.5, 11.0)
    s = wl.random_system(200, box, (1, 2, 3, 4, 5, 6), seed=31, neutral=False)
    M = (24, 27, 22)
    c = 11.0
    cw = window_cw(box, M, 7, c, 4.5)
    plan = lr.Plan(box, s.n, s.ps, 4.5, c=c, c_w=cw, P=7, grid=M, precision=precision,
                   flags=lr.PSWF_FLAG_VIRIAL, device=dev)
    plan.set_points(torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=plan.dtype, device=dev))
    e, _, _ = plan.execute()
    W = plan.virial().cpu().numpy()
    plan.sync()
    ref = DiscretePSWF(GridConfig(box, M, 7, c, 4.5, s.ps, c_w=cw)).virial_fd(s.pos, s.q)
    assert rel_rms(W, ref) <= tol, (rel_rms(W, ref), W, ref)
    E = e.cpu().numpy()
    for ci in range(6):
        # per channel, relative to the channel's energy scale as well (its
        # virial can be much smaller than its energy)
        bound = 3 * tol * max(np.abs(ref[ci]).max(), abs(E[ci]))
        assert np.abs(W[ci] - ref[ci]).max() <= bound, (ci, W[ci], ref[ci])


def test_virial_batch_plan():
    """Batch plans: per-slot virials equal single-structure plans' (FP32)."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    structs = [wl.random_system(n, b, (1, 6), seed=n, neutral=True)
               for n, b in ((80, (9.0, 10.0, 9.5)), (150, (11.0, 9.0, 12.0)))]
    M = (28, 28, 28)
    plan = lr.BatchPlan((12.0, 12.0, 12.0), 4, 230, 2, (1, 6), 4.0, grid=M, flags=lr.PSWF_FLAG_VIRIAL, device=dev)
    off = np.array([0, 80, 230], dtype=np.int64)
    plan.set_points(np.array([s.box for s in structs]), np.array([s.ps for s in structs], dtype=np.int32), off,
                    torch.tensor(np.concatenate([s.pos for s in structs]), device=dev),
                    torch.tensor(np.concatenate([s.q for s in structs], axis=1), dtype=torch.float32, device=dev))
    plan.execute()
    W = plan.virial().cpu().numpy()
    info = plan.info
    for i, s in enumerate(structs):
        sp = lr.Plan(s.box, s.n, s.ps, 4.0, c=info["c"], c_w=info["c_w"], P=info["P"], grid=M,
                     flags=lr.PSWF_FLAG_VIRIAL, device=dev)
        sp.set_points(torch.tensor(s.pos, device=dev), torch.tensor(s.q, dtype=torch.float32, device=dev))
        sp.execute()
        assert np.allclose(W[i], sp.virial().cpu().numpy(), rtol=1e-5, atol=1e-8)
    assert np.all(W[2:] == 0.0)
