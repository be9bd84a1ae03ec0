"""Real-space complement on the GPU (pswf_real_space).

* Against the oracle's real-space sum (oracle/realspace.py, FP64 autograd):
  per-channel energies, potentials and the total force, all six exponents,
  atoms far outside the box (FP64 1e-10, FP32 2e-6 relative RMS).
* The complete lattice sum from the GPU alone, reciprocal part
  (pswf_execute) + real-space part - self energy, against Ewald (O3) on the
  ionic-melt sub-box at its benchmarked parameters: the 1e-5 relative force
  tolerance the parameters are chosen for.
* The same on the 64-charge box (L = 12 A, p = 1, r_c = 4) and the
  water-like box at its benchmarked parameters (forces within 1e-5 of
  Ewald, energies within 1e-5 of the per-atom energy scale), and the NaCl
  rock-salt crystal's energy against the Madelung constant.
* The full-size melt (4,194,304 atoms, r_c = 7, K = 4), the configuration
  the benchmark times: potentials of every channel and forces of seeded
  sampled atoms against the oracle's per-atom neighbour sums.
* General cells: a sheared cell against the oracle's lattice sum (FP64
  1e-10, FP32 2e-6), and the melt sub-box rotated into a general cell:
  reciprocal + real space - self against Ewald of the unrotated box, forces
  rotated, within 1e-5.
* Cells with a height below 3 r_c (no cell list: the direct sum over all
  pairs and images): a box at r_c = L/2 and a small sheared cell with r_c
  above its heights, against the oracle (FP64 1e-10, FP32 2e-6).
* Non-finite positions are reported (PSWF_ENONFINITE) in both modes.
* Plans without PSWF_FLAG_REAL_SPACE, or direct-sum plans above 16384 atoms,
  are refused; no atoms give zero energies; a cell holding more than 2048 atoms
  is reported (PSWF_ECELL) by the next synchronising call."""
import math

import numpy as np
import pytest

from conftest import rel_rms
from gpu_helpers import TOL_FP32, window_cw
from paper_2606_06617_b300 import workloads as wl

pytestmark = pytest.mark.gpu

C = math.log(3.0 / 1e-5)


@pytest.mark.parametrize("ps", [(1, 2, 3, 4, 5, 6), (1,), (6, 1, 4, 2)])
@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, TOL_FP32)])
def test_real_space_matches_oracle(precision, tol, ps):
    """Cell list (3 x 3 x 3 at r_c = 4), atoms up to two boxes outside the
    cell.  One channel takes the FP32 plans' direct scatter (its record does
    not fit an accumulator row), two to sixteen the record scatter and
    unpack."""
    import torch
    from oracle.realspace import real_space
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    box = (13.0, 14.5, 12.5)
    r_c = 4.0
    s = wl.random_system(300, box, ps, seed=41, neutral=False)
    s.pos = s.pos + np.random.default_rng(2).integers(-2, 3, size=s.pos.shape) * np.asarray(box)
    plan = lr.Plan(box, s.n, s.ps, r_c, c=C, P=6, grid=(28, 30, 26), precision=precision,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    e, phi, f = plan.real_space(torch.tensor(s.pos, device=dev), torch.tensor(s.q, device=dev))
    plan.sync()
    e, phi, f = e.cpu().numpy(), phi.cpu().double().numpy(), f.cpu().double().numpy()
    F = np.zeros((s.n, 3))
    for c, p in enumerate(s.ps):
        o = real_space(s.pos, s.q[c], box, p, C, r_c)
        assert abs(e[c] - o["E"]) <= tol * abs(o["E"]), (c, e[c], o["E"])
        assert rel_rms(phi[c], o["phi"]) <= tol, (c, rel_rms(phi[c], o["phi"]))
        F += o["F"]
    assert rel_rms(f, F) <= tol, rel_rms(f, F)
    assert abs(e[-1] - e[:-1].sum()) <= 1e-12 * abs(e[:-1]).sum()


@pytest.mark.parametrize("precision,tol,reach", [(1, 1e-10, 50), (0, TOL_FP32, 5000)])
def test_real_space_distant_images(precision, tol, reach):
    """Atoms moved by up to +-reach box lengths, others exactly on the cell's
    faces or just below zero: the binning wraps them (FP32 plans form the
    fixed-point cell coordinates as one rounded integer and take the cell
    modulo n_c), and the results equal the oracle's on the unmoved atoms.
    (Moving an atom by 5000 boxes already rounds its double coordinates by
    1.5e-11 A, beyond the FP64 bound's reach on close pairs; 50 boxes round
    them by 1e-13 A.)"""
    import torch
    from oracle.realspace import real_space
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    box = (13.0, 14.5, 12.5)
    r_c = 4.0
    s = wl.random_system(300, box, (1, 4), seed=43, neutral=False)
    rng = np.random.default_rng(5)
    base = s.pos.copy()
    base[:3] = [[0.0, 0.0, 0.0], [box[0], 7.0, 3.0], [5.0, -1e-12, box[2]]]
    moved = base + rng.integers(-reach, reach + 1, size=base.shape) * np.asarray(box)
    moved[:3] = base[:3]
    plan = lr.Plan(box, s.n, s.ps, r_c, c=C, P=6, grid=(28, 30, 26), precision=precision,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    e, phi, f = plan.real_space(torch.tensor(moved, device=dev), torch.tensor(s.q, device=dev))
    plan.sync()
    e, phi, f = e.cpu().numpy(), phi.cpu().double().numpy(), f.cpu().double().numpy()
    F = np.zeros((s.n, 3))
    for c, p in enumerate(s.ps):
        o = real_space(base, s.q[c], box, p, C, r_c)
        assert abs(e[c] - o["E"]) <= tol * abs(o["E"]), (c, e[c], o["E"])
        assert rel_rms(phi[c], o["phi"]) <= tol, (c, rel_rms(phi[c], o["phi"]))
        F += o["F"]
    assert rel_rms(f, F) <= tol, rel_rms(f, F)


@pytest.mark.parametrize("precision", [1, 0])
def test_gpu_total_matches_ewald(precision):
    """Ionic melt parameters (r_c = 7, c = log(3e5), P = 7, h = 0.911 A) on a
    density-matched sub-box (L = 21.875 A, 24^3, 1024 atoms)."""
    import torch
    from oracle.ewald import ewald
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    L = 350.0 * 24 / 384
    s = wl.ionic_melt(int(round(4194304 * (L / 350.0) ** 3)), L, seed=3)
    M = (24, 24, 24)
    r_c = 7.0
    cw = window_cw(s.box, M, 7, C, r_c)
    plan = lr.Plan(s.box, s.n, s.ps, r_c, c=C, c_w=cw, P=7, grid=M, precision=precision,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    pos = torch.tensor(s.pos, device=dev)
    q = torch.tensor(s.q, dtype=plan.dtype, device=dev)
    plan.set_points(pos, q)
    e_k, phi_k, f_k = plan.execute()
    e_r, phi_r, f_r = plan.real_space(pos, q)
    plan.sync()
    self_e = plan.self_energy()
    F = f_k.cpu().double().numpy() + f_r.cpu().double().numpy()
    E = e_k.cpu().numpy()[:-1] + e_r.cpu().numpy()[:-1] - self_e
    F_ew = np.zeros_like(F)
    for c, p in enumerate(s.ps):
        ew = ewald(s.pos, s.q[c], s.box, p)
        F_ew += ew["F"]
        assert abs(E[c] - ew["E"]) <= 1e-5 * max(abs(ew["E"]), 1e-3 * np.abs(s.q[c]).sum()), (c, E[c], ew["E"])
    assert rel_rms(F, F_ew) <= 1e-5, rel_rms(F, F_ew)


def test_real_space_refusals():
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    plan = lr.Plan((13.0, 13.0, 13.0), 10, (1,), 4.0, P=6, grid=(26, 26, 26), device=dev)
    pos = torch.zeros(10, 3, dtype=torch.float64, device=dev)
    q = torch.zeros(1, 10, dtype=torch.float32, device=dev)
    with pytest.raises(lr.PswfError) as e:
        plan.real_space(pos, q)
    assert e.value.status == -8
    with pytest.raises(lr.PswfError) as e:   # a height below 3 r_c: direct sum, at most 16384 atoms
        lr.Plan((11.0, 13.0, 13.0), 20000, (1,), 4.0, P=6, grid=(26, 26, 26), flags=lr.PSWF_FLAG_REAL_SPACE,
                device=dev)
    assert e.value.status == -1


def _nearest(pos, i, box):
    d = pos - pos[i]
    d -= box * np.round(d / box)
    r2 = np.einsum("nd,nd->n", d, d)
    r2[i] = np.inf
    return float(np.sqrt(r2.min()))


@pytest.mark.slow
@pytest.mark.parametrize("precision,tol", [(0, TOL_FP32), (1, 1e-10)])
def test_full_size_melt_sampled_atoms(precision, tol):
    """48 seeded atoms of the full-size melt.  Uniform random positions put
    a few atoms closer than 0.1 A to a neighbour; there the FP32 path's
    fixed-point displacement (w / 2^29 = 1.3e-8 A) bounds a term's relative
    error by p 1.3e-8 / r (8e-7 at p = 6, r = 0.1 A), so FP32 samples are
    drawn among atoms with no neighbour closer than 0.1 A (all but about
    4e-4 of them); FP64 samples are any atoms."""
    import torch
    from oracle.mollifiers import Mollifier
    from oracle.realspace import real_space_atoms
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.ionic_melt(4194304, 350.0, seed=0)
    box = np.asarray(s.box)
    r_c = 7.0
    c = math.log(3.0 / 1e-5)
    plan = lr.Plan(s.box, s.n, s.ps, r_c, tol=1e-5, P=7, grid=384, precision=precision,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    e, phi, f = plan.real_space(torch.tensor(s.pos, device=dev), torch.tensor(s.q, device=dev))
    plan.sync()
    phi, f = phi.cpu().double().numpy(), f.cpu().double().numpy()
    rng = np.random.default_rng(17)
    idx = []
    while len(idx) < 48:
        i = int(rng.integers(s.n))
        if precision == 1 or _nearest(s.pos, i, box) >= 0.1:
            idx.append(i)
    moll = Mollifier(c, r_c)
    F = np.zeros((len(idx), 3))
    for ch, p in enumerate(s.ps):
        o_phi, o_F = real_space_atoms(idx, s.pos, s.q[ch], box, p, c, r_c, moll)
        assert rel_rms(phi[ch, idx], o_phi) <= tol, (ch, rel_rms(phi[ch, idx], o_phi))
        F += o_F
    assert rel_rms(f[idx], F) <= tol, rel_rms(f[idx], F)
    assert abs(e.cpu().numpy()[-1] - e.cpu().numpy()[:-1].sum()) <= 1e-12 * np.abs(e.cpu().numpy()[:-1]).sum()


def _close_pair_bounds(idx, pos, q, box, p, r_c, moll, rel, dx):
    """Per-atom error bounds of the FP32 path for atoms with close
    neighbours: each pair term (|q_j f_p(r)| for phi, |q_i q_j f_p'(r)| for
    the force components) carries a relative error rel (rounding) plus the
    one of the fixed-point displacement, dx = 1.3e-8 A: (p + 1) dx / r for
    f_p ~ r^-p and (p + 2) dx / r for its derivative."""
    b_phi = np.zeros(len(idx))
    b_f = np.zeros(len(idx))
    for k, i in enumerate(idx):
        d = pos - pos[i]
        d -= box * np.round(d / box)
        r2 = np.einsum("nd,nd->n", d, d)
        nb = np.nonzero((r2 < r_c * r_c) & (r2 > 0.0))[0]
        r = np.sqrt(r2[nb])
        f = (1.0 - moll.G(p, r)) / r ** p
        h = 1e-6 * r
        fp = ((1.0 - moll.G(p, r + h)) / (r + h) ** p - (1.0 - moll.G(p, r - h)) / (r - h) ** p) / (2 * h)
        b_phi[k] = np.sum(np.abs(q[nb] * f) * (rel + (p + 1) * dx / r))
        b_f[k] = np.sum(np.abs(q[i] * q[nb] * fp) * (rel + (p + 2) * dx / r))
    return b_phi, b_f


@pytest.mark.slow
def test_full_size_melt_close_pairs():
    """Atoms of the full-size melt with a neighbour closer than 0.1 A (the
    ones the sampled test leaves out in FP32), element by element against the
    oracle within their own bounds: relative rounding 2e-6 on every pair term
    plus the fixed-point displacement's p 1.3e-8 A / r (section on the
    real-space records).  The closest pairs of 4.2M uniform atoms are ~0.01 A
    apart, where 1/r^6 terms dominate the potential."""
    import torch
    from scipy.spatial import cKDTree
    from oracle.mollifiers import Mollifier
    from oracle.realspace import real_space_atoms
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    s = wl.ionic_melt(4194304, 350.0, seed=0)
    box = np.asarray(s.box)
    r_c = 7.0
    c = math.log(3.0 / 1e-5)
    plan = lr.Plan(s.box, s.n, s.ps, r_c, tol=1e-5, P=7, grid=384, precision=0,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    e, phi, f = plan.real_space(torch.tensor(s.pos, device=dev), torch.tensor(s.q, device=dev))
    plan.sync()
    phi, f = phi.cpu().double().numpy(), f.cpu().double().numpy()
    wrapped = s.pos - box * np.floor(s.pos / box)
    pairs = cKDTree(wrapped, boxsize=box).query_pairs(0.1, output_type="ndarray")
    assert len(pairs) > 100
    close = np.unique(pairs.ravel())
    order = np.argsort(np.linalg.norm(np.diff(wrapped[pairs], axis=1)[:, 0] -
                                      box * np.round(np.diff(wrapped[pairs], axis=1)[:, 0] / box), axis=1))
    # the 8 closest pairs' atoms and 24 more drawn at random among the close ones
    rng = np.random.default_rng(23)
    idx = list(dict.fromkeys([int(a) for a in pairs[order[:8]].ravel()] +
                             [int(a) for a in rng.choice(close, 24, replace=False)]))
    moll = Mollifier(c, r_c)
    F = np.zeros((len(idx), 3))
    bF = np.zeros(len(idx))
    for ch, p in enumerate(s.ps):
        o_phi, o_F = real_space_atoms(idx, s.pos, s.q[ch], box, p, c, r_c, moll)
        b_phi, b_f = _close_pair_bounds(idx, wrapped, s.q[ch], box, p, r_c, moll, 2e-6, 1.3e-8)
        err = np.abs(phi[ch, idx] - o_phi)
        assert np.all(err <= b_phi), (ch, p, np.max(err / b_phi))
        F += o_F
        bF += b_f
    err = np.max(np.abs(f[idx] - F), axis=1)
    assert np.all(err <= bF), np.max(err / bF)


def _gpu_total(s, M, P, r_c, tol, precision):
    """E_c and F of reciprocal part + real-space part - self energy, all on
    the GPU."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    c = math.log(3.0 / tol)
    cw = window_cw(s.box, M, P, c, r_c)
    plan = lr.Plan(s.box, s.n, s.ps, r_c, c=c, c_w=cw, P=P, grid=M, precision=precision,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    pos = torch.tensor(s.pos, device=dev)
    q = torch.tensor(s.q, dtype=plan.dtype, device=dev)
    plan.set_points(pos, q)
    e_k, _, f_k = plan.execute()
    e_r, _, f_r = plan.real_space(pos, q)
    plan.sync()
    E = e_k.cpu().numpy()[:-1] + e_r.cpu().numpy()[:-1] - plan.self_energy()
    return E, f_k.cpu().double().numpy() + f_r.cpu().double().numpy()


def _energy_scale(q, phi):
    """1/2 sum_i |q_i phi_i|: the size of the per-atom energies, against which
    an energy of cancelling charges (random +-1) is measured."""
    return 0.5 * float(np.sum(np.abs(q * phi)))


@pytest.mark.parametrize("precision", [1, 0])
def test_gpu_total_random_charges_box(precision):
    """64 charges (+-1, minimum separation 1 A) in L = 12 A, p = 1, r_c = 4
    (the largest the cell list takes: 3 cells per edge).  A 1e-5 force error
    then needs the mollifier of tol 5e-6 (c = log(6e5); with c = log(3e5)
    the oracle's total stays at 1.2e-5 on any grid): P = 8, grid 28^3
    (oracle total 6.9e-6 from Ewald).  The energy (-0.169, from cancelling
    terms) is measured against the per-atom energy scale."""
    from oracle.ewald import ewald
    s = wl.random_charges(64, 12.0, 1.0, seed=5)
    E, F = _gpu_total(s, (28, 28, 28), 8, 4.0, 5e-6, precision)
    ew = ewald(s.pos, s.q[0], s.box, 1)
    assert abs(E[0] - ew["E"]) <= 1e-5 * _energy_scale(s.q[0], ew["phi"]), (E[0], ew["E"])
    assert rel_rms(F, ew["F"]) <= 1e-5, rel_rms(F, ew["F"])


@pytest.mark.parametrize("precision", [1, 0])
def test_gpu_total_water_parameters(precision):
    """Water-like box at its benchmarked parameters (h = 31 / 64 A, P = 8,
    r_c = 4, tol 5e-6): the 648-atom box of the same density, 38^3."""
    from oracle.ewald import ewald
    s = wl.water_box(n_side=6, L=18.6, seed=4)
    E, F = _gpu_total(s, (38, 38, 38), 8, 4.0, 5e-6, precision)
    F_ew = np.zeros_like(F)
    for c, p in enumerate(s.ps):
        ew = ewald(s.pos, s.q[c], s.box, p)
        F_ew += ew["F"]
        assert abs(E[c] - ew["E"]) <= 1e-5 * _energy_scale(s.q[c], ew["phi"]), (c, E[c], ew["E"])
    assert rel_rms(F, F_ew) <= 1e-5, rel_rms(F, F_ew)


def test_gpu_total_nacl_madelung():
    """Rock salt, 2 x 2 x 2 conventional cells (64 ions, a = 5.64 A): the
    energy is -N M / (2 d), d = a / 2, M = 1.747564594633 (the Madelung
    constant of rock salt), and every force vanishes by symmetry."""
    s = wl.nacl(5.64, 2)
    M_nacl = 1.747564594633
    d = 5.64 / 2
    E, F = _gpu_total(s, (28, 28, 28), 7, 3.7, 1e-5, 1)
    ref = -s.n * M_nacl / (2 * d)
    assert abs(E[0] - ref) <= 1e-5 * abs(ref), (E[0], ref)
    assert np.abs(F).max() <= 1e-5 * s.n / d ** 2


def test_real_space_empty_and_tiny():
    """n = 0 gives zero energies; a 5-atom system in a 3 x 3 x 3 cell list
    (most cells empty) matches the oracle."""
    import torch
    from oracle.realspace import real_space
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    box = (12.5, 13.0, 14.0)
    plan = lr.Plan(box, 8, (2,), 4.0, c=C, P=6, grid=(26, 26, 28), precision=1,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    e, _, _ = plan.real_space(torch.zeros(0, 3, dtype=torch.float64, device=dev),
                              torch.zeros(1, 0, dtype=torch.float64, device=dev))
    plan.sync()
    assert np.all(e.cpu().numpy() == 0.0)
    rng = np.random.default_rng(3)
    pos = rng.uniform(0.0, 1.0, size=(5, 3)) * np.asarray(box)
    q = rng.normal(size=(1, 5))
    e, phi, f = plan.real_space(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    plan.sync()
    o = real_space(pos, q[0], box, 2, C, 4.0)
    assert abs(e.cpu().numpy()[0] - o["E"]) <= 1e-10 * max(1.0, abs(o["E"]))
    assert np.allclose(phi.cpu().numpy()[0], o["phi"], rtol=1e-10, atol=1e-12)
    assert np.allclose(f.cpu().numpy(), o["F"], rtol=1e-10, atol=1e-12)


def test_real_space_overfull_cell_is_reported():
    """2100 atoms inside one 4.3 A cell: the queue cannot encode the cell,
    its pairs are left out and pswf_sync returns PSWF_ECELL (-9)."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    box = (13.0, 13.0, 13.0)
    n = 2100
    rng = np.random.default_rng(4)
    pos = 5.0 + rng.uniform(0.0, 3.0, size=(n, 3))
    q = rng.normal(size=(1, n))
    plan = lr.Plan(box, n, (1,), 4.0, c=C, P=6, grid=(26, 26, 26), flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    plan.real_space(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    with pytest.raises(lr.PswfError) as e:
        plan.sync()
    assert e.value.status == -9


SHEARED = np.array([[19.2, 0.0, 0.0], [4.5, 18.0, 0.0], [-3.0, 3.5, 17.5]])


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, TOL_FP32)])
def test_real_space_sheared_cell_matches_oracle(precision, tol):
    """Sheared cell (heights 17.5-18.0 A, 4 list cells per edge at r_c = 4),
    p = 1 and 6, atoms up to one cell outside."""
    import torch
    from oracle.realspace import real_space
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(21)
    n = 500
    pos = rng.uniform(-1.0, 2.0, size=(n, 3)) @ SHEARED
    q = rng.normal(size=(2, n))
    plan = lr.Plan(None, n, (1, 6), 4.0, c=C, P=6, grid=(40, 36, 36), precision=precision,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev, cell=SHEARED)
    e, phi, f = plan.real_space(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    plan.sync()
    e, phi, f = e.cpu().numpy(), phi.cpu().double().numpy(), f.cpu().double().numpy()
    F = np.zeros((n, 3))
    for c, p in enumerate((1, 6)):
        o = real_space(pos, q[c], SHEARED, p, C, 4.0)
        assert abs(e[c] - o["E"]) <= tol * abs(o["E"]), (c, e[c], o["E"])
        assert rel_rms(phi[c], o["phi"]) <= tol, (c, rel_rms(phi[c], o["phi"]))
        F += o["F"]
    assert rel_rms(f, F) <= tol, rel_rms(f, F)


@pytest.mark.parametrize("precision", [1, 0])
def test_gpu_total_rotated_melt_box_matches_ewald(precision):
    """The ionic-melt sub-box (L = 21.875 A, 1024 atoms, r_c = 7, P = 7,
    24^3) rotated into a general cell H = L R^T: the complete lattice sum
    from the GPU against Ewald of the unrotated box (forces rotated back)."""
    import torch
    from oracle.ewald import ewald
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    L = 350.0 * 24 / 384
    s = wl.ionic_melt(int(round(4194304 * (L / 350.0) ** 3)), L, seed=3)
    th, ph = 0.5, 0.3
    Rz = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    Rx = np.array([[1.0, 0.0, 0.0], [0.0, math.cos(ph), -math.sin(ph)], [0.0, math.sin(ph), math.cos(ph)]])
    R = Rx @ Rz
    H = np.diag(s.box) @ R.T
    M = (24, 24, 24)
    cw = window_cw(s.box, M, 7, C, 7.0)
    plan = lr.Plan(None, s.n, s.ps, 7.0, c=C, c_w=cw, P=7, grid=M, precision=precision,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev, cell=H)
    pos = torch.tensor(s.pos @ R.T, device=dev)
    q = torch.tensor(s.q, dtype=plan.dtype, device=dev)
    plan.set_points(pos, q)
    e_k, _, f_k = plan.execute()
    e_r, _, f_r = plan.real_space(pos, q)
    plan.sync()
    E = e_k.cpu().numpy()[:-1] + e_r.cpu().numpy()[:-1] - plan.self_energy()
    F = (f_k.cpu().double().numpy() + f_r.cpu().double().numpy()) @ R   # back to the box frame
    F_ew = np.zeros_like(F)
    for c, p in enumerate(s.ps):
        ew = ewald(s.pos, s.q[c], s.box, p)
        F_ew += ew["F"]
        assert abs(E[c] - ew["E"]) <= 1e-5 * _energy_scale(s.q[c], ew["phi"]), (c, E[c], ew["E"])
    assert rel_rms(F, F_ew) <= 1e-5, rel_rms(F, F_ew)


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, TOL_FP32)])
def test_real_space_sixteen_channels(precision, tol):
    """K = 16 (the largest channel class of the pair kernel), exponents
    cycling through 1..6, against the oracle channel by channel.  Random
    non-neutral charges can make a channel's energy a small difference of
    large pair terms (p = 5 here: E = -1.04), so energies are measured
    against the per-atom energy scale 1/2 sum |q_i phi_i|."""
    import torch
    from oracle.realspace import real_space
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    box = (12.6, 13.2, 14.1)
    ps = tuple(1 + (c % 6) for c in range(16))
    rng = np.random.default_rng(31)
    n = 260
    pos = rng.uniform(-0.5, 1.5, size=(n, 3)) * np.asarray(box)
    q = rng.normal(size=(16, n))
    plan = lr.Plan(box, n, ps, 4.0, c=C, P=6, grid=(26, 28, 30), precision=precision,
                   flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    e, phi, f = plan.real_space(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    plan.sync()
    e, phi, f = e.cpu().numpy(), phi.cpu().double().numpy(), f.cpu().double().numpy()
    F = np.zeros((n, 3))
    for c, p in enumerate(ps):
        o = real_space(pos, q[c], box, p, C, 4.0)
        scale = max(abs(o["E"]), _energy_scale(q[c], o["phi"]))
        assert abs(e[c] - o["E"]) <= tol * scale, (c, e[c], o["E"], scale)
        assert rel_rms(phi[c], o["phi"]) <= tol, (c, rel_rms(phi[c], o["phi"]))
        F += o["F"]
    assert rel_rms(f, F) <= tol, rel_rms(f, F)


@pytest.mark.parametrize("precision,tol", [(1, 1e-10), (0, TOL_FP32)])
def test_real_space_direct_sum_small_cells(precision, tol):
    """No cell list: the 64-charge box (L = 12 A) at r_c = 6 = L/2 (minimum
    image), and the sheared cell scaled to edges of about 9.5 A with
    r_c = 6 above its heights (images up to two cells away); p = 1, 4, 6."""
    import torch
    from oracle.realspace import real_space
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(41)
    s = wl.random_charges(64, 12.0, 1.0, seed=6)
    cases = [(np.diag(s.box), s.pos, rng.normal(size=(3, 64)), (24, 24, 24))]
    H = SHEARED / 2.0
    pos = rng.uniform(-0.5, 1.5, size=(90, 3)) @ H
    cases.append((H, pos, rng.normal(size=(3, 90)), (24, 24, 24)))
    ps = (1, 4, 6)
    for H, pos, q, M in cases:
        n = len(pos)
        plan = lr.Plan(None, n, ps, 6.0, c=C, P=6, grid=M, precision=precision, flags=lr.PSWF_FLAG_REAL_SPACE,
                       device=dev, cell=H)
        e, phi, f = plan.real_space(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
        plan.sync()
        e, phi, f = e.cpu().numpy(), phi.cpu().double().numpy(), f.cpu().double().numpy()
        F = np.zeros((n, 3))
        for c, p in enumerate(ps):
            o = real_space(pos, q[c], H, p, C, 6.0)
            scale = max(abs(o["E"]), _energy_scale(q[c], o["phi"]))
            assert abs(e[c] - o["E"]) <= tol * scale, (c, e[c], o["E"])
            assert rel_rms(phi[c], o["phi"]) <= tol, (c, rel_rms(phi[c], o["phi"]))
            F += o["F"]
        assert rel_rms(f, F) <= tol, rel_rms(f, F)


@pytest.mark.parametrize("box", [(13.0, 13.0, 13.0), (9.0, 9.0, 9.0)])   # cell list; direct sum
def test_real_space_nonfinite_positions_reported(box):
    """A NaN or Inf coordinate is binned at 0 and reported as
    PSWF_ENONFINITE (-6) by the next synchronising call."""
    import torch
    from paper_2606_06617_b300 import lr
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    pos = rng.uniform(0.0, 1.0, size=(40, 3)) * np.asarray(box)
    pos[7, 1] = np.nan
    pos[19, 2] = np.inf
    q = rng.normal(size=(1, 40))
    plan = lr.Plan(box, 40, (1,), 4.0, c=C, P=6, grid=(26, 26, 26), flags=lr.PSWF_FLAG_REAL_SPACE, device=dev)
    plan.real_space(torch.tensor(pos, device=dev), torch.tensor(q, device=dev))
    with pytest.raises(lr.PswfError) as e:
        plan.sync()
    assert e.value.status == -6
