"""Pins of the oracle's real-space complement (oracle/realspace.py).

* Brute force: the pair sum over an explicit, wide range of periodic images
  (every image within 5 cells) on a handful of atoms, some placed several
  cells away from the primary cell, equals the oracle's energy; its forces
  are -dE/dr by central differences.
* Large cutoff limit: with G_p = 0 (r_c far beyond every pair) the term is
  the bare 1/r^p pair sum, checked on two atoms at a known distance.
* The per-atom direct sum (real_space_atoms: minimum image, f_p' by
  autograd in r) equals the potentials and forces that real_space gets by
  differentiating the total energy in q and r.
* General cells: a sheared cell against brute force over every image within
  5 cells; a rotated box equals the box (rotated forces); a unimodular
  change of the cell vectors (same lattice) changes nothing; a diagonal cell
  is the box."""
import math

import numpy as np
import pytest

C = math.log(3.0 / 1e-5)


def _brute(pos, q, box, p, r_c, moll):
    box = np.asarray(box, dtype=float)
    E = 0.0
    rng = range(-5, 6)
    for i in range(len(pos)):
        for j in range(len(pos)):
            for a in rng:
                for b in rng:
                    for cc in rng:
                        d = pos[j] + np.array([a, b, cc]) * box - pos[i]
                        r = float(np.linalg.norm(d))
                        if 0.0 < r < r_c:
                            E += 0.5 * q[i] * q[j] * (1.0 - moll.G(p, r)) / r ** p
    return E


def test_real_space_matches_brute_force_over_images():
    from oracle.mollifiers import Mollifier
    from oracle.realspace import real_space
    rng = np.random.default_rng(7)
    box = (9.0, 10.0, 9.5)
    r_c = 4.0
    pos = rng.uniform(0.0, 1.0, size=(14, 3)) * np.asarray(box)
    pos[:7] += rng.integers(-3, 4, size=(7, 3)) * np.asarray(box)      # far images
    q = rng.normal(size=14)
    moll = Mollifier(C, r_c)
    for p in (1, 3, 6):
        o = real_space(pos, q, box, p, C, r_c, moll)
        ref = _brute(pos, q, box, p, r_c, moll)
        assert abs(o["E"] - ref) <= 1e-12 * max(1.0, abs(ref)), (p, o["E"], ref)
    o = real_space(pos, q, box, 1, C, r_c, moll)
    eps = 1e-6
    for i, d in ((0, 0), (3, 2), (10, 1)):
        pp, pm = pos.copy(), pos.copy()
        pp[i, d] += eps
        pm[i, d] -= eps
        g = (real_space(pp, q, box, 1, C, r_c, moll)["E"] - real_space(pm, q, box, 1, C, r_c, moll)["E"]) / (2 * eps)
        assert abs(-g - o["F"][i, d]) <= 1e-6 * max(1.0, abs(g)), (i, d, -g, o["F"][i, d])


def test_real_space_bare_pair_beyond_the_mollifier():
    """Two atoms 1.5 A apart in a 40 A box with r_c = 4: G_p(1.5 / 4) is
    tiny but not zero, so compare against the bare pair term with the
    mollifier applied by hand; and phi_i = q_j (1 - G) / r^p."""
    from oracle.mollifiers import Mollifier
    from oracle.realspace import real_space
    moll = Mollifier(C, 4.0)
    pos = np.array([[1.0, 2.0, 3.0], [2.5, 2.0, 3.0]])
    q = np.array([0.7, -1.3])
    for p in (1, 2, 6):
        g = (1.0 - moll.G(p, 1.5)) / 1.5 ** p
        o = real_space(pos, q, (40.0, 40.0, 40.0), p, C, 4.0, moll)
        assert abs(o["E"] - q[0] * q[1] * g) <= 1e-14
        assert np.allclose(o["phi"], [q[1] * g, q[0] * g], rtol=1e-13)


def test_per_atom_sums_match_the_energy_derivatives():
    from oracle.mollifiers import Mollifier
    from oracle.realspace import real_space, real_space_atoms
    rng = np.random.default_rng(9)
    box = (9.0, 8.5, 10.0)
    r_c = 4.0
    pos = rng.uniform(0.0, 1.0, size=(60, 3)) * np.asarray(box)
    pos[:10] += rng.integers(-2, 3, size=(10, 3)) * np.asarray(box)
    q = rng.normal(size=60)
    moll = Mollifier(C, r_c)
    idx = [0, 3, 11, 25, 59]
    for p in (1, 4, 6):
        o = real_space(pos, q, box, p, C, r_c, moll)
        phi, F = real_space_atoms(idx, pos, q, box, p, C, r_c, moll)
        assert np.allclose(phi, o["phi"][idx], rtol=1e-12, atol=1e-14)
        assert np.allclose(F, o["F"][idx], rtol=1e-11, atol=1e-13)


SHEARED = np.array([[13.0, 0.0, 0.0], [3.5, 12.0, 0.0], [-2.0, 2.5, 11.0]])


def _brute_cell(pos, q, H, p, r_c, moll):
    E = 0.0
    rng = range(-5, 6)
    for i in range(len(pos)):
        for j in range(len(pos)):
            for a in rng:
                for b in rng:
                    for cc in rng:
                        d = pos[j] + np.array([a, b, cc], dtype=float) @ H - pos[i]
                        r = float(np.linalg.norm(d))
                        if 0.0 < r < r_c:
                            E += 0.5 * q[i] * q[j] * (1.0 - moll.G(p, r)) / r ** p
    return E


def test_real_space_sheared_cell_brute_force():
    from oracle.mollifiers import Mollifier
    from oracle.realspace import real_space
    rng = np.random.default_rng(12)
    pos = rng.uniform(-1.0, 2.0, size=(12, 3)) @ SHEARED
    q = rng.normal(size=12)
    moll = Mollifier(C, 4.0)
    for p in (1, 6):
        o = real_space(pos, q, SHEARED, p, C, 4.0, moll)
        ref = _brute_cell(pos, q, SHEARED, p, 4.0, moll)
        assert abs(o["E"] - ref) <= 1e-12 * max(1.0, abs(ref)), (p, o["E"], ref)


def test_real_space_cell_invariances():
    import math
    from oracle.mollifiers import Mollifier
    from oracle.realspace import real_space
    rng = np.random.default_rng(13)
    moll = Mollifier(C, 4.0)
    box = (11.0, 12.5, 10.0)
    pos = rng.uniform(0.0, 1.0, size=(40, 3)) * np.asarray(box)
    q = rng.normal(size=40)
    th = 0.7
    Rz = np.array([[math.cos(th), -math.sin(th), 0.0], [math.sin(th), math.cos(th), 0.0], [0.0, 0.0, 1.0]])
    a = real_space(pos, q, box, 4, C, 4.0, moll)
    b = real_space(pos @ Rz.T, q, np.diag(box) @ Rz.T, 4, C, 4.0, moll)
    d = real_space(pos, q, np.diag(box), 4, C, 4.0, moll)
    assert abs(a["E"] - b["E"]) <= 1e-12 * abs(a["E"])
    assert np.allclose(b["F"], a["F"] @ Rz.T, rtol=1e-10, atol=1e-12)
    assert a["E"] == d["E"]
    U = np.array([[1, 0, 0], [1, 1, 0], [0, -1, 1]], dtype=float)
    pos2 = rng.uniform(0.0, 1.0, size=(30, 3)) @ SHEARED
    q2 = rng.normal(size=30)
    e1 = real_space(pos2, q2, SHEARED, 2, C, 4.0, moll)
    e2 = real_space(pos2, q2, U @ SHEARED, 2, C, 4.0, moll)
    assert abs(e1["E"] - e2["E"]) <= 1e-12 * abs(e1["E"])
    assert np.allclose(e1["F"], e2["F"], rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("p,cell", [(1, False), (6, False), (4, True)])
def test_real_space_vjp_matches_finite_differences(p, cell):
    """The oracle's VJP of the real-space outputs (double autograd) against
    central differences of L = gE E + gphi . phi + gF . F built from the
    forward outputs of real_space itself (a dropped term, a wrong sign or a
    missing second-derivative term of the force fails it)."""
    import math
    from oracle.realspace import real_space, real_space_vjp
    from paper_2606_06617_b300 import workloads as wl
    s = wl.random_system(24, (7.0, 7.5, 8.0), (p,), seed=20 + p, neutral=False)
    box = np.asarray(s.box)
    if cell:
        box = np.array([[7.0, 0.0, 0.0], [1.2, 7.5, 0.0], [-0.8, 0.9, 8.0]])
    c, rc = math.log(3e5), 3.2
    rng = np.random.default_rng(p)
    gE, gphi, gF = 0.7, rng.normal(size=s.n), rng.normal(size=(s.n, 3))

    def L(pos, q):
        r = real_space(pos, q, box, p, c, rc)
        return gE * r["E"] + float(np.dot(gphi, r["phi"])) + float(np.sum(gF * r["F"]))

    gq, gp = real_space_vjp(s.pos, s.q[0], box, p, c, rc, gE, gphi, gF)
    h = 1e-5
    for k in (0, 5, 11):
        qp, qm = s.q[0].copy(), s.q[0].copy()
        qp[k] += h
        qm[k] -= h
        fd = (L(s.pos, qp) - L(s.pos, qm)) / (2 * h)
        assert abs(fd - gq[k]) <= 1e-6 * max(1.0, abs(gq[k])), (k, fd, gq[k])
        for d in range(3):
            pp, pm = s.pos.copy(), s.pos.copy()
            pp[k, d] += h
            pm[k, d] -= h
            fd = (L(pp, s.q[0]) - L(pm, s.q[0])) / (2 * h)
            assert abs(fd - gp[k, d]) <= 1e-5 * max(1.0, abs(gp[k, d])), (k, d, fd, gp[k, d])
