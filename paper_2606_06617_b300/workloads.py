"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws positions, boxes, latent charges and arrival times
(numpy PCG64); it holds none of the PSWF-LR arithmetic, so both the CUDA
path's tests/bench and the CPU oracle may use it.  The paper's own benchmark
systems (NaCl crystals, SWM4-NDP water, LiPF6/DMC electrolyte; Methods,
"Performance comparison in differentiable long-range evaluations") are not
available here; these recipes stand in for them.

Conventions: positions are float64 arrays [N, 3] in Angstrom, boxes are
orthorhombic edge lengths (L_x, L_y, L_z), latent charges are float64
arrays [K, N] (one row per channel), ``ps`` lists each channel's exponent.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class System:
    pos: np.ndarray            # [N, 3]
    q: np.ndarray              # [K, N]
    box: tuple                 # (L_x, L_y, L_z)
    ps: tuple                  # exponent per channel
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _neutral(rng, K, N, scale=1.0):
    q = rng.standard_normal((K, N)) * scale
    return q - q.mean(axis=1, keepdims=True)


def _uniform_min_sep(rng, n, box, min_sep, max_tries=2_000_000):
    """Uniform positions with a minimum pairwise (minimum-image) separation,
    by sequential rejection on a cell grid."""
    box = np.asarray(box, dtype=np.float64)
    nc = np.maximum((box // max(min_sep, 1e-9)).astype(int), 1)
    cells: dict = {}
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place atoms at this density / separation")
        x = rng.random(3) * box
        ci = tuple((x / box * nc).astype(int) % nc)
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    key = ((ci[0] + dx) % nc[0], (ci[1] + dy) % nc[1], (ci[2] + dz) % nc[2])
                    for y in cells.get(key, ()):
                        d = x - y
                        d -= box * np.round(d / box)
                        if d @ d < min_sep * min_sep:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            out.append(x)
            cells.setdefault(ci, []).append(x)
    return np.array(out).reshape(-1, 3)


# ---- small parity case: 64 point charges ---------------------------------
def random_charges(n: int = 64, L: float = 12.0, min_sep: float = 1.0, seed: int = 0) -> System:
    """n/2 charges +1 and n/2 charges -1, uniform in a cubic box with a
    minimum separation; one channel p = 1."""
    rng = np.random.default_rng(seed)
    pos = _uniform_min_sep(rng, n, (L, L, L), min_sep)
    q = np.concatenate([np.ones(n // 2), -np.ones(n - n // 2)])[None, :]
    return System(pos, q, (L, L, L), (1,), name=f"random_charges_{n}")


def nacl(a: float = 5.64, ncell: int = 2) -> System:
    """Rock-salt crystal of ncell^3 conventional cells (8 ions each)."""
    base = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    pos, q = [], []
    for i in range(ncell):
        for j in range(ncell):
            for k in range(ncell):
                off = np.array([i, j, k], dtype=np.float64)
                pos += list((base + off) * a)
                q += [1.0] * 4
                pos += list((base + np.array([.5, 0, 0]) + off) * a)
                q += [-1.0] * 4
    L = ncell * a
    pos = np.mod(np.array(pos), L)
    return System(pos, np.array(q)[None, :], (L, L, L), (1,), name=f"nacl_{ncell}")


# ---- water-like box --------------------------------------------------------
def _random_rotations(rng, n):
    qv = rng.standard_normal((n, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z); R[:, 0, 1] = 2 * (x * y - z * w); R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w); R[:, 1, 1] = 1 - 2 * (x * x + z * z); R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w); R[:, 2, 1] = 2 * (y * z + x * w); R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def water_box(n_side: int = 10, L: float = 31.0, seed: int = 0) -> System:
    """n_side^3 three-site molecules: O on a jittered cubic lattice (spacing
    L / n_side, jitter U(-0.3, 0.3)), O-H 0.96 A, H-O-H 104.5 deg, uniformly
    random orientation.  Channel 0 (p = 1): O -0.8, H +0.4.  Channel 1
    (p = 6): per-atom coefficients |N(1, 0.2)| (not neutral)."""
    rng = np.random.default_rng(seed)
    sp = L / n_side
    g = (np.arange(n_side) + 0.5) * sp
    O = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    O = O + rng.uniform(-0.3, 0.3, O.shape)
    half = np.deg2rad(104.5) / 2
    h1 = 0.96 * np.array([np.sin(half), np.cos(half), 0.0])
    h2 = 0.96 * np.array([-np.sin(half), np.cos(half), 0.0])
    R = _random_rotations(rng, len(O))
    pos = np.stack([O, O + R @ h1, O + R @ h2], 1).reshape(-1, 3)
    pos = np.mod(pos, L)
    q1 = np.tile([-0.8, 0.4, 0.4], len(O))
    q6 = np.abs(rng.normal(1.0, 0.2, len(pos)))
    return System(pos, np.stack([q1, q6]), (L, L, L), (1, 6), name=f"water_{len(pos)}")


# ---- large ionic melt ----------------------------------------------------------
def ionic_melt(N: int = 4194304, L: float = 350.0, seed: int = 0) -> System:
    """N atoms uniform in a cubic box.  Channel 0 (p = 1): charges +1 / -1,
    exactly half each, shuffled.  Channels 1..3 (p = 2, 4, 6): N(0, 1) with
    the channel mean subtracted (neutral)."""
    rng = np.random.default_rng(seed)
    pos = rng.random((N, 3)) * L
    q0 = np.concatenate([np.ones(N // 2), -np.ones(N - N // 2)])
    rng.shuffle(q0)
    q = np.concatenate([q0[None, :], _neutral(rng, 3, N)], 0)
    return System(pos, q, (L, L, L), (1, 2, 4, 6), name=f"ionic_melt_{N}")


# ---- serving stream ---------------------------------------------------------------
@dataclass
class Request:
    rid: int
    t_arrival: float
    system: System


def serving_stream(n_req: int = 4096, rate: float = 2000.0, K: int = 8,
                   n_min: int = 32, n_max: int = 2048, density: float = 0.1,
                   seed: int = 0):
    """Requests with atom counts log-uniform in [n_min, n_max], orthorhombic
    boxes of the given number density with aspect ratios U(1, 1.5), K neutral
    N(0, 1) channels that all share one exponent drawn from {1, 6} per
    request, and Poisson arrivals at ``rate`` requests/s."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_req)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n_req):
        n = int(np.floor(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        n = min(max(n, n_min), n_max)
        a = rng.uniform(1.0, 1.5, 3)
        V = n / density
        box = tuple(float(v) for v in a * (V / np.prod(a)) ** (1.0 / 3.0))
        pos = rng.random((n, 3)) * np.asarray(box)
        p = int(rng.choice([1, 6]))
        q = _neutral(rng, K, n)
        out.append(Request(i, float(t[i]), System(pos, q, box, (p,) * K, name=f"req{i}")))
    return out


# ---- training-step batch ----------------------------------------------------------
def training_batch(n_struct: int = 64, K: int = 16, n_lo: int = 200, n_hi: int = 600,
                   density: float = 0.1, min_sep: float = 0.8, seed: int = 0):
    """Structures with N ~ U{n_lo..n_hi}, cubic boxes at the given density,
    min separation ``min_sep``, K neutral N(0, 1) channels with exponents
    alternating 1, 6, 1, 6, ..."""
    rng = np.random.default_rng(seed)
    ps = tuple(1 if c % 2 == 0 else 6 for c in range(K))
    out = []
    for s in range(n_struct):
        n = int(rng.integers(n_lo, n_hi + 1))
        L = (n / density) ** (1.0 / 3.0)
        pos = _uniform_min_sep(rng, n, (L, L, L), min_sep)
        q = _neutral(rng, K, n)
        out.append(System(pos, q, (L, L, L), ps, name=f"train{s}"))
    return out


def random_system(n: int, box, ps, seed: int = 0, neutral: bool = True) -> System:
    """Generic helper for parity tests: uniform positions, N(0,1) channels."""
    rng = np.random.default_rng(seed)
    box = tuple(float(b) for b in box)
    pos = rng.random((n, 3)) * np.asarray(box)
    K = len(ps)
    q = _neutral(rng, K, n) if neutral else rng.standard_normal((K, n))
    return System(pos, q, box, tuple(ps), name=f"random_{n}")
