"""Thin ctypes binding of libpswf_lr.so (include/pswf_lr.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
library.  PyTorch supplies device memory (outputs and the plan workspace) and
the current CUDA stream.  If the library is missing this module raises on
first use; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PSWF_LR_LIBRARY selects another build of the same library (for example
# libpswf_lr_checked.so, the bounds-checked build the tests use)
LIB_PATH = os.environ.get("PSWF_LR_LIBRARY") or os.path.join(_HERE, "libpswf_lr.so")
LIB_CHECKED_PATH = os.path.join(_HERE, "libpswf_lr_checked.so")

PSWF_ETIMEOUT = -5
PSWF_SUBMIT_BORROW = 1
PSWF_EBOUNDS = -10
PSWF_FLAG_BACKWARD = 1
PSWF_FLAG_VIRIAL = 2
PSWF_FLAG_REAL_SPACE = 4
PSWF_TRANSFORM_FULL = 0
PSWF_TRANSFORM_PRUNED = 1
PSWF_TRANSFORM_PRUNED_X = 2
PSWF_TRANSFORM_OWN = 3


class PswfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class PswfOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("r_c", ctypes.c_double), ("c", ctypes.c_double),
                ("c_w", ctypes.c_double), ("eta", ctypes.c_double), ("P", ctypes.c_int),
                ("grid", ctypes.c_int * 3), ("precision", ctypes.c_int), ("flags", ctypes.c_int)]


class PswfInfo(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("c_w", ctypes.c_double), ("r_c", ctypes.c_double),
                ("k_c", ctypes.c_double), ("eta", ctypes.c_double), ("tol", ctypes.c_double),
                ("est_err_spread", ctypes.c_double), ("est_err_band", ctypes.c_double),
                ("lambda0", ctypes.c_double), ("C0", ctypes.c_double),
                ("box", ctypes.c_double * 3), ("h", ctypes.c_double * 3), ("grid", ctypes.c_int * 3),
                ("P", ctypes.c_int), ("K", ctypes.c_int), ("precision", ctypes.c_int),
                ("deg_window", ctypes.c_int), ("deg_mult", ctypes.c_int), ("flags", ctypes.c_int),
                ("n_max", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("B", ctypes.c_int), ("batch", ctypes.c_int), ("transform", ctypes.c_int),
                ("nkx", ctypes.c_int), ("cell", ctypes.c_double * 9),
                ("deg_real", ctypes.c_int)]


MAX_BUCKETS = 16


class PswfServerOpts(ctypes.Structure):
    _fields_ = [("r_c", ctypes.c_double), ("tol", ctypes.c_double), ("c", ctypes.c_double),
                ("h_max", ctypes.c_double), ("K", ctypes.c_int), ("npset", ctypes.c_int),
                ("pset", ctypes.c_int * 6), ("nbucket", ctypes.c_int), ("grid", ctypes.c_int * MAX_BUCKETS),
                ("b_max", ctypes.c_int * MAX_BUCKETS), ("n_max", ctypes.c_int64 * MAX_BUCKETS),
                ("inflight", ctypes.c_int), ("precision", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("P", ctypes.c_int)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

# name -> (argtypes, restype); mirrors include/pswf_lr.h
SIGNATURES = {
    "pswf_opts_default": ([ctypes.POINTER(PswfOpts)], None),
    "pswf_plan_params": ([_dp, ctypes.c_int, _ip, ctypes.POINTER(PswfOpts), ctypes.POINTER(PswfInfo)], ctypes.c_int),
    "pswf_plan_create": ([_dp, _i64, ctypes.c_int, _ip, ctypes.POINTER(PswfOpts), _vp, ctypes.POINTER(_vp)],
                         ctypes.c_int),
    "pswf_plan_create_cell": ([_dp, _i64, ctypes.c_int, _ip, ctypes.POINTER(PswfOpts), _vp, ctypes.POINTER(_vp)],
                         ctypes.c_int),
    "pswf_plan_info": ([_vp, ctypes.POINTER(PswfInfo)], ctypes.c_int),
    "pswf_plan_set_workspace": ([_vp, _vp, _i64], ctypes.c_int),
    "pswf_plan_set_stream": ([_vp, _vp], ctypes.c_int),
    "pswf_set_points": ([_vp, _i64, _vp, ctypes.c_int, _vp], ctypes.c_int),
    "pswf_execute": ([_vp, _vp, _vp, _vp], ctypes.c_int),
    "pswf_backward": ([_vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "pswf_self_energy": ([_vp, _dp], ctypes.c_int),
    "pswf_virial": ([_vp, _vp], ctypes.c_int),
    "pswf_stress": ([_vp, _vp], ctypes.c_int),
    "pswf_real_space": ([_vp, _i64, _vp, ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
    "pswf_real_space_backward": ([_vp, _i64, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "pswf_sync": ([_vp], ctypes.c_int),
    "pswf_sync_for": ([_vp, ctypes.c_double], ctypes.c_int),
    "pswf_compute_host": ([_vp, _i64, _dp, _dp, _dp, _dp, _dp], ctypes.c_int),
    "pswf_compute_host_real": ([_vp, _i64, _dp, _vp, _dp, _vp, _vp], ctypes.c_int),
    "pswf_plan_destroy": ([_vp], None),
    "pswf_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "pswf_plan_last_error": ([_vp, ctypes.c_char_p, ctypes.c_int], ctypes.c_int),
    "pswf_self_energy_noalloc": ([_vp, _i64, _vp, _vp, _vp], ctypes.c_int),
    "pswf_profile_enable": ([_vp, ctypes.c_int], ctypes.c_int),
    "pswf_profile_read": ([_vp, _dp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "pswf_batch_plan_create": ([_dp, ctypes.c_int, _i64, ctypes.c_int, _ip, ctypes.c_int, ctypes.POINTER(PswfOpts),
                                _vp, ctypes.POINTER(_vp)], ctypes.c_int),
    "pswf_batch_set_points": ([_vp, ctypes.c_int, _dp, _ip, ctypes.POINTER(ctypes.c_int64), _vp, ctypes.c_int, _vp],
                              ctypes.c_int),
    "pswf_server_opts_default": ([ctypes.POINTER(PswfServerOpts)], None),
    "pswf_server_create": ([ctypes.POINTER(PswfServerOpts), ctypes.POINTER(_vp)], ctypes.c_int),
    "pswf_server_route": ([_vp, _i64, _dp, ctypes.POINTER(PswfInfo)], ctypes.c_int),
    "pswf_server_submit": ([_vp, _i64, _dp, _ip, _dp, _dp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "pswf_server_wait": ([_vp, _i64, _dp, _dp, _dp, _dp], ctypes.c_int),
    "pswf_server_wait_for": ([_vp, _i64, ctypes.c_double, _dp, _dp, _dp, _dp], ctypes.c_int),
    "pswf_server_pause": ([_vp, ctypes.c_int], ctypes.c_int),
    "pswf_server_submit_many": ([_vp, _i64, ctypes.POINTER(ctypes.c_int64), _dp, _ip, ctypes.POINTER(_dp),
                                 ctypes.POINTER(_dp), ctypes.POINTER(ctypes.c_int64), ctypes.c_int], ctypes.c_int),
    "pswf_server_wait_many": ([_vp, _i64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), _dp, _dp,
                               _dp, _dp], ctypes.c_int),
    "pswf_server_stats": ([_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "pswf_server_last_error": ([_vp, ctypes.c_char_p, ctypes.c_int], ctypes.c_int),
    "pswf_server_destroy": ([_vp], None),
}

NSTAGE = 11
STAGES = ("set_points", "spread", "fft_fwd", "multiply", "fft_inv", "interp", "backward", "other", "real_space",
          "h2d", "d2h")


def lib():
    """Loads libpswf_lr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_2606_06617_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status: int, handle=None):
    if status == 0:
        return
    L = lib()
    msg = L.pswf_strerror(status).decode()
    if handle:
        buf = ctypes.create_string_buffer(512)
        L.pswf_plan_last_error(handle, buf, 512)
        if buf.value:
            msg = f"{msg}: {buf.value.decode()}"
    raise PswfError(status, msg)


def make_opts(r_c: float, tol: float = 1e-5, c: float = 0.0, c_w: float = 0.0, eta: float = 0.0,
              P: int = 0, grid=None, precision: int = 0, flags: int = 0) -> PswfOpts:
    o = PswfOpts()
    lib().pswf_opts_default(ctypes.byref(o))
    o.tol, o.r_c, o.c, o.c_w, o.eta, o.P = tol, r_c, c, c_w, eta, P
    if grid is not None:
        g = [int(grid)] * 3 if np.isscalar(grid) else [int(x) for x in grid]
        for d in range(3):
            o.grid[d] = g[d]
    o.precision, o.flags = precision, flags
    return o


def _info_dict(info: PswfInfo) -> dict:
    out = {}
    for name, _ in PswfInfo._fields_:
        v = getattr(info, name)
        out[name] = list(v) if isinstance(v, ctypes.Array) else v
    return out


def plan_params(box, ps, **opts) -> dict:
    """Host-only parameter selection (no GPU).  ``opts`` as make_opts."""
    L = lib()
    box_a = (ctypes.c_double * 3)(*[float(b) for b in box])
    p_a = (ctypes.c_int * len(ps))(*[int(p) for p in ps])
    o = make_opts(**opts)
    info = PswfInfo()
    _check(L.pswf_plan_params(box_a, len(ps), p_a, ctypes.byref(o), ctypes.byref(info)))
    return _info_dict(info)


class Plan:
    """One periodic system: PSWF-LR plan with a torch-allocated workspace.

    Calls enqueue on the current torch CUDA stream of the plan's device."""

    def __init__(self, box, n_max: int, ps, r_c: float, *, tol: float = 1e-5, c: float = 0.0,
                 c_w: float = 0.0, eta: float = 0.0, P: int = 0, grid=None, precision: int = 0,
                 flags: int = 0, device=None, cell=None):
        """box: three edge lengths of an orthorhombic box, or None with
        cell: 3 x 3 lattice vectors as rows (general cell,
        pswf_plan_create_cell)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("PSWF-LR needs a CUDA device")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.K = len(ps)
        self.ps = tuple(int(p) for p in ps)
        if cell is not None:
            import numpy as np
            cell_a = (ctypes.c_double * 9)(*[float(x) for x in np.asarray(cell, dtype=np.float64).reshape(9)])
            self.box = tuple(float(x) for x in np.linalg.norm(np.asarray(cell, dtype=np.float64).reshape(3, 3), axis=1))
        else:
            cell_a = None
            self.box = tuple(float(b) for b in box)
        self.dtype = torch.float64 if precision == 1 else torch.float32
        L = lib()
        box_a = (ctypes.c_double * 3)(*self.box)
        p_a = (ctypes.c_int * self.K)(*self.ps)
        o = make_opts(r_c=r_c, tol=tol, c=c, c_w=c_w, eta=eta, P=P, grid=grid, precision=precision, flags=flags)
        h = _vp()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            if cell_a is not None:
                _check(L.pswf_plan_create_cell(cell_a, int(n_max), self.K, p_a, ctypes.byref(o), _vp(stream),
                                               ctypes.byref(h)))
            else:
                _check(L.pswf_plan_create(box_a, int(n_max), self.K, p_a, ctypes.byref(o), _vp(stream),
                                          ctypes.byref(h)))
        self._h = h
        self.n_max = int(n_max)
        info = PswfInfo()
        _check(L.pswf_plan_info(self._h, ctypes.byref(info)), self._h)
        self.info = _info_dict(info)
        nbytes = max(int(self.info["workspace_bytes"]), 256)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self._ws.data_ptr() + 255) & ~255
        with torch.cuda.device(self.device):
            _check(L.pswf_plan_set_workspace(self._h, _vp(aligned), nbytes), self._h)
        self.n = None
        self.flags = int(flags)
        self.generation = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            try:
                lib().pswf_plan_destroy(h)
            except Exception:
                pass
            self._h = None

    def _stream(self):
        import torch
        _check(lib().pswf_plan_set_stream(self._h, _vp(torch.cuda.current_stream(self.device).cuda_stream)), self._h)

    def set_points(self, pos, q):
        """pos: cuda tensor [n, 3] float32/float64; q: cuda tensor [K, n]."""
        import torch
        if not (pos.is_cuda and q.is_cuda) or pos.device != self.device or q.device != self.device:
            raise ValueError("pos and q must be CUDA tensors on the plan's device")
        if pos.dtype not in (torch.float32, torch.float64):
            pos = pos.double()
        pos = pos.contiguous()
        q = q.to(self.dtype).contiguous()
        n = pos.shape[0]
        if pos.shape != (n, 3) or q.shape != (self.K, n):
            raise ValueError("pos must be [n, 3] and q [K, n]")
        self._stream()
        _check(lib().pswf_set_points(self._h, n, _vp(pos.data_ptr()), 1 if pos.dtype == torch.float64 else 0,
                                     _vp(q.data_ptr())), self._h)
        self._keep = (pos, q)
        self.n = n
        self.generation += 1

    def execute(self, energy: bool = True, phi: bool = True, forces: bool = True, out=None):
        """Returns (energy [K+1] float64, phi [K, n] or None, forces [n, 3] or None) on the device."""
        import torch
        if self.n is None:
            raise PswfError(-8, "execute before set_points")
        n = self.n
        if out is not None:
            e, ph, f = out
        else:
            e = torch.empty(self.K + 1, dtype=torch.float64, device=self.device) if energy else None
            ph = torch.empty(self.K, n, dtype=self.dtype, device=self.device) if phi else None
            f = torch.empty(n, 3, dtype=self.dtype, device=self.device) if forces else None
        ptr = lambda t: _vp(t.data_ptr() if (t is not None and t.numel() > 0) else 0)
        self._stream()
        _check(lib().pswf_execute(self._h, ptr(e), ptr(ph), ptr(f)), self._h)
        return e, ph, f

    def backward(self, g_energy=None, g_phi=None, g_forces=None, grad_q: bool = True, grad_pos: bool = True):
        import torch
        n = self.n
        gq = torch.empty(self.K, n, dtype=self.dtype, device=self.device) if grad_q else None
        gr = torch.empty(n, 3, dtype=self.dtype, device=self.device) if grad_pos else None
        ge = g_energy.to(torch.float64).contiguous() if g_energy is not None else None
        gp = g_phi.to(self.dtype).contiguous() if g_phi is not None else None
        gf = g_forces.to(self.dtype).contiguous() if g_forces is not None else None
        ptr = lambda t: _vp(t.data_ptr() if (t is not None and t.numel() > 0) else 0)
        self._stream()
        _check(lib().pswf_backward(self._h, ptr(ge), ptr(gp), ptr(gf), ptr(gq), ptr(gr)), self._h)
        return gq, gr

    def virial(self):
        """Diagonal virial W[c, d] = -L_d dE_c/dL_d of the last execute (device
        float64 [K, 3]; batch plans [B, K, 3]); needs flags=PSWF_FLAG_VIRIAL."""
        import torch
        B = getattr(self, "B", None)
        shape = (self.K, 3) if B is None else (B, self.K, 3)
        out = torch.empty(*shape, dtype=torch.float64, device=self.device)
        self._stream()
        _check(lib().pswf_virial(self._h, _vp(out.data_ptr())), self._h)
        return out

    def stress(self):
        """Virial tensor components (xx, yy, zz, xy, xz, yz) of the last
        execute, W_ab = -dE_c / d epsilon_ab at fixed fractional coordinates
        (device float64 [K, 6]; batch plans [B, K, 6]); needs
        flags=PSWF_FLAG_VIRIAL."""
        import torch
        B = getattr(self, "B", None)
        shape = (self.K, 6) if B is None else (B, self.K, 6)
        out = torch.empty(*shape, dtype=torch.float64, device=self.device)
        self._stream()
        _check(lib().pswf_stress(self._h, _vp(out.data_ptr())), self._h)
        return out

    def real_space(self, pos, q, out=None):
        """Real-space complement (pswf_real_space) of positions pos [n, 3] and
        charges q [K, n] (device tensors): returns (energy float64 [K + 1],
        phi [K, n], forces [n, 3]); needs flags=PSWF_FLAG_REAL_SPACE.  out =
        (energy, phi, forces) device tensors of those shapes to fill."""
        import torch
        n = int(pos.shape[0])
        pos = pos.contiguous()
        q = q.to(self.dtype).contiguous()
        if out is not None:
            energy, phi, forces = out
        else:
            energy = torch.empty(self.K + 1, dtype=torch.float64, device=self.device)
            phi = torch.empty(self.K, n, dtype=self.dtype, device=self.device)
            forces = torch.empty(n, 3, dtype=self.dtype, device=self.device)
        self._stream()
        self.rs_generation = getattr(self, "rs_generation", 0) + 1
        pdt = 1 if pos.dtype == torch.float64 else 0
        _check(lib().pswf_real_space(self._h, n, _vp(pos.data_ptr()), pdt, _vp(q.data_ptr()),
                                     _vp(energy.data_ptr()), _vp(phi.data_ptr()), _vp(forces.data_ptr())), self._h)
        return energy, phi, forces

    def real_space_backward(self, pos, q, g_energy=None, g_phi=None, g_forces=None, grad_q: bool = True,
                            grad_pos: bool = True):
        """VJP of the last real_space call's (energy, phi, forces) on the same
        pos and q: returns (grad_q [K, n] or None, grad_pos [n, 3] or None)
        for upstream g_energy [K] (float64), g_phi [K, n], g_forces [n, 3]
        (device tensors, each may be None)."""
        import torch
        n = int(pos.shape[0])
        pos = pos.contiguous()
        q = q.to(self.dtype).contiguous()
        gq = torch.empty(self.K, n, dtype=self.dtype, device=self.device) if grad_q else None
        gr = torch.empty(n, 3, dtype=self.dtype, device=self.device) if grad_pos else None
        ge = g_energy.to(torch.float64).contiguous() if g_energy is not None else None
        gp = g_phi.to(self.dtype).contiguous() if g_phi is not None else None
        gf = g_forces.to(self.dtype).contiguous() if g_forces is not None else None
        ptr = lambda t: _vp(t.data_ptr() if (t is not None and t.numel() > 0) else 0)
        self._stream()
        pdt = 1 if pos.dtype == torch.float64 else 0
        _check(lib().pswf_real_space_backward(self._h, n, ptr(pos), pdt, ptr(q), ptr(ge), ptr(gp), ptr(gf), ptr(gq),
                                              ptr(gr)), self._h)
        return gq, gr

    def self_coefficients(self, q):
        """s_c with E_self^(c) = s_c sum_i (q_i^c)^2 (device float64 [K]),
        from the device self energies of charges q [K, n] (the plan's
        noalloc entry point, so nothing is allocated on the plan's side)."""
        import torch
        qd = q.to(self.dtype).contiguous()
        ones = torch.ones(self.K, 1, dtype=self.dtype, device=self.device)
        out = torch.empty(self.K, dtype=torch.float64, device=self.device)
        self._stream()
        _check(lib().pswf_self_energy_noalloc(self._h, 1, _vp(ones.data_ptr()), _vp(out.data_ptr()),
                                              _vp(torch.cuda.current_stream(self.device).cuda_stream)), self._h)
        return out   # one unit charge per channel: E_self = s_c

    def self_energy(self) -> np.ndarray:
        out = (ctypes.c_double * self.K)()
        self._stream()
        _check(lib().pswf_self_energy(self._h, out), self._h)
        return np.array(out[:])

    def sync(self, timeout_ms: float | None = None):
        """Waits for the plan's stream; with timeout_ms, raises PswfError
        (status PSWF_ETIMEOUT = -5) if the work is still running then."""
        if timeout_ms is None:
            _check(lib().pswf_sync(self._h), self._h)
        else:
            _check(lib().pswf_sync_for(self._h, float(timeout_ms)), self._h)

    def profile(self, enable: bool = True):
        """Record CUDA events around each stage of later calls."""
        _check(lib().pswf_profile_enable(self._h, 1 if enable else 0), self._h)

    def profile_read(self):
        """(stage ms dict, own-kernel launch counts dict) since the last read."""
        ms = (ctypes.c_double * NSTAGE)()
        nl = (ctypes.c_int64 * NSTAGE)()
        _check(lib().pswf_profile_read(self._h, ms, nl), self._h)
        return dict(zip(STAGES, ms[:])), dict(zip(STAGES, nl[:]))

    def compute_host(self, pos: np.ndarray, q: np.ndarray, phi: bool = True, forces: bool = True, out=None,
                     real: bool = False):
        """End-to-end from host arrays; returns numpy (energy, phi, forces).
        real=False: charges and results float64 (pswf_compute_host);
        real=True: charges and results in the plan's precision
        (pswf_compute_host_real).  Positions and energies are float64.
        out = (energy [K+1], phi [K, n] or None, forces [n, 3] or None)
        C-contiguous arrays of those dtypes to fill instead of new ones."""
        import torch
        rdt = (np.float32 if self.dtype == torch.float32 else np.float64) if real else np.float64
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=rdt)
        n = pos.shape[0]
        if out is not None:
            e, ph, f = out
            for a, shape, dt in ((e, (self.K + 1,), np.float64), (ph, (self.K, n), rdt), (f, (n, 3), rdt)):
                if a is not None and (a.dtype != dt or a.shape != shape or not a.flags.c_contiguous):
                    raise ValueError("out arrays must be C-contiguous, of shapes [K+1], [K, n], [n, 3] and the "
                                     "dtypes float64, then float64 or (real=True) the plan's precision")
        else:
            e = np.empty(self.K + 1)
            ph = np.empty((self.K, n), dtype=rdt) if phi else None
            f = np.empty((n, 3), dtype=rdt) if forces else None
        dp = lambda a: a.ctypes.data_as(_dp) if a is not None else ctypes.cast(0, _dp)
        vp = lambda a: ctypes.c_void_p(a.ctypes.data) if a is not None else None
        self._stream()
        if real:
            _check(lib().pswf_compute_host_real(self._h, n, dp(pos), vp(q), dp(e), vp(ph), vp(f)), self._h)
        else:
            _check(lib().pswf_compute_host(self._h, n, dp(pos), dp(q), dp(e), dp(ph), dp(f)), self._h)
        return e, ph, f


class BatchPlan(Plan):
    """Up to b_max independent structures per call on one grid size (see
    pswf_batch_plan_create).  execute() returns energy [b_max, K+1] and phi /
    forces over the concatenated atoms (buffers of n_max rows)."""

    def __init__(self, box_max, b_max: int, n_max: int, K: int, pset, r_c: float, *, tol: float = 1e-5,
                 c: float = 0.0, c_w: float = 0.0, eta: float = 0.0, P: int = 0, grid=None, precision: int = 0,
                 flags: int = 0, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("PSWF-LR needs a CUDA device")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.K = int(K)
        self.B = int(b_max)
        self.pset = tuple(int(p) for p in pset)
        self.box = tuple(float(b) for b in box_max)
        self.dtype = torch.float64 if precision == 1 else torch.float32
        L = lib()
        box_a = (ctypes.c_double * 3)(*self.box)
        p_a = (ctypes.c_int * len(self.pset))(*self.pset)
        o = make_opts(r_c=r_c, tol=tol, c=c, c_w=c_w, eta=eta, P=P, grid=grid, precision=precision, flags=flags)
        h = _vp()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            _check(L.pswf_batch_plan_create(box_a, self.B, int(n_max), self.K, p_a, len(self.pset), ctypes.byref(o),
                                            _vp(stream), ctypes.byref(h)))
        self._h = h
        self.n_max = int(n_max)
        info = PswfInfo()
        _check(L.pswf_plan_info(self._h, ctypes.byref(info)), self._h)
        self.info = _info_dict(info)
        nbytes = max(int(self.info["workspace_bytes"]), 256)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        aligned = (self._ws.data_ptr() + 255) & ~255
        with torch.cuda.device(self.device):
            _check(L.pswf_plan_set_workspace(self._h, _vp(aligned), nbytes), self._h)
        self.n = None
        self.flags = int(flags)
        self.generation = 0

    def set_points(self, boxes, ps, offsets, pos, q):
        """boxes [b, 3], ps [b, K] (host), offsets [b+1] (host int64),
        pos cuda [n, 3], q cuda [K, n] over the concatenated atoms."""
        import torch
        boxes = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
        b = boxes.shape[0]
        ps = np.ascontiguousarray(ps, dtype=np.int32).reshape(b, self.K)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        if offsets.shape != (b + 1,):
            raise ValueError("offsets must have b + 1 entries")
        n = int(offsets[-1]) if b > 0 else 0
        if pos.dtype not in (torch.float32, torch.float64):
            pos = pos.double()
        pos = pos.contiguous()
        q = q.to(self.dtype).contiguous()
        if pos.shape != (n, 3) or q.shape != (self.K, n):
            raise ValueError("pos must be [n, 3] and q [K, n] with n = offsets[-1]")
        self._stream()
        self._tables = (boxes, ps, offsets)
        _check(lib().pswf_batch_set_points(self._h, b, boxes.ctypes.data_as(_dp), ps.ctypes.data_as(_ip),
                                           offsets.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                           _vp(pos.data_ptr() if n else 0), 1 if pos.dtype == torch.float64 else 0,
                                           _vp(q.data_ptr() if n else 0)), self._h)
        self._keep = (pos, q)
        self.n = n
        self.generation += 1

    def execute(self, energy: bool = True, phi: bool = True, forces: bool = True, out=None):
        """Returns (energy [b_max, K+1], phi [K, n_max] or None, forces [n_max, 3] or None)."""
        import torch
        if self.n is None:
            raise PswfError(-8, "execute before set_points")
        if out is None:
            e = torch.empty(self.B, self.K + 1, dtype=torch.float64, device=self.device) if energy else None
            ph = torch.empty(self.K, self.n_max, dtype=self.dtype, device=self.device) if phi else None
            f = torch.empty(self.n_max, 3, dtype=self.dtype, device=self.device) if forces else None
            out = (e, ph, f)
        e, ph, f = out
        ptr = lambda t: _vp(t.data_ptr() if (t is not None and t.numel() > 0) else 0)
        self._stream()
        _check(lib().pswf_execute(self._h, ptr(e), ptr(ph), ptr(f)), self._h)
        return e, ph, f

    def self_energy(self) -> np.ndarray:
        out = (ctypes.c_double * (self.B * self.K))()
        self._stream()
        _check(lib().pswf_self_energy(self._h, out), self._h)
        return np.array(out[:]).reshape(self.B, self.K)


class Server:
    """Continuous-batching request server (pswf_server_*).  buckets: list of
    (grid, b_max, n_max) with ascending grids."""

    def __init__(self, K: int, pset, r_c: float, buckets, *, tol: float = 1e-5, c: float = 0.0, h_max: float = 0.0,
                 inflight: int = 2, precision: int = 0, use_graphs: bool = True, P: int = 0, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("PSWF-LR needs a CUDA device")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.K = int(K)
        L = lib()
        o = PswfServerOpts()
        L.pswf_server_opts_default(ctypes.byref(o))
        o.r_c, o.tol, o.c, o.h_max, o.K = r_c, tol, c, h_max, self.K
        pset = [int(p) for p in pset]
        o.npset = len(pset)
        for i, p in enumerate(pset):
            o.pset[i] = p
        o.nbucket = len(buckets)
        for i, (g, b, n) in enumerate(buckets):
            o.grid[i], o.b_max[i], o.n_max[i] = int(g), int(b), int(n)
        o.inflight, o.precision, o.use_graphs, o.P = inflight, precision, 1 if use_graphs else 0, P
        h = _vp()
        with torch.cuda.device(self.device):
            st = L.pswf_server_create(ctypes.byref(o), ctypes.byref(h))
        if st:
            raise PswfError(st, f"{L.pswf_strerror(st).decode()}: server creation failed")
        self._h = h

    def route(self, n: int, box) -> tuple:
        """(bucket index, plan info dict of that bucket)."""
        box_a = (ctypes.c_double * 3)(*[float(b) for b in box])
        info = PswfInfo()
        r = lib().pswf_server_route(self._h, int(n), box_a, ctypes.byref(info))
        if r < 0:
            raise PswfError(r, "no bucket holds this structure")
        return r, _info_dict(info)

    def submit(self, pos: np.ndarray, q: np.ndarray, box, ps) -> int:
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        q = np.ascontiguousarray(q, dtype=np.float64)
        n = pos.shape[0]
        if q.shape != (self.K, n):
            raise ValueError("q must be [K, n]")
        box_a = (ctypes.c_double * 3)(*[float(b) for b in box])
        ps_a = (ctypes.c_int * self.K)(*[int(p) for p in ps])
        t = ctypes.c_int64()
        self._check(lib().pswf_server_submit(self._h, n, box_a, ps_a, pos.ctypes.data_as(_dp), q.ctypes.data_as(_dp),
                                             ctypes.byref(t)))
        self._n = getattr(self, "_n", {})
        self._n[t.value] = n
        return t.value

    def wait(self, ticket: int, phi: bool = True, forces: bool = True, timeout_ms: float | None = None):
        """(energy [K+1], phi [K, n] or None, forces [n, 3] or None, latency ms).
        With timeout_ms, raises PswfError (status PSWF_ETIMEOUT = -5) if the
        structure is not done by then; the ticket stays valid."""
        n = self._n[ticket]
        e = np.empty(self.K + 1)
        ph = np.empty((self.K, n)) if phi else None
        f = np.empty((n, 3)) if forces else None
        lat = ctypes.c_double()
        dp = lambda a: a.ctypes.data_as(_dp) if a is not None else ctypes.cast(0, _dp)
        t = -1.0 if timeout_ms is None else float(timeout_ms)
        st = lib().pswf_server_wait_for(self._h, ticket, t, dp(e), dp(ph), dp(f), ctypes.byref(lat))
        if st != PSWF_ETIMEOUT:
            del self._n[ticket]   # released by the server (done or failed)
            getattr(self, "_borrowed", {}).pop(ticket, None)
        self._check(st)
        return e, ph, f, lat.value

    def submit_many(self, structures, borrow: bool = False):
        """Submits [(pos [n, 3], q [K, n], box, ps), ...] in one call
        (pswf_server_submit_many; each structure's arrays are passed by
        address, float64 C-contiguous ones without a copy); returns
        (tickets, offsets) int64 arrays, offsets the running atom counts.
        borrow=True (PSWF_SUBMIT_BORROW): the server reads the arrays when
        it stages their batch instead of copying them now; they stay
        referenced by this object until wait_many releases the tickets, and
        the caller must not change them before that."""
        count = len(structures)
        pos_l = [np.ascontiguousarray(st[0], dtype=np.float64) for st in structures]
        q_l = [np.ascontiguousarray(st[1], dtype=np.float64) for st in structures]
        ns = np.fromiter((a.shape[0] for a in pos_l), dtype=np.int64, count=count)
        if any(qq.shape != (self.K, int(n)) for qq, n in zip(q_l, ns)):
            raise ValueError("q must be [K, n]")
        boxes = np.ascontiguousarray(np.array([st[2] for st in structures], dtype=np.float64).reshape(count, 3))
        ps = np.ascontiguousarray(np.array([st[3] for st in structures], dtype=np.int32).reshape(count, self.K))
        pos_a = np.fromiter((a.ctypes.data for a in pos_l), dtype=np.uintp, count=count)
        q_a = np.fromiter((a.ctypes.data for a in q_l), dtype=np.uintp, count=count)
        off = np.zeros(count + 1, dtype=np.int64)
        off[1:] = np.cumsum(ns)
        tk = np.zeros(count, dtype=np.int64)
        i64p, dpp = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_dp)
        st = lib().pswf_server_submit_many(self._h, count, ns.ctypes.data_as(i64p), boxes.ctypes.data_as(_dp),
                                           ps.ctypes.data_as(_ip), pos_a.ctypes.data_as(dpp), q_a.ctypes.data_as(dpp),
                                           tk.ctypes.data_as(i64p), PSWF_SUBMIT_BORROW if borrow else 0)
        # the structures submitted before an error have their tickets written
        self._n = getattr(self, "_n", {})
        self._borrowed = getattr(self, "_borrowed", {})
        for t, n, a, b in zip(tk.tolist(), ns.tolist(), pos_l, q_l):
            if t == 0:
                break
            self._n[t] = n
            if borrow:   # referenced by the server until the ticket is released
                self._borrowed[t] = (a, b)
        self._check(st)
        return tk, off

    def wait_many(self, tickets, offsets, phi: bool = False, forces: bool = True):
        """Waits for submit_many's tickets (pswf_server_wait_many): returns
        (energies [count, K+1], phi [K * n_total] (structure i's [K, n_i] at
        K * offsets[i]) or None, forces [n_total, 3] or None, latencies ms
        [count])."""
        tickets = np.ascontiguousarray(tickets, dtype=np.int64)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        count, ntot = len(tickets), int(offsets[-1]) if len(offsets) else 0
        e = np.empty((count, self.K + 1))
        ph = np.empty(self.K * ntot) if phi else None
        f = np.empty((ntot, 3)) if forces else None
        lat = np.empty(count)
        dp = lambda a: a.ctypes.data_as(_dp) if a is not None else ctypes.cast(0, _dp)
        i64p = ctypes.POINTER(ctypes.c_int64)
        st = lib().pswf_server_wait_many(self._h, count, tickets.ctypes.data_as(i64p), offsets.ctypes.data_as(i64p),
                                         dp(e), dp(ph), dp(f), dp(lat))
        for t in tickets.tolist():   # every ticket is released by the call
            getattr(self, "_n", {}).pop(t, None)
            getattr(self, "_borrowed", {}).pop(t, None)
        self._check(st)
        return e, ph, f, lat

    def pause(self, pause: bool = True):
        """Holds back new batches (pause=True) or resumes them."""
        self._check(lib().pswf_server_pause(self._h, int(bool(pause))))

    def stats(self) -> dict:
        b, r, a = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        st = lib().pswf_server_stats(self._h, ctypes.byref(b), ctypes.byref(r), ctypes.byref(a))
        return {"batches": b.value, "requests": r.value, "atoms": a.value, "status": st}

    def _check(self, st: int):
        if st:
            buf = ctypes.create_string_buffer(512)
            lib().pswf_server_last_error(self._h, buf, 512)
            raise PswfError(st, f"{lib().pswf_strerror(st).decode()}: {buf.value.decode()}")

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().pswf_server_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def serving_buckets(K: int, h_max: float, grids=(16, 24, 32, 40, 48, 56, 64, 72), n_cap: int = 2048,
                    density: float = 0.1, target_atoms: int = 16384):
    """Bucket list for structures up to n_cap atoms at the given density:
    per grid, structures per batch so that a batch holds about target_atoms
    (at least 4), and the atom capacity for that many of the largest
    structures the grid admits."""
    out = []
    for g in grids:
        n_struct = int(min(n_cap, math.ceil(density * (g * h_max) ** 3 * 1.05)))
        b = max(4, min(64, target_atoms // max(n_struct, 1)))
        out.append((g, b, b * n_struct))
    return out


def _make_function():
    import torch

    class _LongRange(torch.autograd.Function):
        """(pos [n,3], q [K,n]) -> (E [K], phi [K,n], F [n,3]) through one
        plan; the backward is the plan's hand-written VJP (pswf_backward),
        which needs a plan created with PSWF_FLAG_BACKWARD."""

        @staticmethod
        def forward(ctx, pos, q, plan):
            plan.set_points(pos.detach(), q.detach())
            e, ph, f = plan.execute()
            ctx.plan = plan
            ctx.gen = plan.generation
            ctx.pos_dtype = pos.dtype
            ctx.q_dtype = q.dtype
            return e[:-1].clone(), ph, f

        @staticmethod
        @torch.autograd.function.once_differentiable
        def backward(ctx, g_e, g_phi, g_f):
            plan = ctx.plan
            if plan.generation != ctx.gen:
                raise PswfError(-8, "the plan was re-run since this forward; its backward state is gone")
            need_q, need_pos = ctx.needs_input_grad[1], ctx.needs_input_grad[0]
            if not (need_q or need_pos):
                return None, None, None
            gq, gr = plan.backward(g_e, g_phi, g_f, grad_q=need_q, grad_pos=need_pos)
            gr = gr.to(ctx.pos_dtype) if gr is not None else None
            gq = gq.to(ctx.q_dtype) if gq is not None else None
            return gr, gq, None

    class _Complete(torch.autograd.Function):
        """(pos [n,3], q [K,n]) -> the complete sum per channel (E_total [K],
        phi_total [K,n], F_total [n,3]): reciprocal part (pswf_execute) +
        real-space complement (pswf_real_space) - self energy, with the
        backward through pswf_backward, pswf_real_space_backward and the
        self term E_self_c = s_c sum_i (q_i^c)^2."""

        @staticmethod
        def forward(ctx, pos, q, plan):
            pd, qd = pos.detach().contiguous(), q.detach().to(plan.dtype).contiguous()
            plan.set_points(pd, qd)
            e_k, ph_k, f_k = plan.execute()
            e_r, ph_r, f_r = plan.real_space(pd, qd)
            s = plan.self_coefficients(qd)
            qq = qd.to(torch.float64)
            E = e_k[:-1] + e_r[:-1] - s * (qq * qq).sum(1)
            phi = ph_k + ph_r - (2.0 * s[:, None] * qq).to(ph_k.dtype)
            ctx.plan, ctx.gen, ctx.rs_gen = plan, plan.generation, plan.rs_generation
            ctx.pos_dtype, ctx.q_dtype = pos.dtype, q.dtype
            ctx.save_for_backward(pd, qd, s)
            return E, phi, f_k + f_r

        @staticmethod
        @torch.autograd.function.once_differentiable
        def backward(ctx, g_e, g_phi, g_f):
            plan = ctx.plan
            if plan.generation != ctx.gen or plan.rs_generation != ctx.rs_gen:
                raise PswfError(-8, "the plan was re-run since this forward; its backward state is gone")
            pd, qd, s = ctx.saved_tensors
            need_q, need_pos = ctx.needs_input_grad[1], ctx.needs_input_grad[0]
            if not (need_q or need_pos):
                return None, None, None
            gq, gr = plan.backward(g_e, g_phi, g_f, grad_q=need_q, grad_pos=need_pos)
            gq_r, gr_r = plan.real_space_backward(pd, qd, g_e, g_phi, g_f, grad_q=need_q, grad_pos=need_pos)
            if need_q:
                ge = g_e if g_e is not None else torch.zeros_like(s)
                gself = 2.0 * s[:, None] * (ge[:, None] * qd.to(torch.float64)
                                            + (g_phi.to(torch.float64) if g_phi is not None else 0.0))
                gq = (gq.to(torch.float64) + gq_r.to(torch.float64) - gself).to(ctx.q_dtype)
            if need_pos:
                gr = (gr + gr_r).to(ctx.pos_dtype)
            return gr, gq, None

    return _LongRange, _Complete


_FN = None


def long_range(plan: "Plan", pos, q):
    """Differentiable long-range evaluation: returns (E [K] float64, phi
    [K, n], forces [n, 3]) with gradients to pos and q through the plan's
    backward kernels.  The plan must be created with flags=PSWF_FLAG_BACKWARD,
    and calls on one plan are sequential: a later forward on the same plan
    replaces the state the pending backward needs (the binding checks this
    through a generation counter)."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    if not (plan.flags & PSWF_FLAG_BACKWARD):
        raise PswfError(-8, "long_range needs a plan created with flags=PSWF_FLAG_BACKWARD")
    return _FN[0].apply(pos, q, plan)


def complete_sum(plan: "Plan", pos, q):
    """Differentiable complete lattice sum per channel (Methods,
    "Implementation details": reciprocal part + real-space complement -
    self energy): returns (E [K] float64, phi [K, n], forces [n, 3]) with
    gradients to pos and q through the plan's backward kernels and the
    real-space backward.  The plan needs flags PSWF_FLAG_BACKWARD |
    PSWF_FLAG_REAL_SPACE; calls on one plan are sequential (generation
    counters guard the pending backward)."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    need = PSWF_FLAG_BACKWARD | PSWF_FLAG_REAL_SPACE
    if (plan.flags & need) != need:
        raise PswfError(-8, "complete_sum needs a plan created with PSWF_FLAG_BACKWARD | PSWF_FLAG_REAL_SPACE")
    return _FN[1].apply(pos, q, plan)
