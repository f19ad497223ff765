"""Plain FP64 CPU oracle of the per-step bond loop (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never calls it, and it
shares no code with the CUDA path: the arithmetic lives in ``ppm_oracle.c``
(plain C, FP64, ``-ffp-contract=off``); this module only builds it and
marshals numpy arrays through ctypes.

Each wrapped function cites the passage of Menon & Song (arXiv:2203.05562)
it follows; see ``ppm_oracle.c`` for the loops themselves.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppm_oracle.c")
_LIB = os.path.join(_HERE, "libppm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, FP64, no contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "ppm_oracle.h")))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("model", C.c_int32),
        ("dx", C.c_double), ("horizon_factor", C.c_double),
        ("rho", C.c_double), ("K", C.c_double), ("mu", C.c_double),
        ("M", C.c_double), ("lambda_t", C.c_double), ("kappa_t", C.c_double),
        ("pc0", C.c_double), ("eta", C.c_double),
        ("suction", C.c_double), ("vg_alpha", C.c_double), ("vg_n", C.c_double),
        ("b1", C.c_double), ("b2", C.c_double),
        ("gravity", C.c_double * 3), ("dt", C.c_double),
        ("rebuild_every", C.c_int32), ("init_stress", C.c_int32), ("visc_form", C.c_int32),
        ("newton_max_iter", C.c_int32), ("newton_tol", C.c_double),
        ("lock_lateral", C.c_int32), ("bc", C.c_int32), ("load_rate", C.c_double),
        ("elastic", C.c_int32), ("load_layers", C.c_int32),
        ("halt_on_unstable", C.c_int32), ("contact", C.c_int32),
        ("contact_modulus", C.c_double), ("friction", C.c_double), ("contact_cutoff", C.c_double),
        ("energy_tol", C.c_double), ("plane_strain", C.c_int32),
        ("coupled", C.c_int32), ("porosity", C.c_double), ("rho_s", C.c_double),
        ("rho_w", C.c_double), ("wr_a1", C.c_double), ("wr_a2", C.c_double), ("wr_n", C.c_double),
    ]


class State(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("cap", C.c_int64), ("nbonds", C.c_int64),
        ("u", C.c_void_p), ("v", C.c_void_p), ("a", C.c_void_p),
        ("sig", C.c_void_p), ("pc", C.c_void_p), ("eps_s", C.c_void_p),
        ("fint", C.c_void_p), ("tforce", C.c_void_p),
        ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("rev", C.c_void_p),
        ("step", C.c_int64),
        ("W_int", C.c_double), ("W_ext", C.c_double), ("W_kin", C.c_double), ("W_kin0", C.c_double),
        ("n_plastic", C.c_int64), ("n_nonconv", C.c_int64), ("n_singular", C.c_int64),
        ("n_overflow", C.c_int64), ("unstable", C.c_int64), ("halted_step", C.c_int64),
        ("unstable_step", C.c_int64), ("J", C.c_void_p),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp, ip, pp = C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(Params)
            L.ppmo_saturation.restype = C.c_double
            L.ppmo_saturation.argtypes = [C.c_double, C.c_double, C.c_double]
            L.ppmo_time_step.restype = C.c_double
            L.ppmo_time_step.argtypes = [pp]
            L.ppmo_family.restype = C.c_int64
            L.ppmo_family.argtypes = [C.c_int64, dp, ip, C.c_double, C.c_int64, ip, ip, ip]
            L.ppmo_reference_positions.restype = None
            L.ppmo_reference_positions.argtypes = [pp, dp]
            L.ppmo_bond_kinematics.argtypes = [pp, C.c_int64, dp, dp, ip, ip, dp, dp, ip, ip]
            L.ppmo_full_horizon_L.argtypes = [pp, C.c_int64, dp, dp, ip, ip, dp]
            L.ppmo_material_update.argtypes = [pp, dp, C.c_double, dp, C.c_double, dp, dp, dp, ip]
            L.ppmo_return_residual.restype = None
            L.ppmo_return_residual.argtypes = [pp, C.c_double, C.c_double, C.c_double, C.c_double,
                                               dp, dp, dp]
            L.ppmo_internal_force.argtypes = [pp, C.c_int64, dp, dp, ip, ip, ip, dp]
            L.ppmo_init.argtypes = [pp, dp, C.POINTER(State)]
            L.ppmo_step.argtypes = [pp, C.POINTER(State), C.c_int]
            L.ppmo_init_with_stress.argtypes = [pp, dp, dp, C.POINTER(State)]
            L.ppmo_init_state.argtypes = [pp, dp, dp, dp, C.POINTER(State)]
            L.ppmo_initial_stress.restype = None
            L.ppmo_initial_stress.argtypes = [pp, dp]
            L.ppmo_objective_gradient.argtypes = [pp, dp, C.c_int, C.c_int64, dp, dp]
            for name in ("ppmo_coupled_saturation", "ppmo_coupled_density"):
                getattr(L, name).restype = C.c_double
                getattr(L, name).argtypes = [pp, C.c_double, C.c_double]
            L.ppmo_coupled_porosity.restype = C.c_double
            L.ppmo_coupled_porosity.argtypes = [pp, C.c_double]
            L.ppmo_critical_time_step.restype = C.c_double
            L.ppmo_critical_time_step.argtypes = [pp, C.POINTER(State)]
            L.ppmo_num_threads.restype = C.c_int
            L.ppmo_set_num_threads.argtypes = [C.c_int]
            L.ppmo_set_num_threads.restype = None
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def make_params(cfg: dict) -> Params:
    """Fill the oracle's parameter struct from a configuration dict
    (keys as produced by ``ppm_inputs.config``)."""
    p = Params()
    for name, _ in Params._fields_:
        if name in ("gravity", "pad_"):
            continue
        if name in cfg:
            setattr(p, name, cfg[name])
    g = cfg.get("gravity", (0.0, 0.0, -9.81))
    for c in range(3):
        p.gravity[c] = g[c]
    return p


def saturation(suction, alpha, n):
    """van Genuchten S_r standing in for the garbled Eq. 15."""
    return lib().ppmo_saturation(suction, alpha, n)


def coupled_saturation(cfg, J, suction):
    """Eq. 15 as read (R37): S_r at volume ratio J and suction."""
    return lib().ppmo_coupled_saturation(C.byref(make_params(cfg)), float(J), float(suction))


def coupled_porosity(cfg, J):
    """Eq. 16: porosity at volume ratio J."""
    return lib().ppmo_coupled_porosity(C.byref(make_params(cfg)), float(J))


def coupled_density(cfg, J, suction):
    """Eq. 48 per current volume: rho_s (1 - phi) + rho_w S_r phi."""
    return lib().ppmo_coupled_density(C.byref(make_params(cfg)), float(J), float(suction))


def time_step(cfg) -> float:
    return lib().ppmo_time_step(C.byref(make_params(cfg)))


def reference_positions(cfg) -> np.ndarray:
    p = make_params(cfg)
    n = p.nx * p.ny * p.nz
    X0 = np.zeros(3 * n)
    lib().ppmo_reference_positions(C.byref(p), _d(X0))
    return X0.reshape(3, n)


def family(x: np.ndarray, delta: float, group=None, cap=None):
    """Eq. 1 by brute force.  x: (3, n).  Returns (row_ptr, col, rev)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[1]
    if cap is None:
        cap = max(1, n * 256)
    row_ptr = np.zeros(n + 1, np.int32)
    col = np.zeros(cap, np.int32)
    rev = np.zeros(cap, np.int32)
    g = None
    if group is not None:
        g = np.ascontiguousarray(group, dtype=np.int32)
    B = lib().ppmo_family(n, _d(x), _i(g) if g is not None else None, delta, cap,
                          _i(row_ptr), _i(col), _i(rev))
    if B < 0:
        raise RuntimeError(f"family exceeds capacity {cap}")
    return row_ptr, col[:B].copy(), rev[:B].copy()


def bond_kinematics(cfg, x, vel, row_ptr, col):
    """Eq. 23, 25: per-bond K_b (B,6), L_b (B,3,3), |S_b| and active flag."""
    p = make_params(cfg)
    x = np.ascontiguousarray(x, np.float64)
    vel = np.ascontiguousarray(vel, np.float64)
    n = x.shape[1]
    B = int(row_ptr[n])
    Kb = np.zeros((max(B, 1), 6))
    Lb = np.zeros((max(B, 1), 9))
    cnt = np.zeros(max(B, 1), np.int32)
    act = np.zeros(max(B, 1), np.int32)
    rp = np.ascontiguousarray(row_ptr, np.int32)
    cl = np.ascontiguousarray(col, np.int32)
    lib().ppmo_bond_kinematics(C.byref(p), n, _d(x), _d(vel), _i(rp), _i(cl),
                               _d(Kb), _d(Lb), _i(cnt), _i(act))
    return Kb[:B], Lb[:B].reshape(B, 3, 3), cnt[:B], act[:B]


def full_horizon_L(cfg, x, vel, row_ptr, col):
    """Eq. 5 and 8: standard (full-horizon) velocity gradient per point."""
    p = make_params(cfg)
    x = np.ascontiguousarray(x, np.float64)
    vel = np.ascontiguousarray(vel, np.float64)
    n = x.shape[1]
    L = np.zeros((n, 9))
    lib().ppmo_full_horizon_L(C.byref(p), n, _d(x), _d(vel),
                              _i(np.ascontiguousarray(row_ptr, np.int32)),
                              _i(np.ascontiguousarray(col, np.int32)), _d(L))
    return L.reshape(n, 3, 3)


def material_update(cfg, sig, pc, L, dt):
    """Sec. 2.3 / 3.2.1 at one point: returns (sig6, pc, deps_s, flags)."""
    p = make_params(cfg)
    s_in = np.ascontiguousarray(sig, np.float64)
    Lf = np.ascontiguousarray(np.asarray(L, np.float64).reshape(9))
    s_out = np.zeros(6)
    pc_out = np.zeros(1)
    des = np.zeros(1)
    fl = np.zeros(1, np.int32)
    rc = lib().ppmo_material_update(C.byref(p), _d(s_in), float(pc), _d(Lf), float(dt),
                                    _d(s_out), _d(pc_out), _d(des), _i(fl))
    if rc != 0:
        raise RuntimeError("material update failed")
    return s_out, float(pc_out[0]), float(des[0]), int(fl[0])


def return_residual(cfg, c, p_tr, q_tr, pc_n, x):
    """Eq. 73-75 residual and exact Jacobian at x = (p, q, pc)."""
    p = make_params(cfg)
    xv = np.ascontiguousarray(x, np.float64)
    r = np.zeros(3)
    J = np.zeros(9)
    lib().ppmo_return_residual(C.byref(p), c, p_tr, q_tr, pc_n, _d(xv), _d(r), _d(J))
    return r, J.reshape(3, 3)


def internal_force(cfg, x, sig, row_ptr, col, rev):
    """Eq. 49 with every bond carrying its point's stress: f (3, n)."""
    p = make_params(cfg)
    x = np.ascontiguousarray(x, np.float64)
    sig = np.ascontiguousarray(sig, np.float64)
    n = x.shape[1]
    f = np.zeros(3 * n)
    lib().ppmo_internal_force(C.byref(p), n, _d(x), _d(sig),
                              _i(np.ascontiguousarray(row_ptr, np.int32)),
                              _i(np.ascontiguousarray(col, np.int32)),
                              _i(np.ascontiguousarray(rev, np.int32)), _d(f))
    return f.reshape(3, n)


def objective(cfg, v0, n_steps):
    """J = sum over the top layer of u_x^2 + u_y^2 after n_steps (forward only)."""
    r = Run(cfg, v0)
    r.step(n_steps)
    nxy = r.p.nx * r.p.ny
    top = slice(r.n - nxy, r.n)
    return float((r.u[0, top] ** 2).sum() + (r.u[1, top] ** 2).sum())


def objective_gradient(cfg, v0, n_steps, cap_per_point=256):
    """J and dJ/d(M, eta, suction, pc0) by the reverse of every step."""
    p = make_params(cfg)
    n = p.nx * p.ny * p.nz
    v = np.ascontiguousarray(v0, np.float64).reshape(3 * n) if v0 is not None else None
    J = np.zeros(1)
    g = np.zeros(4)
    rc = lib().ppmo_objective_gradient(C.byref(p), _d(v) if v is not None else None, int(n_steps),
                                       n * cap_per_point, _d(J), _d(g))
    if rc != 0:
        raise RuntimeError(f"ppmo_objective_gradient failed ({rc})")
    return float(J[0]), g


def initial_stress(cfg) -> np.ndarray:
    """R13 geostatic initial effective stress (6, n), O(n)."""
    p = make_params(cfg)
    n = p.nx * p.ny * p.nz
    sig = np.zeros(6 * n)
    lib().ppmo_initial_stress(C.byref(p), _d(sig))
    return sig.reshape(6, n)


def set_threads(t: int):
    lib().ppmo_set_num_threads(int(t))


def num_threads() -> int:
    return int(lib().ppmo_num_threads())


class Run:
    """One soil column stepped by the oracle (Alg. 2).  Arrays are numpy
    views in the oracle's component-major layout."""

    def __init__(self, cfg: dict, v0: np.ndarray | None = None, cap_per_point: int = 256,
                 sig0: np.ndarray | None = None, u0: np.ndarray | None = None):
        self.cfg = dict(cfg)
        self.p = make_params(self.cfg)
        n = self.p.nx * self.p.ny * self.p.nz
        self.n = n
        cap = max(1, n * cap_per_point)
        self.u = np.zeros((3, n))
        self.v = np.zeros((3, n))
        self.a = np.zeros((3, n))
        self.sig = np.zeros((6, n))
        self.pc = np.zeros(n)
        self.eps_s = np.zeros(n)
        self.fint = np.zeros((3, n))
        self.tforce = np.zeros((3, cap))
        self.row_ptr = np.zeros(n + 1, np.int32)
        self.col = np.zeros(cap, np.int32)
        self.rev = np.zeros(cap, np.int32)
        self.J = np.ones(n)
        s = State()
        s.n, s.cap = n, cap
        for name in ("u", "v", "a", "sig", "pc", "eps_s", "fint", "tforce", "row_ptr", "col", "rev", "J"):
            setattr(s, name, getattr(self, name).ctypes.data)
        self.s = s
        v0a = None if v0 is None else np.ascontiguousarray(v0, np.float64).reshape(3 * n)
        self._v0 = v0a
        s0 = None if sig0 is None else np.ascontiguousarray(sig0, np.float64).reshape(6 * n)
        self._sig0 = s0
        u0a = None if u0 is None else np.ascontiguousarray(u0, np.float64).reshape(3 * n)
        self._u0 = u0a
        rc = lib().ppmo_init_state(C.byref(self.p), _d(u0a) if u0a is not None else None,
                                   _d(v0a) if v0a is not None else None,
                                   _d(s0) if s0 is not None else None, C.byref(s))
        if rc != 0:
            raise RuntimeError(f"ppmo_init failed ({rc})")

    def step(self, n_steps: int = 1):
        rc = lib().ppmo_step(C.byref(self.p), C.byref(self.s), int(n_steps))
        if rc != 0:
            raise RuntimeError(f"ppmo_step failed ({rc})")

    @property
    def nbonds(self) -> int:
        return int(self.s.nbonds)

    def critical_time_step(self) -> float:
        """Eq. 65 (reading R30) over the current family and positions."""
        return float(lib().ppmo_critical_time_step(C.byref(self.p), C.byref(self.s)))

    @property
    def steps_done(self) -> int:
        return int(self.s.step)

    def family(self):
        B = self.nbonds
        return self.row_ptr.copy(), self.col[:B].copy(), self.rev[:B].copy()

    def positions(self):
        return reference_positions(self.cfg) + self.u

    def energies(self):
        s = self.s
        return dict(W_int=s.W_int, W_ext=s.W_ext, W_kin=s.W_kin, W_kin0=s.W_kin0)

    def counters(self):
        s = self.s
        return dict(plastic=s.n_plastic, nonconv=s.n_nonconv, singular=s.n_singular,
                    overflow=s.n_overflow, unstable=s.unstable, halted_step=s.halted_step,
                    unstable_step=s.unstable_step)
