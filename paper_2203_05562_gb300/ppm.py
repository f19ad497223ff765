"""ctypes binding of the C ABI in ``include/ppm.h``.

Argument marshalling only: every step of the bond loop runs in the CUDA
library.  PyTorch supplies the device workspace (``torch.empty``) and the
current CUDA stream.  If the compiled library is missing this module raises;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

FP64, MIXED = 0, 1
SUBHORIZON, STANDARD, SUBHORIZON_CONJUGATE = 0, 1, 2
FIELD = dict(u=0, v=1, a=2, sigma=3, pc=4, eps_s=5, fint=6, row_ptr=7, col=8, rev=9, tforce=10, J=11)
_NCOMP = dict(u=3, v=3, a=3, sigma=6, pc=1, eps_s=1, fint=3, J=1)
STATUS_BITS = dict(nonconv=1, singular=2, nonfinite=4, family_full=8, row_full=16, unstable=32,
                   halted=64, tc_timeout=128)


class PPMError(RuntimeError):
    pass


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("model", C.c_int32),
        ("dx", C.c_double), ("horizon_factor", C.c_double),
        ("rho", C.c_double), ("K", C.c_double), ("mu", C.c_double),
        ("M", C.c_double), ("lambda_t", C.c_double), ("kappa_t", C.c_double),
        ("pc0", C.c_double), ("eta", C.c_double), ("suction", C.c_double),
        ("vg_alpha", C.c_double), ("vg_n", C.c_double), ("b1", C.c_double), ("b2", C.c_double),
        ("gravity", C.c_double * 3), ("dt", C.c_double),
        ("rebuild_every", C.c_int32), ("init_stress", C.c_int32), ("visc_form", C.c_int32),
        ("newton_max_iter", C.c_int32), ("newton_tol", C.c_double),
        ("lock_lateral", C.c_int32), ("precision", C.c_int32), ("max_family", C.c_int32),
        ("use_graph", C.c_int32), ("bond_tile", C.c_int32), ("bc", C.c_int32),
        ("load_rate", C.c_double), ("elastic", C.c_int32), ("load_layers", C.c_int32),
        ("halt_on_unstable", C.c_int32), ("contact", C.c_int32),
        ("contact_modulus", C.c_double), ("friction", C.c_double), ("contact_cutoff", C.c_double),
        ("energy_tol", C.c_double), ("plane_strain", C.c_int32),
        ("coupled", C.c_int32), ("porosity", C.c_double), ("rho_s", C.c_double),
        ("rho_w", C.c_double), ("wr_a1", C.c_double), ("wr_a2", C.c_double), ("wr_n", C.c_double),
        ("points_per_block", C.c_int32), ("bond_grid", C.c_int32), ("gather_lanes", C.c_int32),
        ("withhold_tc_product", C.c_int32),
    ]


class Column(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("pad_", C.c_int32),
                ("suction", C.c_double), ("M", C.c_double)]


class Counters(C.Structure):
    _fields_ = [("steps", C.c_int64), ("nbonds", C.c_int64), ("bond_steps", C.c_int64),
                ("plastic", C.c_int64), ("nonconv", C.c_int64), ("singular", C.c_int64),
                ("rebuilds", C.c_int64), ("pairs", C.c_int64), ("launches", C.c_int64),
                ("returns_fp64", C.c_int64), ("bond_tile", C.c_int32), ("halted_step", C.c_int32),
                ("status", C.c_uint32), ("unstable_step", C.c_int32),
                ("W_int", C.c_double), ("W_ext", C.c_double), ("W_kin", C.c_double),
                ("W_kin0", C.c_double), ("points_per_block", C.c_int32), ("bond_blocks", C.c_int32),
                ("gather_lanes", C.c_int32)]


_lib = None
_lock = threading.Lock()


def library(build_if_missing: bool = True):
    """Load ``libppm.so`` (building it in-tree when sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(path):
                raise PPMError(f"CUDA library {path} is missing; run the package build")
            L = C.CDLL(path)
            vp, pp, szp = C.c_void_p, C.POINTER(Params), C.POINTER(C.c_size_t)
            L.ppm_workspace_size.argtypes = [pp, C.c_int, C.POINTER(Column), szp]
            L.ppm_init.argtypes = [pp, C.c_int, C.POINTER(Column), vp, C.c_size_t, vp,
                                   C.POINTER(vp)]
            L.ppm_build_families.argtypes = [vp]
            L.ppm_step.argtypes = [vp, C.c_int]
            L.ppm_step_timed.argtypes = [vp, C.c_int, C.POINTER(C.c_double)]
            L.ppm_read_state.argtypes = [vp, C.c_int, vp, C.c_size_t, C.c_int]
            L.ppm_write_state.argtypes = [vp, C.c_int, vp, C.c_size_t, C.c_int]
            L.ppm_num_bonds.argtypes = [vp, C.POINTER(C.c_int64)]
            L.ppm_critical_time_step.argtypes = [vp, C.POINTER(C.c_double)]
            L.ppm_status.argtypes = [vp, C.POINTER(Counters)]
            L.ppm_info.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
            L.ppm_error_string.restype = C.c_char_p
            L.ppm_error_string.argtypes = [C.c_int]
            L.ppm_family_noalloc.argtypes = [C.c_int64, vp, C.c_double, C.c_int, vp, vp, vp,
                                             C.c_int64, vp, C.POINTER(C.c_int64)]
            L.ppm_adjoint_workspace_size.argtypes = [vp, C.c_int, C.c_int, szp]
            L.ppm_adjoint_forward.argtypes = [vp, C.c_int, C.c_int, vp, C.c_size_t]
            L.ppm_adjoint_reverse.argtypes = [vp, vp, C.c_int, C.POINTER(C.c_double)]
            L.ppm_measure_fp32_peak.argtypes = [vp, C.POINTER(C.c_double)]
            L.ppm_struct_size.restype = C.c_size_t
            L.ppm_struct_size.argtypes = [C.c_int]
            L.ppm_destroy.restype = None
            L.ppm_destroy.argtypes = [vp]
            for which, cls in ((0, Params), (1, Column), (2, Counters)):
                if L.ppm_struct_size(which) != C.sizeof(cls):
                    raise PPMError(f"ABI layout mismatch for {cls.__name__}")
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = library().ppm_error_string(rc).decode()
        raise PPMError(f"{what}: {msg} ({rc})")


def make_params(cfg: dict, precision=None, model=None, use_graph=True, max_family=0,
                bond_tile=32, points_per_block=0, bond_grid=0) -> Params:
    p = Params()
    for name, _ in Params._fields_:
        if name in ("gravity", "precision", "use_graph", "max_family", "model", "pad_",
                    "bond_tile", "points_per_block", "bond_grid"):
            continue
        if name in cfg:
            setattr(p, name, cfg[name])
    g = cfg.get("gravity", (0.0, 0.0, -9.81))
    for c in range(3):
        p.gravity[c] = g[c]
    prec = cfg.get("precision", "fp64") if precision is None else precision
    if isinstance(prec, str):
        prec = {"fp64": FP64, "mixed": MIXED}[prec]
    p.precision = prec
    p.model = cfg.get("model", 0) if model is None else model
    p.use_graph = int(use_graph)
    p.max_family = int(cfg.get("max_family", max_family))
    p.bond_tile = int(cfg.get("bond_tile", bond_tile))
    p.points_per_block = int(cfg.get("points_per_block", points_per_block))
    p.bond_grid = int(cfg.get("bond_grid", bond_grid))
    return p


def measure_fp32_peak() -> float:
    """Measured FP32 multiply-add rate of the current device (TFLOP/s),
    through ``ppm_measure_fp32_peak`` on the current stream."""
    import torch

    out = C.c_double(0.0)
    _check(library().ppm_measure_fp32_peak(C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                           C.byref(out)), "ppm_measure_fp32_peak")
    return float(out.value)


def family_noalloc(x, delta: float, max_family: int = 192, cap: int | None = None):
    """Family of the points x (torch CUDA tensor (3, n), float64) through
    ``ppm_family_noalloc``, which allocates no device memory itself; the
    output tensors are allocated here by the caller side.  Returns
    (row_ptr, col, rev) as CUDA tensors."""
    import torch

    if x.dtype != torch.float64 or not x.is_cuda or x.dim() != 2 or x.shape[0] != 3:
        raise PPMError("x must be a (3, n) float64 CUDA tensor")
    x = x.contiguous()
    n = x.shape[1]
    cap = n * max_family if cap is None else cap
    row_ptr = torch.empty(n + 1, dtype=torch.int32, device=x.device)
    col = torch.empty(max(cap, 1), dtype=torch.int32, device=x.device)
    rev = torch.empty(max(cap, 1), dtype=torch.int32, device=x.device)
    nb = C.c_int64(0)
    # the library uses the current device's copy of its scratch array
    with torch.cuda.device(x.device):
        stream = torch.cuda.current_stream(x.device).cuda_stream
        _check(library().ppm_family_noalloc(n, C.c_void_p(x.data_ptr()), float(delta),
                                            int(max_family), C.c_void_p(row_ptr.data_ptr()),
                                            C.c_void_p(col.data_ptr()), C.c_void_p(rev.data_ptr()),
                                            cap, C.c_void_p(stream), C.byref(nb)),
               "ppm_family_noalloc")
    B = int(nb.value)
    return row_ptr, col[:B], rev[:B]


class Simulation:
    """One context of the library: a soil column, or an ensemble of columns
    when ``columns`` (a list of dicts with nx, ny, nz, suction, M) is given."""

    def __init__(self, cfg: dict, columns=None, precision=None, model=None, device=None,
                 use_graph=True, max_family=0, bond_tile=32, points_per_block=0, bond_grid=0):
        import torch

        if not torch.cuda.is_available():
            raise PPMError("no CUDA device available")
        self._torch = torch
        L = library()
        self.params = make_params(cfg, precision, model, use_graph, max_family, bond_tile,
                                  points_per_block, bond_grid)
        self.fp64 = self.params.precision == FP64
        self.dtype = np.float64 if self.fp64 else np.float32
        self.tdtype = torch.float64 if self.fp64 else torch.float32
        cols = None
        ncols = 0
        if columns:
            ncols = len(columns)
            cols = (Column * ncols)()
            for q, cdef in enumerate(columns):
                cols[q].nx, cols[q].ny, cols[q].nz = cdef["nx"], cdef["ny"], cdef["nz"]
                cols[q].suction, cols[q].M = cdef["suction"], cdef["M"]
        self._cols = cols
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        nbytes = C.c_size_t(0)
        _check(L.ppm_workspace_size(C.byref(self.params), ncols, cols, C.byref(nbytes)),
               "ppm_workspace_size")
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8,
                                         device=self.device)
            base = self.workspace.data_ptr()
            aligned = (base + 255) // 256 * 256
            self.stream = torch.cuda.current_stream(self.device)
            ctx = C.c_void_p()
            _check(L.ppm_init(C.byref(self.params), ncols, cols, C.c_void_p(aligned),
                              C.c_size_t(nbytes.value), C.c_void_p(self.stream.cuda_stream),
                              C.byref(ctx)), "ppm_init")
        self._ctx = ctx
        dt = C.c_double(0)
        n = C.c_int64(0)
        _check(L.ppm_info(ctx, C.byref(dt), C.byref(n)), "ppm_info")
        self.dt = dt.value
        self.n = int(n.value)

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if getattr(self, "_ctx", None):
            library().ppm_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the four calls of the method --------------------------------------
    def build_families(self):
        _check(library().ppm_build_families(self._ctx), "ppm_build_families")

    def step(self, n_steps: int = 1):
        _check(library().ppm_step(self._ctx, int(n_steps)), "ppm_step")

    def step_timed(self, n_steps: int = 1):
        ms = (C.c_double * 3)(0.0, 0.0, 0.0)
        _check(library().ppm_step_timed(self._ctx, int(n_steps), ms), "ppm_step_timed")
        return [ms[0], ms[1], ms[2]]

    # -- adjoint -----------------------------------------------------------
    def adjoint_forward(self, n_steps: int, ckpt_every: int):
        """Run n_steps from the initial state keeping checkpoints for the
        reverse sweep (workspace allocated here with torch)."""
        nbytes = C.c_size_t(0)
        _check(library().ppm_adjoint_workspace_size(self._ctx, int(n_steps), int(ckpt_every),
                                                    C.byref(nbytes)), "ppm_adjoint_workspace_size")
        self._adj_ws = self._torch.empty(int(nbytes.value) + 256, dtype=self._torch.uint8,
                                         device=self.device)
        base = (self._adj_ws.data_ptr() + 255) // 256 * 256
        _check(library().ppm_adjoint_forward(self._ctx, int(n_steps), int(ckpt_every),
                                             C.c_void_p(base), nbytes.value), "ppm_adjoint_forward")

    def adjoint_reverse(self, dJ_du):
        """dJ/d(M, eta, suction, pc0) for dJ/du of the final displacement
        (a (3, n) float64 CUDA tensor or numpy array)."""
        grad = (C.c_double * 4)()
        if hasattr(dJ_du, "data_ptr"):
            t = dJ_du.to(device=self.device, dtype=self._torch.float64).contiguous()
            _check(library().ppm_adjoint_reverse(self._ctx, C.c_void_p(t.data_ptr()), 1, grad),
                   "ppm_adjoint_reverse")
        else:
            a = np.ascontiguousarray(np.asarray(dJ_du, np.float64).reshape(3 * self.n))
            _check(library().ppm_adjoint_reverse(self._ctx, C.c_void_p(a.ctypes.data), 0, grad),
                   "ppm_adjoint_reverse")
        return np.array([grad[q] for q in range(4)])

    def critical_time_step(self) -> float:
        """Eq. 65 over the current family and positions (ppm_critical_time_step)."""
        dt = C.c_double(0.0)
        _check(library().ppm_critical_time_step(self._ctx, C.byref(dt)), "ppm_critical_time_step")
        return float(dt.value)

    def num_bonds(self) -> int:
        nb = C.c_int64(0)
        _check(library().ppm_num_bonds(self._ctx, C.byref(nb)), "ppm_num_bonds")
        return int(nb.value)

    def _shape(self, field):
        if field in _NCOMP:
            return (_NCOMP[field], self.n) if _NCOMP[field] > 1 else (self.n,), self.dtype
        if field == "row_ptr":
            return (self.n + 1,), np.int32
        nb = self.num_bonds()
        if field in ("col", "rev"):
            return (nb,), np.int32
        if field == "tforce":
            return (3, nb), self.dtype
        raise KeyError(field)

    def read(self, field: str, device: bool = False, out=None):
        """A state field as a numpy array (or a torch tensor on the device):
        u, v, a, fint (3, n); sigma (6, n: xx, yy, zz, yz, xz, xy); pc, eps_s
        and J (the volume ratio of the coupled mode) (n,); row_ptr, col,
        rev and tforce for the family.  ``out`` may be a preallocated host
        numpy array (e.g. pinned)."""
        shape, dt = self._shape(field)
        if out is not None:
            if out.dtype != dt or out.size != int(np.prod(shape)) or not out.flags.c_contiguous:
                raise PPMError(f"out must be a contiguous {np.dtype(dt).name} array of {shape}")
            _check(library().ppm_read_state(self._ctx, FIELD[field], C.c_void_p(out.ctypes.data),
                                            out.nbytes, 0), "ppm_read_state")
            return out
        if device:
            tdt = {np.int32: self._torch.int32, np.float32: self._torch.float32,
                   np.float64: self._torch.float64}[dt]
            out = self._torch.empty(shape, dtype=tdt, device=self.device)
            nbytes = out.numel() * out.element_size()
            _check(library().ppm_read_state(self._ctx, FIELD[field], C.c_void_p(out.data_ptr()),
                                            nbytes, 1), "ppm_read_state")
            return out
        out = np.empty(shape, dtype=dt)
        _check(library().ppm_read_state(self._ctx, FIELD[field], C.c_void_p(out.ctypes.data),
                                        out.nbytes, 0), "ppm_read_state")
        return out

    def write(self, field: str, values):
        """Overwrites a state field (numpy array or torch tensor, the layout
        of ``read``).  Writing u makes the next step rebuild the family;
        family fields are read-only."""
        if hasattr(values, "data_ptr"):
            t = values.to(device=self.device, dtype=self.tdtype).contiguous()
            _check(library().ppm_write_state(self._ctx, FIELD[field], C.c_void_p(t.data_ptr()),
                                             t.numel() * t.element_size(), 1), "ppm_write_state")
            return
        shape, dt = self._shape(field)
        a = np.ascontiguousarray(np.asarray(values, dtype=dt).reshape(shape))
        _check(library().ppm_write_state(self._ctx, FIELD[field], C.c_void_p(a.ctypes.data),
                                         a.nbytes, 0), "ppm_write_state")

    def status(self) -> dict:
        """Counters and energies of ``ppm_status`` with the status bits as
        names in ``flags`` (nonconv, singular, nonfinite, family_full,
        row_full, unstable, halted, tc_timeout)."""
        c = Counters()
        _check(library().ppm_status(self._ctx, C.byref(c)), "ppm_status")
        out = {name: getattr(c, name) for name, _ in Counters._fields_ if "pad" not in name}
        out["flags"] = [k for k, b in STATUS_BITS.items() if c.status & b]
        return out
