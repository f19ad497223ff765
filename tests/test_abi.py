"""The C-ABI library builds, loads and exports every declared symbol, and
rejects invalid parameters -- all without a GPU."""
import ctypes as C
import os
import re

import pytest

import ppm_inputs as pi
from paper_2203_05562_gb300 import ppm as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ppm_\w+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = P.library()
    names = declared_functions()
    assert "ppm_step" in names and "ppm_init" in names
    for name in names:
        assert hasattr(L, name), name


def test_struct_layout_matches_binding():
    L = P.library()
    assert L.ppm_struct_size(0) == C.sizeof(P.Params)
    assert L.ppm_struct_size(1) == C.sizeof(P.Column)
    assert L.ppm_struct_size(2) == C.sizeof(P.Counters)


def _ws(cfg, **kw):
    p = P.make_params(cfg, **kw)
    n = C.c_size_t(0)
    rc = P.library().ppm_workspace_size(C.byref(p), 0, None, C.byref(n))
    return rc, n.value


def test_workspace_size_and_invalid_parameters():
    cfg = pi.config(0)
    rc, nbytes = _ws(cfg, precision=P.FP64)
    assert rc == 0 and nbytes > 0
    rc2, nbytes_mixed = _ws(cfg, precision=P.MIXED)
    assert rc2 == 0 and nbytes_mixed < nbytes
    for bad in (dict(dx=0.0), dict(K=-1.0), dict(b1=0.5), dict(lambda_t=0.01),
                dict(nz=0), dict(nx=2000), dict(newton_max_iter=0), dict(max_family=300)):
        rc, _ = _ws(dict(cfg, **bad))
        assert rc == -1, bad
    rc, _ = _ws(cfg, model=5)
    assert rc == -1


def test_error_strings():
    L = P.library()
    assert L.ppm_error_string(0) == b"ok"
    assert b"workspace" in L.ppm_error_string(-2)


def test_init_rejects_null_and_misaligned_workspace():
    L = P.library()
    p = P.make_params(pi.config(0))
    ctx = C.c_void_p()
    assert L.ppm_init(C.byref(p), 0, None, None, 0, None, C.byref(ctx)) == -1
    assert L.ppm_init(C.byref(p), 0, None, C.c_void_p(0x1001), 1 << 30, None, C.byref(ctx)) == -1
    assert not ctx.value


def _ws_cols(cfg, columns):
    p = P.make_params(cfg)
    cols = (P.Column * len(columns))()
    for q, c in enumerate(columns):
        cols[q].nx, cols[q].ny, cols[q].nz = c["nx"], c["ny"], c["nz"]
        cols[q].suction, cols[q].M = c["suction"], c["M"]
    n = C.c_size_t(0)
    return P.library().ppm_workspace_size(C.byref(p), len(columns), cols, C.byref(n))


def test_the_later_parameters_are_validated():
    # the energy tolerance, the substrate, plane strain (y period > 4 delta),
    # the coupled mode (material ranges) and the launch-shape switches, without a GPU
    cfg = pi.small_config(6, 13, 5)
    assert _ws(cfg)[0] == 0
    good = [dict(energy_tol=5e-2), dict(contact=1), dict(plane_strain=1), dict(coupled=1),
            dict(plane_strain=1, contact=1, coupled=1, halt_on_unstable=1),
            dict(bond_tile=128), dict(points_per_block=2, bond_grid=2), dict(gather_lanes=8),
            dict(withhold_tc_product=1)]
    for kw in good:
        assert _ws(dict(cfg, **kw))[0] == 0, kw
    bad = [dict(energy_tol=-1e-2), dict(energy_tol=float("inf")), dict(contact=2),
           dict(contact=1, contact_cutoff=0.0), dict(contact=1, friction=-0.1),
           dict(plane_strain=2), dict(plane_strain=1, ny=12), dict(coupled=2),
           dict(coupled=1, porosity=0.0), dict(coupled=1, porosity=1.0),
           dict(coupled=1, rho_s=0.0), dict(coupled=1, wr_a1=0.0), dict(coupled=1, wr_n=1.0),
           dict(coupled=1, wr_a2=-1.0), dict(halt_on_unstable=2), dict(bond_tile=96),
           dict(points_per_block=3), dict(bond_grid=3), dict(gather_lanes=5),
           dict(withhold_tc_product=2)]
    for kw in bad:
        assert _ws(dict(cfg, **kw))[0] == -1, kw
    # plane strain and the coupled mode take one column
    two = [dict(nx=6, ny=13, nz=5, suction=1e3, M=1.2)] * 2
    assert _ws_cols(cfg, two) == 0
    assert _ws_cols(dict(cfg, plane_strain=1), two) == -1
    assert _ws_cols(dict(cfg, coupled=1), two) == -1
