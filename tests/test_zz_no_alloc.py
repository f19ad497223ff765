"""The allocation-free family entry point (ppm_family_noalloc) against the
regular one (ppm_build_families of a context) on the same positions.

The regular entry point takes its scratch from a workspace the caller
allocates; the allocation-free one uses a fixed array inside the library,
for callers that cannot allocate device memory (real-time loops that must
not enter the allocator, hosts whose device memory belongs to another
allocator).  Both must give the same family, bit for bit, on calls in a
row: the array keeps the last call's contents, so a later call must not see
an earlier call's leftovers (a large column first, then a smaller perturbed
one, then again after calls that ran out of space).  This file is collected
last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import ppm_inputs as pi

pytestmark = pytest.mark.gpu

PPM_EINVAL, PPM_ENOSPACE = -1, -2


def _context_family(cfg, u):
    from paper_2203_05562_gb300 import Simulation
    sim = Simulation(cfg, precision="fp64")
    sim.write("u", u)
    sim.build_families()
    out = sim.read("row_ptr"), sim.read("col"), sim.read("rev")
    sim.close()
    return out


def _positions(cfg, u):
    n = pi.num_points(cfg)
    idx = np.arange(n)
    ijk = np.stack([idx % cfg["nx"], (idx // cfg["nx"]) % cfg["ny"], idx // (cfg["nx"] * cfg["ny"])])
    return ijk.astype(np.float64) * cfg["dx"] + u          # (ix * dx) + u, each rounded once


def _raw_call(x, delta, max_family, cap):
    """ppm_family_noalloc through ctypes; returns (rc, row_ptr, nbonds)."""
    import torch
    from paper_2203_05562_gb300.ppm import library
    n = x.shape[1]
    row_ptr = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
    col = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    rev = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    nb = C.c_int64(-1)
    rc = library().ppm_family_noalloc(n, C.c_void_p(x.data_ptr()), float(delta), int(max_family),
                                      C.c_void_p(row_ptr.data_ptr()), C.c_void_p(col.data_ptr()),
                                      C.c_void_p(rev.data_ptr()), int(cap),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                      C.byref(nb))
    torch.cuda.synchronize()
    return rc, row_ptr.cpu().numpy(), nb.value


def _check_against_regular(cfg, amp, seed):
    import torch
    from paper_2203_05562_gb300.ppm import family_noalloc
    u = pi.perturbation(cfg, amp * cfg["dx"], seed=seed)
    rp, col, rev = _context_family(cfg, u)
    x = torch.from_numpy(_positions(cfg, u)).cuda()
    delta = cfg["horizon_factor"] * cfg["dx"]
    grp, gcol, grev = family_noalloc(x, delta, max_family=192)
    torch.cuda.synchronize()
    assert np.array_equal(grp.cpu().numpy(), rp)
    assert np.array_equal(gcol.cpu().numpy(), col)
    assert np.array_equal(grev.cpu().numpy(), rev)
    return x, delta, rp


def test_no_alloc_family_matches_regular_entry_point_on_calls_in_a_row():
    # the 128,000-point column first, then a smaller perturbed column whose
    # cell grid, counts and scan occupy only part of what the first call wrote
    _check_against_regular(pi.config(1), 0.0, seed=31)
    _check_against_regular(pi.small_config(20, 20, 40, dx=0.0025), 0.3, seed=32)


def test_no_alloc_reports_running_out_of_space_and_recovers():
    import torch
    cfg = pi.small_config(20, 20, 40, dx=0.0025)
    x, delta, rp = _check_against_regular(cfg, 0.2, seed=33)
    nbonds = int(rp[-1])
    # bonds beyond cap: every row empty, no bonds reported
    rc, grp, nb = _raw_call(x, delta, 192, nbonds - 1)
    assert rc == PPM_ENOSPACE and nb == 0 and np.all(grp == 0)
    # rows beyond max_family: those points get empty rows, the others keep theirs
    rc, grp, nb = _raw_call(x, delta, 100, nbonds)
    assert rc == PPM_ENOSPACE
    full = np.diff(rp) > 100
    assert full.any() and np.all(np.diff(grp)[full] == 0)
    assert np.array_equal(np.diff(grp)[~full], np.diff(rp)[~full]) and nb == int(grp[-1])
    # the next call starts clean: the same family as the regular entry point
    _check_against_regular(pi.small_config(12, 10, 9, dx=0.0025), 0.25, seed=34)


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2203_05562_gb300.ppm import library

    L = library()
    n = 262145
    buf = torch.zeros(1, dtype=torch.int32, device="cuda")
    nb = C.c_int64(-1)
    rc = L.ppm_family_noalloc(n, C.c_void_p(buf.data_ptr()), 0.01, 192, C.c_void_p(buf.data_ptr()),
                              C.c_void_p(buf.data_ptr()), C.c_void_p(buf.data_ptr()), 1, None,
                              C.byref(nb))
    assert rc == PPM_EINVAL and nb.value == -1
