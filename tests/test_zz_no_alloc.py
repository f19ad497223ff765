"""The allocation-free family entry point (ppm_family_noalloc) against the
regular one (ppm_build_families of a context) on the same positions.

The regular entry point takes its scratch from a workspace the caller
allocates; the allocation-free one uses a fixed array inside the library,
for callers that cannot allocate device memory (for instance while a stream
is being captured into a CUDA graph).  Both must give the same family, bit
for bit, on two calls in a row -- the second call must not see the first
call's leftovers.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import ppm_inputs as pi

pytestmark = pytest.mark.gpu


def _context_family(cfg, u):
    from paper_2203_05562_gb300 import Simulation
    sim = Simulation(cfg, precision="fp64")
    sim.write("u", u)
    sim.build_families()
    return sim.read("row_ptr"), sim.read("col"), sim.read("rev")


def _positions(cfg, u):
    n = pi.num_points(cfg)
    idx = np.arange(n)
    ijk = np.stack([idx % cfg["nx"], (idx // cfg["nx"]) % cfg["ny"], idx // (cfg["nx"] * cfg["ny"])])
    return ijk.astype(np.float64) * cfg["dx"] + u          # (ix * dx) + u, each rounded once


def test_no_alloc_family_matches_regular_entry_point_twice():
    import torch
    from paper_2203_05562_gb300.ppm import family_noalloc, library

    cases = [pi.small_config(20, 20, 40, dx=0.0025), pi.config(1)]
    amps = [0.3, 0.0]
    for rnd, (cfg, amp) in enumerate(zip(cases, amps)):
        u = pi.perturbation(cfg, amp * cfg["dx"], seed=31 + rnd)
        rp, col, rev = _context_family(cfg, u)
        x = torch.from_numpy(_positions(cfg, u)).cuda()
        delta = cfg["horizon_factor"] * cfg["dx"]
        grp, gcol, grev = family_noalloc(x, delta, max_family=192)
        torch.cuda.synchronize()
        assert np.array_equal(grp.cpu().numpy(), rp)
        assert np.array_equal(gcol.cpu().numpy(), col)
        assert np.array_equal(grev.cpu().numpy(), rev)


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
    assert rc == -1 and nb.value == -1
