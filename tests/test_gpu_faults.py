"""Failure detection through the status word, with faults injected in the
inputs only (no device fault is ever provoked): a non-finite velocity, a
return solve allowed a single Newton step, two coincident points, and a
family capacity smaller than the horizon holds.  Each is reported (or, for
the coincident points, harmless) and the run carries on; where the oracle
defines the result, the GPU matches it."""
import numpy as np
import pytest

import ppm_inputs as pi
from gpu_helpers import gpu_run, oracle_run, state_errors

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_a_non_finite_velocity_is_reported(precision):
    cfg = pi.small_config(6, 6, 8, rebuild_every=1)
    v0 = pi.initial_velocity(cfg, std=1e-4, seed=2)
    v0[0, 100] = np.nan
    sim = gpu_run(cfg, 3, precision, v0=v0)
    st = sim.status()
    assert "nonfinite" in st["flags"]
    # the run carries on (the non-finite values spread a horizon per step and
    # points whose position is not finite drop out of the family search) and
    # the family arrays stay well formed
    sim.step(2)
    rp = sim.read("row_ptr")
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == sim.num_bonds() < 19464
    col = sim.read("col")
    assert col.size == 0 or (col.min() >= 0 and col.max() < rp.size - 1)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_a_single_newton_step_is_reported_as_not_converged(precision):
    cfg = pi.small_config(5, 5, 7, suction=50e3, newton_max_iter=1, rebuild_every=2)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=3)
    sim = gpu_run(cfg, 4, precision, v0=v0)
    st = sim.status()
    assert st["nonconv"] > 0 and "nonconv" in st["flags"]
    if precision == "fp64":
        run = oracle_run(cfg, 4, v0)
        assert st["nonconv"] == run.counters()["nonconv"]
        err = state_errors(sim, run)
        assert max(err.values()) <= FP64_TOL, err


def test_coincident_points_stay_finite():
    # a zero-length bond is in the family, adds nothing to K and carries no
    # force state (nothing divides by a bond length on the step path)
    cfg = pi.small_config(5, 5, 6, rebuild_every=1)
    n = pi.num_points(cfg)
    u = np.zeros((3, n))
    u[0, 31] = -cfg["dx"]            # point 31 moved onto its x-neighbour 30
    for precision in ("fp64", "mixed"):
        sim = gpu_run(cfg, 3, precision, v0=pi.initial_velocity(cfg, std=1e-4, seed=4), u=u)
        rp, col = sim.read("row_ptr"), sim.read("col")
        assert 30 in col[rp[31]:rp[32]] and 31 in col[rp[30]:rp[31]]
        assert np.isfinite(sim.read("a")).all() and np.isfinite(sim.read("sigma")).all()
        assert "nonfinite" not in sim.status()["flags"]


def test_a_family_cap_below_the_horizon_is_reported():
    cfg = pi.small_config(6, 6, 6, max_family=40)
    sim = gpu_run(cfg, 2, "mixed", v0=pi.initial_velocity(cfg, std=1e-4, seed=5))
    st = sim.status()
    assert "row_full" in st["flags"]
    # interior points (122 neighbours) lost their rows; surface corners kept theirs
    rp = sim.read("row_ptr")
    lens = np.diff(rp)
    assert lens.max() <= 40 and (lens == 0).sum() > 0
