"""The energy terms of Eqs. 66-69 on the GPU.

The residual of Eq. 69 equals (dt^2 / 8) (sum m |a_n|^2 - sum m |a_0|^2)
identically for the explicit scheme (the derivation is in the oracle's pin
of the same identity).  At the full size of the column-collapse workload,
where the oracle cannot follow step by step, this is a property that the
GPU's energy accounting must satisfy whatever the state; at small sizes
the tolerance of the check (reading R34) decides the same flags and the same
hard stop as the oracle."""
import numpy as np
import pytest

import ppm_inputs as pi
from gpu_helpers import gpu_run, oracle_run

pytestmark = pytest.mark.gpu


def identity_terms(sim, cfg, a0_sq):
    st = sim.status()
    m = cfg["rho"] * cfg["dx"] ** 3
    a = sim.read("a").astype(np.float64)
    resid = st["W_int"] + st["W_kin"] - st["W_ext"] - st["W_kin0"]
    pred = sim.dt ** 2 / 8.0 * (m * float((a * a).sum()) - a0_sq)
    scale = max(st["W_kin"], abs(st["W_int"]), abs(st["W_ext"]), st["W_kin0"])
    return resid, pred, scale


@pytest.mark.parametrize("name,precision,tol", [
    ("column_10x10x20_fp64", "fp64", 1e-9),
    ("collapse_40x40x80_mixed", "mixed", 2e-2),
])
def test_the_eq69_residual_identity_at_full_size(name, precision, tol):
    from paper_2203_05562_gb300 import Simulation
    cfg = pi.config(name)
    sim = Simulation(cfg, precision=precision, bond_tile=0)
    sim.write("v", pi.initial_velocity(cfg))
    sim.step(0)                                   # the initial pass: a_0 and W_kin0
    m = cfg["rho"] * cfg["dx"] ** 3
    a0 = sim.read("a").astype(np.float64)
    a0_sq = m * float((a0 * a0).sum())
    seen = 0.0
    for _ in range(8):
        sim.step(25)
        resid, pred, scale = identity_terms(sim, cfg, a0_sq)
        # FP32 state: the identity holds to the rounding of v and a, a small
        # fraction of the residual itself
        assert abs(resid - pred) <= tol * abs(pred) + 1e-12 * scale, (sim.status()["steps"], resid, pred)
        seen = max(seen, abs(pred) / scale)
    assert seen > 1e-5                           # the residual is not trivially zero


def test_the_check_tolerance_matches_oracle():
    # a column released from rest trips 1e-2 in its first steps, not 5e-2
    cfg = pi.small_config(6, 6, 10, suction=20e3, model=2, contact=1, rebuild_every=1)
    v0 = pi.initial_velocity(cfg, std=1e-4, seed=1)
    for tol in (0.0, 5e-2):
        c = dict(cfg, energy_tol=tol)
        run = oracle_run(c, 40, v0)
        sim = gpu_run(c, 40, "fp64", v0=v0)
        st = sim.status()
        assert ("unstable" in st["flags"]) == bool(run.counters()["unstable"])
        assert bool(run.counters()["unstable"]) == (tol == 0.0)
        assert st["unstable_step"] == run.counters()["unstable_step"]


@pytest.mark.parametrize("tol", [5e-2, 1e-1])
def test_a_looser_tolerance_stops_eq51_at_the_oracle_step(tol):
    cfg = pi.small_config(12, 4, 4, suction=0.0, model=0, bc=1, load_rate=0.05,
                          gravity=(0.0, 0.0, 0.0), elastic=1, init_stress=1, rebuild_every=0,
                          halt_on_unstable=1, energy_tol=tol)
    v0 = np.zeros((3, pi.num_points(cfg)))
    run = oracle_run(cfg, 400, v0)
    h = run.counters()["halted_step"]
    assert 0 < h < 400
    sim = gpu_run(cfg, 400, "fp64", v0=v0)
    assert sim.status()["halted_step"] == h


def test_a_negative_tolerance_is_rejected():
    from paper_2203_05562_gb300 import Simulation
    cfg = pi.small_config(4, 4, 4, energy_tol=-1e-2)
    with pytest.raises(RuntimeError):
        Simulation(cfg, precision="fp64")
