"""The coupled mode on the GPU against the oracle (Eq. 15-16, 48-49;
reading R37): every state field and the volume ratio within 1e-10 (FP64)
and the displacement within 1e-3 relative L2 (mixed) for the three force
states, with the substrate and in plane strain; the volume ratio of a
uniform dilation in closed form; the rejected configurations."""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi
from gpu_helpers import gpu_run, oracle_run, rel_inf, rel_l2, state_errors

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10
MIXED_TOL = 1e-3


def coupled(**kw):
    base = dict(nx=5, ny=5, nz=7, coupled=1, suction=30e3, pc0=5e3, rebuild_every=2)
    base.update(kw)
    return pi.small_config(**base)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_coupled_mode_matches_oracle(model):
    cfg = coupled(model=model)
    v0 = pi.initial_velocity(cfg, std=1e-2, seed=41)
    run = oracle_run(cfg, 12, v0)
    assert np.abs(run.J - 1.0).max() > 1e-7 and run.counters()["plastic"] > 0
    sim = gpu_run(cfg, 12, "fp64", v0=v0)
    err = state_errors(sim, run)
    err["J"] = rel_inf(sim.read("J") - 1.0, run.J - 1.0)
    assert max(err.values()) <= FP64_TOL, err
    st, ce = sim.status(), run.energies()
    scale = max(abs(ce["W_int"]), abs(ce["W_ext"]), ce["W_kin"])
    for key in ("W_int", "W_ext", "W_kin"):
        assert abs(st[key] - ce[key]) <= FP64_TOL * scale, key
    sim = gpu_run(cfg, 12, "mixed", v0=v0)
    assert rel_l2(sim.read("u"), run.u) <= MIXED_TOL


def test_coupled_plane_strain_on_the_substrate_matches_oracle():
    cfg = coupled(nx=8, ny=13, nz=6, plane_strain=1, contact=1, friction=0.25, model=2)
    v = pi.initial_velocity(dict(cfg, ny=1), std=1e-2, seed=42)
    v[1] = 0.0
    v0 = v.reshape(3, cfg["nz"], 1, cfg["nx"]).repeat(cfg["ny"], axis=2).reshape(3, -1)
    run = oracle_run(cfg, 12, v0)
    sim = gpu_run(cfg, 12, "fp64", v0=v0)
    err = state_errors(sim, run)
    err["J"] = rel_inf(sim.read("J") - 1.0, run.J - 1.0)
    assert max(err.values()) <= FP64_TOL, err


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_the_volume_ratio_of_a_uniform_dilation(precision, tol):
    cfg = coupled(nx=5, ny=4, nz=6, suction=0.0, init_stress=1, elastic=1,
                  gravity=(0.0, 0.0, 0.0), contact=1, rebuild_every=0)
    edot = 2.0
    sim = gpu_run(cfg, 1, precision, v0=edot * oracle.reference_positions(cfg))
    want = np.exp(3.0 * sim.dt * edot / (1.0 + edot * sim.dt))
    assert np.allclose(sim.read("J"), want, rtol=tol, atol=0)


def test_coupled_mode_rejections():
    from paper_2203_05562_gb300 import Simulation
    with pytest.raises(RuntimeError):
        Simulation(coupled(), columns=[dict(nx=4, ny=4, nz=4, suction=1e3, M=1.2)] * 2,
                   precision="mixed")
    with pytest.raises(RuntimeError):
        Simulation(coupled(porosity=1.0), precision="fp64")
    sim = Simulation(coupled(model=1), precision="fp64")
    with pytest.raises(RuntimeError):
        sim.adjoint_forward(2, 1)
