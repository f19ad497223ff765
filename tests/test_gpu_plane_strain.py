"""The plane-strain variant on the GPU against the oracle (reading R35):
the family with its periodic images bit-exact (FP64 path), every state
field within 1e-10 (FP64) and displacement within 1e-3 relative L2 (mixed)
for the three force states, on the substrate, the critical time step, the
y-invariance of a y-invariant start at a larger size, and the rejected
configurations."""
import numpy as np
import pytest

import ppm_inputs as pi
from gpu_helpers import gpu_run, oracle_run, rel_l2, state_errors

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10
MIXED_TOL = 1e-3


def slab(**kw):
    base = dict(nx=9, ny=13, nz=8, plane_strain=1, suction=20e3, pc0=5e3, rebuild_every=1)
    base.update(kw)
    return pi.small_config(**base)


def in_plane_velocity(cfg, seed, std=1e-3):
    v = pi.initial_velocity(dict(cfg, ny=1), std=std, seed=seed)
    v[1] = 0.0
    return v.reshape(3, cfg["nz"], 1, cfg["nx"]).repeat(cfg["ny"], axis=2).reshape(3, -1)


def test_the_periodic_family_is_bit_exact_after_displaced_rebuilds():
    cfg = slab()
    v0 = in_plane_velocity(cfg, seed=31, std=0.3)        # large: members change
    run = oracle_run(cfg, 3, v0)
    sim = gpu_run(cfg, 3, "fp64", v0=v0)
    rp, col, rev = run.family()
    assert np.array_equal(sim.read("row_ptr"), rp)
    assert np.array_equal(sim.read("col"), col) and np.array_equal(sim.read("rev"), rev)
    assert np.diff(rp).max() == 122


@pytest.mark.parametrize("model", [0, 1, 2])
def test_plane_strain_matches_oracle(model):
    cfg = slab(model=model)
    v0 = in_plane_velocity(cfg, seed=32)
    run = oracle_run(cfg, 12, v0)
    assert run.counters()["plastic"] > 0
    sim = gpu_run(cfg, 12, "fp64", v0=v0)
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err
    st, ce = sim.status(), run.energies()
    scale = max(abs(ce["W_int"]), abs(ce["W_ext"]), ce["W_kin"])
    for key in ("W_int", "W_ext", "W_kin"):
        assert abs(st[key] - ce[key]) <= FP64_TOL * scale, key
    sim = gpu_run(cfg, 12, "mixed", v0=v0)
    assert rel_l2(sim.read("u"), run.u) <= MIXED_TOL


def test_a_plane_strain_slab_on_the_substrate_matches_oracle():
    cfg = slab(model=2, contact=1, friction=0.25, rebuild_every=2)
    v0 = in_plane_velocity(cfg, seed=33)
    run = oracle_run(cfg, 12, v0)
    sim = gpu_run(cfg, 12, "fp64", v0=v0)
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_plane_strain_critical_time_step_matches_oracle(precision, tol):
    cfg = slab(rebuild_every=2)
    v0 = in_plane_velocity(cfg, seed=34, std=1e-2)
    run = oracle_run(cfg, 6, v0)
    sim = gpu_run(cfg, 6, precision, v0=v0)
    got, want = sim.critical_time_step(), run.critical_time_step()
    assert np.isfinite(want) and abs(got - want) <= tol * want, (got, want)


def test_a_y_invariant_start_stays_y_invariant_in_the_mixed_path():
    # 40 x 13 x 40 (the 2-D collapse of aspect 1): the layers' families list
    # the same members in different orders, so the layers agree to rounding
    cfg = slab(nx=40, nz=40, rebuild_every=50, model=2, contact=1)
    v0 = in_plane_velocity(cfg, seed=35)
    sim = gpu_run(cfg, 500, "mixed", v0=v0)
    u = sim.read("u").reshape(3, cfg["nz"], cfg["ny"], cfg["nx"]).astype(np.float64)
    assert np.all(u[1] == 0.0)
    spread = np.abs(u - u[:, :, :1, :]).max()
    assert spread <= 1e-4 * np.abs(u).max(), spread


def test_plane_strain_rejections():
    from paper_2203_05562_gb300 import Simulation
    with pytest.raises(RuntimeError):
        Simulation(slab(ny=12), precision="fp64")              # 12 dx < 4 delta
    with pytest.raises(RuntimeError):
        Simulation(slab(), columns=[dict(nx=9, ny=13, nz=8, suction=0.0, M=1.2)] * 2,
                   precision="mixed")
    sim = Simulation(slab(model=1), precision="fp64")
    with pytest.raises(RuntimeError):
        sim.adjoint_forward(2, 1)
