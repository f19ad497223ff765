"""Pins of the coupled mode in the oracle (Eq. 15-16, 48-49; reading R37):
the degree of saturation of Eq. 15 reduces to the van Genuchten curve when
it does not depend on the void ratio and behaves as a retention curve
must; the solid mass is conserved exactly; the volume ratio follows a
uniform dilation in closed form and a rigid motion leaves it at one; a
compacting column gains saturation where it compacts."""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi


def coupled(**kw):
    base = dict(coupled=1, rebuild_every=1)
    base.update(kw)
    return pi.small_config(**base)


def test_eq15_reduces_to_van_genuchten_without_the_void_ratio():
    cfg = coupled(wr_a2=0.0)
    for s in (1e3, 2e4, 5e4):
        want = oracle.saturation(s, cfg["wr_a1"], cfg["wr_n"])
        assert oracle.coupled_saturation(cfg, 1.0, s) == pytest.approx(want, rel=1e-14)


def test_eq15_is_a_retention_curve():
    cfg = coupled()
    assert oracle.coupled_saturation(cfg, 1.0, 0.0) == 1.0
    s = np.linspace(1e3, 1e5, 50)
    sr = np.array([oracle.coupled_saturation(cfg, 1.0, v) for v in s])
    assert np.all(np.diff(sr) < 0) and np.all((sr > 0) & (sr < 1))
    # denser soil (smaller J, smaller void ratio) holds more water; no voids: saturated
    J = np.linspace(0.85, 1.15, 31)
    srj = np.array([oracle.coupled_saturation(cfg, v, 25e3) for v in J])
    assert np.all(np.diff(srj) < 0)
    assert oracle.coupled_saturation(cfg, 1.0 - cfg["porosity"], 25e3) == 1.0
    # Eq. 16
    assert oracle.coupled_porosity(cfg, 1.0) == pytest.approx(cfg["porosity"], rel=1e-15)
    assert oracle.coupled_porosity(cfg, 1.0 - cfg["porosity"]) == pytest.approx(0.0, abs=1e-15)


def test_the_solid_mass_is_conserved_exactly():
    cfg = coupled(nx=5, ny=5, nz=7, suction=30e3, pc0=5e3)
    run = oracle.Run(cfg, pi.initial_velocity(cfg, std=1e-2, seed=3))
    run.step(40)
    assert np.abs(run.J - 1.0).max() > 1e-6           # the volumes did change
    phi = np.array([oracle.coupled_porosity(cfg, j) for j in run.J])
    V0 = cfg["dx"] ** 3
    solid = cfg["rho_s"] * (1.0 - phi) * run.J * V0
    assert np.allclose(solid, cfg["rho_s"] * (1.0 - cfg["porosity"]) * V0, rtol=1e-14, atol=0)


def test_the_volume_ratio_of_a_uniform_dilation():
    # zero stress, no gravity: v = edot X gives L = edot / (1 + edot dt) I on
    # every bond in the configuration after the predictor, so after one
    # step J = exp(3 dt edot / (1 + edot dt)) at every point
    cfg = coupled(nx=5, ny=4, nz=6, suction=0.0, init_stress=1, elastic=1,
                  gravity=(0.0, 0.0, 0.0), contact=1, rebuild_every=0)
    X = oracle.reference_positions(cfg)
    edot = 2.0
    run = oracle.Run(cfg, edot * X)
    assert np.all(run.a == 0.0)
    dt = oracle.time_step(cfg)
    run.step(1)
    want = np.exp(3.0 * dt * edot / (1.0 + edot * dt))
    assert np.allclose(run.J, want, rtol=1e-12, atol=0)


def test_a_rigid_translation_keeps_the_volume():
    cfg = coupled(nx=4, ny=4, nz=5, suction=0.0, init_stress=1, elastic=1,
                  gravity=(0.0, 0.0, 0.0), contact=1, rebuild_every=1)
    n = pi.num_points(cfg)
    v0 = np.zeros((3, n)); v0[0] = 0.3; v0[2] = 0.1
    run = oracle.Run(cfg, v0)
    run.step(20)
    assert np.all(run.J == 1.0)
    assert np.allclose(run.v[0], 0.3, rtol=1e-13) and np.allclose(run.v[2], 0.1, rtol=1e-13)


def test_a_compacting_column_gains_saturation_where_it_compacts():
    cfg = coupled(nx=5, ny=5, nz=8, suction=30e3, pc0=3e3, rebuild_every=2)
    run = oracle.Run(cfg, np.zeros((3, pi.num_points(cfg))))
    run.step(60)
    J = run.J
    assert J.min() < 1.0 - 1e-5
    s_r = np.array([oracle.coupled_saturation(cfg, j, cfg["suction"]) for j in J])
    s_r0 = oracle.coupled_saturation(cfg, 1.0, cfg["suction"])
    moved = np.abs(J - 1.0) > 1e-9
    assert np.all(np.sign(s_r - s_r0)[moved] == -np.sign(J - 1.0)[moved])
    assert np.isfinite(run.u).all()


def test_the_adjoint_rejects_the_coupled_mode():
    cfg = coupled(nx=4, ny=4, nz=4)
    with pytest.raises(RuntimeError):
        oracle.objective_gradient(cfg, np.zeros((3, pi.num_points(cfg))), 2)
