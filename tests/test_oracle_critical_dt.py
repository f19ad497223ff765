"""Pins of the critical time step of Eq. 65 (reading R30: the micro-modulus
divided by the bond length, C = 18 K / (pi delta^4)) in the oracle: its
scaling with the stiffness, the density and the lattice spacing, and that it
is a stable step for the explicit scheme of Alg. 2 while three times it is
not (the paper calls it conservative for state-based models)."""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi


def column(**kw):
    cfg = pi.small_config(6, 6, 6, suction=0.0, elastic=1, init_stress=1, gravity=(0.0, 0.0, 0.0),
                          bc=1, load_rate=0.0, rebuild_every=0, model=2)
    cfg.update(kw)
    return cfg


def dt_c(cfg, u=None):
    n = pi.num_points(cfg)
    run = oracle.Run(cfg, np.zeros((3, n)))
    if u is not None:
        run.u[:] = u
    return run.critical_time_step()


def test_scales_with_density_stiffness_and_spacing():
    base = column()
    t0 = dt_c(base)
    assert t0 > 0 and np.isfinite(t0)
    assert dt_c(column(K=4 * base["K"])) == pytest.approx(t0 / 2, rel=1e-12)
    assert dt_c(column(rho=4 * base["rho"])) == pytest.approx(2 * t0, rel=1e-12)
    # same horizon in spacings: C ~ dx^-4, V ~ dx^3, 1/|zeta| ~ 1/dx
    assert dt_c(column(dx=2 * base["dx"])) == pytest.approx(2 * t0, rel=1e-12)


def test_the_shortest_bonds_set_the_step():
    # compressing the lattice shortens every bond, so the step shrinks
    cfg = column()
    X = oracle.reference_positions(cfg)
    assert dt_c(cfg, u=-0.05 * (X - X.mean(axis=1, keepdims=True))) < dt_c(cfg)


@pytest.mark.parametrize("factor,stable", [(1.0, True), (3.0, False)])
def test_is_a_stable_step_and_three_times_it_is_not(factor, stable):
    cfg = column()
    cfg["dt"] = factor * dt_c(cfg)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=5)
    run = oracle.Run(cfg, v0)
    run.step(600)
    vmax = float(np.abs(run.v).max())
    assert (vmax < 10 * np.abs(v0).max()) == stable, vmax
