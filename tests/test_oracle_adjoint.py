"""The oracle's reverse (adjoint) sweep against central finite differences
of its own forward run, h = 1e-6 relative, on columns where the gradient
is fixed by the forward model alone."""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi

NAMES = ["M", "eta", "suction", "pc0"]


def fd_gradient(cfg, v0, steps, rel=1e-6):
    g = np.zeros(4)
    for k, name in enumerate(NAMES):
        h = rel * cfg[name]
        cp = dict(cfg, **{name: cfg[name] + h})
        cm = dict(cfg, **{name: cfg[name] - h})
        g[k] = (oracle.objective(cp, v0, steps) - oracle.objective(cm, v0, steps)) / (2 * h)
    return g


@pytest.mark.parametrize("model", [0, 1])
def test_adjoint_matches_finite_differences_on_a_plastic_column(model):
    # suction 50 kPa: S_r s exceeds pc0, every bond yields from the first step
    cfg = pi.small_config(5, 5, 7, suction=50e3, rebuild_every=3, model=model)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=4)
    J, g = oracle.objective_gradient(cfg, v0, 6)
    assert J == pytest.approx(oracle.objective(cfg, v0, 6), rel=1e-14)
    fd = fd_gradient(cfg, v0, 6)
    assert np.all(np.abs(fd) > 0)
    assert np.allclose(g, fd, rtol=1e-4, atol=0), (g, fd)


def test_adjoint_of_an_elastic_column_has_no_plastic_parameter_gradient():
    # the K0 state lies inside the yield surface: only the suction acts
    cfg = pi.small_config(5, 5, 7, suction=10e3, rebuild_every=0)
    v0 = pi.initial_velocity(cfg, std=1e-6, seed=2)
    J, g = oracle.objective_gradient(cfg, v0, 5)
    assert g[0] == 0.0 and g[1] == 0.0 and g[3] == 0.0
    fd = fd_gradient(cfg, v0, 5)
    assert g[2] == pytest.approx(fd[2], rel=1e-5)


def test_adjoint_with_literal_viscosity_and_locked_lateral_motion():
    cfg = pi.small_config(4, 5, 6, suction=40e3, visc_form=1, eta=3e12, lock_lateral=1,
                          rebuild_every=2)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=8)
    _, g = oracle.objective_gradient(cfg, v0, 5)
    fd = fd_gradient(cfg, v0, 5)
    assert np.allclose(g, fd, rtol=1e-4, atol=1e-12 * np.abs(fd).max()), (g, fd)


@pytest.mark.slow
def test_adjoint_matches_finite_differences_on_the_10x10x20_column():
    # the 10x10x20 column with a low preconsolidation so that it yields
    cfg = pi.config(0, pc0=5e3)
    v0 = pi.initial_velocity(cfg)
    J, g = oracle.objective_gradient(cfg, v0, 20)
    fd = fd_gradient(cfg, v0, 20)
    assert np.allclose(g, fd, rtol=1e-4, atol=0), (g, fd)
