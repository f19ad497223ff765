"""GPU adjoint (reverse sweep with checkpoints) against the oracle's
adjoint and against central finite differences of the FP64 oracle."""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi

pytestmark = pytest.mark.gpu
NAMES = ["M", "eta", "suction", "pc0"]


def gpu_gradient(cfg, v0, steps, every, precision):
    import torch
    from paper_2203_05562_gb300.adjoint import ColumnRun, top_surface_runout
    theta = torch.tensor([cfg[k] for k in NAMES], dtype=torch.float64, requires_grad=True)
    u = ColumnRun.apply(theta, cfg, v0, steps, every, precision)
    J = top_surface_runout(u, cfg)
    J.backward()
    return float(J.detach()), theta.grad.numpy().copy()


@pytest.mark.parametrize("model", [0, 1])
def test_fp64_adjoint_matches_oracle_adjoint(model):
    cfg = pi.small_config(5, 5, 7, suction=50e3, rebuild_every=3, model=model)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=4)
    Jo, go = oracle.objective_gradient(cfg, v0, 6)
    J, g = gpu_gradient(cfg, v0, 6, 2, "fp64")
    assert J == pytest.approx(Jo, rel=1e-10)
    assert np.allclose(g, go, rtol=1e-8, atol=0), (g, go)


def test_mixed_adjoint_matches_oracle_adjoint():
    cfg = pi.small_config(5, 5, 7, suction=50e3, rebuild_every=3)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=4)
    _, go = oracle.objective_gradient(cfg, v0, 6)
    _, g = gpu_gradient(cfg, v0, 6, 2, "mixed")
    assert np.allclose(g, go, rtol=1e-3, atol=0), (g, go)


def test_checkpoint_interval_does_not_change_the_gradient():
    cfg = pi.small_config(5, 6, 7, suction=40e3, rebuild_every=4)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=7)
    ref = gpu_gradient(cfg, v0, 9, 9, "mixed")[1]
    for every in (1, 4):
        assert np.array_equal(gpu_gradient(cfg, v0, 9, every, "mixed")[1], ref)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-4), ("mixed", 1e-3)])
def test_adjoint_matches_oracle_finite_differences_on_the_10x10x20_column(precision, tol):
    # the 10x10x20 column with a low preconsolidation so that it yields;
    # central differences h = 1e-6 relative of the FP64 oracle
    cfg = pi.config(0, pc0=5e3)
    v0 = pi.initial_velocity(cfg)
    steps = 20
    _, g = gpu_gradient(cfg, v0, steps, 5, precision)
    fd = np.zeros(4)
    for k, name in enumerate(NAMES):
        h = 1e-6 * cfg[name]
        fd[k] = (oracle.objective(dict(cfg, **{name: cfg[name] + h}), v0, steps) -
                 oracle.objective(dict(cfg, **{name: cfg[name] - h}), v0, steps)) / (2 * h)
    assert np.allclose(g, fd, rtol=tol, atol=0), (g, fd)


@pytest.mark.slow
def test_fp64_adjoint_over_200_steps_matches_oracle_finite_differences():
    # the length of the adjoint workload (200 steps, checkpoints every 20)
    # on the 10x10x20 column that yields (p_c0 = 5 kPa): the FP64 GPU
    # gradient against central differences (h = 1e-6 relative) of the FP64
    # oracle's objective, to 1e-4 relative per parameter
    cfg = pi.config(0, pc0=5e3)
    v0 = pi.initial_velocity(cfg)
    steps = 200
    _, g = gpu_gradient(cfg, v0, steps, 20, "fp64")
    fd = np.zeros(4)
    for k, name in enumerate(NAMES):
        h = 1e-6 * cfg[name]
        fd[k] = (oracle.objective(dict(cfg, **{name: cfg[name] + h}), v0, steps) -
                 oracle.objective(dict(cfg, **{name: cfg[name] - h}), v0, steps)) / (2 * h)
    assert np.all(fd != 0.0)
    assert np.allclose(g, fd, rtol=1e-4, atol=0), (g, fd)


def test_adjoint_leaves_the_final_state():
    from paper_2203_05562_gb300 import Simulation
    cfg = pi.small_config(5, 5, 6, suction=50e3)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=1)
    sim = Simulation(cfg, precision="mixed", use_graph=False)
    sim.write("v", v0)
    sim.adjoint_forward(5, 2)
    u, sig = sim.read("u"), sim.read("sigma")
    sim.adjoint_reverse(np.ones((3, sim.n)))
    assert np.array_equal(sim.read("u"), u) and np.array_equal(sim.read("sigma"), sig)
    assert sim.status()["steps"] == 5
