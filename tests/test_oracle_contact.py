"""Pins of the substrate contact (Sec. 4.2, Eq. 91-93; readings R31-R33) in
the oracle, on a one-layer slab resting on the rigid substrate: the
time-averaged penetration equals the static m g / k, a slab sliding without
friction keeps its speed, with friction it stops after v0^2 / (2 mu_f g)
and stays, and the energy balance of Eq. 69 closes with friction."""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi


def slab(friction):
    return pi.small_config(6, 6, 1, suction=0.0, elastic=1, init_stress=1, contact=1,
                           friction=friction, rebuild_every=0, model=1)


def spring(cfg):
    m = cfg["rho"] * cfg["dx"] ** 3
    k = cfg["contact_modulus"] * cfg["dx"] ** 2 / (cfg["contact_cutoff"] * cfg["dx"])
    return m, k


def test_the_time_averaged_penetration_is_the_static_one():
    cfg = slab(0.0)
    n = pi.num_points(cfg)
    m, k = spring(cfg)
    dt = oracle.time_step(cfg)
    periods = int(round(10 * 2 * np.pi / np.sqrt(k / m) / dt))
    run = oracle.Run(cfg, np.zeros((3, n)))
    mean = 0.0
    for _ in range(periods):
        run.step(1)
        mean += run.u[2].mean() / periods
    g = -cfg["gravity"][2]
    assert mean == pytest.approx(-m * g / k, rel=1e-2)
    assert run.u[2].max() <= 0.0          # it never leaves the substrate's reach upwards


def test_a_frictionless_slab_keeps_its_speed():
    cfg = slab(0.0)
    n = pi.num_points(cfg)
    v0 = np.zeros((3, n)); v0[0] = 0.1
    run = oracle.Run(cfg, v0)
    run.step(500)
    dt = oracle.time_step(cfg)
    assert np.allclose(run.v[0], 0.1, rtol=1e-12, atol=0)
    assert np.allclose(run.u[0], 0.1 * 500 * dt, rtol=1e-9, atol=0)


def test_friction_stops_a_sliding_slab_after_v0_squared_over_2_mu_g():
    mu, v = 0.25, 0.1
    cfg = slab(mu)
    n = pi.num_points(cfg)
    v0 = np.zeros((3, n)); v0[0] = v
    run = oracle.Run(cfg, v0)
    g = -cfg["gravity"][2]
    dt = oracle.time_step(cfg)
    run.step(int(1.3 * v / (mu * g) / dt))
    assert np.all(run.v[0] == 0.0)
    assert run.u[0].mean() == pytest.approx(v * v / (2 * mu * g), rel=1e-3)
    u = run.u.copy()
    run.step(200)
    assert np.array_equal(run.u[0], u[0])      # static friction holds it
    e = run.energies()
    bal = abs(e["W_int"] + e["W_kin"] - e["W_ext"] - e["W_kin0"])
    assert bal <= 1e-6 * max(abs(e["W_int"]), abs(e["W_ext"]), e["W_kin0"])


def test_the_adjoint_rejects_contact():
    cfg = slab(0.25)
    with pytest.raises(RuntimeError):
        oracle.objective_gradient(cfg, np.zeros((3, pi.num_points(cfg))), 2)


def test_two_points_closer_than_the_cutoff_repel_each_other():
    # Eq. 91 between points of the soil (reading R36): in a stress-free block
    # (no force state) with one point moved to 0.5 dx of its x-neighbour, the
    # internal force is the pair's repulsion and nothing else
    cfg = pi.small_config(4, 4, 4, suction=0.0, elastic=1, init_stress=1, contact=1,
                          rebuild_every=0, model=1)
    n = pi.num_points(cfg)
    dx, dc = cfg["dx"], cfg["contact_cutoff"] * cfg["dx"]
    x = oracle.reference_positions(cfg)
    a, b = 1 + 4 + 16, 2 + 4 + 16                  # (1, 1, 1) and (2, 1, 1)
    x[0, a] += 0.5 * dx
    rp, col, rev = oracle.family(x, cfg["horizon_factor"] * dx)
    sig = np.zeros((6, n))
    f = oracle.internal_force(cfg, x, sig, rp, col, rev)
    F = cfg["contact_modulus"] * dx * dx * (dc - 0.5 * dx) / dc
    want = np.zeros((3, n))
    want[0, a], want[0, b] = -F, F
    assert np.allclose(f, want, rtol=0, atol=1e-12 * F)
    f0 = oracle.internal_force(dict(cfg, contact=0), x, sig, rp, col, rev)
    assert np.all(f0 == 0.0)


def test_a_plane_strain_slab_stops_after_the_same_distance():
    # friction with the periodic slab of reading R35: the motion stays in x
    mu, v = 0.5, 0.1
    cfg = pi.small_config(6, 13, 1, suction=0.0, elastic=1, init_stress=1, contact=1,
                          friction=mu, rebuild_every=0, model=1, plane_strain=1)
    n = pi.num_points(cfg)
    v0 = np.zeros((3, n)); v0[0] = v
    run = oracle.Run(cfg, v0)
    g = -cfg["gravity"][2]
    dt = oracle.time_step(cfg)
    run.step(int(1.3 * v / (mu * g) / dt))
    assert np.all(run.v[0] == 0.0) and np.all(run.v[1] == 0.0) and np.all(run.u[1] == 0.0)
    assert run.u[0].mean() == pytest.approx(v * v / (2 * mu * g), rel=1e-3)
