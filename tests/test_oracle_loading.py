"""Pins of the uniaxial-compression boundary condition (the loading of
Sec. 4.1) in the oracle: the loaded end regions (a horizon thick) follow the
prescribed motion exactly, and with the reaction's work counted as external
work the energy balance of Eq. 69 closes for the energy-conserving force
states."""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi

RATE = 0.05     # m/s


def loaded_column(model, nx=12, ny=4, nz=4):
    # the elastic skeleton of Sec. 4.1, no gravity, no suction
    return pi.small_config(nx, ny, nz, suction=0.0, model=model, bc=1, load_rate=RATE,
                           gravity=(0.0, 0.0, 0.0), elastic=1, init_stress=1, rebuild_every=0)


def test_loaded_faces_follow_the_prescribed_motion():
    cfg = loaded_column(2)
    n = pi.num_points(cfg)
    run = oracle.Run(cfg, pi.initial_velocity(cfg, std=1e-4, seed=3))
    steps = 120
    run.step(steps)
    ix = np.arange(n) % cfg["nx"]
    dt = oracle.time_step(cfg)
    nl = int(cfg["horizon_factor"])          # the loaded regions: a horizon thick
    held, driven = ix < nl, ix >= cfg["nx"] - nl
    assert nl == 3
    assert np.all(run.u[0, held] == 0.0) and np.all(run.v[0, held] == 0.0)
    assert np.all(run.v[0, driven] == -RATE)
    assert np.allclose(run.u[0, driven], -RATE * dt * steps, rtol=1e-12, atol=0)
    # the other components and the points between the regions move freely
    assert np.abs(run.u[1:, driven]).max() > 0
    free = ~held & ~driven
    assert np.abs(run.u[0, free]).max() > 0 and np.abs(run.v[0, free] + RATE).max() > 0


@pytest.mark.parametrize("model", [1, 2])
def test_energy_balance_closes_with_the_reaction_work(model):
    cfg = loaded_column(model)
    run = oracle.Run(cfg, np.zeros((3, pi.num_points(cfg))))
    run.step(300)
    e = run.energies()
    # the driven face does all the external work (no gravity)
    assert e["W_ext"] > 0 and e["W_int"] > 0
    bal = abs(e["W_int"] + e["W_kin"] - e["W_ext"] - e["W_kin0"])
    assert bal <= 1e-5 * max(abs(e["W_int"]), abs(e["W_ext"]), abs(e["W_kin"]))


def test_the_printed_eq51_force_state_runs_away_under_compression():
    # Eq. 51 as printed is not power-conjugate (reading R25): under the slow
    # compression the kinetic energy grows without bound while the
    # bookkeeping (boundary work, stored energy) still balances
    cfg = loaded_column(0)
    run = oracle.Run(cfg, np.zeros((3, pi.num_points(cfg))))
    run.step(300)
    e = run.energies()
    assert e["W_kin"] > 1e6 * abs(e["W_ext"])
    bal = abs(e["W_int"] + e["W_kin"] - e["W_ext"] - e["W_kin0"])
    assert bal <= 1e-9 * e["W_kin"]


def test_the_elastic_skeleton_never_yields():
    # the critical-state ellipse ends at p = 0, so bonds that the loading puts
    # in tension yield whatever pc0; the elastic skeleton of Sec. 4.1 does not
    counts = {}
    for elastic in (0, 1):
        cfg = dict(loaded_column(2), elastic=elastic, pc0=1e12)
        run = oracle.Run(cfg, np.zeros((3, pi.num_points(cfg))))
        run.step(200)
        counts[elastic] = run.counters()["plastic"]
    assert counts[0] > 0 and counts[1] == 0


def test_the_energy_check_as_a_hard_stop():
    # halt_on_unstable: the run stops at the first step whose Eq. 69 balance
    # fails, and later steps change nothing (the printed Eq. 51 force state
    # under the compression fails it within a few hundred steps)
    cfg = dict(loaded_column(0), halt_on_unstable=1)
    n = pi.num_points(cfg)
    run = oracle.Run(cfg, np.zeros((3, n)))
    run.step(300)
    h = run.counters()["halted_step"]
    assert 0 < h < 300
    frozen = run.u.copy(), run.v.copy(), run.sig.copy()
    run.step(20)
    assert all(np.array_equal(a, b) for a, b in zip(frozen, (run.u, run.v, run.sig)))
    # the same run without the stop, one step at a time: the balance first fails at h
    free = oracle.Run(dict(cfg, halt_on_unstable=0), np.zeros((3, n)))
    first = None
    for step in range(1, h + 1):
        free.step(1)
        e = free.energies()
        bal = abs(e["W_int"] + e["W_kin"] - e["W_ext"] - e["W_kin0"])
        if first is None and bal > 1e-2 * max(e["W_kin"], abs(e["W_int"]), abs(e["W_ext"]), e["W_kin0"]):
            first = step
    assert first == h
    assert np.array_equal(free.u, frozen[0])
