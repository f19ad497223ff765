"""Pins of the energy bookkeeping of Eqs. 66-69 in the oracle.

With the explicit scheme of Alg. 2 (half-step velocity v_{n+1/2} = v_n +
dt a_n / 2, u_{n+1} = u_n + dt v_{n+1/2}, full-step v_{n+1} = v_{n+1/2} +
dt a_{n+1} / 2), the trapezoidal works of Eqs. 66-67 taken over the
increment dt (u'_n + dt u''_n / 2) and the kinetic energy of Eq. 68 give,
for ANY force law, one step at a time:

    dW_kin = (1/2) du . (F_n + F_{n+1}) + (dt^2 / 8) d(sum_i m |a_i|^2),

so the residual of Eq. 69 is, identically,

    W_int + W_kin - W_ext - W_kin0 = (dt^2 / 8) (sum m |a_n|^2 - sum m |a_0|^2).

Every force must be booked in W_int or W_ext for this to hold: the bond
forces, gravity, the reaction of a prescribed component (reading R20), the
substrate's normal and friction forces and the repulsion between soil points
closer than delta_c (Eq. 91-93).  A dropped term, a wrong
half or a force booked at the wrong velocity breaks it, which makes it an
exact check on all of them at once.  It also says what the check of Eq. 69
measures: the mass-weighted frequency content of the motion against dt, so
that a column released from rest (large high-frequency accelerations, tiny
energies) trips a tolerance of 1e-2 in its first steps while perfectly
stable -- hence the tolerance as a parameter (reading R34)."""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi

CASES = {
    # the column under gravity and suction, critical-state skeleton, family
    # rebuilt every step, for the three force states
    "column_model0": dict(nx=5, ny=5, nz=7, suction=20e3, model=0, rebuild_every=1),
    "column_model1": dict(nx=5, ny=5, nz=7, suction=20e3, model=1, rebuild_every=1),
    "column_model2": dict(nx=5, ny=5, nz=7, suction=20e3, model=2, rebuild_every=1),
    # uniaxial compression: the reaction of the held and driven planes
    "uniaxial": dict(nx=12, ny=4, nz=4, suction=0.0, model=2, bc=1, load_rate=0.05,
                     gravity=(0.0, 0.0, 0.0), elastic=1, init_stress=1, rebuild_every=0),
    # the column on the substrate: normal spring and Coulomb friction
    "contact": dict(nx=5, ny=5, nz=6, suction=20e3, model=2, contact=1, friction=0.25,
                    rebuild_every=2),
    # a slab sliding on the substrate until friction stops it
    "sliding": dict(nx=6, ny=6, nz=1, suction=0.0, elastic=1, init_stress=1, contact=1,
                    friction=0.25, rebuild_every=0, model=1),
    # two points of the column starting closer than delta_c (reading R36)
    "pair": dict(nx=5, ny=5, nz=6, suction=20e3, model=2, contact=1, friction=0.25,
                 rebuild_every=2),
}


def residual_and_identity(run, cfg, a0_sq):
    e = run.energies()
    m = cfg["rho"] * cfg["dx"] ** 3
    dt = oracle.time_step(cfg)
    resid = e["W_int"] + e["W_kin"] - e["W_ext"] - e["W_kin0"]
    pred = dt * dt / 8.0 * (m * float((run.a ** 2).sum()) - a0_sq)
    scale = max(e["W_kin"], abs(e["W_int"]), abs(e["W_ext"]), e["W_kin0"])
    return resid, pred, scale


@pytest.mark.parametrize("case", list(CASES))
def test_the_eq69_residual_is_dt2_over_8_times_the_change_of_sum_m_a2(case):
    cfg = pi.small_config(**CASES[case])
    n = pi.num_points(cfg)
    if case == "sliding":
        v0 = np.zeros((3, n)); v0[0] = 0.1; v0[1] = 0.03
    else:
        v0 = pi.initial_velocity(cfg, std=1e-3, seed=11)
    u0 = None
    if case == "pair":
        u0 = np.zeros((3, n))
        u0[0, 2 + 5 * 2 + 25 * 3] = 0.6 * cfg["dx"]    # (2, 2, 3) to 0.4 dx of (3, 2, 3)
    run = oracle.Run(cfg, v0, u0=u0)
    m = cfg["rho"] * cfg["dx"] ** 3
    a0_sq = m * float((run.a ** 2).sum())
    steps = 400 if case == "sliding" else 60
    nonzero = 0
    for _ in range(steps):
        run.step(1)
        resid, pred, scale = residual_and_identity(run, cfg, a0_sq)
        assert abs(resid - pred) <= 1e-10 * max(scale, abs(pred)), (run.steps_done, resid, pred)
        nonzero += abs(resid) > 1e-6 * scale
    if case == "pair":
        # the pair was pushed apart
        x = oracle.reference_positions(cfg) + run.u
        i, j = 2 + 5 * 2 + 25 * 3, 3 + 5 * 2 + 25 * 3
        assert np.linalg.norm(x[:, j] - x[:, i]) > 0.5 * cfg["dx"]
    # the identity is not met trivially (the sliding slab's accelerations are
    # small beside its kinetic energy; there the friction work, which is as
    # large as that energy, is what the identity checks)
    assert nonzero > 0 or case == "sliding"
    if case == "sliding":
        e = run.energies()
        # the constant deceleration mu_f g has taken about a fifth of it
        assert 0.15 * e["W_kin0"] < e["W_int"] < 0.3 * e["W_kin0"]


def test_a_column_released_from_rest_trips_the_default_tolerance_while_stable():
    # suction puts the column under a sudden isotropic load at t = 0: the
    # residual is a percent of the energies for a few steps and then decays,
    # the motion staying bounded
    cfg = pi.small_config(6, 6, 10, suction=20e3, model=2, contact=1, rebuild_every=1)
    n = pi.num_points(cfg)
    v0 = pi.initial_velocity(cfg, std=1e-4, seed=1)
    runs = {tol: oracle.Run(dict(cfg, energy_tol=tol), v0) for tol in (0.0, 5e-2)}
    ratio = []
    for _ in range(200):
        for r in runs.values():
            r.step(1)
        e = runs[0.0].energies()
        bal = abs(e["W_int"] + e["W_kin"] - e["W_ext"] - e["W_kin0"])
        ratio.append(bal / max(e["W_kin"], abs(e["W_int"]), abs(e["W_ext"]), e["W_kin0"]))
    assert max(ratio[:10]) > 1e-2 and max(ratio[100:]) < 2e-3
    assert runs[0.0].counters()["unstable"] == 1 and runs[5e-2].counters()["unstable"] == 0
    # the first failing step is recorded: one of the first few
    first = next(i + 1 for i, r in enumerate(ratio) if r > 1e-2)
    assert runs[0.0].counters()["unstable_step"] == first <= 10
    assert runs[5e-2].counters()["unstable_step"] == 0
    # the tolerance only changes the diagnosis
    assert np.array_equal(runs[0.0].u, runs[5e-2].u)
    assert np.abs(runs[0.0].v).max() < 0.05


def test_a_looser_tolerance_still_stops_the_printed_eq51_force_state():
    cfg = pi.small_config(12, 4, 4, suction=0.0, model=0, bc=1, load_rate=0.05,
                          gravity=(0.0, 0.0, 0.0), elastic=1, init_stress=1, rebuild_every=0,
                          halt_on_unstable=1)
    halted = {}
    for tol in (0.0, 5e-2, 1e-1):
        run = oracle.Run(dict(cfg, energy_tol=tol), np.zeros((3, pi.num_points(cfg))))
        run.step(400)
        halted[tol] = run.counters()["halted_step"]
    assert 0 < halted[0.0] <= halted[5e-2] <= halted[1e-1] < 400, halted


def test_a_negative_tolerance_is_rejected():
    cfg = pi.small_config(4, 4, 4, energy_tol=-1e-2)
    with pytest.raises(RuntimeError):
        oracle.Run(cfg, np.zeros((3, pi.num_points(cfg))))


@pytest.mark.parametrize("seed", range(16))
def test_the_identity_holds_for_random_combinations_of_the_options(seed):
    # force state, boundary condition, substrate and friction, plane strain,
    # suction, skeleton, initial stress, gravity and rebuild period drawn at
    # random (the coupled mode changes the masses, which the identity assumes
    # constant, and is left out)
    rng = np.random.default_rng(1000 + seed)
    plane = bool(rng.integers(2))
    bc = int(rng.integers(2))
    kw = dict(nx=int(rng.integers(4, 7)), ny=13 if plane else int(rng.integers(3, 6)),
              nz=int(rng.integers(4, 7)), plane_strain=int(plane), model=int(rng.integers(3)),
              bc=bc, load_rate=0.05 if bc else 0.0,
              contact=int(rng.integers(2)) if bc == 0 else 0,
              friction=float(rng.choice([0.0, 0.25, 0.5])),
              suction=float(rng.choice([0.0, 20e3])), elastic=int(rng.integers(2)),
              init_stress=int(rng.integers(2)), rebuild_every=int(rng.choice([0, 1, 3])),
              pc0=float(rng.choice([5e3, 20e3])),
              gravity=(0.0, 0.0, -9.81) if rng.integers(2) else (0.0, 0.0, 0.0))
    cfg = pi.small_config(**kw)
    n = pi.num_points(cfg)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=seed)
    if plane:
        v0 = v0.reshape(3, kw["nz"], kw["ny"], kw["nx"])[:, :, :1, :].repeat(kw["ny"], axis=2).reshape(3, n)
        v0[1] = 0.0
    run = oracle.Run(cfg, v0)
    m = cfg["rho"] * cfg["dx"] ** 3
    a0_sq = m * float((run.a ** 2).sum())
    for _ in range(25):
        run.step(1)
        resid, pred, scale = residual_and_identity(run, cfg, a0_sq)
        assert abs(resid - pred) <= 1e-10 * max(scale, abs(pred)), (kw, run.steps_done, resid, pred)
