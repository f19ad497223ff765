"""Pins of the oracle's bond pass -> point state chain, the sign of the
suction term in the total stress, and the exact interior fraction of the
printed Eq. 51 force state.

Each test checks the oracle against something the mathematics fixes:
- an affine half-step velocity makes every active bond's velocity gradient
  the same matrix A (Eq. 19, 25), so every bond of a point takes the same
  constitutive update, and the point state after one step is one
  single-point update with L = A whatever the bond weights (Sec. 1:
  internal variables on points; the weighted mean must be normalised and
  epsilon_s must accumulate the mean, not the sum);
- an effective stress of -S_r s 1 makes the total stress of Eq. 32 zero, so
  no point, on a surface or inside, carries any force;
- on the interior of an undeformed cubic lattice the force of Eq. 49 with
  the own-bond state of Eq. 51 under a linear stress field is a fixed
  multiple of div(sigma), computed here by enumerating lattice offsets.
"""
import itertools

import numpy as np
import pytest

import oracle
import ppm_inputs as pi


def _affine_start(cfg, A, b, sig0, seed):
    """Deformed start y = X + u0 and the initial velocity that makes the
    half-step velocity of Eq. 60 equal A x_(n+1) + b at the positions of
    Eq. 61 (x_(n+1) = y + dt v_half): v_half = (I - dt A)^-1 (A y + b) and
    v0 = v_half - dt/2 a0, where a0 (the initial pass) does not depend on v0."""
    n = pi.num_points(cfg)
    u0 = pi.perturbation(cfg, 0.2 * cfg["dx"], seed=seed)
    y = oracle.reference_positions(cfg) + u0
    dt = oracle.time_step(cfg)
    probe = oracle.Run(cfg, np.zeros((3, n)), sig0=sig0, u0=u0)
    a0 = probe.a.copy()
    w = np.linalg.solve(np.eye(3) - dt * A, A @ y + b[:, None])
    return u0, w - 0.5 * dt * a0, dt


@pytest.mark.parametrize("plastic", [False, True])
def test_point_state_after_affine_step_is_one_material_update(plastic):
    # the substrate carries the column (no fixed base), so a general affine
    # velocity field is admissible at every point; without friction the
    # initial acceleration does not depend on the initial velocity
    cfg = pi.small_config(6, 5, 7, contact=1, friction=0.0, suction=20e3,
                          pc0=(35e3 if plastic else 200e3))
    n = pi.num_points(cfg)
    rng = np.random.default_rng(17 + plastic)
    sig0 = np.zeros((6, n))
    sig0[:3] = -30e3 + rng.uniform(-2e3, 2e3, size=(3, n))
    sig0[3:] = rng.uniform(-1e3, 1e3, size=(3, n)) * (8.0 if plastic else 1.0)
    A = rng.normal(size=(3, 3)) * 2.0
    b = rng.normal(size=3) * 0.05
    u0, v0, dt = _affine_start(cfg, A, b, sig0, seed=5)
    run = oracle.Run(cfg, v0, sig0=sig0, u0=u0)
    pc_start = run.pc.copy()
    run.step(1)
    n_plastic = 0
    for i in range(n):
        want, pc_want, des_want, flags = oracle.material_update(cfg, sig0[:, i], pc_start[i], A, dt)
        n_plastic += flags & 1
        scale = np.abs(sig0[:, i]).max()
        tol = 1e-9 if plastic else 1e-11
        assert np.abs(run.sig[:, i] - want).max() <= tol * scale, i
        assert abs(run.pc[i] - pc_want) <= tol * abs(pc_start[i]), i
        assert run.eps_s[i] == pytest.approx(des_want, rel=1e-8 if plastic else 1e-10, abs=1e-18), i
    assert (n_plastic > n // 4) if plastic else (n_plastic == 0)
    assert run.counters()["plastic"] > 0 if plastic else run.counters()["plastic"] == 0


@pytest.mark.parametrize("model", [0, 1, 2])
def test_effective_stress_of_minus_suction_carries_no_force(model):
    # Eq. 32: total stress = sigma_bar - S_r p_w 1 = sigma_bar + S_r s 1 (p_w = -s)
    cfg = pi.small_config(6, 5, 7, model=model, suction=30e3, gravity=(0.0, 0.0, 0.0),
                          rebuild_every=0)
    n = pi.num_points(cfg)
    Srs = oracle.saturation(cfg["suction"], cfg["vg_alpha"], cfg["vg_n"]) * cfg["suction"]
    sig0 = np.zeros((6, n))
    sig0[:3] = -Srs
    u0 = pi.perturbation(cfg, 0.2 * cfg["dx"], seed=3)
    run = oracle.Run(cfg, np.zeros((3, n)), sig0=sig0, u0=u0)
    scale = Srs * cfg["dx"] ** 2
    assert np.abs(run.fint).max() <= 1e-12 * scale
    assert np.abs(run.a).max() == 0.0
    # the opposite sign would leave a total stress of -2 S_r s 1, which the
    # surfaces do not balance: forces of the order of S_r s dx^2
    x = run.positions()
    rp, col, rev = oracle.family(x, cfg["horizon_factor"] * cfg["dx"])
    wrong = oracle.internal_force(cfg, x, 3.0 * sig0, rp, col, rev)
    assert np.abs(wrong).max() > 0.1 * scale


def _lattice_ball(r2):
    r = int(np.floor(np.sqrt(r2)))
    return [o for o in itertools.product(range(-r, r + 1), repeat=3)
            if o != (0, 0, 0) and o[0] ** 2 + o[1] ** 2 + o[2] ** 2 <= r2]


def eq51_interior_fraction(r2, comp=2):
    """Interior force of Eq. 49 with the force state of Eq. 51 under
    sigma = c x_comp e_comp (x) e_comp, over V c, on the undeformed lattice
    with |o|^2 <= r2 (omega = 1, uniform volumes).

    T_(ij) = varpi_(ij) sigma_i K_(ij)^-1 zeta_(ij), T_(ji) = varpi_(ji)
    sigma_j K_(ji)^-1 zeta_(ji), zeta_(ji) = -zeta_(ij); by point reflection
    K_(ji) = K_(ij) and varpi_(ji) = varpi_(ij), so the force on i is
    V^2 sum_o varpi(o) (sigma_i + sigma_(i+o)) K(o)^-1 zeta(o).  The sigma_i
    terms cancel in pairs (odd in o); sigma_(i+o) - sigma_i = c o_comp dx.
    With K(o) = V dx^2 Ks(o), Ks(o) = sum over the sub-horizon S(o) = {o' in
    H : |o' - o|^2 <= r2} of o' o'^T, and varpi(o) = |S(o)| / |H| (Eq. 55),
    f_comp / (V c) = sum_o varpi(o) o_comp (Ks(o)^-1 o)_comp."""
    H = _lattice_ball(r2)
    Ha = np.array(H, dtype=np.float64)
    total = 0.0
    for o in Ha:
        d = Ha - o
        S = Ha[(d * d).sum(axis=1) <= r2 + 1e-9]
        Ks = S.T @ S
        varpi = len(S) / len(Ha)
        total += varpi * o[comp] * np.linalg.solve(Ks, o)[comp]
    return total


def test_lattice_fraction_enumeration_is_one_for_the_full_horizon():
    # with S(o) = H the same sum is sum_o o_z^2 / sum_o o_z^2 = 1 (standard
    # correspondence): the enumeration above reduces to the textbook identity
    H = np.array(_lattice_ball(9), dtype=np.float64)
    Ks = H.T @ H
    assert sum(o[2] * np.linalg.solve(Ks, o)[2] for o in H) == pytest.approx(1.0, rel=1e-14)


@pytest.mark.parametrize("comp", [0, 2])
def test_eq51_interior_force_is_the_exact_lattice_fraction(comp):
    cfg = pi.small_config(16, 16, 16, model=0)
    X = oracle.reference_positions(cfg)
    rp, col, rev = oracle.family(X, cfg["horizon_factor"] * cfg["dx"])
    c = 1e6
    sig = np.zeros((6, X.shape[1]))
    sig[comp] = c * X[comp]
    # no suction term: the total stress is then the effective one
    cfg0 = dict(cfg, suction=0.0)
    f = oracle.internal_force(cfg0, X, sig, rp, col, rev)
    ijk = np.round(X / cfg["dx"]).astype(int)
    inner = np.all((ijk >= 7) & (ijk <= 8), axis=0)
    ratio = f[comp, inner] / cfg["dx"] ** 3 / c
    # delta^2 = 9.09 dx^2: the integer lattice distances nearest to it are 9
    # and 10, so the offset ball and every sub-horizon are those of r2 = 9
    want = eq51_interior_fraction(9, comp)
    assert 0.80 < want < 0.86
    assert np.abs(ratio - want).max() <= 1e-9 * want
    # other components of the force vanish on the interior
    others = [q for q in range(3) if q != comp]
    assert np.abs(f[others][:, inner]).max() <= 1e-9 * abs(want) * c * cfg["dx"] ** 3
