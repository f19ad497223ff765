"""Pins of the plane-strain variant in the oracle (reading R35).

The paper's experiments (Secs. 4.1 and 4.2) are two-dimensional.  Plane
strain in the x-z plane is taken as a slab periodic in y (period ny dx,
ny dx > 4 delta) whose y velocity is held at zero: a y-invariant start
stays y-invariant, which is the plane-strain solution of the same
nonlocal model.  Pinned here against what the mathematics fixes: the
family against an independent brute force with explicit periodic images,
the shape tensor of a full interior family against the lattice-ball sum,
the y-invariance of the motion, the elastic plane-strain coupling
sigma_yy = nu (sigma_xx + sigma_zz), and the energy identity of Eq. 69."""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi


def slab(**kw):
    base = dict(nx=8, ny=13, nz=8, plane_strain=1, rebuild_every=0)
    base.update(kw)
    return pi.small_config(**base)


def lattice(cfg):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    i = np.arange(nx * ny * nz)
    return np.stack([i % nx, i // nx % ny, i // (nx * ny)])


def test_the_family_is_the_periodic_brute_force():
    cfg = slab()
    run = oracle.Run(cfg, np.zeros((3, pi.num_points(cfg))))
    rp, col, rev = run.family()
    I = lattice(cfg).astype(np.int64)
    ny, hf = cfg["ny"], cfg["horizon_factor"]
    n = I.shape[1]
    for i in range(n):
        d = I - I[:, i:i + 1]
        dy = np.stack([d[1], d[1] - ny, d[1] + ny])
        dy = dy[np.argmin(np.abs(dy), axis=0), np.arange(n)]
        r2 = d[0] ** 2 + dy ** 2 + d[2] ** 2
        want = np.flatnonzero((r2 <= hf * hf) & (np.arange(n) != i))
        assert np.array_equal(col[rp[i]:rp[i + 1]], want), i
    # every row holds its reverse bond, and each y-layer has the same row lengths
    assert np.array_equal(col[rev], np.repeat(np.arange(n), np.diff(rp)))
    lens = np.diff(rp).reshape(cfg["nz"], ny, cfg["nx"])
    assert np.all(lens == lens[:, :1, :])
    assert lens.max() == 122                     # interior: the full lattice ball


def test_a_full_interior_family_has_the_lattice_ball_shape_tensor():
    cfg = slab(model=1)
    n = pi.num_points(cfg)
    run = oracle.Run(cfg, np.zeros((3, n)))
    rp, col, _ = run.family()
    x = oracle.reference_positions(cfg)
    Kb, _, cnt, act = oracle.bond_kinematics(cfg, x, np.zeros((3, n)), rp, col)
    hf, dx = cfg["horizon_factor"], cfg["dx"]
    r = np.arange(-3, 4)
    g = np.stack(np.meshgrid(r, r, r, indexing="ij")).reshape(3, -1)
    ball = g[:, ((g ** 2).sum(0) <= hf * hf) & ((g ** 2).sum(0) > 0)]
    G = ball @ ball.T                             # integer lattice sum: c I exactly
    assert np.array_equal(G, G[0, 0] * np.eye(3, dtype=G.dtype)) and G[0, 0] == 236
    K = dx ** 5 * G.astype(np.float64)
    I = lattice(cfg)
    # points a horizon away from the x and z faces, in every y-layer (the
    # first and last layers' families cross the periodic boundary)
    inner = np.flatnonzero((I[0] >= 3) & (I[0] < cfg["nx"] - 3) & (I[2] >= 3) & (I[2] < cfg["nz"] - 3))
    assert set(I[1, inner]) == set(range(cfg["ny"]))
    for i in inner:
        b = rp[i]
        assert cnt[b] == 122 and act[b]
        sym = Kb[b]                               # xx, yy, zz, yz, xz, xy
        assert np.allclose(sym[:3], K[0, 0], rtol=1e-12) and np.allclose(sym[3:], 0.0, atol=1e-12 * K[0, 0])


def y_layers(a, cfg):
    return np.asarray(a).reshape(a.shape[0], cfg["nz"], cfg["ny"], cfg["nx"])


def in_plane_velocity(cfg, seed):
    v = pi.initial_velocity(dict(cfg, ny=1), std=1e-3, seed=seed)      # one layer
    v[1] = 0.0
    v = v.reshape(3, cfg["nz"], 1, cfg["nx"]).repeat(cfg["ny"], axis=2)
    return v.reshape(3, -1)


@pytest.mark.parametrize("model", [0, 1, 2])
def test_a_y_invariant_start_stays_y_invariant(model):
    cfg = slab(model=model, suction=20e3, pc0=5e3, rebuild_every=5)
    run = oracle.Run(cfg, in_plane_velocity(cfg, seed=4))
    run.step(40)
    assert run.counters()["plastic"] > 0
    assert np.all(run.u[1] == 0.0) and np.all(run.v[1] == 0.0)
    for name in ("u", "v", "sig"):
        a = y_layers(getattr(run, name), cfg)
        scale = np.abs(a).max()
        assert np.abs(a - a[:, :, :1, :]).max() <= 1e-10 * scale, name
    sig = run.sig
    assert np.abs(sig[3]).max() <= 1e-10 * np.abs(sig).max()     # yz
    assert np.abs(sig[5]).max() <= 1e-10 * np.abs(sig).max()     # xy


def test_the_elastic_plane_strain_coupling():
    # D_yy = 0 on every bond: sigma_yy = lambda tr(eps), sigma_xx + sigma_zz =
    # 2 (lambda + mu) tr(eps), so sigma_yy = nu (sigma_xx + sigma_zz) with
    # nu = lambda / (2 (lambda + mu)) (rotations about y keep both sides)
    cfg = slab(elastic=1, init_stress=1, suction=0.0)
    run = oracle.Run(cfg, in_plane_velocity(cfg, seed=5))
    run.step(60)
    K, mu = cfg["K"], cfg["mu"]
    lam = K - 2.0 * mu / 3.0
    nu = lam / (2.0 * (lam + mu))
    s = run.sig
    assert np.abs(s[1]).max() > 0
    err = np.abs(s[1] - nu * (s[0] + s[2]))
    assert err.max() <= 1e-6 * np.abs(s).max()


def test_the_energy_identity_holds_in_plane_strain():
    cfg = slab(model=2, suction=20e3, rebuild_every=2)
    run = oracle.Run(cfg, in_plane_velocity(cfg, seed=6))
    m = cfg["rho"] * cfg["dx"] ** 3
    dt = oracle.time_step(cfg)
    a0 = m * float((run.a ** 2).sum())
    for _ in range(30):
        run.step(1)
        e = run.energies()
        resid = e["W_int"] + e["W_kin"] - e["W_ext"] - e["W_kin0"]
        pred = dt * dt / 8.0 * (m * float((run.a ** 2).sum()) - a0)
        scale = max(e["W_kin"], abs(e["W_int"]), abs(e["W_ext"]), e["W_kin0"])
        assert abs(resid - pred) <= 1e-10 * max(scale, abs(pred))


def test_too_thin_a_slab_and_the_adjoint_are_rejected():
    with pytest.raises(RuntimeError):
        oracle.Run(slab(ny=12), np.zeros((3, 8 * 12 * 8)))       # 12 dx < 4 delta
    cfg = slab()
    with pytest.raises(RuntimeError):
        oracle.objective_gradient(cfg, np.zeros((3, pi.num_points(cfg))), 2)
