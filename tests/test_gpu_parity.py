"""GPU library against the FP64 CPU oracle on identical seeded inputs.

Tolerances: family CSR and reverse index bit-exact; FP64 path <= 1e-10
relative (max-norm over a field, relative to the field's max) on every
state field; mixed path <= 1e-3 relative L2 on displacement.
"""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi
from gpu_helpers import gpu_run, oracle_run, rel_inf, rel_l2, state_errors

pytestmark = pytest.mark.gpu
FP64_TOL = 1e-10
MIXED_TOL = 1e-3


def _family_gpu(cfg, u, columns=None):
    from paper_2203_05562_gb300 import Simulation
    sim = Simulation(cfg, columns=columns, precision="fp64")
    sim.write("u", u)
    sim.build_families()
    return sim.read("row_ptr"), sim.read("col"), sim.read("rev")


@pytest.mark.parametrize("amp", [0.0, 0.3])
def test_family_bit_exact_fp64(amp):
    cfg = pi.small_config(9, 8, 11)
    u = pi.perturbation(cfg, amp * cfg["dx"], seed=5)
    rp, col, rev = _family_gpu(cfg, u)
    X = oracle.reference_positions(cfg) + u
    orp, ocol, orev = oracle.family(X, cfg["horizon_factor"] * cfg["dx"])
    assert np.array_equal(rp, orp)
    assert np.array_equal(col, ocol)
    assert np.array_equal(rev, orev)


def _pairs(rp, col):
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return set(zip(rows.tolist(), np.asarray(col).tolist()))


@pytest.mark.parametrize("amp", [0.0, 0.3])
def test_mixed_family_against_oracle_within_fp32_rounding_of_the_horizon(amp):
    # The mixed path tests membership (Eq. 1) in FP32 lattice units,
    # (I_j - I_i) + (u_j - u_i) / dx, against (delta / dx)^2 rounded to
    # FP32.  On the same positions (the FP32 displacement, widened) the
    # oracle decides in FP64.  The families must agree except for pairs
    # whose FP64 distance lies within the FP32 rounding of that test of
    # the horizon: each component carries at most about 3e-7 (its rounded
    # difference and offset), the squared sum a few ulps of 9; 2e-5 of
    # delta^2 / dx^2 bounds it.  Pairs planted at the horizon itself
    # exercise the bound; the reverse index must be valid throughout.
    from paper_2203_05562_gb300 import Simulation
    cfg = pi.small_config(9, 8, 11)
    dx, hf = cfg["dx"], cfg["horizon_factor"]
    u = pi.perturbation(cfg, amp * dx, seed=7)
    n = pi.num_points(cfg)
    ijk = np.stack([np.arange(n) % 9, (np.arange(n) // 9) % 8, np.arange(n) // 72])
    # plant pairs at |x_j - x_i| = delta along x (lattice offset 3) in a few rows
    for (iy, iz) in ((2, 3), (5, 6), (4, 8)):
        row = np.where((ijk[1] == iy) & (ijk[2] == iz))[0]
        u[:, row] = 0.0
        u[0, row[3:]] = (hf - 3.0) * dx           # points ix >= 3 shifted by delta - 3 dx
    u32 = u.astype(np.float32)
    sim = Simulation(cfg, precision="mixed")
    sim.write("u", u32.astype(np.float64))
    sim.build_families()
    rp, col, rev = sim.read("row_ptr"), sim.read("col"), sim.read("rev")
    sim.close()
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.array_equal(rev[rev], np.arange(len(col)))
    assert np.array_equal(col[rev], rows)
    X = oracle.reference_positions(cfg) + u32.astype(np.float64)
    orp, ocol, _ = oracle.family(X, hf * dx)
    diff = _pairs(rp, col) ^ _pairs(orp, ocol)
    r2 = np.array([((X[:, j] - X[:, i]) ** 2).sum() / dx ** 2 for (i, j) in diff])
    assert np.all(np.abs(r2 - hf * hf) <= 2e-5 * hf * hf), (len(diff), r2)
    assert len(diff) <= 2 * 3 * 6


def test_family_config0_counts():
    cfg = pi.config(0)
    rp, col, rev = _family_gpu(cfg, np.zeros((3, pi.num_points(cfg))))
    assert len(col) == 179768 and rp[-1] == 179768
    assert np.all(col[rev] == np.repeat(np.arange(len(rp) - 1), np.diff(rp)))


def test_family_ensemble_columns_never_bond():
    cols = [dict(nx=4, ny=5, nz=6, suction=5e3, M=1.1), dict(nx=3, ny=3, nz=9, suction=0.0, M=1.3),
            dict(nx=5, ny=4, nz=4, suction=40e3, M=1.0)]
    cfg = pi.small_config(1, 1, 1)
    n = sum(c["nx"] * c["ny"] * c["nz"] for c in cols)
    rp, col, rev = _family_gpu(cfg, np.zeros((3, n)), columns=cols)
    off = 0
    for c in cols:
        cc = dict(cfg, nx=c["nx"], ny=c["ny"], nz=c["nz"])
        m = pi.num_points(cc)
        orp, ocol, orev = oracle.family(oracle.reference_positions(cc), cfg["horizon_factor"] * cfg["dx"])
        assert np.array_equal(rp[off:off + m + 1] - rp[off], orp)
        assert np.array_equal(col[rp[off]:rp[off + m]] - off, ocol)
        assert np.array_equal(rev[rp[off]:rp[off + m]] - rp[off], orev)
        off += m


def test_fp64_config0_50_steps_matches_oracle():
    cfg = pi.config(0)
    v0 = pi.initial_velocity(cfg)
    run = oracle_run(cfg, 50, v0)
    sim = gpu_run(cfg, 50, "fp64", v0=v0)
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err
    st = sim.status()
    ce = run.energies()
    for key in ("W_int", "W_ext", "W_kin"):
        assert abs(st[key] - ce[key]) <= FP64_TOL * max(abs(ce[key]), ce["W_kin"]), key
    assert st["plastic"] == run.counters()["plastic"]


@pytest.mark.parametrize("model", [0, 1, 2])
def test_fp64_plastic_column_all_models(model):
    # suction 50 kPa: S_r s = 21.7 kPa exceeds pc0, every bond starts plastic
    cfg = pi.small_config(6, 5, 7, suction=50e3, model=model, rebuild_every=2)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=3)
    run = oracle_run(cfg, 8, v0)
    assert run.counters()["plastic"] > 0
    sim = gpu_run(cfg, 8, "fp64", v0=v0)
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err
    assert sim.status()["plastic"] == run.counters()["plastic"]


def test_fp64_switches_zero_stress_locked_no_rebuild():
    cfg = pi.small_config(5, 6, 8, init_stress=1, lock_lateral=1, rebuild_every=0,
                          visc_form=1, eta=5e12)
    v0 = pi.initial_velocity(cfg, std=1e-2, seed=9)
    run = oracle_run(cfg, 6, v0)
    sim = gpu_run(cfg, 6, "fp64", v0=v0)
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err


def test_fp64_ensemble_matches_per_column_oracle():
    cols = [dict(nx=4, ny=4, nz=6, suction=5e3, M=1.1), dict(nx=3, ny=5, nz=5, suction=45e3, M=1.35)]
    cfg = pi.small_config(1, 1, 1, rebuild_every=2)
    n = sum(c["nx"] * c["ny"] * c["nz"] for c in cols)
    v0 = np.random.default_rng(4).normal(0, 1e-4, size=(3, n))
    sim = gpu_run(cfg, 5, "fp64", v0=v0, columns=cols)
    u, sig = sim.read("u"), sim.read("sigma")
    off = 0
    for c in cols:
        cc = dict(cfg, **c)
        m = pi.num_points(cc)
        run = oracle_run(cc, 5, v0[:, off:off + m])
        assert rel_inf(u[:, off:off + m], run.u) <= FP64_TOL
        assert rel_inf(sig[:, off:off + m], run.sig) <= FP64_TOL
        off += m


def test_mixed_config0_50_steps_within_1e3():
    cfg = pi.config(0)
    v0 = pi.initial_velocity(cfg)
    run = oracle_run(cfg, 50, v0)
    sim = gpu_run(cfg, 50, "mixed", v0=v0)
    assert rel_l2(sim.read("u"), run.u) <= MIXED_TOL
    err = state_errors(sim, run, norm=rel_l2)
    assert err["sigma"] <= MIXED_TOL and err["v"] <= 1e-2, err


@pytest.mark.slow
def test_mixed_config1_first_50_steps_within_1e3():
    cfg = pi.config(1)
    v0 = pi.initial_velocity(cfg)
    run = oracle_run(cfg, 50, v0)
    sim = gpu_run(cfg, 50, "mixed", v0=v0)
    assert rel_l2(sim.read("u"), run.u) <= MIXED_TOL
    err = state_errors(sim, run, norm=rel_l2)
    assert err["sigma"] <= MIXED_TOL, err


def test_graph_replay_matches_direct_launches_bitwise():
    cfg = pi.small_config(7, 6, 9, suction=30e3, rebuild_every=3)
    v0 = pi.initial_velocity(cfg, std=1e-3)
    a = gpu_run(cfg, 7, "mixed", v0=v0, use_graph=True)
    b = gpu_run(cfg, 7, "mixed", v0=v0, use_graph=False)
    for f in ("u", "v", "a", "sigma", "pc"):
        assert np.array_equal(a.read(f), b.read(f)), f


def test_runs_are_deterministic():
    cfg = pi.config(0)
    v0 = pi.initial_velocity(cfg)
    a = gpu_run(cfg, 20, "mixed", v0=v0)
    b = gpu_run(cfg, 20, "mixed", v0=v0)
    for f in ("u", "v", "sigma", "pc", "tforce"):
        assert np.array_equal(a.read(f), b.read(f)), f


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 2, 2), (1, 1, 5), (3, 1, 4)])
def test_degenerate_columns(dims):
    cfg = pi.small_config(*dims, suction=20e3, model=0)
    v0 = pi.initial_velocity(cfg, std=1e-3)
    run = oracle_run(cfg, 4, v0)
    sim = gpu_run(cfg, 4, "fp64", v0=v0)
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err
    assert sim.status()["singular"] == run.counters()["singular"]


def test_mixed_plastic_column_fp32_returns_within_1e3():
    # every bond yields from the first step; most returns are solved in FP32
    cfg = pi.small_config(8, 8, 10, suction=50e3, rebuild_every=5)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=12)
    run = oracle_run(cfg, 20, v0)
    sim = gpu_run(cfg, 20, "mixed", v0=v0)
    err = state_errors(sim, run, norm=rel_l2)
    assert err["u"] <= MIXED_TOL and err["sigma"] <= MIXED_TOL and err["pc"] <= MIXED_TOL, err
    st = sim.status()
    assert st["plastic"] > 0 and st["returns_fp64"] < st["plastic"]


def test_mixed_near_apex_returns_use_fp64():
    # zero initial stress and no suction: every state sits at the apex
    cfg = pi.small_config(6, 6, 8, suction=0.0, init_stress=1, rebuild_every=0)
    v0 = pi.initial_velocity(cfg, std=1e-2, seed=21)
    run = oracle_run(cfg, 10, v0)
    sim = gpu_run(cfg, 10, "mixed", v0=v0)
    st = sim.status()
    assert st["returns_fp64"] > 0
    assert rel_l2(sim.read("u"), run.u) <= MIXED_TOL


@pytest.mark.parametrize("tile", [32, 64, 256])
def test_bond_tiles_match_oracle(tile):
    from paper_2203_05562_gb300 import Simulation
    cfg = pi.small_config(7, 6, 9, suction=50e3, rebuild_every=3)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=13)
    run = oracle_run(cfg, 6, v0)
    for precision, tol, norm in (("fp64", FP64_TOL, rel_inf), ("mixed", MIXED_TOL, rel_l2)):
        sim = Simulation(cfg, precision=precision, bond_tile=tile)
        sim.write("v", v0)
        sim.step(6)
        assert sim.status()["bond_tile"] == tile
        err = state_errors(sim, run, norm=norm)
        assert err["u"] <= tol and err["sigma"] <= tol, (precision, err)


@pytest.mark.parametrize("lanes", [4, 8])
def test_gather_lanes_match_oracle(lanes):
    # the force gather with four or eight lanes per point (the autotuner's two
    # candidates), both precisions, plastic bonds and rebuilds every 3 steps
    cfg = pi.small_config(7, 6, 9, suction=50e3, rebuild_every=3, gather_lanes=lanes)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=13)
    run = oracle_run(cfg, 6, v0)
    for precision, tol, norm in (("fp64", FP64_TOL, rel_inf), ("mixed", MIXED_TOL, rel_l2)):
        sim = gpu_run(cfg, 6, precision, v0=v0)
        assert sim.status()["gather_lanes"] == lanes
        err = state_errors(sim, run, norm=norm)
        assert err["u"] <= tol and err["a"] <= 10 * tol, (precision, err)


@pytest.mark.parametrize("model", [0, 2])
@pytest.mark.parametrize("ppb,grid", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_tensor_core_launch_shapes_match_oracle(model, ppb, grid):
    # the mixed path's tensor-core bond kernel (32 threads per point) with
    # one or two points per block, a grid over every point or a persistent
    # resident wave; plastic bonds (suction 50 kPa) and rebuilds every 3 steps
    from paper_2203_05562_gb300 import Simulation
    cfg = pi.small_config(7, 6, 9, suction=50e3, rebuild_every=3, model=model)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=13)
    run = oracle_run(cfg, 6, v0)
    sim = Simulation(cfg, precision="mixed", bond_tile=32, points_per_block=ppb, bond_grid=grid)
    sim.write("v", v0)
    sim.step(6)
    st = sim.status()
    assert st["bond_tile"] == 32 and st["points_per_block"] == ppb
    assert (st["bond_blocks"] > 0) == (grid == 2)
    assert st["plastic"] > 0
    err = state_errors(sim, run, norm=rel_l2)
    assert err["u"] <= MIXED_TOL and err["sigma"] <= MIXED_TOL, err


def test_autotuner_picks_a_tile_and_stays_correct():
    from paper_2203_05562_gb300 import Simulation
    cfg = pi.config(0)
    v0 = pi.initial_velocity(cfg)
    run = oracle_run(cfg, 10, v0)
    sim = Simulation(cfg, precision="mixed", bond_tile=0)
    sim.write("v", v0)
    sim.step(10)
    assert sim.status()["bond_tile"] in (32, 64, 128, 256)
    assert sim.status()["gather_lanes"] in (4, 8)
    assert rel_l2(sim.read("u"), run.u) <= MIXED_TOL


def test_rebuild_period_graph_matches_direct_launches():
    cfg = pi.small_config(6, 7, 9, suction=30e3, rebuild_every=4)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=2)
    a = gpu_run(cfg, 13, "mixed", v0=v0, use_graph=True)    # 3 four-step graphs + singles
    b = gpu_run(cfg, 13, "mixed", v0=v0, use_graph=False)
    for f in ("u", "v", "sigma", "pc"):
        assert np.array_equal(a.read(f), b.read(f)), f
    assert a.status()["rebuilds"] == b.status()["rebuilds"] == 4


def test_mixed_ensemble_matches_per_column_oracle():
    cols = pi.ensemble_columns(count=4, seed=5, n_min=200, n_max=700)
    cfg = pi.config("ensemble_64_columns_mixed", rebuild_every=5)
    n = sum(c["nx"] * c["ny"] * c["nz"] for c in cols)
    v0 = np.random.default_rng(8).normal(0, 1e-6, size=(3, n))
    sim = gpu_run(cfg, 12, "mixed", v0=v0, columns=cols)
    u = sim.read("u")
    off = 0
    for c in cols:
        cc = dict(cfg, **c)
        m = pi.num_points(cc)
        run = oracle_run(cc, 12, v0[:, off:off + m])
        assert rel_l2(u[:, off:off + m], run.u) <= MIXED_TOL
        off += m


@pytest.mark.parametrize("model,elastic", [(0, 0), (1, 0), (2, 0), (2, 1)])
def test_uniaxial_loading_matches_oracle(model, elastic):
    # the loading of Sec. 4.1: the end regions (a horizon thick) held in x and
    # driven at -load_rate, no fixed base; suction 50 kPa so that the returns
    # run too, or the elastic skeleton of that section
    cfg = pi.small_config(10, 5, 6, suction=50e3, model=model, bc=1, load_rate=0.05,
                          rebuild_every=3, elastic=elastic)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=21)
    run = oracle_run(cfg, 10, v0)
    assert (run.counters()["plastic"] > 0) == (elastic == 0)
    sim = gpu_run(cfg, 10, "fp64", v0=v0)
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err
    st, ce = sim.status(), run.energies()
    for key in ("W_int", "W_ext", "W_kin"):
        scale = max(abs(ce["W_int"]), abs(ce["W_ext"]), ce["W_kin"])
        assert abs(st[key] - ce[key]) <= FP64_TOL * scale, key
    sim = gpu_run(cfg, 10, "mixed", v0=v0)
    err = state_errors(sim, run, norm=rel_l2)
    assert err["u"] <= MIXED_TOL and err["sigma"] <= MIXED_TOL, err


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
def test_critical_time_step_matches_oracle(precision, tol):
    # Eq. 65 (reading R30) over a deformed column's family, after some steps
    cfg = pi.small_config(7, 6, 9, suction=30e3, rebuild_every=2)
    v0 = pi.initial_velocity(cfg, std=1e-2, seed=17)
    run = oracle_run(cfg, 6, v0)
    sim = gpu_run(cfg, 6, precision, v0=v0)
    got, want = sim.critical_time_step(), run.critical_time_step()
    assert np.isfinite(want) and abs(got - want) <= tol * want, (got, want)


@pytest.mark.parametrize("use_graph", [True, False])
def test_hard_stop_on_the_energy_check_matches_oracle(use_graph):
    # the Eq. 69 check as a hard stop, decided on the device (so also inside
    # CUDA graphs): the printed Eq. 51 force state under compression fails it
    cfg = pi.small_config(12, 4, 4, suction=0.0, model=0, bc=1, load_rate=0.05,
                          gravity=(0.0, 0.0, 0.0), elastic=1, init_stress=1, rebuild_every=0,
                          halt_on_unstable=1)
    run = oracle_run(cfg, 300, np.zeros((3, pi.num_points(cfg))))
    h = run.counters()["halted_step"]
    assert 0 < h < 300
    sim = gpu_run(cfg, 300, "fp64", v0=np.zeros((3, pi.num_points(cfg))), use_graph=use_graph)
    st = sim.status()
    assert "halted" in st["flags"] and st["halted_step"] == h
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err
    u = sim.read("u")
    sim.step(10)
    assert np.array_equal(sim.read("u"), u)


def test_substrate_contact_sliding_slab_matches_oracle():
    # Sec. 4.2: a one-layer slab sliding on the rigid substrate under friction
    cfg = pi.small_config(6, 6, 1, suction=0.0, elastic=1, init_stress=1, contact=1,
                          friction=0.25, rebuild_every=0, model=1)
    n = pi.num_points(cfg)
    v0 = np.zeros((3, n)); v0[0] = 0.1; v0[1] = 0.03
    run = oracle_run(cfg, 400, v0)
    for precision, tol, norm in (("fp64", FP64_TOL, rel_inf), ("mixed", MIXED_TOL, rel_l2)):
        sim = gpu_run(cfg, 400, precision, v0=v0)
        err = state_errors(sim, run, norm=norm)
        assert err["u"] <= tol and err["v"] <= tol, (precision, err)


@pytest.mark.parametrize("model", [0, 2])
def test_column_on_the_substrate_matches_oracle(model):
    # a plastic column resting on the substrate instead of a fixed base
    cfg = pi.small_config(6, 5, 8, suction=50e3, contact=1, model=model, rebuild_every=2)
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=23)
    run = oracle_run(cfg, 12, v0)
    assert run.counters()["plastic"] > 0
    sim = gpu_run(cfg, 12, "fp64", v0=v0)
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err
    st, ce = sim.status(), run.energies()
    for key in ("W_int", "W_ext", "W_kin"):
        scale = max(abs(ce["W_int"]), abs(ce["W_ext"]), ce["W_kin"])
        assert abs(st[key] - ce[key]) <= FP64_TOL * scale, key
    sim = gpu_run(cfg, 12, "mixed", v0=v0)
    err = state_errors(sim, run, norm=rel_l2)
    assert err["u"] <= MIXED_TOL, err


@pytest.mark.parametrize("model", [0, 1, 2])
def test_points_closer_than_the_cutoff_match_oracle(model):
    # Eq. 91 between points of the soil (reading R36): a point starting at
    # 0.4 dx of its x-neighbour in a column on the substrate
    cfg = pi.small_config(6, 5, 8, suction=50e3, contact=1, model=model, rebuild_every=2)
    n = pi.num_points(cfg)
    u0 = np.zeros((3, n))
    u0[0, 2 + 6 * 2 + 30 * 4] = 0.6 * cfg["dx"]
    v0 = pi.initial_velocity(cfg, std=1e-3, seed=29)
    run = oracle.Run(cfg, v0, u0=u0)
    run.step(12)
    sim = gpu_run(cfg, 12, "fp64", v0=v0, u=u0)
    err = state_errors(sim, run)
    assert max(err.values()) <= FP64_TOL, err
    sim = gpu_run(cfg, 12, "mixed", v0=v0, u=u0)
    err = state_errors(sim, run, norm=rel_l2)
    assert err["u"] <= MIXED_TOL, err
