"""Parity at the workloads' full sizes, in the launch configuration the
benchmark times (autotuned tile, graph replay): sampled points after one
step against oracle runs on lattice patches, plus properties that hold at
any size.

One step changes a point's state through its neighbours within 4 delta
(positions after the predictor depend on the initial accelerations within
2 delta; the force on a point on the positions within 2 delta), so a patch
of +-13 lattice sites (> 4 x 3.015) around a sampled point, with the full
column's initial stress and velocities, gives that point's exact result.
"""
import numpy as np
import pytest

import oracle
import ppm_inputs as pi

pytestmark = pytest.mark.gpu
R = 13


def _patch(cfg, ijk):
    lo = [max(0, ijk[d] - R) for d in range(3)]
    hi = [min(cfg[k] - 1, ijk[d] + R) for d, k in enumerate(("nx", "ny", "nz"))]
    dims = [hi[d] - lo[d] + 1 for d in range(3)]
    gx, gy, gz = np.meshgrid(np.arange(lo[0], hi[0] + 1), np.arange(lo[1], hi[1] + 1),
                             np.arange(lo[2], hi[2] + 1), indexing="ij")
    # patch point order: x fastest, then y, then z
    ids = (gx + cfg["nx"] * (gy + cfg["ny"] * gz)).transpose(2, 1, 0).reshape(-1)
    center = (ijk[0] - lo[0]) + dims[0] * ((ijk[1] - lo[1]) + dims[1] * (ijk[2] - lo[2]))
    return dims, ids, center


def _samples(cfg, count, seed):
    rng = np.random.default_rng(seed)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    pts = [(0, 0, nz - 1), (nx - 1, ny // 2, nz // 2), (nx // 2, ny // 2, nz // 2), (1, ny - 1, 1)]
    while len(pts) < count:
        pts.append(tuple(int(rng.integers(0, m)) for m in (nx, ny, nz)))
    return pts


@pytest.mark.parametrize("name,precision,count", [
    ("collapse_40x40x80_mixed", "fp64", 6),
    ("collapse_40x40x80_mixed", "mixed", 8),
    ("large_64x64x256_mixed", "mixed", 6),
])
def test_sampled_points_after_one_step(name, precision, count):
    from paper_2203_05562_gb300 import Simulation
    cfg = pi.config(name)
    n = pi.num_points(cfg)
    v0 = pi.initial_velocity(cfg)
    sim = Simulation(cfg, precision=precision, bond_tile=0)
    sim.write("v", v0)
    sim.step(1)
    got = {f: sim.read(f).astype(np.float64) for f in ("u", "v", "a", "sigma", "pc")}
    sig0 = oracle.initial_stress(cfg)
    tol = 1e-10 if precision == "fp64" else 1e-4
    for ijk in _samples(cfg, count, seed=11):
        dims, ids, c = _patch(cfg, ijk)
        pcfg = dict(cfg, nx=dims[0], ny=dims[1], nz=dims[2])
        run = oracle.Run(pcfg, v0[:, ids], sig0=sig0[:, ids])
        run.step(1)
        i = ids[c]
        want = {"u": run.u, "v": run.v, "a": run.a, "sigma": run.sig, "pc": run.pc[None]}
        for f, arr in want.items():
            arr = np.atleast_2d(arr)
            g = np.atleast_2d(got[f])[:, i]
            scale = np.abs(arr).max() + 1e-300
            err = np.abs(g - arr[:, c]).max() / scale
            assert err <= tol, (name, precision, ijk, f, err)


def test_full_size_properties_of_the_1m_point_column():
    from paper_2203_05562_gb300 import Simulation
    cfg = pi.config("large_64x64x256_mixed")
    sim = Simulation(cfg, precision="mixed", bond_tile=0)
    sim.write("v", pi.initial_velocity(cfg))
    sim.step(1)
    rp, col, rev = sim.read("row_ptr"), sim.read("col"), sim.read("rev")
    # undeformed lattice count: sum over offsets o != 0, |o| <= 3.015, of prod(n_d - |o_d|)
    total = 0
    for ox in range(-3, 4):
        for oy in range(-3, 4):
            for oz in range(-3, 4):
                if (ox, oy, oz) != (0, 0, 0) and ox * ox + oy * oy + oz * oz <= 3.015 ** 2:
                    total += (64 - abs(ox)) * (64 - abs(oy)) * (256 - abs(oz))
    assert rp[-1] == len(col) == total == 122821992
    assert np.diff(rp).max() == 122
    rows = np.repeat(np.arange(len(rp) - 1, dtype=np.int64), np.diff(rp))
    assert np.all(rev >= 0) and np.array_equal(col[rev], rows)
    # pairwise forces conserve linear momentum at any size
    f = sim.read("fint").astype(np.float64)
    scale = np.abs(f).sum(axis=1)
    assert np.all(np.abs(f.sum(axis=1)) <= 1e-5 * scale)


@pytest.mark.parametrize("shape", [dict(bond_tile=0), dict(bond_tile=32, bond_grid=2)])
def test_ensemble_with_a_60000_point_column_after_one_step(shape):
    # a batched ensemble (the workload's material and spacing) with a column
    # at the upper end of the ensemble's sizes (30 x 30 x 66 = 59,400 points)
    # and two small ones of other suctions and slopes, in the autotuned launch
    # shape and in a persistent wave over all columns: the small columns
    # against full oracle runs, the large one at sampled points against
    # oracle patches, after one step (mixed path, 1e-4)
    from paper_2203_05562_gb300 import Simulation
    base = pi.config("ensemble_64_columns_mixed")
    cols = [dict(nx=30, ny=30, nz=66, suction=35e3, M=1.3),
            dict(nx=10, ny=12, nz=20, suction=5e3, M=1.05),
            dict(nx=14, ny=14, nz=15, suction=48e3, M=1.38)]
    ccfg = [dict(base, nx=c["nx"], ny=c["ny"], nz=c["nz"], suction=c["suction"], M=c["M"]) for c in cols]
    v0s = [pi.initial_velocity(c, std=1e-4, seed=40 + q) for q, c in enumerate(ccfg)]
    sim = Simulation(base, columns=cols, precision="mixed", **shape)
    sim.write("v", np.concatenate(v0s, axis=1))
    sim.step(1)
    st = sim.status()
    if shape.get("bond_grid") == 2:
        assert st["bond_blocks"] > 0
    got = {f: sim.read(f).astype(np.float64) for f in ("u", "v", "a", "sigma", "pc")}
    offsets = np.cumsum([0] + [pi.num_points(c) for c in ccfg])
    tol = 1e-4
    for q, c in enumerate(ccfg):
        sl = slice(offsets[q], offsets[q + 1])
        sig0 = oracle.initial_stress(c)
        if q > 0:                                     # the small columns, whole
            run = oracle.Run(c, v0s[q], sig0=sig0)
            run.step(1)
            want = {"u": run.u, "v": run.v, "a": run.a, "sigma": run.sig, "pc": run.pc[None]}
            for f, arr in want.items():
                g = np.atleast_2d(got[f])[:, sl]
                err = np.abs(g - arr).max() / (np.abs(arr).max() + 1e-300)
                assert err <= tol, (q, f, err)
            continue
        for ijk in _samples(c, 5, seed=17):               # the 59,400-point column, sampled
            dims, ids, ctr = _patch(c, ijk)
            pcfg = dict(c, nx=dims[0], ny=dims[1], nz=dims[2])
            run = oracle.Run(pcfg, v0s[q][:, ids], sig0=sig0[:, ids])
            run.step(1)
            want = {"u": run.u, "v": run.v, "a": run.a, "sigma": run.sig, "pc": run.pc[None]}
            for f, arr in want.items():
                arr = np.atleast_2d(arr)
                g = np.atleast_2d(got[f])[:, offsets[q] + ids[ctr]]
                err = np.abs(g - arr[:, ctr]).max() / (np.abs(arr).max() + 1e-300)
                assert err <= tol, (ijk, f, err)
