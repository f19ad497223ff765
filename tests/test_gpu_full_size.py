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
