"""The column collapse of Sec. 4.2 as the benchmark runs it: plane strain
(a slab 13 planes thick, periodic in y), 0.1 m wide at 2.5 mm, aspect 2,
on the substrate with the soil-soil repulsion, mixed path.  Over the first
0.1 s: no status flag, the Eq. 69 residual equal to (dt^2/8) times the
change of sum m|a|^2, the y-planes equal to within FP32 rounding, and a
smooth substrate letting the column spread further than a rough one."""
import numpy as np
import pytest

import bench

pytestmark = pytest.mark.gpu


def test_the_plane_strain_collapse_on_the_substrate():
    from paper_2203_05562_gb300 import Simulation
    shape = {}
    for mu in (0.0, 0.5):
        cfg = bench.runout_config(2.0, mu, 0.0)
        sim = Simulation(cfg, precision="mixed", bond_tile=0)
        sim.step(0)
        m = cfg["rho"] * cfg["dx"] ** 3
        a0 = sim.read("a").astype(np.float64)
        a0_sq = m * float((a0 * a0).sum())
        sim.step(int(round(0.1 / sim.dt / 50)) * 50)
        st = sim.status()
        assert st["flags"] == [], st["flags"]
        a = sim.read("a").astype(np.float64)
        resid = st["W_int"] + st["W_kin"] - st["W_ext"] - st["W_kin0"]
        pred = sim.dt ** 2 / 8.0 * (m * float((a * a).sum()) - a0_sq)
        scale = max(st["W_kin"], abs(st["W_int"]), abs(st["W_ext"]))
        assert abs(resid - pred) <= 2e-2 * abs(pred) + 1e-6 * scale, (resid, pred)
        u = sim.read("u").reshape(3, cfg["nz"], cfg["ny"], cfg["nx"]).astype(np.float64)
        assert np.all(u[1] == 0.0)
        # the planes list their members in different orders: FP32 rounding,
        # amplified over 17,000 steps of plastic flow (4e-3 measured)
        assert np.abs(u - u[:, :, :1, :]).max() <= 2e-2 * np.abs(u).max()
        shape[mu] = bench.runout_shape(sim, cfg)
    assert shape[0.0]["runout"] > shape[0.5]["runout"] > 1.0, shape
    # both slump; the order of the heights is the final deposits' (later)
    assert shape[0.0]["height"] < 1.0 and shape[0.5]["height"] < 1.0, shape
