"""The benchmark's own measures, checked on the host: the point-to-point
oscillation score of Sec. 4.1 against closed forms, the run-out column's
preconsolidation pressure against the oracle's geostatic state, and the
run-out measure of an undeformed column."""
import numpy as np
import pytest

import bench
import oracle
import ppm_inputs as pi


def grid(cfg):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    i = np.arange(nx * ny * nz)
    return i % nx, i // nx % ny, i // (nx * ny)


@pytest.mark.parametrize("plane_strain", [False, True])
def test_the_oscillation_score_of_closed_form_fields(plane_strain):
    cfg = bench.uniaxial_config(2, plane_strain)
    ix, iy, iz = grid(cfg)
    mean, amp = -30e3, 1.5e3
    flat = bench.oscillation_scores(np.full(ix.size, mean), cfg, 2)
    assert flat["checkerboard"] == 0.0 and flat["cv"] == 0.0 and flat["mean_sxx_Pa"] == mean
    # a linear field equals the mean of its six neighbours
    ramp = mean + 10.0 * ix + 20.0 * iy - 5.0 * iz
    assert bench.oscillation_scores(ramp, cfg, 2)["checkerboard"] == pytest.approx(0.0, abs=1e-12)
    # a checkerboard of amplitude a: every neighbour has the opposite sign
    chk = mean + amp * (-1.0) ** (ix + iy + iz)
    sc = bench.oscillation_scores(chk, cfg, 2)
    assert sc["checkerboard"] == pytest.approx(2 * amp / abs(sc["mean_sxx_Pa"]), rel=1e-12)


@pytest.mark.parametrize("aspect,suction", [(2.0, 0.0), (1.0, 0.0), (2.0, 25e3)])
def test_the_runout_column_is_over_consolidated_by_a_quarter_at_its_base(aspect, suction):
    cfg = dict(bench.runout_config(aspect, 0.25, suction), init_stress=0)
    assert cfg["nx"] == 40 and cfg["ny"] == 13 and cfg["plane_strain"] == 1 and cfg["contact"] == 1
    assert cfg["nz"] == int(round(0.1 / aspect / cfg["dx"]))
    sig = oracle.initial_stress(cfg)
    ix, iy, iz = grid(cfg)
    base = np.flatnonzero(iz == 0)
    p_eff = -(sig[0, base] + sig[1, base] + sig[2, base]) / 3.0     # compression positive
    assert np.allclose(cfg["pc0"], 1.25 * p_eff, rtol=1e-12)


def test_the_runout_of_an_undeformed_column():
    class Still:
        def __init__(self, n):
            self.n = n

        def read(self, field):
            return np.zeros((3, self.n))

    for ps in (True, False):
        cfg = bench.runout_config(2.0, 0.0, 0.0, plane_strain=ps)
        shape = bench.runout_shape(Still(pi.num_points(cfg)), cfg)
        assert shape == {"runout": 1.0, "height": 1.0}
