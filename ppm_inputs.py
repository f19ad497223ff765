"""Seeded synthetic inputs shared by the oracle and the GPU library.

This module holds problem data only -- material constants, lattice sizes,
seeded random draws -- and none of the method's arithmetic.  Both the FP64
CPU oracle and the CUDA library receive exactly these arrays and numbers.

The soil columns stand in for the paper's 2-D column-collapse runs
(Sec. 4.2): the same kind of critical-state soil, synthetic and 3-D, with no
external data.  All quantities are SI (m, s, kg, Pa).
"""
from __future__ import annotations

import math

import numpy as np

#: Material shared by the five workloads (suction and M vary per workload).
MATERIAL = dict(
    horizon_factor=3.015,   # delta = 3.015 dx (about 122 bonds per interior point)
    rho=2000.0,             # kg/m^3
    K=20e6, mu=10e6,        # Pa
    M=1.2, lambda_t=0.1, kappa_t=0.02,
    pc0=20e3,               # Pa (initial preconsolidation, magnitude)
    eta=1000.0,             # Pa s, scaled by pc_n^2 in the default viscosity form
    vg_alpha=0.1e-3,        # 1/Pa  (0.1 1/kPa)
    vg_n=1.5,
    b1=0.0, b2=1.0,
    gravity=(0.0, 0.0, -9.81),
    dt=0.0,                 # 0: 0.3 dx / p-wave speed
    model=0, init_stress=0, visc_form=0,
    newton_max_iter=50, newton_tol=1e-10,
    lock_lateral=0,
    rebuild_every=1,
    bc=0,                   # 0: fixed base layer; 1: uniaxial compression along x
    load_rate=0.0,          # m/s, bc = 1
    elastic=0,              # 1: linear elastic skeleton (no yield), as in Sec. 4.1
    load_layers=0,          # bc = 1: planes held / driven at each end; 0: the horizon's thickness
    halt_on_unstable=0,     # 1: the Eq. 69 energy check stops the run
    contact=0,              # 1: rigid flat substrate (Sec. 4.2) instead of the fixed base
    contact_modulus=4e6,    # C_s, Pa (Sec. 4.2)
    friction=0.25,          # mu_f (Sec. 4.2)
    contact_cutoff=0.8,     # delta_c / dx (Sec. 4.2)
    energy_tol=0.0,         # tolerance of the Eq. 69 energy check; 0: 1e-2
    plane_strain=0,         # 1: plane strain in x-z, y periodic (ny dx > 4 delta), v_y = 0
    coupled=0,              # 1: J-dependent porosity, S_r, volume and mass (Eq. 15-16, 48-49)
    porosity=0.2,           # phi_0 (Sec. 4.2)
    rho_s=2200.0, rho_w=1000.0,   # kg/m^3 (Sec. 4.2)
    wr_a1=0.038, wr_a2=3.49, wr_n=1.25,      # Eq. 15 (Sec. 4.2; a1 read per Pa)
)

#: The five workloads: (description, overrides).
WORKLOADS = {
    "column_10x10x20_fp64": dict(nx=10, ny=10, nz=20, dx=0.005, suction=10e3, steps=50,
                                 rebuild_every=1, precision="fp64", seed=2203),
    "collapse_40x40x80_mixed": dict(nx=40, ny=40, nz=80, dx=0.0025, suction=20e3, steps=2000,
                                    rebuild_every=50, precision="mixed", seed=2204),
    "large_64x64x256_mixed": dict(nx=64, ny=64, nz=256, dx=0.00125, suction=30e3, steps=500,
                                  rebuild_every=50, precision="mixed", seed=2205),
    "ensemble_64_columns_mixed": dict(dx=0.0025, steps=1000, rebuild_every=50,
                                      precision="mixed", seed=2203, columns=64),
    "adjoint_40x40x80": dict(nx=40, ny=40, nz=80, dx=0.0025, suction=20e3, steps=200,
                             rebuild_every=50, precision="mixed", seed=2207, ckpt_every=20),
}

WORKLOAD_ORDER = list(WORKLOADS)


def config(name_or_index, **overrides) -> dict:
    """Full parameter dict of a workload (by name or position 0..4)."""
    name = WORKLOAD_ORDER[name_or_index] if isinstance(name_or_index, int) else name_or_index
    cfg = dict(MATERIAL)
    cfg.update(WORKLOADS[name])
    cfg["name"] = name
    cfg.update(overrides)
    return cfg


def small_config(nx=6, ny=6, nz=8, **overrides) -> dict:
    """A small column with the workload material, for tests."""
    cfg = dict(MATERIAL)
    cfg.update(nx=nx, ny=ny, nz=nz, dx=0.005, suction=10e3, steps=5, rebuild_every=1,
               precision="fp64", seed=7, name=f"column_{nx}x{ny}x{nz}")
    cfg.update(overrides)
    return cfg


def num_points(cfg) -> int:
    return int(cfg["nx"]) * int(cfg["ny"]) * int(cfg["nz"])


def initial_velocity(cfg, std: float = 1e-6, seed: int | None = None) -> np.ndarray:
    """Initial velocities N(0, std) m/s per component, shape (3, n),
    component-major; point id = ix + nx*(iy + ny*iz)."""
    n = num_points(cfg)
    rng = np.random.default_rng(cfg.get("seed", 0) if seed is None else seed)
    return rng.normal(0.0, std, size=(3, n))


def perturbation(cfg, amplitude: float, seed: int) -> np.ndarray:
    """A random displacement field, uniform in [-amplitude, amplitude]."""
    n = num_points(cfg)
    rng = np.random.default_rng(seed)
    return rng.uniform(-amplitude, amplitude, size=(3, n))


def ensemble_columns(count: int = 64, seed: int = 2203, n_min: int = 2000, n_max: int = 60000):
    """Column sizes, suctions and critical-state slopes of the batched
    ensemble: aspect ratio a ~ U[1, 4], target size N* ~ U[n_min, n_max],
    width w = round((N*/a)^(1/3)), height h = round(a w), clipped so that
    w*w*h lies in [n_min, n_max]; suction ~ U[0, 50] kPa, M ~ U[1.0, 1.4]."""
    rng = np.random.default_rng(seed)
    cols = []
    for _ in range(count):
        a = rng.uniform(1.0, 4.0)
        target = rng.uniform(n_min, n_max)
        w = max(2, int(round((target / a) ** (1.0 / 3.0))))
        h = max(2, int(round(a * w)))
        while w * w * h > n_max and h > 2:
            h -= 1
        while w * w * h < n_min:
            h += 1
        s = rng.uniform(0.0, 50e3)
        M = rng.uniform(1.0, 1.4)
        cols.append(dict(nx=w, ny=w, nz=h, suction=s, M=M))
    return cols
