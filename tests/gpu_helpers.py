"""Shared helpers of the GPU parity tests (no arithmetic of the method)."""
import numpy as np

import oracle
import ppm_inputs as pi


def rel_inf(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = np.abs(b).max()
    return float(np.abs(a - b).max() / (scale if scale > 0 else 1.0))


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def gpu_run(cfg, steps, precision, model=None, v0=None, use_graph=True, columns=None, u=None):
    from paper_2203_05562_gb300 import Simulation
    sim = Simulation(cfg, columns=columns, precision=precision, model=model, use_graph=use_graph)
    if v0 is not None:
        sim.write("v", v0)
    if u is not None:
        sim.write("u", u)
    sim.step(steps)
    return sim


def oracle_run(cfg, steps, v0=None):
    r = oracle.Run(cfg, v0)
    r.step(steps)
    return r


def state_errors(sim, run, norm=rel_inf):
    return dict(u=norm(sim.read("u"), run.u), v=norm(sim.read("v"), run.v),
                a=norm(sim.read("a"), run.a), sigma=norm(sim.read("sigma"), run.sig),
                pc=norm(sim.read("pc"), run.pc), eps_s=norm(sim.read("eps_s"), run.eps_s))
