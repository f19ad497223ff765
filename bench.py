"""Throughput of the per-step bond loop on one GB300 (bond-steps/s).

Workload (default): the 40x40x80 mixed-precision column collapse
(128,000 points, dx = 2.5 mm, delta = 3.015 dx, suction 20 kPa; family
rebuilt every 50 steps), inputs seeded and synthetic.  A "step" is one
explicit Newmark step of the whole path: predictor, family search when due,
the fused bond kernel, the force gather with the corrector, and the energy
terms.  The FP64 path is timed on the same column for comparison.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--runout]

Besides the headline, the JSON line carries:
- the roofline of the bond kernel, the HBM figures and the clocks, and the
  bond pass's time in every launch shape (warp tensor-core kernel, its
  persistent wave, the tensor-memory kernel, a scalar tile);
- the end-to-end rate through the API with host buffers;
- the mixed path's error against FP64 (precision);
- the FP64 path, the other force states and the coupled mode;
- the 64-column ensemble, the 1M-point column and the adjoint;
- Eq. 65's critical step, the uniaxial compression of Sec. 4.1 (3-D and plane strain);
- with --runout, the collapse study of Sec. 4.2;
- the oracle's CPU baseline.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload on the host cores.  Under torchrun each rank runs an
independent replica (the column does not shard); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ppm_inputs as pi  # noqa: E402

WORKLOAD = "collapse_40x40x80_mixed"
METRIC = "bond-steps/s (mixed path, 40x40x80 column collapse)"
UNIT = "bond-steps/s"
# FP32 lanes per SM and SM count of GB300; the ALU roof is lanes x 2 flop x clock
SMS, LANES = 152, 128
# algorithmic FP32 flops of the sub-horizon loop: per (bond, family member)
# membership test 8 flops (3 sub, 3 mul, 2 add); per (bond, sub-horizon
# member) 30 flops (15 multiply-adds into K~ and A~)
FLOPS_TEST, FLOPS_PAIR = 8, 30


BOND_SOURCES = ("bond.cu", "bond_device.cuh", "ppm_internal.cuh")


def bond_source_digest():
    """sha256 prefix over the code the bond kernel is compiled from: its
    sources with comments removed and whitespace collapsed, so that only a
    change of code (not of a comment) retires a profile."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in BOND_SOURCES:
        with open(os.path.join(ROOT, "paper_2203_05562_gb300", "csrc", name)) as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the bond kernel from the committed ncu
    summary, or None when the kernel's sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "bond_kernel_collapse_40x40x80.json")
    try:
        with open(path) as f:
            prof = json.load(f)
        digest = bond_source_digest()
    except OSError:
        return None
    if prof.get("bond_src_sha256_16") != digest:
        return None
    return prof.get("dram_bytes_per_launch")


def algorithmic_bytes(nbonds: int, npoints: int, mixed: bool) -> float:
    """DRAM bytes one step must move (R = 4 B mixed, 8 B FP64).
    Per bond: col and rev read (8 B), the force state written at its
    reverse slot (3R), that row read back by the gather (3R).  Per point:
    the bond kernel reads lat, colid, row_ptr (12 B), u, vh, sigma, pc, eps
    (14R) and writes sigma, pc, eps, tsum (11R); the gather reads row_ptr,
    lat (8 B), tsum, vh (6R) and writes fint, a, v (9R); the predictor reads
    u, v, a (9R) and writes u, vh (6R), plus the FP32 displacement
    compensation (read and written, 24 B)."""
    R = 4 if mixed else 8
    return nbonds * (8 + 6 * R) + npoints * (20 + 55 * R + (24 if mixed else 0))


def bond_kernel_bytes(nbonds: int, npoints: int) -> float:
    """DRAM bytes of one launch of the mixed bond kernel: col and rev read,
    the reverse-slot force state written (20 B per bond); per point lat,
    colid, row_ptr, u, vh, sigma, pc, eps read and sigma, pc, eps, tsum
    written (12 + 14 x 4 + 11 x 4 = 112 B)."""
    return nbonds * 20 + npoints * 112


def uniaxial_config(m: int, plane_strain: bool = False) -> dict:
    """The uniaxial compression test of Sec. 4.1, synthetic: in 3-D,
    12,000 points (40 x 15 x 20, spacing 5 mm), or in plane strain (the
    paper's setting) 40 x 13 x 20 with y periodic; K = 25 MPa, mu = 15 MPa,
    skeleton density 2200 kg/m^3 with porosity 0.2, saturated at zero
    suction, the elastic skeleton, horizon m spacings (+0.015 against ties),
    u_x = 0.5 mm over 0.1 s applied by the end regions (a horizon thick) at
    the dynamic time step of 3e-6 s, no gravity."""
    return pi.small_config(40, 13 if plane_strain else 15, 20, dx=0.005, horizon_factor=m + 0.015,
                           K=25e6, mu=15e6, rho=0.8 * 2200.0 + 0.2 * 1000.0, suction=0.0,
                           elastic=1, init_stress=1, gravity=(0.0, 0.0, 0.0), bc=1,
                           load_rate=0.5e-3 / 0.1, dt=3e-6, rebuild_every=0,
                           plane_strain=int(plane_strain))


def oscillation_scores(sxx, cfg, m: int) -> dict:
    """Point-to-point oscillation of sigma_xx over the points at least a
    horizon inside the loaded regions and the lateral faces: the mean of
    |sigma_i - mean of its six lattice neighbours| over |mean sigma|, the
    coefficient of variation, and the mean."""
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    g = np.asarray(sxx, np.float64).reshape(nz, ny, nx)
    mx, my = 2 * m, m
    def sh(dz, dy, dx):
        return g[my + dz:nz - my + dz, my + dy:ny - my + dy, mx + dx:nx - mx + dx]
    core = sh(0, 0, 0)
    nbr = (sh(0, 0, -1) + sh(0, 0, 1) + sh(0, -1, 0) + sh(0, 1, 0) + sh(-1, 0, 0) + sh(1, 0, 0)) / 6
    mean = float(core.mean())
    return {"checkerboard": float(np.abs(core - nbr).mean() / abs(mean)),
            "cv": float(core.std() / abs(mean)), "mean_sxx_Pa": mean}


def uniaxial_compression(steps: int, tile: int, early: int = 10000, plane_strain: bool = False):
    """The three force states (in plane strain the two that conserve
    energy) on the Sec. 4.1 test at m = 2 and 3; the oscillation scores
    after `early` steps (u_x = 0.15 mm) and at the end."""
    import torch
    from paper_2203_05562_gb300 import Simulation
    out = []
    for m in (2, 3):
        cfg = uniaxial_config(m, plane_strain)
        for model in ((1, 2) if plane_strain else (1, 2, 0)):
            sim = Simulation(cfg, precision="mixed", model=model, bond_tile=tile)
            r = {"m": m, "model": model, "steps": steps, "ms": 0.0}
            for tag, upto in (("early", min(early, steps)), ("end", steps)):
                done = 0 if tag == "early" else min(early, steps)
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record(sim.stream)
                sim.step(upto - done)
                ev1.record(sim.stream)
                torch.cuda.synchronize()
                r["ms"] += ev0.elapsed_time(ev1)
                st = sim.status()
                sig = sim.read("sigma")
                snap = {"steps": upto, "flags": st["flags"],
                        "W_kin_over_W_int": st["W_kin"] / abs(st["W_int"]) if st["W_int"] else None}
                if np.isfinite(sig).all():
                    snap.update(oscillation_scores(sig[0], cfg, m))
                r[tag] = snap
            out.append(r)
            del sim
    return out


def runout_config(aspect: float, friction: float, suction: float, plane_strain: bool = True) -> dict:
    """The soil column collapse of Sec. 4.2, synthetic: in plane strain (the
    paper's setting; a slab 13 planes thick, periodic in y) or as a square
    3-D column; 0.1 m wide (40 points at 2.5 mm) and 0.1 / aspect high resting on
    the rigid substrate (C_s = 4 MPa, delta_c = 0.8 dx, friction mu_f),
    released from the K0 geostatic state at a constant suction, with the
    preconsolidation pressure 1.25 x the initial mean effective stress at the
    base (the geostatic part plus S_r s: over-consolidation ratio 1.25
    there), the power-conjugate sub-horizon force state, the family rebuilt
    every 50 steps."""
    dx, nx = 0.0025, 40
    nz = int(round(0.1 / aspect / dx))
    m = pi.MATERIAL
    nu = (3 * m["K"] - 2 * m["mu"]) / (2 * (3 * m["K"] + m["mu"]))
    k0 = nu / (1 - nu)
    p_base = (1 + 2 * k0) / 3 * m["rho"] * -m["gravity"][2] * (nz - 1) * dx
    n_vg = m["vg_n"]
    s_r = (1 + (m["vg_alpha"] * suction) ** n_vg) ** -(1 - 1 / n_vg)
    return pi.small_config(nx, 13 if plane_strain else nx, nz, dx=dx, suction=suction, model=2,
                           contact=1, friction=friction, pc0=1.25 * (p_base + s_r * suction),
                           rebuild_every=50, energy_tol=5e-2, plane_strain=int(plane_strain))


def runout_shape(sim, cfg) -> dict:
    """Run-out (largest horizontal distance from the column's axis over the
    initial half-width; along x in plane strain) and deposit height (over
    the initial height)."""
    nx, ny, nz, dx = cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"]
    i = np.arange(nx * ny * nz)
    x = np.stack([i % nx, i // nx % ny, i // (nx * ny)]) * dx + sim.read("u").astype(np.float64)
    c = (cfg["nx"] - 1) * cfg["dx"] / 2
    reach = np.abs(x[0] - c) if cfg["plane_strain"] else np.maximum(np.abs(x[0] - c), np.abs(x[1] - c))
    return {"runout": float(reach.max() / c),
            "height": float(x[2].max() / ((cfg["nz"] - 1) * cfg["dx"]))}


def collapse_runout(tile: int) -> list:
    """Sec. 4.2.1-4.2.3 in plane strain on the substrate: the dry column at
    aspect 2 on a smooth, an intermediate and a rough substrate (mu_f = 0,
    0.25, 0.5), at suctions 25 and 50 kPa (mu_f = 0.25), and at aspects 1
    and 0.5, each to the end time of the paper's snapshots for that aspect."""
    import torch
    from paper_2203_05562_gb300 import Simulation
    runs = [(2.0, 0.0, 0.0), (2.0, 0.25, 0.0), (2.0, 0.5, 0.0),
            (2.0, 0.25, 25e3), (2.0, 0.25, 50e3), (1.0, 0.25, 0.0), (0.5, 0.25, 0.0)]
    t_end = {2.0: 0.25, 1.0: 0.4, 0.5: 0.5}
    out = []
    for aspect, friction, suction in runs:
        cfg = runout_config(aspect, friction, suction)
        sim = Simulation(cfg, precision="mixed", bond_tile=tile)
        steps = int(round(t_end[aspect] / sim.dt / 50)) * 50
        r = {"aspect": aspect, "friction": friction, "suction_Pa": suction,
             "points": sim.n, "steps": steps, "t_end_s": steps * sim.dt, "snapshots": []}
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, done = 0.0, 0
        for q in (1, 2, 3, 4):
            upto = steps * q // 4 // 50 * 50
            ev0.record(sim.stream)
            sim.step(upto - done)
            ev1.record(sim.stream)
            torch.cuda.synchronize()
            ms += ev0.elapsed_time(ev1)
            done = upto
            st = sim.status()
            r["snapshots"].append(dict(runout_shape(sim, cfg), t_s=done * sim.dt, flags=st["flags"],
                                       unstable_step=st["unstable_step"], W_kin=st["W_kin"],
                                       eq69_residual_over_max=eq69_ratio(st)))
        st = sim.status()
        r.update(ms_per_step=ms / steps, bond_steps_per_s=st["bond_steps"] / (ms * 1e-3))
        out.append(r)
        del sim
    return out


def eq69_ratio(st) -> float:
    """|W_int + W_kin - W_ext - W_kin0| over the largest of the four terms."""
    bal = abs(st["W_int"] + st["W_kin"] - st["W_ext"] - st["W_kin0"])
    return bal / max(st["W_kin"], abs(st["W_int"]), abs(st["W_ext"]), st["W_kin0"])


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.file.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def aggregate_over_ranks(ms: float, bond_steps: float, dist=None, device="cuda"):
    """Whole-job figures of N replicas: the slowest rank's time (max) and
    every rank's bond-steps (sum).  dist is torch.distributed (or None for
    one process); device is where the collective's tensors live ("cuda"
    under NCCL, "cpu" under gloo)."""
    if dist is None:
        return ms, bond_steps
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    b = torch.tensor([bond_steps], dtype=torch.float64, device=device)
    dist.all_reduce(b)
    return float(t.item()), float(b.item())


def oracle_sample(steps: int = 4, single_steps: int = 1):
    """The FP64 CPU oracle, as it stands, on the benchmark's own column: the
    family is built outside the timing (the oracle's search is brute force),
    one warm-up step, then `steps` steps on all the host's threads and
    `single_steps` on one thread (no family rebuild falls in the sample).
    Returns (bond-steps/s, threads, description, single-thread bond-steps/s,
    (steps taken, u, sigma) of the oracle at the end)."""
    import oracle
    cfg = pi.config(WORKLOAD)
    run = oracle.Run(cfg, pi.initial_velocity(cfg))
    run.step(1)                                   # warm-up step
    threads = oracle.num_threads()
    t0 = time.perf_counter()
    run.step(steps)
    rate = run.nbonds * steps / (time.perf_counter() - t0)
    single = None
    if single_steps > 0:
        oracle.set_threads(1)
        t0 = time.perf_counter()
        run.step(single_steps)
        single = run.nbonds * single_steps / (time.perf_counter() - t0)
        oracle.set_threads(threads)
    desc = (f"the full 40x40x80 column ({run.n:,} points, {run.nbonds:,} bonds): {steps} steps on "
            f"{threads} threads and {single_steps} on one, after one warm-up step; family built "
            f"outside the timing, no rebuild in the sample; FP64 oracle")
    return rate, threads, desc, single, (run.steps_done, run.u.copy(), run.sig.copy())


def rel_l2(a, b) -> float:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def precision_report(cfg, tile, u_timed, timed_steps, oracle_state):
    """The mixed path's error against FP64 on the benchmark's column: after
    the oracle's own steps, against the FP64 oracle itself (and the FP64 GPU
    path beside it); and after the timed run, against the FP64 GPU path over
    the same steps (which matches the oracle to 1e-10 in the parity tests)."""
    from paper_2203_05562_gb300 import Simulation
    out = {}
    if oracle_state is not None:
        n_or, u_or, sig_or = oracle_state
        row = {"steps": n_or}
        for prec in ("mixed", "fp64"):
            s = Simulation(cfg, precision=prec, bond_tile=tile)
            s.write("v", pi.initial_velocity(cfg))
            s.step(n_or)
            row[prec] = {"u_rel_l2": rel_l2(s.read("u"), u_or), "sigma_rel_l2": rel_l2(s.read("sigma"), sig_or)}
            del s
        out["against_fp64_oracle"] = row
    s = Simulation(cfg, precision="fp64", bond_tile=0)
    s.write("v", pi.initial_velocity(cfg))
    s.step(timed_steps)
    u64 = s.read("u")
    out["after_timed_run_against_fp64_path"] = {"steps": timed_steps, "u_rel_l2": rel_l2(u_timed, u64)}
    del s
    return out


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    rate, threads, desc, _, _ = oracle_sample(max(1, min(args.steps, 5)), single_steps=0)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "sample": desc},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def align_to_rebuild(warmup: int, rebuild_every: int) -> int:
    """Untimed steps after `warmup` so that the first timed step is one
    that rebuilds the family (a step with index s rebuilds when
    (s + 1) % R == 0): the timed region then holds ceil(K / R) family
    searches for K steps, the whole periods' share when R divides K."""
    if rebuild_every <= 1:
        return 0
    return (rebuild_every - 1 - warmup) % rebuild_every


def time_path(cfg, precision, steps, warmup, stream_sync):
    """Device-timed steps of one precision; returns a dict of figures.  The
    timed region starts at a family rebuild (align_to_rebuild)."""
    import torch
    from paper_2203_05562_gb300 import Simulation
    sim = Simulation(cfg, precision=precision, bond_tile=0)
    sim.write("v", pi.initial_velocity(cfg))
    sim.step(warmup + align_to_rebuild(warmup, cfg.get("rebuild_every", 0)))
    torch.cuda.synchronize()
    st0 = sim.status()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream_sync()
    ev0.record(sim.stream)
    sim.step(steps)
    ev1.record(sim.stream)
    torch.cuda.synchronize()
    stream_sync()
    ms = ev0.elapsed_time(ev1)
    st1 = sim.status()
    return sim, dict(ms=ms, bond_steps=st1["bond_steps"] - st0["bond_steps"],
                     pairs=st1["pairs"] - st0["pairs"], launches=st1["launches"] - st0["launches"],
                     rebuilds=st1["rebuilds"] - st0["rebuilds"], nbonds=st1["nbonds"], status=st1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--standard-steps", type=int, default=100)
    ap.add_argument("--no-uniaxial", action="store_true")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the mixed-vs-FP64 error report (about 25 s)")
    ap.add_argument("--runout", action="store_true",
                    help="also run the column-collapse run-out study of Sec. 4.2 (about 4 min)")
    ap.add_argument("--uniaxial-steps", type=int, default=33334,
                    help="steps of the Sec. 4.1 test (0.1 s at dt = 3e-6 s)")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--large-steps", type=int, default=50)
    ap.add_argument("--tile", type=int, default=32, help="bond-kernel tile for --profile-only")
    ap.add_argument("--ensemble-steps", type=int, default=100)
    ap.add_argument("--profile-only", action="store_true",
                    help="run warm-up + steps of the mixed path only (for ncu captures)")
    ap.add_argument("--profile-adjoint", type=int, default=0,
                    help="with --profile-only: an adjoint of this many steps (checkpoints every "
                         "half of them) instead of plain steps")
    ap.add_argument("--profile-model", type=int, default=0, choices=[0, 1, 2],
                    help="the force state --profile-only runs (0: Eq. 51, 1: standard, 2: power-conjugate)")
    ap.add_argument("--profile-workload", default=WORKLOAD,
                    choices=[WORKLOAD, "large_64x64x256_mixed"],
                    help="the column --profile-only runs")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    cfg = pi.config(WORKLOAD)
    n = pi.num_points(cfg)
    sampler = ClockSampler(local)
    if args.profile_only:
        from paper_2203_05562_gb300 import Simulation
        pcfg = pi.config(args.profile_workload)
        sim = Simulation(pcfg, precision="mixed", model=args.profile_model, use_graph=False,
                         bond_tile=args.tile)
        sim.write("v", pi.initial_velocity(pcfg))
        if args.profile_adjoint > 0:
            sim.adjoint_forward(args.profile_adjoint, max(1, args.profile_adjoint // 2))
            u = sim.read("u", device=True).double()
            nxy = pcfg["nx"] * pcfg["ny"]
            dJ = torch.zeros_like(u)
            dJ[0:2, -nxy:] = 2.0 * u[0:2, -nxy:]
            sim.adjoint_reverse(dJ)
        else:
            sim.step(args.warmup + args.steps)
        torch.cuda.synchronize()
        print(json.dumps({"profile_only": True, "status": sim.status()["flags"]}))
        return 0

    # ---- device-timed mixed path (the headline) ----
    barrier()
    sampler.start()
    sim, fig = time_path(cfg, "mixed", args.steps, args.warmup, barrier)
    clocks = sampler.stop()
    ms, total_bond_steps = aggregate_over_ranks(fig["ms"], float(fig["bond_steps"]), dist)
    value = total_bond_steps / (ms * 1e-3)

    # ---- dominant kernel: per-phase CUDA-event times on the launching stream,
    # over the same warm-up and steps as the headline, on a fresh column ----
    st = sim.status()
    u_timed = sim.read("u")                       # the precision report compares it with FP64
    steps_timed_run = int(st["steps"])            # warm-up, alignment to a rebuild, timed steps
    # Eq. 65 (reading R30) on the column at the end of the run, beside the step used
    critical = {"eq65_s": sim.critical_time_step(), "dt_used_s": sim.dt,
                "note": "micro-modulus over bond length; stable for models 1 and 2 up to at least 2x"}
    del sim
    from paper_2203_05562_gb300 import Simulation
    tile = fig["status"]["bond_tile"]          # the autotuner's choice, reused below
    shape = {"threads_per_point": tile, "points_per_block": fig["status"]["points_per_block"],
             "persistent_blocks": fig["status"]["bond_blocks"],
             "gather_lanes": fig["status"]["gather_lanes"]}
    cfg_t = dict(cfg, gather_lanes=shape["gather_lanes"])   # the autotuner's gather for fixed-shape runs
    shape_kw = dict(bond_tile=tile, points_per_block=shape["points_per_block"],
                    bond_grid=2 if shape["persistent_blocks"] else 1)
    tsim = Simulation(cfg_t, precision="mixed", **shape_kw)
    tsim.write("v", pi.initial_velocity(cfg))
    tsim.step(args.warmup + align_to_rebuild(args.warmup, cfg["rebuild_every"]))
    t0 = tsim.status()
    phase = tsim.step_timed(args.steps)
    t1 = tsim.status()
    nph = args.steps
    bond_ms = phase[1] / nph
    pairs_per_step = (t1["pairs"] - t0["pairs"]) / nph
    nb = fig["nbonds"]
    rp = tsim.read("row_ptr")
    fam_sq = float(np.sum(np.diff(rp).astype(np.float64) ** 2))
    del tsim
    # every launch shape of the bond pass on the same steps (the autotuner's
    # candidates for this workload): event-timed mean ms per bond launch
    shape_ms = {}
    for name, kw in (("warp_tensor_core_32", dict(bond_tile=32, points_per_block=1, bond_grid=1)),
                     ("warp_tensor_core_32_persistent", dict(bond_tile=32, points_per_block=1, bond_grid=2)),
                     ("tensor_memory_tcgen05_128", dict(bond_tile=128)),
                     ("scalar_64", dict(bond_tile=64))):
        ssim = Simulation(cfg, precision="mixed", **kw)
        ssim.write("v", pi.initial_velocity(cfg))
        ssim.step(args.warmup + align_to_rebuild(args.warmup, cfg["rebuild_every"]))
        shape_ms[name] = ssim.step_timed(args.steps)[1] / args.steps
        del ssim
    flops = FLOPS_TEST * fam_sq + FLOPS_PAIR * pairs_per_step
    peaks, peak_kind = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nominal_tflops = SMS * LANES * 2 * sm_max * 1e6 / 1e12
    from paper_2203_05562_gb300.ppm import measure_fp32_peak
    peak_tflops = measure_fp32_peak()             # FMA chains on this GPU, now
    achieved = flops / (bond_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": achieved / peak_tflops, "traffic": profiled_traffic(),
                "traffic_unit": "DRAM bytes per launch (ncu, profiles/)",
                "kernel": ("k_bond_tcw<0> (fused bond kernel, sub-horizon sums on the tensor cores, "
                           "one warp per point)" if tile == 32 else
                           f"k_bond<float,0,{tile}> (fused sub-horizon / constitutive / force state)"),
                "launch_shape": shape,
                "peak_kind": "measured: FP32 FMA chains on every SM (ppm_measure_fp32_peak), this run",
                "peak_nominal": nominal_tflops, "frac_of_nominal": achieved / nominal_tflops,
                "nominal_kind": f"FP32 lanes x 2 x {sm_max:.0f} MHz ({peak_kind} max SM clock)",
                "flops_per_launch": flops,
                "bond_kernel_ms": bond_ms, "bond_kernel_ms_by_launch_shape": shape_ms,
                "gather_ms": phase[2] / nph,
                "predictor_family_ms": phase[0] / nph}

    # ---- batched ensemble: 64 columns in one context, whole rebuild periods as graphs ----
    ens = None
    if not args.no_ensemble:
        ecfg = pi.config("ensemble_64_columns_mixed")
        cols = pi.ensemble_columns(64, seed=ecfg["seed"])
        esim0 = Simulation(ecfg, columns=cols, precision="mixed", bond_tile=0)
        ne = esim0.n
        esim0.write("v", np.random.default_rng(ecfg["seed"]).normal(0, 1e-6, size=(3, ne)))
        esim0.step(args.warmup + align_to_rebuild(args.warmup, ecfg["rebuild_every"]))
        torch.cuda.synchronize()
        e0 = esim0.status()
        eva, evb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        eva.record(esim0.stream)
        esim0.step(args.ensemble_steps)
        evb.record(esim0.stream)
        torch.cuda.synchronize()
        e1 = esim0.status()
        ems = eva.elapsed_time(evb)
        ens = {"workload": "ensemble_64_columns_mixed", "columns": 64, "points": ne,
               "bonds": e1["nbonds"], "steps": args.ensemble_steps,
               "value": (e1["bond_steps"] - e0["bond_steps"]) / (ems * 1e-3), "unit": UNIT,
               "ms_per_step": ems / args.ensemble_steps, "bond_tile": e1["bond_tile"],
               "points_per_block": e1["points_per_block"], "persistent_blocks": e1["bond_blocks"],
               "rebuilds_timed": e1["rebuilds"] - e0["rebuilds"],
               "graph": "one CUDA graph per 50-step rebuild period; the bond pass one launch over all columns"}
        del esim0
        # the cost of the kernel boundaries inside a step: a 64-point column run
        # through the same graphs, whose kernels do almost no work
        tcfg = pi.small_config(4, 4, 4, precision="mixed", rebuild_every=ecfg["rebuild_every"])
        tsim0 = Simulation(tcfg, precision="mixed")
        tsim0.step(ecfg["rebuild_every"])
        torch.cuda.synchronize()
        tsteps = 10 * ecfg["rebuild_every"]
        eva.record(tsim0.stream)
        tsim0.step(tsteps)
        evb.record(tsim0.stream)
        torch.cuda.synchronize()
        floor_ms = eva.elapsed_time(evb) / tsteps
        ens["step_floor_us"] = 1e3 * floor_ms
        ens["step_floor_share"] = floor_ms / ens["ms_per_step"]
        ens["step_floor_note"] = ("ms per step of a 64-point column through the same per-step graph "
                                  "(predictor, bond, gather, energy launches; the family search every "
                                  "rebuild period): the kernel boundaries one persistent launch would remove")
        del tsim0

    # ---- large column (64x64x256, 1,048,576 points), mixed ----
    large = None
    if not args.no_large:
        lcfg = pi.config("large_64x64x256_mixed")
        lsim = Simulation(lcfg, precision="mixed", bond_tile=0)
        lsim.write("v", pi.initial_velocity(lcfg))
        lsim.step(args.warmup + align_to_rebuild(args.warmup, lcfg["rebuild_every"]))
        torch.cuda.synchronize()
        l0 = lsim.status()
        la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        la.record(lsim.stream)
        lsim.step(args.large_steps)
        lb.record(lsim.stream)
        torch.cuda.synchronize()
        l1 = lsim.status()
        lms = la.elapsed_time(lb)
        large = {"workload": "large_64x64x256_mixed", "points": lsim.n, "bonds": l1["nbonds"],
                 "steps": args.large_steps, "value": (l1["bond_steps"] - l0["bond_steps"]) / (lms * 1e-3),
                 "unit": UNIT, "ms_per_step": lms / args.large_steps, "bond_tile": l1["bond_tile"],
                 "points_per_block": l1["points_per_block"], "persistent_blocks": l1["bond_blocks"],
                 "rebuilds_timed": l1["rebuilds"] - l0["rebuilds"]}
        del lsim

    # ---- adjoint: 40x40x80 column, 200 steps, checkpoints every 20 ----
    adj = None
    if not args.no_adjoint:
        # warm-up: a two-step adjoint on a small column loads the adjoint's
        # kernels (modules load lazily, on first launch; about 1.4 s here)
        wcfg = pi.small_config(5, 5, 7, suction=50e3)
        wsim = Simulation(wcfg, precision="mixed", use_graph=False, bond_tile=tile)
        wsim.write("v", pi.initial_velocity(wcfg, std=1e-3, seed=1))
        wsim.adjoint_forward(2, 1)
        wsim.adjoint_reverse(np.zeros((3, wsim.n)))
        torch.cuda.synchronize()
        del wsim
        acfg = pi.config("adjoint_40x40x80")
        av0 = pi.initial_velocity(acfg)
        asim = Simulation(acfg, precision="mixed", use_graph=False, bond_tile=tile)
        asim.write("v", av0)
        ta = time.perf_counter()
        asim.adjoint_forward(acfg["steps"], acfg["ckpt_every"])
        torch.cuda.synchronize()
        tb = time.perf_counter()
        u = asim.read("u", device=True).double()
        nxy = acfg["nx"] * acfg["ny"]
        dJ = torch.zeros_like(u)
        dJ[0:2, -nxy:] = 2.0 * u[0:2, -nxy:]
        g = asim.adjoint_reverse(dJ)
        torch.cuda.synchronize()
        tc = time.perf_counter()
        # the reverse call leaves the context at the final state: repeat it
        # warm (the first call's time varies between machines by about 1.3 s)
        g2 = asim.adjoint_reverse(dJ)
        torch.cuda.synchronize()
        td = time.perf_counter()
        adj = {"workload": "adjoint_40x40x80", "steps": acfg["steps"], "ckpt_every": acfg["ckpt_every"],
               "objective": float((u[0:2, -nxy:] ** 2).sum()),
               "grad": {"M": g[0], "eta": g[1], "suction": g[2], "pc0": g[3]},
               "repeat_bitwise_equal": bool(np.array_equal(np.asarray(g), np.asarray(g2))),
               "forward_s": tb - ta, "reverse_s": td - tc, "reverse_first_call_s": tc - tb,
               "reverse_over_forward": (td - tc) / (tb - ta)}
        del asim

    # ---- FP64 path on the same column (fewer steps: FP64 is ~1/64 rate) ----
    sim64, fig64 = time_path(cfg, "fp64", args.fp64_steps, 1, barrier)
    fp64_rate = fig64["bond_steps"] / (fig64["ms"] * 1e-3)
    del sim64

    # ---- the uniaxial compression test of Sec. 4.1 (NEXT-1 comparison) ----
    uniaxial = None
    if not args.no_uniaxial:
        uniaxial = {"workload": "uniaxial_40x15x20 (Sec. 4.1, dynamic loading, elastic skeleton)",
                    "runs": uniaxial_compression(args.uniaxial_steps, tile),
                    "plane_strain": {"workload": "uniaxial_40x13x20, y periodic",
                                     "runs": uniaxial_compression(args.uniaxial_steps, tile,
                                                                  plane_strain=True)}}

    # ---- run-out of the column collapse on the substrate (Sec. 4.2, opt-in) ----
    runout = None
    if args.runout:
        runout = {"workload": "plane-strain collapse on the substrate, 40 x 13 (periodic) x 0.1/(aspect dx), dx 2.5 mm",
                  "runs": collapse_runout(tile)}

    # ---- standard correspondence (model 1) on the same column ----
    simS, figS = time_path(dict(cfg, model=1), "mixed", args.standard_steps, args.warmup, barrier)
    standard = {"model": "standard correspondence (every sub-horizon is the family)",
                "value": figS["bond_steps"] / (figS["ms"] * 1e-3), "unit": UNIT,
                "steps": args.standard_steps, "ms_per_step": figS["ms"] / args.standard_steps,
                "bond_tile": figS["status"]["bond_tile"]}
    del simS

    # ---- the other modes on the same column: the power-conjugate sub-horizon
    # force state, and the coupled mode (Eq. 15-16, 48-49) on the headline's ----
    other_modes = {}
    for tag, mcfg in (("power_conjugate_subhorizon", dict(cfg, model=2)),
                      ("coupled", dict(cfg, coupled=1))):
        simO, figO = time_path(mcfg, "mixed", args.standard_steps, args.warmup, barrier)
        other_modes[tag] = {"value": figO["bond_steps"] / (figO["ms"] * 1e-3), "unit": UNIT,
                            "steps": args.standard_steps, "ms_per_step": figO["ms"] / args.standard_steps,
                            "bond_tile": figO["status"]["bond_tile"], "flags": figO["status"]["flags"]}
        del simO
        if tag == "power_conjugate_subhorizon":
            # the bond kernel against the FP32 roof: the sender pass's algorithmic
            # flops (as the headline's) plus 9 adds per (receiver, sender) pair
            rsim = Simulation(mcfg, precision="mixed", **shape_kw)
            rsim.write("v", pi.initial_velocity(mcfg))
            rsim.step(args.warmup + align_to_rebuild(args.warmup, mcfg["rebuild_every"]))
            r0s = rsim.status()
            rms = rsim.step_timed(args.steps)[1] / args.steps
            rpairs = (rsim.status()["pairs"] - r0s["pairs"]) / args.steps
            del rsim
            rflops = FLOPS_TEST * fam_sq + (FLOPS_PAIR + 9) * rpairs
            other_modes[tag]["roofline"] = {
                "bound": "alu", "kernel": "k_bond_tcw<2> (sender and receiver passes on the tensor cores)",
                "bond_kernel_ms": rms, "flops_per_launch": rflops,
                "achieved": rflops / (rms * 1e-3) / 1e12, "peak": peak_tflops, "unit": "TFLOP/s",
                "frac": rflops / (rms * 1e-3) / 1e12 / peak_tflops,
                "note": "algorithmic flops: 8 per family pair tested, 30 per sub-horizon pair summed, "
                        "9 per (receiver, sender) pair of the receiver sums"}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    from paper_2203_05562_gb300 import Simulation
    host_v0 = torch.from_numpy(pi.initial_velocity(cfg).astype(np.float32)).pin_memory()
    host_u = torch.empty((3, n), dtype=torch.float32).pin_memory()
    esim = Simulation(cfg_t, precision="mixed", **shape_kw)
    esim.write("v", host_v0.numpy())
    esim.step(args.warmup + align_to_rebuild(args.warmup, cfg["rebuild_every"]))
    torch.cuda.synchronize()
    barrier()
    s0 = esim.status()["bond_steps"]
    t0 = time.perf_counter()
    host_u_np = host_u.numpy()
    esim.write("v", host_v0.numpy())    # this run's input, from pinned host memory
    for _ in range(args.steps):
        esim.step(1)
        esim.read("u", out=host_u_np)   # the step's result back to pinned host memory
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    s1 = esim.status()["bond_steps"]
    e2e_ms, e2e_bond_steps = aggregate_over_ranks(e2e_s * 1e3, float(s1 - s0), dist)
    e2e = {"value": e2e_bond_steps / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": int(host_v0.numel() * 4 / args.steps),
           "d2h_bytes_per_step": int(host_u.numel() * 4)}

    # ---- CPU baseline (oracle, host cores, bounded sample) ----
    cpu = None
    oracle_state = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, threads, desc, single, oracle_state = oracle_sample()
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
               "single_thread": {"value": single, "unit": UNIT, "cores": 1}}

    # ---- the mixed path's error against FP64, per result ----
    precision = None
    if rank == 0 and not args.no_precision:
        precision = precision_report(cfg, tile, u_timed, steps_timed_run, oracle_state)

    # HBM GB/s of both paths: algorithmic bytes per step x steps per second,
    # and the bond kernel's profiled DRAM bytes over its event-timed launch
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    b_mixed = algorithmic_bytes(nb, n, True)
    b_fp64 = algorithmic_bytes(nb, n, False)
    traffic = roofline["traffic"]
    hbm = {"unit": "GB/s", "peak": hbm_peak, "peak_kind": peak_kind,
           "mixed": {"bytes_per_step": b_mixed, "gbs": b_mixed * (value / world / nb) / 1e9,
                     "bond_kernel_algorithmic_gbs": bond_kernel_bytes(nb, n) / (bond_ms * 1e-3) / 1e9,
                     "bond_kernel_dram_gbs": traffic / (bond_ms * 1e-3) / 1e9 if traffic else None},
           "fp64": {"bytes_per_step": b_fp64, "gbs": b_fp64 * (fp64_rate / nb) / 1e9},
           "note": "the path is FP32-issue-bound (roofline above); these are far below the HBM roof"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "points": n, "bonds": nb, "dx": cfg["dx"],
                       "horizon": "3.015 dx", "rebuild_every": cfg["rebuild_every"],
                       "l2": "inputs larger than L2 (force states + family > 129 MB)",
                       "timed_region": "starts at a family rebuild: ceil(steps / rebuild_every) "
                                       "family searches inside",
                       "rebuilds_timed": fig["rebuilds"],
                       "bond_launch_shape": shape,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "fp64_path": {"value": fp64_rate, "unit": UNIT, "steps": args.fp64_steps},
            "mixed_over_fp64": value / world / fp64_rate if fp64_rate > 0 else None,
            "hbm": hbm, "precision": precision, "standard_model": standard, "other_modes": other_modes,
            "uniaxial_compression": uniaxial,
            "collapse_runout": runout,
            "critical_time_step": critical,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "ensemble": ens,
            "large": large, "adjoint": adj,
            "clocks": clocks, "gpu_launches": fig["launches"],
            "status": dict({k: st[k] for k in ("plastic", "nonconv", "singular", "flags", "unstable_step")},
                           eq69_residual_over_max_at_end=eq69_ratio(st)),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
