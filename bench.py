#!/usr/bin/env python3
"""Throughput of the parallel VC-SGC transmutation sweep on one GB300.

Workload: rigid BCC 80x80x80 cells (1,024,000 sites), EAM tabulated on
5000-point grids, 2% B placed at random, T = 600 K, kappa = 1000 (units of
kB T / N), phi scanned over 8 values across the two-phase region -- the 8
phi values run as 8 replicas of one context.  Every colour of the period-4
sublattice schedule trials all its 8,000 sites at once (128 colours).
A step is one sweep of every replica: 8 x 1,024,000 trial moves.

python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Prints one JSON line.  Under torchrun each rank runs its own replicas (the
method does not shard: replicas only) and rank 0 reports the aggregate.
"""
from __future__ import annotations

import argparse
import ctypes
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

from paper_1012_5082_gb300 import inputs as I  # noqa: E402
from paper_1012_5082_gb300 import recipe as RC  # noqa: E402

CELLS = 80
T_K = 600.0
KAPPA = 1000.0
N_PHI = 8
FRAC_B = 0.02
# Parameter recipe (Sec. III C): dmu0 = dmu_S, the driving force at two-phase
# coexistence from kappa = 0 SGC runs of a small lattice (both single-phase
# branches integrated to their crossing), and phi_j = dmu0 - 2 kappa_p N c0_j.
PRESCAN_GRID = np.round(np.arange(-1.85, -1.2499, 0.05), 4)  # eV, 13 points around the crossing
PRESCAN_CELLS, PRESCAN_WARMUP, PRESCAN_SWEEPS = 16, 200, 400
# Algorithmic work of one trial of the fused colour step, by pipe (from the
# source; the compile-time five-shell table holds 33 non-empty (row, shell)
# masks, 25 of them with more than one site):
#   simple integer ops: Philox 60 (4 xor + 2 key adds per round), site decode
#     15, 13 rows x (two effective-species words 3 + 3, funnel shift 1, row
#     address 2) 117, one-bit masks 8 x 2, multi-bit masks 25 x (and, add) 50,
#     own bit 3 -> 261
#   popc: 25;  32-bit multiply pairs (mul.hi + mul.lo): Philox 20
#   FP32: the local exponent, its bound and the screen 20;  MUFU: expf 1
OPS_SIMPLE, OPS_POPC, OPS_MULPAIR, OPS_FP32, OPS_MUFU = 261, 25, 20, 20, 1
OPS_PER_TRIAL = OPS_SIMPLE + OPS_POPC + 2 * OPS_MULPAIR + OPS_FP32 + OPS_MUFU
# Per-SM rates measured on GB300 (per clock): INT32 xor+add 120, popc 20.7,
# multiply pairs 31, FP32 FMA 122, expf 11.3.  Integer ops and popc share
# the ALU pipe; multiplies, FP32 and MUFU run on other pipes in parallel, so
# the floor of a trial is the ALU pipe's time (the larger of the two).
SM_CYCLES_PER_TRIAL = max(OPS_SIMPLE / 120.0 + OPS_POPC / 20.7,
                          OPS_MULPAIR / 31.0 + OPS_FP32 / 122.0 + OPS_MUFU / 11.3)
ALU_PEAK_OPS = OPS_PER_TRIAL * 152 * 2.07e9 / SM_CYCLES_PER_TRIAL
# Nominal HBM bytes of a trial of the gather form over an explicit int32
# neighbour list (58 x 4 B list, own species 1 B, own rho 8 B, species write
# 1 B): the kernels here read no list (bit-packed rows resident on chip)
HBM_BYTES_PER_TRIAL = 242
# a chain of dependent step-shaped launches with programmatic dependent launch
STEP_LATENCY_FLOOR_US = 1.29
METRIC = "VC-SGC trial moves/s"


def c0_grid():
    return 0.02 + np.arange(N_PHI) * 0.48 / 7


def workload(dmu0):
    """The headline lattice, its random 2 % start and the 8 replicas' phi for
    the driving force dmu0 (eV)."""
    lat = I.bcc_lattice(CELLS, CELLS, CELLS)
    types = I.random_types(lat.n, int(round(FRAC_B * lat.n)), seed=1001)
    tab = I.eam_tables()
    c0 = c0_grid()
    return lat, types, tab, RC.phi_grid(dmu0, KAPPA, T_K, c0), c0


def prescan(V, stream, local):
    """Sec. III C (i): dmu_S from kappa = 0 SGC runs of 16^3 lattices started
    in pure A and pure B at each driving force of PRESCAN_GRID."""
    t0 = time.perf_counter()
    c_a, c_b, e_a, e_b = RC.sgc_branches(V, T_K, PRESCAN_GRID, cells=PRESCAN_CELLS, warmup=PRESCAN_WARMUP,
                                         sweeps=PRESCAN_SWEEPS, stream=stream, device=local)
    dmu_s = RC.coexistence(PRESCAN_GRID, c_a, c_b, e_a, e_b)
    return {"dmu_S_eV": dmu_s, "grid_eV": PRESCAN_GRID.tolist(), "c_A_branch": [float(x) for x in c_a],
            "c_B_branch": [float(x) for x in c_b], "e_A_eV": e_a, "e_B_eV": e_b,
            "lattice": f"{PRESCAN_CELLS}^3 BCC, kappa 0, T 600 K, {PRESCAN_WARMUP} + {PRESCAN_SWEEPS} sweeps",
            "seconds": time.perf_counter() - t0}


def _recipe_point(pre, dmu_s, sweeps, trials_per_step, ms, reps):
    return {"prescan": pre,
            "recipe_dmu_S": {"dmu0_eV": dmu_s,
                             "label": "dmu0 = dmu_S, the two-phase coexistence value of steps (i) and (iii) of "
                                      "Sec. III C, on the same supersaturated start", "sweeps": sweeps,
                             "trial_moves_per_s": trials_per_step * sweeps / (ms * 1e-3), "replicas": reps,
                             "accepted_flips_per_s": sum(x["accepted_flips_per_s"] for x in reps)}}


def balanced_dmu(V, stream, local):
    """The driving force at which the first composite move of the random 2 %
    start has no expected drift (recipe.balanced_dmu0 on the dE of every
    site, evaluated by the library)."""
    lat = I.bcc_lattice(CELLS, CELLS, CELLS)
    types = I.random_types(lat.n, int(round(FRAC_B * lat.n)), seed=1001)
    ctx = V.Context(lat, types, I.eam_tables(), -2.0, KAPPA, T_K, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4),
                    stream=stream, device=local)
    de = ctx.delta_e(np.arange(lat.n))
    ctx.close()
    return RC.balanced_dmu0(de, types, T_K)


def config_dict(extra=None):
    d = {"workload": f"rigid BCC {CELLS}^3 cells (1,024,000 sites), EAM 5000-pt tables, "
                     f"2% B, T=600 K, kappa=1000, {N_PHI} phi values as replicas (c0 = 0.02 .. 0.5, "
                     "phi = dmu0 - 2 kappa kB T c0, dmu0 balanced on the random start), "
                     "period-4 sublattice schedule (8,000 trials per colour step)",
         "sites": 2 * CELLS ** 3, "replicas": N_PHI, "trials_per_step": N_PHI * 2 * CELLS ** 3,
         "l2_policy": "L2 flushed between timed sweeps (a 256 MB write on the stream, outside the timed "
                      "intervals); within a sweep the 2.5 MB bit-packed state stays L2-resident"}
    if extra:
        d.update(extra)
    return d


class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def cpu_baseline(lat, types, tab, phi, c0, budget_s=12.0):
    """The oracle, as it stands, on one host core: one replica of the same
    workload, sweeps of the same schedule, about budget_s seconds."""
    import oracle as O

    s = O.System(lat, types, tab)
    s.set_params(float(phi[0]), KAPPA, T_K, c0=float(c0[0]), seed=2001)
    s.schedule_sublattice(lat.cells, (4, 4, 4))
    t0 = time.perf_counter()
    s.parallel_steps(4)
    dt = time.perf_counter() - t0
    n_steps = max(4, int(budget_s / max(dt / 4, 1e-6)))
    t0 = time.perf_counter()
    s.parallel_steps(n_steps)
    dt = time.perf_counter() - t0
    trials = s.obs()["trials"]
    per_step = lat.n // 128
    done = n_steps * per_step
    return {"value": done / dt, "unit": "trial moves/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_steps} colour steps ({done} trial moves, {done / lat.n:.2f} sweeps) of "
                      f"replica 0 of the 80^3 workload, serial FP64 C oracle, {dt:.1f} s",
            "trials_counted": int(trials)}


def md_bench(V, torch, stream, local, steps=20, warmup=3, box=250.0, precision=0):
    """MD atom-steps/s of the hybrid scheme's MD half on the nanocrystal
    workload: 25 nm periodic cube, 16 Voronoi grains of BCC (a = 2.855 A)
    with random centres and orientations, overlaps within 2.0 A removed,
    1% B, Langevin BAOAB at 700 K, dt = 2 fs, FP64; plus one hybrid cycle
    (20 MD steps, then 0.1 N trial moves on the frozen positions)."""
    t0 = time.perf_counter()
    lat = I.nanocrystal(box, 16, seed=1002)
    gen_s = time.perf_counter() - t0
    types = I.random_types(lat.n, int(round(0.01 * lat.n)), seed=1003)
    v = I.maxwell_velocities(types, 700.0, seed=1004)
    tab = I.eam_tables()
    nb = 2 * int(box // 22.0)  # even box count, boxes wider than 2 r_c = 10.6 A
    ctx = V.Context(lat, types, tab, -1.0, KAPPA, 700.0, c0=0.01, schedule=V.SCHED_SPATIAL,
                    sched=(nb, nb, nb, 2, 2, 2), dt=2.0, gamma=0.01, T_md=700.0, stream=stream,
                    device=local, precision=precision)
    ctx.set_velocities(v)
    ctx.md_steps(warmup)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.md_steps(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    n_mc = max(1, int(round(0.1 * lat.n / (nb ** 3 // 8))))  # 0.1 N trial moves
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.hybrid(1, 20, n_mc)
    torch.cuda.synchronize()
    cyc = time.perf_counter() - t0
    o = ctx.observables()
    ctx.close()
    return {"metric": "MD atom-steps/s", "value": lat.n * steps / (ms * 1e-3), "unit": "atom-steps/s",
            "atoms": lat.n, "steps": steps, "ms_per_step": ms / steps,
            "dtype": "f64" if precision == 0 else "f32 tables, f64 sums",
            "workload": "nanocrystal 25 nm, 16 grains, 1% B, Langevin 700 K, dt 2 fs",
            "hybrid_cycle_s": cyc, "hybrid_mc_trials": int(o["trials"]),
            "generate_s": gen_s}


def mc_explicit_bench(V, torch, stream, local, dmu0, steps=256, warmup=16, box=250.0):
    """The MC phase of the hybrid scheme (Sec. IV A) alone: colour steps of the
    general per-pair form on the explicit positions of the 25 nm nanocrystal
    (1% B, T = 700 K, kappa = 1000, SPATIAL boxes of more than 2 r_c in 2 x 2
    x 2 colours, one trial per box per step), FP64 and mixed precision, with
    the mixed form's dE error against the FP64 form on the same state."""
    lat = I.nanocrystal(box, 16, seed=1002)
    types = I.random_types(lat.n, int(round(0.01 * lat.n)), seed=1003)
    tab = I.eam_tables()
    nb = 2 * int(box // 22.0)
    phi = float(RC.phi_grid(dmu0, KAPPA, 700.0, 0.01))
    out = {"workload": f"nanocrystal 25 nm ({lat.n} atoms), 1% B, 700 K, kappa 1000, {nb}^3 boxes in 8 colours"}
    hbm, src = measured_peak_hbm()
    ctxs = {}
    for name, prec in (("fp64", V.PREC_FP64), ("mixed", V.PREC_MIXED)):
        ctx = V.Context(lat, types, tab, phi, KAPPA, 700.0, c0=0.01, schedule=V.SCHED_SPATIAL,
                        sched=(nb, nb, nb, 2, 2, 2), stream=stream, device=local, precision=prec)
        ctx.steps(warmup)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        o0 = ctx.observables()
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.steps(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        o1 = ctx.observables()
        trials = o1["trials"] - o0["trials"]
        v = trials / (ms * 1e-3)
        out[name] = {"trial_moves_per_s": v, "us_per_step": ms * 1e3 / steps, "trials_per_step": trials // steps,
                     "acc_local": (o1["local_accepts"] - o0["local_accepts"]) / max(1, trials),
                     "hbm_nominal": {"bytes_per_trial": HBM_BYTES_PER_TRIAL, "frac": HBM_BYTES_PER_TRIAL * v / 1e9 / hbm,
                                     "peak_gbs": hbm, "peak_source": src}}
        ctxs[name] = ctx
    t = ctxs["fp64"].types()
    ctxs["mixed"].set_types(t)
    sites = np.random.default_rng(8).choice(lat.n, 20000, replace=False)
    err = np.abs(ctxs["mixed"].delta_e(sites) - ctxs["fp64"].delta_e(sites))
    out["mixed_dE_error_vs_fp64"] = {"max_eV": float(err.max()), "rms_eV": float(np.sqrt(np.mean(err ** 2))),
                                     "sampled_sites": int(len(sites))}
    out["speedup_mixed_vs_fp64"] = out["mixed"]["trial_moves_per_s"] / out["fp64"]["trial_moves_per_s"]
    for ctx in ctxs.values():
        ctx.close()
    return out


def ensemble_bench(V, torch, stream, local, steps=20, box=250.0, cg_iters=100):
    """The paper's MD ensemble (Sec. IV B) on the 25 nm nanocrystal: CG
    pre-relaxation (Polak-Ribiere, a fixed budget of iterations), then
    Nose-Hoover NVT and MTK NPT MD steps at 700 K, dt 2 fs, FP64.  The EAM is
    the synthetic one with the rho^2 embedding coefficient that puts the BCC
    crystal at zero pressure at a = 2.855 A (the workloads' coefficient
    leaves it at about -880 kbar, where a barostat collapses the cell)."""
    lat = I.nanocrystal(box, 16, seed=1002)
    types = I.random_types(lat.n, int(round(0.01 * lat.n)), seed=1003)
    tab = I.eam_tables(I.npt_eam_params())
    nb = 2 * int(box // 22.0)
    ctx = V.Context(lat, types, tab, -1.0, KAPPA, 700.0, c0=0.01, schedule=V.SCHED_SPATIAL,
                    sched=(nb, nb, nb, 2, 2, 2), dt=2.0, gamma=0.0, T_md=700.0, stream=stream, device=local)
    e_start = ctx.energy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cg = ctx.minimize(ftol=1e-3, max_iter=cg_iters)
    torch.cuda.synchronize()
    cg_s = time.perf_counter() - t0
    e_relaxed = ctx.energy()
    ctx.set_velocities(I.maxwell_velocities(types, 700.0, seed=1004))
    out = {"workload": "nanocrystal 25 nm, 16 grains, 1% B, zero-pressure EAM, 700 K, dt 2 fs",
           "atoms": lat.n,
           "cg": {"iterations": cg["iterations"], "fmax_eV_per_A": cg["fmax"], "seconds": cg_s,
                  "energy_drop_eV_per_atom": (e_start - e_relaxed) / lat.n}}
    for kind, kw in (("nvt", dict(t_damp=100.0)), ("npt", dict(t_damp=100.0, p_damp=1000.0, p_ext_bar=0.0))):
        ctx.set_ensemble(kind, **kw)
        ctx.md_steps(3)
        s0 = ctx.ensemble_state()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.md_steps(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        s1 = ctx.ensemble_state()
        out[kind] = {"atom_steps_per_s": lat.n * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                     "temperature_K": s1["temperature"], "pressure_bar": s1["pressure_bar"],
                     "conserved_change_eV_per_atom": (s1["conserved"] - s0["conserved"]) / lat.n,
                     "box_A": s1["lx"]}
    ctx.close()
    return out


def mixed_bench(V, torch, stream, local, dmu0, sweeps=40, warmup=3):
    """The mixed-precision form on the 128^3 rigid lattice (4,194,304 sites) x
    8 phi replicas, timed beside the FP64 form on the same workload, with the
    error of the mixed form: per-trial dE (max, rms) over sampled sites on the
    same species, energy per atom, and each chain's mean concentration."""
    cells = 128
    lat = I.bcc_lattice(cells, cells, cells)
    types = I.random_types(lat.n, int(round(FRAC_B * lat.n)), seed=1003)
    tab = I.eam_tables()
    c0 = c0_grid()
    phi = RC.phi_grid(dmu0, KAPPA, T_K, c0)
    seeds = np.arange(N_PHI, dtype=np.uint64) + np.uint64(4001)
    out = {"workload": f"rigid BCC {cells}^3 cells ({lat.n} sites) x {N_PHI} phi replicas, "
                       "period-4 sublattice, T=600 K, kappa=1000"}
    ctxs = {}
    for name, prec in (("fp64", V.PREC_FP64), ("mixed", V.PREC_MIXED)):
        ctx = V.Context(lat, np.tile(types, N_PHI), tab, 0.0, KAPPA, T_K, schedule=V.SCHED_SUBLATTICE,
                        sched=(4, 4, 4), n_replicas=N_PHI, phi_r=phi, c0_r=c0, seed_r=seeds,
                        stream=stream, device=local, precision=prec)
        ctx.sweep(warmup)
        ms = timed_sweeps(torch, stream, ctx, sweeps)
        out[name] = {"value": N_PHI * lat.n * sweeps / (ms * 1e-3), "unit": "trial moves/s",
                     "ms_per_sweep": ms / sweeps,
                     "mean_c": [ctx.observables(r)["mean_c"] for r in range(N_PHI)]}
        ctxs[name] = ctx
    # errors on common species (those of the FP64 chain)
    t = ctxs["fp64"].types(0)
    ctxs["mixed"].set_types(t, 0)
    rng = np.random.default_rng(7)
    sites = rng.choice(lat.n, 200000, replace=False)
    d64 = ctxs["fp64"].delta_e(sites, 0)
    d32 = ctxs["mixed"].delta_e(sites, 0)
    err = np.abs(d32 - d64)
    e64 = ctxs["fp64"].energy(0) / lat.n
    e32 = ctxs["mixed"].energy(0) / lat.n
    dc = np.abs(np.array(out["mixed"]["mean_c"]) - np.array(out["fp64"]["mean_c"]))
    out["error_vs_fp64"] = {"dE_max_eV": float(err.max()), "dE_rms_eV": float(np.sqrt(np.mean(err ** 2))),
                            "energy_per_atom_eV": abs(e32 - e64), "mean_c_abs_max": float(dc.max()),
                            "sampled_sites": int(len(sites))}
    out["speedup_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    for ctx in ctxs.values():
        ctx.close()
    return out


def c4_grid(dmu0):
    """(phi, T, c0) of the 64 replicas: 8 temperatures in 500-900 K x 8
    concentrations c0 = 0.02 .. 0.5 with the same local driving force."""
    phi, T, c0 = [], [], []
    for r in range(64):
        Tr = 500.0 + 400.0 * (r // 8) / 7.0
        c0r = 0.02 + (r % 8) * 0.48 / 7
        T.append(Tr)
        c0.append(c0r)
        phi.append(float(RC.phi_grid(dmu0, KAPPA, Tr, c0r)))
    return phi, T, c0


def c4_batch(V, stream, local, tab, dmu0):
    cells, types = [], []
    for r in range(64):
        L = 24 + 4 * (r % 7)
        n = 2 * L ** 3
        cells.append((L, L, L))
        types.append(I.random_types(n, int(round(FRAC_B * n)), seed=3000 + r))
    phi, T, c0 = c4_grid(dmu0)
    return V.Batch(cells, types, tab, phi, KAPPA, T, c0_r=c0,
                   seed_r=np.arange(64, dtype=np.uint64) + np.uint64(3000), stream=stream, device=local)


class L2Flush:
    """A buffer twice the 129 MB L2, written on the stream between timed
    sweeps so that no sweep starts with the previous one's cache contents."""

    def __init__(self, torch, device):
        self.buf = torch.empty(256 << 20, dtype=torch.uint8, device=device)
        self.k = 0

    def __call__(self, torch, stream):
        self.k = (self.k + 1) & 255
        with torch.cuda.stream(stream):
            self.buf.fill_(self.k)


def timed_sweeps(torch, stream, b, sweeps, flush=None):
    """Device time (ms) of `sweeps` sweeps, each between its own pair of
    events on the stream, L2 flushed before each (outside the events)."""
    flush = flush or L2Flush(torch, torch.cuda.current_device())
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(sweeps)]
    torch.cuda.synchronize()
    for a, z in ev:
        flush(torch, stream)
        a.record(stream)
        b.sweep(1)
        z.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(z) for a, z in ev)


def batch_bench(V, torch, stream, local, dmu0, sweeps=30, warmup=3, surrogate=True):
    """64 replicas of rigid BCC of uneven sizes (L = 24 + 4 (r mod 7) cells,
    27,648 to 221,184 sites) at 8 temperatures in 500-900 K x 8 phi values,
    kappa = 1000, advanced together by one fused launch per colour step
    (CUDA graphs of 64 steps); block size picked by the autotuner.  With
    surrogate: the same run with delayed acceptance by a network trained on
    the sampler's own dE."""
    tab = I.eam_tables()
    b = c4_batch(V, stream, local, tab, dmu0)
    best = b.autotune(steps=64)
    b.sweep(warmup)
    ms = timed_sweeps(torch, stream, b, sweeps)
    total = sum(b.sizes)
    obs = [b.observables(r) for r in range(64)]
    b.close()
    out = {"metric": "aggregate VC-SGC trial moves/s", "value": total * sweeps / (ms * 1e-3),
           "unit": "trial moves/s", "replicas": 64, "sites_total": total, "sweeps": sweeps,
           "ms_per_sweep": ms / sweeps, "block": best,
           "acc_local_sample": [obs[r]["acc_local"] for r in (0, 31, 63)],
           "workload": "64 replicas, L = 24..48 cells, T 500-900 K x 8 phi, kappa 1000, FP64"}
    if surrogate:
        out["delayed_acceptance"] = surrogate_bench(V, torch, stream, local, tab, dmu0, sweeps, warmup, out["value"],
                                                    obs)
    return out


def surrogate_bench(V, torch, stream, local, tab, dmu0, sweeps, warmup, plain_value, plain_obs,
                    n_samples=10_000_000, train_steps=5000, batch=4096, lr=2e-3):
    """Form (4): (descriptor, dE) samples drawn by the sampler itself on 12^3
    replicas of the 10^3 parity workload's EAM at the 64 (phi, T) points,
    training by the GPU kernels, then the 64-replica batch with the network
    as stage 1 of delayed acceptance."""
    phi, T, c0 = c4_grid(dmu0)
    lat = I.bcc_lattice(12, 12, 12)
    types = [I.random_types(lat.n, int(round(c * lat.n)), seed=5000 + r) for r, c in enumerate(c0)]
    gen = V.Batch([(12, 12, 12)] * 64, types, tab, phi, KAPPA, T, c0_r=c0,
                  seed_r=np.arange(64, dtype=np.uint64) + np.uint64(5000), stream=stream, device=local)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xs, Ys, got = [], [], 0
    gen.sweep(4)
    while got < n_samples:
        gen.sweep(2)
        X, Y = gen.features()
        Xs.append(X)
        Ys.append(Y)
        got += X.shape[0]
    X, Y = torch.cat(Xs), torch.cat(Ys)
    del Xs, Ys
    gen.sweep(5)
    Xh, Yh = gen.features()
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    gen.close()
    s = V.Surrogate(I.mlp_init(7, out_bias=float(Y.mean())), stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = s.train(X, Y, batch=batch, steps=train_steps, lr=lr, seed=17)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    g = s.forward(Xh)
    rmse = float(torch.sqrt(((g - Yh) ** 2).mean()))
    b = c4_batch(V, stream, local, tab, dmu0)
    b.set_surrogate(s)
    best = b.autotune(steps=64)
    b.sweep(warmup)
    ms = timed_sweeps(torch, stream, b, sweeps)
    total = sum(b.sizes)
    obs = [b.observables(r) for r in range(64)]
    b.close()
    s.close()
    trials = sum(o["trials"] for o in obs)
    s1 = sum(o["stage1_accepts"] for o in obs)
    acc = sum(o["local_accepts"] for o in obs)
    value = total * sweeps / (ms * 1e-3)
    dc = [abs(obs[r]["mean_c"] - plain_obs[r]["mean_c"]) for r in range(64)]
    return {"value": value, "unit": "trial moves/s", "speedup_vs_plain": value / plain_value,
            "block": best, "stage1_rejection": 1.0 - s1 / trials, "stage2_acceptance": acc / max(1, s1),
            "train_samples": int(X.shape[0]), "sample_gen_s": t_gen, "train_steps": train_steps,
            "train_batch": batch, "train_s": t_train, "train_samples_per_s": train_steps * batch / t_train,
            "loss_first": float(np.mean(hist[:10])), "loss_last": float(np.mean(hist[-100:])),
            "holdout_rmse_eV": rmse, "holdout_std_eV": float(Yh.std()),
            "mean_c_abs_diff_vs_plain": {"mean": float(np.mean(dc)), "max": float(np.max(dc))},
            "network": "10-64-64-1 SiLU, BF16 mma.sync m16n8k16, FP32 accumulate; Adam"}


def ising_bench(V, torch, stream, local, sweeps=30, warmup=3):
    """The Ising-type lattice gas of Sec. II B (BCC, pair interactions to the
    second shell, eps_AA(1) = eps_BB(1) = -10 U, eps_AB(1) = -9.7 U, eps(2) =
    -2 U, U = 0.1 eV, k_B T = 0.8617 U) through the same kernels: throughput on
    80^3 x 8 replicas at c0 = 1/2, and the parallel method's acceptance in the
    paper's set-up (40^3 cells, 64 domains of 10^3 cells in octants, one trial
    per domain per step) against kappa at c0 = 1/2, dmu0 = 0."""
    tab = I.ising_tables()
    T = 1000.0
    kT = I.KB_EV * T
    out = {"workload": "Ising-type lattice gas, BCC, eps(1) -10/-9.7/-10 U, eps(2) -2 U, U = 0.1 eV, T = 1000 K"}
    lat = I.bcc_lattice(CELLS, CELLS, CELLS)
    types = I.random_types(lat.n, lat.n // 2, seed=6001)
    kappa = 100.0
    ctx = V.Context(lat, np.tile(types, N_PHI), tab, -kappa * kT, kappa, T, schedule=V.SCHED_SUBLATTICE,
                    sched=(4, 4, 4), n_replicas=N_PHI, c0=0.5,
                    seed_r=np.arange(N_PHI, dtype=np.uint64) + np.uint64(6001), stream=stream, device=local)
    ctx.sweep(warmup)
    ms = timed_sweeps(torch, stream, ctx, sweeps)
    out["throughput"] = {"value": N_PHI * lat.n * sweeps / (ms * 1e-3), "unit": "trial moves/s",
                         "config": f"{CELLS}^3 x {N_PHI} replicas, period-4 sublattice, c0 = 0.5, kappa = 100"}
    ctx.close()
    lat = I.bcc_lattice(40, 40, 40)
    acc = {}
    for kappa in (10.0, 100.0, 1000.0):
        ctx = V.Context(lat, I.random_types(lat.n, lat.n // 2, seed=6101), tab, -kappa * kT, kappa, T,
                        schedule=V.SCHED_BLOCKS, sched=(5, 5, 5, 2, 2, 2), c0=0.5, seed=6102,
                        stream=stream, device=local)
        ctx.sweep(20)
        o0 = ctx.observables()
        ctx.sweep(30)
        o1 = ctx.observables()
        acc[str(kappa)] = (o1["flips"] - o0["flips"]) / (o1["trials"] - o0["trials"])
        ctx.close()
    out["acceptance_parallel_64_domains"] = acc
    # dmu(c) = phi + 2 kappa_p N <c> at dmu0 = 0 across the gap: the finite
    # system's van der Waals loop (16^3 cells, kappa = 1000, 4 replicas per c0)
    kappa, L, S = 1000.0, 16, 4
    c0s = np.round(np.arange(1, 13) * 0.04 + 0.02, 2)
    c0r = np.repeat(c0s, S)
    lat = I.bcc_lattice(L, L, L)
    types = [I.random_types(lat.n, int(round(c * lat.n)), seed=6200 + q) for q, c in enumerate(c0r)]
    b = V.Batch([(L, L, L)] * len(c0r), types, tab, -2.0 * kappa * kT * c0r, kappa, T,
                seed_r=np.arange(len(c0r), dtype=np.uint64) + 6300, c0_r=c0r, stream=stream, device=local)
    b.sweep(500)
    s0 = b.observables_all()
    b.sweep(1000)
    s1 = b.observables_all()
    b.close()
    c = np.array([(s1[q]["mean_c"] * s1[q]["steps"] - s0[q]["mean_c"] * s0[q]["steps"])
                  / (s1[q]["steps"] - s0[q]["steps"]) for q in range(len(c0r))]).reshape(-1, S)
    dmu = 2.0 * kappa * kT * (c - c0s[:, None])
    out["dmu_of_c_meV"] = {f"{x:.2f}": round(float(v) * 1e3, 3) for x, v in zip(c0s, dmu.mean(axis=1))}
    out["paper_max_acceptance"] = {"parallel": 0.34, "serial": 0.47, "c": 0.5}
    return out


def overlap_bench(V, torch, stream, local, dmu0, sweeps=4, warmup=1):
    """Overlapping, position-weighted domains (Sec. III A) against the plain
    octants on the same cells of the headline lattice (80^3 x 8 replicas,
    the same phi and c0, 2% B start): cells of 10^3 lattice cells, octants =
    blocks of 5^3 in 2x2x2 colours, overlapping = domains of 6^3 with gap 4
    (13.0 A > 2 r_c); one trial per cell per colour step (512 per replica).
    Reports throughput and replica 0's energy per atom after 2, 5, 10 and 20
    sweeps from the supersaturated start (the relaxation the larger trial
    volume is meant to speed up), with the period-4 sublattice beside them."""
    lat, types, tab, phi, c0 = workload(dmu0)
    seeds = np.arange(N_PHI, dtype=np.uint64) + np.uint64(7001)
    out = {"workload": "80^3 x 8 replicas, headline phi/c0, cells of 10^3 lattice cells"}
    for name, kind, sched in (("octants", V.SCHED_BLOCKS, (5, 5, 5, 2, 2, 2)),
                              ("overlapping", V.SCHED_OVERLAP, (10, 10, 10, 4, 4, 4)),
                              ("sublattice", V.SCHED_SUBLATTICE, (4, 4, 4))):
        ctx = V.Context(lat, np.tile(types, N_PHI), tab, 0.0, KAPPA, T_K, schedule=kind, sched=sched,
                        n_replicas=N_PHI, phi_r=phi, c0_r=c0, seed_r=seeds, stream=stream, device=local)
        # replica 0 (c0 = the starting 2 %): energy per atom as the
        # supersaturated start relaxes
        e = {"0": ctx.observables(0)["energy_per_atom"]}
        done = 0
        for k in (2, 5, 10, 20):
            ctx.sweep(k - done)
            done = k
            e[str(k)] = ctx.observables(0)["energy_per_atom"]
        ctx.sweep(warmup)
        ms = timed_sweeps(torch, stream, ctx, sweeps)
        out[name] = {"trial_moves_per_s": N_PHI * lat.n * sweeps / (ms * 1e-3),
                     "trials_per_step": N_PHI * (lat.n // ctx.steps_per_sweep),
                     "us_per_step": ms * 1e3 / (sweeps * ctx.steps_per_sweep),
                     "energy_per_atom_after_sweeps": e}
        ctx.close()
    return out


def multi_bench(V, torch, stream, local, sweeps=10, warmup=2):
    """Multicomponent colour step: 80^3 x 8 replicas, period-4 sublattice,
    K = 3 (one density function) and K = 4 (species-dependent densities,
    re-embedding), 5% of each solute at random, T = 1200 K, kappa = 10."""
    lat = I.bcc_lattice(CELLS, CELLS, CELLS)
    out = {}
    # phi per solute: the local driving forces at which the expected dn of
    # every solute vanishes on the random start (solved once from the dE of
    # every site to every target species), minus 2 kappa kB T c0
    for K, ds, ph in ((3, None, [-1.928, -1.628]), (4, (1.0, 1.25, 0.85, 1.1), [-1.173, -2.037, 0.567])):
        tab = I.eam_tables(I.multi_eam_params(K, dens_scale=ds))
        t = np.stack([I.multi_random_types(lat.n, [int(0.05 * lat.n)] * (K - 1), seed=8000 + r)
                      for r in range(N_PHI)])
        g = V.Multi(lat, t, tab, ph, 10.0, 1200.0, c0=0.05,
                    seed_r=np.arange(N_PHI, dtype=np.uint64) + np.uint64(8100), stream=stream, device=local)
        g.sweep(warmup)
        ms = timed_sweeps(torch, stream, g, sweeps)
        o = g.observables(0)
        out[f"K{K}"] = {"trial_moves_per_s": N_PHI * lat.n * sweeps / (ms * 1e-3),
                        "us_per_step": ms * 1e3 / (sweeps * g.steps_per_sweep),
                        "reembed": ds is not None, "acc_local": o["acc_local"], "acc_global": o["acc_global"],
                        "launches_per_step": 2 if ds is not None else 1}
        g.close()
    # binary with species-dependent densities (f_B = 1.25 f_A), one chain two
    # ways: the binary context's screened re-embedding step (two launches,
    # neighbour lists) and the multicomponent context's with K = 2
    tab = I.eam_tables(I.multi_eam_params(2, dens_scale=(1.0, 1.25)))
    t = np.stack([I.random_types(lat.n, int(0.05 * lat.n), seed=8200 + r) for r in range(N_PHI)])
    seeds = np.arange(N_PHI, dtype=np.uint64) + np.uint64(8300)
    phi_b, kappa_b, T_b, c0_b = -2.2, 100.0, 1200.0, 0.05
    g = V.Multi(lat, t, tab, [phi_b], kappa_b, T_b, c0=c0_b, seed_r=seeds, stream=stream, device=local)
    b = V.Context(lat, t.reshape(-1), tab, phi_b, kappa_b, T_b, schedule=V.SCHED_SUBLATTICE, sched=(4, 4, 4),
                  n_replicas=N_PHI, phi_r=np.full(N_PHI, phi_b), c0_r=np.full(N_PHI, c0_b), seed_r=seeds,
                  stream=stream, device=local)
    res = {}
    for name, obj, sw in (("screened_K2", g, sweeps), ("binary_context", b, sweeps)):
        obj.sweep(warmup)
        ms = timed_sweeps(torch, stream, obj, sw)
        res[name] = {"trial_moves_per_s": N_PHI * lat.n * sw / (ms * 1e-3),
                     "us_per_step": ms * 1e3 / (sw * obj.steps_per_sweep)}
    res["acc_local"] = g.observables(0)["acc_local"]
    g.close()
    b.close()
    out["binary_reembedding"] = res
    out["workload"] = "80^3 x 8 replicas, period-4 sublattice (64,000 trials per colour step)"
    return out


def reembed_da_bench(V, torch, stream, local, sweeps=10, equil=400, train_steps=3000, batch=4096, lr=2e-3):
    """Delayed acceptance on the re-embedding workload (80^3 x 8 replicas,
    f_B = 1.25 f_A, phi = -2.2 eV, kappa = 100, 1200 K, c0 = 5 %, period-4
    sublattice; the binary context runs the two-species multicomponent
    kernels).  The plain rule takes the chains from the random start through
    `equil` sweeps; a surrogate is trained on the descriptors and exact
    targets of that state; then the plain rule and delayed acceptance are
    timed from the same state.  Reports the step time of each, the trial
    moves and accepted flips per second, the stage-1 pass and stage-2
    acceptance fractions, and the energy per atom along the equilibration."""
    lat = I.bcc_lattice(CELLS, CELLS, CELLS)
    tab = I.eam_tables(I.multi_eam_params(2, dens_scale=(1.0, 1.25)))
    t = np.stack([I.random_types(lat.n, int(0.05 * lat.n), seed=8200 + r) for r in range(N_PHI)])
    seeds = np.arange(N_PHI, dtype=np.uint64) + np.uint64(8300)
    g = V.Context(lat, t.reshape(-1), tab, -2.2, 100.0, 1200.0, c0=0.05, schedule=V.SCHED_SUBLATTICE,
                  sched=(4, 4, 4), n_replicas=N_PHI, seed_r=seeds, stream=stream, device=local)

    def mean_obs():
        o = [g.observables(r) for r in range(N_PHI)]
        return o, float(np.mean([q["energy_per_atom"] for q in o])), float(np.mean([q["c"] for q in o]))

    trace, done = [], 0
    for k in sorted({k for k in (0, 50, 100, 200, equil // 2, equil) if k <= equil}):
        g.sweep(k - done)
        done = k
        _, e, c = mean_obs()
        trace.append({"sweeps": k, "energy_per_atom": e, "c": c})
    torch.cuda.synchronize()
    X, Y = g.features()
    s = V.Surrogate(I.mlp_init(7, out_bias=float(Y.mean())), stream=stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = s.train(X, Y, batch=batch, steps=train_steps, lr=lr, seed=19)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    pred = s.forward(X[: 1 << 20])
    rmse = float(torch.sqrt(((pred - Y[: 1 << 20]) ** 2).mean()))
    y_std = float(Y.std())
    del X, Y, pred
    start = [g.types(r) for r in range(N_PHI)]
    out = {"workload": "80^3 x 8 replicas, f_B = 1.25 f_A, phi -2.2 eV, kappa 100, 1200 K, c0 5 %, "
                       "period-4 sublattice (64,000 trials per colour step)",
           "equilibration": trace, "train_s": t_train, "train_steps": train_steps,
           "loss_first_last": [float(hist[:10].mean()), float(hist[-100:].mean())],
           "target_rmse_eV": rmse, "target_std_eV": y_std}
    for mode in ("plain", "delayed"):
        for r in range(N_PHI):
            g.set_types(start[r], r)
        g.set_surrogate(s if mode == "delayed" else None)
        g.sweep(2)
        o0, _, _ = mean_obs()
        ms = timed_sweeps(torch, stream, g, sweeps)
        o1, e, c = mean_obs()
        trials = sum(o1[r]["trials"] - o0[r]["trials"] for r in range(N_PHI))
        s1 = sum(o1[r]["stage1_accepts"] - o0[r]["stage1_accepts"] for r in range(N_PHI))
        acc = sum(o1[r]["local_accepts"] - o0[r]["local_accepts"] for r in range(N_PHI))
        flips = sum(o1[r]["flips"] - o0[r]["flips"] for r in range(N_PHI))
        res = {"us_per_step": ms * 1e3 / (sweeps * g.steps_per_sweep),
               "trial_moves_per_s": N_PHI * lat.n * sweeps / (ms * 1e-3),
               "accepted_flips_per_s": flips / (ms * 1e-3),
               "acc_local": acc / trials, "energy_per_atom": e, "c": c}
        if mode == "delayed":
            res["stage1_pass"] = s1 / trials
            res["stage2_accept"] = acc / max(s1, 1)
        out[mode] = res
    out["speedup"] = out["plain"]["us_per_step"] / out["delayed"]["us_per_step"]
    g.close()
    s.close()
    return out


def schedule_bench(V, torch, stream, local, dmu0, sweeps=2):
    """The schedule autotuner (vcsgc_autotune_schedule) on the headline
    workload: the period-4 sublattice (8,000 trials per replica per colour
    step), octant blocks of 4^3 and 5^3 cells (1,000 and 512 trials) and
    overlapping domains in cells of 10^3 (512 trials), each scored by the
    accepted flips per second it delivers from the random start."""
    lat, types, tab, phi, c0 = workload(dmu0)
    cand = [("sublattice 4^3", V.SCHED_SUBLATTICE, (4, 4, 4, 0, 0, 0)),
            ("octant blocks 4^3", V.SCHED_BLOCKS, (4, 4, 4, 2, 2, 2)),
            ("octant blocks 5^3", V.SCHED_BLOCKS, (5, 5, 5, 2, 2, 2)),
            ("overlapping 10^3, gap 4", V.SCHED_OVERLAP, (10, 10, 10, 4, 4, 4))]
    ctx = V.Context(lat, np.tile(types, N_PHI), tab, 0.0, KAPPA, T_K, schedule=V.SCHED_SUBLATTICE,
                    sched=(4, 4, 4), n_replicas=N_PHI, phi_r=phi, c0_r=c0, seed_r=rank_seeds(0),
                    stream=stream, device=local)
    t0 = time.perf_counter()
    best, scores = ctx.autotune_schedule([(k, s) for _, k, s in cand], sweeps=sweeps)
    dt = time.perf_counter() - t0
    ctx.close()
    return {"workload": "80^3 x 8 replicas, headline phi and c0, from the random start",
            "score": "accepted flips/s of all replicas over the candidate's timed sweeps",
            "scores": {name: float(v) for (name, _, _), v in zip(cand, scores)}, "chosen": cand[best][0],
            "sweeps_per_candidate": 2 * sweeps, "seconds": dt}


def rank_seeds(rank: int, n: int = N_PHI) -> np.ndarray:
    """Philox keys of one rank's replicas.  Ranks run independent replicas
    (the method does not shard: weak scaling), so the keys must differ
    between ranks: rank r takes 2001 + 1000 r + (0 .. n-1)."""
    return np.arange(n, dtype=np.uint64) + np.uint64(2001 + 1000 * rank)


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over the ranks (the slowest rank times the
    job); x itself when there is one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return world * units_per_rank / seconds


def run_reference(args):
    """--impl reference: the CPU oracle times the same workload (replica 0 of
    the headline, with the driving force of its own pre-scan)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O

    lat, types, tab, _, c0 = workload(0.0)
    s = O.System(lat, types, tab)
    dmu_bal = RC.balanced_dmu0([s.delta_e(i) for i in range(lat.n)], types, T_K)
    phi = RC.phi_grid(dmu_bal, KAPPA, T_K, c0)
    s.set_params(float(phi[0]), KAPPA, T_K, c0=float(c0[0]), seed=2001)
    s.schedule_sublattice(lat.cells, (4, 4, 4))
    step_steps = 16  # colour steps per bench step: 128,000 trial moves
    for _ in range(args.warmup):
        s.parallel_steps(step_steps)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.parallel_steps(step_steps)
    dt = time.perf_counter() - t0
    trials = args.steps * step_steps * (lat.n // 128)
    v = trials / dt
    sample = f"{step_steps} colour steps ({step_steps * (lat.n // 128)} trial moves) of replica 0 per step"
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "trial moves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict({"parallelism": f"replicas x{args.gpus}"}),
            "cpu_baseline": {"value": v, "unit": "trial moves/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "trial moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "recipe": {"dmu0_eV": dmu_bal, "rule": "balanced on the random start, from the oracle's dE"}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-md", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-ising", action="store_true")
    ap.add_argument("--no-overlap", action="store_true")
    ap.add_argument("--no-multi", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--md-only", action="store_true", help="only the MD measurement (profiling)")
    ap.add_argument("--md-box", type=float, default=250.0, help="nanocrystal box (A) for --md-only")
    ap.add_argument("--md-mixed", action="store_true", help="the mixed-precision form for --md-only")
    ap.add_argument("--multi-only", action="store_true", help="only the multicomponent measurement (profiling)")
    ap.add_argument("--da-reembed-only", action="store_true",
                    help="only delayed acceptance on the re-embedding workload (profiling)")
    ap.add_argument("--da-equil", type=int, default=400, help="plain sweeps before the surrogate is trained")
    ap.add_argument("--headline-only", action="store_true", help="only the headline and its sampling points")
    ap.add_argument("--no-recipe", action="store_true",
                    help="skip the SGC pre-scan and the dmu_S point (profiling of the headline)")
    ap.add_argument("--launch", default=None,
                    help="FORM,BLOCK,VARIANT: a fixed launch shape of the colour step instead of the autotuner's")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1012_5082_gb300 import vcsgc as V

    if args.md_only:
        print(json.dumps(md_bench(V, torch, torch.cuda.Stream(), local, steps=args.steps, warmup=args.warmup,
                                  box=args.md_box, precision=1 if args.md_mixed else 0)), flush=True)
        return 0
    if args.multi_only:
        print(json.dumps(multi_bench(V, torch, torch.cuda.Stream(), local, sweeps=args.steps,
                                     warmup=args.warmup)), flush=True)
        return 0
    if args.da_reembed_only:
        print(json.dumps(reembed_da_bench(V, torch, torch.cuda.Stream(), local, sweeps=args.steps,
                                          equil=args.da_equil)), flush=True)
        return 0
    stream = torch.cuda.Stream()
    # parameter recipe (Sec. III C): dmu_S from the SGC pre-scan; the balanced
    # driving force of the random start as a second, labelled point
    pre = None if args.no_recipe else prescan(V, stream, local)
    dmu_s = None if args.no_recipe else pre["dmu_S_eV"]
    dmu_bal = balanced_dmu(V, stream, local)
    lat, types, tab, phi, c0 = workload(dmu_bal)
    seeds = rank_seeds(rank)

    def headline_context(phis):
        return V.Context(lat, np.tile(types, N_PHI), tab, 0.0, KAPPA, T_K, schedule=V.SCHED_SUBLATTICE,
                         sched=(4, 4, 4), n_replicas=N_PHI, phi_r=phis, c0_r=c0, seed_r=seeds,
                         stream=stream, device=local)

    ctx = headline_context(phi)
    spw = ctx.steps_per_sweep
    trials_per_step = N_PHI * lat.n
    # launch shape by timing, as a user would (or fixed from the command line)
    if args.launch:
        ctx.set_launch(*[int(x) for x in args.launch.split(",")])
    else:
        ctx.autotune(256)
    launch = ctx.get_launch()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    def sampling(o0, o1, seconds):
        """Per replica over the timed region: local and global acceptance,
        accepted flips per second, concentration at its end."""
        out = []
        for r in range(N_PHI):
            a, b = o0[r], o1[r]
            dt, dg = b["trials"] - a["trials"], b["global_trials"] - a["global_trials"]
            out.append({"c0": float(c0[r]), "c": b["c"],
                        "acc_local": (b["local_accepts"] - a["local_accepts"]) / max(1, dt),
                        "acc_global": (b["global_accepts"] - a["global_accepts"]) / max(1, dg),
                        "accepted_flips_per_s": (b["flips"] - a["flips"]) / seconds})
        return out

    # warm-up (also builds the CUDA graph)
    ctx.sweep(args.warmup)
    flush = L2Flush(torch, local)
    barrier()
    o_start = ctx.observables_all()
    with Clocks(local) as clk:
        barrier()
        ms = timed_sweeps(torch, stream, ctx, args.steps, flush)
        barrier()
    o_end = ctx.observables_all()
    ms_max = max_over_ranks(ms, dist, "cuda")
    value = aggregate(world, trials_per_step * args.steps, ms_max * 1e-3)
    reps = sampling(o_start, o_end, ms * 1e-3)

    # roofline of the dominant kernel: the fused colour step.  Its average time
    # per colour step is the timed region over its steps (the graph's other
    # nodes of the per-step form, the step-base advance and the colour table
    # of the next 64 steps, add ~3 us per 64 launches, ~1 %).
    avg_ms = ms_max / (args.steps * spw)
    trials_per_colour_step = N_PHI * (lat.n // 128)
    achieved = OPS_PER_TRIAL * trials_per_colour_step / (avg_ms * 1e-3) / 1e12
    peak = ALU_PEAK_OPS / 1e12
    hbm_peak, hbm_src = measured_peak_hbm()
    hbm_ach = HBM_BYTES_PER_TRIAL * trials_per_colour_step / (avg_ms * 1e-3) / 1e9
    kname = ("k_lattice_step (one launch per colour step: commit of step k-1, site pick, dE from bit-packed "
             "shell counts, local test, dn reduction)" if launch[0] == 0 else
             "k_cluster_steps (one thread-block cluster per replica, 128 colour steps per launch)")
    roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
            "frac": achieved / peak,
            "peak_source": (f"derived from measured per-SM rates (INT32 120, popc 20.7, multiply pairs 31, FP32 122, "
                            f"expf 11.3 per clock): the ALU pipe needs {SM_CYCLES_PER_TRIAL:.2f} SM cycles per trial "
                            f"({OPS_PER_TRIAL} algorithmic ops), x 152 SMs x 2.07 GHz"),
            # DRAM bytes per launch from an ncu capture of the per-step kernel
            # (256-thread blocks, warm L2, three launches of the timed loop);
            # the cluster form is another kernel, not captured
            "traffic": 255061 if launch[0] == 0 else None,
            "traffic_source": ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --cache-control none, "
                               "k_lattice_step<...,256,...> x 3 (launches 600-602): read 47,360 / 256 / 256 B, "
                               "write 252,672 / 250,368 / 214,272 B; the kernel's own reads are L2-resident, the "
                               "writes are write-backs of lines dirtied before it (the L2 flush between sweeps)"
                               if launch[0] == 0 else None),
            "ops_per_trial": {"simple_int": OPS_SIMPLE, "popc": OPS_POPC, "mul_pairs": OPS_MULPAIR,
                              "fp32": OPS_FP32, "mufu": OPS_MUFU},
            "trials_per_colour_step": trials_per_colour_step, "avg_colour_step_us": avg_ms * 1e3,
            "hbm_nominal": {"bytes_per_trial": HBM_BYTES_PER_TRIAL, "achieved_gbs": hbm_ach, "peak_gbs": hbm_peak,
                            "frac": hbm_ach / hbm_peak, "peak_source": hbm_src,
                            "note": "the gather form's list bytes; this kernel reads no list (measured DRAM ~0)"},
            "step_latency_floor_us": STEP_LATENCY_FLOOR_US}

    recipe_out = {
        "headline": {"dmu0_eV": dmu_bal,
                     "label": "dmu0 = the driving force of the metastable start (Eq. c0's optimality condition on "
                              "the state the run starts from): the first composite move has no expected drift",
                     "replicas": reps, "accepted_flips_per_s": sum(x["accepted_flips_per_s"] for x in reps)}}
    if not args.no_recipe:
        # the second point: the recipe's coexistence driving force dmu_S,
        # which freezes this supersaturated start (every isolated B dissolves
        # locally; the composite moves' dn lies far outside the constraint's
        # width)
        ctx_b = headline_context(RC.phi_grid(dmu_s, KAPPA, T_K, c0))
        ctx_b.set_launch(*launch)
        ctx_b.sweep(args.warmup)
        n_b = min(args.steps, 20)
        ob0 = ctx_b.observables_all()
        ms_b = timed_sweeps(torch, stream, ctx_b, n_b, flush)
        ob1 = ctx_b.observables_all()
        ctx_b.close()
        recipe_out.update(_recipe_point(pre, dmu_s, n_b, trials_per_step, ms_b, sampling(ob0, ob1, ms_b * 1e-3)))

    # end to end through the C ABI with host buffers: every replica's species
    # up from pinned memory, one sweep, observables and species down, every step
    pinned = torch.empty(N_PHI * lat.n, dtype=torch.uint8, pin_memory=True)
    host = pinned.numpy()
    ctx.types_all(host)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_types_all(host)
        ctx.sweep(1)
        obs = ctx.observables_all()
        ctx.types_all(host)
    barrier()
    dt_e2e = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = {"value": aggregate(world, trials_per_step * args.steps, dt_e2e), "unit": "trial moves/s",
           "h2d_bytes_per_step": N_PHI * lat.n,
           "d2h_bytes_per_step": N_PHI * lat.n + N_PHI * ctypes.sizeof(V.Observables),
           "calls_per_step": "vcsgc_set_types_all, vcsgc_sweep(1), vcsgc_observables_all, vcsgc_get_types_all",
           "clock": "host wall clock over all steps"}

    ctx.close()
    launches = (spw * args.steps + 2 * ((spw * args.steps) // 64)) if launch[0] == 0 else args.steps
    line = {"metric": METRIC, "value": value, "unit": "trial moves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": config_dict({"parallelism": f"replicas x{world}"}),
            "launch": {"form": launch[0], "block": launch[1], "variant": launch[2],
                       "chosen_by": "command line" if args.launch else "vcsgc_autotune"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "clocks": clk.summary(), "sampling": recipe_out}
    if not args.headline_only:
        if not args.no_md:
            line["md"] = md_bench(V, torch, stream, local)
            line["md_mixed"] = md_bench(V, torch, stream, local, precision=V.PREC_MIXED)
            line["mc_explicit"] = mc_explicit_bench(V, torch, stream, local, dmu_bal)
        if not args.no_mixed:
            line["mixed_128cubed"] = mixed_bench(V, torch, stream, local, dmu_bal)
        if not args.no_batch:
            line["batch_64"] = batch_bench(V, torch, stream, local, dmu_bal, surrogate=not args.no_surrogate)
        if not args.no_ising:
            line["ising"] = ising_bench(V, torch, stream, local)
        if not args.no_overlap:
            line["overlap"] = overlap_bench(V, torch, stream, local, dmu_bal)
            line["schedule_autotune"] = schedule_bench(V, torch, stream, local, dmu_bal)
        if not args.no_multi:
            line["multicomponent"] = multi_bench(V, torch, stream, local)
            if not args.no_surrogate:
                line["delayed_acceptance_reembedding"] = reembed_da_bench(V, torch, stream, local)
        if not args.no_ensemble and not args.no_md:
            line["md_ensemble"] = ensemble_bench(V, torch, stream, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(lat, types, tab, phi, c0)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
