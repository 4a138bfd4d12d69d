"""Benchmark: LJ MD particle-steps/s on one GB300 (and N independent replicas).

Workload (the large monatomic LJ fluid): fcc 100^3 x 4 = 4,000,000 particles,
density 0.8442, T = 0.722, truncated-shifted LJ eps = sigma = 1, rc = 2.5,
skin 0.3, dt = 0.005, NVE velocity-Verlet with energies every step.  A bench
"step" is one MD step: integrate, list update by the skin rule (amortised),
force, finalize, energy reductions.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
(the reference arm of this method; there is no runnable code in the paper).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LJ MD particle-steps/s (N=4.0M fcc LJ fluid, FP32 forces + double-single integration)"
UNIT = "particle-steps/s"
WORKLOAD = {"workload": "LJ fluid fcc 100^3 x 4 = 4,000,000 particles, rho 0.8442, T 0.722, "
                        "rc 2.5, skin 0.3, dt 0.005, NVE",
            "n_particles": 4000000, "dt": 0.005, "skin": 0.3, "rcut": 2.5,
            "thermo": "every step",
            "l2": "inputs larger than L2 (~2.8 GB working set vs 129 MB L2)"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id is not None:
                cmd += ["-i", str(self.gpu_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def _gpu_smi_id(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ----------------------------------------------------------------------------
# oracle (CPU) timing
# ----------------------------------------------------------------------------
def host_cpu():
    """(nproc, CPU model) of this host, for the CPU-baseline lines."""
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                k, _, v = ln.partition(":")
                k = k.strip().lower()
                if v.strip() and k not in fields:
                    fields[k] = v.strip()
    except OSError:
        pass
    model = fields.get("model name") or fields.get("cpu model") or fields.get("hardware")
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for ln in out.splitlines():
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    model = model or fields.get("model")
    import platform
    return os.cpu_count(), model or platform.machine()


def oracle_sample(nsteps, budget_s=None, ncell=None):
    """Time the FP64 oracle on an fcc sample of the workload (same density,
    temperature and parameters); returns (particle-steps/s, n, steps, secs)."""
    import oracle
    from paper_2406_04210_gb300 import inputs
    if ncell is None:
        # ~6 us per particle-step for a short run incl. the initial list build
        n_target = max(4000, min(4_000_000, budget_s / (6e-6 * max(nsteps, 1))))
        ncell = max(10, int((n_target / 4) ** (1 / 3)))
    s = inputs.fcc_system(ncell, seed=inputs.SEEDS["lj4m"])
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    t0 = time.perf_counter()
    oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, nsteps)
    dt = time.perf_counter() - t0
    return s.n * nsteps / dt, s.n, nsteps, dt


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # warm-up and timed steps on one sample sized to finish in ~2-3 minutes
    total = args.steps + args.warmup
    n_target = max(4000, min(4_000_000, 150.0 / (6e-6 * max(total, 1))))
    if args.ref_n:   # a smaller sample (tests)
        n_target = args.ref_n
    ncell = max(10, int((n_target / 4) ** (1 / 3)))
    import oracle
    from paper_2406_04210_gb300 import inputs
    s = inputs.fcc_system(ncell, seed=inputs.SEEDS["lj4m"])
    lj = oracle.LJ(s.eps, s.sigma, s.rcut)
    w = oracle.run(s.box, s.pos, s.vel, lj, s.skin, s.dt, max(args.warmup, 0))
    t0 = time.perf_counter()
    oracle.run(s.box, w["pos"], w["vel"], lj, s.skin, s.dt, args.steps)
    sec = time.perf_counter() - t0
    value = s.n * args.steps / sec
    sample = (f"fcc {ncell}^3 x 4 = {s.n} particles of the workload's fluid, {args.steps} "
              f"velocity-Verlet steps after {args.warmup} warm-up steps, single thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "nproc": host_cpu()[0], "cpu_model": host_cpu()[1]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def timed_integrate(box, dt, steps, thermo_dev):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    box.integrate(dt, steps, thermo=True, out=thermo_dev)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def timed_call(fn):
    """Milliseconds of fn() on the device (CUDA events on the current stream;
    the library orders its work with that stream)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def bench_adjoint(ljmd, inputs):
    """Adjoint/forward time ratio on the differentiable workload: N = 32,000
    (fcc 20^3 x 4), 200 steps, checkpoints every 20, loss = mean squared
    deviation of the final pair-distance histogram (64 bins on [0, 2.5],
    Gaussian width = bin width) from a target."""
    s = inputs.lj32000()
    nsteps, k = 200, 20
    b = ljmd.from_system(s, "mixed_ds")
    target = b.pair_hist(64, 2.5, 2.5 / 64, 2.8)[0][0] * 0.9
    zeros = np.zeros((s.n, 3))
    res = {}
    for rep in range(3):                      # the first round is warm-up
        b.set_state(s.pos, s.vel)
        t_plain, _ = timed_call(lambda: b.integrate(s.dt, nsteps, thermo=False))
        b.set_state(s.pos, s.vel)
        t_rec, _ = timed_call(lambda: b.integrate(s.dt, nsteps, thermo=False, ckpt_every=k))
        h = b.pair_hist(64, 2.5, 2.5 / 64, 2.8)[0][0]
        coef = 2.0 * (h - target) / 64
        lx_T = b.pair_hist(64, 2.5, 2.5 / 64, 2.8, coef=coef)[1]
        t_adj, out = timed_call(lambda: b.adjoint(lx_T, zeros))
        if rep:
            for key, v in (("forward_ms", t_plain), ("recorded_forward_ms", t_rec), ("adjoint_ms", t_adj)):
                res.setdefault(key, []).append(v)
    med = {key: float(np.median(v)) for key, v in res.items()}
    b.close()
    return {"workload": "fcc 20^3 x 4 = 32,000 particles, rho 0.8442, T 0.722, 200 steps, "
                        "checkpoints every 20, pair-histogram loss (64 bins)",
            "forward_ms": med["forward_ms"], "recorded_forward_ms": med["recorded_forward_ms"],
            "adjoint_ms": med["adjoint_ms"],
            "ratio": med["adjoint_ms"] / med["forward_ms"],
            "ratio_vs_recorded_forward": med["adjoint_ms"] / med["recorded_forward_ms"],
            "dL_deps": float(out[2][0, 0]), "dL_dsigma": float(out[3][0, 0])}


def bench_batched(ljmd, inputs, steps):
    """512 independent boxes, N log-uniform in [500, 20000], rho U[0.6, 0.95],
    T U[0.7, 1.5], advanced together (one launch per phase, graph-captured)."""
    systems = inputs.replica_systems(512, seed=inputs.SEEDS["replicas512"])
    n = [x.n for x in systems]
    pos = np.concatenate([x.pos for x in systems])
    vel = np.concatenate([x.vel for x in systems])
    box = np.stack([x.box for x in systems])
    b = ljmd.Box(pos, box, vel, n=n, precision="mixed_ds")
    b.set_lj(1.0, 1.0, 2.5, 0.3)
    tuning = b.autotune(reps=3, cache=False)
    import torch
    th = torch.zeros((steps, 512, 4), dtype=torch.float64, device="cuda")
    b.integrate(0.005, 20, thermo=True, out=th[:20])
    b.integrate(0.005, min(steps, 100), thermo=True, out=th[:min(steps, 100)])   # step graph of the timed call
    ms, _ = timed_call(lambda: b.integrate(0.005, steps, thermo=True, out=th))
    tot = int(sum(n))
    b.close()
    return {"workload": "512 replicas, N log-uniform [500, 20000], rho U[0.6, 0.95], T U[0.7, 1.5], "
                        "dt 0.005", "particles": tot, "steps": steps, "ms_per_step": ms / steps,
            "value": tot * steps / (ms / 1e3), "unit": UNIT, "tuning": tuning}


def _guarded(fn):
    """Run a secondary measurement; a failure is reported in its place
    instead of ending the run."""
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 - reported, not hidden
        return {"error": f"{type(e).__name__}: {e}"}


def bench_drift(ljmd, inputs, steps):
    """NVE energy drift of the N = 4000 fluid (fcc 10^3 x 4, rho 0.8442,
    T 0.722, dt 0.005) over `steps` steps in each precision: the slope of a
    linear fit of E/N against time (per particle per tau) and the largest
    |E(t) - E(0)|/N, energies recorded every step."""
    s = inputs.lj4000()
    out = {"workload": f"fcc 10^3 x 4 = 4000 particles, rho 0.8442, T 0.722, dt 0.005, {steps} NVE steps "
                       f"({steps * s.dt:g} tau), energies every step"}
    t = (np.arange(steps) + 1) * s.dt
    for prec in ("mixed_ds", "mixed_fp64", "fp64"):
        b = ljmd.from_system(s, prec)
        t0 = time.perf_counter()
        th = b.integrate(s.dt, steps)
        sec = time.perf_counter() - t0
        b.close()
        E = (th[:, 0, 0] + th[:, 0, 1]) / s.n
        slope = float(np.polyfit(t, E - E[0], 1)[0])
        out[prec] = {"drift_per_particle_per_tau": slope,
                     "max_abs_dev_per_particle": float(np.abs(E - E[0]).max()),
                     "E_per_particle_0": float(E[0]), "seconds": sec}
    return out


def bench_binary(ljmd, inputs, steps_mixed, steps_fp64):
    """Binary LJ mixture 80:20 at rho 1.2, N = 256,000, dt 0.003: particle-
    steps/s of the mixed path against the all-FP64 GPU path.  The random
    insertion (minimum separation 0.7) is relaxed on the GPU first by 40
    rounds of 10 MD steps with the velocities zeroed after each round; the
    timed runs then start from the relaxed positions with Maxwell-Boltzmann
    velocities at T = 0.7."""
    s = inputs.binary_random_system(seed=inputs.SEEDS["binary256k"])
    b = ljmd.from_system(s, "mixed_ds")
    zero = np.zeros_like(s.vel)
    b.set_state(s.pos, zero)
    for _ in range(40):
        b.integrate(s.dt, 10, thermo=False)
        pos, _, _ = b.get_state()
        b.set_state(pos, zero)
    pos, _, _ = b.get_state()
    b.close()
    relaxed = inputs.System(s.box, pos, s.vel, s.type, s.eps, s.sigma, s.rcut, s.skin, s.dt, s.T, s.seed)
    out = {"workload": "binary LJ 80:20, N = 256,000, rho 1.2, T 0.7, dt 0.003, rc 2.5 sigma_ab, skin 0.3, "
                       "NVE, energies every step (random insertion relaxed on the GPU)"}
    for prec, k in (("mixed_ds", steps_mixed), ("fp64", steps_fp64)):
        bb = ljmd.from_system(relaxed, prec)
        bb.integrate(s.dt, 20)
        ms, _ = timed_call(lambda: bb.integrate(s.dt, k))
        info = bb.info()
        bb.close()
        out[prec] = {"value": s.n * k / (ms / 1e3), "unit": UNIT, "steps": k, "ms_per_step": ms / k,
                     "rebuilds": int(info.rebuilds)}
    out["mixed_over_fp64"] = out["mixed_ds"]["value"] / out["fp64"]["value"]
    return out


def bench_temperature_sweep(ljmd, inputs, steps, temps=(0.5, 0.722, 1.0, 1.5, 2.0, 3.0)):
    """The truncated-force study of the paper (Sec. 5): N = 100,000, `steps`
    NVE steps per temperature (rho 0.8442, rc 2.5, skin 0.3, dt 0.005).  Per
    temperature: particle-steps/s (no phase events), list builds per step,
    and the phase shares from a profiled run of steps / 10 (a hotter fluid
    moves faster, so the lists are rebuilt more often)."""
    out = {"workload": f"first 100,000 sites of an fcc lattice, rho 0.8442, rc 2.5, skin 0.3, dt 0.005, "
                       f"{steps} NVE steps per temperature, energies every step", "points": []}
    for T in temps:
        s = inputs.fcc_subset_system(100000, 0.8442, T, inputs.SEEDS["lj4m"] + 7)
        b = ljmd.from_system(s, "mixed_ds")
        b.integrate(s.dt, 200)
        i0 = b.info()
        ms, _ = timed_call(lambda: b.integrate(s.dt, steps))
        i1 = b.info()
        b.set_profiling(True)
        b.integrate(s.dt, max(100, steps // 10))
        prof = b.profile()
        b.close()
        tot = sum(v[0] for v in prof.values()) or 1.0
        out["points"].append({"T": T, "value": s.n * steps / (ms / 1e3), "unit": UNIT,
                              "ms_per_step": ms / steps,
                              "rebuilds_per_step": (i1.rebuilds - i0.rebuilds) / steps,
                              "share": {k: v[0] / tot for k, v in prof.items()}})
    return out


def bench_layouts(ljmd, s, tuning, steps=100,
                  layouts=((1.0, "zrun"), (1.0, "morton"), (1.08, "zrun"), (1.15, "zrun"), (1.15, "morton"),
                           (1.22, "zrun"))):
    """A/B of the cell layouts on the same fluid: cell edge over the list
    radius, and the order inside cells (z runs, or a space-filling Morton
    curve over 4 x 4 x 4 sub-cells).  Per layout: in-graph force and list-
    update times per step over `steps` steps (CUDA events in the step graph),
    and one forced list build (binning, sort, list) timed with CUDA events."""
    import torch
    b = ljmd.from_system(s, "mixed_ds")
    b.list_kernel = tuning.get("list_kernel", "auto")
    b.set_tuning(**{k: v for k, v in tuning.items() if k in b.TUNING})
    out = []
    for sc, od in layouts:
        b.set_layout(cell_scale=sc, order=od)
        b.integrate(s.dt, 20, thermo=False)
        b.set_profiling(True)
        b.integrate(s.dt, steps)
        prof = b.profile()
        b.set_profiling(False)
        ms_build, _ = timed_call(lambda: b.neighbour_update(force=True))
        out.append({"cell_scale": sc, "order": od,
                    "force_ms_per_step": prof["force"][0] / steps,
                    "list_update_ms_per_step": prof["list_update"][0] / steps,
                    "forced_build_ms": ms_build})
    b.close()
    torch.cuda.synchronize()
    return {"workload": f"the timed fluid, {steps} steps per layout", "points": out}


def bench_all_pairs(ljmd, inputs, steps_mixed, steps_fp64):
    """The paper's first workload (Sec. 4): untruncated LJ between all pairs,
    velocity-Verlet and the Andersen-like thermostat; N = 2000 (fcc sites,
    rho 0.8442), T_bath 0.722, collision rate 1 per unit time, dt 0.005."""
    s = inputs.fcc_subset_system(2000, 0.8442, 0.722, inputs.SEEDS["lj4000"] + 9)
    inf = np.full((1, 1), np.inf)
    out = {"workload": "all pairs (untruncated LJ, minimum image), N = 2000, rho 0.8442, dt 0.005, "
                       "Andersen-like thermostat T 0.722 rate 1, energies every step"}
    for prec, k in (("mixed_ds", steps_mixed), ("fp64", steps_fp64)):
        b = ljmd.Box(s.pos, s.box, s.vel, s.type, precision=prec)
        b.set_lj(s.eps, s.sigma, inf, s.skin, True)
        b.set_thermostat(0.722, 1.0, 1)
        b.integrate(s.dt, 100)
        ms, _ = timed_call(lambda: b.integrate(s.dt, k))
        th = b.integrate(s.dt, 100)
        b.close()
        out[prec] = {"value": s.n * k / (ms / 1e3), "unit": UNIT, "steps": k, "ms_per_step": ms / k,
                     "T_kin_last100": float(th[:, 0, 3].mean())}
    return out


def _summary(prec, adj, batched, binary, drift, allp, tsweep, layouts=None):
    def g(d, *keys):
        for k in keys:
            if not isinstance(d, dict) or k not in d:
                return None
            d = d[k]
        return d

    def r3(x):
        return float(f"{x:.4g}") if isinstance(x, (int, float)) else x

    out = {"lj4m": {k: r3(v) for k, v in prec.items()}}
    if "fp64" in prec and prec.get("fp64"):
        out["lj4m"]["mixed_ds_over_fp64"] = r3(prec["mixed_ds"] / prec["fp64"])
    out["adjoint_forward_ratio"] = r3(g(adj, "ratio"))
    out["adjoint_over_recorded_forward"] = r3(g(adj, "ratio_vs_recorded_forward"))
    out["replicas512"] = {"value": r3(g(batched, "value")), "steps": g(batched, "steps")}
    out["binary256k"] = {"mixed_ds": r3(g(binary, "mixed_ds", "value")), "fp64": r3(g(binary, "fp64", "value")),
                         "ratio": r3(g(binary, "mixed_over_fp64"))}
    out["drift_lj4000_per_particle_per_tau"] = {p: r3(g(drift, p, "drift_per_particle_per_tau"))
                                                for p in ("mixed_ds", "mixed_fp64", "fp64")}
    out["all_pairs_n2000"] = {"mixed_ds": r3(g(allp, "mixed_ds", "value")), "fp64": r3(g(allp, "fp64", "value"))}
    pts = g(tsweep, "points") or []
    out["tsweep_n100k"] = [[p["T"], r3(p["value"]), r3(p["rebuilds_per_step"])] for p in pts]
    lay = g(layouts, "points") or []
    out["layouts_force_list_build_ms"] = [[p["cell_scale"], p["order"], r3(p["force_ms_per_step"]),
                                           r3(p["forced_build_ms"])] for p in lay]
    return out


def job_throughput(ms_local, n_local, steps, dist=None):
    """Whole-job particle-steps/s over all ranks: the particles every rank
    advanced (summed) times `steps`, over the slowest rank's time (max over
    ranks).  Returns (value, ms_max).  Each rank runs its own box (replicas
    only), so this is the one collective of a multi-GPU run."""
    ms, n = float(ms_local), float(n_local)
    if dist is not None and dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        import torch
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        c = torch.tensor([n], dtype=torch.float64, device=dev)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        ms, n = float(t.item()), float(c.item())
    return n * steps / (ms / 1e3), ms


def run_gpu(args):
    import torch
    from paper_2406_04210_gb300 import build, inputs, ljmd

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0 or world == 1:
        build.build()
    if dist:
        dist.barrier()
    ljmd.load()

    # independent replica per rank (replicas only: the path does not shard)
    s = inputs.fcc_system(args.ncell, seed=inputs.SEEDS["lj4m"] + rank)
    n = s.n
    box = ljmd.from_system(s, "mixed_ds")
    box.list_kernel = args.list_kernel
    box.force_kernel = args.force_kernel
    if args.cond_graph:
        box.graph_conditional = True
    tuning = box.autotune(reps=3, cache=False)        # launch/layout/list-kernel autotuner
    thermo = torch.zeros((max(args.steps, args.warmup, 1), 1, 4), dtype=torch.float64,
                         device="cuda")
    if args.warmup:
        box.integrate(s.dt, args.warmup, thermo=True, out=thermo[: args.warmup])
    # untimed: capture the step graphs the timed call replays (graphs hold up
    # to 100 steps, keyed by their step count) and size the energy ring, so
    # that the timed region launches graphs and does no capture
    for k in sorted({min(args.steps, 100), args.steps % 100} - {0}):
        box.integrate(s.dt, k, thermo=True, out=thermo[:k])
    info0 = box.info()
    sampler = ClockSampler(_gpu_smi_id(local))
    if dist:
        dist.barrier()
    sampler.start()
    ms = timed_integrate(box, s.dt, args.steps, thermo[: args.steps])   # no phase events
    clocks = sampler.stop()
    info1 = box.info()
    launches = int(info1.launches - info0.launches)
    th = thermo[: args.steps].cpu().numpy()
    value, ms = job_throughput(ms, n, args.steps, dist)
    # phase breakdown and the force kernel's in-graph duration: the next K
    # steps again, with CUDA events captured into the step graph
    box.set_profiling(True)
    box.integrate(s.dt, args.steps, thermo=True, out=thermo[: args.steps])
    torch.cuda.synchronize()
    prof = box.profile()

    # roofline of the dominant kernel (pair force), timed in the graph
    fk = "tiles" if box.force_kernel == "tiles" else "chunks"   # "auto" runs the chunk kernel
    f_ms, f_n = prof["force"]
    f_avg = f_ms / max(f_n, 1)
    list_entries = info1.list_entries
    force_bytes = 4 * list_entries + 36 * n      # list + count + own posq + force out
    peak, peak_kind = _peaks()
    achieved = force_bytes / (f_avg / 1e3) / 1e9
    total_prof = sum(v[0] for v in prof.values())
    phases = {k: {"ms_per_step": v[0] / max(args.steps, 1),
                  "share": v[0] / total_prof if total_prof else None} for k, v in prof.items()}
    E = th[:, 0, 0] + th[:, 0, 1]
    box.set_profiling(False)

    # end to end through the C ABI with host buffers: state in, K steps,
    # energies and state out
    pos_h = torch.from_numpy(s.pos).pin_memory()
    vel_h = torch.from_numpy(s.vel).pin_memory()
    pos_o = torch.empty_like(pos_h).pin_memory()
    vel_o = torch.empty_like(vel_h).pin_memory()
    img_o = torch.empty((n, 3), dtype=torch.int32).pin_memory()
    th_h = torch.empty((args.steps, 1, 4), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    box.set_state(pos_h.numpy(), vel_h.numpy())
    box.integrate(s.dt, args.steps, thermo=True, out=th_h.numpy())
    box._check(box._lib.md_get_state(box._h, pos_o.data_ptr(), vel_o.data_ptr(),
                                     img_o.data_ptr()), "md_get_state")
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": n * args.steps / e2e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(48 * n / max(args.steps, 1)),
           "d2h_bytes_per_step": int((60 * n) / max(args.steps, 1) + 32),
           "what": "md_set_state(host x, v) + md_integrate(K steps, host energies) + "
                   "md_get_state(host x, v, images), wall clock"}
    box.close()
    del box

    # other precisions on the same workload
    prec = {"mixed_ds": value / world}
    for p, k in (() if args.quick else (("mixed_fp64", args.steps), ("fp64", max(20, args.steps // 10)))):
        b2 = ljmd.from_system(s, p)
        b2.integrate(s.dt, min(args.warmup, 10) or 1, thermo=True, out=thermo[:10])
        ms2 = timed_integrate(b2, s.dt, k, thermo[:k])
        prec[p] = n * k / (ms2 / 1e3)
        b2.close()

    layouts = _guarded(lambda: bench_layouts(ljmd, s, tuning)) if (args.layouts or not args.quick) else None
    adj = None if args.quick else bench_adjoint(ljmd, inputs)
    batched = None if args.quick else _guarded(lambda: bench_batched(ljmd, inputs, 1000))
    drift = None if args.quick else _guarded(lambda: bench_drift(ljmd, inputs, 100000))
    binary = None if args.quick else _guarded(lambda: bench_binary(ljmd, inputs, 10 * args.steps,
                                                                     max(20, args.steps)))
    tsweep = None if args.quick else _guarded(lambda: bench_temperature_sweep(ljmd, inputs, 50 * args.steps))
    allp = None if args.quick else _guarded(lambda: bench_all_pairs(ljmd, inputs, 20 * args.steps,
                                                                     2 * args.steps))

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1 and not args.quick:
        ps, ns, st, sec = oracle_sample(10, ncell=40)
        nproc, model = host_cpu()
        cpu = {"value": ps, "unit": UNIT, "cores": 1, "kind": "oracle", "nproc": nproc, "cpu_model": model,
               "sample": f"fcc 40^3 x 4 = {ns} particles of the workload's fluid, {st} "
                         f"velocity-Verlet steps incl. the initial list build, "
                         f"{sec:.1f} s on one host core"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / max(args.steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 forces / double-single state",
        "data": "synthetic", "config": dict(WORKLOAD, parallelism=f"replicas{world}"),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (DRAM_BYTES_PER_PARTICLE[fk] * n) if DRAM_BYTES_PER_PARTICLE.get(fk) else None,
                     "kernel": FORCE_KERNEL_NAMES[fk] + " (pair force, energy+virial)",
                     "bytes_per_launch": force_bytes, "avg_launch_ms": f_avg,
                     "peak_kind": f"hbm_gbs of {peak_kind} peaks (copy, burst)"},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
        "phases": phases, "precisions": prec,
        "energy": {"E_per_particle_first": float(E[0] / n), "E_per_particle_last": float(E[-1] / n),
                   "drift_per_particle": float((E[-1] - E[0]) / n)},
        "rebuilds_in_timed_region": int(info1.rebuilds - info0.rebuilds),
        "temperature_sweep": tsweep, "all_pairs": allp, "drift_lj4000": drift, "binary256k": binary,
        "layouts": layouts,
        "adjoint": adj, "batched": batched, "tuning": tuning,
    }
    # the headline figures of the metric's second half and of the other
    # workloads, last in the line and compact
    line["summary"] = _summary(prec, adj, batched, binary, drift, allp, tsweep, layouts)
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


#: DRAM read + write bytes per particle of one force launch (energy variant)
#: per force kernel, from an ncu capture of the 256,000-particle fluid (fcc
#: 40^3 x 4, scaled by the particle count); None when the kernel has changed
#: since.
DRAM_BYTES_PER_PARTICLE = {"chunks": 416.0, "tiles": None}
FORCE_KERNEL_NAMES = {"chunks": "k_force_f32", "tiles": "k_force_tile_f32"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ncell", type=int, default=100,
                    help="fcc cells per edge (100 = the 4.0M-particle workload; smaller for profiling)")
    ap.add_argument("--quick", action="store_true",
                    help="skip the other precisions and the CPU oracle (profiling runs)")
    ap.add_argument("--layouts", action="store_true",
                    help="with --quick: still run the cell-layout A/B")
    ap.add_argument("--list-kernel", default="auto", choices=["auto", "quads", "lanes"],
                    help="list-build kernel (md_set_list_kernel)")
    ap.add_argument("--force-kernel", default="auto", choices=["auto", "chunks", "tiles"],
                    help="FP32 list-form force kernel (md_set_force_kernel)")
    ap.add_argument("--ref-n", type=int, default=0,
                    help="--impl reference: particles of the oracle's sample (default: sized to ~2-3 minutes)")
    ap.add_argument("--cond-graph", action="store_true",
                    help="list update of each step as a conditional graph node (md_set_graph_conditional; "
                         "fewer launches, ~4.5 us slower per step on GB300)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.ncell != 100:
        n = 4 * args.ncell ** 3
        WORKLOAD["workload"] = WORKLOAD["workload"].replace("100^3 x 4 = 4,000,000", f"{args.ncell}^3 x 4 = {n:,}")
        WORKLOAD["n_particles"] = n
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
