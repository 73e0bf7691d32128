"""Throughput of one full WCSPH-RANS advection step with the bidirectional
buffer on GB300, in particle-steps/s.

A "step" is one sph_step advection step: cell-list rebuild, labelling, time
step, B / viscous / k-epsilon sweep, all acoustic sub-steps (momentum and
continuity sweeps, boundary values) and the buffer update.  The workload is
the turbulent straight channel (6 x 2, dp = 0.005, ~480k particles, k-eps
RANS, velocity inlet with 5% Philox fluctuation, zero-pressure outlet) with
FP32 pair sweeps and FP64 integration.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs its own replica of the workload (the
path is replicas-only, no exchange) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s vs plain FP64 at stated error; HBM GB/s; adjoint/forward time"
UNIT = "particle-steps/s"


_T0 = time.perf_counter()


def log(msg: str):
    """Progress on stderr (the JSON line goes to stdout)."""
    sys.stderr.write(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}\n")
    sys.stderr.flush()


def workload(name: str, seed: int = 2):
    from paper_2510_25702_gb300 import cases

    if name == "turbulent_channel":
        return cases.turbulent_channel(length=6.0, height=2.0, dp=0.005, seed=seed)
    if name == "turbulent_channel_small":
        return cases.turbulent_channel(length=0.6, height=0.2, dp=0.005, seed=seed)
    if name == "poiseuille":
        # the pressure-driven channel at its stated pressures (inlet 0.1,
        # outlet 0), in the form that holds its 2000 steps
        return cases.pressure_driven_channel(seed=seed)
    if name == "batched_channels":
        return cases.batched_channels(seed=3 + 100 * (seed - 2))
    if name == "plane_jet":
        return cases.plane_jet(dp=0.002, seed=seed + 2)
    if name == "mixer_3d":
        # the stated 3000-step run holds with the transport-velocity shift and
        # the density reinitialisation on
        return cases.mixer_3d_stable(dp=0.01, seed=seed + 4)
    if name == "mixer_3d_small":
        # 951k fluid + 243k wall particles: the 3D sweeps at a size that a
        # profiler captures quickly, inputs still larger than L2
        return cases.mixer_3d(dp=0.015, seed=seed + 4)
    raise ValueError(name)


def as_list(case):
    return list(case) if isinstance(case, (list, tuple)) else [case]


def describe(case):
    """(name, dim, rans, walls) of a workload that may be a batch of instances."""
    cs = as_list(case)
    name = cs[0].name if len(cs) == 1 else f"batched_channels_{len(cs)}x ({sum(c.n for c in cs)} particles)"
    return name, cs[0].dim, any(c.rans for c in cs), sum(c.nw for c in cs)


# DRAM traffic per launch of the dominant kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum; the command and the summary
# are in profiles/), keyed by the hash of the kernel sources it was taken
# with: a changed source reports null.
NCU_TRAFFIC = {
    # (kernel stage, workload, csrc hash): bytes per launch
    ("advection_sweep", "turbulent_channel", "03b4c48e29e5c736"): 117.3e6,
    ("advection_sweep", "turbulent_channel", "29718dcd43be767d"): 116.0e6,
    ("advection_sweep", "turbulent_channel", "0c8c13fd2cfe5f1c"): 118.0e6,
    ("advection_sweep", "turbulent_channel", "d7457316e402e35f"): 117.5e6,
    ("advection_sweep", "turbulent_channel", "a395c5c7af995f9d"): 117.3e6,
    ("advection_sweep", "turbulent_channel", "ad3089c508c5cf82"): 117.1e6,
    ("advection_sweep", "turbulent_channel", "664e195af6d3036d"): 117.2e6,
    # the same counters: these sources change only the advection sweep's form
    # with the transport shift (X = true), which this workload does not run;
    # every X = false instantiation reports the same registers, stack and
    # spills as on 664e195af6d3036d (ptxas -v)
    ("advection_sweep", "turbulent_channel", "cd30be69af19360e"): 117.2e6,
}


def csrc_hash() -> str:
    import hashlib

    d = os.path.join(ROOT, "paper_2510_25702_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            with open(os.path.join(d, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# algorithmic bytes per live particle and launch, 2D, FP32 packs (16 B),
# FP64 masters (8 B); every array element a kernel needs, once
def algorithmic_bytes(stage: str, dim: int, R: int, rans: bool) -> int:
    pk = 4 * R  # one pack vector
    vec = 8 * dim  # FP64 vector master
    nsym = 3 if dim == 2 else 6
    idx = 2 + 4 + 4  # instance, cell key, label
    if stage == "momentum_sweep":
        rd = idx + 2 * pk + pk * (1 if dim == 2 else 2) + 8 + 8 * nsym + vec + vec + vec + (16 if rans else 0)
        wr = vec + vec + pk
        return rd + wr
    if stage == "continuity_sweep":
        rd = idx + 2 * pk + 8 + 8 + vec + vec
        wr = 8 + 8 + 8 + vec + 2 * pk
        return rd + wr
    if stage == "advection_sweep":
        rd = idx + 2 * pk + (pk + 24 if rans else 0) + 8 + 8 + 8 + vec + vec
        wr = 8 * nsym + vec + (24 if rans else 0) + pk * (1 if dim == 2 else 2) + 8 + 8 + vec + 2 * pk
        return rd + wr
    raise ValueError(stage)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, interval_ms: int = 20):
        self.device = device
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []
        self.span = (0, None)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the first sample arrives once nvidia-smi is up; only then does
            # the timed region start
            t0 = time.perf_counter()
            while not self.lines and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except (OSError, ValueError):
            self.proc = None
        return self

    def begin(self):
        """Mark the start of the timed region: samples before it are left out."""
        self.span = (len(self.lines), None)

    def end(self):
        """Mark the end of the timed region (at least the first sample after
        its start is kept)."""
        self.span = (self.span[0], max(len(self.lines), self.span[0] + 1))

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lo, hi = self.span
        for ln in self.lines[lo:hi]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def sample_case(work: str):
    """The bounded CPU sample of a workload: the same channel physics and
    spacing on a 0.75 x 2 section (60k particles) for the full 6 x 2 channel."""
    from paper_2510_25702_gb300 import cases

    if work == "turbulent_channel":
        return cases.turbulent_channel(length=0.75, height=2.0, dp=0.005, seed=2)
    if work == "batched_channels":
        return cases.batched_channels()[5]
    if work == "plane_jet":
        return cases.plane_jet(dp=0.002, box=0.4)
    if work == "mixer_3d":
        return cases.mixer_3d_stable(dp=0.02)
    return workload(work)


def time_oracle(case, steps: int, warmup: int = 0):
    import oracle

    o = oracle.OracleSim(case)
    for _ in range(warmup):
        o.step(1)
    ps = 0
    t0 = time.perf_counter()
    for _ in range(steps):
        ps += o.n - int(o.a["dead"][: o.n].sum())
        o.step(1)
    dt = time.perf_counter() - t0
    return ps / dt, dt, o


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(work: str, steps: int = 20):
    """The FP64 oracle, as it stands, on the host cores over a bounded sample
    of the workload (10-30 s of CPU work in all): on all cores (OpenMP over
    particles; the reported value) and on one core."""
    import oracle

    case = sample_case(work)
    cores = host_cores()
    oracle.set_threads(cores)
    value, dt, o = time_oracle(case, 2 * steps)
    used = oracle.num_threads()
    oracle.set_threads(1)
    v1, dt1, _ = time_oracle(case, steps)
    oracle.set_threads(cores)
    return {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"{2 * steps} advection steps ({o.stats['n_ac']} sub-steps each) of {case.name} "
                      f"({case.n} particles, a section of the workload), {dt:.1f} s FP64 on {used} threads",
            "one_core": {"value": v1, "cores": 1, "sample": f"{steps} steps, {dt1:.1f} s"}}


def adjoint_bench(steps: int = 200, every: int = 20, dp: float = 0.002):
    """Differentiated window on the plane jet (2 x 2, slot 0.1, dp 0.002,
    about 1M particles, k-eps held over the window, fixed dt, FP64): times
    of the forward (one snapshot), the checkpointed forward and the reverse
    pass over `steps` steps, and a finite-difference check of the gradient
    along one random direction of the 32-point inlet profile."""
    import math

    import torch

    from paper_2510_25702_gb300 import cases, sph
    from paper_2510_25702_gb300.adjoint import Window

    th = 1.0 + 0.1 * np.cos(np.linspace(0.0, 2.0 * np.pi, 32))
    c = cases.plane_jet(dp=dp, theta=th)
    dt_ad = 0.25 * c.h / c.U_ref
    n_ac = max(1, math.ceil(dt_ad / (0.6 * c.h / (c.c0 + c.U_ref))))
    c = c.replace(dt_mode="fixed", dt_ad_fixed=dt_ad, n_ac_fixed=n_ac)
    sim = sph.Simulation(c, precision="fp64")
    log(f"adjoint: created {c.name}")
    # one step with the turbulence held labels the buffer particles (the
    # outlet set S is taken from the labels at the window start); unfrozen
    # k-eps steps at the impulsively started slot would raise nu_t at the
    # slot edges within a few steps beyond what the fixed dt can carry
    Window(sim, 0, 0, [3, 4, 5], 1, 1, 4 * c.dp).forward(th)
    sim.adjoint_release()
    start = sim.save_state()
    win = Window(sim, 0, 0, [3, 4, 5], steps, every, 4 * c.dp)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    # forward of the differentiated map (fixed dt, turbulence held) with one
    # snapshot, then with a snapshot every `every` steps, then the reverse
    once = Window(sim, 0, 0, [3, 4, 5], steps, steps, 4 * c.dp)
    _, t_plain = timed(lambda: once.forward(th))
    log(f"adjoint: forward {t_plain:.2f} s")
    sim.restore_state(start)
    J, t_fwd = timed(lambda: win.forward(th))
    log(f"adjoint: checkpointed forward {t_fwd:.2f} s")
    g, t_bwd = timed(lambda: win.backward())
    log(f"adjoint: backward {t_bwd:.2f} s")
    # the same window with a snapshot at every step (no segment recompute)
    every1 = Window(sim, 0, 0, [3, 4, 5], steps, 1, 4 * c.dp)
    sim.restore_state(start)
    _, t_fwd1 = timed(lambda: every1.forward(th))
    g1, t_bwd1 = timed(lambda: every1.backward())
    log(f"adjoint: every-step snapshots: forward {t_fwd1:.2f} s, backward {t_bwd1:.2f} s")
    u = np.random.default_rng(11).normal(size=th.size)
    u /= np.linalg.norm(u)
    h = 1e-6
    sim.restore_state(start)
    jp = once.forward(th + h * u)
    sim.restore_state(start)
    jm = once.forward(th - h * u)
    fd = (jp - jm) / (2 * h)
    sim.adjoint_release()
    sim.close()
    return {"workload": c.name, "particles": c.n, "window_steps": steps, "checkpoint_every": every,
            "sub_steps": n_ac, "J": J, "forward_plain_s": t_plain, "forward_checkpointed_s": t_fwd,
            "backward_s": t_bwd, "adjoint_over_forward": t_bwd / t_plain,
            "every_step_snapshots": {"forward_s": t_fwd1, "backward_s": t_bwd1,
                                     "adjoint_over_forward": t_bwd1 / t_plain,
                                     "grad_rel_diff": float(np.linalg.norm(g1 - g) / np.linalg.norm(g))},
            "note": "turbulence held and dt fixed over the window in every pass",
            "fd_directional": fd, "adjoint_directional": float(g @ u),
            "fd_rel_err": abs(float(g @ u) - fd) / max(abs(fd), 1e-300), "dtype": "f64"}


def fp32_error(case, sim64, steps: int):
    """The FP32-sweep form against the plain FP64 form after the same number
    of advection steps from the same initial state (`sim64` has taken
    `steps`): relative L2 difference per field over the particles of the
    initial state that both runs still hold, matched by (instance, uid).
    Copies are left out: uids are given in injection order, so one injection
    decision taken differently (a particle within rounding of a buffer line)
    would shift the uids of every later copy."""
    from paper_2510_25702_gb300 import sph

    sim32 = sph.Simulation(case, precision="fp32")
    sim32.step(steps)
    names = ["inst", "uid", "pos", "vel", "rho", "k", "eps"]
    f32, f64 = sim32.read(names), sim64.read(names)
    t32, t64 = sim32.stats()["t"], sim64.stats()["t"]
    sim32.close()
    n0 = np.array([c.n for c in as_list(case)], np.int64)
    keep32 = f32["uid"].astype(np.int64) < n0[f32["inst"]]
    keep64 = f64["uid"].astype(np.int64) < n0[f64["inst"]]
    f32 = {k: v[keep32] for k, v in f32.items()}
    f64 = {k: v[keep64] for k, v in f64.items()}
    k32 = f32["inst"].astype(np.int64) << 32 | f32["uid"].astype(np.int64)
    k64 = f64["inst"].astype(np.int64) << 32 | f64["uid"].astype(np.int64)
    common, i32, i64 = np.intersect1d(k32, k64, assume_unique=True, return_indices=True)
    out = {"steps": steps, "particles_compared": int(common.size),
           "particles_in_one_run_only": int(k32.size + k64.size - 2 * common.size),
           "t_rel_diff": abs(t32 - t64) / max(abs(t64), 1e-300), "rel_l2": {}}
    for name in ("pos", "vel", "rho", "k", "eps"):
        a, b = f32[name][i32], f64[name][i64]
        den = float(np.linalg.norm(b))
        if den > 0:
            out["rel_l2"][name] = float(np.linalg.norm(a - b)) / den
    return out


def probe_error(steps: int, nx: int = 120, ny: int = 40):
    """The FP32-sweep form against the plain FP64 form after `steps`
    advection steps of the 2D turbulent channel, compared on a fixed nx x ny
    grid of probes over the channel by Shepard-normalised SPH interpolation
    (Wendland C2 weights, support 2h): after thousands of steps the two runs
    hold different particles, so the fields are compared at fixed points."""
    from scipy.spatial import cKDTree

    from paper_2510_25702_gb300 import sph

    case = workload("turbulent_channel")
    lo, hi = case.pos[:, :2].min(0), case.pos[:, :2].max(0)
    xs = lo[0] + (np.arange(nx) + 0.5) * (hi[0] - lo[0]) / nx
    ys = lo[1] + (np.arange(ny) + 0.5) * (hi[1] - lo[1]) / ny
    probes = np.stack(np.meshgrid(xs, ys, indexing="ij"), -1).reshape(-1, 2)
    names = ("u", "v", "rho", "k", "eps")
    res = {}
    for prec in ("fp32", "fp64"):
        sim = sph.Simulation(case, precision=prec)
        sim.set_graph(True)
        done = 0
        while done < steps:
            k = min(500, steps - done)
            rc = sim.step_rc(k)
            if rc:
                sim.close()
                return {"workload": case.name, "error": f"{prec}: status {rc} within steps {done}..{done + k}"}
            done += k
        f = sim.read(["pos", "vel", "rho", "mass", "k", "eps"])
        t = sim.stats()["t"]
        sim.close()
        x = f["pos"][:, :2]
        vol = f["mass"] / f["rho"]
        vals = {"u": f["vel"][:, 0], "v": f["vel"][:, 1], "rho": f["rho"], "k": f["k"], "eps": f["eps"]}
        out = {nm: np.zeros(len(probes)) for nm in names}
        for p_i, js in enumerate(cKDTree(x).query_ball_point(probes, 2.0 * case.h)):
            js = np.asarray(js, dtype=np.int64)
            if js.size == 0:
                continue
            q = np.linalg.norm(x[js] - probes[p_i], axis=1) / case.h
            w = (1.0 - 0.5 * q) ** 4 * (1.0 + 2.0 * q) * vol[js]
            for nm in names:
                out[nm][p_i] = (w @ vals[nm][js]) / w.sum()
        res[prec] = (out, t, int(f["pos"].shape[0]))
    (a, ta, na), (b, tb, nb) = res["fp32"], res["fp64"]
    rel = {nm: float(np.linalg.norm(a[nm] - b[nm]) / max(np.linalg.norm(b[nm]), 1e-300)) for nm in names}
    vel = float(np.sqrt(np.sum((a["u"] - b["u"]) ** 2 + (a["v"] - b["v"]) ** 2) / np.sum(b["u"] ** 2 + b["v"] ** 2)))
    return {"workload": case.name, "steps": steps, "probes": [nx, ny], "t_fp32": ta, "t_fp64": tb,
            "particles_fp32": na, "particles_fp64": nb, "rel_l2_velocity": vel, "rel_l2": rel}


def run_reference(args, rank: int):
    """--impl reference: the oracle on all host cores (OpenMP over
    particles), each step one oracle advection step of the bounded sample;
    rank 0 only."""
    if rank != 0:
        return
    import oracle

    oracle.set_threads(host_cores())
    case = sample_case(args.workload)
    value, dt, o = time_oracle(case, max(1, args.steps), warmup=args.warmup)
    used = oracle.num_threads()
    sample = (f"each step one advection step of {case.name} ({case.n} particles, a section of the "
              f"workload), FP64 oracle on {used} threads")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": describe(workload(args.workload))[0], "sample": case.name,
                       "particles": case.n, "rans": bool(case.rans)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--min-timed-s", type=float, default=1.0,
                    help="repeat the K timed steps until the repeats last this long (at least 3 repeats)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="turbulent_channel")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU comparison run")
    ap.add_argument("--no-tune", action="store_true", help="keep the default sweep block sizes")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the differentiated-window timing")
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--adjoint-dp", type=float, default=0.002)
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the differentiated window and print its record (for profiling)")
    ap.add_argument("--probe-steps", type=int, default=5000,
                    help="steps of the FP32-against-FP64 probe-grid comparison in the line (0: skip)")
    ap.add_argument("--probe-error", type=int, default=0, metavar="STEPS",
                    help="only compare the FP32 and FP64 forms of the 2D channel after STEPS steps on a probe grid")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2510_25702_gb300 import build as _b
    from paper_2510_25702_gb300 import sph

    if not os.path.exists(_b.LIB):
        _b.build()
    if args.probe_error > 0:
        rec = probe_error(args.probe_error)
        if rank == 0:
            print(json.dumps(rec))
        return
    if args.adjoint_only:
        rec = adjoint_bench(steps=args.adjoint_steps, every=max(1, args.adjoint_steps // 10), dp=args.adjoint_dp)
        if rank == 0:
            print(json.dumps(rec))
        return
    case = workload(args.workload, seed=2 + rank)
    if args.workload == "batched_channels" and world > 1:
        # instances of one batch partitioned across ranks by particle count
        from paper_2510_25702_gb300.shard import shard_cases

        case = shard_cases(workload(args.workload), world, rank)
    sim = sph.Simulation(case, precision=args.precision)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    wname, wdim, wrans, wwalls = describe(case)
    log(f"created {wname}")
    sim.step(args.warmup)
    log("warm-up done")
    tuned = None
    if not args.no_tune:
        # sweep block sizes, cached per (GPU, workload shape) next to the build
        tuned, hit = sim.autotune(steps=8, cache_path=os.path.join(os.path.dirname(_b.LIB), "autotune.txt"))
        tuned = {"blocks": dict(zip(("list", "adv", "mom", "cont"), tuned)), "from_cache": hit}
    log(f"autotune {tuned}")
    # timed region: K steps replayed from the two captured CUDA graphs
    sim.set_graph(True)
    # one uncaptured step, both graphs captured, then a few replays of each
    # before the clock starts
    sim.step(max(10, args.warmup))
    from paper_2510_25702_gb300.shard import combine_timing

    # The K timed steps are one measurement: a barrier and a synchronise on
    # both sides, CUDA events on the launching stream, the max over ranks.
    # The measurement is repeated (at least 3 times, until the repeats
    # together last min_timed_s) so that the clock record spans the run;
    # value is the median repeat.
    reps = []
    launches = None
    with ClockSampler(local) as clk:
        clk.begin()
        total_ms = 0.0
        while len(reps) < 3 or (total_ms < 1e3 * args.min_timed_s and len(reps) < 1000):
            s0 = sim.stats()
            barrier()
            start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            start.record(stream)
            sim.step(args.steps)
            end.record(stream)
            torch.cuda.synchronize()
            barrier()
            s1 = sim.stats()
            ms_r = start.elapsed_time(end)
            ps_r = 0.5 * (s0["n"] + s1["n"]) * args.steps
            ms_r, ps_r = combine_timing(ms_r, ps_r, dist)
            if launches is None:
                launches = s1["kernel_launches"] - s0["kernel_launches"]
                n0, n1 = s0["n"], s1["n"]
            reps.append((ms_r, ps_r))
            total_ms += ms_r
        clk.end()
    rates = [p / (m * 1e-3) for m, p in reps]
    med = int(np.argsort(rates)[len(rates) // 2])
    ms, particle_steps = reps[med]
    value = rates[med]
    repeats = {"n": len(reps), "ms": [round(m, 4) for m, _ in reps], "value_min": min(rates),
               "value_max": max(rates), "timed_total_ms": total_ms, "statistic": "median"}
    log(f"timed region (graphs) {len(reps)} x {args.steps} steps, median {ms:.2f} ms")

    # the same K steps launched one kernel at a time with CUDA events around
    # every stage on the launching stream: per-kernel durations for the
    # roofline (a graph replay has no per-kernel events)
    sim.set_graph(False)
    sim.set_profiling(2)
    pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0 = sim.stats()
    pa.record(stream)
    sim.step(args.steps)
    pb.record(stream)
    torch.cuda.synchronize()
    e_ms = pa.elapsed_time(pb)
    e1 = sim.stats()
    sim.set_profiling(0)
    stages = sim.stage_times()
    eager = {"value": 0.5 * (e0["n"] + e1["n"]) * args.steps / (e_ms * 1e-3), "ms_per_step": e_ms / args.steps}
    log(f"profiled pass {e_ms:.1f} ms")

    # dominant kernel and its roofline.  The momentum and continuity stages
    # time the first acoustic sub-step (one launch per step each); later
    # sub-steps run in one cooperative launch of their own (stage
    # later_sub_steps), so each stage is one pass over the particles per step
    sweeps = ("advection_sweep", "momentum_sweep", "continuity_sweep")
    dom = max(sweeps, key=lambda s: stages[s][0])
    R = 4 if args.precision == "fp32" else 8
    nbar = 0.5 * (n0 + n1)
    peak, peak_kind = peaks()
    sweep_roofs = {}
    for sw in sweeps:
        sw_ms = stages[sw][0] / args.steps
        bpp = algorithmic_bytes(sw, wdim, R, wrans)
        ach = bpp * nbar / (sw_ms * 1e-3) / 1e9
        sweep_roofs[sw] = {"achieved": ach, "frac": ach / peak, "bytes_per_particle": bpp, "avg_launch_ms": sw_ms}
    per_particle = sweep_roofs[dom]["bytes_per_particle"]
    launch_ms = sweep_roofs[dom]["avg_launch_ms"]
    achieved = sweep_roofs[dom]["achieved"]
    try:
        alu = {"fp32_fma_tflops": sph.measure_fma_peak("fp32") / 1e12,
               "fp64_fma_tflops": sph.measure_fma_peak("fp64") / 1e12,
               "how": "sph_measure_fma_peak: 8 FMA chains per thread, 8 x 256 threads per SM, best of 3"}
    except Exception as exc:  # reported, not fatal
        alu = {"error": str(exc)}

    # end to end through the C ABI: per step the inlet profile goes host ->
    # device (sph_set_profile, from pinned staging), the step is enqueued
    # (sph_step_async), and the step's result -- the FP64 mass and momentum
    # totals of every instance -- comes back into page-locked memory
    # (sph_reduce_mass_momentum_async).  The host waits for step s's totals
    # (an event after their copy) once step s + 1 is enqueued, checks them
    # and counts the live particles from the mass: the device never waits
    # for the host, the host reads every step's result.
    e2e_steps = max(50, args.steps)
    theta = np.array([1.0])
    sim.set_graph(True)
    ninst = len(as_list(case))
    # particle mass of each instance (one mass per instance): live count = mass / m
    m_part = np.array([float(c.mass[0]) for c in as_list(case)])
    ring = [torch.empty(4 * ninst, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]

    def take(buf):
        tot = buf.numpy().reshape(ninst, 4)
        if not np.isfinite(tot).all():
            raise RuntimeError("non-finite totals in the end-to-end loop")
        return float((tot[:, 0] / m_part).sum())

    barrier()
    t0 = time.perf_counter()
    ps = 0.0
    for s in range(e2e_steps):
        sim.set_profile(0, 0, theta)
        sim.step_async(1)
        sim.mass_momentum_async(ring[s % 2])
        done[s % 2].record(stream)
        if s > 0:
            done[(s - 1) % 2].synchronize()
            ps += take(ring[(s - 1) % 2])
    done[(e2e_steps - 1) % 2].synchronize()
    ps += take(ring[(e2e_steps - 1) % 2])
    t1 = time.perf_counter()
    st = sim.stats()
    if st["status"] != 0:
        raise RuntimeError(f"device status {st['status']} in the end-to-end loop")
    # whole job: the slowest rank's wall time, the particle-steps of all ranks
    e2e_ms, ps = combine_timing(1e3 * (t1 - t0), ps, dist)
    e2e = {"value": ps / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": 8 + 8 * theta.size, "d2h_bytes_per_step": 32 * ninst, "steps": e2e_steps,
           "per_step": "sph_set_profile (n_theta and theta moved from page-locked staging by a one-block "
                       "kernel), sph_step_async, sph_reduce_mass_momentum_async (FP64 totals written by the "
                       "reduction into page-locked host memory); the host waits for each step's totals "
                       "after enqueuing the next step and checks them; the status word read once after "
                       "the loop"}

    log("e2e done")
    fp64 = None
    fp32_err = None
    if not args.no_fp64 and args.precision == "fp32" and rank == 0:
        sim64 = sph.Simulation(case, precision="fp64")
        if tuned:
            sim64.autotune(steps=3, cache_path=os.path.join(os.path.dirname(_b.LIB), "autotune.txt"))
        sim64.step(args.warmup)
        # the same K steps in graph replay, repeated like the FP32 form's
        sim64.set_graph(True)
        sim64.step(4)
        done64 = args.warmup + 4
        r64 = []
        while len(r64) < 3 or (sum(m for m, _ in r64) < 5e2 * args.min_timed_s and len(r64) < 200):
            n_a = sim64.stats()["n"]
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sim64.step(args.steps)
            b.record(stream)
            torch.cuda.synchronize()
            done64 += args.steps
            r64.append((a.elapsed_time(b), 0.5 * (n_a + sim64.stats()["n"]) * args.steps))
        rates64 = sorted(p / (m * 1e-3) for m, p in r64)
        fp64 = rates64[len(rates64) // 2]
        fp32_err = fp32_error(case, sim64, done64)
        sim64.close()

    log("fp64 done")
    # the FP32 form against the FP64 form over the scope table's long run of
    # the channel (fields on a fixed probe grid: the particle sets part ways)
    probe = None
    if (args.probe_steps > 0 and args.precision == "fp32" and rank == 0 and not args.no_fp64
            and args.workload == "turbulent_channel"):
        probe = probe_error(args.probe_steps)
        log("probe error done")
    adj = None
    if rank == 0 and not args.no_adjoint:
        adj = adjoint_bench(steps=args.adjoint_steps, every=max(1, args.adjoint_steps // 10), dp=args.adjoint_dp)
        log("adjoint done")

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)

    st = sim.stats()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if (args.workload == "batched_channels" and world > 1) else "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": wname, "particles": int(nbar), "walls": wwalls, "rans": bool(wrans),
                       "sweeps": args.precision, "integration": "f64", "sub_steps": st["n_ac"],
                       "l2": f"working set {st['device_bytes'] / 2**20:.0f} MiB > 129 MB L2, no flush",
                       "parallelism": (f"instances split over {world} ranks" if args.workload == "batched_channels"
                                       and world > 1 else f"replicas x{world}")},
            "repeats": repeats,
            "sweep_rooflines": sweep_roofs, "alu_peaks": alu,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": NCU_TRAFFIC.get((dom, args.workload, csrc_hash())),
                         "csrc": csrc_hash(),
                         "bytes_per_particle": per_particle, "avg_launch_ms": launch_ms,
                         "launch_time": "stage time per step (one launch per step)"},
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
            "stage_timing": "CUDA events around each stage in a second pass of the same K steps launched "
                            "kernel by kernel (value comes from graph replay)",
            "fp64_value": fp64, "fp64_timing": "graph replay of the same K steps, median of repeats",
            "fp32_over_fp64": (value / fp64) if fp64 else None, "fp32_error": fp32_err,
            "fp32_probe_error": probe,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "eager": eager, "autotune": tuned, "adjoint": adj,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
