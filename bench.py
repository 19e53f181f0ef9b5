#!/usr/bin/env python
"""Benchmark of the MOL^T wave solver on one or more GB300s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload 2d|3d|1d|batch|adjoint]
                    [--prec mixed|fp64] [--impl ours|reference]

A "step" is one time step of the scheme of order 2P over the whole synthetic
field: every pass of the hot path (per-axis line sweeps, the ADI combination
and the level update u^{n+1} = 2u^n - u^{n-1} + F[u^n]).  The default workload
is the 2D one: homogeneous Dirichlet unit square, 2048 x 2048 points, P = 3
(6th order), CFL 2, beta = beta_max(3), a seeded Gaussian pulse; inputs are
resident in HBM when the timed region starts.  Metric: point-updates/s
(points x steps / second), summed over all GPUs.  ``--workload batch``: 512
independent Dirichlet squares, n log-uniform in [64, 1024], P in {1, 2, 3},
CFL in [0.5, 4], seeded Gaussians, stepped together through mol_batch_step
(every rank its own 512 problems).  ``--workload adjoint``: gradient of a
receiver misfit (64 receivers, 400 steps) with respect to the initial field of
a 1024^2 Dirichlet problem, P = 2, CFL 2; a step is one adjoint time step.

Prints ONE JSON line (rank 0).  Under torchrun every rank solves its own
problem (independent replicas, weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import shutil
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_1308_3214_gb300 import workloads  # noqa: E402

METRIC = "point-updates/s"
PEAKS_FILE = ROOT / "MEASURED_PEAKS.json"
TRAFFIC_FILE = ROOT / "profiles" / "ncu_traffic.json"
CSRC = ROOT / "paper_1308_3214_gb300" / "csrc"
KERNEL_SOURCES = {
    "single": [CSRC / f for f in ("molt_kernels.cuh", "molt_regs.cuh", "molt_strided_nb.cuh", "molt_tma.cuh",
                                  "molt_passes.cu", "molt_regs.cu", "molt_api.cu")],
    "batch": [CSRC / f for f in ("molt_kernels.cuh", "molt_regs.cuh", "molt_batch.cuh", "molt_batch.cu")],
    "embed": [CSRC / "molt_embed.cu"],
}
FALLBACK_HBM_GBS = 6800.0
FP64_PEAK_GFLOPS = 1250.0


def workload_spec(name: str) -> dict:
    if name == "2d":
        n = 2048
        return dict(name="2d-dirichlet-2048x2048-P3-cfl2-gaussian", shape=(n, n), P=3, cfl=2.0,
                    bc="dirichlet", lo=(0.0, 0.0), hi=(1.0, 1.0), h=1.0 / (n - 1), steps_in_config=500,
                    field=lambda: workloads.gaussian_2d(n, seed=1002))
    if name == "3d":
        n = 256
        L = 2 * math.pi
        return dict(name="3d-periodic-256^3-P2-cfl1.5-fourier16", shape=(n, n, n), P=2, cfl=1.5,
                    bc="periodic", lo=(0.0,) * 3, hi=(L,) * 3, h=L / n, steps_in_config=200,
                    field=lambda: workloads.fourier_3d(n, seed=1003)[0])
    if name == "adjoint":
        n = 1024
        return dict(name="adjoint-2d-dirichlet-1024x1024-P2-cfl2-400steps-64rec", n=n, P=2, cfl=2.0, nsteps=400,
                    nrec=64, bc="dirichlet")
    if name == "batch":
        return dict(name="batch-512-dirichlet-n64..1024-P1..3-cfl0.5..4-gaussian", count=512, seed=1004,
                    steps_in_config=200, bc="dirichlet")
    if name == "source":
        n = 2048
        return dict(name="source-2d-dirichlet-2048x2048-P2-cfl2-pointsource", shape=(n, n), P=2, cfl=2.0,
                    bc="dirichlet", lo=(-1.0, -1.0), hi=(1.0, 1.0), h=2.0 / (n - 1))
    if name == "dirichlet1d":
        n = 10001
        return dict(name="dirichlet1d-10001-P3-cfl2-standing-wave-data", shape=(n,), P=3, cfl=2.0, bc="dirichlet",
                    lo=(0.0,), hi=(1.0,), h=1.0 / (n - 1))
    if name == "embedded":
        n = 2048
        return dict(name="embedded-ellipse-2048x2048-P2-cfl1-gaussian", n=n, P=2, cfl=1.0, bc="dirichlet")
    if name == "toeplitz":
        n = 2048
        return dict(name="toeplitz-experiment-2048x2048-chunk32-d0.5395", shape=(n, n), d=math.exp(-1.234290745253055 / 2))
    if name == "1d":
        n = 256
        L = 2 * math.pi
        return dict(name="1d-periodic-256-P1-cfl1.5-fourier8", shape=(n,), P=1, cfl=1.5, bc="periodic",
                    lo=(0.0,), hi=(L,), h=L / n, steps_in_config=200,
                    field=lambda: workloads.fourier_1d(n, seed=1001))
    raise SystemExit(f"unknown workload {name}")


def bytes_per_point(spec: dict, prec: str) -> dict:
    """Algorithmic HBM bytes per point and step of each pass, the per-unit
    figures of the path's plan (one pass per axis, every field read or written
    once per pass, levels as 8-byte pairs / doubles, staged fields in the
    sweep precision): 2D y pass: u in, the P + 1 stage combinations out
    (8 + t (P + 1)); 2D x pass: those in, u, u^{n-1} in, u^{n+1} out
    (t (P + 1) + 24); 3D: z 8 + t P, y t P + 8 + t (P + 1), x t (P + 1) + 24.
    The roofline's `achieved` uses these."""
    P, nd = spec["P"], len(spec["shape"])
    t = 4 if prec == "mixed" else 8
    if nd == 1:
        return {0: 24}
    if nd == 2:
        return {1: 8 + t * (P + 1), 0: t * (P + 1) + 24}
    return {2: 8 + t * P, 1: t * P + 8 + t * (P + 1), 0: t * (P + 1) + 24}


def bytes_per_point_design(spec: dict, prec: str) -> dict:
    """The bytes these kernels move: in 2D the y pass writes the P powers
    D_y^k u (not P + 1 combinations) and the x pass reads them and takes the
    u term from the pair level it reads anyway (y 8 + t P, x t P + 24);
    otherwise as bytes_per_point."""
    P, nd = spec["P"], len(spec["shape"])
    t = 4 if prec == "mixed" else 8
    if nd == 2:
        return {1: 8 + t * P, 0: t * P + 24}
    return bytes_per_point(spec, prec)


def kernel_sha(family: str = "single") -> str:
    """Hash of the sources the kernels of one family (single-problem or
    batched passes) are compiled from; traffic figures taken on other
    sources are not reported."""
    h = hashlib.sha256()
    for p in KERNEL_SOURCES[family]:
        h.update(p.read_bytes())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""
    QUERY = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def start(self):
        if shutil.which("nvidia-smi") is None:
            return self
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.fh = open(self.path, "w")
        cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-lms", "100"]
        self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        time.sleep(0.3)
        return self

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in Path(self.path).read_text().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            rows.append(f)
        os.unlink(self.path)
        if self.bus_id:
            mine = [r for r in rows if r[1].lower().endswith(self.bus_id.lower()[-12:])]
            rows = mine or rows
        if not rows:
            return None
        idx0 = rows[0][0]
        rows = [r for r in rows if r[0] == idx0]

        def num(x):
            try:
                return float(x)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[2]) for r in rows])
        mx = np.array([num(r[3]) for r in rows])
        pw = np.array([num(r[4]) for r in rows])
        load = pw > np.nanmedian(pw) if len(pw) > 4 else np.ones_like(pw, dtype=bool)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[6 + k].lower().startswith("active"):
                    reasons.add(name)
        sm_load = sm[load] if load.any() else sm
        return {"sm_mhz": float(np.nanmedian(sm_load)), "sm_max_mhz": float(np.nanmax(mx)),
                "reasons": sorted(reasons), "samples": int(len(rows)),
                "power_w_max": float(np.nanmax(pw)) if len(pw) else None}


def read_peak():
    try:
        d = json.loads(PEAKS_FILE.read_text())
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def read_traffic(kernel_axis: int, workload: str, prec: str, family: str = "single"):
    """ncu DRAM bytes per launch of the dominant pass, if taken on the
    current kernel sources."""
    try:
        d = json.loads(TRAFFIC_FILE.read_text())
    except Exception:
        return None
    for e in d.get("entries", []):
        if (e.get("workload") == workload and e.get("prec") == prec and int(e.get("axis", -1)) == kernel_axis
                and e.get("kernel_sha") == kernel_sha(family)):
            return float(e["dram_bytes_per_launch"])
    return None


# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class RankGroup:
    """One process per GPU (the env vars of torch.distributed.run).  With more
    than one rank: a process group (NCCL on GPUs; gloo on the CPU, where the
    tests drive this class), a barrier, and the reductions the JSON line needs:
    the maximum of the ranks' times and the sum of their points.  With one
    rank every call is the identity."""

    def __init__(self, backend: str | None = None):
        self.world, self.rank, self.local = dist_setup()
        self.device = "cpu"
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = backend or ("nccl" if torch.cuda.is_available() else "gloo")
            if backend == "nccl":
                torch.cuda.set_device(self.local)
                dist.init_process_group("nccl", device_id=torch.device("cuda", self.local))
                self.device = "cuda"
            else:
                dist.init_process_group("gloo")

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def _reduce(self, x: float, op: str) -> float:
        if self.world == 1:
            return float(x)
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
        return float(t.item())

    def max(self, x: float) -> float:
        return self._reduce(x, "max")

    def sum(self, x: float) -> float:
        return self._reduce(x, "sum")

    def close(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


TIMED_REGION = ("one call of the public API (mol_step / the solve or adjoint call) over the K timed steps, "
                "level conversions in and out included; CUDA events on the launch stream, the call enqueued "
                "behind a bounded spin kernel so that the host's enqueue latency is not device time (e2e "
                "includes it)")


def hold_stream(ms: float = 60.0):
    """Keep the current stream busy for about `ms` (torch's bounded spin
    kernel) so that the launches enqueued next run back to back: per-pass
    CUDA events then bracket only their kernels, not host launch gaps (a
    70 µs step with two launches and four event records per step can be
    host-bound)."""
    import torch
    torch.cuda._sleep(int(ms * 1e-3 * 2.0e9))


def aggregate_rate(group: RankGroup, points: float, seconds: float) -> float:
    """Whole-job rate: the points all ranks processed over the slowest rank's time."""
    return group.sum(points) / group.max(seconds)


def cpu_oracle_rate(spec: dict, budget_s: float, max_steps: int | None = None, min_side: int = 64):
    """Point-updates/s of the FP64 oracle on a bounded sample of the workload:
    the full field when one step fits the budget, else a smaller grid with the
    same CFL, P and boundary condition."""
    import oracle
    oracle.build()
    nd = len(spec["shape"])
    full = int(np.prod(spec["shape"]))
    P, bc = spec["P"], spec["bc"]
    beta = oracle.beta_max(P)
    # probe: one step on a small grid
    side = spec["shape"][0]
    probe_side = min(side, 256 if nd < 3 else 48)
    probe_shape = (probe_side,) * nd
    u = sample_field(spec, probe_shape)
    nu = beta / spec["cfl"]
    t0 = time.perf_counter()
    oracle.step(u, u, nu, P, beta, bc)
    rate = np.prod(probe_shape) / max(time.perf_counter() - t0, 1e-6)
    steps = max_steps or 3
    pts = min(full, int(rate * budget_s / steps))
    s = max(min_side, int(round(pts ** (1.0 / nd))))
    s = min(s, side)
    shape = (s,) * nd if pts < full else tuple(spec["shape"])
    if max_steps is None and pts >= full:
        # the whole field fits: spend the budget on steps of it (at most 50)
        steps = int(max(3, min(50, rate * budget_s / (2.0 * full))))
    u0 = sample_field(spec, shape)
    u1 = oracle.start(u0, nu, P, beta, bc)
    t0 = time.perf_counter()
    oracle.run(u0, u1, steps, nu, P, beta, bc)
    dt = time.perf_counter() - t0
    return float(np.prod(shape) * steps / dt), shape, steps, dt, oracle.num_threads()


def sample_field(spec: dict, shape):
    nd = len(shape)
    if nd == 2:
        return workloads.gaussian_2d(shape[1], seed=1002, ny=shape[0])
    if nd == 3:
        return workloads.fourier_3d(shape[0], seed=1003, shape=shape)[0]
    return workloads.fourier_1d(shape[0], seed=1001)


def run_reference(args, spec):
    """The oracle as it stands on the host cores: each step is one oracle time
    step on a bounded sample of the workload (same CFL, P, boundary)."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle
    oracle.build()
    nd = len(spec["shape"])
    P, bc = spec["P"], spec["bc"]
    beta = oracle.beta_max(P)
    nu = beta / spec["cfl"]
    total_budget = 150.0
    rate0, _, _, _, _ = cpu_oracle_rate(spec, budget_s=3.0, max_steps=1)
    per_step_pts = rate0 * total_budget / max(args.steps + args.warmup, 1)
    full = int(np.prod(spec["shape"]))
    s = int(round(min(per_step_pts, full) ** (1.0 / nd)))
    s = max(16, min(s, spec["shape"][0]))
    shape = (s,) * nd
    u0 = sample_field(spec, shape)
    u1 = oracle.start(u0, nu, P, beta, bc)
    up, uc = oracle.run(u0, u1, args.warmup, nu, P, beta, bc)
    t0 = time.perf_counter()
    up, uc = oracle.run(up, uc, args.steps, nu, P, beta, bc)
    dt = time.perf_counter() - t0
    pts = float(np.prod(shape))
    value = pts * args.steps / dt
    cores = oracle.num_threads()
    sample = f"{'x'.join(map(str, shape))} grid per step (same CFL, P, bc), {args.steps} steps"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": spec["name"], "shape": list(spec["shape"]), "P": P, "cfl": spec["cfl"], "bc": bc,
                       "beta": beta, "prec": "fp64", "levels": "f64",
                       "timed_region": "host wall clock over the K oracle steps of the sample",
                       "l2": "host run (the oracle on the CPU cores; no GPU cache)",
                       "parallelism": f"{cores} OpenMP threads over lines", "tuning": None},
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample,
                             "sampled_shape": list(shape)},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--workload", default="2d", choices=["2d", "3d", "1d", "batch", "adjoint", "source", "dirichlet1d",
                                                        "embedded", "toeplitz"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="2D default: leave out the batched sub-measurement")
    ap.add_argument("--batch-count", type=int, default=512, help="problems of the batch workload (profiling)")
    ap.add_argument("--tuning", default=None,
                    help="fixed launch variants instead of the autotuner (profiling): res_warps,strided_rpt,"
                         "strided_warps,rows_warps[,rows_persist,strided_nb,strided_stage,rows_nb] for a single "
                         "problem; x_warps_short,x_warps_long,y_rule for the batch")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    spec = workload_spec(args.workload)
    if args.workload == "batch" and args.batch_count != spec["count"]:
        spec["count"] = args.batch_count
        spec["name"] = spec["name"].replace("batch-512", f"batch-{args.batch_count}")
    if args.workload == "batch":
        main_batch(args, spec)
        return
    if args.workload == "adjoint":
        main_adjoint(args, spec)
        return
    if args.workload in ("source", "dirichlet1d"):
        main_extension(args, spec)
        return
    if args.workload == "embedded":
        main_embedded(args, spec)
        return
    if args.workload == "toeplitz":
        main_toeplitz(args, spec)
        return
    if args.impl == "reference":
        run_reference(args, spec)
        return

    import torch
    from paper_1308_3214_gb300 import molt

    group = RankGroup()
    world, rank = group.world, group.rank
    if world == 1:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    barrier, max_over_ranks = group.barrier, group.max

    shape, P = spec["shape"], spec["P"]
    N = int(np.prod(shape))
    dt = spec["cfl"] * spec["h"]

    def make(prec):
        return molt.Solver(shape, dt=dt, P=P, bc=spec["bc"], prec=prec, lo=spec["lo"], hi=spec["hi"])

    u0_host = spec["field"]()
    solver = make(args.prec)
    if args.tuning:
        solver.set_tuning(*[int(v) for v in args.tuning.split(",")])
        tuning = solver.tuning()
    else:
        tuning = solver.autotune()          # once per problem, as a user would

    def timed_steps(s, nsteps, warm):
        """Region A: nsteps through mol_step as a user runs it (CUDA-graph time
        loop), timed with CUDA events on the launch stream.  Region B, right
        after: the same nsteps with per-pass CUDA events (graphs off) for the
        per-kernel durations of the roofline."""
        up = torch.from_numpy(u0_host).cuda()
        uc = s.start(up)
        s.step(up, uc, warm)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        l0 = s.launches
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        hold_stream()
        ev0.record()
        s.step(up, uc, nsteps)
        ev1.record()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = s.launches - l0
        s.set_pass_timing(True)
        kb = min(nsteps, 100)
        e2 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        hold_stream()
        e2.record()
        s.step(up, uc, kb)
        e3.record()
        torch.cuda.synchronize()
        passes = s.pass_times()
        s.set_pass_timing(False)
        return ms, launches, passes, e2.elapsed_time(e3) * nsteps / kb

    try:
        bus = torch.cuda.get_device_properties(dev_index).pci_bus_id
    except Exception:
        bus = None
    sampler = ClockSampler(bus).start()
    ms, launches, passes, ms_b = timed_steps(solver, args.steps, args.warmup)
    clocks = sampler.stop()
    value = aggregate_rate(group, N * args.steps, ms * 1e-3)
    ms = max_over_ranks(ms)

    # roofline of the dominant pass
    bpp = bytes_per_point(spec, args.prec)
    bpd = bytes_per_point_design(spec, args.prec)
    dom_axis = max(passes, key=lambda a: passes[a][0])
    dom_ms = passes[dom_axis][0] / passes[dom_axis][1]
    alg_bytes = bpp[dom_axis] * N
    achieved = alg_bytes / (dom_ms * 1e-3) / 1e9
    peak, peak_kind = read_peak()
    if tuning.get("rows_warps", 0) > 0:
        how = ("persistent CTAs, next row prefetched into L2" if tuning.get("rows_persist") else "one CTA per row")
        xk = (f"k_contig_rows (x: each row over {tuning['rows_warps']} warps of a CTA, {how}; "
              "Horner + level update)")
    else:
        xk = "k_contig_res / k_contig (x: one row per warp; Horner + level update)"
    nbt = tuning.get("strided_nb", 0)
    stg = {0: "direct loads and stores", 1: "TMA tile loads", 2: "TMA tensor stores",
           3: "TMA loads and stores"}[tuning.get("strided_stage", 0)]
    pk = (f"k_strided_nb ({{}}: powers of D_{{}}, one neighbour exchange per sweep, {stg})" if nbt
          else "k_strided ({}: powers of D_{})")
    yk = ("k_strided_nb_h (y: Horner, P+1 outputs, one neighbour exchange per sweep"
          + (", fields staged in shared memory)" if nbt == 2 else ")") if nbt
          else "k_strided (y: Horner, P+1 outputs)")
    kernel_name = {0: xk, 1: pk.format("y", "y") if len(shape) == 2 else yk, 2: pk.format("z", "z")}[dom_axis]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": read_traffic(dom_axis, spec["name"], args.prec),
                "kernel": kernel_name, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                "alg_bytes_per_launch": alg_bytes,
                "passes": {f"axis{a}": {"ms_per_launch": passes[a][0] / passes[a][1],
                                         "alg_GBps": bpp[a] * N / (passes[a][0] / passes[a][1] * 1e-3) / 1e9,
                                         "frac": bpp[a] * N / (passes[a][0] / passes[a][1] * 1e-3) / 1e9 / peak,
                                         "alg_bytes_per_point": bpp[a],
                                         "moved_bytes_per_point": bpd[a],
                                         "moved_frac": bpd[a] * N / (passes[a][0] / passes[a][1] * 1e-3) / 1e9 / peak}
                           for a in passes},
                "bytes_note": ("achieved counts the plan's per-point bytes (2D: P + 1 staged fields); "
                               "moved_* count what these kernels move (2D: P fields)"),
                "step_alg_GBps": sum(bpp.values()) * N * args.steps / (ms * 1e-3) / 1e9,
                "kernel_timing": (f"per-pass CUDA events over a second region of min(steps, 100) steps, "
                                  f"enqueued behind a spin kernel so that they run back to back "
                                  f"(graphs off, {ms_b / args.steps:.4f} ms/step)")}

    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.prec == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": spec["name"], "shape": list(shape), "P": P, "cfl": spec["cfl"],
                       "bc": spec["bc"], "beta": solver.beta, "prec": args.prec,
                       "levels": "f32 hi+lo pairs" if args.prec == "mixed" else "f64",
                       "timed_region": TIMED_REGION,
                       "l2": "no flush: per-step working set (3 levels + intermediate fields) exceeds the 129 MB L2",
                       "parallelism": f"{world} independent replica(s)", "tuning": tuning},
            "gpu_launches": launches, "roofline": roofline, "clocks": clocks}

    if rank == 0 and not args.no_fp64_compare and args.prec == "mixed":
        s64 = make("fp64")
        s64.autotune()
        k64 = max(3, args.steps // 8)
        ms64, _, p64, _ = timed_steps(s64, k64, 3)
        line["fp64_path"] = {"value": N * k64 / (ms64 * 1e-3), "ms_per_step": ms64 / k64, "steps": k64,
                             "passes_ms_per_launch": {f"axis{a}": p64[a][0] / p64[a][1] for a in p64}}
        s64.close()

    if rank == 0 and not args.no_accuracy and len(shape) == 2:
        line["accuracy"] = accuracy_check(spec, make, molt, torch)
    elif rank == 0 and not args.no_accuracy and len(shape) == 3 and spec["bc"] == "periodic":
        line["accuracy"] = accuracy_check_3d(spec, make, torch, dt)
    elif rank == 0 and not args.no_accuracy and len(shape) == 1 and spec["bc"] == "periodic":
        line["accuracy"] = accuracy_check_1d(spec, make, torch, dt)

    if not args.no_e2e:
        calls, per_call = 2, spec["steps_in_config"]          # the configuration's whole run per call
        pin_in = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        pin_out = torch.empty(shape, dtype=torch.float64, pin_memory=True)
        pin_in.numpy()[...] = u0_host
        solver.solve_host(pin_in.numpy(), per_call, out=pin_out.numpy())      # warm
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(calls):
            solver.solve_host(pin_in.numpy(), per_call, out=pin_out.numpy())
        torch.cuda.synchronize()
        e2e_el = time.perf_counter() - t0
        e2e_value = aggregate_rate(group, N * per_call * calls, e2e_el)
        line["e2e"] = {"value": e2e_value, "unit": METRIC,
                       "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N,
                       "step": f"one mol_solve_host call: copy u0 in, start + {per_call - 1} steps, copy u out",
                       "time_steps_per_step": per_call}

    if len(shape) == 2 and args.prec == "mixed" and not args.no_batch:
        line["batch"] = batch_summary(args, group)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, sshape, ssteps, sdt, cores = cpu_oracle_rate(spec, budget_s=20.0)
        line["cpu_baseline"] = {"value": rate, "unit": METRIC, "cores": cores, "kind": "oracle",
                                "sample": f"{ssteps} oracle steps on a {'x'.join(map(str, sshape))} grid "
                                          f"({sdt:.1f} s), same CFL, P, boundary"}
        import oracle
        oracle.set_threads(1)
        try:
            r1, s1, k1, t1, _ = cpu_oracle_rate(spec, budget_s=5.0)
        finally:
            oracle.set_threads(cores)
        line["cpu_baseline"]["single_thread"] = {
            "value": r1, "unit": METRIC, "cores": 1,
            "sample": f"{k1} oracle steps on a {'x'.join(map(str, s1))} grid ({t1:.1f} s)"}
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    group.close()


# ---------------------------------------------------------------------------
# batched workload
# ---------------------------------------------------------------------------
def batch_set(spec, rank: int = 0):
    """The 512 problems of one rank: (n, P, cfl, u0) each, dt = CFL h."""
    probs = workloads.batch_problems(count=spec["count"], seed=spec["seed"] + 7919 * rank)
    shapes = [(p.n, p.n) for p in probs]
    dts = [p.cfl / (p.n - 1) for p in probs]
    return probs, shapes, dts, [p.P for p in probs]


def batch_oracle_rate(probs, dts, budget_s: float, steps: int = 2):
    """Point-updates/s of the FP64 oracle on the first problems of the list
    (in their seeded order) that fit the budget, `steps` steps each."""
    import oracle
    oracle.build()
    pts = 0.0
    used = 0
    t_all = 0.0
    for p, dt in zip(probs, dts):
        beta = oracle.beta_max(p.P)
        nu = beta / dt / (p.n - 1)
        u1 = oracle.start(p.u0, nu, p.P, beta, "dirichlet")
        t0 = time.perf_counter()
        oracle.run(p.u0, u1, steps, nu, p.P, beta, "dirichlet")
        t_all += time.perf_counter() - t0
        pts += p.n * p.n * steps
        used += 1
        if t_all >= budget_s:
            break
    return pts / t_all, used, steps, t_all, oracle.num_threads()


def batch_summary(args, group):
    """The 512-problem batched workload measured inside the default run: the
    mixed path through mol_batch_step (CUDA-graph loop), per-pass roofline
    fractions against the measured HBM peak (plan bytes 8 + 4 (P_i + 1) for
    the y pass and 4 (P_i + 1) + 24 for the x pass per point, and the bytes
    the batch kernels move), and the float64 path on the same batch."""
    import torch
    from paper_1308_3214_gb300 import molt
    spec = workload_spec("batch")
    probs, shapes, dts, Ps = batch_set(spec, group.rank)
    npts = sum(n * n for n, _ in shapes)
    plan = {1: sum(n * n * (8 + 4 * (P + 1)) for (n, _), P in zip(shapes, Ps)),
            0: sum(n * n * (4 * (P + 1) + 24) for (n, _), P in zip(shapes, Ps))}
    moved = {1: sum(n * n * (8 + 4 * P) for (n, _), P in zip(shapes, Ps)),
             0: sum(n * n * (4 * P + 24) for (n, _), P in zip(shapes, Ps))}
    steps = max(10, min(args.steps, 40))
    peak, _ = read_peak()

    def run(prec, k):
        b = molt.BatchSolver(shapes, dt=dts, P=Ps, prec=prec)
        tun = b.autotune()
        u0 = b.pack([p.u0 for p in probs])
        up = u0.clone()
        uc = b.start(up)
        b.step(up, uc, 3)
        torch.cuda.synchronize()
        group.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hold_stream()
        e0.record()
        b.step(up, uc, k)
        e1.record()
        torch.cuda.synchronize()
        group.barrier()
        ms = e0.elapsed_time(e1)
        b.set_pass_timing(True)
        hold_stream()
        b.step(up, uc, k)
        torch.cuda.synchronize()
        passes = b.pass_times()
        b.set_pass_timing(False)
        out = uc.clone()
        b.close()
        return ms, passes, tun, out

    ms, passes, tun, u_mixed = run("mixed", steps)
    out = {"workload": spec["name"], "problems": len(shapes), "points_per_step": npts, "steps": steps,
           "value": aggregate_rate(group, npts * steps, ms * 1e-3), "unit": METRIC,
           "ms_per_step": group.max(ms) / steps, "tuning": tun, "passes": {}}
    for a in passes:
        t = passes[a][0] / passes[a][1] * 1e-3
        out["passes"][f"axis{a}"] = {
            "ms_per_launch": t * 1e3, "frac": plan[a] / t / 1e9 / peak, "alg_bytes": plan[a],
            "moved_frac": moved[a] / t / 1e9 / peak, "moved_bytes": moved[a],
            "traffic": read_traffic(a, spec["name"], "mixed", "batch")}
    if group.rank == 0 and not args.no_fp64_compare:
        k64 = max(3, steps // 4)
        ms64, p64, _, _ = run("fp64", k64)
        out["fp64_path"] = {"value": npts * k64 / (ms64 * 1e-3), "ms_per_step": ms64 / k64, "steps": k64,
                            "passes_ms_per_launch": {f"axis{a}": p64[a][0] / p64[a][1] for a in p64}}
    return out


def main_toeplitz(args, spec):
    """The chunk-local causal recurrence of a strided sweep at the 2D
    workload's size and decay (d = e^(-beta_max(3)/2)): the in-register scan
    against the 32 x 32 Toeplitz product on the tensor cores.  Not the
    solver's step: a measurement of a design alternative."""
    from paper_1308_3214_gb300 import molt
    if args.impl == "reference":
        print(json.dumps({"impl": "reference", "unavailable": "a kernel design experiment: no reference arm"}))
        return
    n = spec["shape"][0]
    t_scan, t_tc, diff = molt.toeplitz_experiment(n, n, spec["d"], reps=max(args.steps, 10))
    peak, _ = read_peak()
    bytes_ = 8 * n * n
    flops_tc = 3 * 2 * (24 * 16 * 8 * 8) * (n // 32) * (n // 32)   # issued MMA work: 72 m16n8k8 per tile
    line = {"metric": "chunk recurrences/s", "value": n * n / (t_scan * 1e-3), "unit": "points/s", "n_gpus": 1,
            "steps": max(args.steps, 10), "warmup": 3, "ms_per_step": t_scan, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded uniform)",
            "config": {"workload": spec["name"], "shape": [n, n], "d": spec["d"], "chunk": 32},
            "scan": {"ms_per_launch": t_scan, "GBps": bytes_ / (t_scan * 1e-3) / 1e9,
                     "frac_hbm": bytes_ / (t_scan * 1e-3) / 1e9 / peak},
            "tensor_core_toeplitz": {"ms_per_launch": t_tc, "GBps": bytes_ / (t_tc * 1e-3) / 1e9,
                                     "frac_hbm": bytes_ / (t_tc * 1e-3) / 1e9 / peak,
                                     "mma_tflops_issued": flops_tc / (t_tc * 1e-3) / 1e12,
                                     "max_rel_diff_vs_scan": diff},
            "gpu_launches": 2 * (max(args.steps, 10) + 3)}
    print(json.dumps(line), flush=True)


def main_batch(args, spec):
    world, rank, local = dist_setup()
    if args.impl == "reference":
        if rank != 0:
            return
        probs, shapes, dts, Ps = batch_set(spec)
        # warm-up and timed steps, each step a bounded sample of problems
        budget = 150.0 / max(args.steps + args.warmup, 1)
        batch_oracle_rate(probs, dts, budget * args.warmup, steps=1)
        rates = []
        used = 0
        for _ in range(args.steps):
            r, used, _, _, cores = batch_oracle_rate(probs, dts, budget, steps=1)
            rates.append(r)
        value = float(np.mean(rates))
        npts = sum(n * n for n, _ in shapes)
        sample = f"each step: the first {used} of the 512 problems (seeded order), one oracle step each"
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * npts / value,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": spec["name"], "problems": len(shapes), "points_per_step": npts,
                           "n_range": [min(n for n, _ in shapes), max(n for n, _ in shapes)],
                           "P_counts": {str(k): Ps.count(k) for k in (1, 2, 3)}, "prec": "fp64", "levels": "f64",
                           "timed_region": "host wall clock over each step's oracle sample",
                           "l2": "host run (the oracle on the CPU cores; no GPU cache)",
                           "parallelism": f"{cores} OpenMP threads over lines", "tuning": None},
                "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
                "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_1308_3214_gb300 import molt
    group = RankGroup()
    if world == 1:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    barrier, max_over_ranks = group.barrier, group.max

    probs, shapes, dts, Ps = batch_set(spec, rank)
    npts = sum(n * n for n, _ in shapes)
    t = 4 if args.prec == "mixed" else 8
    # plan bytes (P + 1 staged fields per problem; `achieved`) and the bytes
    # the batch kernels move (P powers)
    bpp_tot = {1: sum(n * n * (8 + t * (P + 1)) for (n, _), P in zip(shapes, Ps)),
               0: sum(n * n * (t * (P + 1) + 24) for (n, _), P in zip(shapes, Ps))}
    moved_tot = {1: sum(n * n * (8 + t * P) for (n, _), P in zip(shapes, Ps)),
                 0: sum(n * n * (t * P + 24) for (n, _), P in zip(shapes, Ps))}

    def make(prec, **kw):
        return molt.BatchSolver(shapes, dt=dts, P=Ps, prec=prec, **kw)

    b = make(args.prec)
    if args.tuning:
        xs, xl, yr = [int(v) for v in args.tuning.split(",")]
        b.set_tuning((xs, xl), yr)
        tuning = b.tuning()
    else:
        tuning = b.autotune()
    u0 = b.pack([p.u0 for p in probs])

    def timed(bs, nsteps, warm):
        up = u0.clone()
        uc = bs.start(up)
        bs.step(up, uc, warm)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        l0 = bs.launches
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hold_stream()
        e0.record()
        bs.step(up, uc, nsteps)
        e1.record()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        launches = bs.launches - l0
        bs.set_pass_timing(True)
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record()
        bs.step(up, uc, nsteps)
        e3.record()
        torch.cuda.synchronize()
        passes = bs.pass_times()
        bs.set_pass_timing(False)
        return ms, launches, passes, e2.elapsed_time(e3), uc

    try:
        bus = torch.cuda.get_device_properties(dev_index).pci_bus_id
    except Exception:
        bus = None
    sampler = ClockSampler(bus).start()
    ms, launches, passes, ms_b, _ = timed(b, args.steps, args.warmup)
    clocks = sampler.stop()
    value = aggregate_rate(group, npts * args.steps, ms * 1e-3)
    ms = max_over_ranks(ms)
    peak, peak_kind = read_peak()
    dom_axis = max(passes, key=lambda a: passes[a][0])
    dom_ms = passes[dom_axis][0] / passes[dom_axis][1]
    achieved = bpp_tot[dom_axis] / (dom_ms * 1e-3) / 1e9
    long_x = ("k_batch_xs (one CTA of two warps per row)" if tuning["x_warps"][1] == 0
              else "k_batch_x<LARGE> (one warp per row)")
    kernel_name = {0: f"k_batch_x (x pass: Horner + level update; rows <= 256) + k_batch_xs<8, 2> (rows of "
                      f"257..512) + {long_x} for longer rows",
                   1: "k_batch_y (y pass: powers of D_y)"}[dom_axis]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": read_traffic(dom_axis, spec["name"], args.prec, "batch"),
                "kernel": kernel_name, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                "alg_bytes_per_launch": bpp_tot[dom_axis],
                "passes": {f"axis{a}": {"ms_per_launch": passes[a][0] / passes[a][1],
                                         "alg_GBps": bpp_tot[a] / (passes[a][0] / passes[a][1] * 1e-3) / 1e9,
                                         "alg_bytes": bpp_tot[a], "moved_bytes": moved_tot[a],
                                         "moved_frac": moved_tot[a] / (passes[a][0] / passes[a][1] * 1e-3) / 1e9
                                         / peak} for a in passes},
                "step_alg_GBps": sum(bpp_tot.values()) * args.steps / (ms * 1e-3) / 1e9,
                "kernel_timing": (f"per-pass CUDA events over a second region of {args.steps} steps "
                                  f"(graphs off, {ms_b / args.steps:.4f} ms/step)")}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.prec == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": spec["name"], "problems": len(shapes), "points_per_step": npts,
                       "n_range": [min(n for n, _ in shapes), max(n for n, _ in shapes)],
                       "P_counts": {str(k): Ps.count(k) for k in (1, 2, 3)}, "prec": args.prec,
                       "levels": "f32 hi+lo pairs" if args.prec == "mixed" else "f64",
                       "timed_region": TIMED_REGION,
                       "l2": "no flush: per-step working set (3 levels + intermediate fields) exceeds the 129 MB L2",
                       "parallelism": f"{world} rank(s), each its own {len(shapes)} problems", "tuning": tuning},
            "gpu_launches": launches, "roofline": roofline, "clocks": clocks}

    # end to end right after the device-timed region, before the float64 comparison
    if not args.no_e2e:
        calls, per_call = 3, max(1, min(spec["steps_in_config"], args.steps))
        pin_in = torch.empty(npts, dtype=torch.float64, pin_memory=True)
        pin_out = torch.empty(npts, dtype=torch.float64, pin_memory=True)
        pin_in.numpy()[...] = np.concatenate([p.u0.reshape(-1) for p in probs])
        b.solve_host(pin_in.numpy(), per_call, out=pin_out.numpy())
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(calls):
            b.solve_host(pin_in.numpy(), per_call, out=pin_out.numpy())
        torch.cuda.synchronize()
        e2e_el = time.perf_counter() - t0
        e2e_value = aggregate_rate(group, npts * per_call * calls, e2e_el)
        line["e2e"] = {"value": e2e_value, "unit": METRIC,
                       "h2d_bytes_per_step": 8 * npts, "d2h_bytes_per_step": 8 * npts,
                       "step": f"one mol_batch_solve_host call: copy u0 in, start + {per_call - 1} steps, copy u out",
                       "time_steps_per_step": per_call}

    if rank == 0 and not args.no_fp64_compare and args.prec == "mixed":
        b64 = make("fp64")
        b64.autotune()
        k64 = max(3, args.steps // 8)
        ms64, _, p64, _, _ = timed(b64, k64, 3)
        line["fp64_path"] = {"value": npts * k64 / (ms64 * 1e-3), "ms_per_step": ms64 / k64, "steps": k64,
                             "passes_ms_per_launch": {f"axis{a}": p64[a][0] / p64[a][1] for a in p64}}
        b64.close()

    if rank == 0 and not args.no_accuracy and args.prec == "mixed":
        line["accuracy"] = batch_accuracy(spec, probs, shapes, dts, Ps, make, molt, torch)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, used, ssteps, sdt, cores = batch_oracle_rate(probs, dts, budget_s=20.0)
        line["cpu_baseline"] = {"value": rate, "unit": METRIC, "cores": cores, "kind": "oracle",
                                "sample": f"{ssteps} oracle steps on each of the first {used} problems "
                                          f"(seeded order; {sdt:.1f} s)"}
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    group.close()


# ---------------------------------------------------------------------------
# adjoint workload
# ---------------------------------------------------------------------------
def adjoint_problem(spec, seed_offset: int = 0):
    """u0: seeded Gaussian; targets: traces of a forward run from a second
    seeded Gaussian; receivers: seeded interior nodes."""
    n = spec["n"]
    u0 = workloads.gaussian_2d(n, seed=1005 + seed_offset)
    u_true = workloads.gaussian_2d(n, seed=2005 + seed_offset)
    rec = np.array([iy * n + ix for iy, ix in workloads.receivers_2d(n, spec["nrec"], seed=1005 + seed_offset)],
                   dtype=np.int64)
    return u0, u_true, rec


def extension_inputs(spec, nsteps: int):
    """Inputs of the workloads of the NEXT rows: the point source of the
    paper's Sec. 4.3 example on a 2048^2 grid (discrete delta at the centre,
    f(t) = sin(4 pi t)(1 - exp(-(t/0.2)^2))), or the 1D standing wave
    cos(3 pi x) cos(3 pi t) with its time-dependent end data."""
    n = spec["shape"][0]
    dt = spec["cfl"] * spec["h"]
    t = dt * np.arange(nsteps + 1)
    if spec["name"].startswith("source"):
        g = np.zeros(spec["shape"])
        g[n // 2, n // 2] = 1.0 / spec["h"] ** 2
        f = np.sin(4 * np.pi * t) * (1.0 - np.exp(-(t / 0.2) ** 2))
        return np.zeros(spec["shape"]), dt, g, f
    P = spec["P"]
    d = np.empty((nsteps + 1, 2, P + 1))
    for m in range(P + 1):
        fm = (-(3 * np.pi) ** 2) ** m * np.cos(3 * np.pi * t)
        d[:, 0, m] = fm
        d[:, 1, m] = np.cos(3 * np.pi) * fm
    return np.cos(3 * np.pi * np.linspace(0.0, 1.0, n)), dt, None, d


def main_extension(args, spec):
    """The rows beyond the hot path (source terms, time-dependent Dirichlet
    data): one solve call of K steps, inputs resident; per-pass events of a
    second call; the oracle on a bounded sample."""
    world, rank, local = dist_setup()
    if rank != 0:
        return
    import torch
    from paper_1308_3214_gb300 import molt
    torch.cuda.set_device(0)
    K = args.steps
    u0h, dt, gh, data = extension_inputs(spec, K)
    s = molt.Solver(spec["shape"], dt=dt, P=spec["P"], bc=spec["bc"], prec=args.prec, lo=list(spec["lo"]),
                    hi=list(spec["hi"]))
    u0 = torch.from_numpy(u0h).cuda()
    g = torch.from_numpy(gh).cuda() if gh is not None else None

    def call(nsteps):
        if g is not None:
            return s.solve_source(u0, nsteps, g, data[:nsteps + 1])
        return s.solve_dirichlet(u0, nsteps, data[:nsteps + 1])

    call(args.warmup)
    torch.cuda.synchronize()
    l0 = s.launches
    bus = torch.cuda.get_device_properties(0).pci_bus_id
    sampler = ClockSampler(bus).start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hold_stream()
    e0.record()
    out = call(K)
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    launches = s.launches - l0
    s.set_pass_timing(True)
    call(min(K, 100))
    passes = s.pass_times()
    s.set_pass_timing(False)
    N = int(np.prod(spec["shape"]))
    bpp = bytes_per_point(spec, args.prec)
    dom = max(passes, key=lambda a: passes[a][0])
    dom_ms = passes[dom][0] / passes[dom][1]
    peak, peak_kind = read_peak()
    achieved = bpp[dom] * N / (dom_ms * 1e-3) / 1e9
    line = {"metric": METRIC, "value": N * K / (ms * 1e-3), "unit": METRIC, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": spec["name"], "shape": list(spec["shape"]), "P": spec["P"], "cfl": spec["cfl"],
                       "prec": args.prec, "step": "one call of K steps (solve_source / solve_dirichlet, direct "
                                                  "launches: per-step scalars)", "parallelism": "1 rank",
                       "timed_region": TIMED_REGION},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": None, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
                         "passes": {f"axis{a}": {"ms_per_launch": passes[a][0] / passes[a][1],
                                                  "alg_bytes_per_point": bpp[a]} for a in passes}},
            "clocks": clocks, "finite": bool(torch.isfinite(out).all())}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        beta = oracle.beta_max(spec["P"])
        if gh is not None:
            m = 257                                    # a bounded sample: the same problem on 257^2
            hs = 2.0 / (m - 1)
            dts = spec["cfl"] * hs
            ks = 10
            gs = np.zeros((m, m))
            gs[m // 2, m // 2] = 1.0 / hs ** 2
            ts = dts * np.arange(ks + 1)
            fs = np.sin(4 * np.pi * ts) * (1.0 - np.exp(-(ts / 0.2) ** 2))
            t0 = time.perf_counter()
            oracle.run_source(np.zeros((m, m)), ks, beta / dts * hs, spec["P"], beta, dts ** 2, gs, fs)
            el = time.perf_counter() - t0
            sample = f"{ks} oracle steps of the point-source problem on {m}x{m} ({el:.1f} s)"
            rate = m * m * ks / el
        else:
            ks = 20
            gam = data[:ks + 1] / (beta / dt) ** (2 * np.arange(spec["P"] + 1))
            t0 = time.perf_counter()
            oracle.run_bc(u0h, ks, beta / dt * spec["h"], spec["P"], beta, gam)
            el = time.perf_counter() - t0
            sample = f"{ks} oracle steps of the same problem ({el:.2f} s)"
            rate = N * ks / el
        line["cpu_baseline"] = {"value": rate, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": sample}
    s.close()
    print(json.dumps(line), flush=True)


def embedded_bytes_per_point(P: int, prec: str = "fp64") -> float:
    """Algorithmic bytes of the line-object sweeps per interior point and step.
    float64: C = 4 sweeps (D_x, L_y^{-1}, D_y, L_x^{-1} accumulated: 16 + 16 +
    16 + 24 B), D = 2 sweeps (L_y^{-1}, the subtraction from v: 16 + 24 B);
    Table 3 builds 1 + P(P-1)/2 C's and P - 1 D's per step.
    float32: C of the pair level (8 B in) 12 + 8 + 12 + 12 B; D (D_y v and
    L_y^{-1} v in one sweep that also keeps D_y v for the C of the same field,
    then D_x accumulated) 16 + 12 B; the C of that field, its D_y v already
    formed, 8 + 8 + 12 B; any other C of a float32 field 8 + 8 + 8 + 12 B."""
    nC = 1 + P * (P - 1) // 2
    if prec == "mixed":
        return 44.0 + (P - 1) * (28.0 + 28.0) + (nC - 1 - (P - 1)) * 36.0
    return 88.0 * nC + 40.0 * (P - 1)


def main_embedded(args, spec):
    """The ellipse of Sec. 4.3 (embedded boundary): one mol_embed_step call of
    K steps with the levels resident; per-kind events of a second call; the
    oracle on a bounded sample.  Points = interior nodes of the domain."""
    world, rank, local = dist_setup()
    if rank != 0:
        return
    n, P, cfl = spec["n"], spec["P"], spec["cfl"]
    if args.impl == "reference":
        import oracle
        oracle.build()
        m = 257
        gs = workloads.ellipse_grid(m)
        u0s = workloads.gaussian_embedded(gs, seed=1006, width=0.15)
        beta = oracle.beta_max(P)
        alpha = beta / (cfl * gs.hx)
        oracle.run_embed(u0s, args.warmup, gs, alpha, P, beta)
        t0 = time.perf_counter()
        oracle.run_embed(u0s, args.steps, gs, alpha, P, beta)
        el = time.perf_counter() - t0
        value = gs.mask.sum() * args.steps / el
        sample = f"the ellipse on {m}x{m} ({int(gs.mask.sum())} interior nodes), {args.steps} steps"
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": spec["name"], "sampled_shape": [m, m]},
                "cpu_baseline": {"value": value, "unit": METRIC, "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    import torch
    from paper_1308_3214_gb300 import molt
    torch.cuda.set_device(0)
    g = workloads.ellipse_grid(n)
    npts = int(g.mask.sum())
    dt = cfl * g.hx
    u0h = workloads.gaussian_embedded(g, seed=1006, width=0.15)
    s = molt.EmbedSolver(g, dt=dt, P=P, prec=args.prec)
    K = args.steps
    up = torch.from_numpy(u0h).cuda()
    uc = s.start(up)
    s.step(up, uc, args.warmup)
    torch.cuda.synchronize()
    l0 = s.launches
    bus = torch.cuda.get_device_properties(0).pci_bus_id
    sampler = ClockSampler(bus).start()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hold_stream()
    e0.record(stream)
    s.step(up, uc, K)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    launches = s.launches - l0
    finite = bool(torch.isfinite(uc).all())
    s.set_pass_timing(True)
    kt = min(K, 50)
    s.step(up, uc, kt)
    kinds = s.pass_times()
    s.set_pass_timing(False)
    sweep_ms = kinds["x_sweep"][0] + kinds["y_sweep"][0]
    sweep_launches = kinds["x_sweep"][1] + kinds["y_sweep"][1]
    hbm_peak, peak_kind = read_peak()
    bpp = embedded_bytes_per_point(P, args.prec)
    hbm_achieved = bpp * npts * kt / (sweep_ms * 1e-3) / 1e9
    kinds_ms = {k: v[0] / kt for k, v in kinds.items()}
    if args.prec == "fp64":
        # float64 operations of the sweep per interior node (a node between
        # grid nodes): two 3-point increments (2 x 5 flops), each recurrence's
        # chunk reduction (FMA, 2 flops) and re-scan (FMA, 2 flops) in both
        # directions (8), the homogeneous terms and the sum (9): 27 flops.  The
        # peak is the nominal float64 rate of a GB300 (1.25 TFLOP/s): the
        # sweeps are bound by the narrow float64 pipe, not by HBM.
        flops = 27.0 * npts * sweep_launches
        achieved = flops / (sweep_ms * 1e-3) / 1e9
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                    "frac": achieved / FP64_PEAK_GFLOPS,
                    "traffic": read_traffic(0, spec["name"], "fp64", "embed"),
                    "peak_kind": "nominal float64 rate of a GB300 (no measured float64 peak on this pool)",
                    "kernel": "k_obj_sweep (all line-object sweeps of a step; float64 recurrences)",
                    "flops_per_node_sweep": 27, "hbm": {"achieved_GBps": hbm_achieved, "peak": hbm_peak,
                                                         "frac": hbm_achieved / hbm_peak,
                                                         "alg_bytes_per_point_step": bpp}}
    else:
        # float32 sweeps: at the HBM copy rate the algorithmic bytes take less
        # time than their float32 arithmetic at the nominal rate, so HBM is the
        # roofline; one warp per line object leaves the sweeps latency bound
        roofline = {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": hbm_achieved / hbm_peak,
                    "traffic": read_traffic(0, spec["name"], "mixed", "embed"),
                    "peak_kind": peak_kind,
                    "kernel": "k_obj_sweep32 (all line-object sweeps of a step; float32 difference form)",
                    "alg_bytes_per_point_step": bpp}
    roofline["kinds_ms_per_step"] = kinds_ms
    roofline["sweep_ms_per_launch"] = sweep_ms / max(sweep_launches, 1)
    line = {"metric": METRIC, "value": npts * K / (ms * 1e-3), "unit": METRIC, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": spec["name"], "grid": [n, n], "interior_points": npts, "P": P, "cfl": cfl,
                       "domain": "((x+y)/4)^2 + (x-y)^2 < 1 in [-2.2, 2.2]^2",
                       "levels": "f32 hi+lo pairs" if args.prec == "mixed" else "f64",
                       "step": "mol_embed_step, K steps in one call, levels resident", "parallelism": "1 rank",
                       "timed_region": TIMED_REGION},
            "gpu_launches": launches, "roofline": roofline,
            "clocks": clocks, "finite": finite}
    if not args.no_e2e:
        t0 = time.perf_counter()
        s.solve_host(u0h, K)
        el = time.perf_counter() - t0
        line["e2e"] = {"value": npts * K / el, "unit": METRIC, "h2d_bytes_per_step": 8 * n * n / K,
                       "d2h_bytes_per_step": 8 * n * n / K, "note": "mol_embed_solve_host: u0 in, K steps, u out"}
    if not args.no_fp64_compare and args.prec == "mixed":
        s64 = molt.EmbedSolver(g, dt=dt, P=P, prec="fp64")
        vp = torch.from_numpy(u0h).cuda()
        vc = s64.start(vp)
        s64.step(vp, vc, 3)
        k64 = max(3, K // 4)
        torch.cuda.synchronize()
        e0.record(stream)
        s64.step(vp, vc, k64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        line["fp64_path"] = {"value": npts * k64 / (ms64 * 1e-3), "ms_per_step": ms64 / k64, "steps": k64}
        s64.close()
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        beta = oracle.beta_max(P)
        ks = 60                                        # the workload itself, 60 steps (about 10 s on 16 cores)
        t0 = time.perf_counter()
        oracle.run_embed(u0h, ks, g, beta / (cfl * g.hx), P, beta)
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": npts * ks / el, "unit": METRIC, "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"{ks} oracle steps of the workload ({n}x{n}, "
                                                            f"{npts} interior nodes, {el:.1f} s)"}
    s.close()
    print(json.dumps(line), flush=True)


def main_adjoint(args, spec):
    world, rank, local = dist_setup()
    n, P, nsteps = spec["n"], spec["P"], spec["nsteps"]
    dt = spec["cfl"] / (n - 1)
    if args.impl == "reference":
        if rank != 0:
            return
        import oracle
        oracle.build()
        beta = oracle.beta_max(P)
        # each step: one oracle adjoint step (F^T on the field + injection) on
        # a grid sized so that the whole run stays within a few minutes
        budget = 150.0 / max(args.steps + args.warmup, 1)
        m = 64
        t0 = time.perf_counter()
        oracle.FT(np.zeros((m, m)), beta / spec["cfl"], P, beta, "dirichlet")
        per_pt = (time.perf_counter() - t0) / (m * m)
        m = int(max(32, min(n, math.sqrt(budget / max(per_pt, 1e-12)))))
        rng = np.random.default_rng(1)
        rec = rng.choice(m * m, size=spec["nrec"], replace=False)
        tg = rng.normal(size=(args.warmup + args.steps, rec.size))
        nu = beta / spec["cfl"]
        oracle.adjoint(tg[:args.warmup], (m, m), rec, nu, P, beta, "dirichlet")
        t0 = time.perf_counter()
        oracle.adjoint(tg[:args.steps], (m, m), rec, nu, P, beta, "dirichlet")
        el = time.perf_counter() - t0
        value = m * m * args.steps / el
        cores = oracle.num_threads()
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": spec["name"], "sampled_shape": [m, m]},
                "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle",
                                 "sample": f"{m}x{m} grid, {args.steps} adjoint steps (same CFL, P, 64 receivers)"},
                "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_1308_3214_gb300 import molt
    group = RankGroup()
    if world == 1:
        torch.cuda.set_device(0)
    dev_index = torch.cuda.current_device()
    barrier, max_over_ranks = group.barrier, group.max

    u0h, uth, rec = adjoint_problem(spec, 7919 * rank)
    N = args.steps                                   # adjoint steps timed
    b = molt.Solver((n, n), dt=dt, P=P, bc="dirichlet", prec=args.prec)
    tuning = b.autotune()
    u0 = torch.from_numpy(u0h).cuda()
    d = b.traces(torch.from_numpy(uth).cuda(), rec, max(N, nsteps))
    res = b.traces(u0, rec, max(N, nsteps)) - d
    # warm-up, then the timed adjoint run of N steps (ms = one mol_adjoint call)
    b.adjoint(rec, res[:args.warmup])
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    l0 = b.launches
    sampler = None
    try:
        bus = torch.cuda.get_device_properties(dev_index).pci_bus_id
    except Exception:
        bus = None
    sampler = ClockSampler(bus).start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hold_stream()
    e0.record()
    grad = b.adjoint(rec, res[:N])
    e1.record()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    barrier()
    ms_rank = e0.elapsed_time(e1)
    ms = max_over_ranks(ms_rank)
    launches = b.launches - l0
    # per-pass device times of the adjoint passes
    b.set_pass_timing(True)
    hold_stream()
    b.adjoint(rec, res[:min(N, 100)])
    passes = b.pass_times()
    b.set_pass_timing(False)
    pts = n * n
    value = aggregate_rate(group, pts * N, ms_rank * 1e-3)
    t = 4 if args.prec == "mixed" else 8
    bpp = {1: 8 + t * P, 0: t * P + 24}
    dom_axis = max(passes, key=lambda a: passes[a][0])
    dom_ms = passes[dom_axis][0] / passes[dom_axis][1]
    achieved = bpp[dom_axis] * pts / (dom_ms * 1e-3) / 1e9
    peak, peak_kind = read_peak()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": read_traffic(dom_axis, spec["name"], args.prec, "single"),
                "kernel": {0: "k_contig_rows<ADJ> (x pass: transposed Horner + level update, rows split over warps)",
                           1: "k_strided<KM = 2> (y pass: powers of D_y^T, clusters)"}[dom_axis],
                "peak_kind": f"{peak_kind} hbm_gbs (copy)", "alg_bytes_per_launch": bpp[dom_axis] * pts,
                "passes": {f"axis{a}": {"ms_per_launch": passes[a][0] / passes[a][1],
                                         "alg_GBps": bpp[a] * pts / (passes[a][0] / passes[a][1] * 1e-3) / 1e9,
                                         "alg_bytes_per_point": bpp[a]} for a in passes},
                "kernel_timing": "per-pass CUDA events over a second adjoint run of min(steps, 100) steps, "
                                 "enqueued behind a spin kernel so that they run back to back"}
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": N, "warmup": args.warmup,
            "ms_per_step": ms / N, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": spec["name"], "shape": [n, n], "P": P, "cfl": spec["cfl"], "receivers": int(rec.size),
                       "prec": args.prec, "step": "one adjoint step: mu^n = 2 mu^{n+1} - mu^{n+2} + F^T mu^{n+1} + g^n",
                       "timed_region": TIMED_REGION,
                       "l2": "no flush, and the per-step working set (3 adjoint levels as f32 pairs + P power "
                             "fields, about 40 MB at 1024^2) fits in the 129 MB L2: steps run back to back inside "
                             "one mol_adjoint call, so HBM fractions of this line are not DRAM-bound figures",
                       "parallelism": f"{world} rank(s), each its own problem", "tuning": tuning},
            "gpu_launches": launches, "roofline": roofline, "clocks": clocks}
    # gradient check and mixed-vs-fp64 comparison of the full workload gradient
    if rank == 0 and not args.no_accuracy:
        other = "fp64" if args.prec == "mixed" else "mixed"
        b2 = molt.Solver((n, n), dt=dt, P=P, bc="dirichlet", prec=other)
        r2 = (b2.traces(torch.from_numpy(u0h).cuda(), rec, nsteps)
              - b2.traces(torch.from_numpy(uth).cuda(), rec, nsteps))
        g2 = b2.adjoint(rec, r2)
        g1 = b.adjoint(rec, res[:nsteps])
        line["accuracy"] = {"steps": nsteps, f"rel_l2_grad_{args.prec}_vs_{other}":
                            float(torch.linalg.norm(g1 - g2) / torch.linalg.norm(g2))}
        b2.close()
    if not args.no_e2e:
        # the user's whole job through the public API: host u0 in, traces,
        # loss, backward (adjoint), host gradient out
        pin = torch.empty(pts, dtype=torch.float64, pin_memory=True)
        pin.numpy()[...] = u0h.reshape(-1)
        gout = torch.empty(pts, dtype=torch.float64, pin_memory=True)
        dd = d[:nsteps]

        def job():
            u = pin.view(n, n).cuda(non_blocking=True).requires_grad_(True)
            tr = molt.receiver_traces(u, b, rec, nsteps)
            loss = 0.5 * ((tr - dd) ** 2).sum()
            loss.backward()
            gout.copy_(u.grad.view(-1))
            return float(loss)

        job()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        calls = 3
        for _ in range(calls):
            job()
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        line["e2e"] = {"value": aggregate_rate(group, pts * nsteps * calls, el), "unit": METRIC,
                       "h2d_bytes_per_step": 8 * pts, "d2h_bytes_per_step": 8 * pts + 8,
                       "step": f"one gradient: copy u0 in, {nsteps} forward steps with traces, loss, "
                               f"{nsteps} adjoint steps, copy the gradient out (counted as {nsteps} point-updates)",
                       "time_steps_per_step": nsteps}
    if rank == 0 and not args.no_e2e:
        # the same gradient through checkpoint-and-recompute (mol_adjoint_history,
        # K = 40): the loss's g^n injected by a callback as a dense field
        K = 40
        rec_t = torch.from_numpy(rec).cuda()
        res_all = res[:nsteps]

        def gfun(step, u):
            if step == 0:
                return None
            g = torch.zeros(pts, dtype=torch.float64, device="cuda")
            g.index_put_((rec_t,), res_all[step - 1], accumulate=True)
            return g.view(n, n)

        hist = molt.history_gradient(b, u0, nsteps, gfun, checkpoint_every=K)      # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist = molt.history_gradient(b, u0, nsteps, gfun, checkpoint_every=K)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        ref = b.adjoint(rec, res_all)
        line["history"] = {"value": pts * nsteps / el, "unit": METRIC, "checkpoint_every": K, "steps": nsteps,
                           "seconds": el, "fields_held": 2 * ((nsteps - 1) // K + 1) + min(K, nsteps) + 4,
                           "rel_l2_vs_trace_adjoint": float(torch.linalg.norm(hist - ref) / torch.linalg.norm(ref)),
                           "step": f"one gradient of the trace misfit through mol_adjoint_history: {nsteps} forward "
                                   f"steps keeping (u^(c-1), u^c) every {K}, each segment recomputed on the device, "
                                   f"{nsteps} adjoint steps with g^n from a host callback"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        m = 256
        beta = oracle.beta_max(P)
        rng = np.random.default_rng(1)
        rr = rng.choice(m * m, size=spec["nrec"], replace=False)
        ksteps = 20
        t0 = time.perf_counter()
        oracle.adjoint(rng.normal(size=(ksteps, rr.size)), (m, m), rr, beta / spec["cfl"], P, beta, "dirichlet")
        el = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": m * m * ksteps / el, "unit": METRIC, "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": f"{ksteps} oracle adjoint steps on a {m}x{m} grid "
                                                            f"({el:.1f} s), same CFL and P, 64 receivers"}
    b.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    group.close()


def batch_accuracy(spec, probs, shapes, dts, Ps, make, molt, torch, sample: int = 6):
    """Mixed vs FP64 on the batch after the workload's step count: rel L2 of
    mixed against FP64 for every problem, and on `sample` seeded problems the
    error of each path against FP64 on the grid refined 2x in h and dt."""
    nsteps = spec["steps_in_config"]
    res = {}
    for prec in ("mixed", "fp64"):
        bs = make(prec)
        u = bs.solve_host(np.concatenate([p.u0.reshape(-1) for p in probs]), nsteps)
        res[prec] = [u[o:o + n * n].reshape(n, n) for o, (n, _) in zip(bs.offsets, shapes)]
        bs.close()
    rel = [float(np.linalg.norm(m - d) / max(np.linalg.norm(d), 1e-300)) for m, d in zip(res["mixed"], res["fp64"])]
    rng = np.random.default_rng(17)
    picks = sorted(int(i) for i in rng.choice(len(probs), size=sample, replace=False))
    E = []
    for i in picks:
        n = shapes[i][0]
        nf = 2 * n - 1
        sf = molt.Solver((nf, nf), dt=dts[i] / 2, P=Ps[i], bc="dirichlet", prec="fp64")
        # the same Gaussian on the refined grid: evaluate the generator's recipe at the fine nodes
        uf = workloads.gaussian_2d(nf, seed=spec["seed"] * 7919 + i)
        up = torch.from_numpy(uf).cuda()
        uc = sf.start(up)
        sf.step(up, uc, 2 * nsteps - 1)
        ref = uc.cpu().numpy()[::2, ::2]
        sf.close()
        nr = np.linalg.norm(ref)
        e_m = float(np.linalg.norm(res["mixed"][i] - ref) / nr)
        e_d = float(np.linalg.norm(res["fp64"][i] - ref) / nr)
        E.append({"problem": i, "n": n, "P": Ps[i], "E_mixed": e_m, "E_fp64": e_d,
                  "equal_l2": bool(abs(e_m - e_d) <= 0.05 * e_d)})
    return {"steps": nsteps, "rel_l2_mixed_vs_fp64_max": max(rel), "rel_l2_mixed_vs_fp64_median": float(np.median(rel)),
            "sampled": E, "equal_l2_all_sampled": all(e["equal_l2"] for e in E),
            "reference": "fp64 single-problem solver on (2n-1)^2, dt/2, 2x steps, shared nodes"}


def accuracy_check(spec, make, molt, torch):
    """Mixed vs FP64 at equal L2 error (2D): both paths run the workload's
    step count; E_X = rel L2 against FP64 on the grid refined 2x in h and dt,
    compared on the shared nodes."""
    shape, P = spec["shape"], spec["P"]
    nsteps = spec["steps_in_config"]
    u0 = spec["field"]()
    out = {}
    for prec in ("mixed", "fp64"):
        s = make(prec)
        up = torch.from_numpy(u0).cuda()
        uc = s.start(up)
        s.step(up, uc, nsteps - 1)
        out[prec] = uc.cpu().numpy()
        s.close()
    n = shape[0]
    nf = 2 * n - 1
    hf = 1.0 / (nf - 1)
    sf = molt.Solver((nf, nf), dt=spec["cfl"] * spec["h"] / 2, P=P, bc=spec["bc"], prec="fp64",
                     lo=spec["lo"], hi=spec["hi"])
    del hf
    xf = workloads.gaussian_2d(nf, seed=1002)
    up = torch.from_numpy(xf).cuda()
    uc = sf.start(up)
    sf.step(up, uc, 2 * nsteps - 1)
    ref = uc.cpu().numpy()[::2, ::2]
    sf.close()
    nr = np.linalg.norm(ref)
    e_m = float(np.linalg.norm(out["mixed"] - ref) / nr)
    e_d = float(np.linalg.norm(out["fp64"] - ref) / nr)
    return {"steps": nsteps, "E_mixed": e_m, "E_fp64": e_d,
            "equal_l2": bool(abs(e_m - e_d) <= 0.05 * e_d),
            "rel_l2_mixed_vs_fp64": float(np.linalg.norm(out["mixed"] - out["fp64"]) / np.linalg.norm(out["fp64"])),
            "reference": f"fp64 on {nf}x{nf}, dt/2, {2 * nsteps} steps, shared nodes"}


def accuracy_check_3d(spec, make, torch, dt):
    """Mixed vs FP64 at equal L2 error (3D periodic): both paths run the
    workload's step count from the Fourier field; E_X = rel L2 against the
    exact solution sum_m a_m cos(k_m . x + phi_m) cos(|k_m| t) (c = 1, zero
    initial velocity)."""
    n = spec["shape"][0]
    nsteps = spec["steps_in_config"]
    u0, modes = workloads.fourier_3d(n, seed=1003)
    out = {}
    for prec in ("mixed", "fp64"):
        s = make(prec)
        up = torch.from_numpy(u0).cuda()
        uc = s.start(up)
        s.step(up, uc, nsteps - 1)
        out[prec] = uc.cpu().numpy()
        s.close()
    t = nsteps * dt
    x = workloads.axis_coords(n, 0.0, 2 * np.pi, "periodic")
    exact = np.zeros((n, n, n))
    for kx, ky, kz, amp, ph in modes:
        w = np.sqrt(kx * kx + ky * ky + kz * kz)
        e = (amp * np.cos(w * t)) * np.exp(1j * ph) * (np.exp(1j * kz * x)[:, None, None]
                                                       * np.exp(1j * ky * x)[None, :, None]
                                                       * np.exp(1j * kx * x)[None, None, :])
        exact += e.real
    nr = np.linalg.norm(exact)
    e_m = float(np.linalg.norm(out["mixed"] - exact) / nr)
    e_d = float(np.linalg.norm(out["fp64"] - exact) / nr)
    return {"steps": nsteps, "t": t, "E_mixed": e_m, "E_fp64": e_d,
            "equal_l2": bool(abs(e_m - e_d) <= 0.05 * e_d),
            "rel_l2_mixed_vs_fp64": float(np.linalg.norm(out["mixed"] - out["fp64"]) / np.linalg.norm(out["fp64"])),
            "reference": "exact solution sum_m a_m cos(k_m . x + phi_m) cos(|k_m| t) of the 16 modes"}


def accuracy_check_1d(spec, make, torch, dt):
    """The 1D periodic configuration over its step count: mixed and FP64
    against the exact solution (each Fourier mode times cos(k t); c = 1, zero
    initial velocity) and against the FP64 oracle's own run."""
    import oracle
    oracle.build()
    n, P = spec["shape"][0], spec["P"]
    nsteps = spec["steps_in_config"]
    rng = np.random.default_rng(1001)                    # the coefficients of workloads.fourier_1d
    a, b = rng.normal(size=8), rng.normal(size=8)
    u0 = spec["field"]()
    out = {}
    for prec in ("mixed", "fp64"):
        s = make(prec)
        up = torch.from_numpy(u0).cuda()
        uc = s.start(up)
        s.step(up, uc, nsteps - 1)
        out[prec] = uc.cpu().numpy()
        s.close()
    t = nsteps * dt
    x = workloads.axis_coords(n, 0.0, 2 * np.pi, "periodic")
    exact = sum((a[k - 1] * np.cos(k * x) + b[k - 1] * np.sin(k * x)) * np.cos(k * t) for k in range(1, 9))
    beta = oracle.beta_max(P)
    nu = beta / spec["cfl"]
    u1 = oracle.start(u0, nu, P, beta, "periodic")
    _, ref = oracle.run(u0, u1, nsteps - 1, nu, P, beta, "periodic")
    rel = lambda v, r: float(np.linalg.norm(v - r) / np.linalg.norm(r))
    e_m, e_d = rel(out["mixed"], exact), rel(out["fp64"], exact)
    return {"steps": nsteps, "t": t, "E_mixed": e_m, "E_fp64": e_d, "equal_l2": bool(abs(e_m - e_d) <= 0.05 * e_d),
            "rel_l2_fp64_vs_oracle": rel(out["fp64"], ref), "rel_l2_mixed_vs_oracle": rel(out["mixed"], ref),
            "reference": "exact solution sum_k (a_k cos kx + b_k sin kx) cos(k t), and the oracle's run"}


if __name__ == "__main__":
    main()
