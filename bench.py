"""Benchmark of the fused DG shallow-water stage on one GB300 (or N replicas).

Metric: DOF-updates/s per RK stage (DOF = 3 (p+1)^2 nlon nlat, one update per
DOF per Runge-Kutta stage).  One bench step is the workload of the 360 x 180,
degree 4 configuration: 500 SSP-RK3 time steps (1500 fused stage kernels,
replayed from captured CUDA graphs) plus the compensated mass reduction, on
the seeded synthetic field (depth 5960 m + 200 m of random spherical
harmonics l <= 4, flow from a random stream function, |u| <= 20 m/s).  L2 is
flushed (256 MiB write) before every timed step; each step is timed with CUDA
events on the solver's stream.

The state arrays of that mesh (19.4 MB each) stay in the 129 MB L2 across the
stages of a step, so the roofline object of the line comes from a second,
streaming leg on the 1440 x 720 degree-4 mesh (311 MB per array), timed the
same way.  "At stated L2 error" is reported per field as (i) the deviation of
each precision from the FP64 path on the same mesh and, over a bounded
sample, from the FP64 oracle, and (ii) the FP64 discretisation error: the
FP64 solution against the FP64 solution of the same field on the 2x refined
mesh at degree 4, as functions; the verdict "matches" = (i) <= 0.1 (ii).
Beside the headline the line carries the tensor-core precisions, the FP64
path, the 180 x 90 degree-3 mesh, the learned correction's 72 x 36 degree-1
coarse solver with and without its network attached (`workload_c5`), the
paper's planar timing workload and the end-to-end figure.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (weak scaling).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (nlon, nlat, degree, rk steps per bench step, seed, description)
    "c2": (180, 90, 3, 1000, 2, "180x90 elements, degree 3, SSP-RK3, 1000 steps per bench step, seed 2"),
    "c1": (20, 10, 1, 100, 1, "20x10 elements, degree 1, SSP-RK3, 100 steps per bench step, seed 1"),
    "c3": (360, 180, 4, 500, 3, "360x180 elements, degree 4, SSP-RK3, 500 steps per bench step, seed 3"),
    "r1": (1440, 720, 4, 20, 3, "1440x720 elements, degree 4, SSP-RK3, 20 steps per bench step, seed 3"),
    # profiling size that still streams (78 MB per FP32 array, 3-5 arrays per stage)
    "r2": (720, 360, 4, 20, 3, "720x360 elements, degree 4, SSP-RK3, 20 steps per bench step, seed 3"),
}
ENSEMBLE_DESC = ("256 members, nlat uniform on 20..180, nlon = 2 nlat, degree uniform on 1..4, "
                 "member k seed 1000+k, FP32 SSP-RK3, 10 steps per bench step, one persistent launch per stage")
METRIC = "DOF-updates/s per RK stage (FP32/TC/learned vs FP64 plain) at stated L2 error"
# DRAM bytes per stage launch of the timed kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, mean over the three SSP-RK3
# stages, cold cache); only for kernels unchanged since that capture.
TRAFFIC = {
    ("fp32", "r1"): (998.1e6, "311.5 / 622.9 / 934.6 MB read, 263.1 / 278.5 / 583.9 MB written "
                              "(1.20x the algorithmic 829.4 MB: the increment form's extra word, partly absorbed by L2)"),
    ("fp32", "c3"): (39.41e6, "19.6 / 39.0 / 58.5 MB read, 0 / 0 / 1.1 MB written (the arrays stay in L2)"),
}
CFL = 0.1
FLUSH_BYTES = 256 << 20
# precision -> arithmetic of the path ("+bf16tc": FP32 stage arithmetic with the
# basis contractions on BF16 tensor cores, FP32 accumulation)
# ("x3": split operands, three tensor-core products per K step)
DTYPES = {"fp32": "f32", "fp64": "f64", "fp32_tc_bf16": "f32+bf16tc", "fp32_tc_fp16": "f32+fp16tc",
          "fp32_tc_bf16x3": "f32+bf16x3tc", "fp32_tc_fp16x3": "f32+fp16x3tc"}
KERNELS = {"fp32": "stage_kernel<float, N={n}>", "fp64": "stage_kernel<double, N={n}>",
           "fp32_tc_bf16": "tc_stage_kernel<{n}, bf16>", "fp32_tc_fp16": "tc_stage_kernel<{n}, fp16>",
           "fp32_tc_bf16x3": "tc_stage_kernel<{n}, bf16, split>", "fp32_tc_fp16x3": "tc_stage_kernel<{n}, fp16, split>"}
TC_PRECS = ("fp32_tc_bf16", "fp32_tc_fp16", "fp32_tc_bf16x3", "fp32_tc_fp16x3")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS) + ["c4"])
    ap.add_argument("--precision", default="fp32", choices=sorted(DTYPES))
    ap.add_argument("--rk-steps", type=int, default=0, help="override RK steps per bench step")
    ap.add_argument("--no-extras", action="store_true", help="skip fp64-plain, e2e and cpu legs (profiling)")
    ap.add_argument("--bands", type=int, default=0,
                    help="time the workload split into this many latitude bands on one GPU (band exchange "
                         "through device copies) against the whole-mesh solver")
    return ap.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job(world, units_per_rank, local_ms):
    """Whole-job throughput of N replicas: every rank processed units_per_rank
    units in local_ms; the job took the slowest rank's time.  Returns
    (units per second, max ms)."""
    total_ms = allreduce_max(world, local_ms)
    return world * units_per_rank / (total_ms * 1e-3), total_ms


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[3:7]):
                if flag.lower() in ("active", "1"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def initial_state(s, seed):
    """The seeded field projected onto the modal basis.  Above 200k elements
    (profiling sizes only) the element means of the field (mode 0) are used:
    projection at p + 9 points per direction would take minutes on the host."""
    from paper_2303_11767_gb300 import synth

    field = synth.SmoothField(seed, s.radius)
    if s.nlon * s.nlat <= 200_000:
        return s.project_grid(field.fields_grid)
    lam = (np.arange(s.nlon) + 0.5) * (2 * math.pi / s.nlon)
    th = -0.5 * math.pi + (np.arange(s.nlat) + 0.5) * (math.pi / s.nlat)
    u = np.zeros(s.shape)
    for f, v in enumerate(field.fields_grid(lam, th)):
        u[:, :, f, 0] = 2.0 * v     # phi_0 = 1/2
    return u


def time_device(s, torch, stream, nsteps, dt, K, W, mass_t, flush):
    """Per-step CUDA-event times (ms) of K timed bench steps after W warm-ups."""
    times = []
    with torch.cuda.stream(stream):
        for it in range(W + K):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(nsteps, dt)
            s.total_mass_device(mass_t)
            b.record(stream)
            if it >= W:
                times.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in times]


def cpu_leg(nlon, nlat, p, seed, budget_s, max_steps):
    """The FP64 oracle on the host cores: number of RK steps that fit the budget,
    their wall time, and the resulting state."""
    import oracle as O
    from paper_2303_11767_gb300 import dgswe, synth

    o = O.Oracle.sphere(nlon, nlat, p, synth.EARTH_RADIUS, dgswe.GRAVITY, dgswe.OMEGA)
    cores = os.cpu_count() or 1
    o.set_threads(cores)
    u0 = o.project_tensor(synth.SmoothField(seed).fields_grid)
    dt = o.max_dt(u0, CFL)
    t0 = time.perf_counter()
    o.rhs(u0)
    t_rhs = time.perf_counter() - t0
    nsteps = int(max(1, min(max_steps, budget_s / (3 * t_rhs))))
    t0 = time.perf_counter()
    u1 = o.step(u0, nsteps, dt, 3)
    wall = time.perf_counter() - t0
    return dict(o=o, u0=u0, u1=u1, dt=dt, nsteps=nsteps, wall=wall, cores=cores)


def stage_flops_per_dof(n):
    """Algorithmic flops of one sum-factorised stage per DOF-update (MAC = 2):
    eval 6n^3 + volume 14n^3 MACs, traces and lifts 36n^2 MACs, ~30 flops of
    fluxes and sources per Gauss point, ~50 per Rusanov point (2n per
    element), 5 per DOF for the RK update: (40n^3 + 117n^2 + 100n) / (3n^2)."""
    return (40.0 * n ** 3 + 117.0 * n ** 2 + 100.0 * n) / (3.0 * n ** 2)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def field_errors(x, y):
    return [float(np.linalg.norm(x[..., f, :] - y[..., f, :]) / np.linalg.norm(y[..., f, :])) for f in range(3)]


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle timed on the host cores, each step a
    bounded sample (a few RK steps) of the same workload."""
    if rank != 0:
        return
    nlon, nlat, p, _, seed, desc = WORKLOADS[args.workload]
    dof = 3 * (p + 1) ** 2 * nlon * nlat
    import oracle as O
    from paper_2303_11767_gb300 import dgswe, synth

    o = O.Oracle.sphere(nlon, nlat, p, synth.EARTH_RADIUS, dgswe.GRAVITY, dgswe.OMEGA)
    cores = os.cpu_count() or 1
    o.set_threads(cores)
    u = o.project_tensor(synth.SmoothField(seed).fields_grid)
    dt = o.max_dt(u, CFL)
    t0 = time.perf_counter()
    o.rhs(u)
    t_rhs = time.perf_counter() - t0
    per = int(max(1, min(100, 3.0 / (3 * t_rhs))))     # ~3 s of work per step
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        u = o.step(u, per, dt, 3)
        if it >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = dof * 3 * per * len(times) / total
    sample = f"{per} SSP-RK3 steps of the {desc.split(',')[0]} workload per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "nlon": nlon, "nlat": nlat, "degree": p, "rk_steps_per_step": per},
        "cpu_baseline": {"value": value, "unit": "DOF-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "DOF-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def member_state(nlon, nlat, p, seed):
    """Member k's own seeded field, projected onto its modal basis (the
    library's cos(theta)-weighted projection, through a temporary FP64
    handle of the member's mesh)."""
    from paper_2303_11767_gb300 import dgswe, synth

    with dgswe.Solver(nlon, nlat, p, precision="fp64") as sv:
        return sv.project_grid(synth.SmoothField(seed, sv.radius).fields_grid)


def run_ensemble(args, world, rank, local):
    """The batched ensemble: 256 independent members advanced together."""
    import torch

    from paper_2303_11767_gb300 import dgswe, synth

    torch.cuda.set_device(local)
    dgswe.set_device(local)
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    nsteps = args.rk_steps or 10
    nlon, nlat, deg = synth.ensemble_members(256)
    e = dgswe.Ensemble(nlon, nlat, deg)
    t_init = time.perf_counter()
    for k in range(e.members):
        e.set_state(k, member_state(nlon[k], nlat[k], deg[k], synth.ensemble_member_seed(k)))
    t_init = time.perf_counter() - t_init
    e.set_dt([e.max_dt(k, CFL) for k in range(e.members)])
    e.set_option(dgswe.OPT_STREAM, stream.cuda_stream)
    e.set_option(dgswe.OPT_STEPS_PER_GRAPH, nsteps)
    tile_rows, bps, tuned_ms = e.autotune(trials=2)
    m0 = e.total_mass(0)
    dof = e.total_dof
    times = []
    launches0 = e.stage_launches()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            for it in range(args.warmup + args.steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                e.step(nsteps)
                b.record(stream)
                if it >= args.warmup:
                    times.append((a, b))
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in times]
    launches = (e.stage_launches() - launches0) * args.steps // (args.steps + args.warmup)
    value, total_ms = whole_job(world, dof * 3 * nsteps * args.steps, sum(ms))
    peak, peak_kind = peaks()
    bytes_per_launch = dof * 4 * 8.0 / 3.0
    launch_s = sum(ms) * 1e-3 / max(1, launches)
    achieved = bytes_per_launch / launch_s / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": ENSEMBLE_DESC, "members": e.members, "dof": dof, "rk_steps_per_step": nsteps,
                   "tile_rows": tile_rows, "blocks_per_sm": bps, "autotune_ms_per_step": tuned_ms,
                   "init": f"each member's own seeded field, projected ({t_init:.0f} s on the host)", "cfl": CFL,
                   "l2": "inputs (1.07 GB per state array) exceed L2; flushed before every timed step"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "peak_kind": peak_kind, "kernel": "ensemble_kernel<fp32>",
                     "bytes_per_launch": bytes_per_launch, "launch_us": launch_s * 1e6},
        "gpu_launches": launches, "clocks": clk.summary(),
        "mass_drift_member0": (e.total_mass(0) - m0) / m0,
    }
    if rank == 0:
        print(json.dumps(out))


def prolong(u, r, nf):
    """Modal state of a mesh refined r x r with nf points per direction that
    represents the coarse state exactly (every coarse polynomial restricted to
    a sub-element is a polynomial of degree <= nf - 1 there): per direction
    the transfer T[s][a_f][a_c] = int L_af(x) L_ac((x + 2s + 1)/r - 1) dx,
    exact with an nf-point Gauss rule.  u: [nlat, nlon, 3, nc^2]."""
    from numpy.polynomial import legendre as npleg

    nlat, nlon, nfld, ncp = u.shape
    nc = int(round(math.sqrt(ncp)))
    x, w = npleg.leggauss(max(nf, nc) + 1)

    def L(k, t):
        c = np.zeros(k + 1)
        c[k] = 1.0
        return math.sqrt((2 * k + 1) / 2.0) * npleg.legval(t, c)

    T = np.array([[[np.sum(w * L(af, x) * L(ac, (x + 2 * sub + 1) / r - 1)) for ac in range(nc)] for af in range(nf)]
                  for sub in range(r)])                                   # [r][nf][nc]
    uc = u.reshape(nlat, nlon, nfld, nc, nc)                              # [j][i][f][b][a]
    uf = np.einsum("yBb,xAa,jifba->jyixfBA", T, T, uc)                   # [j][sy][i][sx][f][B][A]
    return np.ascontiguousarray(uf.reshape(nlat * r, nlon * r, nfld, nf * nf))


def accuracy_leg(name, precisions, make64, make_prec):
    """(i) and (ii) of "at stated L2 error" for one workload, per field.
    (ii), the FP64 discretisation error: the FP64 solution after the
    workload's steps against the FP64 solution on the 2x refined mesh at
    degree 4 (the finer discretisation of the same seeded field, projected
    there, advanced to the same time with its own CFL step), both as
    functions: the coarse solution is prolonged exactly onto the fine mesh
    and the relative L2 norm of the difference is taken over the fine modal
    coefficients (orthonormal basis, uniform element Jacobian in (lambda,
    theta)).  It includes the coarse mesh's approximation error of the field.
    (i), the precision error: relative L2 of each precision's state against
    the FP64 state on the same mesh.  A precision matches where
    (i) <= 0.1 (ii)."""
    from paper_2303_11767_gb300 import synth

    nlon, nlat, p, nsteps, seed, desc = WORKLOADS[name]
    s64 = make64(nlon, nlat, p)
    u0 = initial_state(s64, seed)
    s64.set_state(u0)
    dt = s64.max_dt(CFL)
    T = nsteps * dt
    s64.step(nsteps, dt)
    u64 = s64.get_state()
    s64.close()
    t0 = time.perf_counter()
    fine = make64(2 * nlon, 2 * nlat, 4)
    fine.set_state(fine.project_grid(synth.SmoothField(seed, fine.radius).fields_grid))
    t_proj = time.perf_counter() - t0
    dtf = fine.max_dt(CFL)
    mf = int(math.ceil(T / dtf))
    fine.step(mf, T / mf)
    uf = fine.get_state()
    fine.close()
    ref_s = time.perf_counter() - t0
    ii = field_errors(prolong(u64, 2, 5), uf)
    out = {"workload": desc, "T_s": T, "steps": nsteps,
           "reference": f"FP64 on {2 * nlon}x{2 * nlat} degree 4 from its own projection of the field "
                        f"({mf} steps of {T / mf:.3e} s; {ref_s:.1f} s incl. {t_proj:.1f} s projection); "
                        f"coarse solution prolonged exactly onto it",
           "fields": ["h", "hu", "hv"], "ii_fp64_discretisation": ii, "i_vs_fp64": {}, "matches": {}}
    for prec in precisions:
        sv = make_prec(nlon, nlat, p, prec)
        sv.set_state(u0)
        sv.step(nsteps, dt)
        e = field_errors(sv.get_state(), u64)
        sv.close()
        out["i_vs_fp64"][prec] = e
        out["matches"][prec] = [bool(a <= 0.1 * b) for a, b in zip(e, ii)]
    return out


def streaming_leg(prec, torch, stream, flush, make_prec, reps=3, nsteps=20):
    """Per-launch time of the stage kernel on the 1440 x 720 degree-4 mesh,
    whose state arrays (311 MB each in FP32) stream from HBM every stage:
    CUDA events around graph replays of nsteps SSP-RK3 steps, L2 flushed
    before each; the mean launch time over all launches of the timed reps."""
    nlon, nlat, p, _, seed, desc = WORKLOADS["r1"]
    s = make_prec(nlon, nlat, p, prec, nsteps)
    s.set_state(initial_state(s, seed))
    dt = s.max_dt(CFL)
    l0 = s.stage_launches()
    ms = []
    with torch.cuda.stream(stream):
        for it in range(1 + reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.step(nsteps, dt)
            b.record(stream)
            b.synchronize()
            if it:
                ms.append(a.elapsed_time(b))
    launches = (s.stage_launches() - l0) * reps // (reps + 1)
    s.close()
    dof = 3 * (p + 1) ** 2 * nlon * nlat
    launch_s = sum(ms) * 1e-3 / launches
    bpl = dof * 4 * 8.0 / 3.0
    return {"workload": desc, "dof": dof, "launch_us": launch_s * 1e6, "bytes_per_launch": bpl,
            "achieved": bpl / launch_s / 1e9, "value": dof / launch_s, "launches": launches,
            "kernel": KERNELS[prec].format(n=p + 1)}


def run_bands(args, world, rank, local):
    """The latitude-band decomposition on one GPU: the workload's mesh as
    args.bands bands, each an independent handle (dg_create_band), their
    boundary rows exchanged before every stage by device copies on one stream
    (bands.LocalExchange), every stage launched per band (dg_band_stage),
    against the whole-mesh solver (graph replay) in the same run.  Measures
    what the decomposition itself costs: the exchange and the per-band
    launches."""
    import torch

    from paper_2303_11767_gb300 import bands, dgswe

    nlon, nlat, p, nsteps, seed, desc = WORKLOADS[args.workload]
    if args.rk_steps:
        nsteps = args.rk_steps
    dof = 3 * (p + 1) ** 2 * nlon * nlat
    torch.cuda.set_device(local)
    dgswe.set_device(local)
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    whole = dgswe.Solver(nlon, nlat, p, precision=args.precision, check_finite=False)
    whole.set_option(dgswe.OPT_STREAM, stream.cuda_stream)
    whole.set_option(dgswe.OPT_STEPS_PER_GRAPH, min(nsteps, 1024))
    u0 = initial_state(whole, seed)
    whole.set_state(u0)
    dt = whole.max_dt(CFL)
    rows = [bands.band_rows(nlat, args.bands, k) for k in range(args.bands)]
    bs = [dgswe.Solver.band(nlon, nlat, jb, je, p, precision=args.precision, check_finite=False) for jb, je in rows]
    ex = bands.LocalExchange(bs, torch, torch.float64 if args.precision == "fp64" else torch.float32, stream)
    href = bands.reference_depth(None, u0[:, :, 0, 0], 0, 1, torch)
    for b, (jb, je) in zip(bs, rows):
        if args.precision != "fp64":
            b.set_reference_depth(href)
        b.set_state(u0[jb:je])

    def timed(fn):
        ms = []
        with torch.cuda.stream(stream):
            for it in range(args.warmup + args.steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                if it >= args.warmup:
                    ms.append(a.elapsed_time(b))
        return ms

    t_whole = timed(lambda: whole.step(nsteps, dt))
    t_bands = timed(lambda: bands.advance(bs, ex, nsteps, dt, 3))
    same = bool(np.array_equal(np.concatenate([b.get_state() for b in bs], axis=0), whole.get_state())) \
        if args.warmup + args.steps > 0 else None
    v_whole = dof * 3 * nsteps * len(t_whole) / (sum(t_whole) * 1e-3)
    v_bands = dof * 3 * nsteps * len(t_bands) / (sum(t_bands) * 1e-3)
    msg = 2 * bs[0].halo_len * (4 if args.precision != "fp64" else 8)
    out = {
        "metric": METRIC, "value": v_bands, "unit": "DOF-updates/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(t_bands) / len(t_bands), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": desc, "bands": args.bands, "rows": rows, "rk_steps_per_step": nsteps,
                   "exchange": "device copies on one stream, before every stage",
                   "bytes_per_boundary_per_stage": msg},
        "whole_mesh": {"value": v_whole, "ms_per_step": sum(t_whole) / len(t_whole)},
        "bands_over_whole": v_bands / v_whole,
        "bands_equal_whole_bitwise": same,
    }
    print(json.dumps(out))


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "c4":
        run_ensemble(args, world, rank, local)
        return
    if args.bands:
        run_bands(args, world, rank, local)
        return
    import torch

    from paper_2303_11767_gb300 import dgswe, synth

    nlon, nlat, p, nsteps, seed, desc = WORKLOADS[args.workload]
    if args.rk_steps:
        nsteps = args.rk_steps
    dof = 3 * (p + 1) ** 2 * nlon * nlat
    torch.cuda.set_device(local)
    dgswe.set_device(local)
    stream = torch.cuda.Stream()   # shared by the solver, the L2 flush and the events
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    mass_t = torch.zeros(1, dtype=torch.float64, device="cuda")

    def make_mesh(nx, ny, pp, prec, steps_per_graph):
        sv = dgswe.Solver(nx, ny, pp, precision=prec, check_finite=False)
        sv.set_option(dgswe.OPT_STREAM, stream.cuda_stream)
        sv.set_option(dgswe.OPT_STEPS_PER_GRAPH, min(max(steps_per_graph, 1), 1024))
        return sv

    def make(prec):
        return make_mesh(nlon, nlat, p, prec, nsteps)

    s = make(args.precision)
    u0 = initial_state(s, seed)
    s.set_state(u0)
    dt = s.max_dt(CFL)
    m0 = s.total_mass()

    # ---- device-timed leg
    torch.cuda.synchronize()
    barrier(world)
    launches0 = s.stage_launches()
    with ClockSampler(local) as clk:
        times = time_device(s, torch, stream, nsteps, dt, args.steps, args.warmup, mass_t, flush)
    launches = s.stage_launches() - launches0
    barrier(world)
    value, total_ms = whole_job(world, dof * 3 * nsteps * args.steps, sum(times))
    stage_launches_timed = launches * args.steps // (args.steps + args.warmup)
    m1 = s.total_mass()
    s.set_option(dgswe.OPT_CHECK_FINITE, 1)
    s.step(1, dt)                                          # raises if any stage met NaN / h <= 0
    ms_per_step = total_ms / args.steps

    # the fused stage on this workload; algorithmic bytes per launch = the mean
    # 8/3 state words per DOF of SSP-RK3 (u read by all stages, u^n by two, one write)
    word = 8 if args.precision == "fp64" else 4
    bytes_per_launch = dof * word * 8.0 / 3.0
    launch_s = (sum(times) * 1e-3) / max(1, stage_launches_timed)
    peak, peak_kind = peaks()
    achieved = bytes_per_launch / launch_s / 1e9
    traffic = TRAFFIC.get((args.precision, args.workload))
    roofline_here = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic[0] if traffic else None,
                     "traffic_note": traffic[1] if traffic else "no capture of this kernel and workload",
                     "peak_kind": peak_kind, "kernel": KERNELS[args.precision].format(n=p + 1),
                     "bytes_per_launch": bytes_per_launch, "launch_us": launch_s * 1e6, "workload": desc}

    out = {
        "metric": METRIC, "value": value, "unit": "DOF-updates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.precision], "data": "synthetic",
        "config": {"workload": desc, "nlon": nlon, "nlat": nlat, "degree": p, "dof": dof,
                   "rk_steps_per_step": nsteps, "dt": dt, "cfl": CFL, "l2": "flushed before every timed step",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline_here,
        # + the two mass kernels per step; the tensor-core path also permutes
        # u^n (base and low parts) into and out of its lane-contiguous layout
        # once per graph of up to 1024 steps
        "gpu_launches": stage_launches_timed + (6 if args.precision in TC_PRECS else 2) * args.steps,
        "clocks": clk.summary(),
        "mass_drift": (m1 - m0) / m0,
    }

    if not args.no_extras and rank == 0 and world == 1:
        def make_prec(nx, ny, pp, prec, steps_per_graph=64):
            return make_mesh(nx, ny, pp, prec, steps_per_graph)

        # ---- the roofline: the same kernel on the mesh that streams from HBM
        if args.workload != "r1" and args.precision != "fp64":
            leg = streaming_leg(args.precision, torch, stream, flush, make_prec)
            tr = TRAFFIC.get((args.precision, "r1"))
            out["roofline"] = {"bound": "hbm", "achieved": leg["achieved"], "peak": peak, "unit": "GB/s",
                               "frac": leg["achieved"] / peak, "traffic": tr[0] if tr else None,
                               "traffic_note": tr[1] if tr else "no capture of this kernel and workload",
                               "peak_kind": peak_kind, "kernel": leg["kernel"],
                               "bytes_per_launch": leg["bytes_per_launch"], "launch_us": leg["launch_us"],
                               "workload": leg["workload"], "value": leg["value"]}
            out["roofline_timed_workload"] = dict(roofline_here, note="state arrays L2-resident across stages")
            for tcp in ("fp32",) + TC_PRECS:
                if tcp != args.precision:
                    lv = streaming_leg(tcp, torch, stream, flush, make_prec)
                    tr = TRAFFIC.get((tcp, "r1"))
                    out.setdefault("roofline_variants", {})[tcp] = {
                        "achieved": lv["achieved"], "frac": lv["achieved"] / peak, "launch_us": lv["launch_us"],
                        "value": lv["value"], "kernel": lv["kernel"], "traffic": tr[0] if tr else None,
                        "workload": lv["workload"]}

        # ---- FP64 plain path on the same workload
        s64 = make("fp64")
        s64.set_state(u0)
        k64 = max(2, args.steps // 5)
        t64 = time_device(s64, torch, stream, nsteps, dt, k64, 1, mass_t, flush)
        s64.close()
        v64 = dof * 3 * nsteps * k64 / (sum(t64) * 1e-3)
        fp64_peak = dgswe.measure_fp64_peak(5)
        fpd = stage_flops_per_dof(p + 1)
        out["fp64_plain"] = {"value": v64, "ms_per_step": sum(t64) / k64, "dtype": "f64", "steps": k64,
                             "speedup_of_value": value / v64,
                             "roofline": {"bound": "alu", "achieved": v64 * fpd / 1e9, "peak": fp64_peak,
                                          "unit": "GFLOP/s", "frac": v64 * fpd / 1e9 / fp64_peak,
                                          "peak_kind": "measured FP64 FMA probe (dg_measure_fp64_peak)",
                                          "flops_per_dof": fpd}}

        # ---- the tensor-core precisions on the same workload (device-timed)
        for tcp in ("fp32",) + TC_PRECS:
            if tcp == args.precision:
                continue
            stc = make(tcp)
            stc.set_state(u0)
            ktc = max(2, args.steps // 5)
            ttc = time_device(stc, torch, stream, nsteps, dt, ktc, 1, mass_t, flush)
            stc.close()
            vtc = dof * 3 * nsteps * ktc / (sum(ttc) * 1e-3)
            out.setdefault("variants", {})[tcp] = {"value": vtc, "ms_per_step": sum(ttc) / ktc,
                                                   "dtype": DTYPES[tcp], "steps": ktc,
                                                   "kernel": KERNELS[tcp].format(n=p + 1)}

        # ---- the 180 x 90 degree-3 workload, FP32 (kept beside the headline)
        if args.workload != "c2":
            n2, l2_, p2, ns2, sd2, desc2 = WORKLOADS["c2"]
            sc2 = make_mesh(n2, l2_, p2, "fp32", ns2)
            sc2.set_state(initial_state(sc2, sd2))
            dt2 = sc2.max_dt(CFL)
            t2 = time_device(sc2, torch, stream, ns2, dt2, max(2, args.steps // 5), 1, mass_t, flush)
            sc2.close()
            dof2 = 3 * (p2 + 1) ** 2 * n2 * l2_
            out["workload_c2"] = {"workload": desc2, "value": dof2 * 3 * ns2 * len(t2) / (sum(t2) * 1e-3),
                                  "dtype": "f32", "ms_per_step": sum(t2) / len(t2)}

        # ---- the learned correction's coarse solver (72x36 degree 1, FP32),
        #      plain and with the per-element network attached: random-init
        #      weights, input statistics of the synthetic state and a source
        #      scaled far below the tendency (the state keeps its trajectory),
        #      so the difference is what the network's inference costs
        from paper_2303_11767_gb300 import learned

        n5, l5, p5 = learned.COARSE
        ns5, sd5 = 200, 5
        legs5 = {}
        for with_mlp in (False, True):
            sc5 = make_mesh(n5, l5, p5, "fp32", ns5)
            u5 = initial_state(sc5, sd5)
            sc5.set_state(u5)
            dt5 = sc5.max_dt(learned.CFL_COARSE)
            net = None
            if with_mlp:
                net = dgswe.MLP(seed=sd5)
                X = learned.gather_inputs(u5)
                xs = X.std(axis=0)
                xs[xs == 0] = 1.0
                ys = 1e-12 * np.abs(u5).reshape(-1, 12).max(axis=0) + 1e-30
                net.set_normalization(X.mean(axis=0), xs, np.zeros(12), ys)
                sc5.attach_mlp(net)
            t5 = time_device(sc5, torch, stream, ns5, dt5, max(2, args.steps // 5), 1, mass_t, flush)
            sc5.close()
            if net is not None:
                net.close()
            dof5 = 3 * (p5 + 1) ** 2 * n5 * l5
            legs5["learned" if with_mlp else "plain"] = {
                "value": dof5 * 3 * ns5 * len(t5) / (sum(t5) * 1e-3), "ms_per_step": sum(t5) / len(t5)}
        out["workload_c5"] = {"workload": f"{n5}x{l5} elements, degree {p5}, SSP-RK3, {ns5} steps per bench "
                                          f"step, seed {sd5}; learned = the same with the per-element network "
                                          "60-128-128-12 attached (random-init weights)",
                              "dtype": "f32", **legs5,
                              "learned_over_plain_time": legs5["learned"]["ms_per_step"] / legs5["plain"]["ms_per_step"]}

        # ---- the paper's own timing workload (planar geostrophic adjustment,
        #      50x50 elements, 360 RK4 steps of 100 s), FP64 planar kernel, with
        #      the paper's CPU throughput derived from its table as context
        paper = {1: 2.85e6, 2: 1.23e6, 3: 4.02e5}
        legs = {}
        for pp in (1, 2, 3):
            sp = dgswe.Solver.plane_swe(50, 50, pp)
            sp.set_option(dgswe.OPT_STREAM, stream.cuda_stream)
            sp.set_option(dgswe.OPT_STEPS_PER_GRAPH, 360)
            sp.set_option(dgswe.OPT_CHECK_FINITE, 0)
            u_pl = sp.project_grid(synth.geostrophic_adjustment_grid())
            ts = []
            for it in range(4):
                sp.set_state(u_pl)
                with torch.cuda.stream(stream):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    sp.step(360, 100.0)
                    b.record(stream)
                b.synchronize()
                if it:
                    ts.append(a.elapsed_time(b))
            dof_pl = 2500 * 3 * (pp + 1) ** 2
            v_pl = dof_pl * 4 * 360 / (min(ts) * 1e-3)
            legs[f"p{pp}"] = {"value": v_pl, "ms_per_run": min(ts), "paper_cpu_value": paper[pp],
                              "ratio_to_paper_cpu": v_pl / paper[pp]}
            sp.close()
        out["paper_workload"] = {"workload": "planar SWE geostrophic adjustment (Sec. 4.3), 50x50 elements, "
                                             "360 RK4 steps of 100 s, FP64, one-thread-per-element planar kernel",
                                 "unit": "DOF-updates/s", "paper_hardware": "12-core Xeon E5-2690 v3 (CPU only; "
                                 "throughput derived from its total-time table)", **legs}

        # ---- end to end through the C-ABI with pinned host buffers
        hin = torch.empty(s.state_len, dtype=torch.float64, pin_memory=True).numpy()
        hout = torch.empty(s.state_len, dtype=torch.float64, pin_memory=True).numpy()
        hin[:] = u0.reshape(-1)
        se = make(args.precision)
        se.set_option(dgswe.OPT_CHECK_FINITE, 1)
        for it in range(args.warmup + args.steps):
            if it == args.warmup:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            se.set_state(hin)
            se.step(nsteps, dt)
            mass = se.total_mass()
            hout[:] = se.get_state().reshape(-1)
        e2e_s = time.perf_counter() - t0
        se.close()
        out["e2e"] = {"value": dof * 3 * nsteps * args.steps / e2e_s, "unit": "DOF-updates/s",
                      "h2d_bytes_per_step": int(hin.nbytes), "d2h_bytes_per_step": int(hout.nbytes) + 8,
                      "ms_per_step": 1e3 * e2e_s / args.steps, "mass": mass}

        # ---- at stated L2 error: (i) and (ii) on this workload and on 180x90 p = 3
        precs = ["fp32", *TC_PRECS]
        acc = {args.workload: accuracy_leg(args.workload, precs, lambda a, b, c: make_mesh(a, b, c, "fp64", 256),
                                           lambda a, b, c, d: make_mesh(a, b, c, d, 256))}
        if args.workload != "c2":
            acc["c2"] = accuracy_leg("c2", precs, lambda a, b, c: make_mesh(a, b, c, "fp64", 256),
                                     lambda a, b, c, d: make_mesh(a, b, c, d, 256))
        out["at_l2_error"] = acc

        # ---- the oracle on the host cores (bounded sample) and the L2 error
        leg = cpu_leg(nlon, nlat, p, seed, budget_s=15.0, max_steps=nsteps)
        cpu_value = dof * 3 * leg["nsteps"] / leg["wall"]
        o1 = leg["o"]
        o1.set_threads(1)
        t0 = time.perf_counter()
        for _ in range(3):
            o1.rhs(leg["u0"])
        single = 3 * dof / (time.perf_counter() - t0)
        out["cpu_baseline"] = {"value": cpu_value, "unit": "DOF-updates/s", "cores": leg["cores"], "kind": "oracle",
                               "sample": f"{leg['nsteps']} SSP-RK3 steps of the same workload "
                                         f"({3 * leg['nsteps']} stages), FP64, {leg['cores']} threads",
                               "seconds": leg["wall"], "cpu": cpu_model(),
                               "single_thread": {"value": single, "sample": "3 right-hand sides, 1 thread"}}
        errs = {}
        for prec in sorted({"fp32", "fp64", *TC_PRECS, args.precision}):
            sv = make(prec)
            sv.set_state(leg["u0"])
            sv.step(leg["nsteps"], leg["dt"])
            errs[prec] = field_errors(sv.get_state(), leg["u1"])
            sv.close()
        out["l2_error_vs_oracle"] = {"steps": leg["nsteps"], "fields": ["h", "hu", "hv"], **errs}
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
