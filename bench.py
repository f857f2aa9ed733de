"""Benchmark of the fused collide-and-stream step (MLUPS and fraction of the HBM roofline).

Default workload: the large periodic anisotropic decaying flow, 512 x 256 x 256 nodes,
r_y = r_z = 0.5, cs2 = 1/12, nu = 0.005, omega_xi = 1, seeded random solenoidal
velocity (Gaussian spectrum peak k = 4, u_rms = 0.03), FP32 arithmetic; populations
stored as FP32 (the headline value) and as shifted FP32 / BF16 / FP16 (reported
beside it with their velocity error against the FP64 path).

One step = one fused launch over the whole lattice.  The working set (2 x 27 x N
stored values, >= 3.6 GB) is far larger than L2, so no explicit flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With --gpus N > 1 (launched by torchrun) every rank runs an independent replica of
the workload on its own GPU ("replicas only": the update has no collective);
value = total node updates of all ranks / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "MLUPS and % of HBM roofline, plain FP32 vs reduced-precision storage at stated error"
WORKLOADS = {
    "decaying": dict(workload="decaying anisotropic flow 512x256x256, r_y=0.5, r_z=0.5 (periodic)",
                     nx=512, ny=256, nz=256, r_y=0.5, r_z=0.5, cs2=1.0 / 12.0, nu=0.005, omega_xi=1.0,
                     init="seeded solenoidal velocity, spectrum peak k=4, u_rms=0.03, seed 3", corr="local",
                     walls="", force=(0.0, 0.0, 0.0)),
    "channel": dict(workload="wall-bounded channel 768x192x384, r_y=0.25, r_z=1 (walls y, periodic x z)",
                    nx=768, ny=192, nz=384, r_y=0.25, r_z=1.0, cs2=1.0 / 48.0, nu=0.005, omega_xi=1.0,
                    init="laminar Poiseuille u_max=0.02 plus seeded wall-damped solenoidal perturbation of 5 %, "
                         "seed 5; F_x = 8 nu u_max / h^2", corr="local", walls="y", force=None),
}
WORKLOAD = dict(WORKLOADS["decaying"])
STORAGE_BYTES = {"f64": 8, "f32": 4, "f32s": 4, "f16s": 2, "bf16s": 2}


def variant_options(var: str) -> dict:
    """A bench variant is a storage form with optional suffixes: "+sr" stochastic
    rounding of 16-bit stores, "+full" the FULL corrections (density-gradient terms),
    "+pN" the lattice updated as N z-slabs exchanging one-plane halos (same results)."""
    parts = var.split("+")
    sub = [int(p[1:]) for p in parts[1:] if p.startswith("p") and p[1:].isdigit()]
    return {"storage": parts[0], "rounding": "stochastic" if "sr" in parts[1:] else "nearest",
            "corr": "full" if "full" in parts[1:] else None, "subdomains": sub[0] if sub else 1}


def bytes_per_node(var: str) -> int:
    """Algorithmic HBM bytes per node-update: 27 populations read and written; FULL adds
    the density field (compute type) written once and read once (its 6 face neighbours
    reused from cache); a per-node force field would add 12 B (not in the bench workloads)."""
    o = variant_options(var)
    b = 2 * 27 * STORAGE_BYTES[o["storage"]]
    if o["corr"] == "full":      # the density field is held in the compute type
        b += 2 * (8 if o["storage"] == "f64" else 4)
    return b
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch from one ncu
# capture of the named kernel on the 512x128x128 decaying-flow case, scaled by the node
# count; only reported for the kernel those counters were taken on.
TRAFFIC_PER_NODE = {("decaying", "k_step_pair<F32,LOCAL,1,false,periodic>"): (906.026496e6 + 855.318784e6) / 8388608}
VARIANTS = ["f32", "f32s", "bf16s", "f16s", "bf16s+sr", "f16s+sr", "f32+full", "f32+p4"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=5)

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                smax.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def allreduce_max(x: float, dev=None) -> float:
    """Maximum of x over the ranks of the default process group (x itself without one).
    NCCL reduces a device tensor, gloo a host tensor."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    on_dev = dist.get_backend() == "nccl"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev if on_dev else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(nodes_per_rank: int, steps: int, world: int, seconds_max: float) -> float:
    """Whole-job throughput: node updates of all ranks over the slowest rank's time."""
    return nodes_per_rank * steps * world / seconds_max / 1e6


def make_inputs():
    w = WORKLOAD
    if w["walls"] == "y":
        rho, u, fx = synth.channel(w["nx"], w["ny"], w["nz"], w["r_y"], w["r_z"], 0.02, w["nu"], 0.05, seed=5)
        w["force"] = (fx, 0.0, 0.0)
        return rho, u
    rho, u = synth.solenoidal_random(w["nx"], w["ny"], w["nz"], w["r_y"], w["r_z"], 4.0, 0.03, seed=3)
    return rho, u


def run_ours(args, rank, world):
    import torch

    from paper_2107_14774_gb300 import Lattice

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = WORKLOAD
    dims = (w["nx"], w["ny"], w["nz"])
    N = w["nx"] * w["ny"] * w["nz"]
    rho, u = make_inputs()
    rho_t = torch.from_numpy(rho.astype(np.float32)).to(dev)
    u_t = torch.from_numpy(u.astype(np.float32)).to(dev)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.Stream(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

    def barrier():
        if dist is not None:
            dist.barrier()

    variants = args.variants.split(",")
    results = {}
    kernel_ms = {}
    kernel_names = {}
    for var in variants:
        vo = variant_options(var)
        lat = Lattice(*dims, r_y=w["r_y"], r_z=w["r_z"], nu=w["nu"], cs2=w["cs2"], storage=vo["storage"],
                      corr=vo["corr"] or w["corr"], stream=stream, device=dev, kernel=args.kernel,
                      walls=w["walls"], force=w["force"], rounding=vo["rounding"], subdomains=vo["subdomains"])
        with torch.cuda.stream(stream):
            lat.init(rho_t, u_t)
            lat.step(args.warmup)
        stream.synchronize()
        barrier()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        with ClockSampler(dev.index) as clk:
            ev0.record(stream)
            lat.step(args.steps)
            ev1.record(stream)
            ev1.synchronize()
        torch.cuda.synchronize(dev)
        ms = allreduce_max(ev0.elapsed_time(ev1), dev)
        kernel_ms[var] = ms / args.steps
        kernel_names[var] = lat.step_kernel
        results[var] = {"mlups": aggregate_mlups(N, args.steps, world, ms * 1e-3), "ms_per_step": ms / args.steps,
                        "clocks": clk.summary(), "kernel": kernel_names[var]}
        lat.close()
        del lat
        torch.cuda.empty_cache()
    barrier()

    # velocity error of each storage form against the FP64 path after the same steps,
    # at each checkpoint; an FP64 run from an initial velocity perturbed by a seeded
    # solenoidal field of 1e-6 relative amplitude (the spectrum of the flow itself)
    # measures how much the flow amplifies a perturbation of its energetic scales
    checkpoints = sorted({int(v) for v in str(args.error_steps).split(",") if int(v) > 0})
    if not checkpoints:
        for var in variants:
            results[var]["u_rel_err_vs_f64"] = None
        return results, kernel_ms, run_e2e(args, rho, u, dims, stream, dev, world, barrier), N

    def trajectory(storage, u0, kern, cps=None):
        cps = checkpoints if cps is None else cps
        torch.cuda.synchronize(dev)   # inputs were made on the current stream; the lattice uses `stream`
        vo = variant_options(storage)
        lat = Lattice(*dims, r_y=w["r_y"], r_z=w["r_z"], nu=w["nu"], cs2=w["cs2"], storage=vo["storage"],
                      corr=vo["corr"] or w["corr"], stream=stream, device=dev, kernel=kern,
                      walls=w["walls"], force=w["force"], rounding=vo["rounding"])
        out, done = [], 0
        with torch.cuda.stream(stream):
            lat.init(rho_t.to(lat.dtype), u0.to(lat.dtype))
            for cp in cps:
                lat.step(cp - done)
                done = cp
                out.append(lat.moments()[1].double())
        lat.close()
        return out

    def errors(us, ref):
        """u_rel_l2 = |u - u_ref| / |u_ref| (the error the precision target is stated in);
        amp = <u - u_ref, u_ref> / |u_ref|^2, the part of it along the flow (an amplitude
        error, e.g. a systematic gain or loss of momentum per step); u2_mean_rel = the
        relative error of the mean kinetic energy."""
        res = {}
        for cp, a, b in zip(checkpoints, us, ref):
            ke_a, ke_b = float((a * a).sum()), float((b * b).sum())
            res[str(cp)] = {"u_rel_l2": float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)),
                            "amp": float(((a - b) * b).sum()) / ke_b, "u2_mean_rel": abs(ke_a / ke_b - 1.0)}
        return res

    ref = trajectory("f64", u_t.double(), "auto")
    up = torch.from_numpy(synth.solenoidal_random(w["nx"], w["ny"], w["nz"], w["r_y"], w["r_z"], 4.0, 0.03,
                                                  seed=99)[1]).to(dev)
    ccp = [cp for cp in checkpoints if cp <= 1000] or checkpoints[:1]
    control = errors(trajectory("f64", u_t.double() + 1e-6 * up, "auto", ccp), ref)
    del up
    for var in variants:
        vo = variant_options(var)
        if vo["corr"] is not None or vo["subdomains"] > 1:
            # another scheme than the FP64 reference's; or the same state as the undecomposed
            # variant bit for bit (the slab decomposition changes no arithmetic)
            results[var]["u_rel_err_vs_f64"] = None
            continue
        results[var]["u_rel_err_vs_f64"] = errors(trajectory(var, u_t, args.kernel), ref)
    results["_control_f64_perturbed_1e-6"] = control
    del ref
    torch.cuda.empty_cache()
    return results, kernel_ms, run_e2e(args, rho, u, dims, stream, dev, world, barrier), N


def run_e2e(args, rho, u, dims, stream, dev, world, barrier):
    """End-to-end MLUPS through the public API with pinned host buffers."""
    import torch

    from paper_2107_14774_gb300 import Lattice
    if args.no_e2e:
        return None
    w = WORKLOAD
    N = dims[0] * dims[1] * dims[2]
    dist = None
    if world > 1:
        import torch.distributed as dist
    # end to end through the public API with pinned host buffers: every step copies its
    # inputs (rho, u) host->device (lb_init), runs one fused step and reads the resulting
    # fields device->host (lb_moments).  Measured two ways: one context doing that
    # serially, and D contexts on their own streams taking the steps in turn, so that the
    # upload of one step overlaps the download and compute of the steps before it
    # (independent inputs streamed through the library, each step with its own copies in
    # both directions).
    D = max(1, args.e2e_contexts)
    rho_h = torch.from_numpy(rho.astype(np.float32)).pin_memory()
    u_h = torch.from_numpy(u.astype(np.float32)).pin_memory()
    outs = [(torch.empty_like(rho_h).pin_memory(), torch.empty_like(u_h).pin_memory()) for _ in range(D)]
    streams = [stream] + [torch.cuda.Stream(dev) for _ in range(D - 1)]
    lats = [Lattice(*dims, r_y=w["r_y"], r_z=w["r_z"], nu=w["nu"], cs2=w["cs2"], storage="f32", corr=w["corr"],
                    stream=s, device=dev, kernel=args.kernel, walls=w["walls"], force=w["force"]) for s in streams]
    e2e_steps = max(4, min(args.steps, 20))

    def serial(n):
        for _ in range(n):
            lats[0].init(rho_h, u_h).step(1).moments(*outs[0])

    def pipelined(n):
        for i in range(n + D - 1):
            if i < n:
                lats[i % D].init(rho_h, u_h).step(1)          # asynchronous: upload, step
            j = i - (D - 1)
            if j >= 0:
                lats[j % D].moments(*outs[j % D])              # download of step j, waits for it

    # the host link alone, without the library: one step's bytes up, down, and both at once
    up = (torch.empty(rho_h.shape, dtype=rho_h.dtype, device=dev), torch.empty(u_h.shape, dtype=u_h.dtype, device=dev))
    down = (torch.zeros_like(up[0]), torch.zeros_like(up[1]))
    side = torch.cuda.Stream(dev)

    def h2d():
        with torch.cuda.stream(streams[0]):
            up[0].copy_(rho_h, non_blocking=True)
            up[1].copy_(u_h, non_blocking=True)

    def d2h():
        with torch.cuda.stream(side):
            outs[0][0].copy_(down[0], non_blocking=True)
            outs[0][1].copy_(down[1], non_blocking=True)

    def copies(*fns):
        def run(n):
            for _ in range(n):
                for f in fns:
                    f()
                torch.cuda.synchronize(dev)
        return run

    timings = {}
    for name, fn in (("serial", serial), ("pipelined", pipelined), ("h2d", copies(h2d)), ("d2h", copies(d2h)),
                     ("both", copies(h2d, d2h))):
        fn(D + 1)                                      # every context has staged and stepped once
        barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        fn(e2e_steps)
        torch.cuda.synchronize(dev)
        timings[name] = allreduce_max(time.perf_counter() - t0, dev)
    for lat in lats:
        lat.close()
    del up, down
    per_step = {k: 1e3 * v / e2e_steps for k, v in timings.items()}
    e2e = {"value": aggregate_mlups(N, e2e_steps, world, timings["pipelined"]), "unit": "MLUPS",
           "h2d_bytes_per_step": 16 * N, "d2h_bytes_per_step": 16 * N, "contexts": D,
           "what": f"per step: lb_init from pinned host rho,u + lb_step(1) + lb_moments to pinned host; {D} "
                   "contexts on their own streams take the steps in turn (the upload of one step overlaps the "
                   "download and compute of the steps before it)",
           "serial": {"value": aggregate_mlups(N, e2e_steps, world, timings["serial"]), "unit": "MLUPS",
                      "what": "the same with one context, each step's copies and step in sequence"},
           "link_ms_per_step": {"h2d": per_step["h2d"], "d2h": per_step["d2h"], "both_at_once": per_step["both"]},
           "link_bound": {"value": aggregate_mlups(N, e2e_steps, world, max(timings["h2d"], timings["d2h"])),
                          "unit": "MLUPS",
                          "what": "the full-duplex bound: one step's bytes in the slower direction alone, pinned "
                                  "host <-> device copies without the library"}}
    e2e["link_frac"] = e2e["value"] / e2e["link_bound"]["value"]
    return e2e


def oracle_sample(seconds_target=15.0, cores=None):
    """The FP64 oracle as it stands, on the host cores, on a z-slab of the workload."""
    import oracle
    oracle.build()
    w = WORKLOAD
    rho, u = make_inputs()
    wn = 1.0 / (w["nu"] / w["cs2"] + 0.5)
    nzs = 8
    o = oracle.Oracle(w["nx"], w["ny"], nzs, r=w["r_y"], s=w["r_z"], cs2=w["cs2"], omega_nu=wn, omega_xi=1.0,
                      corr=oracle.CORR_LOCAL, threads=cores or 0, walls=w["walls"], force=w["force"])
    f = o.init(rho[:nzs], u[:, :nzs])
    n = w["nx"] * w["ny"] * nzs
    t0 = time.perf_counter()
    f = o.step(f)
    dt = time.perf_counter() - t0
    steps = 1
    # grow the sample to roughly the target duration
    extra = int(max(0, seconds_target / max(dt, 1e-3) - 1))
    extra = min(extra, 20)
    if extra:
        t0 = time.perf_counter()
        f = o.run(f, extra)
        dt += time.perf_counter() - t0
        steps += extra
    return {"value": n * steps / dt / 1e6, "unit": "MLUPS", "cores": o.threads, "kind": "oracle",
            "sample": f"{steps} steps of a {w['nx']}x{w['ny']}x{nzs} z-slab (periodic in z) of the workload "
                      f"(FP64 C oracle, factored form, OpenMP), {dt:.1f} s"}


def reference_steps(steps, warmup, budget_s=90.0):
    """The oracle as it stands, timed step by step on the host cores: every step is one
    oracle step of a z-slab of the workload whose thickness is chosen so that the warm-up
    and timed steps take about `budget_s` seconds in all."""
    import oracle
    oracle.build()
    w = WORKLOAD
    rho, u = make_inputs()
    wn = 1.0 / (w["nu"] / w["cs2"] + 0.5)

    def slab(nzs):
        o = oracle.Oracle(w["nx"], w["ny"], nzs, r=w["r_y"], s=w["r_z"], cs2=w["cs2"], omega_nu=wn, omega_xi=1.0,
                          corr=oracle.CORR_LOCAL, walls=w["walls"], force=w["force"])
        return o, o.init(rho[:nzs], u[:, :nzs])
    o, f = slab(1)
    t0 = time.perf_counter()
    f = o.step(f)
    per_plane = time.perf_counter() - t0
    nzs = int(max(1, min(w["nz"], budget_s / max(steps + warmup, 1) / max(per_plane, 1e-6))))
    o, f = slab(nzs)
    for _ in range(warmup):
        f = o.step(f)
    t0 = time.perf_counter()
    for _ in range(steps):
        f = o.step(f)
    dt = time.perf_counter() - t0
    n = w["nx"] * w["ny"] * nzs
    return {"value": n * steps / dt / 1e6, "unit": "MLUPS", "cores": o.threads, "kind": "oracle",
            "ms_per_step": 1e3 * dt / max(steps, 1),
            "sample": f"each step: one FP64 oracle step (C, factored form, OpenMP) of a {w['nx']}x{w['ny']}x{nzs} "
                      f"z-slab (periodic in z) of the workload; {warmup} warm-up + {steps} timed steps, {dt:.1f} s"}


def run_study(args):
    """Parameter studies of Secs. 6 and 7 through the library (FP32 storage)."""
    from paper_2107_14774_gb300 import studies
    omegas = [float(v) for v in args.omegas.split(",")]
    emit = lambda d: print(json.dumps(d), flush=True)
    t0 = time.time()
    if args.study == "stability":          # Fig. 8: U_max vs omega_nu, both schemes, cs2 = 0.08
        for (nx, ny, nz, r, s) in [(30, 40, 30, 0.75, 1.0), (30, 60, 30, 0.5, 1.0)]:
            for model in ("central", "raw"):
                for wn in omegas:
                    U = studies.max_stable_lid_velocity(nx, ny, nz, r, s, 0.08, wn, 1.0, model, args.study_steps)
                    emit({"study": "stability", "grid": [nx, ny, nz], "r": r, "s": s, "model": model,
                          "omega_nu": wn, "omega_xi": 1.0, "U_max": U, "steps": args.study_steps})
    elif args.study == "xi":               # Fig. 9: U_max vs omega_nu for omega_xi = 0.5, 1.0, 1.4
        for corr in args.study_corr.split(","):
            for wb in (0.5, 1.0, 1.4):
                for wn in omegas:
                    U = studies.max_stable_lid_velocity(30, 60, 30, 0.5, 1.0, 0.08, wn, wb, "central",
                                                        args.study_steps, corr=corr, ramp_steps=args.study_ramp)
                    emit({"study": "xi", "grid": [30, 60, 30], "r": 0.5, "s": 1.0, "model": "central",
                          "corr": corr, "omega_nu": wn, "omega_xi": wb, "U_max": U, "steps": args.study_steps,
                          "lid_ramp_steps": args.study_ramp})
    elif args.study == "reynolds":         # Fig. 10: Re_max at U = 0.2, r = 0.5, s = 1, cs2 = 0.08
        for (nx, ny, nz) in [(40, 80, 40), (50, 100, 50), (90, 180, 90)]:
            for model in ("central", "raw"):
                re = studies.max_stable_reynolds(nx, ny, nz, 0.5, 1.0, 0.08, 0.2, model, args.study_steps)
                emit({"study": "reynolds", "grid": [nx, ny, nz], "r": 0.5, "s": 1.0, "model": model, "U": 0.2,
                      "Re_max": re, "steps": args.study_steps})
    elif args.study == "channel":          # channel 768x192x384 long run, reduced-precision storage vs FP32
        import torch
        from paper_2107_14774_gb300 import Lattice
        w = WORKLOADS["channel"]
        n = (w["nx"], w["ny"], w["nz"])
        rho, u, fx = synth.channel(*n, w["r_y"], w["r_z"], 0.02, w["nu"], 0.05, seed=5)
        h = n[1] * w["r_y"]
        yw = (np.arange(n[1]) + 0.5) * w["r_y"]
        laminar = torch.from_numpy(4 * 0.02 * yw * (h - yw) / h ** 2)
        cps = sorted({int(v) for v in args.study_checkpoints.split(",")})
        rho_t = torch.from_numpy(rho.astype(np.float32)).cuda()
        u_t = torch.from_numpy(u.astype(np.float32)).cuda()
        del rho, u
        stream = torch.cuda.Stream()
        ref = {}
        for var in ["f32"] + [v for v in args.study_variants.split(",") if v != "f32"]:
            vo = variant_options(var)
            lat = Lattice(*n, r_y=w["r_y"], r_z=w["r_z"], nu=w["nu"], cs2=w["cs2"], storage=vo["storage"],
                          corr=w["corr"], stream=stream, walls=w["walls"], force=(fx, 0.0, 0.0),
                          rounding=vo["rounding"])
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                lat.init(rho_t, u_t)
            m0 = lat.reduce()
            done, t0 = 0, time.time()
            for cp in cps:
                lat.step(cp - done)
                done = cp
                m = lat.reduce()
                ut = lat.moments()[1][0].double()             # u_x [nz, ny, nx]
                prof = ut.mean(dim=(0, 2)).cpu()              # mean over x and z: u_x(y)
                rec = {"study": "channel", "variant": var, "kernel": lat.step_kernel, "step": cp,
                       "mass_drift_rel": float(m[0] / m0[0] - 1.0),
                       "profile_vs_laminar_rel_l2": float(torch.linalg.vector_norm(prof - laminar)
                                                          / torch.linalg.vector_norm(laminar)),
                       "profile_centre": float(prof[n[1] // 2]), "laminar_centre": float(laminar[n[1] // 2]),
                       "fluctuation_rms": float((ut - prof.to(ut.device)[None, :, None]).pow(2).mean().sqrt()),
                       "seconds": round(time.time() - t0, 1)}
                if var == "f32":
                    ref[cp] = lat.moments()[1].double().cpu()
                else:
                    uu = lat.moments()[1].double().cpu()
                    rec["u_rel_l2_vs_f32"] = float(torch.linalg.vector_norm(uu - ref[cp]) /
                                                   torch.linalg.vector_norm(ref[cp]))
                    del uu
                emit(rec)
            lat.close()
            torch.cuda.empty_cache()
    elif args.study == "adjoint":          # discrete adjoint, 128x64x64, T = 500, K = 50 and K = 1, FP32
        import torch
        from paper_2107_14774_gb300 import Lattice
        n, T = (128, 64, 64), 500
        rho, u = synth.solenoidal_random(*n, 1.0, 0.5, 4.0, 0.01, seed=4)
        ff = synth.force_field(*n, 1e-5, seed=44)
        lat = Lattice(*n, r_y=1.0, r_z=0.5, nu=0.01, storage="f32", stream=torch.cuda.Stream())
        lat.set_force_field(torch.from_numpy(ff).cuda())
        N = n[0] * n[1] * n[2]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
        torch.cuda.synchronize()
        ev[2].record(lat.stream)
        lat.step(T)
        ev[3].record(lat.stream)
        torch.cuda.synchronize()
        t_fwd = ev[2].elapsed_time(ev[3]) / 1e3
        # K = 50: checkpoints every 50 steps, each segment recomputed once; K = 1: all 500
        # states resident (28 GB), nothing recomputed
        for K in [int(v) for v in args.study_k.split(",")]:
            for rep in range(2):                  # the first call also pages in the allocations
                lat.init(torch.from_numpy(rho).cuda(), torch.from_numpy(u).cuda())
                torch.cuda.synchronize()
                ev[0].record(lat.stream)
                J, dJdF, dJdw = lat.adjoint_ke(T, K)
                ev[1].record(lat.stream)
                torch.cuda.synchronize()
            t_adj = ev[0].elapsed_time(ev[1]) / 1e3
            emit({"study": "adjoint", "grid": list(n), "T": T, "K": K, "J": J, "dJ_domega": list(dJdw),
                  "seconds_adjoint_total": t_adj, "seconds_forward_T_steps": t_fwd, "ratio": t_adj / t_fwd,
                  "node_steps_per_s": N * T / t_adj,
                  "stored_states": (T + K - 1) // K + K - 1})
        lat.close()
    else:                                  # Sec. 6: shallow cavity, cubic vs cuboid, Re = 100, Ma = 0.1
        cubic = studies.shallow_cavity(256, 64, 128, 1.0, 1.0, 1 / 3, 0.1 * (1 / 3) ** 0.5)
        emit({"study": "cavity", "lattice": "cubic 256x64x128", "r": 1.0, "s": 1.0, "cs2": 1 / 3,
              "nodes": cubic["nodes"], "steps": cubic["steps"], "seconds": cubic["seconds"], "stable": cubic["stable"],
              "u_min": float(cubic["u"].min()), "v_max": float(cubic["v"].max()), "v_min": float(cubic["v"].min())})
        for (nx, nz, r, s) in [(104, 40, 0.406, 1.3), (96, 64, 0.375, 0.75), (96, 48, 0.375, 1.0)]:
            c = studies.shallow_cavity(nx, 64, nz, r, s, 0.04, 0.1 * 0.2)
            du = float(np.max(np.abs(np.interp(c["y"], cubic["y"], cubic["u"]) - c["u"])))
            dv = float(np.max(np.abs(np.interp(c["x"], cubic["x"], cubic["v"]) - c["v"])))
            emit({"study": "cavity", "lattice": f"cuboid {nx}x64x{nz}", "r": r, "s": s, "cs2": 0.04,
                  "nodes": c["nodes"], "steps": c["steps"], "seconds": c["seconds"], "stable": c["stable"],
                  "node_ratio": cubic["nodes"] / c["nodes"], "time_ratio": cubic["seconds"] / c["seconds"],
                  "max_abs_du_over_U": du, "max_abs_dv_over_U": dv,
                  "u_min": float(c["u"].min()), "v_max": float(c["v"].max()), "v_min": float(c["v"].min())})
    emit({"study": args.study, "wall_seconds": time.time() - t0})
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--error-steps", default="100,1000,10000",
                    help="comma list of step counts at which each storage form is compared with the FP64 path")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--variants", default=",".join(VARIANTS),
                    help="storage forms to time (comma list of f32,f32s,bf16s,f16s,f64; "
                         "bf16s+sr / f16s+sr: stochastic rounding)")
    ap.add_argument("--workload", default="decaying", choices=sorted(WORKLOADS),
                    help="decaying: 512x256x256 periodic (default); channel: 768x192x384 with y walls")
    ap.add_argument("--kernel", default="auto", choices=["auto", "pair", "one", "staged", "march", "onepass"],
                    help="kernel selection passed to the library (auto = two nodes per thread where possible)")
    ap.add_argument("--dims", default=None,
                    help="NX,NY,NZ override of the lattice size (profiling of a smaller case only)")
    ap.add_argument("--study", default=None, choices=["stability", "xi", "reynolds", "cavity", "adjoint", "channel"],
                    help="run a parameter study of the paper instead of the benchmark (one JSON line per point): "
                         "stability / xi = Sec. 7 Figs. 8 / 9, reynolds = Fig. 10, cavity = Sec. 6, "
                         "adjoint = timing of the checkpointed adjoint on the 128x64x64 case, "
                         "channel = 768x192x384 channel run of reduced-precision storage against FP32")
    ap.add_argument("--e2e-contexts", type=int, default=2,
                    help="contexts taking the end-to-end steps in turn (1: no overlap)")
    ap.add_argument("--study-k", default="50,1",
                    help="adjoint study: checkpoint intervals K to time (1 keeps every state resident)")
    ap.add_argument("--study-corr", default="full,local,none",
                    help="correction modes of the omega_xi study (Fig. 9)")
    ap.add_argument("--study-ramp", type=int, default=0,
                    help="xi study: bring the lid up to speed linearly over this many steps (0: impulsive start)")
    ap.add_argument("--study-checkpoints", default="1000,10000,50000",
                    help="step counts at which the channel study reports (the last is the run length)")
    ap.add_argument("--study-variants", default="f32,bf16s,bf16s+sr,f16s+sr",
                    help="storage forms of the channel study (f32 is the reference run)")
    ap.add_argument("--study-steps", type=int, default=100_000, help="steps a stable run must survive")
    ap.add_argument("--omegas", default="1.5,1.6,1.7,1.8,1.9,1.95,1.98",
                    help="omega_nu values of the stability studies")
    args = ap.parse_args()
    if args.study:
        return run_study(args)
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    WORKLOAD.clear()
    WORKLOAD.update(WORKLOADS[args.workload])
    if args.dims:
        nx, ny, nz = (int(v) for v in args.dims.split(","))
        WORKLOAD.update(nx=nx, ny=ny, nz=nz, workload=WORKLOAD["workload"].split(" ")[0] + f" {nx}x{ny}x{nz} (reduced)")
    config = {k: WORKLOAD[k] for k in ("workload", "r_y", "r_z", "cs2", "nu", "omega_xi", "init", "corr", "walls")}
    config.update(nodes=WORKLOAD["nx"] * WORKLOAD["ny"] * WORKLOAD["nz"], parallelism=f"replicas x{world}",
                  l2="working set (2 x 27 x N stored values) >> 129 MB L2; no flush needed")

    if args.impl == "reference":
        if rank != 0:
            return
        cpu = reference_steps(args.steps, args.warmup)
        line = {"impl": "reference", "metric": METRIC, "value": cpu["value"], "unit": "MLUPS", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": cpu["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config, "cpu_baseline": cpu,
                "e2e": {"value": cpu["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    results, kernel_ms, e2e, N = run_ours(args, rank, world)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    peaks, which = measured_peaks()
    peak = float(peaks["hbm_gbs"])
    main_var = "f32" if "f32" in results else list(results)[0]
    r = results[main_var]
    achieved = bytes_per_node(main_var) * N / (kernel_ms[main_var] * 1e-3) / 1e9
    tpn = TRAFFIC_PER_NODE.get((args.workload, r["kernel"])) if not args.dims else None
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "traffic": round(tpn * N) if tpn else None,
            "peak_source": f"{which} hbm_gbs (copy bandwidth)", "kernel": r["kernel"],
            "algorithmic_bytes_per_launch": bytes_per_node(main_var) * N}
    variants = {}
    control = results.pop("_control_f64_perturbed_1e-6", None)
    for var in results:
        v = results[var]
        ach = bytes_per_node(var) * N / (kernel_ms[var] * 1e-3) / 1e9
        variants[var] = {"mlups": round(v["mlups"], 1), "ms_per_step": round(v["ms_per_step"], 4),
                         "bytes_per_node": bytes_per_node(var), "achieved_gbs": round(ach, 1),
                         "hbm_frac": round(ach / peak, 4), "kernel": v["kernel"],
                         "error_vs_f64": v["u_rel_err_vs_f64"],
                         "clocks": v["clocks"]}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = oracle_sample()
        one = oracle_sample(seconds_target=1.0, cores=1)     # one step on one core
        cpu["single_core"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
    line = {"metric": METRIC, "value": round(r["mlups"], 1), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(r["ms_per_step"], 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if main_var == "f64" else "f32", "data": "synthetic", "config": config,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps,
            "storage": main_var,
            "clocks": r["clocks"], "variants": variants,
            "error_control_f64_perturbed_1e-6": control}
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
