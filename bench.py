#!/usr/bin/env python
"""Benchmark of the dose engine: arc dose evaluations per second, forward +
adjoint, on a 256x256x160 pelvis-like grid at 2 mm with a two-arc VMAT plan
(2 x 178 control points, kernel radius 4 cm by default).

One step = pdrt_dose_forward + pdrt_dose_backward of the whole plan (all
control points), with the dose gradient of a quadratic dose-volume objective
resident in HBM.  value = arcs (178 CPs) evaluated per second, whole job.
The L2 cache (129 MB) is flushed between steps by writing a 256 MB buffer.

--impl reference times the FP64 CPU oracle (the method's plain definition)
on the host cores on a bounded sample (one control point per step at full
grid size), in the same metric.

Multi-GPU: the method's control points are independent, but one plan fits a
GPU; --gpus N runs N independent replicas (one process per GPU via
torch.distributed.run), value = total arcs/s over ranks, no collective on the
data path.
"""
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

METRIC = "arc dose evals/sec fwd+adjoint (256^3-class grid, 178 CPs) vs HBM roofline; warm vs plain"
UNIT = "arc evals/s"
CP_PER_ARC = 178
SMS, FP32_LANES = 152, 128


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pdrt", choices=["pdrt", "reference"])
    ap.add_argument("--r-cm", type=float, default=4.0)
    ap.add_argument("--cpu-sample-cps", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--corrections", action="store_true",
                    help="penumbra, off-axis profile and collimator rotation on (Sec. 2.2.2)")
    ap.add_argument("--warm-cases", type=int, default=20,
                    help="held-out phantoms for the warm-versus-plain figure (0 = skip)")
    ap.add_argument("--workload", default="pelvis256",
                    choices=["pelvis256", "pelvis128", "water64", "paper180", "batch32", "optimise"],
                    help="pelvis256: 256x256x160 @ 2 mm, 2 x 178 CPs (headline); "
                         "pelvis128: 128x128x96 @ 3 mm, 178 CPs (smaller case for profiler captures); "
                         "water64: one static 10 x 10 cm field on 64^3 water at 2.5 mm (R = 2 cm); "
                         "batch32: 32 uneven plans in one CUDA-graph launch (its own JSON line)")
    ap.add_argument("--step-stats", type=int, default=20,
                    help="single steps timed after the run for median / p10 / p90 (0: skip)")
    ap.add_argument("--scratch-gb", type=float, default=24.0,
                    help="plan scratch budget in GB (0 = library default)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations and the 32-plan batch (extra keys)")
    return ap.parse_args()


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def replica_time(ms, world, device):
    """Timed-region length of the slowest replica (max over ranks)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_step, steps, world, ms_max):
    """Whole-job throughput: the units all replicas processed over the
    slowest replica's time (weak scaling: each rank runs the full workload)."""
    return units_per_step * steps * world / (ms_max / 1e3)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _workload(r_cm, name="pelvis256", corrections=False):
    from paper_2512_18863_gb300 import synth
    if name == "pelvis128":
        w = synth.pelvis_arc_128(r_cm=r_cm)
    elif name == "water64":
        w = synth.water_static_64()
    elif name == "paper180":
        w = synth.paper_table_arc()
    else:
        w = synth.pelvis_two_arc_256(r_cm=r_cm)
    if corrections:
        # source penumbra, off-axis profile and a 15 degree collimator angle
        synth.with_corrections(w.machine, 1007, collimator_deg=15.0)
        w = synth.Workload(w.name + "_corrected", w.phantom, w.machine, w.plan)
    return w


def _config(w, world):
    """The workload description both arms print (identical for the ratio)."""
    nz, ny, nx = w.phantom.shape
    return {"workload": w.name, "grid": [nx, ny, nz],
            "spacing_mm": [float(x) for x in w.phantom.spacing],
            "n_cp": int(w.plan.n_cp), "kernel_radius_px": int(w.machine.r_px),
            "step": "forward + adjoint of all control points",
            "l2": "flushed between steps (256 MB write)",
            "parallelism": "replicas" if world > 1 else "single"}


def _subplan(w, sel):
    from paper_2512_18863_gb300 import synth
    return synth.Workload(w.name, w.phantom, w.machine,
                          synth.Plan(w.plan.gantry_deg[sel], w.plan.iso, w.plan.leaves[sel],
                                     w.plan.jaws[sel], w.plan.mu[sel]))


def _objective_grad(D, masks, torch):
    """dL/dD of L = 100 mean_PTV (D - Dp)^2 + sum_s l_s mean_s max(D - d_s, 0)^2
    (prescription Dp = 0.9 x median PTV dose; OAR thresholds 0.5 Dp).  A
    phantom without structures (water) takes L = mean (D - 0.9 max D)^2."""
    if "ptv" not in masks:
        return (2.0 * (D - 0.9 * float(D.max())) / D.numel()).contiguous()
    ptv = masks["ptv"]
    dp = 0.9 * float(D[ptv].median())
    g = torch.zeros_like(D)
    g[ptv] = 100.0 * 2.0 * (D[ptv] - dp) / ptv.sum()
    for name, lam in (("bladder", 1.0), ("rectum", 10.0)):
        m = masks[name]
        ex = torch.clamp(D[m] - 0.5 * dp, min=0.0)
        g[m] += lam * 2.0 * ex / m.sum()
    return g.contiguous()


class _Clocks:
    """nvidia-smi sampling (every 100 ms) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = os.path.join(tempfile.gettempdir(), f"pdrt_clocks_{os.getpid()}.csv")
        self.proc = None
        self.gpu = gpu_index
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(gpu_index), "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def _cpu_model():
    """The host CPU's model name (lscpu), else the architecture."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def _memo_reset(eng):
    """Forget the plan's memoised kernel spectra: every timed step then
    computes the spectra of its slices once (in the forward; its adjoint
    takes them), so no work is carried from one step into the next."""
    if eng.info.get("spectrum_memo_bytes"):
        eng.reset_spectrum_memo()


def _step_stats(eng, leaves, jaws, mu, g, dose, flush, n):
    """Device time of single steps (CUDA events around each, L2 flushed
    before it): median, p10 and p90 of n forward-only and of n forward +
    adjoint steps."""
    import torch
    out = {}
    for name, adj in (("forward", False), ("forward_adjoint", True)):
        ev = []
        for _ in range(n):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            _memo_reset(eng)
            eng.forward(leaves, jaws, mu, out=dose)
            if adj:
                eng.backward(leaves, jaws, mu, g)
            b.record()
            ev.append((a, b))
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        p10, p50, p90 = (float(x) for x in np.percentile(ms, [10, 50, 90]))
        out[name] = {"median_ms": p50, "p10_ms": p10, "p90_ms": p90, "n": int(n)}
    return out


def _cpu_baseline(w, n_cps):
    """FP64 oracle forward + adjoint on n_cps control points at full size."""
    from oracle import oracle
    sel = np.linspace(0, w.plan.n_cp - 1, n_cps).round().astype(int)
    sub = _subplan(w, sel)
    mod = oracle.Model(sub.phantom, sub.machine, sub.plan)
    rng = np.random.default_rng(0)
    g = rng.standard_normal(sub.phantom.shape)
    t0 = time.perf_counter()
    dose = mod.dose()
    grads = mod.dose_grad(g)
    dt = time.perf_counter() - t0
    out = {"value": (n_cps / CP_PER_ARC) / dt, "unit": UNIT, "cores": oracle.num_threads(),
           "kind": "oracle", "cpu_model": _cpu_model(),
           "sample": f"{n_cps} of {w.plan.n_cp} control points (fwd+adjoint) on the full "
                     f"{'x'.join(str(s) for s in w.phantom.shape[::-1])} grid, FP64, OpenMP; "
                     f"{dt:.1f} s"}
    return out, (sub, g, dose, grads)


def _accuracy(sample):
    """The engine on the CPU baseline's sample of control points against the
    oracle's results (outside any timed region): the largest dose deviation
    relative to the maximum dose and the largest gradient deviation relative
    to each class's largest gradient (the parity bars are 1e-4 and 1e-3)."""
    from paper_2512_18863_gb300.engine import DoseEngine
    sub, g, dose_ref, grads_ref = sample
    eng = DoseEngine(sub.phantom, sub.machine, sub.plan.gantry_deg, sub.plan.iso)
    d = eng.forward(sub.plan.leaves, sub.plan.jaws, sub.plan.mu).cpu().numpy().astype(np.float64)
    grads = [t.cpu().numpy().astype(np.float64)
             for t in eng.backward(sub.plan.leaves, sub.plan.jaws, sub.plan.mu, g.astype(np.float32))]
    eng.close()
    rel = lambda a, r: float(np.abs(a - r).max() / max(float(np.abs(r).max()), 1e-300))
    return {"sample": f"the CPU baseline's {sub.plan.n_cp} control points, full grid, same kernel radius",
            "dose_max_err_rel_max": rel(d, dose_ref),
            "grad_max_err_rel_max": {n: rel(a, r) for n, a, r in zip(("leaves", "jaws", "mu"), grads, grads_ref)},
            "bars": {"dose": 1e-4, "grad": 1e-3}}


def _reference(args):
    world, rank, _ = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            dist.destroy_process_group()
            return
    from oracle import oracle
    w = _workload(args.r_cm, args.workload, args.corrections)
    rng = np.random.default_rng(0)
    times = []
    for s in range(args.warmup + args.steps):
        b = int(rng.integers(0, w.plan.n_cp))
        sub = _subplan(w, np.array([b]))
        mod = oracle.Model(sub.phantom, sub.machine, sub.plan)
        g = rng.standard_normal(sub.phantom.shape)
        t0 = time.perf_counter()
        mod.dose()
        mod.dose_grad(g)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_step = float(np.mean(times))
    value = (1.0 / CP_PER_ARC) / per_step
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded pelvis phantom and VMAT arcs)",
           "config": _config(w, world),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                            "kind": "oracle", "cpu_model": _cpu_model(),
                            "sample": "one control point per step (fwd+adjoint), full grid"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch from a
# one-pass ncu capture of the 256x256x160 two-arc plan at R = 20 px, 178
# control points per launch (profiles/dram_pelvis256_2x178_R20.md); the FFT
# entries add the spectrum kernel launched (and timed) with each FFT pass.
# Each entry holds the SHA-256 prefixes of the sources the kernel is built
# from; a figure is reported only while the sources and the workload match
# the capture, else null.
_CAPTURES = {
    "workload": "pelvis256x256x160_2x178cp_R4cm",
    "conv_forward_fft": {"src": ("csrc/k_conv_fft.cu", "csrc/pdrt_impl.cuh"),
                         "sha": "b53b6c4d1f258152+635819d77a80519b", "bytes": 2.1100e9},
    "conv_adjoint_fft": {"src": ("csrc/k_conv_fft.cu", "csrc/pdrt_impl.cuh"),
                         "sha": "b53b6c4d1f258152+635819d77a80519b", "bytes": 2.1730e9},
    "gather_accumulate": {"src": ("csrc/k_gather.cu", "csrc/pdrt_impl.cuh"),
                          "sha": "f9d6a140dfd9f8d7+635819d77a80519b", "bytes": 1.6072e9},
    "gather_transpose": {"src": ("csrc/k_gather.cu", "csrc/pdrt_impl.cuh"),
                         "sha": "f9d6a140dfd9f8d7+635819d77a80519b", "bytes": 1.9807e9},
    "mag_transpose": {"src": ("csrc/k_adjoint.cu", "csrc/pdrt_impl.cuh"),
                      "sha": "7e30bff0a6f71a37+635819d77a80519b", "bytes": 0.4359e9},
}


def _src_sha(paths):
    import hashlib
    out = []
    for rel in paths:
        with open(os.path.join(ROOT, "paper_2512_18863_gb300", rel), "rb") as f:
            out.append(hashlib.sha256(f.read()).hexdigest()[:16])
    return "+".join(out)


def _captured_bytes(kernel, workload):
    """DRAM bytes per launch of `kernel` from the capture, or None when the
    workload or the kernel's sources differ from the captured ones."""
    c = _CAPTURES.get(kernel)
    if not c or workload != _CAPTURES["workload"] or _src_sha(c["src"]) != c["sha"]:
        return None
    return c["bytes"]


def _warm_start(n_cases):
    """Warm versus plain: dose evaluations the optimiser needs from the trained
    network's proposal to reach the plain optimiser's best objective in 100
    evaluations from an open-field start, on held-out phantoms."""
    import os
    from paper_2512_18863_gb300 import warmstart as W
    path = W.default_weights_path()
    if not os.path.exists(path):
        return {"unavailable": "no trained weights at " + os.path.relpath(path)}
    import numpy as np
    d = np.load(path)
    seeds = [int(x) for x in d["test_seeds"][:n_cases]]
    net = W.load_net(path)
    t0 = time.time()
    rows = W.evaluate(net, seeds)
    net.close()
    out = W.summarise(rows)
    out.update({"seconds": time.time() - t0, "held_out_seeds": seeds,
                "trained_on_plans": int(len(d["train_seeds"])),
                "network": "5-layer BF16 CNN (tcgen05, FP32 accumulate)"})
    return out


def _gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2512_18863_gb300 import _lib
    from paper_2512_18863_gb300.engine import DoseEngine

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = _workload(args.r_cm, args.workload, args.corrections)
    eng = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso,
                     scratch_budget_bytes=int(args.scratch_gb * 1e9))
    dev = eng.device
    leaves = torch.tensor(w.plan.leaves, dtype=torch.float32, device=dev)
    jaws = torch.tensor(w.plan.jaws, dtype=torch.float32, device=dev)
    mu = torch.tensor(w.plan.mu, dtype=torch.float32, device=dev)
    masks = {k: torch.tensor(v, device=dev) for k, v in w.phantom.masks.items()}
    dose = torch.empty(w.phantom.shape, dtype=torch.float32, device=dev)
    eng.forward(leaves, jaws, mu, out=dose)
    g = _objective_grad(dose, masks, torch)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2

    def step():
        _memo_reset(eng)
        eng.forward(leaves, jaws, mu, out=dose)
        eng.backward(leaves, jaws, mu, g)
        flush.zero_()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    work = eng.work()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = _lib.pdrt_launch_count()
    eng.profile(True)
    clocks = _Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    prof = eng.profile_read()
    eng.profile(False)
    launches = _lib.pdrt_launch_count() - launches0
    ms_max = replica_time(ms, world, dev)
    arcs_per_step = w.plan.n_cp / CP_PER_ARC
    value = whole_job_value(arcs_per_step, args.steps, world, ms_max)

    roofline = _roofline(prof, work, args.steps, w.name)
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["total_ms"] / args.steps}
               for k, v in prof.items() if not k.startswith("_") and v["launches"]}
    kernel_hbm = _kernel_hbm(prof, w.name)
    # the same step with the spectra kept from step to step (outside the
    # timed region; the headline resets them before every step)
    memo = None
    if eng.info.get("spectrum_memo_bytes"):
        def warm_step():
            eng.forward(leaves, jaws, mu, out=dose)
            eng.backward(leaves, jaws, mu, g)
            flush.zero_()
        for _ in range(2):
            warm_step()
        w0 = torch.cuda.Event(enable_timing=True)
        w1 = torch.cuda.Event(enable_timing=True)
        w0.record()
        for _ in range(args.steps):
            warm_step()
        w1.record()
        torch.cuda.synchronize()
        warm_ms = w0.elapsed_time(w1) / args.steps
        memo = {"headline": "memo reset before every timed step: each step computes its kernel spectra "
                            "once (forward) and its adjoint takes them",
                "bytes": int(eng.info["spectrum_memo_bytes"]), "pmax": int(eng.info["spectrum_memo_pmax"]),
                "kept_across_steps": {"ms_per_step": warm_ms,
                                      "value": arcs_per_step / (warm_ms / 1e3) * world}}
    # per-step distribution (after the timed region, outside it)
    step_ms = (_step_stats(eng, leaves, jaws, mu, g, dose, flush, args.step_stats)
               if args.step_stats > 0 else None)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda t: t.cpu().pin_memory()
        h_leaves, h_jaws, h_mu, h_g = pin(leaves), pin(jaws), pin(mu), pin(g)
        h_dose = torch.empty(dose.shape, dtype=torch.float32).pin_memory()
        h_dl, h_dj, h_dm = (torch.empty(t.shape, dtype=torch.float32).pin_memory()
                            for t in (leaves, jaws, mu))
        d_l, d_j, d_m, d_g = (torch.empty_like(t) for t in (leaves, jaws, mu, g))

        # the 42 MB copies overlap the compute that does not need them: the
        # dose gradient's upload runs beside the forward, the dose's download
        # beside the adjoint (copy stream + events; both inside every step)
        cs = torch.cuda.Stream(device=dev)
        ev_g, ev_f = torch.cuda.Event(), torch.cuda.Event()

        def e2e_step():
            main = torch.cuda.current_stream(dev)
            _memo_reset(eng)
            d_l.copy_(h_leaves, non_blocking=True)
            d_j.copy_(h_jaws, non_blocking=True)
            d_m.copy_(h_mu, non_blocking=True)
            cs.wait_stream(main)          # the previous adjoint has read d_g
            with torch.cuda.stream(cs):
                d_g.copy_(h_g, non_blocking=True)
                ev_g.record(cs)
            eng.forward(d_l, d_j, d_m, out=dose)
            ev_f.record(main)
            cs.wait_event(ev_f)
            with torch.cuda.stream(cs):
                h_dose.copy_(dose, non_blocking=True)
            main.wait_event(ev_g)
            dl, dj, dm = eng.backward(d_l, d_j, d_m, d_g)
            h_dl.copy_(dl, non_blocking=True)
            h_dj.copy_(dj, non_blocking=True)
            h_dm.copy_(dm, non_blocking=True)
            main.wait_stream(cs)          # the dose has left before the next forward
            flush.zero_()

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        el = lambda ts: sum(t.numel() * 4 for t in ts)
        e2e = {"value": arcs_per_step * args.steps * world / dt, "unit": UNIT,
               "h2d_bytes_per_step": el([h_leaves, h_jaws, h_mu, h_g]),
               "d2h_bytes_per_step": el([h_dose, h_dl, h_dj, h_dm])}

    cpu = accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, sample = _cpu_baseline(w, args.cpu_sample_cps)
        accuracy = _accuracy(sample)
    info = eng.info
    # the literal "vs HBM roofline" figure: bytes the method must move per
    # step (dose written, its gradient read, parameters and gradients) over
    # the step time, against the measured copy bandwidth
    alg_bytes = 4 * (2 * dose.numel() + 2 * (leaves.numel() + jaws.numel() + mu.numel()))
    hbm_peak = _measured_peaks().get("hbm_gbs", 6800.0)
    hbm = {"algorithmic_bytes_per_step": alg_bytes,
           "achieved_gbs": alg_bytes / (ms_max / args.steps / 1e3) / 1e9, "peak_gbs": hbm_peak,
           "frac": alg_bytes / (ms_max / args.steps / 1e3) / 1e9 / hbm_peak,
           "note": "the step is bound by the convolution arithmetic, not by HBM"}
    warm = None
    if rank == 0 and world == 1 and args.warm_cases > 0:
        warm = _warm_start(args.warm_cases)
    eng.close()
    sweep = batch32 = None
    if rank == 0 and world == 1 and not args.no_extras:
        sweep = _config_sweep(args, w.name)
        batch32 = _batch32(args, steps=3, warmup=1, report=False)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded pelvis phantom and VMAT arcs)",
               "config": _config(w, world),
               "precision": {"dose": "FP32 throughout; the convolution by FP32 FFTs, the slices "
                                     "beyond the FFT size limit on the tensor cores with a BF16 hi/lo "
                                     "split (three products, FP32 accumulation)",
                             "parity_bar": "max |dD| <= 1e-4 max D, gradients 1e-3 relative "
                                           "(tests against the FP64 oracle)",
                             "measured": "the line's accuracy key: this run's engine against the oracle "
                                         "on the CPU baseline's control points"},
               "roofline": roofline, "kernel_hbm": kernel_hbm,
               "kernels": kernels, "work": work, "gpu_launches": launches,
               "launch": {"scratch_gb": args.scratch_gb,
                          "fft_pmax": info.get("fft_pmax"), "fft_ctas_per_sm": info.get("fft_ctas_per_sm"),
                          "tc_phase": info.get("tc_phase"),
                          "tc_ctas_per_sm": info.get("tc_ctas_per_sm"),
                          "simt_ctas_per_sm": info.get("simt_ctas_per_sm"),
                          "chunk_cp": info.get("chunk_cp")},
               "configs": sweep, "batch32": batch32,
               "hbm_literal": hbm, "warm_start": warm, "step_ms": step_ms,
               "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "accuracy": accuracy,
               "spectrum_memo": memo}
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _roofline(prof, work, steps, workload):
    """Roofline of the dominant kernel.  With the FFT path on it is the FFT
    convolution, bound by the FP32 pipes: achieved = its algorithmic FLOPs
    (work.fft_flops: 2 x 2.5 N log2 N per slice and direction for the real
    2-D transforms, N = Pu Pv, plus the product, plus the kernel spectrum's
    cosine sums once per slice and padded size: the adjoint takes the
    forward's from the memo) over its CUDA-event time (the spectrum kernel's
    included), peak = 152 SM x 128 FP32 lanes x 2 FLOP
    x 2070 MHz.  Otherwise the tensor-core convolution against the measured
    sustained BF16 peak, with the direct convolution's 2 (2R+1)^2 FLOP per
    support point.  The direct-convolution-equivalent rate of all
    convolution kernels is reported beside it."""
    ms = lambda keys: sum(prof[k]["total_ms"] for k in keys if k in prof)
    ln = lambda keys: sum(prof[k]["launches"] for k in keys if k in prof)
    fft_k, tc_k, simt_k = (("conv_forward_fft", "conv_adjoint_fft"), ("conv_forward_tc", "conv_adjoint_tc"),
                           ("conv_forward", "conv_adjoint"))
    fft_ms, tc_ms, conv_ms = ms(fft_k), ms(tc_k), ms(fft_k + tc_k + simt_k)
    alu_peak = SMS * FP32_LANES * 2 * 2070.0e6 / 1e12
    peaks = _measured_peaks()
    direct = 2.0 * work["conv_flops"] * steps / (conv_ms / 1e3) / 1e12 if conv_ms else None
    if fft_ms > 0.5 * conv_ms:
        flops = work["fft_flops"] * steps
        achieved = flops / (fft_ms / 1e3) / 1e12
        n = max(ln(fft_k), 1)
        fb, ab = _captured_bytes("conv_forward_fft", workload), _captured_bytes("conv_adjoint_fft", workload)
        traffic = 0.5 * (fb + ab) if fb and ab else None
        return {"bound": "alu", "kernel": "k_conv_fft (FFT convolution, forward + adjoint)",
                "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                "traffic": traffic,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, one-pass "
                                   "capture at this workload, mean of forward and adjoint" if traffic else None),
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 FLOP x 2070 MHz",
                "flops": "algorithmic FFT: 2 x 2.5 N log2 N per slice and direction (N = Pu Pv) "
                         "+ product + kernel spectrum once per slice and padded size",
                "flops_per_launch": flops / n, "ms_per_launch": fft_ms / n,
                "tc_overflow_ms_per_step": tc_ms / steps,
                "direct_equivalent_tflops": direct}
    if tc_ms > 0.5 * conv_ms:
        flops = 2.0 * work["conv_flops"] * steps
        achieved = flops / (tc_ms / 1e3) / 1e12
        peak = peaks.get("bf16_tflops_sustained", 1700.0)
        n = max(ln(tc_k), 1)
        return {"bound": "tensor", "kernel": "k_conv_tc (tensor-core convolution, forward + adjoint)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "traffic_source": None,
                "peak_source": ("measured bf16 dense sustained (MEASURED_PEAKS.json)"
                                if "bf16_tflops_sustained" in peaks else "fallback 1.7 PFLOP/s bf16 sustained"),
                "flops": "algorithmic: 2 (2R+1)^2 per fluence-support point per pass",
                "flops_per_launch": flops / n, "ms_per_launch": tc_ms / n,
                "tensor_issued_tflops": work.get("mma_flops", 0.0) * steps / (tc_ms / 1e3) / 1e12}
    flops = 2.0 * work["conv_flops"] * steps
    achieved = flops / (conv_ms / 1e3) / 1e12
    n = max(ln(simt_k), 1)
    return {"bound": "alu", "kernel": "k_conv (FP32 SIMT convolution, forward + adjoint)",
            "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
            "traffic": None, "traffic_source": None,
            "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 FLOP x 2070 MHz",
            "flops": "algorithmic: 2 (2R+1)^2 per fluence-support point per pass",
            "flops_per_launch": flops / n, "ms_per_launch": conv_ms / n}


def _kernel_hbm(prof, workload):
    """Achieved DRAM bandwidth of the HBM-side kernels against the measured
    copy bandwidth: captured DRAM bytes per launch over the CUDA-event time
    per launch (null when no capture of the current sources exists)."""
    peak = _measured_peaks().get("hbm_gbs", 6800.0)
    out = {}
    names = {"gather_accumulate": "gather_accumulate", "gather_transpose": "gather_transpose",
             "mag_transpose": "mag_transpose_param_grad", "conv_forward_fft": "conv_forward_fft",
             "conv_adjoint_fft": "conv_adjoint_fft"}
    for key, pk in names.items():
        if pk not in prof or not prof[pk]["launches"]:
            continue
        b = _captured_bytes(key, workload)
        launches = prof[pk]["launches"]
        if key == "mag_transpose":   # the parameter-gradient launch (one per call) shares the timer
            launches = max(launches * 2 // 3, 1)
        per = prof[pk]["total_ms"] / launches
        gbs = b / (per / 1e3) / 1e9 if b else None
        out[key] = {"bytes_per_launch": b, "ms_per_launch": per, "achieved_gbs": gbs, "peak_gbs": peak,
                    "frac": gbs / peak if gbs else None}
    return out


def _timed_steps(eng, leaves, jaws, mu, g, dose, flush, n, adjoint):
    """Median device time of n single steps (CUDA events, L2 flushed before each)."""
    import torch
    ev = []
    for _ in range(n):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        _memo_reset(eng)
        eng.forward(leaves, jaws, mu, out=dose)
        if adjoint:
            eng.backward(leaves, jaws, mu, g)
        b.record()
        ev.append((a, b))
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in ev]))


def _config_sweep(args, headline):
    """The other dose configurations, each on its own plan: the two-arc plan
    at the kernel radii 2 and 8 cm (forward and forward + adjoint), the
    178-CP arc on 128x128x96 at 3 mm (forward) and the static 10 x 10 cm
    field on 64^3 water (forward).  Median of 5 single steps after 2 warm-ups."""
    import torch

    from paper_2512_18863_gb300.engine import DoseEngine
    cases = [("pelvis256", 2.0, True), ("pelvis256", 8.0, True), ("pelvis128", 4.0, False),
             ("water64", 2.0, False)]
    out = {}
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for name, r_cm, adj in cases:
        w = _workload(r_cm, name)
        if w.name == headline:
            continue
        eng = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso,
                         scratch_budget_bytes=int(args.scratch_gb * 1e9))
        dev = eng.device
        t = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
        leaves, jaws, mu = t(w.plan.leaves), t(w.plan.jaws), t(w.plan.mu)
        dose = eng.forward(leaves, jaws, mu)
        masks = {k: torch.tensor(v, device=dev) for k, v in w.phantom.masks.items()}
        g = _objective_grad(dose, masks, torch)
        for _ in range(2):
            eng.forward(leaves, jaws, mu, out=dose)
            if adj:
                eng.backward(leaves, jaws, mu, g)
        row = {"n_cp": int(w.plan.n_cp), "kernel_radius_px": int(w.machine.r_px),
               "forward_ms": _timed_steps(eng, leaves, jaws, mu, g, dose, flush, 5, False)}
        arcs = w.plan.n_cp / CP_PER_ARC
        row["forward_arc_evals_per_s"] = arcs / (row["forward_ms"] / 1e3)
        if adj:
            row["forward_adjoint_ms"] = _timed_steps(eng, leaves, jaws, mu, g, dose, flush, 5, True)
            row["forward_adjoint_arc_evals_per_s"] = arcs / (row["forward_adjoint_ms"] / 1e3)
        row["fft_pmax"] = eng.info.get("fft_pmax")
        out[w.name] = row
        eng.close()
    return out


def _gpu_batch(args):
    _batch32(args, args.steps, args.warmup, report=True)


def _batch32(args, steps, warmup, report):
    """32 plans of uneven grids (96..256 voxels per axis, 2-3 mm) and arcs
    (90-356 CPs): per-plan schedules from the autotuner, then forward +
    adjoint of all plans per CUDA-graph launch.  report: print its own JSON
    line; else return the figures (extra keys of the headline line)."""
    import torch

    from paper_2512_18863_gb300 import synth
    from paper_2512_18863_gb300.batch import DoseBatch
    from paper_2512_18863_gb300.engine import DoseEngine

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    ws = synth.uneven_batch(32)
    budget = int(1.5e9)          # per plan: 32 plans share the GPU
    engines, grads = [], []
    for w in ws:
        e = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso, scratch_budget_bytes=budget)
        masks = {k: torch.tensor(v, device=e.device) for k, v in w.phantom.masks.items()}
        d = e.forward(w.plan.leaves, w.plan.jaws, w.plan.mu)
        g = _objective_grad(d, masks, torch)
        e.autotune(w.plan.leaves, w.plan.jaws, w.plan.mu, g)
        engines.append(e)
        grads.append(g)
    batch = DoseBatch(engines, [w.plan.leaves for w in ws], [w.plan.jaws for w in ws],
                      [w.plan.mu for w in ws], grads, n_branches=len(ws))   # one branch per plan
    for _ in range(warmup):
        for e in engines:
            _memo_reset(e)
        batch.launch()
    torch.cuda.synchronize()
    lat = []
    clocks = _Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    total_ms = 0.0
    for _ in range(steps):
        e0.record()
        for e in engines:
            _memo_reset(e)
        batch.launch()
        e1.record()
        lat.append(batch.plan_times_ms())     # synchronises
        total_ms += e0.elapsed_time(e1)
    clk = clocks.stop()
    lat = np.concatenate(lat)
    n_cp = sum(w.plan.n_cp for w in ws)
    if not report:
        res = {"plans": len(ws), "control_points": n_cp, "steps": steps,
               "plan_evals_per_s": len(ws) * steps / (total_ms / 1e3),
               "arc_evals_per_s": n_cp / CP_PER_ARC * steps / (total_ms / 1e3),
               "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                              "max": float(lat.max())},
               "graph_launch_ms": total_ms / steps, "kernels_per_launch": batch.kernels,
               "schedules": [{"fft_pmax": e.info["fft_pmax"], "tensor_cores": e.info["tensor_cores"],
                              "chunk_cp": e.info["chunk_cp"]} for e in engines]}
        batch.close()
        for e in engines:
            e.close()
        return res
    if rank == 0:
        out = {"metric": "batched dose evals/sec fwd+adjoint (32 uneven plans, one CUDA-graph launch)",
               "value": len(ws) * steps * world / (total_ms / 1e3), "unit": "plan evals/s",
               "n_gpus": world, "steps": steps, "warmup": warmup,
               "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32",
               "data": "synthetic (seeded pelvis phantoms, uneven grids and arcs)",
               "config": {"workload": "batch32_uneven", "plans": len(ws), "control_points": n_cp,
                          "grids": [list(w.phantom.shape[::-1]) for w in ws],
                          "schedules": [{"tensor_cores": e.info["tensor_cores"], "chunk_cp": e.info["chunk_cp"],
                                         "tc_phase": e.info["tc_phase"],
                                         "tc_ctas_per_sm": e.info["tc_ctas_per_sm"]} for e in engines]},
               "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                              "max": float(lat.max())},
               "arc_evals_per_s": n_cp / CP_PER_ARC * steps * world / (total_ms / 1e3),
               "gpu_launches": batch.kernels * steps, "graph_launches": steps,
               "clocks": clk}
        print(json.dumps(out), flush=True)
    batch.close()
    for e in engines:
        e.close()


def _gpu_optimise(args):
    """Gradient plan optimisation (Adam, quadratic objective) of the two-arc
    plan from an open-field start: seconds per 100 iterations (one forward +
    adjoint, objective and Adam step each)."""
    import torch

    from paper_2512_18863_gb300 import optimize as opt
    from paper_2512_18863_gb300.engine import DoseEngine

    torch.cuda.set_device(0)
    w = _workload(args.r_cm, "pelvis256")
    eng = DoseEngine(w.phantom, w.machine, w.plan.gantry_deg, w.plan.iso,
                     scratch_budget_bytes=int(args.scratch_gb * 1e9))
    masks = {k: w.phantom.masks[k] for k in ("ptv", "bladder", "rectum")}
    init = opt.open_field_start(w.plan, w.machine)
    D0 = eng.forward(*init)
    presc = float(D0[torch.as_tensor(masks["ptv"], device=eng.device)].mean())
    opt.optimise(eng, masks, presc, init, n_iter=args.warmup, objective="quadratic")
    torch.cuda.synchronize()
    n = max(args.steps, 1) * 10
    t0 = time.perf_counter()
    res = opt.optimise(eng, masks, presc, init, n_iter=n, objective="quadratic")
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {"metric": "plan optimisation iterations/sec (fwd + adjoint + Adam, two-arc 256x256x160 plan)",
           "value": n / dt, "unit": "iterations/s", "n_gpus": 1, "steps": n, "warmup": args.warmup,
           "ms_per_step": dt / n * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded pelvis phantom and VMAT arcs)",
           "config": _config(w, 1), "seconds_per_100_iterations": dt / n * 100,
           "objective_first_last": [res.history[0], res.history[-1]]}
    print(json.dumps(out), flush=True)
    eng.close()


def main():
    args = _args()
    if args.impl == "reference":
        _reference(args)
    elif args.workload == "batch32":
        _gpu_batch(args)
    elif args.workload == "optimise":
        _gpu_optimise(args)
    else:
        _gpu(args)


if __name__ == "__main__":
    main()
