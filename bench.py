#!/usr/bin/env python3
"""Benchmark: adjoint light paths per second of constant-memory differentiable light
tracing (LRB-3-pass, attached) on the box + 32x32 height-field workload.

One step = one pass of the hot path over one batch of 2^22 light paths at depth 16:
  refit the height field's triangles and BVH bounds (2 kernels)
  -> primal light tracing with sensor connection and splat at every vertex (1 kernel)
  -> film L2 loss and image adjoint (1 kernel)
  -> LRB-3-pass backward, attached gradients w.r.t. the emitted radiance and every
     height-field vertex height including the splat-position derivative (2 kernels:
     pass 2 stores delta_total and the connection-validity mask per path, pass 3
     backpropagates).
Inputs are seeded and synthetic (see paper_2609_32920_gb300.inputs).  `value` is
device-timed with inputs resident in HBM; `e2e` adds the host->device copy of the step's
inputs and the device->host copy of loss and gradients.  The ResLRB and naive-AD
pipelines and the peak device memory of each method versus depth are reported alongside.

`--impl reference` times the FP64 CPU oracle (naive tape AD) on the host cores instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# The headline workload: the largest single-GPU configuration, the caustic slab (a
# dielectric slab with a 128x128 height-field top over a diffuse receiver, 512x512 film,
# 2^24 light paths per step at depth 8, attached height gradients).  The box with a 32x32
# diffuse height field (2^22 paths at depth 16) is timed alongside as a study.
WORKLOADS = {
    "slab512_hm128": dict(paths_log2=24, depth=8, resolution="512x512",
                          geometry="dielectric slab, 128x128 height-field top (32258 + 1016 + 2 triangles) "
                                   "over a 2x2 m diffuse receiver",
                          params="16384 heights (+ Le)"),
    "box256_hm32": dict(paths_log2=22, depth=16, resolution="256x256",
                        geometry="open box of 5 textured walls + 32x32 diffuse height field (1922 triangles)",
                        params="Le (3) + 1024 heights (+ albedo textures)"),
}
WORKLOAD = "slab512_hm128"
N_PATHS = 1 << WORKLOADS[WORKLOAD]["paths_log2"]
DEPTH = WORKLOADS[WORKLOAD]["depth"]
METRIC = "adjoint light paths/s (LRB-3-pass attached: refit + primal + film + backward)"
FLOPS_PER = {"node": 24, "prim": 30, "vertex": 150, "conn": 100}


KERNEL_SOURCES = ("lt_kernels.cu", "lt_device.cuh", "lt_launch.h", "lt_batch.h", "lt_mlp.cuh", "lt_api.cu")


def traffic_profile(workload):
    return os.path.join(ROOT, "profiles", f"traffic_{workload}.md")


def kernel_fingerprint():
    """16 hex digits identifying the compiled kernels: the kernel sources with comments and
    layout removed, and the kernel compiler flags (a comment edit keeps it, a code or flag
    change does not)."""
    import hashlib
    import re

    from paper_2609_32920_gb300 import build as B
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        src = open(os.path.join(ROOT, "paper_2609_32920_gb300", "csrc", f)).read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    h.update(" ".join(B.ARCH + B.FLAGS + B.KERNEL_FLAGS).encode())
    return h.hexdigest()[:16]


def profiled_traffic(workload, key):
    """DRAM bytes per launch of kernel `key` (primal, lrb3_backward) from the committed ncu
    summary of the workload, or None when the compiled kernels have changed since that
    capture (or there is none)."""
    import re
    try:
        text = open(traffic_profile(workload)).read()
        fp = re.search(r"kernel_fingerprint: (\w+)", text).group(1)
        tb = int(re.search(r"traffic_bytes_%s_per_launch: (\d+)" % key, text).group(1))
    except (OSError, AttributeError, ValueError):
        return None
    return tb if fp == kernel_fingerprint() else None


def workload_config(n_paths, workload=None):
    """The `config` object of the JSON line (both arms)."""
    wl = workload or WORKLOAD
    w = WORKLOADS[wl]
    return {"workload": wl, "resolution": w["resolution"], "geometry": w["geometry"], "paths_per_gpu": n_paths,
            "max_depth": w["depth"], "attached": True, "params": w["params"],
            "l2": "flushed between steps (256 MB write outside the timed interval)"}


def make_workload(name):
    """(scene, target scene, paths, depth) of a named workload.  Targets: the caustic of
    another height field (seed 1) for the slab; perturbed albedo and halved heights for the
    box."""
    from paper_2609_32920_gb300 import inputs as I
    w = WORKLOADS[name]
    if name == "slab512_hm128":
        sc = I.slab_scene(512, n=128, seed=0)
        tgt = I.slab_scene(512, n=128, seed=1)
    else:
        sc = I.box_scene(256, heightmap=32)
        tgt = sc.with_params(albedo=I.perturbed_albedo(sc, 0.05, 1), heights=sc.heights * 0.5)
    return sc, tgt, 1 << w["paths_log2"], w["depth"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS),
                    help="timed workload (profiling runs may pick the box)")
    ap.add_argument("--paths-log2", type=int, default=0, help="paths per GPU per step (0: the workload's; "
                                                               "profiling uses fewer)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the per-method and memory-vs-depth sweeps")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU-oracle sample time")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-target study")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched many-scene study")
    ap.add_argument("--no-inverse", action="store_true", help="skip the caustic inverse-rendering study")
    ap.add_argument("--scatter", type=int, default=0, choices=[0, 1, 2, 3],
                    help="gradient and splat scatter mode of the step (profiling runs; lt_render_opts.scatter)")
    ap.add_argument("--profile", action="store_true",
                    help="profiling run: only warm-up and timed steps (no e2e, census, studies or CPU baseline)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ------------------------------------------------------------------ clocks sampler
class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lt_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU oracle timing
def oracle_sample(sc, dI, seconds: float, n_norm: int, depth: int, attached: int = 1):
    """Time the FP64 oracle (naive tape AD) on a bounded sample of the workload's paths."""
    from oracle import oracle as O
    O.build()
    cores = os.cpu_count() or 1
    n = 32
    t0 = time.perf_counter()
    O.gradient(sc, dI, seed=0, n_paths=n, max_depth=depth, attached=attached, n_norm=n_norm, n_threads=cores)
    dt = max(time.perf_counter() - t0, 1e-3)
    n = int(min(1 << 16, max(256, n * seconds / dt)))
    t0 = time.perf_counter()
    O.gradient(sc, dI, seed=0, n_paths=n, max_depth=depth, attached=attached, n_norm=n_norm, n_threads=cores)
    dt = time.perf_counter() - t0
    return n, dt, cores


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2609_32920_gb300 import inputs as I
    sc, _, n_wl, depth = make_workload(args.workload)
    dI = I.smooth_adjoint(sc.W, sc.H, 1)
    # size one step's sample so that the whole warmup + steps run stays within a few minutes
    per_step = max(1.0, min(8.0, 150.0 / max(1, args.steps + args.warmup)))
    n, dt, cores = oracle_sample(sc, dI, per_step, n_wl, depth)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.gradient(sc, dI, seed=i, n_paths=n, max_depth=depth, attached=1, n_norm=n_wl, n_threads=cores)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    value = n / mean
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * mean, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(n_wl, args.workload),
            "cpu_baseline": {"value": value, "unit": "paths/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n} of the workload's {n_wl} paths per step (the same scene, depth and "
                                       f"attached gradient), naive tape reverse-mode AD in FP64 on the host cores"},
            "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------ GPU arm
class Step:
    """One pass of the hot path on a workload: refit the height field (update_tris,
    refit_nodes, refit_big, refit_wide<4>, refit_wide<8>: every width stays current), the
    order of the paths (a counting sort, 4 kernels) and primal light tracing storing the
    paths' connection-validity masks and first connections (1 kernel), film L2 loss and image
    adjoint (1), LRB-3-pass backward in its three-pass form, attached (pass 2 of the
    single-connection paths, pass 2 of the others, pass 3: 3 kernels).  Events around the
    primal (with its sort) and the backward time them on the launching stream."""

    LAUNCHES = 14

    def __init__(self, name, dev, path_offset=0, n_norm=0, n_paths=0, scatter=0):
        import torch

        from paper_2609_32920_gb300 import lt
        self.lt = lt
        sc, tgt, n_wl, depth = make_workload(name)
        self.name, self.sc, self.depth = name, sc, depth
        self.n = n_paths or n_wl
        self.S = S = lt.Scene(sc)
        T_S = lt.Scene(tgt)
        self.target = T_S.primal(T_S.opts(seed=12345, n_paths=self.n, max_depth=depth))
        del T_S
        self.heights = S.heights.clone()
        self.state = S.new_lrb3_state(self.n)
        self.path_offset, self.n_norm = path_offset, n_norm or self.n
        kw = dict(seed=1, n_paths=self.n, max_depth=depth, path_offset=path_offset, n_norm=self.n_norm,
                  lrb3_state=self.state, scatter=scatter)
        self.o_plain = S.opts(**kw)
        self.o_att = S.opts(attached=1, lrb3_mask_ready=1, **kw)
        self.img = S.new_image()
        self.dI = torch.empty_like(self.img)
        self.loss = torch.empty(1, device=dev)
        self.grads = S.new_grads()
        self.stream = torch.cuda.current_stream()

    def __call__(self, ev=None):
        """ev: optional [primal start, primal end, backward start, backward end] events."""
        S, lt, st = self.S, self.lt, self.stream
        S.refit(self.heights)
        if ev:
            ev[0].record(st)
        S.primal(self.o_plain, image=self.img)
        if ev:
            ev[1].record(st)
        lt.film_l2(self.img, self.target, d_image=self.dI, loss=self.loss)
        if ev:
            ev[2].record(st)
        S.backward_lrb3(self.o_att, self.dI, grads=self.grads)
        if ev:
            ev[3].record(st)

    def census(self):
        """Work of one primal and one backward pair (counting kernel variants, untimed)."""
        import torch
        S = self.S
        out = {}
        for key in ("primal", "lrb3_backward"):
            c = torch.zeros(5, dtype=torch.int64, device=self.img.device)
            kw = dict(seed=1, n_paths=self.n, max_depth=self.depth, path_offset=self.path_offset,
                      n_norm=self.n_norm, census=c, lrb3_state=self.state)
            if key == "primal":
                S.primal(S.opts(**kw), image=S.new_image())
            else:
                S.backward_lrb3(S.opts(attached=1, lrb3_mask_ready=1, **kw), self.dI, grads=S.new_grads())
            torch.cuda.synchronize()
            v = [int(x) for x in c.cpu()]
            flops = (FLOPS_PER["node"] * v[1] + FLOPS_PER["prim"] * v[2] + FLOPS_PER["vertex"] * v[3] +
                     FLOPS_PER["conn"] * v[4])
            out[key] = {"rays": v[0], "box_tests": v[1], "prim_tests": v[2], "vertices": v[3], "connections": v[4],
                        "flops": flops}
        return out


def timed_steps(step, steps, flush, barrier):
    """Run `steps` timed steps (L2 flushed before each, outside the timed interval); returns
    per-step, per-primal and per-backward milliseconds."""
    import torch
    st = step.stream
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    ev = [(E(), E()) for _ in range(steps)]
    kev = [[E(), E(), E(), E()] for _ in range(steps)]
    barrier()
    for i in range(steps):
        flush.fill_(i & 0xff)
        ev[i][0].record(st)
        step(kev[i])
        ev[i][1].record(st)
    barrier()
    return ([a.elapsed_time(b) for a, b in ev], [k[0].elapsed_time(k[1]) for k in kev],
            [k[2].elapsed_time(k[3]) for k in kev])


def device_free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2609_32920_gb300 import inputs as I
    from paper_2609_32920_gb300 import lt
    from paper_2609_32920_gb300.shard import max_over_ranks, path_shard

    wl = args.workload
    n_paths = (1 << args.paths_log2) if args.paths_log2 else (1 << WORKLOADS[wl]["paths_log2"])
    # weak scaling: each rank traces its own paths, no data-path collective
    path_offset, _, n_norm = path_shard(rank, ws, n_paths)
    step = Step(wl, dev, path_offset, n_norm, n_paths, args.scatter)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # clocks and throttle reasons are sampled from before the warm-up to the end of the
    # end-to-end timing, so the record spans both timed regions
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.5)  # nvidia-smi's first sample
    for _ in range(args.warmup):
        step()
    step.S.sync_status()
    step_ms, primal_ms, bwd_ms = timed_steps(step, args.steps, flush, barrier)
    total_ms = max_over_ranks(sum(step_ms), dev)
    ms_per_step = total_ms / args.steps
    if args.profile:
        clk = clocks.stop()
        if rank == 0:
            print(json.dumps({"profile": True, "workload": wl, "paths": n_paths, "ms_per_step": ms_per_step,
                              "primal_ms": statistics.median(primal_ms), "backward_ms": statistics.median(bwd_ms),
                              "clocks": clk}))
        return 0
    value = ws * n_paths / (ms_per_step * 1e-3)
    step.S.sync_status()

    # ---------------- end to end through the public API with host buffers
    S = step.S
    alb_h = S.albedo.cpu().pin_memory()
    le_h = S.Le.cpu().pin_memory()
    hts_h = step.heights.cpu().pin_memory()
    tgt_h = step.target.cpu().pin_memory()
    out_h = [torch.empty(g.numel(), dtype=torch.float32).pin_memory() for g in step.grads]
    loss_h = torch.empty(1, dtype=torch.float32).pin_memory()
    h2d = (alb_h.numel() + le_h.numel() + hts_h.numel() + tgt_h.numel()) * 4
    d2h = (sum(g.numel() for g in step.grads) + 1) * 4

    def e2e_step():
        S.albedo.copy_(alb_h, non_blocking=True)
        S.Le.copy_(le_h, non_blocking=True)
        step.heights.copy_(hts_h, non_blocking=True)
        step.target.copy_(tgt_h, non_blocking=True)
        step()
        for g, h in zip(step.grads, out_h):
            h.copy_(g, non_blocking=True)
        loss_h.copy_(step.loss, non_blocking=True)

    for _ in range(2):
        e2e_step()
    barrier()
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(max(3, args.steps // 2))]
    for a, b in e_ev:
        flush.fill_(1)
        a.record(step.stream)
        e2e_step()
        b.record(step.stream)
    barrier()
    e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in e_ev) / len(e_ev), dev)
    e2e_value = ws * n_paths / (e2e_ms * 1e-3)
    clk = clocks.stop()

    # ---------------- roofline of the dominant kernel (census from the counting variants)
    census = step.census()
    sm_max = 2070.0
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        sm_max = float(peaks.get("sm_max_mhz", sm_max))
    except Exception:
        pass
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tflops = sms * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA lanes x 2 x max SM clock
    kernel_ms = {"primal": sum(primal_ms) / len(primal_ms), "lrb3_backward": sum(bwd_ms) / len(bwd_ms)}
    names = {"primal": "k_primal<PLAIN> (primal light tracing, sensor connections, splats, validity masks)",
             "lrb3_backward": "k_lrb3_single + k_lrb3_p2 + k_lrb3_p3 (LRB-3 passes 2 and 3, attached)"}
    rooflines = {}
    for key in kernel_ms:
        ach = census[key]["flops"] / (kernel_ms[key] * 1e-3) / 1e12
        rooflines[key] = {"bound": "alu", "kernel": names[key], "achieved": ach, "peak": peak_tflops,
                          "unit": "TFLOP/s", "frac": ach / peak_tflops,
                          "peak_note": f"derived: {sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                          "traffic": profiled_traffic(wl, key),
                          "traffic_source": os.path.relpath(traffic_profile(wl), ROOT),
                          "kernel_ms": kernel_ms[key], "census": census[key], "flops_per": FLOPS_PER}
    dom = max(kernel_ms, key=kernel_ms.get)
    roofline = dict(rooflines[dom])
    roofline["other"] = {k: {x: rooflines[k][x] for x in ("kernel", "achieved", "frac", "kernel_ms", "traffic")}
                         for k in rooflines if k != dom}

    # ---------------- studies (outside the headline timing)
    studies = {}
    other = "box256_hm32" if wl == "slab512_hm128" else "slab512_hm128"
    if rank == 0:
        studies[other] = workload_study(other, dev, flush, barrier, args.steps)
    if not args.no_sweep:
        studies["scatter"] = scatter_study(step, flush)
        studies["literal_transport"] = literal_study(step, flush)
        studies["methods"], studies["memory_vs_depth"] = method_sweep(step, dev, flush)
        if rank == 0:
            box = Step("box256_hm32", dev)
            studies["box_methods"], studies["box_memory_vs_depth"] = method_sweep(box, dev, flush)
            studies["russian_roulette"] = roulette_study(box, dev, flush)
            del box
    if not args.no_sweep and rank == 0:
        studies["bidirectional"] = bidir_study(dev, flush)
    if not args.no_learned and rank == 0:
        studies["learned_target"] = learned_target_study(dev)
    if not args.no_batch and rank == 0:
        studies["batched"] = batched_study(dev)
    if not args.no_inverse and rank == 0:
        studies["caustic_inverse"] = {
            "configured (lr 1e-3, per-vertex heights, L2)": caustic_inverse_study(dev, lr=1e-3),
            "blurred loss, smooth heights": caustic_inverse_study(dev, lr=2e-4, blur_px=8, smooth_cells=8)}

    # ---------------- CPU baseline: the oracle on the host cores (rank 0, N=1 only)
    cpu = None
    if rank == 0 and ws == 1:
        n, dt, cores = oracle_sample(step.sc, I.smooth_adjoint(step.sc.W, step.sc.H, 1), args.cpu_seconds,
                                     n_paths, step.depth)
        cpu = {"value": n / dt, "unit": "paths/s", "cores": cores, "kind": "oracle",
               "sample": f"{n} of the workload's {n_paths} paths, depth {step.depth}, attached naive tape AD "
                         f"(FP64), one gradient pass"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "paths/s", "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(n_paths, wl),
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": "paths/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": Step.LAUNCHES * args.steps, "clocks": clk,
                "step_ms": {"median": statistics.median(step_ms), "min": min(step_ms), "max": max(step_ms)},
                "primal_ms": statistics.median(primal_ms), "backward_ms": statistics.median(bwd_ms),
                "studies": studies, "lib": lt.version()}
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def workload_study(name, dev, flush, barrier, steps):
    """The same step on another workload (untimed for the headline)."""
    step = Step(name, dev)
    for _ in range(3):
        step()
    step_ms, primal_ms, bwd_ms = timed_steps(step, max(5, steps // 2), flush, barrier)
    step.S.sync_status()
    ms = statistics.median(step_ms)
    return {"config": workload_config(step.n, name), "ms_per_step": ms, "paths_per_s": step.n / (ms * 1e-3),
            "primal_ms": statistics.median(primal_ms), "backward_ms": statistics.median(bwd_ms)}


def scatter_study(step, flush, reps=3):
    """Primal and LRB-3 backward times of the workload for each way of bringing gradients and
    splats to memory (opts.scatter 0-3, see include/lt.h)."""
    import torch
    S, st = step.S, step.stream
    names = {0: "default (46 KB shared-memory arrays, else plain global atomics)",
             1: "shared-memory arrays up to the opt-in limit", 2: "plain global atomics",
             3: "warp-aggregated global atomics for gradients and splats"}
    out = {"workload": f"{step.name}, 2^{step.n.bit_length() - 1} paths, depth {step.depth}, attached"}
    for mode in (0, 1, 2, 3):
        kw = dict(seed=1, n_paths=step.n, max_depth=step.depth, lrb3_state=step.state, scatter=mode)
        op, om = S.opts(**kw), S.opts(attached=1, lrb3_mask_ready=1, **kw)
        p_ms, b_ms = [], []
        for r in range(reps + 1):
            flush.fill_(r)
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(st)
            S.primal(op, image=step.img)
            e[1].record(st)
            S.backward_lrb3(om, step.dI, grads=step.grads)
            e[2].record(st)
            torch.cuda.synchronize()
            if r:
                p_ms.append(e[0].elapsed_time(e[1]))
                b_ms.append(e[1].elapsed_time(e[2]))
        out[str(mode)] = {"mode": names[mode], "primal_ms": statistics.median(p_ms),
                          "backward_ms": statistics.median(b_ms)}
    S.sync_status()
    return out


def literal_study(step, flush, reps=3):
    """The paper-literal attached transport (opts.literal; determinant-guarded inverse, with
    and without Jacobian noise) against the exact chain transport on the workload: time of
    one LRB-3 backward and the relative L2 distance of its height gradient from the exact
    one at the same seed."""
    import torch
    S, st = step.S, step.stream
    kw = dict(seed=1, n_paths=step.n, max_depth=step.depth, attached=1)
    out = {"workload": f"{step.name}, 2^{step.n.bit_length() - 1} paths, depth {step.depth}, attached"}
    variants = (("exact (two kernels, path list)", dict(lrb3_state=step.state, lrb3_mask_ready=1)),
                ("exact (fused)", {}), ("literal, guard only", dict(literal=1)),
                ("literal, Jacobian noise", dict(literal=1, jac_noise=1, noise_seed=3)))
    ref = None
    for name, extra in variants:
        o = S.opts(**kw, **extra)
        ms = []
        for r in range(reps + 1):
            flush.fill_(r)
            S.primal(S.opts(seed=1, n_paths=step.n, max_depth=step.depth, lrb3_state=step.state), image=step.img)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            g = S.backward_lrb3(o, step.dI)
            e1.record(st)
            torch.cuda.synchronize()
            if r:
                ms.append(e0.elapsed_time(e1))
        gh = g[2].double()
        if ref is None:
            ref = gh
        out[name] = {"backward_ms": statistics.median(ms),
                     "height_rel_l2_to_exact": float(torch.linalg.norm(gh - ref) / torch.linalg.norm(ref))}
    S.sync_status()
    return out


def bidir_study(dev, flush, seeds=16, n_log2=21, m_log2=19, depth=6):
    """The bidirectional estimator against the light tracer alone on the box with textured
    walls (256x256, detached albedo and Le): time of one gradient (primal + backward) and the
    mean per-parameter variance of the albedo gradient over seeds; time x variance is the
    efficiency (lower is better)."""
    import torch

    from paper_2609_32920_gb300 import inputs as I
    from paper_2609_32920_gb300 import lt
    sc = I.box_scene(256)
    S = lt.Scene(sc)
    dI = torch.tensor(I.smooth_adjoint(sc.W, sc.H, 3), dtype=torch.float32, device=dev)
    n, m = 1 << n_log2, 1 << m_log2
    st = torch.cuda.current_stream()
    out = {"workload": f"box256 (textured walls), detached, depth {depth}, 2^{n_log2} light paths, "
                       f"2^{m_log2} camera samples, {seeds} seeds"}
    for name, mc in (("light_tracer", 0), ("bidirectional", m)):
        G, ms = [], []
        for s_ in range(seeds + 1):
            o = S.opts(seed=40 + s_, n_paths=n, max_depth=depth)
            b = S.bidir_opts(mc)
            flush.fill_(s_)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            S.bidir_primal(o, b)
            g = S.bidir_backward(o, b, dI)
            e1.record(st)
            torch.cuda.synchronize()
            if s_:
                ms.append(e0.elapsed_time(e1))
                G.append(g[0].double().cpu())
        G = torch.stack(G)
        var = float(G.var(dim=0, unbiased=True).mean())
        out[name] = {"ms_per_gradient": statistics.median(ms), "variance": var,
                     "time_x_variance": statistics.median(ms) * var}
    out["efficiency_gain"] = out["light_tracer"]["time_x_variance"] / out["bidirectional"]["time_x_variance"]
    S.sync_status()
    return out


METHODS = ("lrb3", "lrb3_fused", "lrb2", "reslrb", "naive")


def _pipeline_runner(S, target, dev, n_paths, path_offset, n_norm, flush):
    """run(method, D, reps) -> (median ms, peak extra bytes, device bytes) of one attached
    gradient: primal + film L2 + backward.  lrb3 = two-kernel form with its per-path
    state; lrb3_fused = one fused backward kernel without per-path state; lrb2 = the
    buffered two-pass baseline (per-vertex splat records, linear in depth).  Peak extra
    bytes: torch's peak allocation above the scene's; device bytes: the fall of the
    device's free memory (cudaMemGetInfo) from before the method's buffers are allocated
    to after its first gradient, which also sees what the driver reserves for the kernels
    (local memory of traversal stacks and chain caches)."""
    import torch

    from paper_2609_32920_gb300 import lt
    stream = torch.cuda.current_stream()
    img = S.new_image()
    dI = torch.empty_like(img)
    loss = torch.empty(1, device=dev)
    grads = S.new_grads()

    def run(method, D, timed_reps=3):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free0 = device_free_bytes()
        base = torch.cuda.memory_allocated()
        torch.cuda.reset_peak_memory_stats()
        aux = None
        state = S.new_lrb3_state(n_paths) if method == "lrb3" else None
        o = S.opts(seed=3, n_paths=n_paths, max_depth=D, attached=1, path_offset=path_offset, n_norm=n_norm,
                   lrb3_state=state, lrb3_mask_ready=int(state is not None))
        if method == "reslrb":
            aux = torch.empty((n_paths, 8), dtype=torch.float32, device=dev)
        elif method == "naive":
            aux = torch.empty(S.naive_workspace_bytes(o), dtype=torch.uint8, device=dev)
        elif method == "lrb2":
            aux = torch.empty(S.lrb2_buffer_bytes(o), dtype=torch.uint8, device=dev)

        def once():
            if method.startswith("lrb3"):
                S.primal(o, image=img)
                lt.film_l2(img, target, d_image=dI, loss=loss)
                S.backward_lrb3(o, dI, grads=grads)
            elif method == "reslrb":
                S.primal(o, estimator=lt.EST_RESLRB, image=img, aux=aux)
                lt.film_l2(img, target, d_image=dI, loss=loss)
                S.backward_reslrb(o, dI, aux, grads=grads)
            elif method == "lrb2":
                S.primal(o, estimator=lt.EST_BUFFERED, image=img, aux=aux)
                lt.film_l2(img, target, d_image=dI, loss=loss)
                S.backward_lrb2(o, dI, aux, grads=grads)
            else:
                S.primal(o, estimator=lt.EST_NAIVE, image=img, aux=aux)
                lt.film_l2(img, target, d_image=dI, loss=loss)
                S.backward_naive(o, dI, aux, grads=grads)
        once()
        torch.cuda.synchronize()
        peak = torch.cuda.max_memory_allocated() - base
        dev_bytes = free0 - device_free_bytes()
        ms = []
        for _ in range(timed_reps):
            flush.fill_(2)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            once()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        del aux, state
        torch.cuda.empty_cache()
        return statistics.median(ms), peak, dev_bytes

    return run


def method_sweep(step, dev, flush):
    """Paths/s of each estimator (primal + film + backward, attached) at the workload's depth,
    and the extra device memory of each estimator at depths 4..64 (torch's peak allocation
    and the device's own free-memory drop)."""
    S, n = step.S, step.n
    run = _pipeline_runner(S, step.target, dev, n, step.path_offset, step.n_norm, flush)
    methods = {"workload": f"{step.name}, 2^{n.bit_length() - 1} paths, depth {step.depth}, attached"}
    for m in METHODS:
        ms, peak, dbytes = run(m, step.depth)
        methods[m] = {"paths_per_s": n / (ms * 1e-3), "ms": ms, "extra_bytes": peak, "device_bytes": dbytes}
    memory = {"workload": f"{step.name}, 2^{n.bit_length() - 1} paths, attached"}
    for D in (4, 8, 16, 32, 64):
        memory[str(D)] = {}
        for m in METHODS:
            ms, peak, dbytes = run(m, D, timed_reps=3)
            memory[str(D)][m] = {"extra_bytes": peak, "device_bytes": dbytes, "ms": ms}
    S.sync_status()
    return methods, memory


def roulette_study(step, dev, flush, rr_depth=4, rr_prob=0.8):
    """Time of one attached LRB-3 gradient (primal + film + backward) on the box workload
    with Russian roulette (continue with probability 0.8 after depth 4) and without it,
    at depths 16 and 64."""
    import torch

    from paper_2609_32920_gb300 import lt
    S, n = step.S, step.n
    stream = torch.cuda.current_stream()
    img = S.new_image()
    dI = torch.empty_like(img)
    loss = torch.empty(1, device=dev)
    grads = S.new_grads()
    state = S.new_lrb3_state(n)
    out = {"setting": "continue with probability %g after depth %d" % (rr_prob, rr_depth)}
    for D in (16, 64):
        row = {}
        for name, rr in (("off", {}), ("on", dict(rr_depth=rr_depth, rr_prob=rr_prob))):
            kw = dict(seed=5, n_paths=n, max_depth=D, attached=1, lrb3_state=state, **rr)
            op, om = S.opts(**kw), S.opts(lrb3_mask_ready=1, **kw)

            def once():
                S.primal(op, image=img)
                lt.film_l2(img, step.target, d_image=dI, loss=loss)
                S.backward_lrb3(om, dI, grads=grads)
            once()
            ms = []
            for _ in range(3):
                flush.fill_(3)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                once()
                b.record(stream)
                torch.cuda.synchronize()
                ms.append(a.elapsed_time(b))
            row[name] = {"ms": statistics.median(ms), "paths_per_s": n / (statistics.median(ms) * 1e-3)}
        out[str(D)] = row
    return out


def _learned_one(dev, kind, seeds, paths_log2, depth):
    """Time x gradient variance of ResLRB with the learned reservoir target against ResLRB
    with the luminance target on one workload.  kind "caustic": dielectric 64x64 height
    field over a receiver, 256x256, attached height gradients, image adjoint from an L2 loss
    against the caustic of a different height field.  kind "interior": the box with the
    32x32 height field, image adjoint concentrated in one film region.  Both estimators use
    the same seeds; variance = mean over parameters of the per-parameter variance across
    seeds."""
    import torch

    from paper_2609_32920_gb300 import inputs as I
    from paper_2609_32920_gb300 import lt
    n = 1 << paths_log2
    if kind == "caustic":
        sc = I.slab_scene(256, n=64, seed=0)
        S = lt.Scene(sc)
        T_S = lt.Scene(I.slab_scene(256, n=64, seed=1))
        target = T_S.primal(T_S.opts(seed=7, n_paths=4 * n, max_depth=depth))
        del T_S
        img = S.primal(S.opts(seed=8, n_paths=4 * n, max_depth=depth))
        _, dI = lt.film_l2(img, target)
        gi = 2
    else:
        sc = I.box_scene(256, heightmap=32)
        S = lt.Scene(sc)
        dI = torch.tensor(I.blob_adjoint(sc.W, sc.H, 81), dtype=torch.float32, device=dev)
        gi = 0
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    (f, t, cnt), ms_collect = timed(lambda: S.mlp_collect(S.opts(seed=9, n_paths=n, max_depth=depth, attached=1), dI,
                                                          capacity=1 << 20,
                                                          target_floor=0.01 * float(dI.abs().max())))
    P = lt.mlp_init(0)
    losses, ms_train = timed(lambda: lt.mlp_train(P, f, t, epochs=20, batch=4096, lr=1e-3))
    rec = torch.empty((n, 8), device=dev)
    res = {}
    for name, extra in (("plain", {}), ("learned", {"target": lt.TARGET_MLP, "mlp": P})):
        grads, ms = [], []
        for s_ in range(seeds):
            o = S.opts(seed=100 + s_, n_paths=n, max_depth=depth, attached=1, **extra)
            g, m_ = timed(lambda: (S.primal(o, estimator=lt.EST_RESLRB, aux=rec), S.backward_reslrb(o, dI, rec))[1])
            grads.append(g[gi].cpu().clone())
            ms.append(m_)
        G = torch.stack(grads).double()
        var = float(G.var(dim=0, unbiased=True).mean())
        res[name] = {"ms_per_gradient": statistics.median(ms), "variance": var,
                     "time_x_variance": statistics.median(ms) * var, "mean_grad_norm": float(G.mean(0).norm())}
    conns = cnt / n
    wl = "slab256_hm64 (caustic)" if kind == "caustic" else "box256_hm32 (interior, localized adjoint)"
    return {"workload": "%s depth %d, 2^%d paths per gradient, %d seeds" % (wl, depth, paths_log2, seeds),
            "pairs": int(f.shape[0]), "connections_per_path": conns, "collect_ms": ms_collect, "train_ms": ms_train,
            "train_loss_first_last": [losses[0], losses[-1]], "plain": res["plain"], "learned": res["learned"],
            "efficiency_gain": res["plain"]["time_x_variance"] / res["learned"]["time_x_variance"]}


def learned_target_study(dev):
    return {"caustic": _learned_one(dev, "caustic", 16, 20, 32), "interior": _learned_one(dev, "interior", 16, 20, 16),
            "cfg_stated": learned_stated_study(dev)}


def connection_histogram(S, n, depth, seed, dev):
    """Fraction of the paths with 0, 1, 2, ... valid sensor connections (the plain primal's
    per-path count): the learned target can only pay where paths connect more than once."""
    import torch
    dbg = torch.zeros((n, 4), dtype=torch.float32, device=dev)
    S.primal(S.opts(seed=seed, n_paths=n, max_depth=depth, attached=1, dbg_out=dbg))
    h = torch.bincount(dbg[:, 0].round().long()).cpu()
    del dbg
    return [float(c) / n for c in h]


def learned_stated_study(dev, seeds=16, ref_seeds=256, depth=32):
    """The learned reservoir target at its stated size: ResLRB at depth 32 with 2^24 paths
    per gradient on the caustic workload (slab512_hm128, attached heights), the network
    trained on 2^20 pairs collected by an LRB-3 pass-2 replay; and, because caustic paths
    have about one connection each, on the slab inside the textured box (slabbox256_hm64,
    2^22 paths).  Per workload: time x variance of ResLRB with the luminance and with the
    learned target over `seeds` seeds, and each one's mean gradient error
    ||mean_s g - g_ref|| / ||g_ref|| next to the error that its variance alone predicts
    (sqrt(P Var / S) / ||g_ref||: an unbiased estimator's error matches it), with g_ref the
    LRB-3 gradient averaged over `ref_seeds` seeds."""
    import torch

    from paper_2609_32920_gb300 import inputs as I
    from paper_2609_32920_gb300 import lt
    st = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        out = fn()
        b.record(st)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    res = {}
    for kind in ("caustic", "slab_in_box"):
        if kind == "caustic":
            n = 1 << 24
            sc = I.slab_scene(512, n=128, seed=0)
            S = lt.Scene(sc)
            T_S = lt.Scene(I.slab_scene(512, n=128, seed=1))
            target = T_S.primal(T_S.opts(seed=7, n_paths=n, max_depth=8))
            del T_S
            img = S.primal(S.opts(seed=8, n_paths=n, max_depth=8))
            _, dI = lt.film_l2(img, target)
        else:
            n = 1 << 22
            sc = I.slab_in_box(256, n=64, seed=0)
            S = lt.Scene(sc)
            dI = torch.tensor(I.blob_adjoint(sc.W, sc.H, 81), dtype=torch.float32, device=dev)
        (f, t, cnt), ms_collect = timed(lambda: S.mlp_collect(
            S.opts(seed=9, n_paths=n, max_depth=depth, attached=1), dI, capacity=1 << 20,
            target_floor=0.01 * float(dI.abs().max())))
        P = lt.mlp_init(0)
        losses, ms_train = timed(lambda: lt.mlp_train(P, f, t, epochs=20, batch=4096, lr=1e-3))
        state = S.new_lrb3_state(n)
        ref = torch.zeros(S.n_heights, dtype=torch.float64, device=dev)
        for s_ in range(ref_seeds):
            o = S.opts(seed=20000 + s_, n_paths=n, max_depth=depth, attached=1, lrb3_state=state)
            S.primal(o)
            om = S.opts(seed=20000 + s_, n_paths=n, max_depth=depth, attached=1, lrb3_state=state, lrb3_mask_ready=1)
            ref += S.backward_lrb3(om, dI)[2][: S.n_heights].double()
        ref /= ref_seeds
        rec = torch.empty((n, 8), device=dev)
        row = {"workload": f"{sc.name}, depth {depth}, 2^{n.bit_length() - 1} paths per gradient, attached heights, "
                           f"{seeds} seeds; g_ref = LRB-3 over {ref_seeds} seeds",
               "connections_per_path": cnt / n, "pairs": int(f.shape[0]), "collect_ms": ms_collect,
               "train_ms": ms_train, "train_loss_first_last": [losses[0], losses[-1]]}
        try:
            row["connections_histogram"] = connection_histogram(S, n, depth, 9, dev)
        except Exception as e:  # a diagnostic: its failure leaves the study's numbers standing
            row["connections_histogram"] = "unavailable: %s" % e
        for name, extra in (("luminance", {}), ("learned", {"target": lt.TARGET_MLP, "mlp": P})):
            G, ms = [], []
            for s_ in range(seeds):
                o = S.opts(seed=100 + s_, n_paths=n, max_depth=depth, attached=1, **extra)
                g, m_ = timed(lambda: (S.primal(o, estimator=lt.EST_RESLRB, aux=rec), S.backward_reslrb(o, dI, rec))[1])
                G.append(g[2][: S.n_heights].double())
                ms.append(m_)
            G = torch.stack(G)
            var = float(G.var(dim=0, unbiased=True).mean())
            nref = float(torch.linalg.norm(ref))
            row[name] = {"ms_per_gradient": statistics.median(ms), "variance": var,
                         "time_x_variance": statistics.median(ms) * var,
                         "mean_gradient_error": float(torch.linalg.norm(G.mean(0) - ref)) / nref,
                         "noise_only_error": (S.n_heights * var / seeds) ** 0.5 / nref}
        row["efficiency_gain"] = row["luminance"]["time_x_variance"] / row["learned"]["time_x_variance"]
        S.sync_status()
        res[kind] = row
        del S
    return res


def _gauss1d(sigma, dev):
    import torch
    r = int(3 * sigma + 1)
    x = torch.arange(-r, r + 1, device=dev, dtype=torch.float32)
    k = torch.exp(-x * x / (2 * sigma * sigma))
    return k / k.sum(), r


def blur_image(im, sigma):
    """Separable Gaussian blur of an [H, W, 3] image with zero padding (a symmetric linear
    operator, so it is its own adjoint)."""
    import torch
    if not sigma:
        return im
    k, r = _gauss1d(sigma, im.device)
    x = im.permute(2, 0, 1).unsqueeze(1)
    x = torch.nn.functional.conv2d(x, k.view(1, 1, 1, -1), padding=(0, r))
    x = torch.nn.functional.conv2d(x, k.view(1, 1, -1, 1), padding=(r, 0))
    return x.squeeze(1).permute(1, 2, 0).contiguous()


def blur_field(g, n, sigma):
    """Separable Gaussian blur of an n x n parameter field (edge values repeated)."""
    import torch
    if not sigma:
        return g
    k, r = _gauss1d(sigma, g.device)
    G = g.view(1, 1, n, n)
    G = torch.nn.functional.conv2d(torch.nn.functional.pad(G, (r, r, 0, 0), mode="replicate"), k.view(1, 1, 1, -1))
    G = torch.nn.functional.conv2d(torch.nn.functional.pad(G, (0, 0, r, r), mode="replicate"), k.view(1, 1, -1, 1))
    return G.view(-1)


def caustic_inverse_study(dev, steps=200, paths_log2=24, depth=8, lr=1e-3, blur_px=0, smooth_cells=0):
    """The paper's geometric inverse problem on the caustic workload: starting from a flat
    slab top, recover the 128x128 height field of the dielectric slab (512x512 film) from
    the caustic it casts, by Adam with attached LRB-3 gradients, 2^24 light paths per
    iteration (a new seed each), against a target rendered from the true height field (sum
    of Gaussians, seed 1) at 2^26 paths.  blur_px > 0: the loss compares the two images
    after a Gaussian blur of that standard deviation (pixels), whose adjoint is the blurred
    residual; smooth_cells > 0: Adam moves a latent field z and the heights are z blurred by
    that many cells (the gradient of z is the blurred height gradient).  Reported: the loss,
    the caustic error at 2^26 paths (relative L2, raw and after a 4-pixel blur; a second
    render of the true heights gives the noise floor) and the height error (RMSE, and with
    the mean removed, since a constant offset does not change the caustic)."""
    import torch

    from paper_2609_32920_gb300 import inputs as I
    from paper_2609_32920_gb300 import lt
    n = 1 << paths_log2
    true_sc = I.slab_scene(512, n=128, seed=1)
    T_S = lt.Scene(true_sc)
    target = T_S.primal(T_S.opts(seed=12345, n_paths=4 * n, max_depth=depth))
    del T_S
    sc = I.slab_scene(512, n=128, seed=0, flat=True)
    S = lt.Scene(sc)
    h_true = torch.tensor(true_sc.heights, dtype=torch.float32, device=dev)
    z = torch.zeros_like(h_true).requires_grad_(True)
    opt = torch.optim.Adam([z], lr=lr)
    state = S.new_lrb3_state(n)
    img = S.new_image()
    dI = torch.empty_like(img)
    loss = torch.empty(1, device=dev)
    grads = S.new_grads()
    bt = blur_image(target, blur_px)
    losses = []

    def evaluate(hh):
        S.refit(hh)
        im = S.primal(S.opts(seed=777, n_paths=4 * n, max_depth=depth))
        a, b = blur_image(im, 4), blur_image(target, 4)
        d = hh - h_true
        return {"caustic_rel_l2": float(torch.linalg.norm(im - target) / torch.linalg.norm(target)),
                "caustic_rel_l2_blur4": float(torch.linalg.norm(a - b) / torch.linalg.norm(b)),
                "height_rmse_m": float(torch.sqrt((d ** 2).mean())),
                "height_rmse_shape_m": float(torch.sqrt(((d - d.mean()) ** 2).mean()))}

    ev = {"floor (true heights)": evaluate(h_true), "0": evaluate(torch.zeros_like(h_true))}
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for it in range(steps):
        torch.cuda.synchronize()
        a.record(stream)
        h = blur_field(z.detach(), 128, smooth_cells)
        S.refit(h)
        o = S.opts(seed=1000 + it, n_paths=n, max_depth=depth, attached=1, lrb3_state=state)
        S.primal(o, image=img)
        if blur_px:
            r = blur_image(img, blur_px) - bt
            losses.append((r * r).mean())
            dI = blur_image(2.0 * r / r.numel(), blur_px)
        else:
            lt.film_l2(img, target, d_image=dI, loss=loss)
            losses.append(loss.clone())
        om = S.opts(seed=1000 + it, n_paths=n, max_depth=depth, attached=1, lrb3_state=state, lrb3_mask_ready=1)
        S.backward_lrb3(om, dI, grads=grads)
        z.grad = blur_field(grads[2][: h.numel()].clone(), 128, smooth_cells)
        opt.step()
        b.record(stream)
        torch.cuda.synchronize()
        ms += a.elapsed_time(b)
        if (it + 1) % 100 == 0:
            ev[str(it + 1)] = evaluate(blur_field(z.detach(), 128, smooth_cells))
    S.sync_status()
    L = [float(x) for x in losses]
    return {"workload": "slab512_hm128 (caustic), flat start, 128x128 heights, depth 8, 2^%d paths per "
                        "iteration, %d Adam steps lr %g" % (paths_log2, steps, lr),
            "loss": "L2 of images blurred by %g px" % blur_px if blur_px else "L2 (film_l2)",
            "parameterisation": "heights = latent blurred by %g cells" % smooth_cells if smooth_cells
                                else "per-vertex heights",
            "ms_per_iteration": ms / steps,
            "loss_mean_of_10_at": {str(i): sum(L[i:i + 10]) / 10 for i in range(0, steps, max(10, steps // 5))},
            "eval": ev}


def batched_study(dev, n_scenes=64, reps=3):
    """Many scenes of uneven size (caustic slabs and boxes, height fields 32^2..256^2,
    depth 4..32, 2^16..2^22 paths, attached) in one persistent launch per pass, against the
    same work issued scene by scene.  One iteration = refit + primal + LRB-3 backward of
    every scene.  The batch's launch shape comes from its autotuner (LRB-3 pass)."""
    import torch

    from paper_2609_32920_gb300 import inputs as I
    from paper_2609_32920_gb300 import lt
    t0 = time.time()
    items = []
    for k, spec in enumerate(I.batched_set(n_scenes, seed=0, max_paths_log2=22)):
        S = lt.Scene(spec["scene"])
        it = dict(scene=S, n_paths=spec["n_paths"], max_depth=spec["max_depth"], attached=spec["attached"], seed=k,
                  lrb3_state=True)
        if S.n_heights:
            it["heights"] = S.heights.clone()
        it["d_image"] = torch.tensor(I.smooth_adjoint(S.W, S.H, 500 + k), dtype=torch.float32, device=dev)
        items.append(it)
    build_s = time.time() - t0
    B = lt.Batch(items)
    B.run(lt.PASS_PRIMAL)
    t1 = time.time()
    cfg, tuned_ms = B.tune(lt.PASS_LRB3, reps=1)
    tune_s = time.time() - t1
    stream = torch.cuda.current_stream()

    def timed(fn):
        ms = []
        fn()
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    def batched():
        B.run(lt.PASS_PRIMAL)
        B.run(lt.PASS_LRB3)

    # the same work scene by scene: two-kernel LRB-3 reusing the primal's validity masks
    states = [it["scene"].new_lrb3_state(it["n_paths"]) for it in items]
    opts_p = [it["scene"].opts(seed=it["seed"], n_paths=it["n_paths"], max_depth=it["max_depth"],
                               attached=it["attached"], lrb3_state=st) for it, st in zip(items, states)]
    opts = [it["scene"].opts(seed=it["seed"], n_paths=it["n_paths"], max_depth=it["max_depth"],
                             attached=it["attached"], lrb3_state=st, lrb3_mask_ready=1)
            for it, st in zip(items, states)]
    grads = [it["scene"].new_grads() for it in items]
    imgs = [it["scene"].new_image() for it in items]

    def sequential():
        for it, op, o, g, im in zip(items, opts_p, opts, grads, imgs):
            S = it["scene"]
            if S.n_heights:
                S.refit(it["heights"])
            S.primal(op, image=im)
            S.backward_lrb3(o, it["d_image"], grads=g)

    ms_b = timed(batched)
    ms_s = timed(sequential)
    total = sum(it["n_paths"] for it in items)
    for it in items:
        it["scene"].sync_status()
    return {"workload": "%d scenes: slab/box alternating, height fields 32^2..256^2, depth 4..32, "
                        "2^16..2^22 paths, attached, 128x128 film" % n_scenes,
            "total_paths": total, "tris": sum(it["scene"].src.n_tris for it in items),
            "batched": {"ms_per_iteration": ms_b, "paths_per_s": total / (ms_b * 1e-3), "config": cfg,
                        "tuned_lrb3_pass_ms": tuned_ms, "tune_s": tune_s},
            "per_scene_calls": {"ms_per_iteration": ms_s, "paths_per_s": total / (ms_s * 1e-3)},
            "speedup": ms_s / ms_b, "scene_build_s": build_s}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
