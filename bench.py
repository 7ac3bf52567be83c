"""Benchmark of forward + adjoint light tracing on the procedural office.

One step = one optimisation iteration's hot path: upload the 16 spot lights,
forward pass (2^24 photons, 5 hits), objective + adjoint weights, adjoint
pass (decorrelated seed), gradient. Metric: Msegments/s of forward + adjoint
(a segment is one traced ray, emission or bounce, hit or miss).

  value   device time (CUDA events on the library's stream) of the step's
          kernels with every input already resident in HBM; the L2 cache is
          flushed (256 MiB write) between steps, outside the timed events.
  e2e     the same metric through the C ABI with host buffers: per step the
          light parameters go host->device, the loss and gradient come back
          device->host, and an Adam update runs on the host.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): each rank traces its own 2^24 photons (weak scaling); the
integer texel sums and the gradients are summed across ranks with NCCL.
"""
from __future__ import annotations

import argparse
import hashlib
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

from paper_2310_02043_gb300 import scenes  # noqa: E402

METRIC = "Msegments/s fwd+adjoint"
PHOTONS, HITS = 1 << 24, 5
TARGET_PHOTONS = 1 << 26
KERNELS_PER_STEP = 8          # forward, loss, loss reduction, weight range, adjoint, gradient, 2 gradient reductions
LIGHT_DEV_BYTES = 160         # device light record the library uploads per light
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "trace_kernel_traffic.json")


def workload(name: str = "office"):
    """(scene, lights, ground-truth lights) of a single-design workload: the
    office (16 spots, 2 cm texels) or the Cornell box (1 point light)."""
    if name == "cornell":
        sc = scenes.cornell_box(res=32)
        lights = scenes.cornell_lights()
        truth = scenes.perturb_lights(lights, seed=1, pos_sigma=0.05, intensity_range=(0.8, 1.2))
        return sc, lights, truth
    sc = scenes.office(seed=0, pitch=0.02)
    lights = scenes.office_lights(0)
    truth = scenes.perturb_lights(lights, seed=1, pos_sigma=0.3, angle_sigma=0.1, intensity_range=(0.7, 1.3),
                                  theta_in_delta=np.radians(5.0))
    return sc, lights, truth


# photons per GPU, hits per photon and target photons of each single-design workload
PASS = {"office": (PHOTONS, HITS, TARGET_PHOTONS), "cornell": (1 << 18, 3, 1 << 22)}


def config_of(sc, lights, n_gpus, name: str = "office"):
    photons, hits, target = PASS[name]
    if name == "cornell":
        what = (f"Cornell box 1 m room, front open, 2 boxes ({sc.n_tri} tris), {sc.n_texels} texels (32x32 per "
                f"face), 1 point light, 2^18 photons/GPU, 3 hits, target traced at 2^22")
    else:
        what = (f"procedural office 20x10x3 m, 200 desks/cabinets ({sc.n_tri} tris), {sc.n_texels} texels "
                f"at 2 cm, {lights.shape[0]} spots, 2^24 photons/GPU, 5 hits, target traced at 2^26")
    return {"workload": what, "triangles": sc.n_tri, "texels": sc.n_texels, "lights": int(lights.shape[0]),
            "photons_per_gpu": photons, "hits": hits,
            "l2": "flushed between steps (256 MiB write outside the timed events)",
            "parallelism": f"photon shards x{n_gpus}" if n_gpus > 1 else "single GPU"}


# ---------------------------------------------------------------------------
# Clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device_index = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device_index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def clock_sampler(local):
    import torch
    props = torch.cuda.get_device_properties(local)
    uuid = getattr(props, "uuid", None)
    return ClockSampler(f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else (uuid or local))


# ---------------------------------------------------------------------------
# Roofline helpers
# ---------------------------------------------------------------------------
# FP32 operations the traversal issues (counted from the kernel's arithmetic,
# one fma per slab plane): a node visit forms -o/d once (3 ops) and tests 8
# child boxes, each 6 plane fmas, one 3-input max, one max with 0, one
# 3-input min, the exit scaling and 2 comparisons (12 ops); a watertight
# ray/triangle test is 9 subtractions, 12 shear operations, 9 edge-function
# operations, 2 additions for the determinant, 8 for the distance and 6 sign
# tests (46 ops); every segment also samples a direction and a flux (about
# 40 ops) and computes the hit's texel and normal (about 40).
OPS_PER_NODE = 8 * 12 + 3
OPS_PER_TRI = 46
OPS_PER_SEGMENT = 80
# Algorithmic bytes per segment of the traversal, as the scope defines them:
# an 8-wide node with quantised child boxes (80 B, five 16-byte loads), a
# triangle (48 B, three 16-byte loads), and the texel access (8 B deposit in
# the forward pass, 4 B weight gather in the adjoint); random numbers are
# computed in registers. A visit of a float node staged in shared memory (240
# B) loads the ray's near and far planes (192 B) and the inner-slot mask; a
# visit of a compressed node read through L1 (96 B) loads its header and
# planes (64 B).
NODE_BYTES, TRI_BYTES = 80, 48
NODE_BYTES_LOADED = {True: 196, False: 64}      # staged float node / compressed node through L1
HBM_FALLBACK_GBS = 6800.0


def alu_peak_tflops(sm_mhz):
    """FP32 issue peak: 152 SMs x 128 FP32 lanes x one operation per lane per
    clock (an FMA counts as one operation, as in OPS_PER_*)."""
    return 152 * 128 * sm_mhz * 1e6 / 1e12


def hbm_peak():
    """(GB/s, basis): the measured copy bandwidth, else the fallback figure."""
    try:
        v = json.load(open(MEASURED_PEAKS)).get("hbm_gbs")
        if v:
            return float(v), "of measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError):
        pass
    return HBM_FALLBACK_GBS, "of fallback (6.8 TB/s, one earlier GB300 measurement)"


def traversal_roofline(work, seg_launch, kernel_ms, adjoint, l2_gbs, peak_clock, traffic_per_seg, name, staged=True):
    """Roofline record of one trace launch: algorithmic bytes (per segment from
    the counting kernel, times the launch's segments) over its CUDA-event time
    against the L2 read rate; beside it the same bytes against HBM, the bytes
    the kernel's nodes actually load (staged float nodes or compressed nodes
    through L1), and the FP32 operations against the issue peak."""
    segs = work["segments"]
    nv, tt = work["node_visits"] / segs, work["tri_tests"] / segs
    per_seg = nv * NODE_BYTES + tt * TRI_BYTES + (4 if adjoint else 8)
    per_seg_loaded = nv * NODE_BYTES_LOADED[staged] + tt * TRI_BYTES + (4 if adjoint else 8)
    secs = kernel_ms / 1e3
    achieved = per_seg * seg_launch / secs / 1e9
    ops_seg = nv * OPS_PER_NODE + tt * OPS_PER_TRI + OPS_PER_SEGMENT
    ops = ops_seg * seg_launch / secs / 1e12
    alu = alu_peak_tflops(peak_clock)
    hbm, hbm_basis = hbm_peak()
    return {"bound": "l2", "achieved": achieved, "peak": l2_gbs, "unit": "GB/s", "frac": achieved / l2_gbs,
            "traffic": traffic_per_seg * seg_launch if traffic_per_seg is not None else None,
            "kernel": f"trace_kernel ({'adjoint' if adjoint else 'forward'}, {name})",
            "peak_basis": "L2 read rate of the library's own probe (lt_probe_l2_read: 32 MiB swept with 16-byte "
                          "L2-only loads), measured in this run",
            "bytes_per_segment": {"algorithmic": per_seg, "node_visits": nv, "tri_tests": tt,
                                  "node_bytes": NODE_BYTES, "tri_bytes": TRI_BYTES,
                                  "node_bytes_loaded": NODE_BYTES_LOADED[staged],
                                  "nodes": "staged float nodes" if staged else "compressed nodes through L1",
                                  "as_loaded": per_seg_loaded},
            "hbm": {"achieved": achieved, "peak": hbm, "frac": achieved / hbm, "unit": "GB/s",
                    "peak_basis": hbm_basis},
            "alu": {"achieved": ops, "peak": alu, "frac": ops / alu, "unit": "TFLOP/s",
                    "fp32_ops_per_segment": ops_seg,
                    "peak_basis": f"FP32 issue peak 152 SMs x 128 lanes x {peak_clock:.0f} MHz (derived)"}}


def l2_read_gbs():
    from paper_2310_02043_gb300.lighttrace import probe_l2_read
    return probe_l2_read(0, 32 << 20, 64)


def kernel_hash():
    """Hash of the sources the stored traffic depends on: the tracing kernels
    and the BVH builder (node visits per segment)."""
    h = hashlib.sha256()
    for f in ("lt_kernels.cu", "lt_bvh.cpp"):
        h.update(open(os.path.join(ROOT, "paper_2310_02043_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def stored_traffic(kernel):
    """DRAM bytes per segment from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    try:
        d = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    if d.get("kernel_source_sha256_16") != kernel_hash():
        return None
    return d.get(kernel, {}).get("dram_bytes_per_segment")


# ---------------------------------------------------------------------------
# CPU baseline: the oracle on the host cores, a bounded sample of the workload
# ---------------------------------------------------------------------------
def cpu_baseline(sc, lights, truth, budget_s=15.0, name="office"):
    """The oracle on the host cores over a bounded sample of the workload
    (photons [0, n) of its budget, n sized to about budget_s, capped at the
    whole budget), with a single-thread figure over a smaller sample."""
    import oracle
    oracle.build()
    photons, hits, _ = PASS[name]
    cores = os.cpu_count() or 1
    small = min(1 << 14, photons)
    target = oracle.forward(sc, truth, 77, small, hits)["E"]
    t0 = time.perf_counter()
    oracle.forward(sc, lights, 2, photons, hits, begin=0, end=small)
    probe = time.perf_counter() - t0
    n = int(min(1 << 20, photons, max(small, small * budget_s / 2.0 / max(probe, 1e-3))))
    n = max(small, (n // 4096) * 4096)
    t0 = time.perf_counter()
    f = oracle.forward(sc, lights, 2, photons, hits, begin=0, end=n)
    t1 = time.perf_counter()
    _, w = oracle.loss(sc, f["E"], target, np.ones(sc.n_texels))
    t2 = time.perf_counter()
    _, seg_adj = oracle.adjoint(sc, lights, 3, photons, hits, w, begin=0, end=n)
    t3 = time.perf_counter()
    segs = f["segments"] + seg_adj
    # the same passes on one thread, over a smaller photon range
    n1 = min(1 << 12, photons)
    t4 = time.perf_counter()
    f1 = oracle.forward(sc, lights, 2, photons, hits, begin=0, end=n1, threads=1)
    _, w1 = oracle.loss(sc, f1["E"], target, np.ones(sc.n_texels))
    _, seg1 = oracle.adjoint(sc, lights, 3, photons, hits, w1, begin=0, end=n1, threads=1)
    t5 = time.perf_counter()
    segs1 = f1["segments"] + seg1
    budget = "the whole budget" if n == photons else f"the 2^{photons.bit_length() - 1} budget"
    return {"value": segs / (t3 - t0) / 1e6, "unit": "Msegments/s", "cores": cores, "kind": "oracle",
            "sample": f"photons [0, {n}) of {budget}, forward + loss + adjoint, brute-force FP64 oracle "
                      f"({segs} segments in {t3 - t0:.1f} s: forward {t1 - t0:.1f} s, adjoint {t3 - t2:.1f} s)",
            "single_thread": {"value": segs1 / (t5 - t4) / 1e6, "unit": "Msegments/s",
                              "sample": f"photons [0, {n1}), same passes, one thread ({segs1} segments in "
                                        f"{t5 - t4:.1f} s)"}}


def run_reference(args):
    """Reference arm: the oracle as it stands on the host cores, same metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    name = args.workload if args.workload in PASS else "office"
    photons, hits, _ = PASS[name]
    sc, lights, truth = workload(name)
    import oracle
    oracle.build()
    small = min(1 << 12, photons)
    target = oracle.forward(sc, truth, 77, small * 4, hits)["E"]
    n = min(1 << 13, photons) if name == "office" else photons
    for _ in range(args.warmup):
        oracle.forward(sc, lights, 2, photons, hits, begin=0, end=small)
    times, segs = [], 0
    for k in range(args.steps):
        t0 = time.perf_counter()
        f = oracle.forward(sc, lights, 2 + k, photons, hits, begin=0, end=n)
        _, w = oracle.loss(sc, f["E"], target, np.ones(sc.n_texels))
        _, sa = oracle.adjoint(sc, lights, 3 + k, photons, hits, w, begin=0, end=n)
        times.append(time.perf_counter() - t0)
        segs += f["segments"] + sa
    value = segs / sum(times) / 1e6
    cores = os.cpu_count() or 1
    budget = "the whole budget" if n == photons else f"the 2^{photons.bit_length() - 1} budget"
    line = {"metric": METRIC, "value": value, "unit": "Msegments/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(sc, lights, args.gpus, name),
            "cpu_baseline": {"value": value, "unit": "Msegments/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: photons [0, {n}) of {budget}, forward + loss + adjoint"},
            "e2e": {"value": value, "unit": "Msegments/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
class Adam:
    """Adam (Kingma and Ba; beta1 0.9, beta2 0.999) on the light parameters."""

    def __init__(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = self.v = None
        self.t = 0

    def step(self, x, g):
        if self.m is None:
            self.m, self.v = np.zeros_like(g), np.zeros_like(g)
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return x - self.lr * mh / (np.sqrt(vh) + self.eps)


def apply_update(lights, grad, opt):
    """Adam step on [x, y, z, yaw, pitch, p_int, theta_in] of every spot
    (theta_out stays fixed); keeps 0 <= theta_in < theta_out."""
    x = lights[:, 1:8].copy()
    x = opt.step(x, grad[:, 0:7])
    out = lights.copy()
    out[:, 1:8] = x
    out[:, 7] = np.clip(out[:, 7], 0.0, out[:, 8] - 1e-3)
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2310_02043_gb300 import shard
    from paper_2310_02043_gb300.lighttrace import Tracer

    name = args.workload
    photons, hits, target_photons = PASS[name]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    sc, lights, truth = workload(name)
    tr = Tracer(local, stream.cuda_stream)
    T = tr.upload_scene(sc)

    # Target: traced from the perturbed ("ground-truth") lights.
    tr.set_lights(truth)
    tr.trace_forward(77, target_photons, hits)
    target = torch.empty(T, dtype=torch.float32, device="cuda")
    tr.irradiance(out=target)
    tr.set_target(target)
    tr.set_lights(lights)

    # Work accounting (untimed): node visits and triangle tests per segment.
    work = tr.count_work(5, photons, hits)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    grad_dev = torch.zeros((lights.shape[0], 8), dtype=torch.float64, device="cuda")
    loss_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    # Every rank traces its own range of one common photon budget (weak
    # scaling: `photons` per GPU); the integer texel sums and the gradients
    # are summed across ranks.
    q_view = shard.device_view(tr.texel_accumulator()[0], T) if world > 1 else None
    sp = shard.ShardedPass(tr, rank, world, photons, hits, accumulator=q_view)

    for k in range(args.warmup):
        sp.step(1000 + 7919 * k, 1001 + 7919 * k, grad_dev, loss_dev)
    torch.cuda.synchronize()

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    sampler = clock_sampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    for k in range(args.steps):
        flush.zero_()
        e = ev[k]
        e[0].record(stream)
        sp.forward(1000 + 7919 * (k + 50))
        e[1].record(stream)
        sp.loss(loss_dev)
        e[2].record(stream)
        sp.adjoint(1001 + 7919 * (k + 50), grad_dev)
        e[3].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    st = tr.stats()
    seg_f, seg_a = st["segments_forward"], st["segments_adjoint"]
    t_step = [ev[k][0].elapsed_time(ev[k][3]) for k in range(args.steps)]
    t_fwd = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    t_adj = [ev[k][2].elapsed_time(ev[k][3]) for k in range(args.steps)]
    total_ms = sum(t_step)
    if world > 1:
        tt = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    segs_per_step_all = (seg_f + seg_a) * world
    value = segs_per_step_all * args.steps / (total_ms / 1e3) / 1e6

    # End to end through the C ABI with host buffers and a host Adam update.
    pinned = torch.empty((lights.shape[0], 9), dtype=torch.float64).pin_memory()
    pinned.copy_(torch.from_numpy(lights))
    grad_host = np.zeros((lights.shape[0], 8), np.float64)
    opt = Adam(lr=0.01)
    cur = lights.copy()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        tr.set_lights(pinned.numpy())
        seed = 5000 + 7919 * k
        sp.step(seed, seed + 1, grad_host)
        cur = apply_update(cur, grad_host, opt)
        pinned.copy_(torch.from_numpy(cur))
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    if world > 1:
        tt = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    e2e_value = segs_per_step_all * args.steps / e2e_s / 1e6
    h2d = LIGHT_DEV_BYTES * lights.shape[0]
    d2h = 8 + 8 * 8 * lights.shape[0]

    if rank != 0:
        tr.close()
        if world > 1:
            dist.destroy_process_group()
        return

    # Roofline of the dominant kernel (the slower of the two trace launches),
    # with its per-segment work counted by the counting kernel.
    fwd_ms = statistics.mean(t_fwd)
    adj_ms = statistics.mean(t_adj)
    adjoint_dominant = adj_ms >= fwd_ms
    dom_ms = adj_ms if adjoint_dominant else fwd_ms
    dom = "adjoint" if adjoint_dominant else "forward"
    peak_clock = clocks["sm_max_mhz"] if clocks and clocks.get("sm_max_mhz") else 2070.0
    traffic = stored_traffic(f"trace_kernel_{dom}") if name == "office" else None
    l2 = l2_read_gbs()
    staged = tr.stats()["staged_nodes"] > 0
    roofline = traversal_roofline(work, seg_a if adjoint_dominant else seg_f, dom_ms, adjoint_dominant, l2,
                                  peak_clock, traffic, name, staged)
    other = traversal_roofline(work, seg_f if adjoint_dominant else seg_a, fwd_ms if adjoint_dominant else adj_ms,
                               not adjoint_dominant, l2, peak_clock, None, name, staged)
    roofline["other_trace_kernel"] = {"kernel": other["kernel"], "achieved": other["achieved"], "frac": other["frac"],
                                      "alu_frac": other["alu"]["frac"]}
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(sc, lights, truth, name=name)
    line = {"metric": METRIC, "value": value, "unit": "Msegments/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_of(sc, lights, world, name),
            "e2e": {"value": e2e_value, "unit": "Msegments/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_opt_iter": 1e3 * e2e_s / args.steps},
            "gpu_launches": KERNELS_PER_STEP * args.steps,
            "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
            "kernel_ms": {"forward": fwd_ms, "adjoint": adj_ms,
                          "loss": statistics.mean(ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps))},
            "segments_per_step": {"forward": seg_f, "adjoint": seg_a}}
    print(json.dumps(line), flush=True)
    tr.close()
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# The office's optimisation run: 200 Adam iterations through the autograd layer
# ---------------------------------------------------------------------------
ADAM_STEPS, ADAM_LR = 200, 0.05
# Units of the optimised columns (Adam's steps are lr x these): the size of
# the ground truth's perturbation of each (position 0.3 m, yaw/pitch 0.1 rad,
# intensity parameter 15 % of its mean, inner cone 5 degrees).
ADAM_SCALE = (0.3, 0.3, 0.3, 0.1, 0.1, None, float(np.radians(5.0)), 1.0)
ADAM_OPTIMIZE = ("x", "y", "yaw", "pitch", "p_int", "theta_in")


def run_adam(args):
    """200 Adam iterations (beta 0.9/0.999, lr 0.05 in scaled units) on the 16
    office spots from the 4 x 4 grid towards ground-truth lights perturbed in
    the ceiling plane, 2^24 photons x 5 hits per iteration, decorrelated
    adjoint seeds (Sec. 4.3),
    through optim.adam (TraceObjective: forward + objective, then adjoint
    path replay): the objective and the parameter errors along the way, and
    the wall-clock ms per optimisation iteration."""
    import torch
    from paper_2310_02043_gb300 import optim
    from paper_2310_02043_gb300.lighttrace import Tracer

    torch.cuda.set_device(0)
    sc, lights, _ = workload("office")
    # ground truth moved in the ceiling plane (x, y N(0, 0.3 m), yaw/pitch
    # N(0, 0.1), intensity x U[0.7, 1.3], theta_in +- 5 deg), so that every
    # light stays inside the room
    truth = scenes.perturb_lights_in_plane(lights, 1)
    tr = Tracer(0)
    T = tr.upload_scene(sc)
    tr.set_lights(truth)
    tr.trace_forward(77, TARGET_PHOTONS, HITS)
    target = tr.irradiance()
    area = tr.texel_areas().astype(np.float64)
    norm = 0.5 * float(np.sum(area * target.astype(np.float64) ** 2))
    prob = optim.LightingProblem(sc, target, photons=PHOTONS, hits=HITS, tracer=tr)
    scale = list(ADAM_SCALE)
    scale[5] = 0.15 * float(np.mean(lights[:, 6]))
    # ceiling-mounted spots: z stays fixed (a spot moved through the ceiling
    # plane lights the ceiling's top side from a centimetre away, a jump of
    # the objective that the adjoint, with visibility frozen, does not see)
    rig = optim.LightRig(lights, optimize=ADAM_OPTIMIZE, scale=scale)
    schedule = optim.SeedSchedule(base=11)
    truth_p = truth[:, 1:9]
    # the objective's Monte Carlo floor: the ground-truth lights themselves
    floor = prob.forward_loss(truth, 3)[0] / norm

    def axis(p):
        return np.stack([np.cos(p[:, 4]) * np.cos(p[:, 3]), np.cos(p[:, 4]) * np.sin(p[:, 3]), np.sin(p[:, 4])], 1)

    def errors(r):
        p = r.lights()[:, 1:9]
        cosang = np.clip(np.sum(axis(p) * axis(truth_p), axis=1), -1.0, 1.0)
        return {"position_xy_m": float(np.sqrt(np.mean(np.sum((p[:, 0:2] - truth_p[:, 0:2]) ** 2, axis=1)))),
                "axis_rad": float(np.sqrt(np.mean(np.arccos(cosang) ** 2))),
                "p_int_rel": float(np.sqrt(np.mean(((p[:, 5] - truth_p[:, 5]) / truth_p[:, 5]) ** 2))),
                "theta_in_rad": float(np.sqrt(np.mean((p[:, 6] - truth_p[:, 6]) ** 2)))}

    start_err = errors(rig)
    warm = optim.LightRig(lights, optimize=ADAM_OPTIMIZE, scale=scale)
    optim.adam(prob, warm, max(args.warmup, 1), lr=ADAM_LR, schedule=optim.SeedSchedule(base=5))
    history = []

    def log(k, loss, r):
        if k % 10 == 9 or k == 0:
            history.append({"iteration": k + 1, "relative_objective": loss / norm, **errors(r)})

    clock = clock_sampler(0)
    clock.start()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses, _ = optim.adam(prob, rig, ADAM_STEPS, lr=ADAM_LR, schedule=schedule, callback=log)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = clock.stop()
    ms = 1e3 * wall / ADAM_STEPS
    line = {"metric": "ms per opt-iter (forward + objective + adjoint + Adam step)", "value": ms, "unit": "ms",
            "n_gpus": 1, "steps": ADAM_STEPS, "warmup": max(args.warmup, 1), "ms_per_step": ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(config_of(sc, lights, 1, "office"),
                           workload=f"procedural office ({sc.n_tri} tris, {T} texels at 2 cm), 16 spots from the "
                                    "4x4 grid towards ground-truth spots perturbed in the ceiling plane (target "
                                    "traced at 2^26); x, y, yaw, pitch, p_int, theta_in optimised, z fixed; "
                                    f"{ADAM_STEPS} Adam iterations, lr {ADAM_LR} in scaled units, 2^24 photons x 5 "
                                    "hits each, decorrelated adjoint seeds",
                           l2="not flushed (end-to-end optimisation timing)"),
            "objective": {"first": losses[0] / norm, "last": losses[-1] / norm, "at_ground_truth": floor,
                          "unit": "relative (O / (1/2 sum A E*^2)); the ground truth's value is the Monte Carlo "
                                  "floor of a 2^24-photon trace against the 2^26-photon target"},
            "units": {"lr": ADAM_LR, "scale": dict(zip(("x", "y", "z", "yaw", "pitch", "p_int", "theta_in",
                                                        "theta_out"), scale))},
            "errors": {"start": start_err, "end": errors(rig)}, "history": history,
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": LIGHT_DEV_BYTES * lights.shape[0],
                    "d2h_bytes_per_step": 8 + 8 * 8 * lights.shape[0]},
            "gpu_launches": KERNELS_PER_STEP * ADAM_STEPS, "cpu_baseline": None, "clocks": clocks}
    print(json.dumps(line), flush=True)
    tr.close()


# ---------------------------------------------------------------------------
# Batched designs: 64 candidate designs in one launch per pass
# ---------------------------------------------------------------------------
BATCH_DESIGNS, BATCH_PHOTONS = 64, 1 << 22
BATCH_KERNELS_PER_STEP = 8    # forward, loss, loss reduction, weight range, adjoint, gradient, 2 gradient reductions


def batch_config(sc, counts, shape):
    return {"workload": f"batched designs: {len(counts)} candidate lighting designs, U{{4..32}} spots each "
                        f"({int(counts.sum())} spots), over the procedural office ({sc.n_tri} tris, {sc.n_texels} "
                        f"texels), 2^22 photons per design, 5 hits, one forward + one adjoint launch per step "
                        f"(CUDA graph)",
            "designs": len(counts), "spots": int(counts.sum()), "photons_per_design": BATCH_PHOTONS, "hits": HITS,
            "launch_shape": {"threads": shape[0], "blocks_per_sm": shape[1], "smem_node_bytes": shape[2]},
            "l2": "flushed between steps (256 MiB write outside the timed events); per-design texel arrays "
                  f"{len(counts)} x {sc.n_texels * 16 / 1e6:.0f} MB exceed L2",
            "parallelism": "single GPU"}


def run_batch(args):
    """64 designs x U{4..32} spots x 2^22 photons, one batch step per
    iteration (captured CUDA graph), against the same designs traced one
    single-design pass at a time."""
    import torch
    from paper_2310_02043_gb300 import autotune
    from paper_2310_02043_gb300.lighttrace import Tracer

    torch.cuda.set_device(0)
    sc, _, truth = workload()
    counts, designs = scenes.office_designs(0, BATCH_DESIGNS)
    tr = Tracer(0)
    T = tr.upload_scene(sc)
    tr.set_lights(truth)
    tr.trace_forward(77, TARGET_PHOTONS, HITS)
    target = torch.empty(T, dtype=torch.float32, device="cuda")
    tr.irradiance(out=target)
    tr.set_target(target)
    tr.batch_setup(counts, BATCH_PHOTONS, HITS)
    tr.batch_set_lights(designs)

    key = autotune.workload_key(torch.cuda.get_device_name(0), sc.n_tri, T, BATCH_PHOTONS, HITS, len(counts))
    shape, tuned = autotune.tune(tr, lambda: tr.batch_step(1, 2, use_graph=True), key, repeats=2)

    stream = torch.cuda.ExternalStream(tr.batch_stream())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for k in range(args.warmup):
        tr.batch_step(10 + k, 20 + k, use_graph=True)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = clock_sampler(0)
    sampler.start()
    segs = 0
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev[k][0].record(stream)
        tr.batch_step(100 + 2 * k, 101 + 2 * k, use_graph=True)
        ev[k][1].record(stream)
        st = tr.stats()
        segs += st["segments_forward"] + st["segments_adjoint"]
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_step = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(t_step)
    value = segs / (total_ms / 1e3) / 1e6
    seg_step = segs / args.steps

    # The same designs, one single-design pass each (set_lights, forward,
    # objective, adjoint), on the library's main stream.
    offs = np.concatenate([[0], np.cumsum(counts)])
    main = torch.cuda.current_stream()
    seq_ms, seq_segs = [], 0
    for k in range(max(1, min(args.steps, 3))):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        a.record(main)
        for d in range(len(counts)):
            tr.set_design(d)
            tr.set_lights(designs[offs[d]:offs[d + 1]])
            tr.trace_forward(200 + k, BATCH_PHOTONS, HITS)
            tr.loss(out=torch.empty(1, dtype=torch.float64, device="cuda"))
            tr.trace_adjoint(300 + k, BATCH_PHOTONS, HITS, out=torch.empty((counts[d], 8), dtype=torch.float64,
                                                                           device="cuda"))
            st = tr.stats()
            seq_segs += st["segments_forward"] + st["segments_adjoint"]
        b.record(main)
        torch.cuda.synchronize()
        seq_ms.append(a.elapsed_time(b))
    tr.set_design(0)
    seq_value = seq_segs / (sum(seq_ms) / 1e3) / 1e6

    # End to end: host lights in, objectives and gradients out, host Adam on
    # every design's parameters.
    opt = Adam(lr=0.01)
    cur = designs.copy()
    t0 = time.perf_counter()
    for k in range(args.steps):
        tr.batch_set_lights(cur)
        loss, grad = tr.batch_step(500 + 2 * k, 501 + 2 * k, use_graph=True)
        cur = apply_update(cur, grad, opt)
    e2e_s = time.perf_counter() - t0
    e2e_value = seg_step * args.steps / e2e_s / 1e6
    h2d = 256 + LIGHT_DEV_BYTES * int(counts.sum())
    d2h = 8 * (len(counts) + 8 * int(counts.sum()) + 2)

    # Roofline of the whole step (forward + adjoint launches of all designs):
    # work per segment from the counting kernel on every 16th design
    # (single-design passes with the same design words).
    acc = {"segments": 0, "node_visits": 0, "tri_tests": 0}
    for d in range(0, len(counts), 16):
        tr.set_design(d)
        tr.set_lights(designs[offs[d]:offs[d + 1]])
        w = tr.count_work(100, BATCH_PHOTONS, HITS)
        for key in acc:
            acc[key] += w[key]
    tr.set_design(0)
    step_ms = total_ms / args.steps
    peak_clock = clocks["sm_max_mhz"] if clocks and clocks.get("sm_max_mhz") else 2070.0
    roofline = traversal_roofline(acc, seg_step, step_ms, False, l2_read_gbs(), peak_clock, None,
                                  "whole batch step: forward + adjoint of 64 designs", tr.stats()["staged_nodes"] > 0)
    line = {"metric": METRIC, "value": value, "unit": "Msegments/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": batch_config(sc, counts, shape),
            "e2e": {"value": e2e_value, "unit": "Msegments/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_opt_iter": 1e3 * e2e_s / args.steps},
            "gpu_launches": BATCH_KERNELS_PER_STEP * args.steps,
            "roofline": roofline,
            "sequential": {"value": seq_value, "unit": "Msegments/s", "ms_per_step": statistics.mean(seq_ms),
                           "what": "the same designs as single-design passes, one after another"},
            "autotune_ms": {json.dumps(list(k)): v for k, v in tuned.items()},
            "cpu_baseline": None, "clocks": clocks}
    print(json.dumps(line), flush=True)
    tr.close()


# ---------------------------------------------------------------------------
# Surrogate warm start: time to a target relative loss
# ---------------------------------------------------------------------------
SG_SOLVES, SG_SOLVE_PHOTONS, SG_STEPS, SG_BATCH = 4096, 1 << 20, 2000, 1 << 18
SG_THRESHOLD = 1e-3
# FLOPs per network row: forward 2 x (3 x 64 x 64 + 16 x 64); the design's
# backward kernel recomputes the forward and back-propagates (twice that)
SG_FWD_FLOPS = 2 * (3 * 64 * 64 + 16 * 64)


def run_surrogate(args):
    """Office at 10 cm texels, 16 spots: the seconds of optimisation until the
    tracer-judged relative objective reaches 1e-3, by adjoint light tracing
    alone and by a surrogate warm start followed by the tracer."""
    import torch
    from paper_2310_02043_gb300 import warmstart
    from paper_2310_02043_gb300.lighttrace import Tracer

    torch.cuda.set_device(0)
    sc = scenes.office(seed=0, pitch=0.1)
    tr = Tracer(0)
    T = tr.upload_scene(sc)
    area = tr.texel_areas()
    sg, info = warmstart.fit(tr, SG_SOLVES, SG_SOLVE_PHOTONS, HITS, SG_STEPS, SG_BATCH)
    # network step and design timing (CUDA events on the current stream)
    stream = torch.cuda.current_stream()
    start = scenes.office_lights(0)
    truth = scenes.perturb_lights_in_plane(start, 3)
    tr.set_lights(truth)
    tr.trace_forward(77, TARGET_PHOTONS, HITS)
    target = torch.empty(T, dtype=torch.float32, device="cuda")
    tr.irradiance(out=target)
    prob = warmstart.SurrogateProblem(sg, target)
    for _ in range(args.warmup):
        prob.forward_loss(start)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_rep = 20
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(n_rep):
        sg.design(start, target)
    b.record(stream)
    torch.cuda.synchronize()
    design_ms = a.elapsed_time(b) / n_rep
    sg.set_kernels(tcgen05=False)    # the same call with the mma.sync kernels, for comparison
    sg.design(start, target)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(n_rep):
        sg.design(start, target)
    b.record(stream)
    torch.cuda.synchronize()
    design_ms_mma = a.elapsed_time(b) / n_rep
    sg.set_kernels()
    rows = 16 * ((T + 15) // 16 * 16)
    design_flops = rows * SG_FWD_FLOPS * 2   # forward + the input gradient (no weight gradient)
    peaks = json.load(open(MEASURED_PEAKS)) if os.path.exists(MEASURED_PEAKS) else {}
    peak = peaks.get("bf16_tflops")
    peak_basis = "measured bf16 burst (MEASURED_PEAKS.json bf16_tflops), of measured"
    if not peak:
        peak, peak_basis = 1900.0, "of fallback (1.9 PFLOP/s bf16 burst, one earlier GB300 measurement)"
    a.record(stream)
    for k in range(n_rep):
        sg.train_step(99, SG_BATCH, 1e-4)
    b.record(stream)
    torch.cuda.synchronize()
    train_ms = a.elapsed_time(b) / n_rep
    sg.set_kernels(train_tcgen05=True)   # the training network on tcgen05, for comparison
    sg.train_step(99, SG_BATCH, 0.0)
    torch.cuda.synchronize()
    a.record(stream)
    for k in range(n_rep):
        sg.train_step(99, SG_BATCH, 0.0)
    b.record(stream)
    torch.cuda.synchronize()
    train_ms_tc = a.elapsed_time(b) / n_rep
    sg.set_kernels()
    held = scenes.surrogate_training_lights(777, 8)
    errs = []
    for L in held:
        tr.set_lights(L[None])
        tr.trace_forward(5, 1 << 24, HITS)
        E = tr.irradiance().astype(np.float64)
        K = sg.response(L).astype(np.float64)
        errs.append(float(np.sum(area * (K - E) ** 2) / np.sum(area * E ** 2)))

    clock = clock_sampler(0)
    clock.start()
    plain_s, plain_hist, _ = warmstart.time_to_loss(tr, sc, start, target, [("tracer", 1 << 22, 2000, 0.02)],
                                                    SG_THRESHOLD, area, max_seconds=60)
    warm_s, warm_hist, _ = warmstart.time_to_loss(
        tr, sc, start, target, [("surrogate", prob, 400, 0.02), ("tracer", 1 << 22, 2000, 0.02)], SG_THRESHOLD,
        area, max_seconds=60)
    # a tighter target: the surrogate's optimum no longer suffices and the
    # tracer refines from it
    tight = SG_THRESHOLD / 2
    plain_t, plain_thist, _ = warmstart.time_to_loss(tr, sc, start, target, [("tracer", 1 << 22, 4000, 0.02)],
                                                     tight, area, max_seconds=60)
    warm_t, warm_thist, _ = warmstart.time_to_loss(
        tr, sc, start, target, [("surrogate", prob, 200, 0.02), ("tracer", 1 << 22, 4000, 0.01)], tight, area,
        max_seconds=60)
    clocks = clock.stop()
    fit_s = info["solve_s"] + info["train_s"]
    line = {"metric": "s to relative loss 1e-3 (surrogate warm start + tracer)", "value": warm_s,
            "unit": "s", "n_gpus": 1, "steps": len(warm_hist), "warmup": args.warmup,
            "ms_per_step": None if warm_s is None else 1e3 * warm_s / max(1, warm_hist[-1][1]),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 network, f32 tracer",
            "data": "synthetic",
            "config": {"workload": f"procedural office ({sc.n_tri} tris, {T} texels at 10 cm), 16 spots from the "
                                   "4x4 grid to a target traced at 2^26 from perturbed spots; Adam lr 0.02; "
                                   "tracer 2^22 photons x 5 hits per iteration; relative loss judged every 10 "
                                   "iterations by two independent 2^24-photon traces (untimed)",
                       "surrogate": f"{SG_SOLVES} single-spot solves at 2^20 photons, {SG_STEPS} Adam steps at "
                                    f"batch 2^18", "l2": "not flushed (end-to-end optimisation timing)"},
            "plain_tracer_s": plain_s, "speedup": (plain_s / warm_s) if (plain_s and warm_s) else None,
            "fit_s": {"solves": info["solve_s"], "train": info["train_s"], "total": fit_s},
            "warm_incl_fit_s": None if warm_s is None else warm_s + fit_s,
            "heldout_rel_l2": errs, "design_ms": design_ms, "design_ms_mma_sync_forward": design_ms_mma,
            "train_step_ms": train_ms, "train_step_ms_tcgen05": train_ms_tc,
            "roofline": {"bound": "tensor", "achieved": design_flops / (design_ms / 1e3) / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "frac": design_flops / (design_ms / 1e3) / 1e12 / peak, "traffic": None,
                         "kernel": "sg_design (network forward + backward over 16 spots x all texels)",
                         "peak_basis": peak_basis},
            "tight": {"threshold": tight, "plain_s": plain_t, "warm_s": warm_t,
                      "history": {"plain": plain_thist, "warm": warm_thist}},
            "history": {"plain": plain_hist, "warm": warm_hist}, "cpu_baseline": None, "clocks": clocks,
            "e2e": {"value": warm_s, "unit": "s", "h2d_bytes_per_step": 16 * 36, "d2h_bytes_per_step": 16 * 64 + 8},
            "gpu_launches": None}
    print(json.dumps(line), flush=True)
    sg.close()
    tr.close()


# ---------------------------------------------------------------------------
# Large building: 64 area lights, 2^26 photons, 6 hits
# ---------------------------------------------------------------------------
BLD_PHOTONS, BLD_HITS = 1 << 26, 6


def run_building(args):
    """Forward + objective + adjoint on the procedural building (961,792
    tris, 17.2 M texels at 4.5 cm, 64 ceiling-panel area lights), and
    L-BFGS on the 64 powers with adjoint path replay (ms per evaluation)."""
    import torch
    from paper_2310_02043_gb300 import optim
    from paper_2310_02043_gb300.lighttrace import Tracer

    torch.cuda.set_device(0)
    sc, L = scenes.building(), scenes.building_lights()
    tr = Tracer(0)
    t0 = time.perf_counter()
    T = tr.upload_scene(sc)
    upload_s = time.perf_counter() - t0
    truth = L.copy()
    truth[:, 6] *= np.sqrt(np.random.default_rng(5).uniform(0.6, 1.4, L.shape[0]))
    truth[:, 1:3] += np.random.default_rng(6).normal(0.0, 0.3, (L.shape[0], 2))
    tr.set_lights(truth)
    tr.trace_forward(77, BLD_PHOTONS, BLD_HITS)
    target = torch.empty(T, dtype=torch.float32, device="cuda")
    tr.irradiance(out=target)
    tr.set_target(target)
    tr.set_lights(L)
    work = tr.count_work(5, 1 << 24, BLD_HITS)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    grad = torch.zeros((L.shape[0], 8), dtype=torch.float64, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in range(args.warmup):
        tr.trace_forward(100 + k, BLD_PHOTONS, BLD_HITS)
        tr.loss(out=loss)
        tr.trace_adjoint(200 + k, BLD_PHOTONS, BLD_HITS, out=grad)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    clock = clock_sampler(0)
    clock.start()
    segs = 0
    for k in range(args.steps):
        flush.zero_()
        e = ev[k]
        e[0].record(stream)
        tr.trace_forward(1000 + 2 * k, BLD_PHOTONS, BLD_HITS)
        tr.loss(out=loss)
        e[1].record(stream)
        tr.trace_adjoint(1001 + 2 * k, BLD_PHOTONS, BLD_HITS, out=grad)
        e[2].record(stream)
        torch.cuda.synchronize()
        st = tr.stats()
        segs += st["segments_forward"] + st["segments_adjoint"]
        seg_adj = st["segments_adjoint"]
    clocks = clock.stop()
    t_f = [e[0].elapsed_time(e[1]) for e in ev]
    t_a = [e[1].elapsed_time(e[2]) for e in ev]
    total_ms = sum(t_f) + sum(t_a)
    value = segs / (total_ms / 1e3) / 1e6
    # end to end: L-BFGS on the 64 powers, host parameters, 2^26 photons per evaluation
    start = L.copy()
    start[:, 6] *= np.sqrt(np.random.default_rng(7).uniform(0.5, 1.5, L.shape[0]))
    prob = optim.LightingProblem(sc, target.cpu().numpy(), photons=BLD_PHOTONS, hits=BLD_HITS, tracer=tr)
    rig = optim.LightRig(start, optimize=("p_int",))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trace = optim.lbfgs(prob, rig, max_iter=max(2, args.steps), seed=9)
    torch.cuda.synchronize()
    lbfgs_s = time.perf_counter() - t0
    evals = prob.evaluations
    e2e_value = evals * BLD_PHOTONS * BLD_HITS * 2 / lbfgs_s / 1e6
    fwd_ms = statistics.mean(t_f)
    adj_ms = statistics.mean(t_a)
    peak_clock = clocks["sm_max_mhz"] if clocks and clocks.get("sm_max_mhz") else 2070.0
    traffic = None
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "trace_kernel_building_traffic.json")))
        if d.get("kernel_source_sha256_16") == kernel_hash():
            traffic = d["trace_kernel_adjoint"]["dram_bytes_per_segment"]
    except (OSError, ValueError, KeyError):
        pass
    # the adjoint launch (its time excludes the objective, which the forward
    # interval includes)
    roofline = traversal_roofline(work, seg_adj, adj_ms, True,
                                  l2_read_gbs(), peak_clock, traffic, "building, BVH through L1/L2", staged=False)
    line = {"metric": METRIC, "value": value, "unit": "Msegments/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"procedural building: 8 storeys 48x24 m, {sc.n_tri} tris (tessellated floors, "
                                   f"walls, columns, partitions, furniture), {T} texels at 4.5 cm, 64 rectangular "
                                   "area lights, 2^26 photons, 6 hits",
                       "triangles": sc.n_tri, "texels": T, "bvh_nodes": tr.stats()["n_nodes"], "lights": 64,
                       "photons": BLD_PHOTONS, "hits": BLD_HITS, "scene_upload_s": upload_s,
                       "l2": "flushed between steps (256 MiB write outside the timed events)",
                       "parallelism": "single GPU"},
            "e2e": {"value": e2e_value, "unit": "Msegments/s", "h2d_bytes_per_step": LIGHT_DEV_BYTES * 64,
                    "d2h_bytes_per_step": 8 + 64 * 64, "what": "L-BFGS (strong Wolfe) on the 64 powers",
                    "evaluations": evals, "ms_per_evaluation": 1e3 * lbfgs_s / max(1, evals),
                    "objective": [trace[0], trace[-1]]},
            "gpu_launches": KERNELS_PER_STEP * args.steps,
            "roofline": roofline,
            "kernel_ms": {"forward_and_loss": fwd_ms, "adjoint": adj_ms},
            "cpu_baseline": None, "clocks": clocks}
    print(json.dumps(line), flush=True)
    tr.close()


def run_profile_building(args):
    """One forward + loss + adjoint of the building at --photons (for ncu)."""
    import torch
    from paper_2310_02043_gb300.lighttrace import Tracer
    torch.cuda.set_device(0)
    sc, L = scenes.building(), scenes.building_lights()
    tr = Tracer(0)
    T = tr.upload_scene(sc)
    tr.set_target(np.zeros(T, np.float32))
    tr.set_lights(L)
    tr.trace_forward(2, args.photons, BLD_HITS)
    tr.loss()
    tr.trace_adjoint(3, args.photons, BLD_HITS)
    st = tr.stats()
    tr.close()
    print(json.dumps({"profile_case": "building", "photons": args.photons, "segments_forward": st["segments_forward"],
                      "segments_adjoint": st["segments_adjoint"]}))


def run_profile_surrogate(args):
    """A small surrogate fit (64 solves at 2^18 photons), 5 training steps at
    batch 2^18 and 3 design evaluations of the 16 office spots (for ncu)."""
    import torch
    from paper_2310_02043_gb300 import warmstart
    from paper_2310_02043_gb300.lighttrace import Tracer
    torch.cuda.set_device(0)
    sc = scenes.office(seed=0, pitch=0.1)
    tr = Tracer(0)
    T = tr.upload_scene(sc)
    sg, _ = warmstart.fit(tr, 64, 1 << 18, HITS, 5, SG_BATCH)
    target = torch.zeros(T, dtype=torch.float32, device="cuda")
    for _ in range(3):
        sg.design(scenes.office_lights(0), target)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": "surrogate", "texels": T}))
    sg.close()
    tr.close()


def run_profile_case(args):
    """One forward + loss + adjoint of the office at --photons (for ncu)."""
    import torch
    from paper_2310_02043_gb300.lighttrace import Tracer
    torch.cuda.set_device(0)
    name = args.workload if args.workload in PASS else "office"
    hits = PASS[name][1]
    sc, lights, _ = workload(name)
    tr = Tracer(0)
    T = tr.upload_scene(sc)
    tr.set_target(np.zeros(T, np.float32))
    tr.set_lights(lights)
    tr.trace_forward(2, args.photons, hits)
    tr.loss()
    tr.trace_adjoint(3, args.photons, hits)
    st = tr.stats()
    tr.close()
    print(json.dumps({"profile_case": True, "photons": args.photons, "segments_forward": st["segments_forward"],
                      "segments_adjoint": st["segments_adjoint"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", action="store_true",
                    help="run one forward + loss + adjoint at --photons and exit (for profilers)")
    ap.add_argument("--photons", type=int, default=1 << 20)
    ap.add_argument("--workload", choices=["office", "cornell", "adam", "batch", "surrogate", "building"],
                    default="office",
                    help="office: one design, 16 spots (default); cornell: the Cornell box, 1 point light, 2^18 "
                         "photons, 3 hits; adam: 200 Adam iterations on the office; batch: 64 designs in one launch per pass; surrogate: time to a target "
                         "loss with the surrogate warm start; building: 961,792 tris, 64 area lights, 2^26 photons, "
                         "6 hits")
    args = ap.parse_args()
    if args.workload == "batch" and args.impl == "ours" and not args.profile_only:
        run_batch(args)
        return
    if args.workload == "surrogate" and args.impl == "ours":
        run_profile_surrogate(args) if args.profile_only else run_surrogate(args)
        return
    if args.workload == "adam" and args.impl == "ours":
        run_adam(args)
        return
    if args.workload == "building" and args.impl == "ours":
        run_profile_building(args) if args.profile_only else run_building(args)
        return
    if args.profile_only:
        run_profile_case(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
