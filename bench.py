#!/usr/bin/env python3
"""Benchmark of the shearlet-regularised segmentation ADMM on GB300.

One step = one whole solve on the 512 x 512 workload (grayscale, K = 4 labels,
J = 4 scales / 61 filters, 500 ADMM iterations, curved Bezier regions with
oriented gratings and noise sigma = 0.05): data term and zero state
(seg_admm_reset), 500 iterations (graph replays), label readout.  The metric
is Mpixel*label*ADMM-iteration per second summed over all ranks.  The work
plan is autotuned on the image before the timed region (--no-tune keeps the
default).  At N = 1 the line also carries `batched`: the same metric for the
64-image uneven batch (one graph per iteration with a branch per image), one
timed step of 300 iterations after three short warm-up steps, beside the same
images solved one after another through the single-image path (--no-batch
skips both), `differentiable`: 16 images of 256 x 256 through the unrolled
forward and reverse sweeps beside the same images solved one after another
(--no-differentiable skips it), and `workloads`: the 2048 x 2048 RGB image
(K = 8, J = 5, 20 of its iterations per step) and the 64 x 64 image (K = 3,
J = 2, 200 iterations) through the same path, and the TV-regularised model of
Sec. 4 on the 512 x 512 image (`tv512`, gamma = 1, lambda = 1/12, 100
iterations) and the NL-means-regularised model of Sec. 4 on it (`nl512`, the
paper's p = 5, varpi = 15, a = 2, mt = 5, gamma = 1/5, lambda = 1/32, 100
iterations; graph built once); the line, tv512 and nl512 carry each model's
label error against the generator's label map (--no-legs skips them).  The
line reports the dominant kernel's HBM roofline and, for the whole iteration,
the method's algorithmic bytes and FP32 operations over the plain iteration
time against the measured HBM bandwidth and the FP32 peak from the unit
counts.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 is launched by torchrun: every rank solves its own copy of the image
(independent problems, no collective on the data path; weak scaling), and the
`batched` leg shards the 64 images whole across the ranks by LPT on their cost
(strong scaling of the fixed batch; the time is the largest over the ranks).
--impl reference times the FP64 CPU oracle (the baseline arm) on a bounded
sample of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1112_1805_gb300 import synth  # noqa: E402

METRIC = "Mpixel·label·ADMM-iter/s, batched vs plain, at ≤1e-4 err; HBM % of peak"
UNIT = "Mpixel·label·iter/s"
WORKLOAD = "bezier512"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--cpu-iters", type=int, default=2, help="oracle iterations in the CPU-baseline sample")
    ap.add_argument("--workload", choices=["bezier512", "batch", "differentiable", "rgb2048", "tv512", "nl512"],
                    default="bezier512",
                    help="bezier512 (default line), the uneven batch of 64 images, the unrolled workload, the "
                         "2048 x 2048 RGB image (K = 8, J = 5; 20 iterations per step unless --iters is given), or "
                         "the 512 x 512 image with the TV or NL-means regulariser of Sec. 4")
    ap.add_argument("--images", type=int, default=16, help="images of the differentiable workload")
    ap.add_argument("--no-differentiable", action="store_true",
                    help="skip the unrolled forward+reverse measurement the default line carries under 'differentiable'")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched measurement that the default line carries under 'batched'")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the 2048 x 2048 RGB and 64 x 64 legs that the default line carries under 'workloads'")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the default work plan instead of autotuning it before the timed region")
    ap.add_argument("--plan", default="",
                    help="fixed work plan fields for profiling runs, e.g. 'wave_mib=256,row_kernel=2' (implies "
                         "--no-tune for the main workload)")
    ap.add_argument("--iters", type=int, default=0,
                    help="ADMM iterations per step for short profiling runs (default: the workload's 500)")
    return ap.parse_args()


def workload_config(wl, extra=None):
    bv_mb = 4 * wl.K * wl.eta * wl.H * wl.W / 1e6
    scene = ("seeded ellipses on a background label, N(0, 0.05^2) noise" if wl.name in ("ellipses64", "unrolled256")
             else "seeded closed-Bezier regions with oriented gratings (amplitude 0.15) and N(0, 0.05^2) noise")
    l2 = (f"no flush: per-iteration working set (b_v {bv_mb:.0f} MB + coefficient spectra) exceeds the 129 MB L2"
          if bv_mb > 129 else f"L2-resident (b_v {bv_mb:.1f} MB): no flush, a latency-bound size")
    cfg = {
        "workload": f"{wl.name}: {wl.H}x{wl.W} {'RGB' if wl.C == 3 else 'gray'}, K={wl.K}, J={wl.J} (eta={wl.eta}), "
                    f"{wl.iters} ADMM iterations, {scene}",
        "H": wl.H, "W": wl.W, "C": wl.C, "K": wl.K, "J": wl.J, "eta": wl.eta, "iters_per_step": wl.iters,
        "lambda": wl.lam, "gamma": wl.gamma, "Lambda": [round(float(x), 6) for x in wl.Lambda()],
        "l2": l2,
        "parallelism": "replicas (one independent image per GPU)",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, n = [], None, set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            n += 1
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        loaded = [x for x in sm if smax and x > 0.5 * smax] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": n}


# ---------------------------------------------------------------------------
# roofline bookkeeping: algorithmic bytes per launch of each kernel
# ---------------------------------------------------------------------------
def kernel_bytes(wl):
    """Compulsory DRAM bytes of one iteration per kernel kind: every operand the
    kind must read from, and every result it must leave in, device memory.
    Coefficient spectra of a wave of filters are scratch that stays in L2 and
    are not counted; the dual b_v (read and written once per iteration) is."""
    H, W, K, eta = wl.H, wl.W, wl.K, wl.eta
    P, Ph = H * W, H * (W // 2 + 1)
    return {
        "row_ustep": K * (2 * Ph * 8 + 6 * P * 4),  # T in, row spectra of u out; s, w, b_w in; u, w, b_w out
        "col_fwd": K * 2 * Ph * 8,                  # row spectra in, 2-D spectra of u out
        "col_fan": K * Ph * 8 + eta * Ph * 4,       # spectra of u and the filter bank in
        "row_shrink": K * eta * P * 8,              # b_v in and out
        "col_gather": eta * Ph * 4,                 # the filter bank in
        "col_reduce_inv": K * Ph * 8 * 2,           # group sums in (at least one), T out
    }


def iteration_bytes(wl):
    """Algorithmic HBM bytes of one iteration: per pixel and label 8 eta (b_v
    read and written) + 24 (s, w, b_w in; u, w, b_w out, as FP32) + the filter
    bank read once per label, 4 eta (W/2+1)/W / K per pixel and label when the
    bank is shared by the K labels of a wave (it is re-read per label here)."""
    P, K, eta = wl.H * wl.W, wl.K, wl.eta
    per = 8 * eta + 24 + 4 * eta * (wl.W // 2 + 1) / wl.W
    return int(per * P * K)


def iteration_flops(wl):
    """FP32 operations of one iteration as the method's arithmetic (not the
    instructions issued): per (label, filter) one inverse and one forward real
    2-D FFT of H x W at 2.5 P log2 P each (the radix-2 count of a real
    transform), the filter product on the half plane in both directions
    (4 H (W/2+1)) and the shrinkage and dual update (6 per coefficient); per
    label the forward FFT of u and the inverse FFT of the synthesis sum, the
    u-step (4 per pixel) and the simplex projection (about 4 K per pixel)."""
    import math

    P, K, eta = wl.H * wl.W, wl.K, wl.eta
    Ph = wl.H * (wl.W // 2 + 1)
    fft2 = 2.5 * P * math.log2(P)
    per_pair = 2 * fft2 + 4 * Ph + 6 * P
    per_label = 2 * fft2 + 4 * P + 4 * K * P
    return K * (eta * per_pair + per_label)


def fp32_peak_tflops(sm_mhz):
    """FP32 peak of the GPU from its unit counts: SMs x 128 FP32 lanes x 2
    (an FMA counted as two operations) x SM clock."""
    import torch

    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = sm_mhz or 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12, sms, mhz


def source_sha() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1112_1805_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_1112_1805_gb300", "csrc", f), "rb") as fp:
            h.update(fp.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel: str, plan=None):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources and with the same wave size (a launch's work
    depends on it); else None."""
    try:
        with open(TRAFFIC_FILE) as fp:
            t = json.load(fp)
    except (OSError, ValueError):
        return None
    if t.get("source_sha") != source_sha():
        return None
    if plan is not None and "wave_mib" in t and plan.get("wave_mib") != t["wave_mib"]:
        return None
    k = t.get("kernels", {}).get(kernel)
    return None if k is None else float(k["dram_bytes_per_launch"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fp:
            p = json.load(fp)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(wl, img, iters: int):
    import oracle

    oracle.build()
    cb = wl.codebook()
    t0 = time.perf_counter()
    s = oracle.data_term(img, cb)
    st = oracle.zero_state(wl.K, wl.J, wl.H, wl.W)
    oracle.admm_iterate(st, s, wl.J, wl.Lambda(), wl.gamma, iters)
    dt = time.perf_counter() - t0
    units = wl.H * wl.W * wl.K * iters
    return units / dt / 1e6, dt, oracle.get_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    img, lab, wl = synth.make_workload_image(WORKLOAD)
    for _ in range(args.warmup):
        oracle_sample(wl, img, 1)
    vals, times = [], []
    cores = 0
    for _ in range(args.steps):
        v, dt, cores = oracle_sample(wl, img, 1)
        vals.append(v)
        times.append(dt)
    value = wl.H * wl.W * wl.K * len(times) / sum(times) / 1e6
    sample = (f"{wl.name} at full size, data term + 1 ADMM iteration per step (filter bank built per step, as the "
              f"oracle does), FP64, {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wl, {"iters_per_step": 1}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    import dataclasses

    name = "rgb2048" if args.workload == "rgb2048" else WORKLOAD
    img, lab, wl = synth.make_workload_image(name)
    if args.iters > 0:
        wl = dataclasses.replace(wl, iters=args.iters)
    elif name == "rgb2048":
        wl = dataclasses.replace(wl, iters=20)
    # the CPU-baseline leg runs first (rank 0, N = 1), before any GPU work
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and name == WORKLOAD:
        v, dt, cores = oracle_sample(wl, img, args.cpu_iters)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{wl.name} at full size, data term + {args.cpu_iters} ADMM iterations "
                         f"({dt:.1f} s, FP64, filter bank built inside the timed call)"}

    img32 = np.ascontiguousarray(img, dtype=np.float32)
    f_dev = torch.tensor(img32, device="cuda")
    fb = FilterBank(wl.H, wl.W, wl.J)
    seg = ShearletSegmenter(fb, f_dev, wl.codebook(), wl.Lambda(), wl.gamma)
    # work plan: autotuned on this image before the timed region (iterate restored)
    if args.plan:
        fixed = seg.plan()
        for kv in args.plan.split(","):
            k, v = kv.split("=")
            fixed[k.strip()] = int(v)
        seg.set_plan(fixed)
        plan = seg.plan()
    else:
        plan = seg.plan() if args.no_tune else seg.tune(10)
    labels_dev = torch.empty((wl.H, wl.W), dtype=torch.int32, device="cuda")
    st = seg.stream
    units_per_step = wl.H * wl.W * wl.K * wl.iters

    def device_step():
        B.seg_admm_reset(seg.handle, f_dev.data_ptr(), False)
        B.seg_admm_step(seg.handle, wl.iters)
        B.seg_admm_get(seg.handle, B.SEG_LABELS, labels_dev.data_ptr(), False)

    for _ in range(args.warmup):
        device_step()
    seg.synchronize()
    torch.cuda.synchronize()
    label_error = float((labels_dev.cpu().numpy() != lab).mean())

    # timed region: K steps bracketed by barrier + synchronize, CUDA events on the state's stream
    clocks = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    ktimes = []
    for _ in range(args.steps):
        device_step()
        try:
            ktimes.append(B.seg_admm_kernel_times(seg.handle))  # last iteration of this step
        except B.ShearsegError:  # more launches per iteration than timing marks
            ktimes.append(None)
    ev1.record(st)
    ev1.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    t = torch.tensor([ms_total], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = units_per_step * args.steps * world / (ms_max / 1000.0) / 1e6

    # end-to-end through the public API with host buffers (pinned), copies inside
    host_img = torch.from_numpy(img32).pin_memory()
    host_labels = torch.empty((wl.H, wl.W), dtype=torch.int32).pin_memory()
    seg.get_host(B.SEG_LABELS, host_labels)
    barrier()
    e2e_times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        seg.reset(host_img)
        seg.step(wl.iters)
        seg.get_host(B.SEG_LABELS, host_labels)  # synchronises
        e2e_times.append(time.perf_counter() - t0)
    et = torch.tensor([sum(e2e_times)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(et, op=dist.ReduceOp.MAX)
    e2e_value = units_per_step * args.steps * world / float(et.item()) / 1e6

    # roofline of the dominant kernel kind (largest share of the iteration)
    roofline, iteration, n_launch = None, None, None
    if ktimes and all(t is not None for t in ktimes):
        kinds = [k for k in ktimes[0] if ktimes[0][k][1] > 0]
        mean_ms = {k: statistics.mean(t[k][0] for t in ktimes) for k in kinds}
        n_launch = {k: ktimes[0][k][1] for k in kinds}
        dom = max(mean_ms, key=mean_ms.get)
        kb = kernel_bytes(wl)
        peak, peak_kind = peaks()
        achieved = kb[dom] / (mean_ms[dom] / 1000.0) / 1e9
        it_ms = sum(mean_ms.values())
        traffic = measured_traffic(dom, plan)
        roofline = {
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": dom, "launches_per_iteration": n_launch[dom],
            "kernel_ms_per_launch": mean_ms[dom] / n_launch[dom],
            "algorithmic_bytes_per_launch": kb[dom] / n_launch[dom], "peak_source": f"{peak_kind} hbm_gbs",
        }
        if traffic is not None:
            # the same launch in DRAM bytes (ncu) over its live CUDA-event time
            roofline["traffic_gbs"] = traffic / (mean_ms[dom] / n_launch[dom] / 1000.0) / 1e9
            roofline["traffic_frac"] = roofline["traffic_gbs"] / peak
        # whole iteration: the method's bytes and flops over the plain graph's
        # time per iteration (the step's time over its iterations: it also
        # holds the reset and the readout, so this slightly understates)
        plain_ms = ms_max / args.steps / wl.iters
        iter_alg = iteration_bytes(wl)
        flops = iteration_flops(wl)
        fpk, sms, mhz = fp32_peak_tflops(clk["sm_mhz"])
        iteration = {"instrumented_ms": it_ms, "kernel_ms": mean_ms, "launches": n_launch,
                     "plain_ms": plain_ms, "algorithmic_bytes": iter_alg,
                     "hbm_frac_algorithmic": iter_alg / (plain_ms / 1000.0) / 1e9 / peak,
                     "fp32": {"flops": flops, "achieved_tflops": flops / (plain_ms / 1000.0) / 1e12,
                              "peak_tflops": fpk, "frac": flops / (plain_ms / 1000.0) / 1e12 / fpk,
                              "peak_derivation": f"{sms} SMs x 128 FP32 lanes x 2 (FMA) x {mhz:.0f} MHz "
                                                 "(median SM clock under load)"}}
    launches_per_step = 2 + (sum(n_launch.values()) * wl.iters if n_launch else 0) + 1
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(wl),
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                   "samples": clk["samples"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(host_img.numel() * 4),
                "d2h_bytes_per_step": int(host_labels.numel() * 4)},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline,
        "plan": plan,
        "iteration": iteration,
        "label_error": label_error,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    seg.close()
    fb.close()
    if rank == 0 and world == 1 and not args.no_legs and name == WORKLOAD:
        # the other single-image workloads: 2048 x 2048 RGB (K = 8, J = 5; 20 of
        # its 1000 iterations per step) and 64 x 64 (K = 3, J = 2, 200 iterations)
        line["workloads"] = {"rgb2048": measure_leg("rgb2048", 20, 3, 3, not args.no_tune),
                             "ellipses64": measure_leg("ellipses64", 200, 5, 3, not args.no_tune),
                             "tv512": measure_tv(100, 5, 3),
                             "nl512": measure_nl(100, 3, 2)}
    if not args.no_batch and name == WORKLOAD:
        # the batched form on the same GPUs (the plain state is released
        # first): the 64-image batch sharded over the ranks
        b = measure_batch(300, 1, 3, 30, not args.no_tune, rank, world)
        if rank == 0:
            line["batched"] = b
    if rank == 0 and world == 1 and not args.no_differentiable and name == WORKLOAD:
        line["differentiable"] = measure_differentiable(2, 1)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def measure_leg(name: str, iters: int, steps: int, warmup: int, tune: bool):
    """Another single-image workload on the same GPU, timed like the main
    line (reset + `iters` graph-replayed iterations + label readout per step,
    CUDA events on the state's stream), with the roofline of its dominant
    kernel kind and the whole iteration's algorithmic bytes and flops."""
    import dataclasses

    import torch

    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    img, _, wl = synth.make_workload_image(name)
    wl = dataclasses.replace(wl, iters=iters)
    f_dev = torch.tensor(np.ascontiguousarray(img, dtype=np.float32), device="cuda")
    fb = FilterBank(wl.H, wl.W, wl.J)
    seg = ShearletSegmenter(fb, f_dev, wl.codebook(), wl.Lambda(), wl.gamma)
    plan = seg.tune(3) if tune else seg.plan()
    labels_dev = torch.empty((wl.H, wl.W), dtype=torch.int32, device="cuda")

    def device_step():
        B.seg_admm_reset(seg.handle, f_dev.data_ptr(), False)
        B.seg_admm_step(seg.handle, wl.iters)
        B.seg_admm_get(seg.handle, B.SEG_LABELS, labels_dev.data_ptr(), False)

    for _ in range(warmup):
        device_step()
    seg.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(seg.stream)
    kt = []
    for _ in range(steps):
        device_step()
        try:
            kt.append(B.seg_admm_kernel_times(seg.handle))
        except B.ShearsegError:
            kt.append(None)
    ev1.record(seg.stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    seg.close()
    fb.close()
    del f_dev
    torch.cuda.empty_cache()
    units = wl.H * wl.W * wl.K * wl.iters * steps
    plain_ms = ms / steps / wl.iters
    peak, peak_kind = peaks()
    out = {"value": units / (ms / 1000.0) / 1e6, "unit": UNIT, "steps": steps, "warmup": warmup,
           "iters_per_step": wl.iters, "ms_per_step": ms / steps, "plan": plan,
           "config": workload_config(wl),
           "iteration": {"plain_ms": plain_ms, "algorithmic_bytes": iteration_bytes(wl),
                         "hbm_frac_algorithmic": iteration_bytes(wl) / (plain_ms / 1000.0) / 1e9 / peak,
                         "fp32_tflops": iteration_flops(wl) / (plain_ms / 1000.0) / 1e12}}
    if kt and all(t is not None for t in kt):
        kinds = [k for k in kt[0] if kt[0][k][1] > 0]
        mean_ms = {k: statistics.mean(t[k][0] for t in kt) for k in kinds}
        n_launch = {k: kt[0][k][1] for k in kinds}
        dom = max(mean_ms, key=mean_ms.get)
        kb = kernel_bytes(wl)
        achieved = kb[dom] / (mean_ms[dom] / 1000.0) / 1e9
        out["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                           "frac": achieved / peak, "launches_per_iteration": n_launch[dom],
                           "kernel_ms_per_launch": mean_ms[dom] / n_launch[dom],
                           "peak_source": f"{peak_kind} hbm_gbs"}
        out["iteration"]["kernel_ms"] = mean_ms
        out["iteration"]["launches"] = n_launch
    return out


def tv_kernel_bytes(H, W, K):
    """Compulsory DRAM bytes of one TV iteration per kernel: the u-step's three
    transforms (right-hand side in, half spectra through, u out; the symbol
    read once) and the two pointwise kernels (the prox kernel reads u, b_v,
    b_w, s and writes b_v, d, w, b_w, q: 48 B per pixel and label; the
    right-hand side reads q and d and writes rhs: 16 B)."""
    P, Ph = H * W, H * (W // 2 + 1)
    return {"tv_row_fwd": K * (P * 4 + Ph * 8), "tv_col_solve": K * 2 * Ph * 8 + Ph * 4,
            "tv_row_inv": K * (Ph * 8 + P * 4), "tv_prox": K * P * 48, "tv_rhs": K * P * 16}


def measure_tv(iters: int, steps: int, warmup: int, lam: float = 1.0 / 12.0):
    """The TV-regularised model of Sec. 4 on the 512 x 512 textured image
    (K = 4) with the paper's TV weights of its stripes and fish runs (gamma =
    1, lambda = 1/12, 100 iterations): the comparison model on the same
    image and GPU.  Also the label error of both models against the
    generator's label map (the paper's comparison on curved textures)."""
    import torch

    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import TVSegmenter

    img, lab, wl = synth.make_workload_image("bezier512")
    f_dev = torch.tensor(np.ascontiguousarray(img, dtype=np.float32), device="cuda")
    seg = TVSegmenter(f_dev, wl.codebook(), lam, 1.0)
    labels_dev = torch.empty((wl.H, wl.W), dtype=torch.int32, device="cuda")

    def device_step():
        B.tv_admm_reset(seg.handle, f_dev.data_ptr(), False)
        B.tv_admm_step(seg.handle, iters)
        B.tv_admm_get(seg.handle, B.SEG_LABELS, labels_dev.data_ptr(), False)

    for _ in range(warmup):
        device_step()
    seg.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(seg.stream)
    for _ in range(steps):
        device_step()
    ev1.record(seg.stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    label_error = float((labels_dev.cpu().numpy() != lab).mean())
    kt = seg.kernel_times(5)
    seg.close()
    units = wl.H * wl.W * wl.K * iters * steps
    kb = tv_kernel_bytes(wl.H, wl.W, wl.K)
    dom = max(kt, key=kt.get)
    peak, peak_kind = peaks()
    achieved = kb[dom] / (kt[dom] / 1000.0) / 1e9
    return {"value": units / (ms / 1000.0) / 1e6, "unit": UNIT, "steps": steps, "warmup": warmup,
            "iters_per_step": iters, "ms_per_step": ms / steps, "label_error": label_error,
            "kernel_ms": kt, "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                                          "unit": "GB/s", "frac": achieved / peak,
                                          "peak_source": f"{peak_kind} hbm_gbs"},
            "workload": f"tv512: bezier512's image (512x512 gray, K=4) with the TV regulariser of Sec. 4 "
                        f"(labels coupled per pixel, periodic forward differences), gamma=1, lambda=1/12, "
                        f"{iters} ADMM iterations per step"}


def measure_nl(iters: int, steps: int, warmup: int, lam: float = 1.0 / 32.0, gamma: float = 0.2):
    """The NL-means-regularised model of Sec. 4 on the 512 x 512 textured
    image (K = 4) with the paper's NL settings (p = 5, varpi = 15, a = 2,
    mt = 5; gamma = 1/5, lambda = 1/32, 100 iterations).  The neighbour
    graph depends on the image only: it is built once (timed separately) and
    the timed steps run the iterations from the zero state."""
    import torch

    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import NLSegmenter

    img, lab, wl = synth.make_workload_image("bezier512")
    f_dev = torch.tensor(np.ascontiguousarray(img, dtype=np.float32), device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seg = NLSegmenter(f_dev, wl.codebook(), lam, gamma)
    graph_s = time.perf_counter() - t0
    nbr, deg, cheb = seg.graph()
    zero_k = torch.zeros((wl.K, wl.H, wl.W), device="cuda")
    zero_v = torch.zeros((wl.K, seg.m, wl.H, wl.W), device="cuda")

    def zero_state():
        for what, z in ((B.SEG_BV, zero_v), (B.SEG_V, zero_v), (B.SEG_W, zero_k), (B.SEG_BW, zero_k),
                        (B.SEG_U, zero_k)):
            seg.set(what, z)

    ms = 0.0
    for step in range(warmup + steps):
        zero_state()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(seg.stream)
        seg.step(iters)
        ev1.record(seg.stream)
        ev1.synchronize()
        if step >= warmup:
            ms += ev0.elapsed_time(ev1)
    label_error = float((seg.labels().cpu().numpy() != lab).mean())
    kt = seg.kernel_times(3)
    seg.close()
    P, K, m = wl.H * wl.W, wl.K, 2 * 5
    units = P * K * iters * steps
    # Chebyshev step: x, rhs, d in; x, d out (20 B per pixel and label) + the
    # neighbour offsets and counts (2 m + 1 B per pixel)
    solve_bytes = cheb * (K * P * 20 + P * (2 * m + 1))
    peak, peak_kind = peaks()
    achieved = solve_bytes / (kt["nl_solve"] / 1000.0) / 1e9
    return {"value": units / (ms / 1000.0) / 1e6, "unit": UNIT, "steps": steps, "warmup": warmup,
            "iters_per_step": iters, "ms_per_step": ms / steps, "label_error": label_error, "kernel_ms": kt,
            "graph_build_s": graph_s, "chebyshev_steps_per_u_step": cheb, "mean_neighbours": float(deg.mean()),
            "roofline": {"bound": "hbm", "kernel": "nl_solve (Chebyshev steps)", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs"},
            "workload": f"nl512: bezier512's image (512x512 gray, K=4) with the NL-means regulariser of Sec. 4 "
                        f"(p=5, varpi=15, a=2, mt=5), gamma=1/5, lambda=1/32, {iters} ADMM iterations per step "
                        f"from the zero state; the graph (built once per image, graph_build_s) is not in the steps"}


def measure_batch(iters: int, steps: int, warmup_steps: int, warmup_iters: int, tune: bool, rank: int = 0,
                  world: int = 1):
    """The uneven batch: 64 seeded images (384 x 640 first, sides 128..1024), K
    in 2..6, J = floor(log2(min side)/2).  With N ranks the images are sharded
    whole by LPT on their cost (shard.share; no collective on the data path)
    and each rank solves its share as one batch (one CUDA graph per
    iteration); the time is the largest over the ranks (strong scaling: the
    batch is fixed).  Returns the summed Mpixel*label*iter/s and its timing;
    at N = 1 also the same images solved one after another."""
    import torch
    import torch.distributed as dist

    from paper_1112_1805_gb300 import shard
    from paper_1112_1805_gb300.api import ShearletBatch

    shapes = synth.batch_shapes()
    rng = np.random.default_rng(synth.seed_for(3))
    host, cbs, lams, units = [], [], [], 0
    for H, W, K, J in shapes:  # every rank draws every image, in order, and keeps its share
        cb = np.array([[0.2 + 0.6 * k / (K - 1)] for k in range(K)])
        img, _ = synth.ellipse_image(H, W, cb, rng)
        host.append(img.astype(np.float32))
        cbs.append(cb)
        lams.append(synth.scale_weights(0.1, J))
        units += H * W * K * iters
    mine = shard.share(shapes, rank, world)
    imgs = [torch.tensor(host[i], device="cuda") for i in mine]
    batch = ShearletBatch(imgs, [cbs[i] for i in mine], [lams[i] for i in mine], 1.0)
    if tune:
        batch.tune(5)
    for _ in range(warmup_steps):
        batch.step(warmup_iters)
    batch.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(batch.stream)
    for _ in range(steps):
        batch.step(iters)
    ev1.record(batch.stream)
    ev1.synchronize()
    t = torch.tensor([ev0.elapsed_time(ev1)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    plans = [batch.image(j).plan() for j in range(len(mine))]
    lanes = batch.lanes
    batch.close()
    value = units * steps / (ms / 1000.0) / 1e6
    out = {"value": value, "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
           "warmup": warmup_steps, "tuned": tune, "n_ranks": world, "images_per_rank_max": max(
               len(shard.share(shapes, r, world)) for r in range(world)),
           "workload": f"batch: {len(shapes)} images, sides 128..1024 (first 384x640), K 2..6, "
                       f"J = floor(log2(min side)/2), {iters} iterations per step, one graph per iteration "
                       f"with the images in concurrent lanes (tuned; 0 = one per image); {world} rank(s), images "
                       f"sharded whole by LPT on H W K eta "
                       f"(strong scaling of the fixed batch); sequential_value: the same images one after "
                       f"another through the single-image path with the batch's plans"}
    out["sms"] = sorted({p.get("sms", 0) for p in plans if p.get("fast")})
    out["lanes"] = lanes
    if world == 1:
        seq = measure_sequential(shapes, imgs, [cbs[i] for i in mine], [lams[i] for i in mine], plans)
        out["sequential_value"] = seq
        out["speedup_vs_sequential"] = value / seq
    return out


def measure_sequential(shapes, imgs, cbs, lams, plans, iters: int = 20, warmup: int = 3):
    """The batch's images solved one after another through the plain
    single-image path (own filter bank and state, the plan the batch tuned
    for the image's shape, with its grids on all SMs: a share of them pays only
    when images run side by side), `iters` graph-replayed iterations each after
    `warmup`; the summed Mpixel*label*iter/s over the summed per-image times."""
    import torch

    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    total_ms, units = 0.0, 0
    for i, (H, W, K, J) in enumerate(shapes):
        fb = FilterBank(H, W, J)
        seg = ShearletSegmenter(fb, imgs[i], cbs[i], lams[i].tolist(), 1.0)
        seg.set_plan(dict(plans[i], sms=0))
        seg.step(warmup)
        seg.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(seg.stream)
        seg.step(iters)
        b.record(seg.stream)
        b.synchronize()
        total_ms += a.elapsed_time(b)
        units += H * W * K * iters
        seg.close()
        fb.close()
    return units / (total_ms / 1000.0) / 1e6


def measure_differentiable(steps: int, warmup: int, n_images: int = 16):
    """The differentiable workload: n_images seeded 256 x 256 images (K = 4,
    J = 3), each T = 50 unrolled ADMM iterations from the zero state with
    checkpoints every 10, then the reverse sweep for a fixed cotangent of w
    (gradients w.r.t. codebook, Lambda and the image).  Units per image and
    pass: H*W*K*T, one forward + reverse pass counted once."""
    import torch

    from paper_1112_1805_gb300 import binding as B
    from paper_1112_1805_gb300.api import FilterBank, ShearletSegmenter

    wl = synth.WORKLOADS["unrolled256"]
    T, ck = wl.iters, 10
    fb = FilterBank(wl.H, wl.W, wl.J)
    segs, cots = [], []
    gen = torch.Generator(device="cuda").manual_seed(synth.seed_for(wl.index))
    for i in range(n_images):
        img, _, _ = synth.make_workload_image("unrolled256", i)
        segs.append(ShearletSegmenter(fb, torch.tensor(img.astype(np.float32), device="cuda"), wl.codebook(),
                                      wl.Lambda(), wl.gamma))
        cots.append(1e-3 * torch.randn((wl.K, wl.H, wl.W), device="cuda", generator=gen))
    torch.cuda.synchronize()
    # one tuning run on the first image; the same-shaped others take its plan
    plan = segs[0].tune(10)
    for sg in segs[1:]:
        sg.set_plan(plan)

    fbars = [torch.empty((1, wl.H, wl.W), device="cuda") for _ in segs]

    def one_pass():
        # every image's forward and reverse sweep is queued on its own stream,
        # then the gradients are read back
        for sg, c in zip(segs, cots):
            B.seg_admm_unrolled_fwd(sg.handle, T, ck)
            B.seg_admm_unrolled_bwd_enqueue(sg.handle, c.data_ptr())
        for sg, fb_ in zip(segs, fbars):
            B.seg_admm_unrolled_grads(sg.handle, wl.K, 1, wl.J, fb_.data_ptr())

    for _ in range(warmup):
        one_pass()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one_pass()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    # the plain iteration on the same images for comparison, T iterations per
    # image: all images queued at once on their own streams (forward only), and
    # one image after another through the single-image path (like for like
    # with the plain line: one solve at a time)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(segs[0].stream)
    for sg in segs:
        B.seg_admm_step(sg.handle, T)
    for sg in segs:
        sg.synchronize()
    e1.record(segs[0].stream)
    torch.cuda.synchronize()
    plain_ms = e0.elapsed_time(e1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sg in segs:
        B.seg_admm_step(sg.handle, T)
        sg.synchronize()
    seq_s = time.perf_counter() - t0
    units = n_images * wl.H * wl.W * wl.K * T
    for sg in segs:
        sg.close()
    fb.close()
    return {"value": units / dt / 1e6, "unit": UNIT, "ms_per_step": dt * 1000.0, "steps": steps, "warmup": warmup,
            "forward_only_value": units / (plain_ms / 1000.0) / 1e6,
            "plain_sequential_value": units / seq_s / 1e6,
            "vs_plain_sequential": (units / dt) / (units / seq_s),
            "plan": {k: plan[k] for k in ("wave_mib", "col_ctas_per_sm")},
            "workload": f"{n_images} x 256x256 gray, K=4, J=3 (eta=29), {T} unrolled ADMM iterations from zero with "
                        f"checkpoints every {ck}, reverse sweep for a fixed cotangent of w (gradients w.r.t. "
                        f"codebook, Lambda, image); one forward+reverse pass counted as {T} iterations"}


def run_differentiable(args):
    """The differentiable workload as the bench line itself (--workload differentiable)."""
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    d = measure_differentiable(args.steps, args.warmup, args.images)
    line = {"metric": METRIC, "value": d["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": d["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": d["workload"], "images": args.images},
            "forward_only_value": d["forward_only_value"]}
    print(json.dumps(line))
    return 0


def run_batch(args):
    """The batch as the bench line itself (--workload batch)."""
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    iters = args.iters or 300
    b = measure_batch(iters, args.steps, args.warmup, iters, not args.no_tune)
    line = {"metric": METRIC, "value": b["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": b["workload"], "images": 64, "iters_per_step": iters, "tuned": b["tuned"]},
            "sequential_value": b.get("sequential_value"), "speedup_vs_sequential": b.get("speedup_vs_sequential"),
            "sms": b.get("sms"), "lanes": b.get("lanes")}
    print(json.dumps(line))
    return 0


def run_comparison_model(args):
    """The TV or NL-means leg as the bench line itself (--workload tv512 / nl512)."""
    import torch

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    iters = args.iters or 100
    d = measure_tv(iters, args.steps, args.warmup) if args.workload == "tv512" else \
        measure_nl(iters, args.steps, args.warmup)
    line = {"metric": METRIC, "value": d["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": d["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": d["workload"], "iters_per_step": iters}, "roofline": d["roofline"],
            "kernel_ms": d["kernel_ms"], "label_error": d["label_error"]}
    print(json.dumps(line))
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("tv512", "nl512"):
        return run_comparison_model(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "differentiable":
        return run_differentiable(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
