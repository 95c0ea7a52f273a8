#!/usr/bin/env python
"""Throughput of one differentiable-rendering step on B300.

A step is the whole hot path once over a 512x512 image of the DeepSDF-shaped
decoder (8 hidden layers of 512, latent 256, skip at layer 4): ray generation
with unit-sphere initialisation, up to 50 march iterations (active-ray
compaction, decoder queries, converge/step), depth / silhouette / mask, the
L1 depth loss against a depth map rendered from a second seeded latent, and
the latent gradient (exact implicit adjoint, FP64 reductions).  Normals are
rendered only with --normals (the L1 depth loss does not use them).

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle on a
bounded crop of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

FLOP_PER_QUERY = 3_146_752          # 8x512 decoder, latent folded into per-shape biases
EPS_MID = 2e-4                      # FP16 stage of the BF16 march (hand-over to FP32-class)
# dram__bytes_read.sum + dram__bytes_write.sum of one mlp_tc_kernel launch (ncu, the
# first march launch of a 256x256 trace: 65,536 rows); the weights dominate it, so it
# is not scaled by rows.  Taken on the current kernel; None once the kernel changes.
TC_TRAFFIC_BYTES = 6317056 + 5888
TC_TRAFFIC_NOTE = ("ncu dram read+write, first march launch of a 256x256 BF16 trace "
                   "(65,536 rows; weights once + ray state read and written by the step "
                   "warps), not scaled")
SIZE = 512
MAX_STEPS = 50
WORKLOAD = ("DeepSDF-shaped decoder 8x512 (latent 256, skip@4, ReLU, tanh), geometric init "
            "r=0.6 + seeded perturbation, z ~ N(0, 0.01^2); 512x512 forward+backward, "
            "L1 depth loss vs a depth map of a second seeded latent, 50 steps, eps 5e-5, "
            "alpha 1.5, exact implicit latent gradient")


def max_over_ranks(values, device):
    """Element-wise maximum of `values` over all ranks of the default process
    group (the slowest rank's time is the job's time)."""
    import torch
    t = torch.tensor([float(v) for v in values], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_rate(units_per_rank_step, world, steps, max_total_ms):
    """Whole-job throughput: the units every rank processed over `steps`,
    divided by the slowest rank's time."""
    return units_per_rank_step * world * steps / (max_total_ms * 1e-3)


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
            "sm_max_mhz": 2032.0}, "fallback"


def make_workload(spec):
    import synth
    Ws, bs = synth.make_decoder(spec, seed=0)
    Z = synth.make_latents(spec, 2, seed=0)
    vp = synth.random_viewpoints(5, seed=0)[0]
    cam = synth.look_at_camera(vp, SIZE, SIZE, shape=0)
    return Ws, bs, Z, cam


# ----------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"dist_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- our arm

class Step:
    """Preallocated buffers and C structs for one fwd+bwd step through the C ABI."""

    def __init__(self, api, dec, ws, cam, params, z, tgt_depth, normals=False):
        import torch
        from ctypes import byref, c_void_p
        from paper_1911_13225_b300 import _abi
        self.api, self.dec, self.ws, self.params = api, dec, ws, params
        self.torch = torch
        self.z = z
        self.tgt = tgt_depth
        n = SIZE * SIZE
        self.res = api.alloc_result(n, params.k_min, z.device, normals=normals)
        dev = z.device
        self.g_depth = torch.empty(n, device=dev)
        self.dz = torch.zeros_like(z)
        self.loss = torch.zeros(1, device=dev, dtype=torch.float64)
        self.cam_c = api.camera_array([cam])
        self.p_c = params.c()
        self.o_c = self.res.c()
        self.w_c = _abi.LossWeights(1.0, 0.0, 0.0, 0.0)
        self.lib = _abi.lib()
        self.byref, self.vp, self.check = byref, c_void_p, _abi.check

    def __call__(self, stream):
        P = lambda t: self.vp(t.data_ptr())
        L, b, s = self.lib, self.byref, self.vp(stream.cuda_stream)
        n = SIZE * SIZE
        self.check(L.dist_trace_fwd(self.dec.handle, P(self.z), 2, self.cam_c, 1, b(self.p_c),
                                    b(self.o_c), self.ws.handle, s), "dist_trace_fwd")
        self.check(L.dist_loss(n, P(self.res.depth), P(self.res.mask), P(self.res.sil), None,
                               P(self.tgt), None, None, P(self.z), 2, self.z.shape[1], b(self.w_c),
                               P(self.loss), P(self.g_depth), None, None, P(self.dz),
                               self.ws.handle, s), "dist_loss")
        self.check(L.dist_trace_bwd(self.dec.handle, P(self.z), 2, self.cam_c, 1, b(self.p_c),
                                    b(self.o_c), P(self.g_depth), None, None, P(self.dz),
                                    self.ws.handle, s), "dist_trace_bwd")


def run_ours(args, rank, world, local_rank):
    import torch
    import synth
    from paper_1911_13225_b300 import api, _abi
    from ctypes import byref, c_double, c_int64

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z, cam = make_workload(spec)
    dec = api.Decoder.from_spec(spec, Ws, bs)
    precision = args.precision
    if precision == "auto":
        precision = "bf16" if dec.has_bf16 else "fp32"
    params = api.TraceParams(max_steps=MAX_STEPS, precision=precision, eps_bf16=args.eps_lo,
                             refine_steps=args.refine, alpha_refine=args.alpha_refine,
                             refine_engine=args.refine_engine, refine_rule=args.refine_rule,
                             coarse_levels=args.coarse_levels,
                             latency_mode=args.latency_mode,
                             eps_mid=args.eps_mid if precision == "bf16" else 0.0)
    ws = api.Workspace(SIZE * SIZE, MAX_STEPS)
    z = torch.from_numpy(Z).to(dev)
    # target: depth of the second latent (untimed setup)
    tgt = api.trace(dec, z, [dict(cam, shape=1)], params, ws).depth.clone()
    stream = torch.cuda.current_stream()
    step = Step(api, dec, ws, cam, params, z, tgt, normals=args.normals)
    flush = torch.empty(256 * 1024 * 1024 // 4, device=dev)

    for _ in range(args.warmup):
        step(stream)
    torch.cuda.synchronize()

    # device-timed region: inputs resident, L2 flushed between steps (untimed)
    L = _abi.lib()
    step.res.queries.zero_()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    gpu_index = local_rank
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        gpu_index = vis.split(",")[local_rank]
    clocks = ClockSampler(gpu_index)
    clocks.start()

    def timed_steps(profiled):
        # K steps, L2 flushed before each (outside its events); profiled:
        # the library also records CUDA events around every decoder and
        # adjoint launch (per-kernel times for the roofline and breakdown)
        L.dist_profile_enable(1 if profiled else 0)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            step(stream)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        L.dist_profile_enable(0)
        return float(sum(a.elapsed_time(b) for a, b in evs))

    total_ms = timed_steps(False)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    queries = step.res.queries.cpu().numpy().astype(np.int64)
    # the same K steps again with per-launch events: events between the
    # decoder launches stop programmatic dependent launch from overlapping a
    # launch's prologue with its predecessor, so they are kept out of the
    # pass that gives `value`
    prof_total_ms = timed_steps(True)
    ms_arr = (c_double * 3)()
    cnt_arr = (c_int64 * 3)()
    all_launches = c_int64()
    _abi.check(L.dist_profile_read(ms_arr, cnt_arr, byref(all_launches)), "dist_profile_read")
    hits = int(step.res.mask.sum().item())
    accuracy = accuracy_vs_oracle(step.res, precision)

    # end to end through the C ABI: pinned host inputs in, loss and dz out
    z_host = torch.from_numpy(Z).pin_memory()
    tgt_host = tgt.cpu().pin_memory()
    loss_host = torch.zeros(1, dtype=torch.float64).pin_memory()
    dz_host = torch.zeros_like(z_host).pin_memory()
    e2e_steps = max(3, args.steps // 2)
    e2e_total = 0.0
    for _ in range(e2e_steps):
        # L2 flushed before every step as in the device-timed loop, outside
        # the timed region (each step is timed on the host from here)
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step.z.copy_(z_host, non_blocking=True)
        step.tgt.copy_(tgt_host, non_blocking=True)
        step(stream)
        loss_host.copy_(step.loss, non_blocking=True)
        dz_host.copy_(step.dz, non_blocking=True)
        stream.synchronize()
        e2e_total += time.perf_counter() - t0
    e2e_s = e2e_total / e2e_steps

    if world > 1:
        total_ms, e2e_s = max_over_ranks([total_ms, e2e_s], dev)
    if rank != 0:
        return None

    ms_per_step = total_ms / args.steps
    rays = SIZE * SIZE
    value = job_rate(rays, world, args.steps, total_ms)
    peaks, peak_src = load_peaks()
    if precision in ("bf16", "fp16"):
        k_ms, k_q, k_n = ms_arr[0], queries[0], cnt_arr[0]
        fused = args.refine_engine == "tc" and args.refine == 0
        if fused:
            # one launch per step decodes the 16-bit rows and the FP32-class
            # rows (4 tensor FLOP per algorithmic FLOP for the latter)
            k_q = queries[0] + queries[1]
        achieved = k_q * FLOP_PER_QUERY / (k_ms * 1e-3) / 1e12 if k_ms > 0 else 0.0
        peak = peaks["bf16_tflops"]
        roof = {"bound": "tensor",
                "kernel": f"mlp_tc_kernel ({precision.upper()} tcgen05 decoder"
                          + (" + FP16-stage rows" if fused and params.eps_mid > 0 else "")
                          + (" + FP32-class rows in the same launch" if fused else "")
                          + "; fp16 and bf16 share the dense tensor rate)"
                          + (" with mlp_tc_wide_kernel on the march's small steps"
                             " (latency mode); achieved = per-step average over both"
                             if fused and args.latency_mode else ""),
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_source": f"{peak_src} bf16 burst",
                "traffic": TC_TRAFFIC_BYTES,
                "traffic_note": TC_TRAFFIC_NOTE}
        if fused:
            tq = queries[0] + 4 * queries[1]
            roof["tensor_tflops_executed"] = tq * FLOP_PER_QUERY / (k_ms * 1e-3) / 1e12 \
                if k_ms > 0 else 0.0
    elif precision == "fp32_tc":
        # the fused march decodes the FP32-class list in mlp_tc_kernel (and
        # the latency-mode kernel); a deferred list would count as kind 1
        k_ms, k_q, k_n = ms_arr[0] + ms_arr[1], queries[1], cnt_arr[0] + cnt_arr[1]
        achieved = k_q * FLOP_PER_QUERY / (k_ms * 1e-3) / 1e12 if k_ms > 0 else 0.0
        peak = peaks["bf16_tflops"]
        roof = {"bound": "tensor",
                "kernel": "mlp_tc_kernel, FP32-class rows only (two-term FP16 split, "
                          "4 tensor FLOP per algorithmic FLOP, so frac <= 0.25)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "peak_source": f"{peak_src} bf16 burst",
                "traffic": None}
    else:
        k_ms, k_q, k_n = ms_arr[1], queries[1], cnt_arr[1]
        achieved = k_q * FLOP_PER_QUERY / (k_ms * 1e-3) / 1e12 if k_ms > 0 else 0.0
        # FP32 FMA peak: 148 SMs x 128 lanes x 2 FLOP x max SM clock
        peak = 148 * 128 * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": "mlp_fp32_fwd_kernel (FP32 SIMT decoder)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "peak_source": "derived: 148 SM x 128 FP32 FMA/clk x 2 x max SM clock",
                "traffic": None}
    roof["mlp_ms_per_step"] = k_ms / args.steps
    roof["mlp_launches_per_step"] = k_n / args.steps
    roof["queries_per_step"] = float(k_q) / args.steps
    roof["timing"] = ("per-launch CUDA events on the launching stream over a second pass of "
                      "the same K steps (profiled_ms_per_step), kept out of the pass that "
                      "gives value")
    breakdown = {"march_tc_ms": ms_arr[0] / args.steps,
                 "march_fp32_list_ms": ms_arr[1] / args.steps,
                 "adjoint_ms": ms_arr[2] / args.steps,
                 "other_ms": prof_total_ms / args.steps
                 - (ms_arr[0] + ms_arr[1] + ms_arr[2]) / args.steps,
                 "profiled_ms_per_step": prof_total_ms / args.steps}
    bi = z_host.numel() * 4 + tgt_host.numel() * 4
    bo = 8 + dz_host.numel() * 4
    line = {
        "metric": "rays/s (pixels traced per second, forward+backward)",
        "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"bf16": "bf16", "fp16": "f16", "fp32": "f32", "fp32_tc": "f16x2"}[precision],
        "data": "synthetic (seeded decoder, latents and camera; no DeepSDF weights)",
        "config": {"workload": WORKLOAD.replace("512x512", f"{SIZE}x{SIZE}"),
                   "rays_per_step": rays, "precision": precision,
                   "eps_lo": args.eps_lo, "eps_mid": args.eps_mid if precision == "bf16" else 0.0,
                   "refine_steps": args.refine,
                   "refine_engine": args.refine_engine, "refine_rule": args.refine_rule,
                   "coarse_levels": args.coarse_levels, "latency_mode": args.latency_mode,
                   "normals": "rendered (analytic, adjoint at the hits)" if args.normals
                              else "not rendered (unused by the L1 depth loss)",
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed between timed steps (256 MB write, untimed)"},
        "sdf_queries_per_s": float(queries.sum()) * world / (total_ms * 1e-3),
        # the same queries over the decoder launches' own time (forward march only)
        "march_sdf_queries_per_s": (float(queries.sum()) / args.steps * world /
                                    ((breakdown["march_tc_ms"] + breakdown["march_fp32_list_ms"])
                                     * 1e-3)) if (breakdown["march_tc_ms"] +
                                                  breakdown["march_fp32_list_ms"]) > 0 else None,
        "queries_per_step": {"lowp": float(queries[0]) / args.steps,
                             "fp32": float(queries[1]) / args.steps},
        "hits": hits,
        "accuracy_vs_oracle": accuracy,
        "fp32_class_queries": ({"tc": "tensor cores, every operand a sum of two FP16 numbers "
                                      "(FP32-class; the accumulator truncates: f within 5e-6 "
                                      "of FP64)",
                                "simt": "FP32 CUDA cores"}[args.refine_engine]
                               if precision in ("bf16", "fp16") else None),
        "e2e": {"value": rays * world / e2e_s, "unit": "rays/s", "h2d_bytes_per_step": bi,
                "d2h_bytes_per_step": bo,
                "note": "host-timed per step (pinned copies in, loss and dz out, stream "
                        "synchronised); L2 flushed before each step outside the timed region, "
                        "as for value"},
        "gpu_launches": int(all_launches.value),
        "gpu_launches_note": "library kernel launches in K steps (counted on the profiled pass, "
                             "which runs the same K steps)",
        "step_breakdown_ms": breakdown,
        "roofline": roof,
        "clocks": clk,
    }
    line["fp32_trace"] = fp32_trace_rate(api, dec, cam, z, tgt, stream)
    # (coarse-to-fine needs the fused tensor-core march: refine_steps 0, TC engine)
    if args.coarse_levels == 0 and precision in ("bf16", "fp16") and args.refine == 0 \
            and args.refine_engine == "tc":
        line["coarse_to_fine"] = coarse_to_fine_rate(api, dec, ws, cam, params, z, tgt, stream,
                                                     flush, args.steps, args.normals)
        if precision == "bf16" and args.refine == 0:
            line["fp16"] = fp16_rate(api, dec, ws, cam, params, z, tgt, stream, flush,
                                     args.steps, args.normals)
            if params.eps_mid > 0:
                line["bf16_without_fp16_stage"] = two_stage_rate(api, dec, ws, cam, params, z, tgt,
                                                                 stream, flush, args.steps,
                                                                 args.normals)
    line["roofline"]["large_launch"] = large_launch_rate(api, dec, z, precision, peaks["bf16_tflops"])
    if not args.no_side_configs and SIZE == 512:
        line["small_32x32"] = small_rate(dev, stream)
        line["five_views_256"] = five_views_rate(api, dec, z, stream, flush)
        line["inverse_32x8_224"] = inverse_rate(api, dec, spec, dev, args.inverse_steps)
    if not args.no_serve:
        line["serving"] = run_serving(args, dec, params, dev)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_crop)
    return line


# ------------------------------------------------- accuracy against the oracle

GOLDEN = os.path.join(ROOT, "tests", "golden", "full_masks.npz")


def accuracy_vs_oracle(res, precision):
    """The benchmark view's hit mask and depth against the FP64 oracle's,
    stored by tests/golden/make_full_masks.py (an oracle-only script): mask
    mismatches in all and outside the excluded rays (16-bit march: silhouette
    rays at the 1e-3 |SDF| margin; FP32: threshold-ambiguous rays), and the
    depth error on the hits both share outside them."""
    if SIZE != 512 or not os.path.exists(GOLDEN):
        return None
    with np.load(GOLDEN) as g:
        n = int(g["b512/n"])
        gm = np.unpackbits(g["b512/mask"])[:n].astype(bool)
        ex = np.unpackbits(g["b512/sil" if precision != "fp32" else "b512/amb32"])[:n].astype(bool)
        if "b512/depth_hits" not in g.files:
            return None
        gd = np.full(n, np.inf)
        gd[gm] = g["b512/depth_hits"].astype(np.float64)
    m = res.mask.cpu().numpy().astype(bool)
    d = res.depth.cpu().numpy().astype(np.float64)
    both = m & gm & ~ex
    err = np.abs(d[both] - gd[both])
    return {"mask_mismatches": int((m != gm).sum()),
            "mask_mismatches_outside_excluded": int(((m != gm) & ~ex).sum()),
            "excluded": "silhouette rays at the 1e-3 |SDF| margin" if precision != "fp32"
                        else "threshold-ambiguous rays (FP32 vs FP64 branch)",
            "excluded_frac": float(ex.mean()),
            "depth_err_q50": float(np.quantile(err, 0.5)), "depth_err_q99": float(np.quantile(err, 0.99)),
            "depth_err_max": float(err.max()), "hits_compared": int(both.sum()),
            "reference": "FP64 oracle, stored by tests/golden/make_full_masks.py"}


# ------------------------------------------------- FP32 trace, large launches

def variant_rate(api, dec, ws, cam, p2, z, tgt, stream, flush, steps, normals):
    """The same fwd+bwd step with trace parameters p2, timed like the main
    line: (ms per step, queries per step, hits)."""
    import torch
    step = Step(api, dec, ws, cam, p2, z, tgt, normals=normals)
    for _ in range(3):
        step(stream)
    torch.cuda.synchronize()
    step.res.queries.zero_()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        evs[i][0].record(stream)
        step(stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    q = step.res.queries.cpu().numpy().astype(np.float64) / steps
    return ms, q, int(step.res.mask.sum().item()), accuracy_vs_oracle(step.res, p2.precision)


def coarse_to_fine_rate(api, dec, ws, cam, params, z, tgt, stream, flush, steps, normals):
    """The same fwd+bwd step with the paper's coarse-to-fine tracing (Sec. 3.2:
    start at 1/4 resolution per side, split every ray into four after every
    three iterations), timed like the main line."""
    import dataclasses
    # (coarse-to-fine runs the two-stage march: no FP16 stage)
    p2 = dataclasses.replace(params, coarse_levels=2, coarse_every=3, eps_mid=0.0)
    ms, q, hits, _ = variant_rate(api, dec, ws, cam, p2, z, tgt, stream, flush, steps, normals)
    return {"value": SIZE * SIZE / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms,
            "coarse_levels": 2, "coarse_every": 3,
            "queries_per_step": {"lowp": float(q[0]), "fp32": float(q[1])},
            "hits": hits,
            "note": "same step with coarse-to-fine tracing (Sec. 3.2); child rays inherit by "
                    "the stated reading, so depths differ from the exact per-pixel trace near "
                    "silhouettes"}


def fp16_rate(api, dec, ws, cam, params, z, tgt, stream, flush, steps, normals):
    """The same fwd+bwd step with FP16 operands (10 mantissa bits against
    BF16's 7), which resolve |f| well enough to hand over to the FP32-class
    queries at |f| < 2e-4 instead of 1e-3."""
    import dataclasses
    p2 = dataclasses.replace(params, precision="fp16", eps_bf16=2e-4, refine_steps=0,
                             coarse_levels=0)
    ms, q, hits, acc = variant_rate(api, dec, ws, cam, p2, z, tgt, stream, flush, steps, normals)
    return {"value": SIZE * SIZE / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms,
            "dtype": "fp16", "eps_lo": 2e-4, "refine_steps": 0,
            "queries_per_step": {"lowp": float(q[0]), "fp32": float(q[1])},
            "hits": hits, "accuracy_vs_oracle": acc,
            "note": "FP16 GEMM operands (same tensor rate as BF16), FP32-class convergence after "
                    "the hand-over; on this view depth vs the FP32 trace q99 7.8e-5 (BF16 "
                    "default: 1.2e-4)"}


def two_stage_rate(api, dec, ws, cam, params, z, tgt, stream, flush, steps, normals):
    """The same fwd+bwd step with the BF16 march handing over straight to the
    FP32-class queries (no FP16 stage), timed like the main line."""
    import dataclasses
    p2 = dataclasses.replace(params, eps_mid=0.0)
    ms, q, hits, acc = variant_rate(api, dec, ws, cam, p2, z, tgt, stream, flush, steps, normals)
    return {"value": SIZE * SIZE / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms,
            "eps_mid": 0.0, "queries_per_step": {"lowp": float(q[0]), "fp32": float(q[1])},
            "hits": hits, "accuracy_vs_oracle": acc,
            "note": "BF16 march, FP32-class queries from |f| < eps_lo on (the FP16 stage off)"}


def fp32_trace_rate(api, dec, cam, z, tgt, stream, steps=3):
    """The plain FP32 GPU trace (CUDA-core decoder, FP32 adjoint) on the same
    workload and step, timed the same way (after one warm-up step)."""
    import torch
    p32 = api.TraceParams(max_steps=MAX_STEPS, precision="fp32")
    ws = api.Workspace(SIZE * SIZE, MAX_STEPS)
    step = Step(api, dec, ws, cam, p32, z, tgt)
    step(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": SIZE * SIZE / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms,
            "steps": steps, "note": "precision fp32: mlp_fp32_fwd_kernel + FP32 adjoint",
            "accuracy_vs_oracle": accuracy_vs_oracle(step.res, "fp32")}


def large_launch_rate(api, dec, z, precision, peak, n=262144 * 2, reps=5):
    """The decoder kernel alone on one large launch (dist_sdf_eval, n random
    points in the unit ball region): the rate the march's first steps run at."""
    import torch
    if precision not in ("bf16", "fp16", "fp32_tc"):
        return None
    dev = z.device
    g = torch.Generator(device="cpu").manual_seed(7)
    pts = (torch.rand(n, 3, generator=g) * 1.4 - 0.7).to(dev)
    sh = torch.zeros(n, dtype=torch.int32, device=dev)
    ws = api.Workspace(n)
    for _ in range(2):
        api.sdf_eval(dec, z, pts, sh, ws, precision=precision)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        api.sdf_eval(dec, z, pts, sh, ws, precision=precision)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    tf = n * FLOP_PER_QUERY / (ms * 1e-3) / 1e12
    return {"rows": n, "ms": ms, "achieved": tf, "peak": peak, "frac": tf / peak,
            "note": "dist_sdf_eval of one launch (fold + pack + decoder), algorithmic FLOPs"}


# ------------------------------------------ the other configurations' lines

def small_rate(dev, stream, steps=20):
    """The small configuration: a 4 x 128 decoder (latent 64, no skip),
    32 x 32 image from (0, 0, 2.5), FP32 forward trace (depth, normals, mask),
    50 steps -- latency-bound: a few tiles per step."""
    import torch
    import synth
    from paper_1911_13225_b300 import api
    spec = synth.SMALL_SPEC
    Ws, bs = synth.make_decoder(spec, seed=0)
    Z = synth.make_latents(spec, 1, seed=0)
    dec = api.Decoder.from_spec(spec, Ws, bs)
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 32, 32)
    ws = api.Workspace(32 * 32, MAX_STEPS)
    z = torch.from_numpy(Z).to(dev)
    p = api.TraceParams(max_steps=MAX_STEPS)
    res = api.alloc_result(32 * 32, 1, dev, normals=True)
    cam_c = api.camera_array([cam])
    for _ in range(3):
        api.trace(dec, z, [cam], p, ws, normals=True, out=res, cam_c=cam_c, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        api.trace(dec, z, [cam], p, ws, normals=True, out=res, cam_c=cam_c, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": 32 * 32 / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms,
            "hits": int(res.mask.sum().item()),
            "note": "4x128 decoder, latent 64, 32x32 from (0, 0, 2.5), FP32 forward with analytic "
                    "normals, 50 steps; back-to-back traces (inputs L2-resident)"}


def five_views_rate(api, dec, z, stream, flush, steps=5):
    """Forward trace of 5 seeded viewpoints (radius 2.5) at 256x256 in one
    call (327,680 rays), latent 0 of the benchmark's, 50 steps: BF16 tcgen05
    march with the FP16 stage and FP32-class convergence against the plain
    FP32 trace, both device-timed with L2 flushed between steps."""
    import torch
    import synth
    cams = [synth.look_at_camera(vp, 256, 256) for vp in synth.random_viewpoints(5, seed=0)]
    n = api.n_pixels(cams)
    ws = api.Workspace(n, MAX_STEPS)
    cam_c = api.camera_array(cams)
    out = {"rays_per_step": n, "note": "5 views x 256x256 in one dist_trace_fwd call, forward "
           "only (depth, silhouette, mask), 50 steps, eps 5e-5, alpha 1.5"}
    for prec in ("bf16", "fp32"):
        p = api.TraceParams(max_steps=MAX_STEPS, precision=prec,
                            eps_mid=EPS_MID if prec == "bf16" else 0.0)
        res = api.alloc_result(n, 1, z.device, normals=False)
        for _ in range(2):
            api.trace(dec, z, cams, p, ws, out=res, cam_c=cam_c, stream=stream)
        torch.cuda.synchronize()
        res.queries.zero_()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for i in range(steps):
            flush.zero_()
            evs[i][0].record(stream)
            api.trace(dec, z, cams, p, ws, out=res, cam_c=cam_c, stream=stream)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in evs) / steps
        q = res.queries.cpu().numpy().astype(np.float64) / steps
        out[prec] = {"value": n / (ms * 1e-3), "unit": "rays/s", "ms_per_step": ms,
                     "queries_per_step": {"lowp": float(q[0]), "fp32": float(q[1])},
                     "hits": int(res.mask.sum().item())}
    out["bf16_over_fp32"] = out["bf16"]["value"] / out["fp32"]["value"]
    return out


def inverse_rate(api, dec, spec, dev, steps=3):
    """The inverse-optimisation batch: 32 shapes (seeded target latents) x 8
    ring views (elevation 20 deg, radius 2.5) at 224x224 = 12,845,056 rays,
    all in one call per library entry point.  One Adam step = trace (BF16
    march with the FP16 stage, central-difference normals, delta 1e-3) + depth
    and normal losses
    (weights 10 and 1) + latent gradient + Adam (lr 1e-2, z0 = 0), device-timed
    after one warm-up step (the ray state alone is 411 MB, far above L2)."""
    import torch
    import synth
    from paper_1911_13225_b300.inverse import InverseProblem
    ring = synth.ring_viewpoints(8)
    cams = [synth.look_at_camera(ring[v], 224, 224, shape=s) for s in range(32) for v in range(8)]
    n = api.n_pixels(cams)
    params = api.TraceParams(max_steps=MAX_STEPS, precision="bf16", normal_delta=1e-3,
                             eps_mid=EPS_MID)
    ws = api.Workspace(n, MAX_STEPS)
    z_true = torch.from_numpy(synth.make_latents(spec, 32, seed=3)).to(dev)
    tgt = api.trace(dec, z_true, cams, params, ws, normals=True)
    prob = InverseProblem(dec, cams, 32, tgt.depth.clone(), tgt.normal.clone(), params=params,
                          ws=ws, lr=1e-2, w_depth=10.0, w_normal=1.0)
    del tgt
    stream = torch.cuda.current_stream()
    loss0 = float(prob.step(stream))
    torch.cuda.synchronize()
    prob.res.queries.zero_()
    from ctypes import byref, c_double, c_int64
    from paper_1911_13225_b300 import _abi
    L = _abi.lib()
    L.dist_profile_enable(1)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    for i in range(steps):
        evs[i][0].record(stream)
        prob.step(stream)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    L.dist_profile_enable(0)
    ms_arr, cnt_arr, all_l = (c_double * 3)(), (c_int64 * 3)(), c_int64()
    _abi.check(L.dist_profile_read(ms_arr, cnt_arr, byref(all_l)), "dist_profile_read")
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    q = prob.res.queries.cpu().numpy().astype(np.float64) / steps
    assert dec.device_error() == 0
    brk = {"march_decoder_s": (ms_arr[0] + ms_arr[1]) / steps * 1e-3,
           "adjoint_s": ms_arr[2] / steps * 1e-3,
           "rest_s": ms * 1e-3 - (ms_arr[0] + ms_arr[1] + ms_arr[2]) / steps * 1e-3,
           "note": "adjoint: the BF16 depth adjoint plus the FP32-class tensor-core "
                   "adjoint of the six central-difference probes per hit (the normal "
                   "term's latent gradient subtracts Jacobians 2e-3 apart, so it needs "
                   "FP32-class operands); rest: mostly the FP32-class queries of those "
                   "probes (normals and their coefficients)"}
    return {"value": n / (ms * 1e-3), "unit": "rays/s", "s_per_adam_step": ms * 1e-3,
            "rays_per_step": n, "steps": steps,
            "march_queries_per_step": {"lowp": float(q[0]), "fp32": float(q[1])},
            "loss_step1": loss0, "loss_last": float(prob.loss.item()),
            "breakdown": brk,
            "note": "32 shapes x 8 views x 224x224 per Adam step, one call per entry point "
                    "(dist_trace_fwd with central-difference normals, dist_loss, "
                    "dist_trace_bwd, dist_adam_step); the paper's Tab. 1 unit is the time "
                    "of one such optimisation step"}


# ----------------------------------------------------------------- serving

SERVE_SIZES = (64, 128, 256, 512)


def serve_requests(n, seed=777):
    """Seeded mixed load: 70% render, 30% render+backward, square images with
    sides uniform over SERVE_SIZES, a N(0, 0.01^2) 256-d latent per request,
    viewpoints uniform on the radius-2.5 sphere."""
    import synth
    rng = np.random.default_rng(seed)
    vps = synth.random_viewpoints(n, seed=seed)
    out = []
    for i in range(n):
        side = int(rng.choice(SERVE_SIZES))
        kind = "backward" if rng.random() < 0.3 else "render"
        z = rng.normal(0.0, 0.01, 256).astype(np.float32)
        z_tgt = rng.normal(0.0, 0.01, 256).astype(np.float32)
        out.append((synth.look_at_camera(vps[i], side, side, shape=0), z, kind, z_tgt))
    return out


def run_serving(args, dec, params, dev):
    """Continuous-batching server under a Poisson stream of the mixed load:
    saturated throughput first (all requests submitted at once), then arrivals
    at `load` x that rate; latency = arrival -> poll-done."""
    import torch
    from paper_1911_13225_b300 import api, _abi
    from paper_1911_13225_b300.serve import Server
    reqs = serve_requests(args.serve_requests)
    ws = api.Workspace(512 * 512, MAX_STEPS)
    tgts = []
    for cam, z, kind, z_tgt in reqs:      # targets of the backward requests (untimed)
        if kind == "backward":
            zt = torch.from_numpy(z_tgt[None]).to(dev)
            tgts.append(api.trace(dec, zt, [cam], params, ws).depth.cpu().numpy())
        else:
            tgts.append(None)
    srv = Server(dec, params, max_rays=4 * 512 * 512, mem_budget=8 << 30, max_requests=64)

    def submit(i):
        cam, z, kind, _ = reqs[i]
        try:
            return srv.submit(cam, z, kind, tgts[i])
        except _abi.DistError as e:
            if e.status == _abi.DIST_E_BUSY:
                return None
            raise

    def drive(arrivals):
        """Submit request i at time arrivals[i] (from t0); returns latencies."""
        n = len(arrivals)
        pending, live, lat = 0, {}, np.zeros(n)
        t0 = time.perf_counter()
        while pending < n or live:
            now = time.perf_counter() - t0
            while pending < n and arrivals[pending] <= now:
                t = submit(pending)
                if t is None:
                    break
                live[pending] = t
                pending += 1
            for i in list(live):
                if srv.poll(live[i]):
                    lat[i] = (live[i].t_done - t0) - arrivals[i]
                    del live[i]
            time.sleep(5e-5)
        return lat, time.perf_counter() - t0

    rays = np.array([int(c["H"]) * int(c["W"]) for c, _, _, _ in reqs], dtype=np.float64)
    drive(np.zeros(min(16, len(reqs))))                      # warm-up
    _, t_sat = drive(np.zeros(len(reqs)))
    sat_req_s = len(reqs) / t_sat
    # Poisson arrivals at each load (fraction of the saturated request rate)
    loads = sorted(set([float(x) for x in args.serve_loads.split(",") if x] + [args.serve_load]))
    by_load = {}
    for load in loads:
        rng = np.random.default_rng(4242)
        arr = np.cumsum(rng.exponential(1.0 / (load * sat_req_s), len(reqs)))
        arr -= arr[0]
        lat_l, t_l = drive(arr)
        by_load[load] = (lat_l, t_l)
    lat, t_run = by_load[args.serve_load]
    srv.close()

    # the plain per-request FP32 CUDA-core trace (+ backward), one at a time
    p32 = api.TraceParams(max_steps=MAX_STEPS, precision="fp32")
    sample = list(range(min(args.serve_fp32_sample, len(reqs))))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sample:
        cam, z, kind, _ = reqs[i]
        zt = torch.from_numpy(z[None]).to(dev)
        res = api.trace(dec, zt, [cam], p32, ws)
        if kind == "backward":
            tg = {"depth": torch.from_numpy(tgts[i]).to(dev)}
            _, gd, _, _, dz = api.loss(res, tg, zt, ws)
            api.backward(dec, zt, [cam], p32, ws, res, g_depth=gd, dz=dz)
        torch.cuda.synchronize()
    t32 = time.perf_counter() - t0
    return {
        "requests": len(reqs), "mix": "70% render / 30% render+backward (L1 depth), sides "
        "uniform over {64,128,256,512}, seeded 256-d latents, shared 8x512 decoder",
        "admission": "device-memory budget 8 GiB, 64 slots, 4x512^2 pooled rays",
        "saturated_rays_per_s": float(rays.sum() / t_sat),
        "saturated_requests_per_s": sat_req_s,
        "load": args.serve_load,
        "poisson_rays_per_s": float(rays.sum() / t_run),
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "by_load": {f"{load:g}": {"poisson_rays_per_s": float(rays.sum() / t_l),
                                   "p50_ms": float(np.percentile(lat_l, 50) * 1e3),
                                   "p99_ms": float(np.percentile(lat_l, 99) * 1e3)}
                    for load, (lat_l, t_l) in by_load.items()},
        "fp32_per_request_rays_per_s": float(rays[sample].sum() / t32),
        "fp32_sample_requests": len(sample),
    }


# ------------------------------------------------------------ oracle arm

def _crop_camera(cam, crop):
    c = dict(cam)
    x0 = (SIZE - crop) // 2
    c["cx"] = cam["cx"] - x0
    c["cy"] = cam["cy"] - x0
    c["H"] = crop
    c["W"] = crop
    return c


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return max(int(i.get("num_threads", 1)) for i in threadpool_info()) or 1
    except Exception:
        return os.cpu_count() or 1


def oracle_sdf(spec, Ws, bs, Z):
    from oracle.mlp import from_synth
    from oracle.sdf import MLPSDF
    return MLPSDF(from_synth(Ws, bs, spec), Z.astype(np.float64))


def oracle_target(sdf, cam):
    """The L1 target: depth of the second latent (rendered once, untimed)."""
    from oracle import tracer
    return tracer.render(sdf, [dict(cam, shape=1)], max_steps=MAX_STEPS, with_normals=False)["depth"]


def oracle_step(spec, sdf, cam, tgt_depth):
    """The oracle's step on `cam`: forward render, L1 loss, exact latent gradient."""
    from oracle import tracer
    from oracle.grad import latent_vjp
    from oracle.loss import loss_terms
    out = tracer.render(sdf, [cam], max_steps=MAX_STEPS, with_normals=False)
    L, gd, _, _ = loss_terms(out, {"depth": tgt_depth})
    G = latent_vjp(sdf, out, 2, spec.latent_dim, g_depth=gd)
    return L, G


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_crop_rate(spec, sdf, cam, crop):
    c = _crop_camera(cam, crop)
    tgt = oracle_target(sdf, c)
    t0 = time.perf_counter()
    oracle_step(spec, sdf, c, tgt)
    dt = time.perf_counter() - t0
    return crop * crop / dt, dt


def _oracle_one_thread(crop):
    """The oracle's crop rate in a child process whose BLAS runs one thread."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-crop-rate", str(crop)],
                       capture_output=True, text=True, env=env, timeout=600)
    if r.returncode != 0:
        return None, None
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["rate"], d["s"]


def cpu_baseline(crop, crop_1t=32):
    """The FP64 oracle's step on central crops of the benchmark view, on all
    host threads (numpy/BLAS) and on one; the full 512x512 step time is
    extrapolated from the all-thread per-ray rate (the crop is the image's
    centre, where more rays hit and march longer than at the border, so the
    extrapolation overstates the full image's time)."""
    import synth
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z, cam = make_workload(spec)
    sdf = oracle_sdf(spec, Ws, bs, Z)
    rate, dt = _oracle_crop_rate(spec, sdf, cam, crop)
    rate1, dt1 = _oracle_one_thread(crop_1t)
    return {"value": rate, "unit": "rays/s", "cores": _blas_threads(),
            "kind": "oracle", "cpu_model": _cpu_model(), "host_cpus": os.cpu_count(),
            "sample": f"central {crop}x{crop} crop of the 512x512 view (same decoder, latents, "
                      f"camera, target rendered beforehand); forward + L1 loss + exact latent "
                      f"gradient; {dt:.1f} s wall",
            "one_thread": ({"value": rate1, "unit": "rays/s", "cores": 1,
                            "sample": f"central {crop_1t}x{crop_1t} crop, {dt1:.1f} s wall "
                                      f"(BLAS limited to one thread)"}
                           if rate1 is not None else None),
            "extrapolated_512x512_step_s": SIZE * SIZE / rate,
            "extrapolation": "512x512 rays / the all-thread crop rate (labelled extrapolated; "
                             "not measured)"}


def run_reference(args):
    import synth
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z, cam = make_workload(spec)
    c = _crop_camera(cam, args.ref_crop)
    sdf = oracle_sdf(spec, Ws, bs, Z)
    tgt = oracle_target(sdf, c)
    for _ in range(args.warmup):
        oracle_step(spec, sdf, c, tgt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(spec, sdf, c, tgt)
    dt = time.perf_counter() - t0
    v = args.ref_crop ** 2 * args.steps / dt
    return {
        "impl": "reference", "metric": "rays/s (pixels traced per second, forward+backward)",
        "value": v, "unit": "rays/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{args.ref_crop}x{args.ref_crop} crop"},
        "cpu_baseline": {"value": v, "unit": "rays/s", "cores": _blas_threads(), "kind": "oracle",
                         "sample": f"central {args.ref_crop}x{args.ref_crop} crop of the "
                                   f"512x512 view per step"},
        "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="auto",
                    choices=["auto", "bf16", "fp16", "fp32", "fp32_tc"])
    ap.add_argument("--refine-engine", default="tc", choices=["tc", "simt"],
                    help="kernel of the FP32-class queries after a BF16/FP16 hand-over")
    ap.add_argument("--refine-rule", default="march", choices=["march", "secant"],
                    help="step rule of the FP32-class queries after a BF16/FP16 hand-over")
    ap.add_argument("--eps-lo", type=float, default=1e-3,
                    help="|f| below which a BF16/FP16 ray switches to FP32 queries")
    ap.add_argument("--eps-mid", type=float, default=EPS_MID,
                    help="BF16 march: > 0 = FP16 queries between the BF16 march and the "
                         "FP32-class queries, handing over at this |f|")
    ap.add_argument("--refine", type=int, default=0,
                    help="0: FP32 convergence to eps; n: accept after n FP32 queries")
    ap.add_argument("--alpha-refine", type=float, default=0.0,
                    help="step factor of the FP32 phase after a tensor-core march (0: alpha)")
    ap.add_argument("--size", type=int, default=512,
                    help="image side (512 is the benchmark workload; smaller for profiling)")
    ap.add_argument("--cpu-crop", type=int, default=96)
    ap.add_argument("--ref-crop", type=int, default=48)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--normals", action="store_true",
                    help="also render analytic normals in the forward pass")
    ap.add_argument("--coarse-levels", type=int, default=0,
                    help="coarse-to-fine tracing for the main line (0: exact per-pixel trace; "
                         "the coarse_to_fine key reports 2 beside it)")
    ap.add_argument("--latency-mode", type=int, default=1, choices=[0, 1],
                    help="1: steps with few tiles spread each tile over a four-SM cluster")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-side-configs", action="store_true",
                    help="skip the 5-view 256x256 and the 32x8x224^2 inverse-step lines")
    ap.add_argument("--inverse-steps", type=int, default=3,
                    help="timed Adam steps of the 32x8x224^2 inverse-step line")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-loads", default="0.5,0.95",
                    help="further Poisson loads reported under serving.by_load")
    ap.add_argument("--serve-load", type=float, default=0.8,
                    help="Poisson arrival rate as a fraction of the saturated request rate")
    ap.add_argument("--serve-fp32-sample", type=int, default=12)
    ap.add_argument("--oracle-crop-rate", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_crop_rate:
        # (child of cpu_baseline: the oracle's rate on one crop, printed as JSON)
        import synth
        spec = synth.DEEPSDF_SPEC
        Ws, bs, Z, cam = make_workload(spec)
        rate, dt = _oracle_crop_rate(spec, oracle_sdf(spec, Ws, bs, Z), cam, args.oracle_crop_rate)
        print(json.dumps({"rate": rate, "s": dt}), flush=True)
        return
    global SIZE
    SIZE = args.size
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
