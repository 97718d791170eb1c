"""Benchmark of one DVGOv2 training iteration (forward + backward + TV + Adam)
on GB300, in fwd+bwd ray-samples/s (samples after bbox and occupancy
culling).

Default workload: the 160^3 DVGO-sized scene (10 blobs, occupancy mask,
colour MLP 39-128-128-3 in FP32, 8192 rays, TV, sparse Adam), seeded
synthetic inputs.  Each timed step is bracketed by CUDA events on the
launching stream after an L2 flush (a 256 MB memset outside the events).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload dvgo_160|dvgo_160_bf16|small_64|unbounded_320]
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

METRIC = "fwd+bwd ray-samples/s"
FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dvgo_160")
    ap.add_argument("--rays", type=int, default=0,
                    help="rays per step (0: the workload's own count; smaller for profiler captures)")
    ap.add_argument("--tv-dense", action="store_true")
    ap.add_argument("--mlp", default="f32tc", choices=["f32tc", "f32"],
                    help="colour MLP of the FP32 workloads: tensor cores with split-FP16 "
                         "operands (FP32 accuracy) or the CUDA cores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the BF16 / learned-proposal comparison")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the second workload (unbounded_320) of the default run")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch the step's kernels one by one instead of replaying a CUDA graph")
    ap.add_argument("--profile-only", action="store_true",
                    help="run warmup+steps with no clock sampling or CPU baseline (for ncu)")
    return ap.parse_args()


def precision_of(workload, mlp="f32"):
    """Trainer precision of a workload: the BF16 form, else the FP32 form with
    its colour MLP on the tensor cores ("f32tc") or on the CUDA cores ("f32")."""
    return "bf16" if workload.endswith("bf16") else mlp


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------- ours
def kernel_flops_bytes(tr):
    """Counts of one step that the algorithmic-work formulas use: samples, live
    samples, and the distinct grid voxels and bricks the trilinear corners of
    all samples / of the live samples touch (the lower corner follows the
    sampler's border clamp; measurement only, outside every timed region)."""
    import torch
    torch.cuda.synchronize()
    S = int(tr.ray_off[-1].item())
    S_live = int(tr.live_count.item())
    Gx, Gy, Gz = tr.G
    cfg = tr.cfg
    dev = tr.xyz.device
    Gt = torch.tensor([Gx, Gy, Gz], dtype=torch.float32, device=dev)
    scale = (Gt - 1) / (cfg.bbox_max - cfg.bbox_min)
    offs = torch.tensor([(k >> 2) * Gx * Gy + ((k >> 1) & 1) * Gx + (k & 1) for k in range(8)],
                        dtype=torch.int64, device=dev)

    def distinct(xyz):
        u = ((xyz - cfg.bbox_min) * scale).clamp(min=0)
        u = torch.minimum(u, Gt - 1).floor().to(torch.int64)
        u = torch.minimum(u, (Gt - 2).to(torch.int64))
        base = (u[:, 2] * Gy + u[:, 1]) * Gx + u[:, 0]
        vox = torch.unique((base[:, None] + offs).reshape(-1))
        x, y, z = vox % Gx, (vox // Gx) % Gy, vox // (Gx * Gy)
        nbx, nby = (Gx + 7) // 8, (Gy + 7) // 8
        bricks = torch.unique(((z // 8) * nby + y // 8) * nbx + x // 8)
        return int(vox.numel()), int(bricks.numel())

    V_all, _ = distinct(tr.xyz[:S])
    V_live, B_live = distinct(tr.xyz[tr.live_idx[:S_live].long()])
    return dict(S=S, S_live=S_live, R=tr.R, V_all=V_all, V_live=V_live, B_live=B_live)


def per_kernel_times(tr, batches, flush, reps=5):
    """Duration of each C-ABI call of one step, CUDA events on the launching
    stream (the current stream), L2 flushed before each step as in the timed
    run.  Calls are keyed "name#k", k the call's position among the step's
    calls of that name (e.g. density then feature for the grid calls)."""
    import torch
    from paper_2206_05085_gb300 import _lib as L
    orig = L._call
    stream = torch.cuda.current_stream()
    events = []
    seen = {}

    def timed(name, *args):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        orig(name, *args)
        e1.record(stream)
        k = seen.get(name, 0)
        seen[name] = k + 1
        events.append((f"{name}#{k}", e0, e1))

    L._call = timed
    try:
        for r in range(reps):
            flush.zero_()
            # the host enqueues the whole step while the GPU spins (~1 ms), so
            # that no interval includes host-side launch time
            torch.cuda._sleep(2_000_000)
            seen.clear()
            o, d, t = batches[r % len(batches)]
            tr.step(o, d, t)
    finally:
        L._call = orig
    torch.cuda.synchronize()
    acc = {}
    for key, e0, e1 in events:
        acc.setdefault(key, []).append(e0.elapsed_time(e1))
    return {key: sum(ts) / len(ts) for key, ts in acc.items()}


def by_entry_point(calls):
    """Per C-ABI entry point: ms per step, calls per step, ms per call."""
    out = {}
    for key, ms in calls.items():
        name = key.split("#")[0]
        r = out.setdefault(name, {"ms_per_step": 0.0, "calls_per_step": 0})
        r["ms_per_step"] += ms
        r["calls_per_step"] += 1
    for r in out.values():
        r["ms_per_call"] = r["ms_per_step"] / r["calls_per_step"]
    return out


def l2_read_gbs(mb=32, reps=40):
    """L2 read rate: one launch of the library's read probe over a buffer well
    inside L2 (152 x 4 blocks, each pass over the whole buffer; the best of
    three launches after a warm-up).  The denominator of the gathers' logical
    (per-corner) traffic."""
    import torch
    from paper_2206_05085_gb300 import _lib as L
    nbytes = mb << 20
    buf = torch.ones(nbytes // 4, device="cuda")
    sink = torch.zeros(152 * 4, device="cuda")
    L.read_probe(buf, nbytes, 2, sink)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        L.read_probe(buf, nbytes, reps, sink)
        e1.record()
        e1.synchronize()
        best = max(best, nbytes * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def reduce_over_ranks(total_ms, e2e_ms, samples, device):
    """Whole-job figures of an N-rank run: the slowest rank's times (max)
    and the samples of all ranks (sum); unchanged without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return total_ms, e2e_ms, samples
    t = torch.tensor([total_ms, e2e_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    s = torch.tensor([samples], dtype=torch.float64, device=device)
    dist.all_reduce(s)
    return float(t[0]), float(t[1]), float(s[0])


def prepare(workload, mlp, rank, n_batches, rays=0):
    """Trainer of a workload and its ray batches resident in HBM (seed =
    1000 * rank + batch), with the sample and live-sample count of each batch
    (deterministic: the occupancy mask is fixed).  The trainer is re-created
    after the counting passes, so the optimizer starts clean."""
    import torch
    from paper_2206_05085_gb300 import synth, train
    cfg = synth.CONFIGS[workload]
    if rays:
        import dataclasses
        cfg = dataclasses.replace(cfg, n_rays=int(rays))
    rp = synth.render_params(cfg)
    prec = precision_of(workload, mlp)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    tr = train.Trainer(cfg, rp, D, Fg, P, n_rays=cfg.n_rays, precision=prec)
    batches, host_batches = [], []
    for i in range(min(n_batches, 8)):
        seed = 1000 * rank + i
        o, d = synth.rays(cfg, seed=seed)
        t = synth.target_rgb(cfg, seed=seed)
        host_batches.append((o, d, t))
        batches.append(tuple(torch.from_numpy(a).cuda() for a in (o, d, t)))
    S_of, SL_of = [], []
    for o, d, t in batches:
        tr.forward(o, d, t)
        torch.cuda.synchronize()
        S_of.append(int(tr.ray_off[-1].item()))
        SL_of.append(int(tr.live_count.item()))
    del tr
    tr = train.Trainer(cfg, rp, D, Fg, P, n_rays=cfg.n_rays, precision=prec)
    return dict(tr=tr, batches=batches, host_batches=host_batches, S_of=S_of, SL_of=SL_of, cfg=cfg,
                rp=rp, prec=prec)


def timed_steps(w, steps, warmup, flush, tv_dense, graph=True, clocks=None, world=1):
    """warmup untimed steps, then `steps` steps each bracketed by CUDA events
    on the launching stream (L2 flushed before each, outside the events).
    With graph, the step is one CUDA graph replay; each replay first copies
    its batch into the graph's input buffers (inside the events)."""
    import torch
    tr, batches, S_of, SL_of = w["tr"], w["batches"], w["S_of"], w["SL_of"]
    stream = torch.cuda.current_stream()
    for i in range(warmup):
        tr.step(*batches[i % len(batches)], tv_dense=tv_dense)
    torch.cuda.synchronize()
    g, g_in = None, None
    if graph:
        g, g_in = tr.capture(*batches[0], tv_dense=tv_dense)
        torch.cuda.synchronize()

    def one_step(o, d, t):
        if g is None:
            return tr.step(o, d, t, tv_dense=tv_dense)
        for dst, src in zip(g_in, (o, d, t)):
            dst.copy_(src, non_blocking=True)
        g.replay()
        return tr.loss

    if clocks:
        clocks.start()
        time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev, samples, live = [], 0, 0
    for i in range(steps):
        flush.zero_()
        b = (warmup + i) % len(batches)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step(*batches[b])
        e1.record(stream)
        ev.append((e0, e1))
        samples += S_of[b]
        live += SL_of[b]
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    return dict(total_ms=total_ms, samples=samples, live=live, graph=g, g_in=g_in)


def run_ours(args, rank, world):
    import torch
    from paper_2206_05085_gb300 import _lib as L
    from paper_2206_05085_gb300 import build as B
    B.build()
    torch.cuda.set_device(rank % max(torch.cuda.device_count(), 1))
    w = prepare(args.workload, args.mlp, rank, args.warmup + args.steps, args.rays)
    tr, batches, host_batches = w["tr"], w["batches"], w["host_batches"]
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    if args.profile_only:
        for i in range(args.warmup + args.steps):
            tr.step(*batches[i % len(batches)], tv_dense=args.tv_dense)
        torch.cuda.synchronize()
        return None
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    tm = timed_steps(w, args.steps, args.warmup, flush, args.tv_dense, graph=not args.no_graph,
                     clocks=clocks, world=world)
    graph, g_in = tm["graph"], tm["g_in"]

    # end-to-end through the public API with host buffers: pinned H2D of the
    # step's rays and targets, D2H of the loss, inside the timed region
    pinned = [tuple(torch.from_numpy(a).pin_memory() for a in hb) for hb in host_batches]
    dev_in = [torch.empty_like(x) for x in batches[0]]
    loss_host = torch.empty(3, dtype=torch.float32).pin_memory()
    e2e_ms = []
    h2d_bytes = sum(x.numel() * x.element_size() for x in pinned[0])
    for i in range(args.steps):
        flush.zero_()
        b = (args.warmup + i) % len(pinned)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dst_in = dev_in if graph is None else g_in
        for dst, src in zip(dst_in, pinned[b]):
            dst.copy_(src, non_blocking=True)
        if graph is None:
            loss = tr.step(dst_in[0], dst_in[1], dst_in[2], tv_dense=args.tv_dense)
        else:
            graph.replay()
            loss = tr.loss
        loss_host.copy_(loss, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    clock_info = clocks.stop() if clocks else None
    # device status word of the kernels with range checks and bounded waits,
    # read once after all timed steps (this call synchronises)
    status = L.device_status()

    calls = per_kernel_times(tr, batches[:1], flush, reps=5)
    l2_gbs = l2_read_gbs()
    kt = by_entry_point(calls)
    counts = kernel_flops_bytes(tr)
    S, S_live = counts["S"], counts["S_live"]
    total_ms, e2e_total, samples = reduce_over_ranks(tm["total_ms"], sum(e2e_ms), tm["samples"], "cuda")
    _, _, live = reduce_over_ranks(tm["total_ms"], 0.0, tm["live"], "cuda")
    return dict(total_ms=total_ms, steps=args.steps, l2_gbs=l2_gbs, samples=samples, live=live,
                e2e_total_ms=e2e_total, e2e_samples=samples, kt=kt, calls=calls, counts=counts,
                clocks=clock_info, S=S, S_live=S_live, h2d=h2d_bytes, cfg=w["cfg"], rp=w["rp"],
                prec=w["prec"], tr=tr, status=status)


def run_secondary(workload, mlp, steps=20, warmup=3):
    """A second workload in the same run (one GPU, rank 0): the same timed
    loop (CUDA graph replays, L2 flushed before each step), its per-call
    times and the memory-kernel record of its counts."""
    import torch
    from paper_2206_05085_gb300 import _lib as L
    w = prepare(workload, mlp, 0, warmup + steps)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    tm = timed_steps(w, steps, warmup, flush, False)
    status = L.device_status()
    tr = w["tr"]
    calls = per_kernel_times(tr, w["batches"][:1], flush, reps=3)
    counts = kernel_flops_bytes(tr)
    res = dict(total_ms=tm["total_ms"], steps=steps, samples=tm["samples"], live=tm["live"],
               kt=by_entry_point(calls), calls=calls, counts=counts, S=counts["S"],
               S_live=counts["S_live"], prec=w["prec"], cfg=w["cfg"], status=status)
    del w, tr
    torch.cuda.empty_cache()
    return res


# Algorithmic work per unit of each kernel (the roofline numerators).
# Colour MLP, per live sample: forward 2*(39*128 + 128*128 + 128*3) FLOP; backward
# twice the forward (the two products of every layer: the input gradient and the
# weight gradient), 87,040 FLOP.  What a kernel recomputes (the tensor-core
# backward takes layer 2 again from the stored layer inputs) is not counted.
MLP_FWD_FLOP = 2 * (39 * 128 + 128 * 128 + 128 * 3)
MLP_BWD_FLOP = 2 * MLP_FWD_FLOP
# Tensor-core MMAs issued per algorithmic product: the FP32 form splits every
# operand into two FP16 terms (hi*hi + hi*lo + lo*hi: 3); the BF16 form keeps
# weights as one term (products with a weight matrix: 2) and splits both
# operands of a weight gradient (3).  The inverse is the fraction of the tensor
# peak a kernel can reach in algorithmic FLOP/s.
MMA_CEILING = {("f32tc", "fwd"): 1 / 3, ("f32tc", "bwd"): 1 / 3, ("bf16", "fwd"): 1 / 2,
               # backward: dW2 (3) and g_h1 (2) of 128x128, dW1 (3) of 128x40, g_k0 (2) of 128x12
               ("bf16", "bwd"): (2 * 16384 + 5120 + 1536) / (5 * 16384 + 3 * 5120 + 2 * 1536)}
# kernels launched per C-ABI call (others launch one); the tensor-core MLP
# backward runs the backward and the partial-gradient reduction
# kernels each C-ABI call launches (the rest launch one): sampling counts,
# scans and fills; the live list scans and fills; the device-side Adam step
# advances its step count, then updates
KERNELS_PER_CALL = {"dvgo_sample_rays": 3, "dvgo_live_samples": 2, "dvgo_touched_compact": 1,
                    "dvgo_adam_step_multi_dev": 2}


def roofline(res, peaks, mk=None):
    """Roofline record of the dominant kernel (largest share of the step).
    The kernel is timed per call, alone on the stream: the burst tensor peak
    is its denominator."""
    kt = res["kt"]
    name, rec = max(kt.items(), key=lambda kv: kv[1]["ms_per_step"])
    S_live, prec = res["S_live"], res["prec"]
    ms = rec["ms_per_call"]
    fp32_peak = 152 * 128 * 2 * 2070e6 / 1e12   # FP32 FMA TFLOP/s at the maximum SM clock
    out = {"kernel": name}
    if name in ("dvgo_rgbnet_bwd", "dvgo_rgbnet_fwd"):
        way = "fwd" if name.endswith("fwd") else "bwd"
        per = MLP_FWD_FLOP if way == "fwd" else MLP_BWD_FLOP
        flop = per * S_live
        achieved = flop / (ms * 1e-3) / 1e12
        if prec in ("bf16", "f32tc"):
            bound, unit = "tensor", "TFLOP/s"
            peak = peaks.get("bf16_tflops", 1900.0)
            peak_src = ("bf16_tflops of measured (burst; FP16 runs at the BF16 rate)" if "bf16_tflops" in peaks
                        else "1.9 PFLOP/s bf16 burst (fallback)")
            ceil = MMA_CEILING[(prec, way)]
            out["mma_ceiling_frac"] = round(ceil, 4)
            out["frac_of_mma_ceiling"] = round(achieved / (peak * ceil), 4)
        else:
            bound, peak, unit = "alu", round(fp32_peak, 2), "TFLOP/s"
            peak_src = "FP32 FMA: 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz (derived)"
        out.update(bound=bound, achieved=round(achieved, 2), peak=peak, unit=unit,
                   frac=round(achieved / peak, 4), flop_per_unit=per, units=S_live,
                   peak_source=peak_src)
    else:
        # a memory kernel: its algorithmic bytes (memory_kernels) over its time
        peak = peaks.get("hbm_gbs", 6800.0)
        b = (mk or {}).get("kernels", {}).get(name + "#0", {}).get("bytes")
        ach = b / (ms * 1e-3) / 1e9 if b else None
        out.update(bound="hbm", achieved=round(ach, 1) if ach else None, peak=peak, unit="GB/s",
                   frac=round(ach / peak, 4) if ach else None, bytes_per_launch=b,
                   peak_source="hbm_gbs of measured" if "hbm_gbs" in peaks else "6800 GB/s (fallback)")
    out["traffic"] = traffic_for(name, prec, S_live)
    out["ms_per_call"] = round(ms, 4)
    out["share"] = round(rec["ms_per_step"] / sum(v["ms_per_step"] for v in kt.values()), 3)
    return out


def memory_kernels(res, peaks):
    """Achieved bandwidth of the memory-bound kernels of one step: algorithmic
    bytes per launch (what the method must move; formulas below, per sample /
    per live sample / per distinct voxel / per ray) / CUDA-event duration,
    against the measured HBM copy peak."""
    c, calls, prec = res["counts"], res["calls"], res["prec"]
    S, SL, R, Va, Vl, Bl = c["S"], c["S_live"], c["R"], c["V_all"], c["V_live"], c["B_live"]
    F = 12
    e = 2 if prec == "bf16" else 4          # bytes per grid element the renderer reads
    sh = 2 if prec == "bf16" else 0         # BF16 shadow written by Adam
    ent_d, ent_f = Bl * 512, Bl * 512 * F   # grid entries in the touched bricks
    # the feature query is the step's only dvgo_sample_grid_fwd once the density
    # query is fused into the weights pass, else the second one
    fused_density = "dvgo_density_alpha_fwd#0" in calls
    dens_key = None if fused_density else "dvgo_sample_grid_fwd#0"
    feat_key = "dvgo_sample_grid_fwd#0" if fused_density else "dvgo_sample_grid_fwd#1"
    algo = {
        # xyz + value out per sample, each distinct corner voxel once
        feat_key: SL * (4 + 12 + 4 * F) + Vl * e * F,
        # raw in, w and T out per sample; ray_off, n_live, T_end per ray
        "dvgo_alpha_weights_fwd#0": S * 12 + R * 16,
        # the density query fused in: xyz in per sample up to the halt, each distinct
        # queried voxel once; raw, w, T out per sample
        "dvgo_density_alpha_fwd#0": SL * 12 + Vl * e + S * 12 + R * 16,
        "dvgo_composite_rgb_fwd#0": SL * 16 + R * 28,
        "dvgo_distortion_fwd#0": SL * 12 + R * 16,
        "dvgo_distortion_bwd#0": SL * 16 + R * 12,
        # w, rgb, m, ds in per live sample; colour and L_r out per ray
        "dvgo_composite_distortion_fwd#0": SL * 24 + R * 32,
        # ... with the photometric loss: target in, g_color out per ray
        "dvgo_composite_distortion_loss_fwd#0": SL * 24 + R * 56,
        # g_w, raw, T, rgb in and g_raw out per live sample, g_raw zeroed past the halt
        "dvgo_composite_bwd#0": SL * 28 + (S - SL) * 4 + R * 24,
        # w, m (twice), ds, raw, T, rgb in and g_raw out per live sample
        "dvgo_composite_distortion_bwd#0": SL * 40 + (S - SL) * 4 + R * 24,
        # both in one pass: w, rgb, m, ds, raw, T in and g_raw out per live sample
        # (g_raw zeroed past the halt); target in, colour, L_r, g_color out per ray
        "dvgo_composite_distortion_loss_fwd_bwd#0": SL * 32 + S * 4 + R * 56,
        # g, xyz, index per live sample; FP32 gradient read-modify-write per distinct voxel
        "dvgo_sample_grid_bwd#0": SL * (4 + 12 + 4) + Vl * 8,
        "dvgo_sample_grid_bwd#1": SL * (4 * F + 12 + 4) + Vl * 8 * F,
        "dvgo_sample_grid_bwd2#0": SL * (4 + 4 * F + 12 + 4) + Vl * 8 * (1 + F),
        # sparse TV: the gradient of every entry of a touched brick is read; entries
        # with a non-zero gradient (the distinct voxels the scatter reached) also
        # read their value and write the gradient back
        "dvgo_tv_add_grad#0": ent_d * 4 + Vl * (e + 4),
        "dvgo_tv_add_grad#1": ent_f * 4 + Vl * F * (e + 4),
        # Adam: g of every entry of a touched brick; where g != 0, p, m, v in and
        # p, m, v, g (and the BF16 shadow) out
        "dvgo_adam_step#0": ent_d * 4 + Vl * (28 + sh),
        "dvgo_adam_step#1": ent_f * 4 + Vl * F * (28 + sh),
        # both grids in one launch (the colour MLP's 22019 entries ride along: 32 B each)
        "dvgo_tv_add_grad_multi#0": (ent_d + ent_f) * 4 + Vl * (1 + F) * (e + 4),
        "dvgo_adam_step_multi#0": (ent_d + ent_f) * 4 + Vl * (1 + F) * (28 + sh) + 22019 * 32,
        "dvgo_adam_step_multi_dev#0": (ent_d + ent_f) * 4 + Vl * (1 + F) * (28 + sh) + 22019 * 32,
    }
    if dens_key:
        algo[dens_key] = S * (12 + 4) + Va * e
    peak = peaks.get("hbm_gbs", 6800.0)
    out = {}
    for key, b in algo.items():
        if key not in calls:
            continue
        ms = calls[key]
        gbs = b / (ms * 1e-3) / 1e9
        out[key] = {"bytes": int(b), "ms": round(ms, 4), "achieved_gbs": round(gbs, 1),
                    "frac": round(gbs / peak, 3)}
    tot_b = sum(v["bytes"] for v in out.values())
    tot_ms = sum(v["ms"] for v in out.values())
    # logical gather traffic (8 corners x channels per sample) against the L2 read rate
    l2 = res.get("l2_gbs")
    gather = {}
    queries = [(feat_key, SL, F)] + ([(dens_key, S, 1)] if dens_key else
                                     [("dvgo_density_alpha_fwd#0", SL, 1)])
    for key, n, ch in queries:
        if key in calls and l2:
            b = n * 8 * ch * e
            gbs = b / (calls[key] * 1e-3) / 1e9
            gather[key] = {"logical_bytes": int(b), "effective_gbs": round(gbs, 1),
                           "frac_of_l2": round(gbs / l2, 3)}
    # what one iteration must move: every touched grid point (13 channels) is read
    # by the forward, re-read by the adjoint, its FP32 gradient read-modify-written
    # and its Adam state (p, g, m, v in; p, m, v out) moved once; step index and
    # ray id per sample written once, read twice; rays, colours, targets, loss per ray
    V_t = Bl * 512
    it_b = V_t * (1 + F) * (e + e + 8 + 28 + sh) + S * 24 + R * 48
    step_ms = res["total_ms"] / max(res.get("steps", 1), 1)
    it_gbs = it_b / (step_ms * 1e-3) / 1e9
    return {"peak_gbs": peak, "peak_source": "hbm_gbs of measured" if "hbm_gbs" in peaks
            else "6800 GB/s (fallback)",
            "counts": c, "kernels": out,
            "all": {"bytes": tot_b, "ms": round(tot_ms, 4),
                    "achieved_gbs": round(tot_b / (tot_ms * 1e-3) / 1e9, 1),
                    "frac": round(tot_b / (tot_ms * 1e-3) / 1e9 / peak, 3)},
            "l2_read_gbs": round(l2, 1) if l2 else None,
            "gather_effective": gather,
            "iteration": {"bytes": int(it_b), "touched_points": int(V_t), "ms": round(step_ms, 4),
                          "achieved_gbs": round(it_gbs, 1), "frac": round(it_gbs / peak, 3)}}


def traffic_for(name, prec, units):
    """DRAM bytes per launch from the committed ncu capture (profiles/traffic.json),
    scaled by units processed; None if the kernel source changed since."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(f"{name}:{prec}")
        if not rec:
            return None
        src = os.path.join(ROOT, rec["source"])
        if hashlib.sha1(open(src, "rb").read()).hexdigest() != rec["sha1"]:
            return None
        return int(rec["dram_bytes"] * units / rec["units"])
    except (OSError, ValueError, KeyError):
        return None


def fine_params(rp, factor=4):
    """Render parameters of a converged reference render: the same sampler
    with a step `factor` times finer (and the alpha interval scaled with it,
    so the density integral is unchanged)."""
    import dataclasses
    return dataclasses.replace(rp, step=float(np.float32(rp.step / factor)),
                               max_steps=rp.max_steps * factor,
                               interval=float(np.float32(rp.interval / factor)))


def forms_report(args):
    """The BF16, low-weight-cull and learned-proposal forms against the plain
    FP32 form on the same rays.  Two references: the converged render (the
    plain FP32 renderer with a 4x finer step: how far a form's arithmetic
    moves the render) and the held-out truth scene (train.heldout_truth_render:
    the model's grids refined 2x plus detail they cannot hold, rendered
    converged; the plain render scores about 33 dB against it, near the
    paper's Table 1 figure for Synthetic-NeRF).  Reported: PSNR of each
    render against both and against the plain render, the gap between a
    form's PSNR against the truth and the plain form's (the <= 0.1 dB
    criterion), and the iteration time of each (CUDA events, mean of 10
    steps)."""
    import torch
    from paper_2206_05085_gb300 import proposal, synth, train
    psnr = proposal.psnr
    out = {}
    cfg = synth.CFG2
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    st = torch.cuda.current_stream()

    def timed(fn, n=10):
        for _ in range(3):
            fn()
        ev = []
        for _ in range(n):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            ev.append((a, b))
        torch.cuda.synchronize()
        return sum(x.elapsed_time(y) for x, y in ev) / n

    def render(cfg_, rp_, prec, o, d, t, R):
        tr = train.Trainer(cfg_, rp_, D, Fg, P, n_rays=R, precision=prec)
        tr.forward(o, d, t)
        c = tr.color.clone()
        del tr
        torch.cuda.empty_cache()
        return c

    # BF16 vs FP32 on the dvgo_160 scene: timing at the workload's 8192 rays
    o, d = synth.rays(cfg, seed=11)
    t = synth.target_rgb(cfg, seed=11)
    to, td, tt = (torch.from_numpy(a).cuda() for a in (o, d, t))
    ms = {}
    for prec in ("f32", "f32tc", "bf16"):
        tr = train.Trainer(cfg, rp, D, Fg, P, n_rays=cfg.n_rays, precision=prec)
        ms[prec] = timed(lambda: tr.step(to, td, tt))
        del tr
    torch.cuda.empty_cache()
    # quality on 4096 of those rays
    Rq = 4096
    qo, qd, qt = to[:Rq].contiguous(), td[:Rq].contiguous(), tt[:Rq].contiguous()
    colors = {prec: render(cfg, rp, prec, qo, qd, qt, Rq) for prec in ("f32", "f32tc", "bf16")}
    gt = render(cfg, fine_params(rp), "f32tc", qo, qd, qt, Rq)
    truth = train.heldout_truth_render(cfg, rp, D, Fg, P, qo, qd, qt)
    out["references"] = {
        "converged": "the plain FP32 render with a 4x finer step, 4096 rays",
        "heldout_truth": (f"the grids refined to the 2x lattice plus N(0, {train.TRUTH_DETAIL_STD}^2) "
                          "detail in density and features, rendered with a 4x finer step, 4096 rays"),
        "plain_psnr_vs_converged_db": round(psnr(colors["f32tc"], gt), 3),
        "plain_psnr_vs_heldout_truth_db": round(psnr(colors["f32tc"], truth), 3)}
    out["fp32_mlp_on_cuda_cores"] = {
        "psnr_vs_tensor_core_fp32_render_db": round(psnr(colors["f32"], colors["f32tc"]), 2),
        "ms_per_step_cuda_cores": round(ms["f32"], 3), "ms_per_step_tensor_cores": round(ms["f32tc"], 3)}
    p_plain = psnr(colors["f32tc"], truth)
    p_bf = psnr(colors["bf16"], truth)
    # the low-weight cull of the colour query (w < 1e-4), and the progressive mask update
    trc = train.Trainer(cfg, rp, D, Fg, P, n_rays=cfg.n_rays, precision="f32tc", w_min=1e-4)
    ms_cull = timed(lambda: trc.step(to, td, tt))
    del trc
    trm = train.Trainer(cfg, rp, D, Fg, P, n_rays=cfg.n_rays, precision="f32tc", mask_update=True)
    ms_mask = timed(lambda: trm.step(to, td, tt))
    del trm
    trc = train.Trainer(cfg, rp, D, Fg, P, n_rays=Rq, precision="f32tc", w_min=1e-4)
    trc.forward(qo, qd, qt)
    c_cull = trc.color.clone()
    n_q, n_l = int(trc.query_count.item()), int(trc.live_count.item())
    del trc
    torch.cuda.empty_cache()
    out["low_weight_cull"] = {
        "w_min": 1e-4, "colour_queries": n_q, "live_samples": n_l,
        "psnr_vs_full_render_db": round(psnr(c_cull, colors["f32tc"]), 2),
        "psnr_vs_converged_db": round(psnr(c_cull, gt), 3),
        "psnr_vs_heldout_truth_db": round(psnr(c_cull, truth), 3),
        "psnr_gap_db": round(abs(psnr(c_cull, truth) - p_plain), 4),
        "ms_per_step_8192_rays": round(ms_cull, 3)}
    out["mask_update"] = {"ms_per_step_8192_rays": round(ms_mask, 3),
                          "without_ms_per_step_8192_rays": round(ms["f32tc"], 3)}
    out["bf16"] = {"psnr_vs_fp32_render_db": round(psnr(colors["bf16"], colors["f32tc"]), 2),
                   "psnr_vs_converged_db": round(psnr(colors["bf16"], gt), 3),
                   "psnr_vs_heldout_truth_db": round(p_bf, 3),
                   "fp32_psnr_vs_heldout_truth_db": round(p_plain, 3),
                   "psnr_gap_db": round(abs(p_bf - p_plain), 4),
                   "ms_per_step_8192_rays": round(ms["bf16"], 3),
                   "fp32_ms_per_step_8192_rays": round(ms["f32tc"], 3)}
    # learned proposal vs dense candidates (<= 512 / ray), 16384 rays
    cfg5 = synth.CFG5
    R = cfg5.n_rays
    dense, prop_tr, prop = proposal.make_forms(cfg5, rp, D, Fg, P, synth.proposal_params(), R,
                                               precision=args.mlp)
    batches = [tuple(torch.from_numpy(a).cuda() for a in synth.rays(cfg5, seed=500 + i, n_rays=R))
               for i in range(8)]
    t0 = time.perf_counter()
    for it in range(400):
        ro, rd = batches[it % len(batches)]
        prop.train_step(ro, rd)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    o5, d5 = synth.rays(cfg5, seed=9)
    t5 = synth.target_rgb(cfg5, seed=9)
    to5, td5, tt5 = (torch.from_numpy(a).cuda() for a in (o5, d5, t5))
    dense.forward(to5, td5, tt5)
    c_dense = dense.color.clone()
    s_dense = int(dense.ray_off[-1].item())
    prop.select_into(prop_tr, to5, td5)
    prop_tr.forward(to5, td5, tt5, sample=False)
    c_prop = prop_tr.color.clone()
    s_prop = int(prop_tr.ray_off[-1].item())
    # the same budget without the network (64 evenly spaced picks), and the
    # picks without their spans (each keeping its one-candidate interval)
    others = {}
    for name, kw in (("uniform", dict(uniform=True)), ("no_spans", dict(spans=False))):
        prop.select_into(prop_tr, to5, td5, **kw)
        prop_tr.forward(to5, td5, tt5, sample=False)
        others[name] = prop_tr.color.clone()
    ms_dense = timed(lambda: dense.step(to5, td5, tt5))

    def prop_step():
        prop.select_into(prop_tr, to5, td5)
        prop_tr.step(to5, td5, tt5, sample=False)
    ms_prop = timed(prop_step)
    rp_c = proposal.candidate_params(cfg5, rp)
    del dense, prop_tr
    torch.cuda.empty_cache()
    # references on 4096 of the rays: the dense candidates 4x finer, and the held-out truth
    q5 = [x[:Rq].contiguous() for x in (to5, td5, tt5)]
    gt5 = render(cfg5, fine_params(rp_c), args.mlp, *q5, Rq)
    truth5 = train.heldout_truth_render(cfg5, rp_c, D, Fg, P, *q5)
    pd, pp = psnr(c_dense[:Rq], truth5), psnr(c_prop[:Rq], truth5)
    out["proposal"] = {
        "rays": R, "samples_dense": s_dense, "samples_proposal": s_prop,
        "psnr_vs_dense_render_db": round(psnr(c_prop, c_dense), 2),
        "uniform_draws_psnr_vs_dense_render_db": round(psnr(others["uniform"], c_dense), 2),
        "without_spans_psnr_vs_dense_render_db": round(psnr(others["no_spans"], c_dense), 2),
        "psnr_vs_converged_db": round(psnr(c_prop[:Rq], gt5), 3),
        "dense_psnr_vs_converged_db": round(psnr(c_dense[:Rq], gt5), 3),
        "psnr_vs_heldout_truth_db": round(pp, 3), "dense_psnr_vs_heldout_truth_db": round(pd, 3),
        "psnr_gap_db": round(abs(pp - pd), 4),
        "ms_per_step_dense": round(ms_dense, 3), "ms_per_step_proposal": round(ms_prop, 3),
        "proposal_training": f"400 steps x {R} rays on the plain renderer's weights, {train_s:.1f} s"}
    return out


def oracle_errors(mlp):
    """Second product of the oracle leg: on the first rays of each form's
    workload, the relative error (max|x - ref| / max|ref| per tensor) of every
    output and gradient of one GPU training step, and of the parameters after
    its TV + Adam update, against the same step composed from the FP64 oracle
    (the learned-proposal form: on the rays whose picks equal the oracle's);
    for the proposal network, its output and parameter gradients."""
    import torch
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    from conftest import rel_err
    from paper_2206_05085_gb300 import _lib as L
    from paper_2206_05085_gb300 import synth
    from step_parity import (error_table, gpu_proposal_step, gpu_step, mlp_grad_errors,
                             oracle_proposal_step, oracle_step)
    oracle.build()
    out = {"definition": "max|gpu - oracle| / max|oracle| per tensor; FP64 oracle on the same rays"}
    n = 64
    for form, workload, prec, tau, tol in (("fp32", "dvgo_160", mlp, 1e-6, 1e-5),
                                           ("bf16", "dvgo_160_bf16", "bf16", 1e-5, 2e-3)):
        cfg = synth.CONFIGS[workload]
        rp = synth.render_params(cfg)
        D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
        o, d = synth.rays(cfg, seed=0)
        t = synth.target_rgb(cfg, seed=0)
        o, d, t = o[:n], d[:n], t[:n]
        gpu = gpu_step(cfg, rp, D, Fg, P, o, d, t, prec, False)
        fb, opt, Pr = oracle_step(cfg, rp, D, Fg, P, o, d, t, prec, False)
        e = error_table(gpu, fb, opt, cfg, rp, Pr, tau)
        rec = {k: (float(f"{v:.3g}") if isinstance(v, float) else v) for k, v in e.items()}
        rec.update(workload=workload, rays=n, tolerance=tol, relu_tau=tau,
                   max_error=float(f"{max(v for k, v in e.items() if isinstance(v, float) and not k.endswith(('max_step', '_raw'))):.3g}"))
        out[form] = rec
        del gpu, fb, opt
        torch.cuda.empty_cache()
    # the learned-proposal form (FP32 step on <= 64 picks of <= 512 candidates per ray)
    import dataclasses
    from paper_2206_05085_gb300 import proposal
    cfg = synth.CONFIGS["dvgo_160_proposal"]
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    PP = (synth.proposal_params() * 3.0).astype(np.float32)
    o, d = synth.rays(cfg, seed=0)
    t = synth.target_rgb(cfg, seed=0)
    o, d, t = o[:n], d[:n], t[:n]
    gpu = gpu_proposal_step(cfg, rp, D, Fg, P, PP, o, d, t, mlp, False)
    fb, opt, Pr, sel, n_sel = oracle_proposal_step(cfg, rp, D, Fg, P, PP, o, d, t, mlp, False)
    agree = np.array([n_sel[r] == gpu["n_sel"][r] and np.array_equal(sel[r], gpu["sel"][r])
                      for r in range(n)])
    if not agree.all():
        o, d, t = o[agree], d[agree], t[agree]
        gpu = gpu_proposal_step(cfg, rp, D, Fg, P, PP, o, d, t, mlp, False)
        fb, opt, Pr, sel, n_sel = oracle_proposal_step(cfg, rp, D, Fg, P, PP, o, d, t, mlp, False)
    rp_p = dataclasses.replace(proposal.candidate_params(cfg, rp), max_steps=proposal.N_DRAW)
    e = error_table(gpu, fb, opt, cfg, rp_p, Pr, 1e-6)
    e["delta"] = rel_err(gpu["delta"], fb["delta"])
    rec = {k: (float(f"{v:.3g}") if isinstance(v, float) else v) for k, v in e.items()}
    rec.update(workload="dvgo_160_proposal", rays=int(len(o)), rays_with_other_picks=int(n - len(o)),
               tolerance=1e-5, relu_tau=1e-6,
               max_error=float(f"{max(v for k, v in e.items() if isinstance(v, float) and not k.endswith(('max_step', '_raw'))):.3g}"))
    out["proposal_form"] = rec
    del gpu, fb, opt
    torch.cuda.empty_cache()
    # learned proposal network (BF16 form) on 8192 points of the bbox
    rng = np.random.default_rng(31)
    m = 8192
    xyz = rng.uniform(-1, 1, (m, 3)).astype(np.float32)
    pp = synth.proposal_params()
    pr = synth.bf16_round(pp)
    g = rng.normal(size=m).astype(np.float32)
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    lg = torch.empty(m, device="cuda")
    L.proposal_fwd(dv(xyz), None, m, None, dv(pp), lg)
    gpp = torch.zeros(pp.size, device="cuda")
    L.proposal_bwd(dv(g), dv(xyz), None, m, None, dv(pp), gpp)
    x = oracle.freq_encode(xyz, 6)
    ref = oracle.mlp_fwd(synth.PROPOSAL_DIMS, pr, x, False)[:, 0]
    got, ggot = lg.cpu().numpy(), gpp.cpu().numpy()
    prop = {"points": m, "tolerance": 2e-3, "relu_tau": 2e-5, "logits": float(f"{rel_err(got, ref):.3g}")}
    raw, adj, n_amb = mlp_grad_errors(synth.PROPOSAL_DIMS, pr, x, g[:, None], ggot, 2e-5, out_sigmoid=False)
    for nm in raw:
        prop["g_" + nm] = float(f"{adj[nm]:.3g}")
        prop["g_" + nm + "_raw"] = float(f"{raw[nm]:.3g}")
    prop["relu_ambiguous_points"] = n_amb
    out["proposal_network"] = prop
    return out


def cpu_baseline(workload, max_seconds=20.0):
    """The FP64 oracle timed on the host on a bounded slice of the workload."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    from oracle_step import forward_backward
    from paper_2206_05085_gb300 import synth
    oracle.build()
    cfg = synth.CONFIGS[workload]
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    if precision_of(workload) == "bf16":
        D, Fg, P = synth.bf16_round(D), synth.bf16_round(Fg), synth.bf16_round(P)
    o, d = synth.rays(cfg, seed=0)
    t = synth.target_rgb(cfg, seed=0)
    n = 64
    samples, t0 = 0, time.perf_counter()
    start = 0
    while True:
        sl = slice(start, start + n)
        fb = forward_backward(cfg, rp, D, Fg, P, o[sl], d[sl], t[sl])
        samples += fb["smp"].S
        start += n
        el = time.perf_counter() - t0
        if el > max_seconds or start >= cfg.n_rays:
            break
    return {"value": samples / el, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{start} of {cfg.n_rays} rays of {workload}, forward+backward, "
                      f"single-threaded FP64 C oracle, {el:.1f} s"}


def _oracle_worker(job):
    """One spawned process: the FP64 oracle's forward + backward over its
    share of 64-ray slices until the time budget is spent."""
    workload, slices, max_seconds = job
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle
    from oracle_step import forward_backward
    from paper_2206_05085_gb300 import synth
    oracle.build()
    cfg = synth.CONFIGS[workload]
    rp = synth.render_params(cfg)
    D, Fg, P = synth.density_grid(cfg), synth.feature_grid(cfg), synth.mlp_params()
    if precision_of(workload) == "bf16":
        D, Fg, P = synth.bf16_round(D), synth.bf16_round(Fg), synth.bf16_round(P)
    o, d = synth.rays(cfg, seed=0)
    t = synth.target_rgb(cfg, seed=0)
    samples, rays, t0 = 0, 0, time.perf_counter()
    for a, b in slices:
        fb = forward_backward(cfg, rp, D, Fg, P, o[a:b], d[a:b], t[a:b])
        samples += fb["smp"].S
        rays += b - a
        if time.perf_counter() - t0 > max_seconds:
            break
    return samples, rays, time.perf_counter() - t0


def cpu_baseline_all_cores(workload, max_seconds=20.0):
    """The same oracle on every host core: one spawned process per core, each
    on its own slices of the workload's rays (the oracle itself unchanged)."""
    import multiprocessing
    from paper_2206_05085_gb300 import synth
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    R, n = synth.CONFIGS[workload].n_rays, 64
    slices = [(a, min(a + n, R)) for a in range(0, R, n)]
    jobs = [(workload, slices[i::cores], max_seconds) for i in range(cores)]
    with multiprocessing.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    samples = sum(r[0] for r in res)
    rays = sum(r[1] for r in res)
    el = max(r[2] for r in res)
    return {"value": samples / el, "unit": METRIC, "cores": cores, "kind": "oracle",
            "sample": f"{rays} of {R} rays of {workload}, forward+backward, FP64 C oracle, "
                      f"{cores} processes, {el:.1f} s"}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        cb = cpu_baseline(args.workload, max_seconds=max(5.0, 2.0 * (args.steps + args.warmup)))
        line = {"impl": "reference", "metric": METRIC, "value": round(cb["value"], 1),
                "unit": "ray-samples/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload},
                "cpu_baseline": cb,
                "e2e": {"value": round(cb["value"], 1), "unit": "ray-samples/s",
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    res = run_ours(args, rank, world)
    if res is None or rank != 0:
        return
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    cfg, rp = res["cfg"], res["rp"]
    value = res["samples"] / (res["total_ms"] * 1e-3)
    e2e = res["e2e_samples"] / (res["e2e_total_ms"] * 1e-3)
    per_call = dict(KERNELS_PER_CALL)
    if res["prec"] == "f32tc":
        per_call["dvgo_rgbnet_bwd"] = 2
    launches_per_step = sum(v["calls_per_step"] * per_call.get(k, 1) for k, v in res["kt"].items())
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "ray-samples/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(res["total_ms"] / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16" if res["prec"] == "bf16" else "f32", "data": "synthetic",
        "config": {"workload": cfg.name, "grid": cfg.grid, "rays": cfg.n_rays,
                   "samples_per_step": res["S"], "live_samples_per_step": res["S_live"],
                   "mlp": "39-128-128-3",
                   "mlp_precision": {"f32tc": "FP32 accuracy on tcgen05 (split-FP16 operands)",
                                     "f32": "FP32 on the CUDA cores",
                                     "bf16": "BF16 on tcgen05 (stored BF16 weights, two-term "
                                             "BF16 activations and gradients)"}[res["prec"]],
                   "tv_dense": bool(args.tv_dense), "l2": "flushed (256 MB memset) before each timed step",
                   "launch": "one CUDA graph per step" if not args.no_graph else "eager kernel launches",
                   "parallelism": "replicas" if args.gpus > 1 else "single"},
        "e2e": {"value": round(e2e, 1), "unit": "ray-samples/s", "h2d_bytes_per_step": res["h2d"],
                "d2h_bytes_per_step": 12},
        # samples in front of each ray's halt: the ones the feature query, the
        # colour MLP and the grid adjoints process
        "live_samples_per_s": round(res["live"] / (res["total_ms"] * 1e-3), 1),
        "device_status": res["status"],
        "gpu_launches": launches_per_step * args.steps,
        "roofline": roofline(res, peaks, memory_kernels(res, peaks)),
        "memory_kernels": memory_kernels(res, peaks),
        "kernels_ms_per_step": {k: round(v["ms_per_step"], 4) for k, v in res["kt"].items()},
        "clocks": res["clocks"],
    }
    # second workloads, timed the same way: the 320^3 contracted scene (grids far
    # larger than L2, 1.57 GB per FP32 feature array: the HBM-bound case of the
    # memory kernels) and the forward-facing 384^2 x 256 layer stack (NDC sampling)
    for name in (() if args.no_secondary or world > 1 else ("unbounded_320", "forward_facing_384")):
        if name == args.workload:
            continue
        sec = run_secondary(name, args.mlp)
        sec["l2_gbs"] = res["l2_gbs"]
        line[name] = {
            "value": round(sec["samples"] / (sec["total_ms"] * 1e-3), 1), "unit": "ray-samples/s",
            "live_samples_per_s": round(sec["live"] / (sec["total_ms"] * 1e-3), 1),
            "ms_per_step": round(sec["total_ms"] / sec["steps"], 4), "steps": sec["steps"], "warmup": 3,
            "samples_per_step": sec["S"], "live_samples_per_step": sec["S_live"],
            "device_status": sec["status"],
            "roofline": roofline(sec, peaks, memory_kernels(sec, peaks)),
            "memory_kernels": memory_kernels(sec, peaks),
            "kernels_ms_per_step": {k: round(v["ms_per_step"], 4) for k, v in sec["kt"].items()}}
    if not args.no_forms and world == 1:
        line["forms"] = forms_report(args)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(args.workload)
        line["cpu_baseline_all_cores"] = cpu_baseline_all_cores(args.workload)
        line["errors_vs_oracle"] = oracle_errors(args.mlp)
    bad = [v for v in [line["device_status"]] + [line.get(k, {}).get("device_status", 0)
                                                  for k in ("unbounded_320", "forward_facing_384")] if v]
    if bad:
        # a kernel reported a range or wait failure: the numbers above are not valid
        line["error"] = f"device status {bad[0]} after the timed steps"
        print(json.dumps(line))
        sys.exit(1)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
