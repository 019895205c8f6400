"""Throughput of the GB300 convolution library on the ResNet-50 bottleneck layer
set (BF16 NHWC, batch 32, bias + ReLU), plus the plain FP32 kernel on the same
layers, the FP8 workload, the grouped 64-problem launch and the backward pass.

One JSON line on rank 0. A "step" is one forward pass over the four layers
(1x1 256->64, 3x3 64->64, 1x1 64->256 at 56x56, 3x3 stride-2 128->128
56->28), each on its own synthetic batch. The timed region replays a CUDA
graph holding K steps; inputs rotate over four buffer sets (~750 MB in all,
well over the 129 MB L2), so every step reads its inputs from HBM.

--impl reference times the FP64 CPU oracle (the "reference arm" of this
comparison) on a bounded sample of the same workload on the host's cores.
Under torchrun every rank runs the same per-rank workload (weak scaling; the
layers shard over the batch with no exchange); rank 0 reports the total.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# max |y - y_oracle| / sum|x||w| allowed for BF16 outputs (twice the 2^-9 output rounding)
PARITY_TOL_BF16_OUT = 4e-3

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return dict(PEAKS_FALLBACK), "fallback"


# The sources the forward layer kernels are built from (kernels, shared
# headers, tensor maps, dispatch and planning): a change to any of them
# invalidates the recorded DRAM traffic.
FWD_SOURCES = ("api.cu", "tc_fwd.cu", "tc_fwd_t.cu", "tc_fwd_shift.cu", "tmap.cu", "epilogue.cuh",
               "launch.cuh", "ptx.cuh", "internal.h")


def csrc_sha1():
    import hashlib
    d = os.path.join(ROOT, "paper_2207_00257_gb300", "csrc")
    files = [os.path.join(d, n) for n in FWD_SOURCES]
    h = hashlib.sha1()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def ncu_traffic(tag):
    """DRAM bytes (read + write) per launch of this layer's kernel from the
    committed ncu record, or None if the kernel sources changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_dram_traffic.json")) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("csrc_sha1") != csrc_sha1() or tag not in rec.get("per_launch", {}):
        return None
    r = rec["per_launch"][tag]
    return r["dram_read"] + r["dram_write"]


# ---------------------------------------------------------------------------
# clocks sampling (nvidia-smi) during the measured region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self, t0, t1):
        rows = [p for (t, p) in self.rows if t0 <= t <= t1] or [p for (_, p) in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None

        sm = sorted(v for v in (num(r[1]) for r in rows) if v is not None)
        smax = max((v for v in (num(r[2]) for r in rows) if v is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for i, n in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(n)
        pw = [v for v in (num(r[3]) for r in rows) if v is not None]
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(rows),
                "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def layer_bytes(sh, eb_in, eb_out):
    x = sh.N * sh.H * sh.W * sh.C * eb_in
    w = sh.K * sh.R * sh.S * sh.C * eb_in
    y = sh.N * sh.P * sh.Q * sh.K * eb_out
    return x + w + sh.K * 4 + y


class Layer:
    """One convolution with its buffer sets, launched through the C ABI."""

    def __init__(self, sh, dtype, sets, seed, dev, relu=True):
        import torch
        from paper_2207_00257_gb300 import binding as B
        from paper_2207_00257_gb300.synth import make_inputs
        self.sh = sh
        self.dtype = dtype
        self.xs, self.ys = [], []
        x, w, b, _ = make_inputs(sh, seed)
        self.x_master = x
        self.w = w.to(dtype).to(dev)
        self.b = b.to(dev)
        self.w_master = w
        self.b_master = b
        for i in range(sets):
            xi = x if i == 0 else make_inputs(sh, seed + 7919 * i, bias=False)[0]
            self.xs.append(xi.to(dtype).to(dev))
            self.ys.append(torch.empty(sh.y_shape(), dtype=dtype, device=dev))
        ind = {torch.bfloat16: B.GBCONV_BF16, torch.float32: B.GBCONV_F32}[dtype]
        self.prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                              ind, ind, B.GBCONV_NHWC,
                              B.GBCONV_FLAG_BIAS | (B.GBCONV_FLAG_RELU if relu else 0))
        self.B = B

    def launch(self, i, stream):
        s = self.B.conv2d_fwd(self.prob, self.xs[i].data_ptr(), self.w.data_ptr(),
                              self.b.data_ptr(), 0, 0, self.ys[i].data_ptr(), 0, 0, stream)
        self.B.check(s, "conv2d_fwd")


def capture_steps(launch_fns, steps, nsets, torch, timed_events=True):
    """Captures `steps` steps into one CUDA graph. launch_fns: list of
    callables f(set_index, stream). Returns (graph, events[steps][len][2])."""
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    def ev():
        # "external" events become record nodes of the graph, so they can be timed
        return torch.cuda.Event(enable_timing=True, external=True)

    evs = [[(ev(), ev()) for _ in launch_fns] for _ in range(steps)] if timed_events else None
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            for st in range(steps):
                for j, f in enumerate(launch_fns):
                    if timed_events:
                        evs[st][j][0].record(stream)
                    f(st % nsets, stream.cuda_stream)
                    if timed_events:
                        evs[st][j][1].record(stream)
    return g, evs


def replay_timed(g, torch, dist_on):
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    start.record()
    g.replay()
    end.record()
    torch.cuda.synchronize()
    t1 = time.time()
    if dist_on:
        import torch.distributed as dist
        dist.barrier()
    return start.elapsed_time(end), t0, t1


def max_over_ranks(v, torch, dist_on):
    if not dist_on:
        return v
    from paper_2207_00257_gb300.distributed import max_over_ranks as mor
    return mor(v, device="cuda")


def bench_layers(layers, steps, warmup, nsets, torch, dist_on, sampler=None):
    """Times `steps` graph-replayed steps over `layers`. Returns dict with
    ms_per_step and per-layer average launch durations (us)."""
    fns = [lay.launch for lay in layers]
    # warm-up: eager steps (sets attributes, tensor maps), then graph warm-up replays
    for st in range(max(warmup, 1)):
        for f in fns:
            f(st % nsets, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    gw, _ = capture_steps(fns, nsets, nsets, torch, timed_events=False)
    for _ in range(max(warmup, 1)):
        gw.replay()
    torch.cuda.synchronize()
    # Headline: a graph of K steps with nothing between the launches, so each
    # kernel's launch overlaps the previous one's tail (programmatic launch).
    g, _ = capture_steps(fns, steps, nsets, torch, timed_events=False)
    g.replay()  # one untimed replay of the timed graph itself
    torch.cuda.synchronize()
    ms, t0, t1 = replay_timed(g, torch, dist_on)
    ms = max_over_ranks(ms, torch, dist_on)
    # Per-kernel durations: the same K steps with an event pair around every
    # launch (the events serialise the launches, so these include each
    # kernel's full launch and ramp).
    ge, evs = capture_steps(fns, steps, nsets, torch)
    ge.replay()
    torch.cuda.synchronize()
    ms_ev, _, _ = replay_timed(ge, torch, dist_on)
    per = [sum(evs[s][j][0].elapsed_time(evs[s][j][1]) for s in range(steps)) / steps * 1e3
           for j in range(len(fns))]
    return {"ms_total": ms, "ms_per_step": ms / steps, "launch_us": per, "t0": t0, "t1": t1,
            "ms_per_step_serialised": ms_ev / steps}


def resnet_report(layers, res, pk, eb):
    out = []
    for lay, us in zip(layers, res["launch_us"]):
        sh = lay.sh
        by = layer_bytes(sh, eb, eb)
        tf = sh.flops / (us * 1e-6) / 1e12
        gbs = by / (us * 1e-6) / 1e9
        ai = sh.flops / by
        attain = min(pk["bf16_tflops"], ai * pk["hbm_gbs"] / 1e3)
        out.append({"layer": sh.tag, "us": round(us, 2), "tflops": round(tf, 1),
                    "gbs": round(gbs, 1), "ai_flop_per_byte": round(ai, 1),
                    "frac_of_bf16_peak": round(tf / pk["bf16_tflops"], 4),
                    "frac_of_hbm": round(gbs / pk["hbm_gbs"], 4),
                    "frac_of_attainable": round(tf / attain, 4),
                    "bound": "hbm" if ai * pk["hbm_gbs"] / 1e3 < pk["bf16_tflops"] else "tensor",
                    "algorithmic_bytes": by, "dram_bytes_ncu": ncu_traffic(sh.tag)})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline BF16 layer set (skip FP32/FP8/grouped/backward)")
    ap.add_argument("--sections", default="fp32,fp8,grouped,backward,fused,groups,nll",
                    help="comma list of extra workloads to run after the headline layer set")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline leg")
    ap.add_argument("--jsonl", default=os.environ.get("GBCONV_BENCH_JSONL"),
                    help="also append one JSON record per result (headline, each layer, each "
                         "extra workload) to this file (default: $GBCONV_BENCH_JSONL, else none)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world, local)


def run_ours(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    dist_on = world > 1
    if dist_on:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2207_00257_gb300.synth import resnet_layers
    dev = torch.device("cuda", local)
    pk, pk_kind = peaks()
    nsets = 4
    layers = [Layer(sh, torch.bfloat16, nsets, 100 + i + 1000 * rank, dev)
              for i, sh in enumerate(resnet_layers(32))]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    res = bench_layers(layers, args.steps, args.warmup, nsets, torch, dist_on)
    flops_step = sum(l.sh.flops for l in layers)
    from paper_2207_00257_gb300.distributed import weak_scaling_rate
    value = weak_scaling_rate(flops_step * args.steps, world, res["ms_total"] * 1e-3) / 1e12
    per_layer = resnet_report(layers, res, pk, 2)
    # Each layer alone, K launches back to back in one graph (programmatic
    # launch overlapping consecutive launches): the per-layer cost inside the
    # headline step.
    for lay, row in zip(layers, per_layer):
        r1 = bench_layers([lay], max(3, min(args.steps, 50)), 1, nsets, torch, dist_on)
        row["us_overlapped"] = round(r1["ms_per_step"] * 1e3, 2)
        row["tflops_overlapped"] = round(lay.sh.flops / (r1["ms_per_step"] * 1e-3) / 1e12, 1)
    # Dominant kernel: the layer with the largest share of the step, by its
    # back-to-back launch time (K launches of that layer alone in one graph,
    # CUDA events around the graph, divided by K): the cost it adds to the
    # headline step, where each launch overlaps its neighbours' launch and
    # ramp. The event-separated time of one launch (events around every
    # launch, so no overlap) is reported beside it.
    j = max(range(len(layers)), key=lambda i: per_layer[i]["us_overlapped"])
    dom = per_layer[j]
    sh = layers[j].sh
    by = layer_bytes(sh, 2, 2)
    us = dom["us_overlapped"]
    if dom["bound"] == "tensor":
        ach = sh.flops / (us * 1e-6) / 1e12
        roof = {"bound": "tensor", "achieved": round(ach, 1), "peak": pk["bf16_tflops"],
                "unit": "TFLOP/s", "frac": round(ach / pk["bf16_tflops"], 4)}
    else:
        ach = by / (us * 1e-6) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(ach / pk["hbm_gbs"], 4)}
    roof.update({"kernel": f"forward kernel of {sh.tag}", "traffic": ncu_traffic(sh.tag),
                 "launch_us": us, "launch_timing": "back-to-back launches of this layer in one graph",
                 "launch_us_event_separated": dom["us"],
                 "algorithmic_bytes_per_launch": by,
                 "flops_per_launch": sh.flops, "peak_source": pk_kind + " (burst)"})
    clocks_window = (res["t0"], res["t1"])
    out = {
        "metric": "conv2d TFLOP/s & % of tensor peak, BF16/FP8 vs FP32 at stated rel err",
        "value": round(value, 2), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(res["ms_per_step"], 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded N(0,1) activations, He-normal weights, U[-0.1,0.1] bias)",
        "config": {"workload": "resnet50_bottleneck_layers_bf16_nhwc_batch32",
                   "layers": [l.sh.tag for l in layers], "global_batch": 32 * world,
                   "per_gpu_batch": 32, "epilogue": "bias+relu", "accumulate": "fp32",
                   "l2": f"inputs/outputs rotated over {nsets} buffer sets "
                         f"({nsets * sum(layer_bytes(l.sh, 2, 2) for l in layers) / 1e6:.0f} MB > 129 MB L2)",
                   "timing": "CUDA graph of K steps, CUDA events on the launch stream",
                   "parallelism": f"dp{world} (batch shards, no exchange)"},
        "frac_of_bf16_peak": round(value / world / pk["bf16_tflops"], 4),
        "ms_per_step_with_launch_events": round(res["ms_per_step_serialised"], 5),
        "layers": per_layer,
        "roofline": roof,
        "gpu_launches": len(layers) * args.steps,
    }
    # ---- e2e through the public API with host buffers ----
    out["e2e"] = e2e_resnet(layers, torch, dist_on, world, max(3, min(args.steps, 20)))
    # ---- extras: FP32 kernel, FP8, grouped, backward ----
    if not args.no_extras:
        sections = [x for x in args.sections.split(",") if x]
        fns = {"fp32": bench_fp32, "fp8": bench_fp8, "grouped": bench_grouped,
               "backward": bench_backward, "fused": bench_fused, "groups": bench_groups,
               "nll": bench_nll}
        for name in sections:
            try:
                out[name] = fns[name](torch, dev, args, dist_on, pk)
            except Exception as e:  # an extra workload never takes the headline line down
                torch.cuda.synchronize()
                out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
    sampler.stop()
    out["clocks"] = sampler.summary(*clocks_window)
    parity_bad = {}
    if rank == 0 and world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(layers, torch)
        # the step's outputs against the oracle: BF16 output rounding bounds the
        # normalised error by 2^-9; anything above twice that is a wrong result
        parity_bad = {k: v for k, v in out["cpu_baseline"]["max_normalised_err_bf16_vs_oracle"].items()
                      if not v <= PARITY_TOL_BF16_OUT}
        out["parity_ok"] = not parity_bad
    if rank == 0:
        print(json.dumps(out), flush=True)
        if args.jsonl:
            write_records(args.jsonl, out)
    if parity_bad:
        sys.stderr.write(f"bench: outputs differ from the FP64 oracle beyond {PARITY_TOL_BF16_OUT}: "
                         f"{parity_bad}\n")
        raise SystemExit(3)
    if dist_on:
        import torch.distributed as dist
        dist.destroy_process_group()


def write_records(path, out):
    """One JSON line per result: the headline, each layer of the step, each
    extra workload; every record carries the run's workload, clocks and
    oracle baseline so that it stands on its own."""
    common = {"time": time.strftime("%Y-%m-%dT%H:%M:%S"), "n_gpus": out["n_gpus"],
              "clocks": out.get("clocks"), "cpu_baseline": out.get("cpu_baseline")}
    recs = [dict(common, kind="headline", **{k: out[k] for k in (
        "metric", "value", "unit", "ms_per_step", "dtype", "config", "roofline", "e2e")})]
    for row in out.get("layers", []):
        recs.append(dict(common, kind="layer", **row))
    for name in ("fp32", "fp8", "grouped", "backward", "fused", "groups", "nll"):
        if name in out:
            recs.append(dict(common, kind=name, result=out[name]))
    with open(path, "a") as f:
        for r in recs:
            f.write(json.dumps(r) + "\n")


def e2e_resnet(layers, torch, dist_on, world, steps):
    """Same metric through the user call, with the copies in the timed region:
    per step and layer, the pinned host -> device copy of its input,
    conv2d_fwd through the public functional API, and the device -> pinned
    host copy of y. The copies run on their own streams (one per direction,
    so both copy engines and the C2C link's two directions work at once) and
    the inputs and outputs are double-buffered across steps: the upload of the
    next layer overlaps the convolution of this one and the download of the
    previous one. The serial form (everything on one stream) is timed too."""
    from paper_2207_00257_gb300 import functional as F
    hx = [l.xs[0].cpu().pin_memory() for l in layers]
    hy = [torch.empty(l.ys[0].shape, dtype=l.ys[0].dtype).pin_memory() for l in layers]
    dx = [[torch.empty_like(l.xs[0]) for _ in range(2)] for l in layers]
    dy = [[torch.empty_like(l.ys[0]) for _ in range(2)] for l in layers]
    s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    h2d_done = [[ev(), ev()] for _ in layers]
    conv_done = [[ev(), ev()] for _ in layers]
    d2h_done = [[ev(), ev()] for _ in layers]
    first = [[True, True] for _ in layers]

    def step(k):
        b = k & 1
        for i, l in enumerate(layers):
            with torch.cuda.stream(s_in):
                if not first[i][b]:
                    s_in.wait_event(conv_done[i][b])  # the convolution of step k-2 has read it
                dx[i][b].copy_(hx[i], non_blocking=True)
                h2d_done[i][b].record(s_in)
            with torch.cuda.stream(s_c):
                s_c.wait_event(h2d_done[i][b])
                if not first[i][b]:
                    s_c.wait_event(d2h_done[i][b])  # the download of step k-2 has read y
                F.conv2d(dx[i][b], l.w, l.b, l.sh.stride, l.sh.pad, l.sh.dil, True, "NHWC",
                         out=dy[i][b])
                conv_done[i][b].record(s_c)
            with torch.cuda.stream(s_out):
                s_out.wait_event(conv_done[i][b])
                hy[i].copy_(dy[i][b], non_blocking=True)
                d2h_done[i][b].record(s_out)
            first[i][b] = False

    def serial_step():
        st = torch.cuda.current_stream()
        for l, h, d, o in zip(layers, hx, dx, hy):
            d[0].copy_(h, non_blocking=True)
            y = F.conv2d(d[0], l.w, l.b, l.sh.stride, l.sh.pad, l.sh.dil, True, "NHWC", out=l.ys[0])
            o.copy_(y, non_blocking=True)

    def timed(run, n):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if dist_on:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        t0 = torch.cuda.current_stream()
        e0.record(t0)
        for sx in (s_in, s_c, s_out):
            sx.wait_event(e0)
        for k in range(n):
            run(k)
        for sx in (s_in, s_c, s_out):
            t0.wait_stream(sx)
        e1.record(t0)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), torch, dist_on)

    for k in range(4):  # warm-up, both forms
        step(k)
    serial_step()
    torch.cuda.synchronize()
    ms = timed(lambda k: step(k + 4), steps)
    ms_serial = timed(lambda k: serial_step(), steps)
    flops = sum(l.sh.flops for l in layers) * steps * world
    h2d = sum(t.numel() * t.element_size() for t in hx)
    d2h = sum(t.numel() * t.element_size() for t in hy)
    return {"value": round(flops / (ms * 1e-3) / 1e12, 2), "unit": "TFLOP/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "ms_per_step": round(ms / steps, 4),
            "link_gbs": round((h2d + d2h) / (ms / steps * 1e-3) / 1e9, 1),
            "pipeline": "H2D, compute and D2H on three streams, inputs/outputs double-buffered",
            "serial_ms_per_step": round(ms_serial / steps, 4),
            "serial_tflops": round(flops / (ms_serial * 1e-3) / 1e12, 2)}


def bench_fp32(torch, dev, args, dist_on, pk):
    from paper_2207_00257_gb300.synth import resnet_layers
    layers = [Layer(sh, torch.float32, 2, 100 + i, dev) for i, sh in enumerate(resnet_layers(32))]
    steps = max(3, min(args.steps, 20))
    res = bench_layers(layers, steps, 3, 2, torch, dist_on)
    flops = sum(l.sh.flops for l in layers)
    prop = torch.cuda.get_device_properties(dev)
    # FP32 CUDA-core peak: 128 FFMA lanes per SM x 2 flops x SMs x max SM clock,
    # and the FFMA probe's measured rate beside it (the roofline uses the probe)
    fp32_nominal = 2 * 128 * prop.multi_processor_count * 2.070e9 / 1e12
    from paper_2207_00257_gb300 import binding as B
    st, fp32_measured = B.gbconv_measure_ffma_tflops(20000, torch.cuda.current_stream().cuda_stream)
    B.check(st, "gbconv_measure_ffma_tflops")
    fp32_peak = fp32_measured
    v = flops / (res["ms_per_step"] * 1e-3) / 1e12
    rows = []
    for lay, us in zip(layers, res["launch_us"]):
        rows.append({"layer": lay.sh.tag, "us": round(us, 1),
                     "tflops": round(lay.sh.flops / (us * 1e-6) / 1e12, 2)})
    del layers
    torch.cuda.empty_cache()
    return {"tflops": round(v, 2), "ms_per_step": round(res["ms_per_step"], 4),
            "fp32_peak_tflops": round(fp32_peak, 1),
            "fp32_peak_note": "measured: FFMA probe kernel (gbconv_measure_ffma_tflops, CUDA events)",
            "fp32_nominal_tflops": round(fp32_nominal, 1),
            "fp32_nominal_note": "2 x 128 FFMA lanes x SMs x 2070 MHz (max clock)",
            "frac_of_fp32_peak": round(v / fp32_peak, 4),
            "frac_of_fp32_nominal": round(v / fp32_nominal, 4), "layers": rows,
            "kernel": "simt_igemm (FP32 FFMA, no tensor cores)"}


def bench_fp8(torch, dev, args, dist_on, pk):
    from paper_2207_00257_gb300 import binding as B
    from paper_2207_00257_gb300.synth import config_fp8, make_inputs
    sh = config_fp8()
    x, w, b, _ = make_inputs(sh, 3, "relu_normal", "he")
    nsets = 2
    xs = [x.to(dev)] + [make_inputs(sh, 3 + 11 * i, "relu_normal", "he", bias=False)[0].to(dev)
                        for i in range(1, nsets)]
    xq = [torch.empty(sh.x_shape(), dtype=torch.uint8, device=dev) for _ in range(nsets)]
    xsc = [torch.empty(1, dtype=torch.float32, device=dev) for _ in range(nsets)]
    wq = torch.empty(sh.w_shape(), dtype=torch.uint8, device=dev)
    wsc = torch.empty(sh.K, dtype=torch.float32, device=dev)
    wd = w.to(dev)
    st = torch.cuda.current_stream().cuda_stream
    B.check(B.gbconv_quantize_e4m3(wd.data_ptr(), B.GBCONV_F32, sh.K, wd.numel() // sh.K,
                                   wq.data_ptr(), wsc.data_ptr(), st), "quant w")
    bd = b.to(dev)
    ys = [torch.empty(sh.y_shape(), dtype=torch.bfloat16, device=dev) for _ in range(nsets)]
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_E4M3, B.GBCONV_BF16, B.GBCONV_NHWC, B.GBCONV_FLAG_BIAS)

    def quant(i, stream):
        B.check(B.gbconv_quantize_e4m3(xs[i].data_ptr(), B.GBCONV_F32, 1, xs[i].numel(),
                                       xq[i].data_ptr(), xsc[i].data_ptr(), stream), "quant x")

    def conv(i, stream):
        B.check(B.conv2d_fwd(prob, xq[i].data_ptr(), wq.data_ptr(), bd.data_ptr(),
                             xsc[i].data_ptr(), wsc.data_ptr(), ys[i].data_ptr(), 0, 0, stream),
                "fp8 conv")

    class L:
        def __init__(s, f):
            s.launch = f

    steps = max(3, min(args.steps, 50))
    res = bench_layers([L(quant), L(conv)], steps, 3, nsets, torch, dist_on)
    conv_us = res["launch_us"][1]
    # the convolution alone, back-to-back launches in one graph (as the headline layers)
    res_c = bench_layers([L(conv)], steps, 3, nsets, torch, dist_on)
    conv_b2b_us = res_c["ms_per_step"] * 1e3
    tf_conv = sh.flops / (conv_b2b_us * 1e-6) / 1e12
    tf_step = sh.flops / (res["ms_per_step"] * 1e-3) / 1e12
    fp8_peak, fp8_note = measure_fp8_peak(torch, dev)
    return {"workload": sh.tag, "tflops_conv_kernel": round(tf_conv, 1),
            "tflops_with_activation_quantisation": round(tf_step, 1),
            "conv_us": round(conv_b2b_us, 2),
            "conv_us_event_separated": round(conv_us, 2),
            "quant_us": round(res["launch_us"][0], 2),
            "fp8_peak_tflops": round(fp8_peak, 1),
            "fp8_peak_note": fp8_note,
            "frac_of_fp8_peak": round(tf_conv / fp8_peak, 4)}


def measure_fp8_peak(torch, dev):
    """Dense E4M3 tensor-core peak of this GPU: cuBLASLt through
    torch._scaled_mm on 8192^3 (per-tensor scales, BF16 output), best of 10
    launches timed with CUDA events after 3 warm-ups; the larger of the two
    accumulation modes."""
    n = 8192
    g = torch.Generator(device=dev).manual_seed(11)
    a = torch.randn(n, n, device=dev, generator=g).to(torch.float8_e4m3fn)
    b = torch.randn(n, n, device=dev, generator=g).to(torch.float8_e4m3fn).t()  # column-major
    one = torch.ones((), device=dev, dtype=torch.float32)
    best = {}
    for fast in (False, True):
        def mm():
            return torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16,
                                    use_fast_accum=fast)
        for _ in range(3):
            mm()
        torch.cuda.synchronize()
        ms = []
        for _ in range(10):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            mm()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        best[fast] = 2 * n ** 3 / (min(ms) * 1e-3) / 1e12
    del a, b
    torch.cuda.empty_cache()
    peak = max(best.values())
    return peak, (f"measured: torch._scaled_mm E4M3 {n}^3 (cuBLASLt), best of 10, CUDA events; "
                  f"{best[False]:.0f} TF (fp32 accumulate) / {best[True]:.0f} TF (fast accumulate)")


def bench_grouped(torch, dev, args, dist_on, pk):
    from paper_2207_00257_gb300 import binding as B
    from paper_2207_00257_gb300.synth import grouped_problems, make_inputs
    shapes = grouped_problems()
    xs, ws, bs, ys, probs = [], [], [], [], []
    for i, sh in enumerate(shapes):
        x, w, b, _ = make_inputs(sh, 1000 + i)
        xs.append(x.bfloat16().to(dev))
        ws.append(w.bfloat16().to(dev))
        bs.append(b.to(dev))
        ys.append(torch.empty(sh.y_shape(), dtype=torch.bfloat16, device=dev))
        probs.append(B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, 1,
                               B.GBCONV_BF16, B.GBCONV_BF16, B.GBCONV_NHWC,
                               B.GBCONV_FLAG_BIAS | B.GBCONV_FLAG_RELU))
    flops = sum(s.flops for s in shapes)
    xp = [t.data_ptr() for t in xs]
    wp = [t.data_ptr() for t in ws]
    bp = [t.data_ptr() for t in bs]
    yp = [t.data_ptr() for t in ys]

    def grouped(i, stream):
        B.check(B.conv2d_grouped(len(probs), probs, xp, wp, bp, yp, 0, 0, stream), "grouped")

    def separate(i, stream):
        for k, p in enumerate(probs):
            B.check(B.conv2d_fwd(p, xp[k], wp[k], bp[k], 0, 0, yp[k], 0, 0, stream), "fwd")

    class L:
        def __init__(s, f):
            s.launch = f

    steps = max(3, min(args.steps, 10))
    # heuristic tile widths, then each problem tuned once (outside the timed
    # region) as the grouped launch's body, then the tuned grouped launch
    rh = bench_layers([L(grouped)], steps, 3, 1, torch, dist_on)
    st = torch.cuda.current_stream().cuda_stream
    t0 = time.time()
    widths = []
    for k, p in enumerate(probs):
        s_, c = B.gbconv_tune(B.GBCONV_OP_GROUPED, p, xp[k], wp[k], bp[k], yp[k], 0, 0, 3, st)
        B.check(s_, "gbconv_tune(grouped)")
        widths.append(c.block_n)
    tune_s = time.time() - t0
    rg = bench_layers([L(grouped)], steps, 3, 1, torch, dist_on)
    rs = bench_layers([L(separate)], steps, 3, 1, torch, dist_on)
    B.gbconv_shutdown()  # clears the tuning table again
    del xs, ws, ys
    torch.cuda.empty_cache()
    tf = lambda r: round(flops / (r["ms_per_step"] * 1e-3) / 1e12, 1)
    return {"problems": len(shapes), "tflop_per_step": round(flops / 1e12, 4),
            "grouped_ms": round(rg["ms_per_step"], 4), "grouped_tflops": tf(rg),
            "grouped_tuning": "per-problem tile width tuned as the grouped launch's body "
                              f"(gbconv_tune GBCONV_OP_GROUPED, {tune_s:.1f} s for 64 problems)",
            "tuned_block_n": widths,
            "heuristic_grouped_ms": round(rh["ms_per_step"], 4), "heuristic_grouped_tflops": tf(rh),
            "separate_launches_ms": round(rs["ms_per_step"], 4), "separate_launches_tflops": tf(rs),
            "both_in_cuda_graphs": True,
            "frac_of_bf16_peak": round(flops / (rg["ms_per_step"] * 1e-3) / 1e12 / pk["bf16_tflops"], 4)}


def bench_backward(torch, dev, args, dist_on, pk):
    from paper_2207_00257_gb300 import binding as B
    from paper_2207_00257_gb300.synth import config_backward, make_inputs
    sh = config_backward()
    x, w, b, g = make_inputs(sh, 5, grad=True)
    xb, wb, gb = x.bfloat16().to(dev), w.bfloat16().to(dev), g.bfloat16().to(dev)
    dx = torch.empty(sh.x_shape(), dtype=torch.bfloat16, device=dev)
    dw = torch.empty(sh.w_shape(), dtype=torch.float32, device=dev)
    db = torch.empty(sh.K, dtype=torch.float32, device=dev)
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_BF16, B.GBCONV_BF16, B.GBCONV_NHWC, 0)
    s1, nd = B.gbconv_workspace_size(B.GBCONV_OP_DGRAD, prob)
    s2, nw = B.gbconv_workspace_size(B.GBCONV_OP_WGRAD, prob)
    wsd = torch.empty(max(nd, 1), dtype=torch.uint8, device=dev)
    wsw = torch.empty(max(nw, 1), dtype=torch.uint8, device=dev)

    def dgrad(i, stream):
        B.check(B.conv2d_dgrad(prob, gb.data_ptr(), wb.data_ptr(), dx.data_ptr(),
                               wsd.data_ptr(), nd, stream), "dgrad")

    def wgrad(i, stream):
        B.check(B.conv2d_wgrad(prob, xb.data_ptr(), gb.data_ptr(), dw.data_ptr(), db.data_ptr(),
                               wsw.data_ptr(), nw, stream), "wgrad")

    class L:
        def __init__(s, f):
            s.launch = f

    # data gradient of the strided ResNet layer (3x3 stride 2, 128 -> 128, 56 -> 28):
    # sub-pixel phases on the tensor cores (workspace, and the allocation-free
    # entry point's static scratch), and the CUDA-core gather kernel
    from paper_2207_00257_gb300.synth import resnet_layers
    s2 = resnet_layers(32)[3]
    _, w2, _, g2 = make_inputs(s2, 6, grad=True)
    w2b, g2b = w2.bfloat16().to(dev), g2.bfloat16().to(dev)
    dx2 = torch.empty(s2.x_shape(), dtype=torch.bfloat16, device=dev)
    prob2 = B.problem(s2.N, s2.C, s2.H, s2.W, s2.K, s2.R, s2.S, s2.stride, s2.pad, s2.dil,
                      B.GBCONV_BF16, B.GBCONV_BF16, B.GBCONV_NHWC, 0)
    _, nd2 = B.gbconv_workspace_size(B.GBCONV_OP_DGRAD, prob2)
    wsd2 = torch.empty(max(nd2, 1), dtype=torch.uint8, device=dev)

    def dgrad_s2(i, stream):
        B.check(B.conv2d_dgrad(prob2, g2b.data_ptr(), w2b.data_ptr(), dx2.data_ptr(),
                               wsd2.data_ptr(), nd2, stream), "dgrad s2")

    def dgrad_s2_noalloc(i, stream):
        B.check(B.conv2d_dgrad_noalloc(prob2, g2b.data_ptr(), w2b.data_ptr(), dx2.data_ptr(),
                                       stream), "dgrad s2 (static scratch)")

    steps = max(3, min(args.steps, 20))
    res = bench_layers([L(dgrad), L(wgrad), L(dgrad_s2), L(dgrad_s2_noalloc)], steps, 3, 1,
                       torch, dist_on)
    # the CUDA-core gather kernel on the same strided layer, by its stored config
    B.check(B.gbconv_set_config(B.GBCONV_OP_DGRAD, prob2,
                                B.gbconv_config_t(0, 0, 0, 0, B.GBCONV_ALGO_SIMT)), "set_config")
    try:
        res_cc = bench_layers([L(dgrad_s2)], max(3, min(args.steps, 5)), 3, 1, torch, dist_on)
    finally:
        B.check(B.gbconv_set_config(B.GBCONV_OP_DGRAD, prob2,
                                    B.gbconv_config_t(0, 0, 0, 0, B.GBCONV_ALGO_AUTO)), "set_config")
    cc_us = res_cc["launch_us"][0]
    # the weight gradient on the band kernel (one unit per filter row: dy and
    # one x band per row, a third of the per-tap kernel's shared-memory ingest)
    split_tap = B.gbconv_get_config(B.GBCONV_OP_WGRAD, prob)[1].split_k
    B.check(B.gbconv_set_config(B.GBCONV_OP_WGRAD, prob,
                                B.gbconv_config_t(0, 0, 0, 0, B.GBCONV_ALGO_SHIFT)), "set_config")
    try:
        _, nwb = B.gbconv_workspace_size(B.GBCONV_OP_WGRAD, prob)
        wsb = torch.empty(max(nwb, 1), dtype=torch.uint8, device=dev)

        def wgrad_band(i, stream):
            B.check(B.conv2d_wgrad(prob, xb.data_ptr(), gb.data_ptr(), dw.data_ptr(), db.data_ptr(),
                                   wsb.data_ptr(), nwb, stream), "wgrad band")
        res_band = bench_layers([L(wgrad_band)], steps, 3, 1, torch, dist_on)
        split_band = B.gbconv_get_config(B.GBCONV_OP_WGRAD, prob)[1].split_k
    finally:
        B.gbconv_shutdown()  # back to the default weight-gradient config
        del wsb
    band_us = res_band["launch_us"][0]
    # algorithmic shared-memory ingest of the two kernels (dy and x, BF16):
    # per tap (R*S = 9 loads of each) vs per filter row (3 loads of each, over
    # Wx = 57 positions per 56-wide row)
    m_bytes = sh.N * sh.H * sh.W * sh.C * 2
    f = sh.flops
    f2 = s2.flops
    return {"workload": sh.tag, "dgrad_us": round(res["launch_us"][0], 1),
            "wgrad_us": round(res["launch_us"][1], 1),
            "dgrad_tflops": round(f / (res["launch_us"][0] * 1e-6) / 1e12, 1),
            "wgrad_tflops": round(f / (res["launch_us"][1] * 1e-6) / 1e12, 1),
            "wgrad_split_k": split_tap,
            "wgrad_band": {"us": round(band_us, 1),
                           "tflops": round(f / (band_us * 1e-6) / 1e12, 1),
                           "split_k": split_band,
                           "smem_ingest_mb": round(3 * 2 * m_bytes * 57 / 56 / 1e6, 1),
                           "per_tap_smem_ingest_mb": round(9 * 2 * m_bytes / 1e6, 1)},
            "dgrad_stride2": {"workload": "dgrad_" + s2.tag,
                              "subpixel_tc_us": round(res["launch_us"][2], 1),
                              "subpixel_tc_tflops": round(f2 / (res["launch_us"][2] * 1e-6) / 1e12, 1),
                              "subpixel_tc_static_scratch_us": round(res["launch_us"][3], 1),
                              "cuda_core_us": round(cc_us, 1),
                              "cuda_core_tflops": round(f2 / (cc_us * 1e-6) / 1e12, 2)}}


def bench_fused(torch, dev, args, dist_on, pk):
    """End of a ResNet-50 bottleneck block (1x1 64 -> 256 at 56x56, batch 32):
    convolution, inference batch norm, identity-shortcut add and ReLU. Fused:
    one conv2d_fwd_fused launch with the folded (scale, shift) and the
    shortcut as residual. Unfused: the plain forward followed by the same
    epilogue as PyTorch elementwise operations (reference point only)."""
    from paper_2207_00257_gb300 import binding as B
    from paper_2207_00257_gb300 import functional as F
    from paper_2207_00257_gb300.synth import make_inputs, resnet_layers
    sh = resnet_layers(32)[2]
    x, w, b, _ = make_inputs(sh, 7)
    g = torch.Generator().manual_seed(8)
    xb, wb = x.bfloat16().to(dev), w.bfloat16().to(dev)
    gamma = (torch.rand(sh.K, generator=g) + 0.5).to(dev)
    beta, mean = torch.randn(sh.K, generator=g).to(dev), (0.1 * torch.randn(sh.K, generator=g)).to(dev)
    var = (torch.rand(sh.K, generator=g) + 0.5).to(dev)
    scale, shift = F.bn_fold(gamma, beta, mean, var, 1e-5, bias=b.to(dev))
    z = torch.randn(sh.y_shape(), generator=g).bfloat16().to(dev)
    y = torch.empty(sh.y_shape(), dtype=torch.bfloat16, device=dev)
    y2 = torch.empty_like(y)
    prob = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                     B.GBCONV_BF16, B.GBCONV_BF16, B.GBCONV_NHWC, B.GBCONV_FLAG_BIAS |
                     B.GBCONV_FLAG_RELU)
    prob0 = B.problem(sh.N, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                      B.GBCONV_BF16, B.GBCONV_BF16, B.GBCONV_NHWC, 0)
    sc4 = scale.view(1, 1, 1, -1)
    sh4 = shift.view(1, 1, 1, -1)

    def fused(i, stream):
        B.check(B.conv2d_fwd_fused(prob, xb.data_ptr(), wb.data_ptr(), shift.data_ptr(),
                                   scale.data_ptr(), z.data_ptr(), 0, 0, y.data_ptr(), 0, 0,
                                   stream), "fused")

    def unfused(i, stream):
        B.check(B.conv2d_fwd(prob0, xb.data_ptr(), wb.data_ptr(), 0, 0, 0, y2.data_ptr(), 0, 0,
                             stream), "conv")
        s = torch.cuda.ExternalStream(stream)
        with torch.cuda.stream(s):
            torch.relu_(y2.float().mul_(sc4).add_(sh4).add_(z.float())).to(torch.bfloat16)

    class L:
        def __init__(s, f):
            s.launch = f

    steps = max(3, min(args.steps, 20))
    res = bench_layers([L(fused), L(unfused)], steps, 3, 1, torch, dist_on)
    rb = bench_layers([L(fused)], max(3, min(args.steps, 50)), 1, 1, torch, dist_on)
    ub = rb["ms_per_step"] * 1e3
    nbytes = (xb.numel() + wb.numel() + z.numel() + y.numel()) * 2
    f = sh.flops
    return {"workload": "bottleneck_end_" + sh.tag + "_bn_residual_relu",
            "fused_us": round(res["launch_us"][0], 1),
            "fused_us_back_to_back": round(ub, 2),
            "fused_frac_of_hbm_back_to_back": round(nbytes / (ub * 1e-6) / 1e9 / pk["hbm_gbs"], 3),
            "fused_tflops": round(f / (res["launch_us"][0] * 1e-6) / 1e12, 1),
            "unfused_conv_plus_torch_elementwise_us": round(res["launch_us"][1], 1),
            "bytes_fused_MB": round((xb.numel() + wb.numel() + z.numel() + y.numel()) * 2 / 1e6, 1)}


def bench_groups(torch, dev, args, dist_on, pk):
    """Channel-grouped layers, batch 32, BF16 NHWC: a depthwise 3x3 (G = C = K
    = 128 at 56x56, memory-bound: reported against HBM), a ResNeXt-style 3x3
    with 32 groups of 4 channels (C = K = 128 at 56x56, CUDA cores), and a
    two-group 3x3 (C = K = 256 at 28x28, tensor cores per group)."""
    from paper_2207_00257_gb300 import binding as B
    cases = [("depthwise_3x3_128ch_56", 128, 56, 128, 128),
             ("resnext_3x3_32x4ch_56", 128, 56, 128, 32),
             ("two_groups_3x3_256ch_28", 256, 28, 256, 2)]
    layers, meta = [], []
    g = torch.Generator().manual_seed(9)
    for tag, C, HW, K, G in cases:
        x = torch.randn(32, HW, HW, C, generator=g).bfloat16().to(dev)
        w = (torch.randn(K, 3, 3, C // G, generator=g) / (3 * (C // G) ** 0.5)).bfloat16().to(dev)
        b = (torch.rand(K, generator=g) * 0.2 - 0.1).to(dev)
        y = torch.empty(32, HW, HW, K, dtype=torch.bfloat16, device=dev)
        prob = B.problem(32, C, HW, HW, K, 3, 3, 1, 1, 1, B.GBCONV_BF16, B.GBCONV_BF16,
                         B.GBCONV_NHWC, B.GBCONV_FLAG_BIAS | B.GBCONV_FLAG_RELU, G)

        def launch(i, stream, prob=prob, x=x, w=w, b=b, y=y):
            B.check(B.conv2d_fwd(prob, x.data_ptr(), w.data_ptr(), b.data_ptr(), 0, 0,
                                 y.data_ptr(), 0, 0, stream), "grouped-channel conv")

        class L:
            pass
        lay = L()
        lay.launch = launch
        layers.append(lay)
        flops = 2 * 32 * K * HW * HW * (C // G) * 9
        nbytes = (x.numel() + y.numel()) * 2 + w.numel() * 2 + K * 4
        meta.append((tag, G, flops, nbytes))
    steps = max(3, min(args.steps, 20))
    res = bench_layers(layers, steps, 3, 1, torch, dist_on)
    out = []
    for lay, (tag, G, flops, nbytes), us in zip(layers, meta, res["launch_us"]):
        # back to back (K launches of this layer alone in one graph, each
        # overlapping its neighbours' launch and ramp), as the headline layers
        r1 = bench_layers([lay], max(3, min(args.steps, 50)), 1, 1, torch, dist_on)
        ub = r1["ms_per_step"] * 1e3
        out.append({"workload": tag, "groups": G, "us_event_separated": round(us, 1),
                    "us_back_to_back": round(ub, 2),
                    "tflops": round(flops / (ub * 1e-6) / 1e12, 2),
                    "gbs": round(nbytes / (ub * 1e-6) / 1e9, 1),
                    "frac_of_hbm": round(nbytes / (ub * 1e-6) / 1e9 / pk["hbm_gbs"], 3),
                    "frac_of_hbm_event_separated": round(nbytes / (us * 1e-6) / 1e9 / pk["hbm_gbs"], 3)})
    return out


def bench_nll(torch, dev, args, dist_on, pk):
    """Negative log-likelihood loss after a 1000-class classifier: forward
    (two-pass reduction) and gradient, batch 32 (the ResNet-50 workload) and
    a 65536-row batch (memory-bound: [N][C] read once, written once)."""
    from paper_2207_00257_gb300 import binding as B
    out = []
    for N in (32, 65536):
        C = 1000
        g = torch.Generator().manual_seed(10)
        logp = torch.log_softmax(torch.randn(N, C, generator=g), dim=1).to(dev)
        t = torch.randint(0, C, (N,), generator=g).to(dev)
        o = torch.empty(1, device=dev)
        tw = torch.empty(1, device=dev)
        go = torch.ones(1, device=dev)
        gi = torch.empty(N, C, device=dev)
        _, nb = B.gbconv_nll_workspace_size(N)
        ws = torch.empty(max(nb, 4), dtype=torch.uint8, device=dev)

        def fwd(i, stream, logp=logp, t=t, o=o, tw=tw, ws=ws, nb=nb, N=N):
            B.check(B.gbconv_nll_loss_fwd(logp.data_ptr(), t.data_ptr(), 0, N, C, -100, 1,
                                          o.data_ptr(), tw.data_ptr(), ws.data_ptr(), nb, stream),
                    "nll fwd")

        def bwd(i, stream, t=t, tw=tw, go=go, gi=gi, N=N):
            B.check(B.gbconv_nll_loss_bwd(go.data_ptr(), t.data_ptr(), 0, N, C, -100, 1,
                                          tw.data_ptr(), gi.data_ptr(), stream), "nll bwd")

        class L:
            def __init__(s, f):
                s.launch = f
        res = bench_layers([L(fwd), L(bwd)], max(3, min(args.steps, 20)), 3, 1, torch, dist_on)
        out.append({"N": N, "C": C, "fwd_us": round(res["launch_us"][0], 2),
                    "bwd_us": round(res["launch_us"][1], 2),
                    "bwd_gbs": round(N * C * 4 / (res["launch_us"][1] * 1e-6) / 1e9, 1)})
    return out


# ---------------------------------------------------------------------------
# the FP64 CPU oracle: cpu_baseline leg and the reference arm
# ---------------------------------------------------------------------------
def oracle_sample_run(images, nthreads=0):
    """Runs the oracle on the first `images` images of each ResNet layer
    (seeded inputs of the bench's buffer set 0). Returns (seconds, flops, outputs)."""
    import numpy as np
    import torch
    import oracle
    from paper_2207_00257_gb300.synth import make_inputs, resnet_layers
    outs, secs, flops = [], 0.0, 0
    for i, sh in enumerate(resnet_layers(32)):
        x, w, b, _ = make_inputs(sh, 100 + i)
        xs = x[:images].bfloat16().double().numpy()
        wd = w.bfloat16().double().numpy()
        p = oracle.Conv(images, sh.C, sh.H, sh.W, sh.K, sh.R, sh.S, sh.stride, sh.pad, sh.dil,
                        "NHWC")
        t = time.perf_counter()
        y, bound = oracle.conv2d_fwd(p, xs, wd, b.double().numpy(), relu=True,
                                     nthreads=nthreads, with_bound=True)
        secs += time.perf_counter() - t
        flops += p.flops
        outs.append((y, bound))
    return secs, flops, outs


def cpu_baseline(layers, torch):
    import numpy as np
    import oracle
    images = int(os.environ.get("GBCONV_CPU_SAMPLE_IMAGES", "32"))
    secs, flops, outs = oracle_sample_run(images)
    errs = {}
    # refresh the outputs of buffer set 0 (the oracle's inputs) and compare
    stream = torch.cuda.current_stream().cuda_stream
    for lay in layers:
        lay.launch(0, stream)
    torch.cuda.synchronize()
    for lay, (y, bound) in zip(layers, outs):
        got = lay.ys[0][:images].double().cpu().numpy()
        errs[lay.sh.tag] = float(f"{oracle.max_normalised_error(got, y, bound):.3e}")
    return {"value": round(flops / secs / 1e12, 6), "unit": "TFLOP/s", "cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"first {images} of 32 images of each of the 4 layers "
                      f"({flops / 1e9:.2f} GFLOP, FP64 six-loop, all host threads)",
            "seconds": round(secs, 2),
            "max_normalised_err_bf16_vs_oracle": errs}


def run_reference(args, rank, world):
    if rank != 0:
        return
    images = 1
    for _ in range(args.warmup):
        oracle_sample_run(images)
    secs, flops = 0.0, 0
    for _ in range(args.steps):
        s, f, _ = oracle_sample_run(images)
        secs += s
        flops += f
    value = flops / secs / 1e12
    out = {"impl": "reference", "metric": "conv2d TFLOP/s & % of tensor peak, BF16/FP8 vs FP32 at stated rel err",
           "value": round(value, 6), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": "resnet50_bottleneck_layers_bf16_nhwc_batch32",
                                           "sample_per_step": f"{images} of 32 images per layer"},
           "cpu_baseline": {"value": round(value, 6), "unit": "TFLOP/s", "cores": os.cpu_count(),
                            "kind": "oracle",
                            "sample": f"first {images} image(s) of each of the 4 layers per step"},
           "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
