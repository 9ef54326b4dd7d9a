"""Benchmark: Gaussian beam summation throughput on one GB300 (or N, as replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: the large open-plane case (point source 2 m above a ground plane
with reflection coefficient 0.9, 65,536 Fibonacci rays, <= 3 reflections,
1 km paths; 256 x 256 receivers at 1.5 m over [-500, 500]^2 m; six octave
bands 125-4000 Hz), synthetic and seeded.  One step is the whole path: fan +
FP64 trace + scan + compaction + segment prepass + beam summation + merge,
through the library's gbt_solve.  Metric: (receiver, segment, frequency)
evaluations per second.  L2 is flushed (256 MiB write) between timed steps
and excluded from the per-step CUDA-event times.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own
replica of the workload (weak scaling, no collective on the data path).
On the default workload the line also carries `forms` (rank 0, outside the
timed steps): the same step with the exact tile pre-cull; the 32-source
batch against one launch per source and per (source, frequency); the
differentiable city's forward, forward + backward and autograd training
step; the tracer alone for each nearest-hit search; the time synthesis of
the field into 2,048 samples.  `--workload` selects
another workload (open_plane_small, city, diff_city, big_city) and
`--tile-cull` times the pre-culled step as the main one.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GBS segment x receiver evals/s at <=1e-4 rel L2; batched & fwd+bwd vs plain"
UNIT = "evals/s"
# Algorithmic work of the method, in FP32/ALU lane issue slots:
# per tested (receiver, segment) pair about 20 (projection onto the segment, s, n^2, window,
# the frequency-independent cutoff); per kept (pair, frequency) about 45 FP32 slots for the
# beam term (1/E, Gaussian amplitude, phase with its range reduction, complex product) plus
# about 12 for the compensated accumulation, i.e. 57, and 4 MUFU operations (RCP, EX2, SIN,
# COS) on the separate special-function pipe, whose time at 16-32 lanes per clock per SM
# stays below the FP32 time on every workload here (open plane: 7 %), so the FP32/ALU issue
# rate is the roofline.
OPS_PER_PAIR = 20
OPS_PER_KEPT = 57
LANES_PER_SM_CLK = 128          # FP32 lanes per SM per clock (4 SMSPs x 32)
KERNEL_TAG = "gbs_fwd_kernel<6,LINE,fwd,plain> warp-autonomous, paired survivors"
# DRAM bytes (read + write) per launch of the dominant kernel, from an ncu capture of this
# exact kernel version (profiles/gbs_fwd_open_plane_64k_rays_256x256_6f.md); a changed
# kernel gets a new tag and no entry until it is captured again.
KERNEL_TRAFFIC = {"gbs_fwd_kernel<6,LINE,fwd,plain> warp-autonomous, paired survivors": 194647296}


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


WORKLOADS = ("open_plane_large", "open_plane_small", "city", "diff_city", "big_city")


def _workload(name: str = "open_plane_large"):
    """The metric is quoted on open_plane_large (default); the others can be measured on
    request with --workload (the batched city is measured as a form)."""
    from paper_2501_13382_gb300 import inputs as I
    return {"open_plane_large": I.open_plane_large, "open_plane_small": I.open_plane_small,
            "city": I.city, "diff_city": I.diff_city, "big_city": I.big_city}[name]()


def _oracle_sample(w, budget_s: float, seed: int = 17):
    """Time the FP64 oracle (trace + sum) on a seeded receiver sample sized to ~budget_s."""
    from oracle import oracle as O
    from paper_2501_13382_gb300 import inputs as I
    src = w.sources[0]
    t0 = time.perf_counter()
    tr = O.trace(w.scene, src)
    t_trace = time.perf_counter() - t0
    n = 16
    while True:
        idx = I.receiver_subset(w.receivers, n, seed)
        t0 = time.perf_counter()
        p = O.gbs_sum(tr, w.receivers[idx], w.freqs, w.beam_b[0], w.scene.c, w.scene.gamma,
                      window=w.window, cutoff=w.cutoff)
        dt = time.perf_counter() - t0
        if dt >= budget_s * 0.3 or n >= w.receivers.shape[0]:
            break
        n = min(w.receivers.shape[0], int(n * max(2.0, budget_s * 0.5 / max(dt, 1e-3))))
    evals = float(len(idx)) * tr.n_seg * len(w.freqs)
    return {"idx": idx, "p": p, "evals": evals, "t_sum": dt, "t_trace": t_trace,
            "n_seg": tr.n_seg}


def aggregate_ranks(torch, ms, e2e_ms, evals, steps, world, dist=None, device="cuda"):
    """Whole-job rates over `world` replicas: the slowest rank's timed totals (max over ranks)
    and every rank's `evals` per step.  Returns (ms_per_step, value, e2e_value)."""
    if dist is not None:
        t = torch.tensor([ms, e2e_ms], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, e2e_ms = float(t[0]), float(t[1])
    ms_per_step = ms / steps
    return (ms_per_step, world * evals / (ms_per_step * 1e-3),
            world * evals / (e2e_ms / steps * 1e-3))


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the same workload and metric."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2501_13382_gb300 import inputs as I
    w = _workload(args.workload)
    n_sample = 48
    idx = I.receiver_subset(w.receivers, n_sample, 23)
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        tr = O.trace(w.scene, w.sources[0])
        O.gbs_sum(tr, w.receivers[idx], w.freqs, w.beam_b[0], w.scene.c, w.scene.gamma,
                  window=w.window, cutoff=w.cutoff)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    evals = float(n_sample) * tr.n_seg * len(w.freqs)
    sec = float(np.sum(times))
    value = evals * len(times) / sec
    cores = O.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "rays": w.sources[0].n_rays, "segments": tr.n_seg,
                       "receivers_per_step": n_sample, "freqs": len(w.freqs),
                       "parallelism": "cpu-openmp"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n_sample} seeded receivers of {w.receivers.shape[0]} "
                                       f"per step, full fan trace each step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _events(torch, n):
    return [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(n)]


def _timed(torch, stream, fn, steps, flush=None):
    """Sum of per-step CUDA-event times (flush between steps, outside the events)."""
    ev = _events(torch, steps)
    for i in range(steps):
        if flush is not None:
            flush.zero_()
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return float(sum(a.elapsed_time(b) for a, b in ev))


def bench_tile_cull(G, torch, stream, sc, w, recv, gam, order, out, flush, steps, n_seg):
    """The same open-plane step with the per-warp segment pre-cull (identical field)."""
    src = w.sources[0]
    freqs, bb = list(w.freqs), list(w.beam_b[0])

    def step():
        G.gbs_solve(sc, src, recv, freqs, bb, gam, order=order, window=w.window, cutoff=w.cutoff,
                    out=out, tile_cull=True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    G.gbt_timing_enable(True)
    G.gbt_timing_read(reset=True)
    ms = _timed(torch, stream, step, steps, flush)
    G.gbt_timing_enable(False)
    n_k, k_ms = G.gbt_timing_read(reset=True)
    tr = G.Trace(sc, src)
    st = G.sum_stats(tr, recv, freqs, bb, gam, order=order, window=w.window, cutoff=w.cutoff,
                     tile_cull=True)
    tr.close()
    evals = float(recv.shape[0]) * n_seg * len(freqs)
    return {"value": evals / (ms / steps * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
            "kernel_ms": k_ms / max(n_k, 1), "pairs_tested": st["pairs_tested"],
            "pairs": st["pairs"], "note": "same kept triples as testing every pair; field equal up to FP32 regrouping"}


def bench_batched(G, torch, stream, steps=5):
    """Batched city: 32 sources (log-uniform 4,096-262,144 rays), 8 frequencies, receivers
    128 x 128.  One graph-replayed batch submit (form chosen by the autotuner, and each form
    on its own) vs one gbt_sum launch per source (8 frequencies each) and vs one launch per
    (source, frequency)."""
    from paper_2501_13382_gb300 import inputs as I
    w = I.batched_city()
    recv_np = I.receiver_grid(128, 250.0, 1.5)
    sc = G.Scene(w.scene)
    gam = torch.as_tensor(w.scene.gamma, device="cuda")
    recv = torch.as_tensor(recv_np, device="cuda")
    order = G.recv_order(recv)
    insts, evals = [], 0.0
    for i, src in enumerate(w.sources):
        tr = G.Trace(sc, src)
        n_seg = tr.info().n_segments
        evals += float(recv.shape[0]) * n_seg * len(w.freqs)
        insts.append(dict(trace=tr, recv=recv, freqs=list(w.freqs), beam_b=list(w.beam_b[i]),
                          gamma=gam, order=order))
    outs = [torch.empty((len(w.freqs), recv.shape[0]), dtype=torch.complex64, device="cuda")
            for _ in insts]

    def plain():
        for d, o in zip(insts, outs):
            G.gbs_sum(d["trace"], recv, d["freqs"], d["beam_b"], gam, order=order,
                      window=w.window, out=o)

    outs_f = [torch.empty_like(o) for o in outs]

    def plain_per_frequency():
        for d, o in zip(insts, outs_f):
            for fi in range(len(d["freqs"])):
                G.gbs_sum(d["trace"], recv, [d["freqs"][fi]], [d["beam_b"][fi]], gam,
                          order=order, window=w.window, out=o[fi:fi + 1])
    plain_per_frequency()
    plain()
    torch.cuda.synchronize()
    t_p = _timed(torch, stream, plain, steps) / steps
    t_pf = _timed(torch, stream, plain_per_frequency, max(1, steps // 2)) / max(1, steps // 2)
    err_pf = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
                 for a, b in zip(outs_f, outs))
    forms = {}
    for name, form in (("auto", G.BATCH_AUTO), ("fused", G.BATCH_FUSED),
                       ("concurrent", G.BATCH_CONCURRENT)):
        batch = G.Batch(insts, window=w.window, use_graph=True, autotune=True, form=form)
        batch.submit()
        torch.cuda.synchronize()
        t_b = _timed(torch, stream, batch.submit, steps) / steps
        err = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
                  for a, b in zip(batch.outputs, outs))
        batch.close()
        forms[name] = {"value": evals / (t_b * 1e-3), "ms": t_b, "rel_l2_vs_plain": err}
    return {"workload": "batched_city_32src_8f_128x128", "evals": evals,
            "batched": forms["auto"], "fused_autotuned": forms["fused"],
            "concurrent": forms["concurrent"],
            "plain_per_instance": {"value": evals / (t_p * 1e-3), "ms": t_p},
            "plain_per_source_frequency": {"value": evals / (t_pf * 1e-3), "ms": t_pf,
                                           "launches_of_gbs_sum": len(insts) * len(w.freqs),
                                           "rel_l2_vs_plain": err_pf},
            "speedup": t_p / forms["auto"]["ms"],
            "speedup_vs_per_source_frequency": t_pf / forms["auto"]["ms"]}


def bench_fwd_bwd(G, torch, stream, steps=5):
    """Differentiable city: 262,144 rays, <= 6 reflections, 128 x 128 receivers, 4 frequencies;
    forward + backward (gradients for 9 reflection coefficients and 4 beam parameters) vs
    forward alone, and the training step of the workload (L2 loss against the seeded target
    field, through the torch.autograd.Function)."""
    from paper_2501_13382_gb300 import inputs as I
    w = I.diff_city()
    sc = G.Scene(w.scene)
    src = w.sources[0]
    tr = G.Trace(sc, src)
    n_seg = tr.info().n_segments
    recv = torch.as_tensor(w.receivers, device="cuda")
    order = G.recv_order(recv)
    gam = torch.as_tensor(w.scene.gamma, device="cuda")
    freqs, bb = list(w.freqs), list(w.beam_b[0])
    out = torch.empty((len(freqs), recv.shape[0]), dtype=torch.complex64, device="cuda")
    g = torch.ones_like(out)
    evals = float(recv.shape[0]) * n_seg * len(freqs)
    res = {"workload": w.name, "evals": evals}
    for name, cull in (("dense", False), ("tile_cull", True)):
        def fwd():
            G.gbs_sum(tr, recv, freqs, bb, gam, order=order, window=w.window, out=out,
                      tile_cull=cull)

        def fwd_bwd():
            fwd()
            G.gbs_sum_backward(tr, recv, freqs, bb, gam, g, order=order, window=w.window,
                               tile_cull=cull)
        fwd_bwd()
        torch.cuda.synchronize()
        t_f = _timed(torch, stream, fwd, steps) / steps
        t_fb = _timed(torch, stream, fwd_bwd, steps) / steps
        r = {"forward": {"value": evals / (t_f * 1e-3), "ms": t_f},
             "forward_backward": {"value": evals / (t_fb * 1e-3), "ms": t_fb},
             "backward_over_forward": (t_fb - t_f) / t_f}
        # the training step of the workload: L2 loss against the field of the seeded target
        # coefficients, forward and backward through the torch.autograd.Function
        from paper_2501_13382_gb300.autograd import gbs_field
        target = G.gbs_sum(tr, recv, freqs, bb,
                           torch.as_tensor(w.extra["target_gamma"], device="cuda"),
                           order=order, window=w.window)
        gam_p = torch.tensor(w.scene.gamma, device="cuda", requires_grad=True)

        def train_step():
            gam_p.grad = None
            p = gbs_field(tr, recv, freqs, bb, gam_p, order=order, window=w.window,
                          tile_cull=cull)
            (p - target).abs().pow(2).sum().backward()
        train_step()
        torch.cuda.synchronize()
        t_a = _timed(torch, stream, train_step, steps) / steps
        r["autograd_loss_step"] = {"value": evals / (t_a * 1e-3), "ms": t_a}
        if cull:
            res["tile_cull"] = r
        else:
            res.update(r)
    tr.close()
    return res


def bench_trace(G, torch, stream, steps=5):
    """The tracer alone (fan, nearest hits, reflections, scan and compaction into the
    segment list) for each nearest-hit search: the synthetic city (768 triangles, kept in
    shared memory, 1,048,576 rays) and the large city (12,288 triangles, 262,144 rays)."""
    from paper_2501_13382_gb300 import inputs as I
    res = {}
    for name, w in (("city_768_tris_1M_rays", I.city()),
                    ("big_city_12k_tris_256k_rays", I.big_city())):
        src = w.sources[0]
        r = {"triangles": int(w.scene.n_tri), "rays": int(src.n_rays)}
        accels = [("auto", G.ACCEL_AUTO), ("bvh", G.ACCEL_BVH), ("linear", G.ACCEL_LINEAR)]
        for an, a in accels:
            sc = G.Scene(w.scene, accel=a)
            t = G.Trace(sc, src)
            n_seg = int(t.info().n_segments)
            t.close()
            ev = _events(torch, steps)
            for i in range(steps):
                ev[i][0].record(stream)
                t = G.Trace(sc, src)
                ev[i][1].record(stream)
                t.close()
            ms = float(np.median([a0.elapsed_time(b0) for a0, b0 in ev]))
            r[an] = {"ms": ms, "rays_per_s": src.n_rays / (ms * 1e-3), "segments": n_seg}
            sc.close()
        res[name] = r
    return res


def bench_synthesis(G, torch, stream, field, freqs, steps=5):
    """Time synthesis of the open-plane field (6 bands x 65,536 receivers) into 2,048
    samples at 16 kHz: the kernel writes 2,048 x 65,536 floats, so it is bound by HBM."""
    n_t, dt = 2048, 1.0 / 16000.0
    out = torch.empty((n_t, field.shape[1]), dtype=torch.float32, device="cuda")
    amp = [1.0] * len(freqs)

    def step():
        G.synthesize(field, list(freqs), amp, 0.0, dt, n_t, out=out)
    step()
    torch.cuda.synchronize()
    ms = _timed(torch, stream, step, steps) / steps
    bytes_out = out.numel() * 4
    peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f).get("hbm_gbs"))
    except Exception:
        pass
    gbs = bytes_out / (ms * 1e-3) / 1e9
    return {"samples": n_t, "receivers": int(field.shape[1]), "freqs": len(freqs), "ms": ms,
            "output_GB_per_s": gbs, "hbm_peak_GB_per_s": peak,
            "frac": (gbs / peak) if peak else None,
            "note": "ms includes forming the FP64 phasors on the host and their upload"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of oracle work for the CPU baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end loop")
    ap.add_argument("--workload", default="open_plane_large", choices=WORKLOADS)
    ap.add_argument("--tile-cull", action="store_true",
                    help="time the tile-cull variant as the main step")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the tile-cull, batched and forward+backward forms")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2501_13382_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if dist:
        dist.barrier()
    from paper_2501_13382_gb300 import gbt as G

    w = _workload(args.workload)
    src = w.sources[0]
    stream = torch.cuda.current_stream()
    sc = G.Scene(w.scene)
    recv = torch.as_tensor(w.receivers, device="cuda")
    gam = torch.as_tensor(w.scene.gamma, device="cuda")
    freqs = list(w.freqs)
    bb = list(w.beam_b[0])
    order = G.recv_order(recv)
    out = torch.empty((len(freqs), recv.shape[0]), dtype=torch.complex64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # work statistics (outside the timed region)
    tr = G.Trace(sc, src)
    st = G.sum_stats(tr, recv, freqs, bb, gam, order=order, window=w.window, cutoff=w.cutoff,
                     tile_cull=args.tile_cull)
    n_seg = st["n_segments"]
    tr.close()
    evals = float(recv.shape[0]) * n_seg * len(freqs)

    def step():
        G.gbs_solve(sc, src, recv, freqs, bb, gam, order=order, window=w.window,
                    cutoff=w.cutoff, out=out, tile_cull=args.tile_cull)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    time.sleep(0.3)
    G.gbt_timing_enable(True)
    G.gbt_timing_read(reset=True)
    G.gbt_launches_read(reset=True)
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    launches = G.gbt_launches_read(reset=True)
    G.gbt_timing_enable(False)
    n_k, k_ms = G.gbt_timing_read(reset=True)
    ms = float(sum(a.elapsed_time(b) for a, b in ev))
    # e2e: host receivers in, host field out, through the public API each step
    host_recv = torch.as_tensor(w.receivers).pin_memory()
    host_out = torch.empty(out.shape, dtype=torch.complex64).pin_memory()
    recv_e = torch.empty_like(recv)

    def step_e2e():
        recv_e.copy_(host_recv, non_blocking=True)
        o = G.recv_order(recv_e)
        G.gbs_solve(sc, src, recv_e, freqs, bb, gam, order=o, window=w.window,
                    cutoff=w.cutoff, out=out, tile_cull=args.tile_cull)
        host_out.copy_(out, non_blocking=True)

    e2e_ms = float("nan")
    if not args.no_e2e:
        for _ in range(2):
            step_e2e()
        torch.cuda.synchronize()
        e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
        for i in range(args.steps):
            flush.zero_()
            e2e_ev[i][0].record(stream)
            step_e2e()
            e2e_ev[i][1].record(stream)
        torch.cuda.synchronize()
        e2e_ms = float(sum(a.elapsed_time(b) for a, b in e2e_ev))
    clk.stop()
    G.gbt_sync()

    ms_per_step, value, e2e_value = aggregate_ranks(torch, ms, e2e_ms, evals, args.steps, world,
                                                    dist)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    clocks = clk.summary()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    kern_ms = k_ms / max(n_k, 1)
    ops = OPS_PER_PAIR * float(st["pairs_tested"]) + OPS_PER_KEPT * float(st["triples_kept"])
    achieved = ops / (kern_ms * 1e-3) / 1e12
    mhz = clocks["sm_mhz"] or 1492.0
    peak = n_sm * LANES_PER_SM_CLK * mhz * 1e6 / 1e12
    tag = KERNEL_TAG if (args.workload == "open_plane_large" and not args.tile_cull) else None
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-op/s",
                "frac": achieved / peak, "traffic": KERNEL_TRAFFIC.get(tag),
                "kernel": KERNEL_TAG, "kernel_ms": kern_ms, "kernel_launches": n_k,
                "ops_per_launch": ops,
                "peak_basis": f"{n_sm} SMs x {LANES_PER_SM_CLK} lanes x median SM clock "
                              f"{mhz:.0f} MHz under load"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "rays": src.n_rays, "segments": n_seg,
                       "receivers": int(recv.shape[0]), "freqs": len(freqs),
                       "pairs": st["pairs"], "pairs_prefiltered": st["pairs_prefiltered"],
                       "triples_kept": st["triples_kept"], "pairs_tested": st["pairs_tested"],
                       "tile_cull": bool(args.tile_cull), "l2": "flushed between steps (256 MiB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(recv.numel() * 4),
                    "d2h_bytes_per_step": int(out.numel() * 8)},
            "gpu_launches": launches,
            "clocks": clocks}

    if not args.no_forms and args.workload == "open_plane_large" and not args.tile_cull:
        line["forms"] = {
            "tile_cull": bench_tile_cull(G, torch, stream, sc, w, recv, gam, order, out, flush,
                                         min(args.steps, 50), n_seg),
            "batched": bench_batched(G, torch, stream),
            "fwd_bwd": bench_fwd_bwd(G, torch, stream),
            "trace": bench_trace(G, torch, stream),
            "synthesis": bench_synthesis(G, torch, stream, out, w.freqs),
        }
        # the forms overwrite `out`; recompute the measured workload's field for the check
        G.gbs_solve(sc, src, recv, list(w.freqs), list(w.beam_b[0]), gam, order=order,
                    window=w.window, cutoff=w.cutoff, out=out)
        torch.cuda.synchronize()

    if world == 1 and not args.no_cpu:
        # CPU baseline + accuracy check of this run's field on the oracle's sample
        samp = _oracle_sample(w, args.cpu_budget)
        from oracle import oracle as O
        pg = out.cpu().numpy().astype(np.complex128)[:, samp["idx"]]
        err = float(np.linalg.norm(pg - samp["p"]) / np.linalg.norm(samp["p"]))
        cpu_value = samp["evals"] / (samp["t_sum"] + samp["t_trace"])
        line["cpu_baseline"] = {"value": cpu_value, "unit": UNIT, "cores": O.num_threads(),
                                "kind": "oracle",
                                "sample": f"{len(samp['idx'])} seeded receivers x {samp['n_seg']} "
                                          f"segments x {len(freqs)} freqs, FP64 trace + sum"}
        line["accuracy"] = {"rel_l2_vs_oracle": err, "receivers_checked": len(samp["idx"])}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
