"""Benchmark: Gaussian beam summation throughput on one GB300 (or N, as replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--cull tile|none]

Workload (default): the synthetic city, the largest single-GPU configuration -- a ground
plane plus 64 seeded box buildings (768 triangles, reflection coefficients U(0.7, 0.95)),
1,048,576 Fibonacci rays from (0, 0, 5) m, <= 8 reflections, 1 km paths; 512 x 512
receivers at 1.5 m over [-250, 250]^2 m; 1 kHz; synthetic and seeded.  One step is the
whole path through the library's gbt_solve: fan + FP64 trace (BVH) + scan + compaction +
segment prepass + the exact tile pre-cull (per-tile segment lists) + beam summation + merge.
Metric: (receiver, segment, frequency) evaluations per second, counting every pair of the
method (the pre-cull skips only pairs that provably contribute nothing).  L2 is flushed
(256 MiB write) between timed steps and excluded from the per-step CUDA-event times.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own replica of the
workload (weak scaling, no collective on the data path).  On the default workload the
line also carries `forms` (rank 0, outside the timed steps): the city testing every pair;
the large open plane (65,536 rays, 256^2 receivers, 6 bands) with and without the
pre-cull and on the all-FP64 GPU path; the small open plane; the 32-source batched city
at 512^2 receivers against one launch per source and per (source, frequency); the
differentiable city's forward, forward + backward and autograd training step; the city with
propagation losses; the tracer
alone; the time synthesis of a field into 2,048 samples.  The reference arm
(`--impl reference`) times the FP64 CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
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
# stays below the FP32 time on every workload here, so the FP32/ALU issue rate is the
# roofline.
OPS_PER_PAIR = 20
OPS_PER_KEPT = 57
LANES_PER_SM_CLK = 128          # FP32 lanes per SM per clock (4 SMSPs x 32)
# Revision of the pair kernel's source.  DRAM bytes (read + write) per launch of the
# dominant kernel come from an ncu capture of one revision, instantiation and workload;
# a changed kernel gets a new revision and no entry until it is captured again.
KERNEL_REV = "rev10"
KERNEL_TRAFFIC = {
    ("gbs_fwd_kernel<1,SEGMENT,fwd,plain> tile segment lists [rev10]",
     "city_1M_rays_512x512_1kHz"): 5284817920,
    ("gbs_fwd_kernel<1,SEGMENT,fwd,plain> every pair [rev10]",
     "city_1M_rays_512x512_1kHz"): 241523122432,
    ("gbs_fwd_kernel<6,LINE,fwd,plain> tile segment lists [rev10]",
     "open_plane_64k_rays_256x256_6f"): 468206080,
    ("gbs_fwd_kernel<6,LINE,fwd,plain> every pair [rev10]",
     "open_plane_64k_rays_256x256_6f"): 195008000,
}
WORKLOADS = ("city", "open_plane_large", "open_plane_small", "diff_city", "big_city")


def kernel_tag(nf: int, window: int, cull: bool) -> str:
    """Name of the pair-kernel instantiation a sum with nf frequencies launches."""
    inst = next((v for v in (1, 2, 4, 6, 8) if nf <= v), 8)
    win = "LINE" if window == 1 else "SEGMENT"
    return (f"gbs_fwd_kernel<{inst},{win},fwd,plain> "
            f"{'tile segment lists' if cull else 'every pair'} [{KERNEL_REV}]")


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


def _workload(name: str = "city", rays: int = 0, recv_side: int = 0):
    """A named workload; rays / recv_side resize the city (smaller cases for profiling)."""
    from paper_2501_13382_gb300 import inputs as I
    if name == "city" and (rays or recv_side):
        return I.city(rays or (1 << 20), recv_side or 512)
    return {"open_plane_large": I.open_plane_large, "open_plane_small": I.open_plane_small,
            "city": I.city, "diff_city": I.diff_city, "big_city": I.big_city}[name]()


def workload_config(w) -> dict:
    """The `config` object of both arms: what the workload is, independent of the arm."""
    src = w.sources[0]
    return {"workload": w.name, "triangles": int(w.scene.n_tri), "rays": int(src.n_rays),
            "max_reflections": int(src.max_reflections), "receivers": int(w.receivers.shape[0]),
            "freqs": int(len(w.freqs)), "window": "LINE" if w.window == 1 else "SEGMENT",
            "parallelism": "one replica per rank"}


def oracle_rate(w, budget_s: float, seed: int = 17, tr=None):
    """The FP64 oracle on the workload: one full trace, then the sum on a seeded receiver
    sample sized to about budget_s.  The sum's cost is exactly linear in the receivers, so
    the whole workload's time is t_trace + t_sum * N / n; returns that rate and the
    sample's field (for the accuracy check)."""
    from oracle import oracle as O
    from paper_2501_13382_gb300 import inputs as I
    src = w.sources[0]
    t_trace = 0.0
    if tr is None:
        t0 = time.perf_counter()
        tr = O.trace(w.scene, src)
        t_trace = time.perf_counter() - t0
    nr = int(w.receivers.shape[0])
    n = min(nr, 32 * O.num_threads())   # OpenMP: chunks of 16 receivers; keep every core busy
    while True:
        idx = I.receiver_subset(w.receivers, n, seed)
        t0 = time.perf_counter()
        p = O.gbs_sum(tr, w.receivers[idx], w.freqs, w.beam_b[0], w.scene.c, w.scene.gamma,
                      window=w.window, cutoff=w.cutoff)
        dt = time.perf_counter() - t0
        if dt >= budget_s * 0.3 or n >= nr:
            break
        n = min(nr, int(n * min(64.0, max(2.0, budget_s * 0.5 / max(dt, 1e-3)))))
    evals_total = float(nr) * tr.n_seg * len(w.freqs)
    t_whole = t_trace + dt * nr / len(idx)
    return {"idx": idx, "p": p, "tr": tr, "n_seg": tr.n_seg, "t_trace": t_trace, "t_sum": dt,
            "value": evals_total / t_whole, "t_whole": t_whole}


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
    """Reference arm: the FP64 CPU oracle as it stands, on the same workload and metric.
    The fan is traced once; each step sums a seeded receiver sample (the cost of the sum is
    exactly linear in the receivers), and the whole workload's time per step is the trace
    plus the sample's time scaled to every receiver."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return None
    from oracle import oracle as O
    from paper_2501_13382_gb300 import inputs as I
    w = _workload(args.workload, getattr(args, "rays", 0), getattr(args, "recv_side", 0))
    src = w.sources[0]
    t0 = time.perf_counter()
    tr = O.trace(w.scene, src)
    t_trace = time.perf_counter() - t0
    nr = int(w.receivers.shape[0])
    # sample size: every core busy (OpenMP hands out receivers in chunks of 16), at least
    # 0.1 s per step
    n = min(nr, 32 * O.num_threads())
    while n < nr:
        idx = I.receiver_subset(w.receivers, n, 23)
        t0 = time.perf_counter()
        O.gbs_sum(tr, w.receivers[idx], w.freqs, w.beam_b[0], w.scene.c, w.scene.gamma,
                  window=w.window, cutoff=w.cutoff)
        dt = time.perf_counter() - t0
        if dt >= 0.1:
            break
        n = min(nr, n * 4)
    whole = []
    for step in range(args.warmup + args.steps):
        idx = I.receiver_subset(w.receivers, n, 23 + step)
        t0 = time.perf_counter()
        O.gbs_sum(tr, w.receivers[idx], w.freqs, w.beam_b[0], w.scene.c, w.scene.gamma,
                  window=w.window, cutoff=w.cutoff)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            whole.append(t_trace + dt * nr / len(idx))
    evals = float(nr) * tr.n_seg * len(w.freqs)
    t_step = float(np.mean(whole))
    value = evals / t_step
    cores = O.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": getattr(args, "gpus", 1), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w),
            "work": {"segments": int(tr.n_seg), "evals_per_step": evals},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"fan traced once ({t_trace:.2f} s, {tr.n_seg} segments); "
                                       f"each step sums {n} seeded receivers of {nr}, and the "
                                       f"step's time is the trace plus that sum scaled to all "
                                       f"{nr} receivers"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return None


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


def _peak_tlane(torch, mhz):
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return n_sm * LANES_PER_SM_CLK * mhz * 1e6 / 1e12, n_sm


def roofline_of(torch, st, kern_ms, n_launch, tag, workload, mhz):
    """FP32/ALU roofline of the pair kernel: the algorithmic lane operations of one launch
    (from the counting pass) over its CUDA-event duration."""
    ops = OPS_PER_PAIR * float(st["pairs_tested"]) + OPS_PER_KEPT * float(st["triples_kept"])
    peak, n_sm = _peak_tlane(torch, mhz)
    achieved = ops / (kern_ms * 1e-3) / 1e12 if kern_ms > 0 else 0.0
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-op/s",
            "frac": achieved / peak, "traffic": KERNEL_TRAFFIC.get((tag, workload)),
            "kernel": tag, "kernel_ms": kern_ms, "kernel_launches": n_launch,
            "ops_per_launch": ops,
            "peak_basis": f"{n_sm} SMs x {LANES_PER_SM_CLK} lanes x median SM clock "
                          f"{mhz:.0f} MHz under load"}


class Problem:
    """A workload's device state: scene, receivers, order, reflection coefficients, output."""

    def __init__(self, G, torch, w):
        self.w = w
        self.src = w.sources[0]
        self.sc = G.Scene(w.scene)
        self.recv = torch.as_tensor(w.receivers, device="cuda")
        self.gam = torch.as_tensor(w.scene.gamma, device="cuda")
        self.freqs = list(w.freqs)
        self.bb = list(w.beam_b[0])
        self.order = G.recv_order(self.recv)
        self.out = torch.empty((len(self.freqs), self.recv.shape[0]), dtype=torch.complex64,
                               device="cuda")

    def stats(self, G, cull):
        tr = G.Trace(self.sc, self.src)
        st = G.sum_stats(tr, self.recv, self.freqs, self.bb, self.gam, order=self.order,
                         window=self.w.window, cutoff=self.w.cutoff, tile_cull=cull)
        tr.close()
        return st

    def solve(self, G, cull, recv=None, order=None):
        G.gbs_solve(self.sc, self.src, self.recv if recv is None else recv, self.freqs, self.bb,
                    self.gam, order=self.order if order is None else order,
                    window=self.w.window, cutoff=self.w.cutoff, out=self.out, tile_cull=cull)


def time_solve(G, torch, stream, pb, cull, steps, flush, warmup=2):
    """Per-step time of the whole path (trace + sum) and the pair kernel's own time."""
    for _ in range(warmup):
        pb.solve(G, cull)
    torch.cuda.synchronize()
    G.gbt_timing_enable(True)
    G.gbt_timing_read(reset=True)
    ms = _timed(torch, stream, lambda: pb.solve(G, cull), steps, flush)
    G.gbt_timing_enable(False)
    n_k, k_ms = G.gbt_timing_read(reset=True)
    return ms / steps, k_ms / max(n_k, 1)


def bench_solve_form(G, torch, stream, w, cull, steps, flush, mhz, st=None):
    """One workload's step (trace + sum through gbt_solve) with its pair-kernel roofline."""
    pb = Problem(G, torch, w)
    st = st or pb.stats(G, cull)
    evals = float(pb.recv.shape[0]) * st["n_segments"] * len(pb.freqs)
    ms, kms = time_solve(G, torch, stream, pb, cull, steps, flush)
    tag = kernel_tag(len(pb.freqs), w.window, cull)
    return {"workload": w.name, "tile_cull": bool(cull), "value": evals / (ms * 1e-3),
            "unit": UNIT, "ms_per_step": ms, "steps": steps,
            "work": {"segments": st["n_segments"], "pairs": st["pairs"],
                     "pairs_tested": st["pairs_tested"], "triples_kept": st["triples_kept"]},
            "roofline": roofline_of(torch, st, kms, steps, tag, w.name, mhz)}


def bench_losses(G, torch, stream, w, steps, flush, mhz):
    """The city step with propagation losses: the paper's atmosphere (20 C, 70 %, 1 atm;
    ISO 9613-1 absorption) and a porous ground (200 kPa s m^-2, Delany-Bazley) under hard
    buildings, with the pre-cull; against the lossless step and the oracle on a sample."""
    from oracle import oracle as O
    from paper_2501_13382_gb300 import inputs as I
    pb = Problem(G, torch, w)
    absorb = list(G.air_absorption(pb.freqs, 20.0, 70.0, 101.325))
    sigma = np.full(w.scene.n_materials, -10.0, np.float32)
    sigma[0] = 200.0
    sg = torch.as_tensor(sigma, device="cuda")

    def step():
        G.gbs_solve(pb.sc, pb.src, pb.recv, pb.freqs, pb.bb, pb.gam, order=pb.order,
                    window=w.window, cutoff=w.cutoff, out=pb.out, tile_cull=True,
                    absorption=absorb, flow_resistivity=sg)
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    G.gbt_timing_enable(True)
    G.gbt_timing_read(reset=True)
    ms = _timed(torch, stream, step, steps, flush) / steps
    G.gbt_timing_enable(False)
    n_k, k_ms = G.gbt_timing_read(reset=True)
    st = pb.stats(G, True)
    evals = float(pb.recv.shape[0]) * st["n_segments"] * len(pb.freqs)
    idx = I.receiver_subset(w.receivers, 256, 31)
    otr = O.trace(w.scene, pb.src)
    po = O.gbs_sum(otr, w.receivers[idx], w.freqs, w.beam_b[0], w.scene.c, w.scene.gamma,
                   window=w.window, cutoff=w.cutoff, absorption=absorb,
                   sigma=sigma.astype(np.float64), scene=w.scene)
    pg = pb.out.cpu().numpy().astype(np.complex128)[:, idx]
    tag = kernel_tag(len(pb.freqs), w.window, True).replace(",fwd,", ",fwd+losses,")
    return {"workload": w.name, "atmosphere": "20 C, 70 %, 101.325 kPa",
            "absorption_np_per_m": absorb, "ground_flow_resistivity_kPa_s_m2": 200.0,
            "value": evals / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "rel_l2_vs_oracle": float(np.linalg.norm(pg - po) / np.linalg.norm(po)),
            "receivers_checked": int(len(idx)),
            "roofline": roofline_of(torch, st, k_ms / max(n_k, 1), n_k, tag, w.name, mhz)}


def bench_f64(G, torch, stream, w, steps=2):
    """The all-FP64 GPU path (every step of the sum in FP64) against the FP32 path with
    float-float phase on the same trace, and both against the FP64 oracle on a sample."""
    from oracle import oracle as O
    from paper_2501_13382_gb300 import inputs as I
    pb = Problem(G, torch, w)
    tr = G.Trace(pb.sc, pb.src)
    n_seg = tr.info().n_segments
    evals = float(pb.recv.shape[0]) * n_seg * len(pb.freqs)
    res = {"workload": w.name, "evals": evals}
    fields = {}
    for name, prec in (("f32", G.PRECISION_F32), ("f64", G.PRECISION_F64)):
        out = torch.empty_like(pb.out)

        def step():
            G.gbs_sum(tr, pb.recv, pb.freqs, pb.bb, pb.gam, order=pb.order, window=w.window,
                      cutoff=w.cutoff, precision=prec, out=out)
        step()
        torch.cuda.synchronize()
        n = steps if prec == G.PRECISION_F64 else 10
        ms = _timed(torch, stream, step, n) / n
        fields[name] = out
        res[name] = {"value": evals / (ms * 1e-3), "unit": UNIT, "ms": ms}
    idx = I.receiver_subset(w.receivers, 512, 29)
    po = O.gbs_sum(O.trace(w.scene, pb.src), w.receivers[idx], w.freqs, w.beam_b[0], w.scene.c,
                   w.scene.gamma, window=w.window, cutoff=w.cutoff)
    for name, out in fields.items():
        pg = out.cpu().numpy().astype(np.complex128)[:, idx]
        res[name]["rel_l2_vs_oracle"] = float(np.linalg.norm(pg - po) / np.linalg.norm(po))
    res["receivers_checked"] = int(len(idx))
    res["f64_over_f32_time"] = res["f64"]["ms"] / res["f32"]["ms"]
    tr.close()
    return res


def bench_batched(G, torch, stream, steps=3, cull=True):
    """Batched city: 32 sources (log-uniform 4,096-262,144 rays), 8 frequencies, 512 x 512
    receivers, with the tile pre-cull.  One graph-replayed batch submit (form chosen by the
    autotuner, and each form on its own) vs one gbt_sum launch per source (8 frequencies
    each) and vs one launch per (source, frequency), the configuration's baseline."""
    from paper_2501_13382_gb300 import inputs as I
    w = I.batched_city()
    sc = G.Scene(w.scene)
    gam = torch.as_tensor(w.scene.gamma, device="cuda")
    recv = torch.as_tensor(w.receivers, device="cuda")
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
                      window=w.window, out=o, tile_cull=cull)

    outs_f = [torch.empty_like(o) for o in outs]

    def plain_per_frequency():
        for d, o in zip(insts, outs_f):
            for fi in range(len(d["freqs"])):
                G.gbs_sum(d["trace"], recv, [d["freqs"][fi]], [d["beam_b"][fi]], gam,
                          order=order, window=w.window, out=o[fi:fi + 1], tile_cull=cull)
    plain_per_frequency()
    plain()
    torch.cuda.synchronize()
    t_p = _timed(torch, stream, plain, steps) / steps
    t_pf = _timed(torch, stream, plain_per_frequency, 1)
    err_pf = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
                 for a, b in zip(outs_f, outs))
    forms = {}
    for name, form in (("auto", G.BATCH_AUTO), ("fused", G.BATCH_FUSED),
                       ("concurrent", G.BATCH_CONCURRENT)):
        batch = G.Batch(insts, window=w.window, use_graph=True, autotune=True, form=form,
                        tile_cull=cull)
        batch.submit()
        torch.cuda.synchronize()
        t_b = _timed(torch, stream, batch.submit, steps) / steps
        err = max(float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
                  for a, b in zip(batch.outputs, outs))
        batch.close()
        forms[name] = {"value": evals / (t_b * 1e-3), "ms": t_b, "rel_l2_vs_plain": err}
    for d in insts:
        d["trace"].close()
    return {"workload": w.name, "tile_cull": bool(cull), "evals": evals,
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
            torch.cuda.synchronize()
            ms = float(np.median([a0.elapsed_time(b0) for a0, b0 in ev]))
            r[an] = {"ms": ms, "rays_per_s": src.n_rays / (ms * 1e-3), "segments": n_seg}
            sc.close()
        res[name] = r
    return res


def bench_synthesis(G, torch, stream, steps=5):
    """Time synthesis of the large open plane's field (6 bands x 65,536 receivers) into
    2,048 samples at 16 kHz: the kernel writes 2,048 x 65,536 floats, so it is bound by
    writing them to HBM."""
    w = _workload("open_plane_large")
    pb = Problem(G, torch, w)
    pb.solve(G, True)
    field, freqs = pb.out, pb.freqs
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
            "note": "gbt_synthesize call (device phasor table + sum), CUDA events on its stream"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=12.0,
                    help="seconds of oracle summation for the CPU baseline")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end loop")
    ap.add_argument("--workload", default="city", choices=WORKLOADS)
    ap.add_argument("--cull", default="tile", choices=["tile", "none"],
                    help="tile: the exact tile pre-cull (default); none: test every pair")
    ap.add_argument("--rays", type=int, default=0,
                    help="city only: rays of the fan (default 1,048,576; smaller for profiling)")
    ap.add_argument("--recv-side", type=int, default=0,
                    help="city only: receivers per grid side (default 512)")
    ap.add_argument("--no-forms", action="store_true", help="skip the other forms")
    ap.add_argument("--forms", default="",
                    help="comma-separated subset of forms to run (default: all)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        run_reference(args)
        return
    cull = args.cull == "tile"

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

    w = _workload(args.workload, args.rays, args.recv_side)
    stream = torch.cuda.current_stream()
    pb = Problem(G, torch, w)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # work statistics (outside the timed region)
    st = pb.stats(G, cull)
    n_seg = st["n_segments"]
    evals = float(pb.recv.shape[0]) * n_seg * len(pb.freqs)

    for _ in range(args.warmup):
        pb.solve(G, cull)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    ev = _events(torch, args.steps)
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
        pb.solve(G, cull)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    launches = G.gbt_launches_read(reset=True)
    G.gbt_timing_enable(False)
    n_k, k_ms = G.gbt_timing_read(reset=True)
    ms = float(sum(a.elapsed_time(b) for a, b in ev))
    # e2e: host receivers in, host field out, through the public API each step
    host_recv = torch.as_tensor(w.receivers).pin_memory()
    host_out = torch.empty(pb.out.shape, dtype=torch.complex64).pin_memory()
    recv_e = torch.empty_like(pb.recv)

    def step_e2e():
        recv_e.copy_(host_recv, non_blocking=True)
        o = G.recv_order(recv_e)
        pb.solve(G, cull, recv=recv_e, order=o)
        host_out.copy_(pb.out, non_blocking=True)

    e2e_ms = float("nan")
    if not args.no_e2e:
        for _ in range(2):
            step_e2e()
        torch.cuda.synchronize()
        e2e_ms = _timed(torch, stream, step_e2e, args.steps, flush)
    clk.stop()
    G.gbt_sync()

    ms_per_step, value, e2e_value = aggregate_ranks(torch, ms, e2e_ms, evals, args.steps, world,
                                                    dist)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    clocks = clk.summary()
    mhz = clocks["sm_mhz"] or 1492.0
    tag = kernel_tag(len(pb.freqs), w.window, cull)
    roofline = roofline_of(torch, st, k_ms / max(n_k, 1), n_k, tag, w.name, mhz)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(w),
            "work": {"segments": n_seg, "evals_per_step": evals, "pairs": st["pairs"],
                     "pairs_prefiltered": st["pairs_prefiltered"],
                     "triples_kept": st["triples_kept"], "pairs_tested": st["pairs_tested"],
                     "tile_cull": cull},
            "timing": {"l2": "flushed between steps (256 MiB write), outside the step events"},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(pb.recv.numel() * 4),
                    "d2h_bytes_per_step": int(pb.out.numel() * 8)},
            "gpu_launches": launches,
            "clocks": clocks}

    wanted = set(f for f in args.forms.split(",") if f) or None

    def want(name):
        return wanted is None or name in wanted

    if (not args.no_forms and args.workload == "city" and cull and not args.rays
            and not args.recv_side):
        forms = {}
        if want("dense"):
            forms["dense"] = bench_solve_form(G, torch, stream, w, False, 3, flush, mhz)
        if want("losses"):
            forms["losses"] = bench_losses(G, torch, stream, w, 10, flush, mhz)
        if want("open_plane_large"):
            op = _workload("open_plane_large")
            forms["open_plane_large"] = {
                "tile_cull": bench_solve_form(G, torch, stream, op, True, 20, flush, mhz),
                "dense": bench_solve_form(G, torch, stream, op, False, 20, flush, mhz)}
        if want("f64"):
            forms["f64"] = bench_f64(G, torch, stream, _workload("open_plane_large"))
        if want("open_plane_small"):
            forms["open_plane_small"] = bench_solve_form(
                G, torch, stream, _workload("open_plane_small"), False, 50, flush, mhz)
        if want("batched"):
            forms["batched"] = bench_batched(G, torch, stream)
        if want("fwd_bwd"):
            forms["fwd_bwd"] = bench_fwd_bwd(G, torch, stream)
        if want("trace"):
            forms["trace"] = bench_trace(G, torch, stream)
        if want("synthesis"):
            forms["synthesis"] = bench_synthesis(G, torch, stream)
        line["forms"] = forms
        # the forms overwrite device state; recompute the measured workload's field
        pb.solve(G, cull)
        torch.cuda.synchronize()
    G.gbt_sync()

    if world == 1 and not args.no_cpu:
        # CPU baseline + accuracy check of this run's field on the oracle's sample
        from oracle import oracle as O
        samp = oracle_rate(w, args.cpu_budget)
        pg = pb.out.cpu().numpy().astype(np.complex128)[:, samp["idx"]]
        err = float(np.linalg.norm(pg - samp["p"]) / np.linalg.norm(samp["p"]))
        nr = int(w.receivers.shape[0])
        line["cpu_baseline"] = {
            "value": samp["value"], "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"FP64 trace of the whole fan ({samp['t_trace']:.2f} s, {samp['n_seg']} "
                      f"segments) + sum over {len(samp['idx'])} seeded receivers of {nr} "
                      f"({samp['t_sum']:.2f} s), the sum scaled linearly to all {nr} receivers"}
        line["accuracy"] = {"rel_l2_vs_oracle": err, "receivers_checked": int(len(samp["idx"]))}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
