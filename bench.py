#!/usr/bin/env python
"""TNVAN hot-path benchmark on GB300.

One step = one iteration of Algorithm 1 over every instance of the 16x16
Edwards-Anderson workload (Gaussian J, open boundary, W = every 4th column,
leftover 16x3 strips, MADE 64-128-128-64, beta in {0.2, 0.4, 0.6, 0.8, 1.0},
16384 samples per beta):
  sample + log q (Eq. 6-8) -> strip contraction log Z_R (Eq. 3-4)
  -> F_q / log Z_IS reduction (Eq. 9) -> REINFORCE backward (Eq. 10)
  -> contraction adjoint d log Z_R / d beta and d / d J -> Adam update.
Metric: samples per second (all instances, all ranks).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank draws its own 16384 samples per beta (own Philox
stream) for one shared set of networks: the ranks exchange their Eq. 9
statistics (all-gather) and sum their gradients (all-reduce) every step
(weak scaling; paper_2504_12037_gb300/dp.py); rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle on the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIG = 2
METRIC = "samples/sec (sample+contract+reduce) and |F_q-F_exact|/N; mixed vs FP32 on one GB300"
UNIT = "samples/s"
FP32_LANES_PER_SM = 128
# fallbacks when MEASURED_PEAKS.json is absent (one earlier GB300 measurement)
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}


def measured_peaks():
    """Roofline denominators: the measured copy bandwidth and cuBLAS
    BF16 throughput of the GB300s, else the fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        out = {k: float(d[k]) for k in FALLBACK_PEAKS if k in d}
        if "bf16_tflops" in out and "hbm_gbs" in out:
            out.setdefault("sm_max_mhz", FALLBACK_PEAKS["sm_max_mhz"])
            out["source"] = "MEASURED_PEAKS.json, of measured"
            return out
    except (OSError, ValueError, KeyError):
        pass
    return dict(FALLBACK_PEAKS, source="fallback (MEASURED_PEAKS.json absent), of fallback")
# dram__bytes_read.sum + dram__bytes_write.sum per whole-batch launch from an ncu
# capture of the kernel as it is built now, on the same workload (see profiles/);
# None for kernels not captured since their last change
NCU_TRAFFIC = {"sample_tc": 623872}


def args_():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "tf32", "bf16"],
                    help="headline mode (bf16: network on the tensor cores, contractions FP32)")
    ap.add_argument("--compare", default="fp32", help="second mode timed beside the headline ('' = none)")
    ap.add_argument("--acc-steps", type=int, default=150, help="training steps before the accuracy estimate")
    ap.add_argument("--no-graph", action="store_true", help="skip the CUDA-graph replay timing")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default="",
                    help="six or seven comma-separated ints for Context.set_tuning instead of autotuning "
                         "(sample tile, strip tile, backward CTAs, adjoint tile, TC group, overlap 2=on 1=off)")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", type=int, default=2, choices=[1, 2, 3, 4, 5],
                    help="2 (default): the 16x16 EA headline; 1, 3, 4, 5: the other synthetic workloads "
                         "(4x4 +-J, SK N=64, random 3-regular N=256, 64 mixed-size EA instances), each its own line")
    ap.add_argument("--adjoint", action="store_true",
                    help="with --workload 1, 3, 4, 5: include the contraction adjoint (d/dbeta, d/dJ) in the step "
                         "(the 16x16 headline always does)")
    ap.add_argument("--sampler-only", type=int, default=-1, metavar="PLAN",
                    help="with --workload: build the workload, pin the tensor-core sampler plan PLAN (0 = default) "
                         "and draw two BF16 batches, nothing else (a short command for ncu captures)")
    ap.add_argument("--train-steps", type=int, default=0,
                    help="with --workload 5: Adam steps of the accuracy run (oracle checks at steps 1, 100 and "
                         "the last)")
    ap.add_argument("--planned", action="store_true",
                    help="also time the training step on random regular graphs (n = 1000, d = 3) whose width "
                         "sets come from the width-set finder")
    ap.add_argument("--ferro40", type=int, default=0, metavar="STEPS",
                    help="also train the 40x40 open ferromagnet (W = every 13th column) at T = 1, 2, T_c, 3, 4, 5 "
                         "for STEPS Adam steps and report |F - F_exact| / |F_exact| against the Kac-Ward value")
    ap.add_argument("--ferro-batch", type=int, default=1000, help="--ferro40: samples per temperature and step")
    ap.add_argument("--ferro-lr", type=float, default=0.01,
                    help="--ferro40: Adam learning rate (divided by 10 for the last third of the steps)")
    ap.add_argument("--ferro-period", type=int, default=13,
                    help="--ferro40: W = columns c with c %% P == P - 1 (strips of P - 1 columns)")
    ap.add_argument("--sweep", action="store_true",
                    help="also time the captured step over per-instance batches 2^8 .. 2^18 (the asymptote)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        sm, smax, reasons = [], [], set()
        with open(self.file.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(self.NAMES, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work per sample (used for the roofline figures)
# ---------------------------------------------------------------------------
def made_macs(D, hidden):
    """Masked multiply-adds of one MADE forward pass (each unit once), one or
    two hidden layers."""
    import numpy as np
    cyc = max(D - 1, 1)
    d1 = np.sort(np.arange(hidden[0]) % cyc + 1)
    c1 = lambda d: int((d1 <= d).sum())
    l1 = int(d1.sum())                       # unit of degree d reads inputs 1..d
    if len(hidden) == 1:
        lo = sum(c1(i) for i in range(D))    # output i reads units of degree <= i
        return l1 + lo, (l1, 0, lo)
    d2 = np.sort(np.arange(hidden[1]) % cyc + 1)
    c2 = lambda d: int((d2 <= d).sum())
    l2 = sum(c1(int(d)) for d in d2)         # layer-2 unit reads layer-1 units of degree <= d
    lo = sum(c2(i) for i in range(D))        # output i reads layer-2 units of degree <= i
    return l1 + l2 + lo, (l1, l2, lo)


def strip_flops(w, L):
    """FP32 operations of one strip chain (per sample): each of L-1 vertical
    steps applies w Kronecker 2x2 factors (2^w outputs x 3 ops) and a diagonal
    (2^w mults); renormalisation adds 2^w mults + 2^w max per row."""
    nx = 1 << w
    return (L - 1) * (w * nx * 3 + nx) + L * 2 * nx


def sampler_latency_bound(model, w, prec, ms_full, n_sm, stream):
    """The sampler's latency bound: every sample is a chain of D dependent
    steps (Eq. 8) and an SM holds at most 2 x 128 samples in flight (TMEM: 128
    lanes, two CTAs of <= 256 columns), so the batch takes at least
    t_step x D x (samples / (2 x 128 x SMs)), with t_step the per-step
    latency of one full wave, measured here: the same kernel timed alone on a
    batch that fills exactly one wave of resident CTAs."""
    import torch

    n_inst = len(w.graphs)
    per_inst = (2 * n_sm * 128) // n_inst // 128 * 128  # one wave of CTAs over the instances
    bufs = model.buffers(per_inst)
    for i in range(3):
        model.sample(per_inst, 5, i, prec, bufs, stream)
    torch.cuda.synchronize()
    model.ctx.profile(True)
    for i in range(5):
        model.sample(per_inst, 5, 10 + i, prec, bufs, stream)
    torch.cuda.synchronize()
    model.ctx.profile(False)
    prof = model.ctx.profile_read()
    ms_wave, n = prof.get("sample_tc", (float("nan"), 1))
    ms_wave /= n
    D = max(len(W) for W in w.widths_sets)
    in_flight = 2 * n_sm * 128
    total = n_inst * w.batch
    bound = ms_wave * total / (per_inst * n_inst)  # = t_step x D x total / in_flight
    return {"model": "t_step x D x samples / samples_in_flight", "samples_in_flight": in_flight,
            "wave_samples": per_inst * n_inst, "wave_ms": ms_wave, "t_step_us": ms_wave / D * 1e3,
            "bound_ms": bound, "measured_ms": ms_full, "frac": bound / ms_full}


def parity_run(model, step, name, bufs, B):
    """One more step of the timed kind (`step`, the timed path with its tuning),
    with what the oracle needs to check it copied to the host: the parameters
    the step sampled with, the samples, log q and log Z_R of sampled rows (every
    1021st sample and the tile edges), the whole batch's log q and log Z_R and
    the step's statistics rows."""
    import numpy as np
    import torch

    p_before = model.params.cpu().numpy().copy()
    step(3 * 10 ** 6)
    torch.cuda.synchronize()
    st = model.step_stats().cpu().numpy()
    spins, logq, logZR = bufs
    rows = np.unique(np.concatenate([np.arange(0, B, 1021), [r for r in (0, 127, 128, 255, 256, B - 1) if r < B]]))
    lq, lz = logq.cpu().numpy(), logZR.cpu().numpy()
    return {"precision": name, "params": p_before, "offsets": np.asarray(model.offsets), "rows": rows,
            "spins": [model.spins_of(spins, k, B).cpu().numpy()[rows] for k in range(model.n)],
            "logq": lq.reshape(model.n, B), "logZR": lz.reshape(model.n, B), "stats": st}


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2504_12037_gb300 import tnvan as tv
    from paper_2504_12037_gb300 import workloads as wl
    from paper_2504_12037_gb300.model import TNVAN

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    PREC = {"fp32": tv.FP32, "tf32": tv.TF32, "bf16": tv.BF16}
    prec = PREC[a.precision]
    w = wl.workload(CONFIG)
    B = w.batch
    n_inst = len(w.graphs)
    stream = torch.cuda.current_stream()
    seed = 12037 + 7919 * rank
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    props = torch.cuda.get_device_properties(local)
    gpu_id = f"GPU-{props.uuid}" if hasattr(props, "uuid") else str(local)

    def timed(mode: int, steps: int, warmup: int, sample_clocks: bool):
        model = TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas, device=local, seed=1000 * rank + 1)
        model.ctx.reserve(B)
        if a.tuning:
            tuned = tuple(int(v) for v in a.tuning.split(","))
            tuned = tuned + (0,) * (7 - len(tuned))  # a 6-value tuning leaves the backward form at its default
            model.ctx.set_tuning(tuned)
        else:
            tuned = None if a.no_autotune else model.ctx.autotune(model.betas, B, mode)
        dbeta = torch.empty(n_inst * B, dtype=torch.float64, device="cuda")
        dJ = torch.empty(sum(model.n_edges), dtype=torch.float64, device="cuda")
        model.tuned = tuned
        if world > 1:
            # one set of networks trained on all ranks' samples: local sampling
            # and contraction, statistics all-gather, gradient all-reduce, Adam
            from paper_2504_12037_gb300.dp import DataParallelStep

            dps = DataParallelStep(model, B, mode, 0.01, dbeta=dbeta, dJ=dJ)
            bufs = dps.out

            def step(i):
                dps(12037, i, stream)
        else:
            bufs = model.buffers(B)

            def step(i):
                model.train_step(B, seed, i, mode, 0.01, bufs, dbeta, dJ, stream)

        for i in range(warmup):
            step(i)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = ClockSampler(gpu_id) if sample_clocks else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        model.ctx.profile(True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        for i in range(steps):
            flush.zero_()  # evict L2 between timed steps (not inside the timed interval)
            starts[i].record(stream)
            step(warmup + i)
            ends[i].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        model.ctx.profile(False)
        ms = sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)) / steps
        prof = model.ctx.profile_read()
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return model, bufs, dbeta, dJ, step, float(t.item()), prof, clocks

    def graph_time(model, mode, bufs, dbeta, dJ):
        """The same step as one CUDA-graph replay (model.capture_train_step); ms per step."""
        cs = model.capture_train_step(B, seed, mode, 0.01, bufs, dbeta, dJ)
        for _ in range(a.warmup):
            cs.replay()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        gs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
        ge = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
        for i in range(a.steps):
            flush.zero_()  # evict L2 between replays (outside the timed interval)
            gs[i].record(stream)
            cs.replay()
            ge[i].record(stream)
        torch.cuda.synchronize()
        ms_g = sum(x.elapsed_time(y) for x, y in zip(gs, ge)) / a.steps
        tg = torch.tensor([ms_g], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(tg, op=dist.ReduceOp.MAX)
        return float(tg.item()), cs

    # clocks are sampled from before the eager timed steps to after the graph replays
    model, (spins, logq, logZR), dbeta, dJ, step, ms_eager, prof, clocks = timed(prec, a.steps, a.warmup, True)
    samples_step = n_inst * B * world
    graph = None
    captured = None
    # every rank takes the parity step (a data-parallel step is collective); rank 0 checks it
    parity_runs = [parity_run(model, step, a.precision, (spins, logq, logZR), B)]
    if not a.no_graph and world == 1:
        ms_g, captured = graph_time(model, prec, (spins, logq, logZR), dbeta, dJ)
        graph = {"value": samples_step / (ms_g / 1e3), "ms_per_step": ms_g,
                 "note": "whole training step captured once, replayed; Philox step from a device counter"}
    clk = clocks.stop() if clocks else None
    eager = {"value": samples_step / (ms_eager / 1e3), "ms_per_step": ms_eager,
             "note": "the same step launched call by call from Python (host launch overhead included)"}
    # headline: the replayed graph (how a training loop runs the step), else the eager steps
    ms_max = graph["ms_per_step"] if graph else ms_eager
    value = samples_step / (ms_max / 1e3)
    compare = None
    if a.compare and a.compare != a.precision:
        m_c, b_c, db_c, dj_c, step_c, ms_c, prof_c, _ = timed(PREC[a.compare], a.steps, a.warmup, False)
        parity_runs.append(parity_run(m_c, step_c, a.compare, b_c, B))
        ms_cg = None if (a.no_graph or world > 1) else graph_time(m_c, PREC[a.compare], b_c, db_c, dj_c)[0]
        ms_ch = ms_cg if ms_cg else ms_c
        compare = {"precision": a.compare, "value": samples_step / (ms_ch / 1e3), "ms_per_step": ms_ch,
                   "eager_ms_per_step": ms_c,
                   "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]} for k, v in prof_c.items()}}

    # ----- end to end through the public API with host buffers -----
    # Every step: the step's input from pinned host memory (which Philox step
    # and Adam t to run, into the captured step's device counter), the step,
    # and the step's results read back to pinned host memory (samples, log q,
    # log Z_R and the step's Eq. 9 rows: F_q, F_IS, stderr, log Z_IS, ... per
    # instance, reduced inside the step).  With a captured step the outputs
    # alternate between two captures of the step (two buffer sets), so step
    # i's read-back runs on a copy stream while step i + 1 computes.
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    fe_last = None
    if captured is not None:
        db2 = torch.empty_like(dbeta)
        dj2 = torch.empty_like(dJ)
        slots = [captured, model.capture_train_step(B, seed, prec, 0.01, model.buffers(B), db2, dj2)]
        cs = torch.cuda.Stream()
        h_out = [(torch.empty(spins.numel(), dtype=torch.int8, pin_memory=True),
                  torch.empty(logq.numel(), dtype=torch.float32, pin_memory=True),
                  torch.empty(logZR.numel(), dtype=torch.float64, pin_memory=True)) for _ in range(2)]
        h_ctr = [torch.zeros(1, dtype=torch.int64, pin_memory=True) for _ in range(2)]
        h_st = [torch.zeros(n_inst, 8, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        ran = [torch.cuda.Event() for _ in range(2)]
        read = [torch.cuda.Event() for _ in range(2)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(a.e2e_steps + 1):
            if i < a.e2e_steps:
                j = i % 2
                if i >= 2:
                    stream.wait_event(read[j])  # slot j's buffers have been read back
                h_ctr[j][0] = 10 ** 6 + i
                slots[j].counter.copy_(h_ctr[j], non_blocking=True)
                slots[j].replay()
                ran[j].record(stream)
            if i >= 1:
                jp = (i - 1) % 2
                sp_, lq_, lz_ = slots[jp].out
                cs.wait_event(ran[jp])
                with torch.cuda.stream(cs):
                    h_st[jp].copy_(slots[jp].stats, non_blocking=True)  # the step's statistics
                    h_out[jp][0].copy_(sp_, non_blocking=True)
                    h_out[jp][1].copy_(lq_, non_blocking=True)
                    h_out[jp][2].copy_(lz_, non_blocking=True)
                read[jp].record(cs)
        cs.synchronize()
        stream.synchronize()
        t_e2e = (time.perf_counter() - t0) / max(a.e2e_steps, 1)
        fe_last = h_st[(a.e2e_steps - 1) % 2].numpy().copy()
    else:
        h_spins = torch.empty(spins.numel(), dtype=torch.int8, pin_memory=True)
        h_logq = torch.empty(logq.numel(), dtype=torch.float32, pin_memory=True)
        h_logZR = torch.empty(logZR.numel(), dtype=torch.float64, pin_memory=True)
        h_st = torch.zeros(n_inst, 8, dtype=torch.float64, pin_memory=True)
        d_st = torch.empty(n_inst * 8, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(a.e2e_steps):
            step(10 ** 6 + i)
            h_st.copy_(model.step_stats(d_st, stream), non_blocking=True)  # the step's statistics
            h_spins.copy_(spins, non_blocking=True)
            h_logq.copy_(logq, non_blocking=True)
            h_logZR.copy_(logZR, non_blocking=True)
            stream.synchronize()
        t_e2e = (time.perf_counter() - t0) / max(a.e2e_steps, 1)
    te = torch.tensor([t_e2e], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(te, op=dist.ReduceOp.MAX)
    e2e = {"value": samples_step / float(te.item()), "unit": UNIT,
           "h2d_bytes_per_step": 8 if captured is not None else 8 * n_inst,
           "path": ("model.capture_train_step replays (two buffer sets; read-back of step i beside step i + 1)"
                    if captured is not None else "model.train_step"),
           "d2h_bytes_per_step": int(spins.numel() + 4 * logq.numel() + 8 * logZR.numel() + 64 * n_inst),
           "statistics": "F_q, F_IS, stderr, log Z_IS of every step reduced on the device inside the step "
                         "and read back with its samples"}

    # ----- per-kernel durations: the same step with the overlapped side-stream
    # schedule off, so that every kernel's events bracket it alone -----
    base = tuple(model.tuned) if model.tuned else (0, 0, 0, 0, 0, 0)
    model.ctx.set_tuning(base[:5] + (1,) + base[6:])
    for i in range(2):
        step(2 * 10 ** 6 + i)
    torch.cuda.synchronize()
    model.ctx.profile(True)
    for i in range(3):
        flush.zero_()
        step(2 * 10 ** 6 + 2 + i)
    torch.cuda.synchronize()
    model.ctx.profile(False)
    prof_seq = model.ctx.profile_read()
    model.ctx.set_tuning(base)
    prof_overlapped = prof
    prof = prof_seq

    # ----- roofline of the dominant kernel -----
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    D, H = model.D[0], w.hidden
    macs, parts = made_macs(D, H)
    strips = 4
    # algorithmic FLOPs per sample of each kernel (masked network, strip chains)
    per_sample = {
        "sample": 2.0 * macs, "sample_tc": 2.0 * macs,
        "backward": 2.0 * macs * 3, "bwd_fused": 2.0 * macs * 3,  # forward, delta, weight gradient
        "strips": strips * strip_flops(3, 16),
        "strips+dbeta": strips * 2 * strip_flops(3, 16),
        "strips_dbeta": strips * 2 * strip_flops(3, 16),
        "strips_adj": strips * 4 * strip_flops(3, 16),  # forward sweep (1x) + backward sweep (3x)
    }
    flop_launch = per_sample.get(dom_name, float("nan")) * n_inst * B
    achieved = flop_launch / (dom_ms / dom_n / 1e3) / 1e12 if dom_n else float("nan")
    note = None
    peaks = measured_peaks()
    n_sm = props.multi_processor_count
    if dom_name in ("sample_tc", "bwd_fused"):
        # BF16 operands on tcgen05: the tensor roofline (the sampler is bound by its
        # chain of D dependent steps per sample, Eq. 8, far below it)
        peak, bound = peaks["bf16_tflops"], "tensor"
        src = f"bf16_tflops (burst) from {peaks['source']}"
        if dom_name == "sample_tc":
            note = f"latency-bound: {D} dependent steps per sample; masked MACs counted once"
    else:
        peak = n_sm * FP32_LANES_PER_SM * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        bound = "alu"
        src = (f"derived: {n_sm} SMs (queried) x {FP32_LANES_PER_SM} FP32 lanes x 2 FLOP x "
               f"{peaks['sm_max_mhz']:.0f} MHz ({peaks['source']})")
    roofline = {"bound": bound, "kernel": dom_name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": NCU_TRAFFIC.get(dom_name), "peak_source": src,
                "flop_per_launch": flop_launch, "ms_per_launch": dom_ms / dom_n}
    if note:
        roofline["note"] = note
    if dom_name == "sample_tc":
        roofline["latency_bound"] = sampler_latency_bound(model, w, prec, dom_ms / dom_n, n_sm, stream)
    kernels = {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]} for k, v in prof.items()}
    launches_per_step = sum(v[1] for v in prof_overlapped.values()) / a.steps

    # ----- accuracy: both modes trained from the same start, then F_q / N -----
    accuracy = None
    if a.acc_steps > 0:
        accuracy = {"train_steps": a.acc_steps, "batch_per_beta": B, "betas": w.betas}
        for name in [a.precision] + ([a.compare] if compare else []):
            m2 = TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas, device=local, seed=77)
            b2 = m2.buffers(B)
            for i in range(a.acc_steps):
                m2.train_step(B, 4242, i, PREC[name], 0.01, b2, None, None, stream)
            sp2, lq2, lz2 = m2.sample(B, 999, 10 ** 7, PREC[name], b2, stream)
            fe = m2.free_energy(B, lz2, lq2, stream)
            accuracy[name] = {"F_q_per_spin": [float(x) / 256 for x in fe[:, 0]],
                              "F_IS_per_spin": [float(x) / 256 for x in fe[:, 1]],
                              "stderr_per_spin": [float(x) / 256 for x in fe[:, 2]]}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "tf32": "tf32", "bf16": "bf16"}[a.precision],
        "data": "synthetic (seeded EA couplings; random-init MADE)",
        "config": {**headline_config(w, B),
                   "precision": f"{a.precision}: network (sampler, backward) in {a.precision} on the "
                                "tensor cores with FP32 accumulation; contractions FP32; reductions FP64"
                                if a.precision != "fp32" else "fp32 everywhere, FP64 reductions",
                   "timing": ("CUDA-graph replay of the whole step (captured once; fresh Philox step per replay "
                              "from a device counter)" if graph else "eager steps"),
                   "l2": "flushed (256 MB write) between timed steps", "parallelism": f"dp{world}" if world > 1 else "single GPU"},
        "clocks": clk, "e2e": e2e, "gpu_launches": int(round(launches_per_step * a.steps)),
        "roofline": roofline, "kernels": kernels,
        "kernels_note": "per-launch CUDA-event times of 3 steps with the overlapped side-stream schedule off",
        "compare": compare, "accuracy": accuracy,
        "graph": graph, "eager": eager, "autotuned": {"sample_tile": None if not model.tuned else model.tuned[0],
                                      "strip_tile": None if not model.tuned else model.tuned[1],
                                      "bwd_ctas_per_instance": None if not model.tuned else model.tuned[2],
                                      "strip_adjoint_tile": None if not model.tuned else model.tuned[3],
                                      "tc_sampler_group_steps": None if not model.tuned else model.tuned[4],
                                      "overlapped_schedule": None if not model.tuned else model.tuned[5] == 2,
                                      "backward_form": None if not model.tuned else model.tuned[6]},
    }
    if a.sweep:
        # samples/s of the whole captured step against the batch: per-instance
        # batches 2^8 .. 2^18 (5 instances: 1,280 .. 1,310,720 samples per step),
        # each autotuned, L2 flushed between replays
        sweep = []
        for lb in range(8, 19, 2):
            Bs = 1 << lb
            ms_ = TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas, device=local, seed=1000 * rank + 3)
            ms_.ctx.reserve(Bs)
            ms_.ctx.autotune(ms_.betas, Bs, prec)
            dbs = torch.empty(n_inst * Bs, dtype=torch.float64, device="cuda")
            djs = torch.empty(sum(ms_.n_edges), dtype=torch.float64, device="cuda")
            cap = ms_.capture_train_step(Bs, seed, prec, 0.01, ms_.buffers(Bs), dbs, djs)
            for _ in range(3):
                cap.replay()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
            for e0, e1 in ev:
                flush.zero_()
                e0.record(stream)
                cap.replay()
                e1.record(stream)
            torch.cuda.synchronize()
            t_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / len(ev)
            sweep.append({"batch_per_instance": Bs, "samples_per_step": n_inst * Bs * world, "ms_per_step": t_ms,
                          "value": n_inst * Bs * world / (t_ms / 1e3)})
            del cap, ms_
        out["sweep"] = sweep
    if a.planned:
        # random regular graph, n = 1000, d = 3, J = +-1, beta = 0.5 (the paper's
        # Fig. 3(a,b) setting), batch 10,000; W and R's elimination order from
        # tnvan_find_width_set at several width bounds; the captured training
        # step (BF16 sampler, elimination contraction, d/dbeta, d/dJ, Adam)
        planned = []
        g = wl.random_regular(1000, 3, 12037 + 7000)
        Bp = 10000
        for wu in (1, 4, 8):
            t0 = time.time()
            Wp, op, wp, _ = tv.find_width_set(g.n, g.ei, g.ej, wu, restarts=4, seed=1)
            t_plan = time.time() - t0
            mp = TNVAN([g], [Wp], [128, 128], [0.5], device=local, seed=1000 * rank + 5, elim_orders=[op])
            info = mp.ctx.instance_info(0)
            mp.ctx.reserve(Bp)
            mp.ctx.autotune(mp.betas, Bp, prec)
            dbs = torch.empty(Bp, dtype=torch.float64, device="cuda")
            djs = torch.empty(g.m, dtype=torch.float64, device="cuda")
            cap = mp.capture_train_step(Bp, seed, prec, 0.01, mp.buffers(Bp), dbs, djs)
            for _ in range(3):
                cap.replay()
            torch.cuda.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
            for e0, e1 in ev:
                flush.zero_()
                e0.record(stream)
                cap.replay()
                e1.record(stream)
            torch.cuda.synchronize()
            t_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / len(ev)
            # per-kernel device times of two eager steps (profiling hooks)
            bp = mp.buffers(Bp)
            mp.ctx.profile(True)
            for i in range(2):
                mp.train_step(Bp, seed, 10 ** 6 + i, prec, 0.01, bp, dbs, djs, stream)
            torch.cuda.synchronize()
            mp.ctx.profile(False)
            kern = {k: round(v[0] / v[1], 4) for k, v in mp.ctx.profile_read().items()}
            planned.append({"w_u": wu, "ms_per_launch": kern, "n_w": len(Wp), "width": wp, "finder_s": t_plan,
                            "components": info["n_components"], "max_component": info["max_component"],
                            "arena_floats": info["arena"], "arena_live_floats": info["arena_live"],
                            "batch": Bp * world, "ms_per_step": t_ms, "value": Bp * world / (t_ms / 1e3)})
            del cap, mp
        out["planned_rrg_n1000_d3"] = planned
    ferro = None
    if a.ferro40 > 0:
        # the paper's first experiment (Sec. 4, Fig. 2): training steps in FP32,
        # then F_q and F_IS from one large batch per temperature
        wf = wl.ferromagnet_columns(period=a.ferro_period, batch=a.ferro_batch)
        mf = TNVAN(wf.graphs, wf.widths_sets, wf.hidden, wf.betas, device=local, seed=1000 * rank + 9,
                   elim_orders=wf.elim_orders)
        bf = mf.buffers(wf.batch)
        t0 = time.time()
        for i in range(a.ferro40):
            lr = a.ferro_lr if 3 * i < 2 * a.ferro40 else a.ferro_lr / 10
            mf.train_step(wf.batch, 40 + rank, i, tv.FP32, lr, bf, None, None, stream)
        torch.cuda.synchronize()
        t_train = time.time() - t0
        Bf = 16384
        spf, lqf, lzf = mf.sample(Bf, 4040 + rank, 10 ** 7, tv.FP32)
        fe = mf.free_energy(Bf, lzf, lqf)
        N = wf.graphs[0].n
        ferro = {"workload": wf.name, "train_steps": a.ferro40, "train_batch": wf.batch, "made": wf.hidden,
                 "lr": [a.ferro_lr, a.ferro_lr / 10], "W_size": int(len(wf.widths_sets[0])),
                 "train_s": t_train, "eval_batch": Bf, "T": [1.0 / b for b in wf.betas],
                 "F_q_per_spin": [float(x) / N for x in fe[:, 0]], "F_IS_per_spin": [float(x) / N for x in fe[:, 1]],
                 "stderr_per_spin": [float(x) / N for x in fe[:, 2]]}
        # magnetisation and susceptibility (Sec. 3) from a smaller batch: the
        # exact conditional moments of M per sample, importance-weighted
        Bm = 2048
        spm, lqm, lzm = mf.sample(Bm, 4141 + rank, 10 ** 7 + 1, tv.FP32)
        t0 = time.time()
        mag = mf.ctx.magnetisation(mf.betas, Bm, spm, lzm, lqm)
        torch.cuda.synchronize()
        ferro["magnetisation"] = {"batch": Bm, "s": time.time() - t0,
                                  "rms_M_per_spin": [float(np.sqrt(max(r[1], 0.0))) / N for r in mag],
                                  "M_per_spin": [float(r[0]) / N for r in mag],
                                  "chi_per_spin": [float(r[2]) for r in mag], "ess": [float(r[5]) for r in mag]}
    if rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, model.params.cpu().numpy(), model.offsets, budget_s=15.0)
        # the oracle's exact free energy of the lattice (single-site transfer matrix, 2^16 states)
        f_exact = oracle_exact_f(w)
        out["cpu_baseline"]["F_exact_per_spin"] = f_exact
        if accuracy:
            for name in [k for k in accuracy if isinstance(accuracy[k], dict)]:
                accuracy[name]["abs_F_q_minus_F_exact_per_spin"] = [
                    abs(fq - fe) for fq, fe in zip(accuracy[name]["F_q_per_spin"], f_exact)]
        # the oracle on sampled rows of one timed-path step per precision
        out["parity"] = oracle_parity(w, parity_runs, check_stats=world == 1)
        if ferro is not None:
            ferro.update(oracle_ferro_exact(wl.ferromagnet_columns(period=a.ferro_period), ferro))
    if ferro is not None:
        out["ferromagnet_40x40"] = ferro
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# the other workloads (--workload 1, 3, 4, 5): one JSON line each
# ---------------------------------------------------------------------------
def oracle_log_zr(g, W, beta, s):
    """The oracle's log Z_R (Eq. 4) of given width-set rows, by topology."""
    from oracle import dense, general, ising, transfer

    if g.topology == 1:
        return dense.log_zr_dense(g.n, g.ei, g.ej, g.J, beta, W, s)
    if g.topology == 2:
        return general.log_zr_general(g.n, g.ei, g.ej, g.J, beta, W, s)
    if g.n <= 16:
        return ising.log_zr_enum(g.n, g.ei, g.ej, g.J, beta, W, s)
    return transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, beta, W, s, g.Lx)


def run_workload(a):
    """One synthetic workload: the captured training step in BF16 (headline)
    and FP32, per-kernel times, the dominant kernel's roofline, end to end
    through host buffers, and (rank 0, oracle leg) parity on sampled rows,
    the oracle timed on a bounded sample, and for workload 5 an Adam run with
    oracle checks along it."""
    import numpy as np
    import torch

    from paper_2504_12037_gb300 import tnvan as tv
    from paper_2504_12037_gb300 import workloads as wl
    from paper_2504_12037_gb300.model import TNVAN

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    w = wl.workload(a.workload)
    B = w.batch
    n_inst = len(w.graphs)
    stream = torch.cuda.current_stream()
    seed = 12037 + 7919 * rank
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    props = torch.cuda.get_device_properties(local)
    gpu_id = f"GPU-{props.uuid}" if hasattr(props, "uuid") else str(local)
    samples_step = n_inst * B * world
    PREC = {"fp32": tv.FP32, "bf16": tv.BF16}
    if a.sampler_only >= 0:
        m = TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas, device=local, seed=1)
        m.ctx.set_tuning((0, 0, 0, 0, a.sampler_only, 0))
        t0 = time.perf_counter()
        for i in range(2):
            m.sample(B, 1, i, tv.BF16)
        torch.cuda.synchronize()
        print(json.dumps({"workload": w.name, "sampler_only": a.sampler_only, "s": time.perf_counter() - t0}))
        return

    def measure(name, sample_clocks):
        mode = PREC[name]
        m = TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas, device=local, seed=1000 * rank + 1)
        m.ctx.reserve(B)
        tuned = m.ctx.autotune(m.betas, B, mode)
        dbeta = torch.empty(n_inst * B, dtype=torch.float64, device="cuda") if a.adjoint else None
        dJ = torch.empty(sum(m.n_edges), dtype=torch.float64, device="cuda") if a.adjoint else None
        cs = m.capture_train_step(B, seed, mode, 0.01, None, dbeta, dJ)
        for _ in range(a.warmup):
            cs.replay()
        torch.cuda.synchronize()
        clocks = ClockSampler(gpu_id) if sample_clocks else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
        for e0, e1 in ev:
            flush.zero_()  # evict L2 between replays (outside the timed interval)
            e0.record(stream)
            cs.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = sum(e0.elapsed_time(e1) for e0, e1 in ev) / a.steps
        clk = clocks.stop() if clocks else None
        # per-kernel times: eager steps with the overlapped schedule off
        base = tuple(tuned)
        m.ctx.set_tuning(base[:5] + (1,) + base[6:])
        bufs = m.buffers(B)
        m.train_step(B, seed, 10 ** 6, mode, 0.01, bufs, dbeta, dJ, stream)
        torch.cuda.synchronize()
        m.ctx.profile(True)
        for i in range(3):
            flush.zero_()
            m.train_step(B, seed, 10 ** 6 + 1 + i, mode, 0.01, bufs, dbeta, dJ, stream)
        torch.cuda.synchronize()
        m.ctx.profile(False)
        prof = m.ctx.profile_read()
        m.ctx.set_tuning(base)
        # launches per step of the captured form (overlapped schedule on)
        m.ctx.profile(True)
        m.train_step(B, seed, 10 ** 6 + 9, mode, 0.01, bufs, dbeta, dJ, stream)
        torch.cuda.synchronize()
        m.ctx.profile(False)
        launches = sum(v[1] for v in m.ctx.profile_read().values())
        run = parity_run(m, lambda i: m.train_step(B, seed, i, mode, 0.01, bufs, dbeta, dJ, stream), name, bufs, B)
        return {"model": m, "cs": cs, "ms": ms, "clocks": clk, "prof": prof, "tuned": tuned, "run": run,
                "launches": launches}

    head = measure("bf16", True)
    cmp_ = measure("fp32", False)
    m, cs = head["model"], head["cs"]
    # end to end: counter upload, one replay, samples / log q / log Z_R and the
    # step's statistics read back to pinned host memory, every step
    h_ctr = torch.zeros(1, dtype=torch.int64, pin_memory=True)
    sp_, lq_, lz_ = cs.out
    h_out = (torch.empty(sp_.numel(), dtype=torch.int8, pin_memory=True),
             torch.empty(lq_.numel(), dtype=torch.float32, pin_memory=True),
             torch.empty(lz_.numel(), dtype=torch.float64, pin_memory=True),
             torch.empty(n_inst, 8, dtype=torch.float64, pin_memory=True))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(a.e2e_steps):
        h_ctr[0] = 10 ** 7 + i
        cs.counter.copy_(h_ctr, non_blocking=True)
        cs.replay()
        for h, d in zip(h_out, (sp_, lq_, lz_, cs.stats)):
            h.copy_(d, non_blocking=True)
        stream.synchronize()
    t_e2e = (time.perf_counter() - t0) / max(a.e2e_steps, 1)
    prof = head["prof"]
    dom_name, (dom_ms, dom_n) = max(prof.items(), key=lambda kv: kv[1][0])
    peaks = measured_peaks()
    macs = [made_macs(len(W), w.hidden)[0] for W in w.widths_sets]
    roofline = {"kernel": dom_name, "ms_per_launch": dom_ms / dom_n}
    if dom_name == "dense" and any(g.topology == 1 for g in w.graphs):
        # the leftover block as a [B x 256] x [256 x 256] product (BF16 tensor cores)
        flop = 2.0 * 256 * 256 * B * sum(1 for g in w.graphs if g.topology == 1)
        ach = flop / (dom_ms / dom_n / 1e3) / 1e12
        roofline.update({"bound": "tensor", "achieved": ach, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                         "frac": ach / peaks["bf16_tflops"], "flop_per_launch": flop, "traffic": None,
                         "peak_source": peaks["source"],
                         "note": "dense_table_kernel (the 256 x 256 table per beta) and dense_tc_kernel together"})
    elif dom_name in ("sample_tc", "bwd_fused", "sample", "backward"):
        mult = 3 if dom_name in ("bwd_fused", "backward") else 1
        flop = 2.0 * mult * sum(macs) * B
        ach = flop / (dom_ms / dom_n / 1e3) / 1e12
        tensor = dom_name in ("sample_tc", "bwd_fused")
        peak = peaks["bf16_tflops"] if tensor else props.multi_processor_count * FP32_LANES_PER_SM * 2 * \
            peaks["sm_max_mhz"] * 1e6 / 1e12
        roofline.update({"bound": "tensor" if tensor else "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "flop_per_launch": flop, "traffic": None,
                         "peak_source": peaks["source"], "note": "masked MACs counted once per unit"})
    else:
        roofline.update({"bound": None, "note": "no algorithmic work formula for this kernel"})
    out = {
        "metric": METRIC, "value": samples_step / (head["ms"] / 1e3), "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": head["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded couplings; random-init MADE)",
        "config": {"workload": w.name, "instances": n_inst, "batch_per_instance": B, "made": w.hidden,
                   "betas": sorted(set(float(b) for b in w.betas)),
                   "width_set_sizes": sorted(set(int(len(W)) for W in w.widths_sets)),
                   "step": ("sample+contract+reduce+REINFORCE backward+d/dbeta+d/dJ+Adam" if a.adjoint
                            else "sample+contract+reduce+REINFORCE backward+Adam"),
                   "timing": "CUDA-graph replay of the whole step", "l2": "flushed (256 MB write) between steps",
                   "parallelism": "single GPU"},
        "clocks": head["clocks"],
        "e2e": {"value": samples_step / t_e2e, "unit": UNIT, "h2d_bytes_per_step": 8,
                "d2h_bytes_per_step": int(sp_.numel() + 4 * lq_.numel() + 8 * lz_.numel() + 64 * n_inst)},
        "gpu_launches": int(head["launches"] * a.steps), "roofline": roofline,
        "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]} for k, v in prof.items()},
        "autotuned": list(head["tuned"]),
        "compare": {"precision": "fp32", "value": samples_step / (cmp_["ms"] / 1e3), "ms_per_step": cmp_["ms"],
                    "kernels": {k: {"ms_per_launch": v[0] / v[1], "launches": v[1]}
                                for k, v in cmp_["prof"].items()}},
    }
    traj = None
    if a.workload == 5 and a.train_steps > 0:
        # Adam from the same start; at steps 1, 100 and the last: the step's
        # statistics and, for a few instances of each size, the rows the
        # oracle checks
        mt = TNVAN(w.graphs, w.widths_sets, w.hidden, w.betas, device=local, seed=77)
        bt = mt.buffers(B)
        checks = sorted(set([1, min(100, a.train_steps), a.train_steps]))
        picks = []
        for L in sorted(set(g.Lx for g in w.graphs)):
            picks += [k for k, g in enumerate(w.graphs) if g.Lx == L][:2]
        traj = {"train_steps": a.train_steps, "checked_steps": checks, "instances_checked": picks, "runs": []}
        # the gradient at step 1 (before the first update), through the C-ABI
        # backward on the GPU's own samples: FP32 sampler + FP32 backward, and
        # the step's BF16 samples + BF16 backward
        gchk = {"params": mt.params.cpu().numpy().copy(), "offsets": np.asarray(mt.offsets), "runs": {}}
        for name, prec in (("fp32", tv.FP32), ("bf16", tv.BF16)):
            sp_g, lq_g, lz_g = mt.sample(B, 4242, 1, prec)
            gg = torch.full_like(mt.params, float("nan"))
            mt.ctx.backward(mt.betas, B, sp_g, lz_g, lq_g, prec, gg)
            torch.cuda.synchronize()
            gchk["runs"][name] = {"spins": {k: mt.spins_of(sp_g, k, B).cpu().numpy() for k in picks},
                                  "grad": gg.cpu().numpy()}
        traj["grad_check"] = gchk
        t0 = time.time()
        for i in range(1, a.train_steps + 1):
            if i in checks:
                p_before = mt.params.cpu().numpy().copy()
            mt.train_step(B, 4242, i, tv.BF16, 0.01, bt, None, None, stream)
            if i in checks:
                torch.cuda.synchronize()
                st = mt.step_stats().cpu().numpy()
                rows = np.arange(0, B, 97)
                traj["runs"].append({"step": i, "params": p_before, "offsets": np.asarray(mt.offsets),
                                     "stats": st, "rows": rows,
                                     "spins": {k: mt.spins_of(bt[0], k, B).cpu().numpy()[rows] for k in picks},
                                     "logq": {k: bt[1][k * B:(k + 1) * B].cpu().numpy()[rows] for k in picks},
                                     "logZR": {k: bt[2][k * B:(k + 1) * B].cpu().numpy()[rows] for k in picks}})
        torch.cuda.synchronize()
        traj["train_s"] = time.time() - t0
    if rank == 0 and not a.no_cpu_baseline:
        out["parity"] = oracle_parity_any(w, [head["run"], cmp_["run"]])
        out["cpu_baseline"] = cpu_baseline_any(w, head["model"].params.cpu().numpy(), head["model"].offsets)
        if traj is not None:
            out["train_run"] = oracle_train_checks(w, traj)
    print(json.dumps(out), flush=True)


def oracle_parity_any(w, runs, max_inst=8):
    """oracle_parity for any topology, on at most max_inst instances."""
    import numpy as np
    import torch

    from oracle import estimators as est
    from oracle import made

    out = {}
    ks = list(range(len(w.graphs)))[:max_inst]
    for r in runs:
        e_q = e_z = e_red = 0.0
        for k in ks:
            g, W, beta = w.graphs[k], w.widths_sets[k], w.betas[k]
            th = torch.as_tensor(r["params"][r["offsets"][k]:r["offsets"][k + 1]].astype(np.float64))
            s = torch.as_tensor(r["spins"][k].astype(np.float64))
            lq_or = made.log_q(th, len(W), w.hidden, s).numpy()
            lz_or = oracle_log_zr(g, W, beta, s).detach().numpy()
            e_q = max(e_q, float(np.abs(r["logq"][k][r["rows"]] - lq_or).max()) / g.n)
            e_z = max(e_z, float(np.abs(r["logZR"][k][r["rows"]] - lz_or).max()) / g.n)
            fe = est.free_energies(r["logZR"][k], r["logq"][k].astype(np.float64), beta)
            e_red = max(e_red, abs(r["stats"][k][0] - fe["F_q"]) / g.n, abs(r["stats"][k][1] - fe["F_IS"]) / g.n)
        out[r["precision"]] = {"instances_checked": len(ks), "rows_per_instance": int(len(r["rows"])),
                               "max_abs_dlogq_per_spin": e_q, "max_abs_dlogZR_per_spin": e_z,
                               "reduction_max_abs_dF_per_spin": e_red}
    out["tolerance_per_spin"] = {"fp32": 1e-6, "reduced_precision": 1e-3}
    return out


def cpu_baseline_any(w, params, offsets, budget_s=10.0, n_b=64):
    """The oracle (sampling replay, log q, log Z_R by topology, estimators) on
    a bounded sample: n_b samples per instance, instances in turn, until about
    budget_s has elapsed."""
    import numpy as np
    import torch

    from oracle import estimators as est
    from oracle import made, philox

    torch.set_num_threads(os.cpu_count() or 1)
    done = 0
    t0 = time.perf_counter()
    k = 0
    while True:
        g, W, beta = w.graphs[k % len(w.graphs)], w.widths_sets[k % len(w.graphs)], w.betas[k % len(w.graphs)]
        kk = k % len(w.graphs)
        th = torch.as_tensor(params[offsets[kk]:offsets[kk + 1]].astype(np.float64))
        u = philox.uniforms(1, k, kk, n_b, len(W))
        s, _ = made.sample(th, len(W), w.hidden, u)
        lq = made.log_q(th, len(W), w.hidden, s)
        lz = oracle_log_zr(g, W, beta, s)
        est.free_energies(lz.detach(), lq.detach(), beta)
        done += n_b
        k += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    return {"value": done / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{k} instance batches x {n_b} samples (FP64 sampling replay, log q, log Z_R, estimators) "
                      f"in {dt:.1f} s"}


def oracle_train_checks(w, traj):
    """At each checked step of the Adam run: |F_q(rows, GPU) - F_q(rows, oracle)|
    / N on the same parameters and samples, the step's F_q / N and, for each
    checked instance, the exact F / N (Kac-Ward determinant) and |F_q - F| / N."""
    import numpy as np
    import torch

    from oracle import kacward, made

    f_ex = {}
    for k in traj["instances_checked"]:
        g = w.graphs[k]
        f_ex[k] = -kacward.log_z_kac_ward(g.Lx, g.Ly, g.ei, g.ej, g.J, w.betas[k]) / w.betas[k] / g.n
    out = {"train_steps": traj["train_steps"], "train_s": traj["train_s"], "checks": []}
    for r in traj["runs"]:
        rec = {"step": r["step"], "instances": []}
        for k in traj["instances_checked"]:
            g, W, beta = w.graphs[k], w.widths_sets[k], w.betas[k]
            th = torch.as_tensor(r["params"][r["offsets"][k]:r["offsets"][k + 1]].astype(np.float64))
            s = torch.as_tensor(r["spins"][k].astype(np.float64))
            lq_or = made.log_q(th, len(W), w.hidden, s).numpy()
            lz_or = oracle_log_zr(g, W, beta, s).detach().numpy()
            f_gpu = -float((r["logZR"][k] - r["logq"][k].astype(np.float64)).mean()) / beta
            f_or = -float((lz_or - lq_or).mean()) / beta
            fq = float(r["stats"][k][0]) / g.n
            rec["instances"].append({"instance": k, "L": g.Lx, "abs_dFq_rows_per_spin": abs(f_gpu - f_or) / g.n,
                                     "F_q_per_spin": fq, "F_exact_per_spin": f_ex[k],
                                     "abs_F_q_minus_F_exact_per_spin": abs(fq - f_ex[k])})
        out["checks"].append(rec)
    if "grad_check" in traj:
        out["grad_check_step1"] = oracle_grad_checks(w, traj["instances_checked"], traj["grad_check"])
    return out


def oracle_grad_checks(w, picks, gchk, n_dir=3, h=1e-4):
    """The Eq. 10 gradient at the first step against the oracle, per checked
    instance, on the GPU's own samples: the oracle's surrogate gradient (its
    own FP64 log q, log Z_R and weights) against the GPU backward (FP32: max
    |delta| / max |g|; BF16: relative Frobenius error and cosine), and central
    finite differences (step h) of the oracle's surrogate sum_b w_b log q_theta(s_b)
    along n_dir random unit directions v against g_FP32 . v."""
    import numpy as np
    import torch

    from oracle import estimators as est
    from oracle import made

    rng = np.random.default_rng(5)
    res = {"fp32_max_rel": 0.0, "bf16_max_rel_fro": 0.0, "bf16_min_cos": 1.0, "fd_max_rel": 0.0,
           "fd_step": h, "fd_directions": n_dir, "instances": len(picks)}
    for k in picks:
        g, W, beta = w.graphs[k], w.widths_sets[k], w.betas[k]
        D = len(W)
        o0, o1 = int(gchk["offsets"][k]), int(gchk["offsets"][k + 1])
        th = gchk["params"][o0:o1].astype(np.float64)
        for name, r in gchk["runs"].items():
            s = torch.as_tensor(r["spins"][k].astype(np.float64))
            lq = made.log_q(torch.as_tensor(th), D, w.hidden, s)
            lz = oracle_log_zr(g, W, beta, s).detach()
            wts = est.reinforce_weights(lz, lq, beta)
            ref = est.surrogate_grad(th, D, w.hidden, s, wts).numpy()
            gk = r["grad"][o0:o1].astype(np.float64)
            if name == "fp32":
                res["fp32_max_rel"] = max(res["fp32_max_rel"], float(np.abs(gk - ref).max() / np.abs(ref).max()))
                for _ in range(n_dir):
                    v = rng.normal(size=th.shape)
                    v /= np.linalg.norm(v)
                    fp = float((wts * made.log_q(torch.as_tensor(th + h * v), D, w.hidden, s)).sum())
                    fm = float((wts * made.log_q(torch.as_tensor(th - h * v), D, w.hidden, s)).sum())
                    fd = (fp - fm) / (2 * h)
                    res["fd_max_rel"] = max(res["fd_max_rel"], abs(float(gk @ v) - fd) / np.linalg.norm(ref))
            else:
                res["bf16_max_rel_fro"] = max(res["bf16_max_rel_fro"],
                                              float(np.linalg.norm(gk - ref) / np.linalg.norm(ref)))
                res["bf16_min_cos"] = min(res["bf16_min_cos"],
                                          float(gk @ ref / (np.linalg.norm(gk) * np.linalg.norm(ref))))
    res["note"] = ("fd_max_rel = |g_FP32 . v - FD| / |g_oracle| over the directions; the oracle's weights use "
                   "its own FP64 log q and log Z_R")
    return res


# ---------------------------------------------------------------------------
# the FP64 oracle as the CPU baseline / reference arm
# ---------------------------------------------------------------------------
def oracle_step(w, params, offsets, n_b, seed, step):
    """One oracle iteration of Algorithm 1 on n_b samples per instance."""
    import numpy as np
    import torch

    from oracle import estimators as est
    from oracle import made, philox, transfer

    done = 0
    for k, (g, W, beta) in enumerate(zip(w.graphs, w.widths_sets, w.betas)):
        D = len(W)
        th = torch.as_tensor(params[offsets[k]:offsets[k + 1]].astype(np.float64))
        u = philox.uniforms(seed, step, k, n_b, D)
        s, _ = made.sample(th, D, w.hidden, u)
        lq = made.log_q(th, D, w.hidden, s)
        bt = torch.tensor(beta, dtype=torch.float64, requires_grad=True)
        Jt = torch.tensor(g.J, dtype=torch.float64, requires_grad=True)
        lz = transfer.log_zr_lattice(g.n, g.ei, g.ej, Jt, bt, W, s, g.Lx)
        est.free_energies(lz.detach(), lq.detach(), beta)
        wts = est.reinforce_weights(lz.detach(), lq.detach(), beta)
        grad = est.surrogate_grad(th.numpy(), D, w.hidden, s, wts)
        torch.autograd.grad(lz.sum(), [bt, Jt])  # adjoint: d/dbeta and d/dJ
        est.adam_step(th.numpy(), grad.numpy(), np.zeros(th.numel()), np.zeros(th.numel()), 1)
        done += n_b
    return done


def oracle_parity(w, runs, check_stats=True):
    """Errors of the GPU step against the FP64 oracle, per precision: on the
    sampled rows of the GPU's own samples, max |delta log q| / N (the oracle's
    log q on the parameters the step sampled with), max |delta log Z_R| / N and
    |delta F_q| / N of those rows' mean; over the whole batch, the step's
    F_q / F_IS / stderr / log Z_IS rows against the oracle's estimators on the
    GPU's log q and log Z_R (the reduction's own error)."""
    import numpy as np
    import torch

    from oracle import estimators as est
    from oracle import made, transfer

    out = {}
    for r in runs:
        e_q = e_z = e_f = e_red = e_lz = 0.0
        for k, (g, W, beta) in enumerate(zip(w.graphs, w.widths_sets, w.betas)):
            D = len(W)
            th = torch.as_tensor(r["params"][r["offsets"][k]:r["offsets"][k + 1]].astype(np.float64))
            s = torch.as_tensor(r["spins"][k].astype(np.float64))
            lq_or = made.log_q(th, D, w.hidden, s).numpy()
            lz_or = transfer.log_zr_lattice(g.n, g.ei, g.ej, g.J, beta, W, s, g.Lx).numpy()
            lq = r["logq"][k][r["rows"]].astype(np.float64)
            lz = r["logZR"][k][r["rows"]]
            e_q = max(e_q, float(np.abs(lq - lq_or).max()) / g.n)
            e_z = max(e_z, float(np.abs(lz - lz_or).max()) / g.n)
            e_f = max(e_f, abs(float((lz - lq).mean() - (lz_or - lq_or).mean())) / beta / g.n)
            if check_stats:
                fe = est.free_energies(r["logZR"][k], r["logq"][k].astype(np.float64), beta)
                st = r["stats"][k]
                e_red = max(e_red, abs(st[0] - fe["F_q"]) / g.n, abs(st[1] - fe["F_IS"]) / g.n)
                e_lz = max(e_lz, abs(st[3] - fe["logZ_IS"]) / g.n)
        out[r["precision"]] = {
            "rows_per_instance": int(len(r["rows"])), "max_abs_dlogq_per_spin": e_q,
            "max_abs_dlogZR_per_spin": e_z, "abs_dFq_rows_per_spin": e_f,
            "reduction_max_abs_dF_per_spin": e_red if check_stats else None,
            "reduction_max_abs_dlogZ_IS_per_spin": e_lz if check_stats else None}
    out["tolerance_per_spin"] = {"fp32": 1e-6, "reduced_precision": 1e-3}
    return out


def oracle_ferro_exact(wf, ferro):
    """Exact F / N of the open ferromagnet at each temperature (the oracle's
    Kac-Ward determinant) and the relative errors of the trained F_q and F_IS."""
    from oracle import kacward

    g = wf.graphs[0]
    L = int(round(g.n ** 0.5))
    f_ex = [-kacward.log_z_kac_ward(L, L, g.ei, g.ej, g.J, b) / b / g.n for b in wf.betas]
    return {"F_exact_per_spin": f_ex, "exact": "Kac-Ward determinant (oracle, FP64)",
            "rel_err_F_q": [abs(f - e) / abs(e) for f, e in zip(ferro["F_q_per_spin"], f_ex)],
            "rel_err_F_IS": [abs(f - e) / abs(e) for f, e in zip(ferro["F_IS_per_spin"], f_ex)]}


def oracle_exact_f(w):
    """Exact F / N of each instance from the oracle's single-site transfer matrix."""
    from oracle import transfer

    out = []
    for g, beta in zip(w.graphs, w.betas):
        lz = float(transfer.log_z_helical(g.Lx, g.Ly, g.ei, g.ej, g.J, beta))
        out.append(-lz / beta / g.n)
    return out


def cpu_baseline(w, params, offsets, budget_s=15.0, n_b=2048):
    """The oracle, as it stands, on a bounded sample of the workload: repeated
    oracle steps of n_b samples per beta until about budget_s has elapsed."""
    import torch

    torch.set_num_threads(os.cpu_count() or 1)
    done, steps = 0, 0
    t0 = time.perf_counter()
    while True:
        done += oracle_step(w, params, offsets, n_b, 1, steps)
        steps += 1
        dt = time.perf_counter() - t0
        if dt >= budget_s or steps >= 50:
            break
    return {"value": done / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{steps} oracle steps x {n_b} samples per beta x {len(w.graphs)} betas "
                      f"(FP64 sampling replay, strip transfer matrices, estimators, autograd gradient "
                      f"and adjoint, Adam) in {dt:.1f} s"}


def headline_config(w, batch_per_beta):
    """The 16x16 workload's configuration keys both arms report."""
    return {"workload": w.name, "lattice": "16x16 open", "couplings": "N(0,1)", "betas": w.betas,
            "batch_per_beta": batch_per_beta, "instances": len(w.graphs),
            "width_set": "every 4th column (64 spins)", "made": [64] + w.hidden + [64],
            "step": "sample+contract+reduce+REINFORCE backward+d/dbeta+d/dJ+Adam"}


def run_reference(a):
    import numpy as np

    from paper_2504_12037_gb300 import workloads as wl

    rank, world, local = dist_env()
    if rank != 0:
        return
    w = wl.workload(CONFIG)
    params = np.concatenate([wl.made_params(len(W), w.hidden, 1 + k) for k, W in enumerate(w.widths_sets)])
    sizes = [wl.made_param_count(len(W), w.hidden) for W in w.widths_sets]
    offsets = np.concatenate([[0], np.cumsum(sizes)])
    import torch

    torch.set_num_threads(os.cpu_count() or 1)
    n_b = 16
    for i in range(a.warmup):
        oracle_step(w, params, offsets, n_b, 1, i)
    t0 = time.perf_counter()
    done = 0
    for i in range(a.steps):
        done += oracle_step(w, params, offsets, n_b, 1, a.warmup + i)
    dt = time.perf_counter() - t0
    value = done / dt
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {**headline_config(w, w.batch), "precision": "fp64 (the oracle, as it stands)",
                      "timing": "host cores, wall clock; each step a bounded sample of the workload's batch",
                      "parallelism": "host threads"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                            "sample": f"{n_b} of the {w.batch} samples per beta x {len(w.graphs)} betas per step"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    a = args_()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload != CONFIG:
        run_workload(a)
    else:
        run_ours(a)
