#!/usr/bin/env python3
"""Benchmark: signals/s to a certified KKT tolerance of 1e-6 for batch-mode MPL.

One step = one bmpl_solve of the whole batch (every outer iteration of every
signal until each is certified), inputs resident in HBM when timing starts.
Default workload: the large mixed-precision batch (A 4096 x 65536 Gaussian,
unit-norm atoms, p = 1024 signals, k ~ U[100, 400], N(0, 1) values,
sigma = 1e-3, lambda_i = 0.01 ||A^T b_i||_inf, rho = 100, active sets up to
1024 atoms), the largest single-GPU batch of the method's workloads.  The
reported path is BF16 correlation + learned warm start; plain FP32 without the
warm start is timed alongside under the same autotuner policy.  The first 64
signals are also solved by the FP64 oracle, which gives the per-result error
and the host-core baseline.

Prints one JSON line.  Under torchrun each rank solves its own batch (the
signals are independent, eq. 3), so scaling is weak and there is no collective
on the data path; rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "signals/sec to KKT tol 1e-6 (mixed+warm-start vs plain FP32 BMPL, 1 GB300)"
UNIT = "signals/s"
TOL = 1e-6
FP32_LANES_PER_SM = 128

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the kernels the roofline block
# can report, per workload, from an ncu capture of the current kernel; absent until one exists.
TRAFFIC = {
    # all k_finish launches of one solve of the 4096 x 65536 batch: 534.6 MB read + 5.3 MB
    # written over the 9 launches of a 64-signal solve (8.44 MB per signal), scaled to 1024
    # signals (per-signal work is independent of the batch); per step, like the entry's
    # bytes_per_step
    ("c3", "k_finish"): 8.64e9,
}

# active-set capacity per workload (supports reach ~570 atoms on c3, ~290 on c5)
SMAX = {"c1": None, "c2": None, "c3": 1024, "c4": 512, "c5": 512}
# signals of the disjoint training stream for the warm-start proposal
TRAIN_SIGNALS = {"c1": 256, "c2": 16384, "c3": 8192, "c4": 8192, "c5": 50000}
# signals per step of the reference arm (the FP64 oracle on the host cores)
REF_SIGNALS = {"c1": 1, "c2": 64, "c3": 16, "c4": 64, "c5": 32}
# signals the oracle solves for the per-result error and the CPU baseline
ERR_SIGNALS = 64


def workload_desc(cfg: str, P, path: str) -> dict:
    meta = P.meta
    if "classes" in meta:
        what = (f"{cfg}: A = [D I] {P.n}x{P.m}, D {meta['classes']} classes x {meta['per_class']} atoms of "
                f"rank-{meta['rank']} subspaces (pixel-like, unit norm), I for occlusion; p={P.p} queries with "
                f"{int(100 * meta['corrupt'])}% of pixels corrupted")
    else:
        what = (f"{cfg}: A {P.n}x{P.m} Gaussian unit-norm atoms, p={P.p} signals, "
                f"k~U[{meta.get('kmin')},{meta.get('kmax')}], sigma={meta.get('sigma')}")
    return {
        "workload": f"{what}, lambda_i={meta.get('lam_frac')}*||A^T b_i||_inf, rho={P.rho}, tol={TOL}",
        "n": P.n, "m": P.m, "p": P.p, "rho": P.rho, "tol": TOL, "path": path,
        "l2": "flushed between timed steps (256 MiB write)",
    }


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def rank_problem(synth, cfg: str, rank: int, p=None, seed_shift: int = 0):
    """Rank r's batch: the shared dictionary and its own signals (the generator's signal
    seed moves by 1000 per rank), so the ranks solve disjoint independent problems."""
    return synth.make_config(cfg, p=p, seed_shift=seed_shift + 1000 * rank)


def max_over_ranks(x: float, dist, device) -> float:
    """Slowest rank's figure (seconds or ms); x itself on one process."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, p: int, steps: int, seconds: float) -> float:
    """Whole-job signals/s: every rank solved p signals per step."""
    return world * p * steps / seconds


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
            "source": "fallback"}


def cpu_baseline(cfg: str, P, max_signals: int, single_signals: int = None) -> tuple:
    """The FP64 oracle on the host cores over the first signals of the batch (OpenMP across
    signals), and on one core over fewer.  Returns (baseline entry, oracle solutions of the
    all-cores sample)."""
    import oracle
    k = min(P.p, max_signals)
    idx = np.arange(k)
    threads = oracle.num_threads()
    t0 = time.perf_counter()
    Xo, _ = oracle.bmpl(P.At, P.B[idx], P.lam[idx], P.rho, threads=threads)
    dt = time.perf_counter() - t0
    # the paper's convention is one core: the same oracle on one thread, a smaller sample
    k1 = min(k, single_signals if single_signals else (32 if P.n * P.m <= (1 << 24) else 4))
    t1 = time.perf_counter()
    oracle.bmpl(P.At, P.B[:k1], P.lam[:k1], P.rho, threads=1)
    dt1 = time.perf_counter() - t1
    extra = (f"; rate extrapolated linearly to the whole batch of {P.p} (signals are independent): "
             f"{P.p / (k / dt):.1f} s estimated" if k < P.p else "")
    entry = {"value": k / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
             "sample": f"first {k} of the {P.p} signals of {cfg}, FP64 Algorithm 1 with exact finish, "
                       f"OpenMP over signals, {dt:.2f} s wall{extra}",
             "extrapolated": k < P.p,
             "single_core": {"value": k1 / dt1, "unit": UNIT, "cores": 1,
                             "sample": f"first {k1} signals of {cfg}, one thread, {dt1:.2f} s wall"}}
    return entry, Xo


def error_vs_oracle(P, X64, Xo) -> dict:
    """Per-result error of the GPU solutions against the FP64 oracle on the same signals:
    relative objective difference, relative Frobenius error of X and support mismatches
    (coefficients above 1e-3 max|x|), with the acceptance tolerances."""
    k = Xo.shape[0]
    A64 = P.At.astype(np.float64)
    rel_obj = []
    mism_sig, mism_ent = 0, 0
    for i in range(k):
        b = P.B[i].astype(np.float64)
        lam = float(P.lam[i])
        def f(x):
            r = b - A64.T @ x
            return lam * np.abs(x).sum() + 0.5 * r @ r
        fo = f(Xo[i])
        rel_obj.append(abs(f(X64[i]) - fo) / abs(fo) if fo != 0 else abs(f(X64[i])))
        xm = np.abs(Xo[i]).max()
        sg = np.abs(X64[i]) > 1e-3 * xm
        so = np.abs(Xo[i]) > 1e-3 * xm
        d = int(np.count_nonzero(sg ^ so))
        mism_ent += d
        mism_sig += int(d > 0)
    den = np.linalg.norm(Xo)
    xrel = float(np.linalg.norm(X64 - Xo) / den) if den > 0 else float(np.linalg.norm(X64))
    ro = float(max(rel_obj)) if rel_obj else 0.0
    return {"signals": k, "rel_objective_max": ro, "x_rel_fro": xrel, "support_mismatch_signals": mism_sig,
            "support_mismatch_entries": mism_ent,
            "tolerances": {"rel_objective": 1e-6, "x_rel_fro": 1e-4, "support_frac": 1e-3},
            "within": bool(ro <= 1e-6 and xrel <= 1e-4 and mism_sig == 0)}


def run_reference(args, rank: int, world: int) -> None:
    """The oracle as the reference arm (CPU, rank 0 only): each step solves a bounded sample
    of the workload's signals on the host cores; signals/s is that sample's rate."""
    if rank != 0:
        return
    from paper_1302_5010_gb300 import synth
    import oracle
    P = synth.make_config(args.config)
    k = min(P.p, args.ref_signals or REF_SIGNALS.get(args.config, 16))
    threads = oracle.num_threads()
    for _ in range(args.warmup):
        oracle.bmpl(P.At, P.B[:1], P.lam[:1], P.rho, threads=threads)
    times = []
    for s in range(args.steps):
        idx = (np.arange(k) + s * k) % P.p
        t0 = time.perf_counter()
        oracle.bmpl(P.At, P.B[idx], P.lam[idx], P.rho, threads=threads)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = k * args.steps / tot
    sample = (f"{k} of the {P.p} signals of {args.config} per step (consecutive slices), FP64 Algorithm 1 "
              f"with exact finish, OpenMP over signals; signals are independent, so the rate stands for "
              f"the whole batch")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": workload_desc(args.config, P, "oracle-fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def correlation_microbench(args) -> None:
    """The correlation GEMM alone (worst-case analysis product A^T R) on an
    n x m dictionary and p residuals, through mpl_correlate; for profiling."""
    import torch
    from paper_1302_5010_gb300 import mpl
    n, m, p = args.corr_shape
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((m, n), device="cuda", generator=g)
    A /= A.norm(dim=1, keepdim=True)
    R = torch.randn((p, n), device="cuda", generator=g) * 0.3
    s = mpl.Solver(A, precision=1 if args.path == "mixed" else 0,
                   **({"gemm_tile": args.gemm_tile} if args.path == "mixed" else {}))
    C = torch.empty((p, m), device="cuda")
    for _ in range(max(args.warmup, 1)):
        s.correlate(R, C)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        s.correlate(R, C)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"microbench": "correlation", "path": args.path, "n": n, "m": m, "p": p,
                      "gemm_tile": args.gemm_tile if args.path == "mixed" else None,
                      "ms_per_call": ms, "tflops_incl_staging": 2.0 * n * m * p / ms / 1e9}))
    s.close()


def train_proposal(args, mpl, torch, solver, P_train, dev) -> dict:
    """Offline (untimed): solve a disjoint training stream of signals with the cold
    solver, then train the warm-start proposal on their supports."""
    t0 = time.perf_counter()
    Bt = torch.from_numpy(P_train.B).to(dev)
    lt = torch.from_numpy(P_train.lam).to(dev)
    Xt = torch.zeros((P_train.p, P_train.m), dtype=torch.float32, device=dev)
    res = solver.solve(Bt, lt, Xt, TOL)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = solver.train_proposal(Bt, lt, Xt, epochs=args.train_epochs)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return {"signals": P_train.p, "solve_s": t1 - t0, "train_s": t2 - t1, "epochs": args.train_epochs,
            "loss_first": float(losses[0]) if len(losses) else None,
            "loss_last": float(losses[-1]) if len(losses) else None,
            "labels_certified": bool(np.all(res.stats["status"] == mpl.MPL_SIG_CERTIFIED)),
            "outer_iters_cold_mean": float(np.mean(res.stats["outer_iters"]))}


def kernel_rooflines(P, precision: int, phase: dict, work: dict, pk: dict, sms: int) -> dict:
    """Roofline entry of each phase's kernel: algorithmic work (device-counted FLOPs or bytes)
    over the kernel's CUDA-event time inside the timed steps, against the measured peak of the
    unit that bounds it (HBM copy bandwidth, dense BF16, or the FP32 FMA rate from unit counts
    and the maximum SM clock)."""
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    fp32_note = f"FP32 FMA: {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 FLOP x max SM clock (nominal units)"
    hbm = pk["hbm_gbs"]
    hbm_note = f"HBM copy bandwidth, of {pk['source']}"
    out = {}

    def entry(kernel, bound, amount, ms, peak, unit, note, amount_key):
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ach = amount / (ms / 1e3) / scale if ms > 0 else 0.0
        return {"kernel": kernel, "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                "frac": ach / peak if peak else None, "peak_note": note, "ms_per_step": ms, amount_key: amount}

    cols = work["gemm_columns"]
    flops = 2.0 * P.n * P.m * cols
    if precision == 0:
        out["correlation"] = entry("k_corr_f32", "alu", flops, phase["correlation"], fp32_peak, "TFLOP/s",
                                   fp32_note, "flop_per_step")
    else:
        out["correlation"] = entry("k_corr_bf16", "tensor", flops, phase["correlation"], pk["bf16_tflops"],
                                   "TFLOP/s", f"dense bf16 burst, of {pk['source']}", "flop_per_step")
    out["correlation"]["identity_route_ms_per_step"] = phase.get("qroute", 0.0)
    out["correlation"]["identity_route_columns_per_step"] = work["qroute_columns"]
    # the finish streams the support's atom columns (exact residuals and correlations) and
    # Gram rows (its solves): at peak its bytes take longer than its FP32 work, so HBM bounds it
    out["finish"] = entry("k_finish", "hbm", work["finish_bytes"], phase["finish"], hbm, "GB/s",
                          hbm_note + "; one CTA per signal, latency-bound sweeps", "bytes_per_step")
    out["finish"]["flop_per_step"] = work["finish_flops"]
    if work["apg_global_elems"] > 0.5 * work["apg_elems"]:
        out["master"] = entry("k_apg", "hbm", 4.0 * work["apg_global_elems"], phase["master"], hbm, "GB/s",
                              hbm_note + "; Gram blocks above the shared-memory size streamed per product",
                              "bytes_per_step")
    else:
        out["master"] = entry("k_apg", "alu", 2.0 * work["apg_elems"], phase["master"], fp32_peak, "TFLOP/s",
                              fp32_note + "; Gram blocks resident in shared memory", "flop_per_step")
    out["selection"] = entry("k_select", "hbm", 4.0 * P.m * cols, phase["selection"], hbm, "GB/s",
                             hbm_note + "; one read of the score rows (the re-score band and any second "
                                        "pass come on top)", "bytes_per_step")
    out["residual"] = entry("k_residual", "hbm", work["residual_bytes"], phase["residual"], hbm, "GB/s",
                            hbm_note, "bytes_per_step")
    out["gram"] = entry("k_gram_gather" if work["qgram"] else "k_gram_async", "hbm", work["gram_bytes"],
                        phase["gram"], hbm, "GB/s", hbm_note, "bytes_per_step")
    return out


def timed_path(args, mpl, torch, P, dev, precision: int, world: int, dist, local: int, warm: bool = False,
               P_train=None, smax=None, want_x64: int = 0) -> dict:
    """Warm up, then time exactly args.steps solves of the whole batch (device events, L2
    flushed between steps), then the same through the C ABI with pinned host buffers."""
    At = torch.from_numpy(P.At).to(dev)
    B = torch.from_numpy(P.B).to(dev)
    lam = torch.from_numpy(P.lam).to(dev)
    X = torch.empty((P.p, P.m), dtype=torch.float32, device=dev)
    opts = {"smax": smax} if smax else {}
    solver = mpl.Solver(At, rho=P.rho, precision=precision, **opts)
    training = None
    if warm:
        training = train_proposal(args, mpl, torch, solver, P_train, dev)
        solver.set(mpl.MPL_OPT_WARM_START, 2)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2
    stream = torch.cuda.current_stream()
    # one-time tuning on the batch (identity route, handshake cadence, Gram from Q), like the layout
    # work of mpl_create it is outside the timed region
    tune = None
    if args.tune:
        vals = [int(v) for v in args.tune.split(",")]
        qr, se, qg = (vals + [0])[:3]
        solver.set(mpl.MPL_OPT_QROUTE, qr)
        solver.set(mpl.MPL_OPT_SYNC_EVERY, se)
        solver.set(mpl.MPL_OPT_QGRAM, qg)
        tune = {"qroute": qr, "sync_every": se, "qgram": qg, "fixed": True}
    elif not args.no_autotune:
        tune = solver.autotune(B, lam, TOL, stream)
    nph = 16

    def timed_steps(profile: bool, clocks=None):
        """W untimed solves (they capture the iteration graphs of this mode), then exactly
        args.steps solves timed by device events, the L2 flushed before each."""
        solver.set(mpl.MPL_OPT_PROFILE, 1 if profile else 0)
        for _ in range(args.warmup):
            solver.solve(B, lam, X, TOL, stream)
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        step_ms, phase_tot, launches, certified = [], np.zeros(nph), 0, True
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(args.steps):
            flush.fill_(1.0)
            ev0.record(stream)
            rc = mpl.bmpl_solve(solver.h, B, P.p, lam, X, TOL, stream)
            ev1.record(stream)
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            ph = np.zeros(nph)
            v = mpl.mpl_get_phase_times(solver.h)
            ph[:len(v)] = v
            phase_tot += ph
            launches += solver.launches()
            st = mpl.mpl_get_stats(solver.h, P.p)
            certified &= bool(rc == mpl.MPL_OK and np.all(st["status"] == mpl.MPL_SIG_CERTIFIED))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        return step_ms, phase_tot, launches, certified, clk

    # the reported time: plain graph replays, nothing but the solve in the timed region
    clocks = ClockSampler(local)
    step_ms, _, launches, certified, clk = timed_steps(False, clocks)
    tot_ms = max_over_ranks(float(sum(step_ms)), dist, dev)
    value = aggregate_rate(world, P.p, args.steps, tot_ms / 1e3)
    # the kernels' own times for the roofline: the same steps again with event nodes around
    # every phase in the captured graphs
    prof_ms, phase_tot, _, certified_p, _ = timed_steps(True)
    certified &= certified_p
    X64 = None
    if want_x64:
        # the certified FP64 iterates of the first signals, for the error against the oracle
        Xd = torch.zeros((P.p, P.m), dtype=torch.float64, device=dev)
        solver.solution_f64(Xd)
        X64 = Xd[:want_x64].cpu().numpy()
        del Xd

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    solver.set(mpl.MPL_OPT_PROFILE, 0)
    Bh = torch.from_numpy(P.B).pin_memory()
    lamh = torch.from_numpy(P.lam).pin_memory()
    Xh = torch.zeros((P.p, P.m), dtype=torch.float32).pin_memory()
    mpl.bmpl_solve(solver.h, Bh, P.p, lamh, Xh, TOL, stream)  # same graphs, staged inputs
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        mpl.bmpl_solve(solver.h, Bh, P.p, lamh, Xh, TOL, stream)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    nbytes = lambda t: t.numel() * t.element_size()
    e2e = {"value": aggregate_rate(world, P.p, args.steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(nbytes(Bh) + nbytes(lamh)), "d2h_bytes_per_step": int(nbytes(Xh))}
    stats = mpl.mpl_get_stats(solver.h, P.p)
    qgram = int(solver.get(mpl.MPL_OPT_QGRAM))
    solver.close()
    del flush
    # roofline of every phase's kernel; the one with the most time per step is the dominant one
    pk = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    names = ["total", "correlation", "selection", "gram", "finish", "master", "residual"]
    phase = {nm: phase_tot[i] / args.steps for i, nm in enumerate(names)}
    phase["qroute"] = phase_tot[10] / args.steps
    work = {"gemm_columns": (phase_tot[7] - phase_tot[9]) / args.steps, "qroute_columns": phase_tot[9] / args.steps,
            "finish_flops": phase_tot[8] / args.steps, "apg_elems": phase_tot[11] / args.steps,
            "apg_global_elems": phase_tot[12] / args.steps, "residual_bytes": phase_tot[13] / args.steps,
            "gram_bytes": phase_tot[14] / args.steps, "finish_bytes": phase_tot[15] / args.steps, "qgram": qgram}
    kern = kernel_rooflines(P, precision, phase, work, pk, sms)
    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    roof = dict(kern[dom])
    tr = TRAFFIC.get((args.config, roof["kernel"]))
    roof["traffic"] = tr
    roof["traffic_unit"] = "bytes per step (all launches of the kernel in one solve)"
    # summed event times per phase (the finish runs on a second stream, so phases overlap)
    roof["phase_ms_per_step"] = {k: round(v, 4) for k, v in phase.items() if v > 0}
    roof["events_pass_ms_per_step"] = float(sum(prof_ms)) / args.steps
    return {"value": value, "tot_ms": tot_ms, "e2e": e2e, "launches": launches, "clocks": clk, "autotune": tune,
            "certified": certified, "roofline": roof, "gemm": kern["correlation"], "kernels": kern,
            "training": training, "X64": X64,
            "outer_iters_mean": float(np.mean(stats["outer_iters"])),
            "active_size_mean": float(np.mean(stats["active_size"]))}


def solve_once(args):
    """Profiling target: args.warmup solves (graph capture, Q build), then one solve of the
    workload args.solve_once (first args.solve_p signals) with fixed options, printing the
    kernel launches of each so that an ncu capture can skip the warm-up."""
    import torch
    from paper_1302_5010_gb300 import mpl, synth
    P = synth.make_config(args.solve_once, p=args.solve_p)
    dev = torch.device("cuda", 0)
    At = torch.from_numpy(P.At).to(dev)
    B = torch.from_numpy(P.B).to(dev)
    lam = torch.from_numpy(P.lam).to(dev)
    opts = dict(qgram=args.solve_qgram, graph=args.solve_graph, sync_every=args.solve_sync,
                qroute=args.solve_qroute, reentry=args.solve_reentry, omega=args.solve_omega)
    if SMAX.get(args.solve_once):
        opts["smax"] = SMAX[args.solve_once]
    if args.path == "mixed":
        opts["gemm_tile"] = args.gemm_tile
    s = mpl.Solver(At, rho=P.rho, precision=1 if args.path == "mixed" else 0, **opts)
    X = torch.empty((P.p, P.m), dtype=torch.float32, device=dev)
    before = 0
    for _ in range(args.warmup):
        s.solve(B, lam, X, TOL)
        torch.cuda.synchronize()
        before += s.launches()
    r = s.solve(B, lam, X, TOL)
    torch.cuda.synchronize()
    if args.solve_train > 0:
        # the warm start's proposal network trained on the solved batch (its training kernels)
        s.train_proposal(B, lam, X, epochs=args.solve_train)
        torch.cuda.synchronize()
    print(json.dumps({"solve_once": args.solve_once, "p": P.p, "path": args.path, "options": opts,
                      "launches_before": before, "launches": s.launches(),
                      "certified": int(np.sum(r.stats["status"] == mpl.MPL_SIG_CERTIFIED))}), flush=True)
    s.close()


def omp_compare(args):
    """lambda = 0 (least squares on the growing support, the reduction to orthogonal matching
    pursuit in Sec. 2.5) on the shape of the paper's Sec. 5.1 batch comparison: A 4096 x 16384
    Gaussian, k ~ U[400, 600], sigma = 1e-3, every signal stopped by ||xi|| <= r_2 (eq. stop1)
    at 1.5 sigma sqrt(n).  rho = 1 is batch OMP (one atom per worst-case analysis, the Gram
    block read from Q = A^T A); the multi-atom rows add rho atoms per analysis as Algorithm 1
    does.  One JSON line per run (warm-up solve, then one event-timed solve)."""
    import torch
    from paper_1302_5010_gb300 import mpl, synth
    P = synth.small_problem(4096, 16384, args.omp_compare, 400, 600, rho=1, lam_frac=0.0, sigma=1e-3, seed=51)
    r2 = 1.5 * 1e-3 * np.sqrt(P.n)
    dev = torch.device("cuda", 0)
    At = torch.from_numpy(P.At).to(dev)
    B = torch.from_numpy(P.B).to(dev)
    lam = torch.zeros(P.p, dtype=torch.float32, device=dev)
    Xt = P.X_true.astype(np.float64)
    supp_true = [set(np.flatnonzero(Xt[i]).tolist()) for i in range(P.p)]
    for rho in (1, 25, 50, 100):
        s = mpl.Solver(At, rho=rho, precision=1, smax=1024, stop_r2=r2, qgram=1, max_outer=1024)
        X = torch.empty((P.p, P.m), dtype=torch.float32, device=dev)
        s.solve(B, lam, X)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = s.solve(B, lam, X)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        X64 = np.zeros((P.p, P.m))
        s.solution_f64(X64)
        st = r.stats
        exact = sum(set(np.flatnonzero(X64[i]).tolist()) == supp_true[i] for i in range(P.p))
        rel = float(np.linalg.norm(X64 - Xt) / np.linalg.norm(Xt))
        res = np.linalg.norm(P.B.astype(np.float64) - X64 @ P.At.astype(np.float64), axis=1)
        print(json.dumps({"metric": "lambda = 0, 4096 x 16384, k~U[400,600]: time to ||xi|| <= r2",
                          "rho": rho, "p": P.p, "ms": round(ms, 2), "signals_per_s": round(P.p / ms * 1e3, 1),
                          "outer_mean": float(st["outer_iters"].mean()), "outer_max": int(st["outer_iters"].max()),
                          "early_stopped": int(np.sum(st["status"] == mpl.MPL_SIG_EARLY_STOP)),
                          "support_exact": int(exact), "rel_error_vs_x_true": rel,
                          "max_residual_over_r2": float(res.max() / r2), "S_mean": float(st["active_size"].mean())}),
              flush=True)
        s.close()


def streaming_warm_vs_cold(args, mpl, torch, dev) -> dict:
    """The streaming workload (2048 x 32768, 4096 signals arriving in batches of 512): every
    batch solved to the KKT tolerance by the mixed path, cold and with the learned warm
    start, the proposal trained on 50000 signals of the same generator (disjoint seed)
    solved and certified by the same solver.  Each mode: one untimed pass over the batches
    (graph capture), then one pass timed by device events per batch."""
    cfg = "c5"
    P = rank_problem(synth_mod(), cfg, 0)
    ntrain = args.c5_train or TRAIN_SIGNALS[cfg]
    Pt = rank_problem(synth_mod(), cfg, 0, p=ntrain, seed_shift=9000)
    At = torch.from_numpy(P.At).to(dev)
    B = torch.from_numpy(P.B).to(dev)
    lam = torch.from_numpy(P.lam).to(dev)
    bs = 512
    solver = mpl.Solver(At, rho=P.rho, precision=1, smax=SMAX[cfg])
    stream = torch.cuda.current_stream()
    X = torch.empty((bs, P.m), dtype=torch.float32, device=dev)
    tune = solver.autotune(B[:bs], lam[:bs], TOL, stream)

    def one_pass(timed: bool):
        ms, outer, cert = [], [], True
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for c0 in range(0, P.p, bs):
            ev0.record(stream)
            res = solver.solve(B[c0:c0 + bs], lam[c0:c0 + bs], X, TOL, stream)
            ev1.record(stream)
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
            outer.append(res.stats["outer_iters"].astype(np.float64))
            cert &= bool(res.status == mpl.MPL_OK and np.all(res.stats["status"] == mpl.MPL_SIG_CERTIFIED))
        o = np.concatenate(outer)
        return {"signals_per_s": P.p / (sum(ms) / 1e3), "ms_per_batch": float(np.mean(ms)),
                "outer_iters_mean": float(o.mean()), "outer_iters_max": int(o.max()), "certified_all": cert}

    one_pass(False)
    cold = one_pass(True)
    # training stream: solved cold in chunks, then the proposal trained on its supports
    t0 = time.perf_counter()
    Bt = torch.from_numpy(Pt.B).to(dev)
    lt = torch.from_numpy(Pt.lam).to(dev)
    Xt = torch.zeros((Pt.p, Pt.m), dtype=torch.float32, device=dev)
    labels_ok = True
    for c0 in range(0, Pt.p, 4096):
        r = solver.solve(Bt[c0:c0 + 4096], lt[c0:c0 + 4096], Xt[c0:c0 + 4096], TOL, stream)
        labels_ok &= bool(np.all(r.stats["status"] == mpl.MPL_SIG_CERTIFIED))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    losses = solver.train_proposal(Bt, lt, Xt, epochs=args.train_epochs)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    del Xt
    solver.set(mpl.MPL_OPT_WARM_START, 2)
    one_pass(False)
    warm = one_pass(True)
    warm["active"] = bool(solver.get(mpl.MPL_OPT_WARM_CANDIDATES) > P.rho)
    solver.close()
    return {"workload": "c5: A 2048x32768 Gaussian, 4096 signals in batches of 512, k~U[50,200], rho 50",
            "cold": cold, "warm": warm, "speedup_warm_vs_cold": warm["signals_per_s"] / cold["signals_per_s"],
            "autotune": tune,
            "training": {"signals": Pt.p, "labels_certified": labels_ok, "solve_s": t1 - t0, "train_s": t2 - t1,
                         "epochs": args.train_epochs, "loss_first": float(losses[0]) if len(losses) else None,
                         "loss_last": float(losses[-1]) if len(losses) else None}}


def synth_mod():
    from paper_1302_5010_gb300 import synth
    return synth


def big_dictionary_run(args):
    """Single-signal MPL and SMPL (omega = 3) on the big dictionary of the paper's Sec. 4.6:
    A 2^12 x 2^20 Gaussian (16 GiB in FP32, drawn on the device), a k-sparse N(0, 1) code,
    noise U[-0.01, 0.01], lambda = 0.005 ||A^T b||_inf and the stopping rule of eq. (stop_con)
    at 1e-5, as in the paper's experiments (Sec. 4.1).  With one signal every correlation is
    a matrix-vector product over the whole dictionary.  For each path (mixed BF16, plain
    FP32) and omega: a warm-up solve, then args.steps solves timed by device events, then one
    solve with event nodes around the phases.  One JSON line each (not a bench line)."""
    import torch
    from paper_1302_5010_gb300 import mpl, synth

    assert torch.cuda.is_available(), "needs a CUDA device"
    dev = torch.device("cuda", 0)
    n, m = args.big_shape
    t0 = time.perf_counter()
    At, b, lam, supp, vals = synth.big_dictionary_device(n, m, args.big_k, device="cuda")
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    x_true = torch.zeros(m, dtype=torch.float64, device=dev)
    x_true[supp] = vals
    stream = torch.cuda.current_stream()
    for precision in (1, 0):
        for omega in (1, 3):
            s = mpl.Solver(At, rho=args.big_rho, precision=precision, smax=1024, stop_eps=1e-5, omega=omega)
            X = torch.empty((1, m), dtype=torch.float32, device=dev)
            res = s.solve(b, lam, X, TOL, stream)  # warm-up: BF16 copy, graphs
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ms = []
            for _ in range(max(args.steps, 1)):
                ev0.record(stream)
                res = s.solve(b, lam, X, TOL, stream)
                ev1.record(stream)
                ev1.synchronize()
                ms.append(ev0.elapsed_time(ev1))
            s.set(mpl.MPL_OPT_PROFILE, 1)
            s.solve(b, lam, X, TOL, stream)
            torch.cuda.synchronize()
            ph = s.phase_times()
            s.set(mpl.MPL_OPT_PROFILE, 0)
            X64 = torch.zeros((1, m), dtype=torch.float64, device=dev)
            s.solution_f64(X64)
            st = res.stats
            err = float(torch.linalg.vector_norm(X64[0] - x_true) / torch.linalg.vector_norm(x_true))
            found = torch.abs(X64[0]) > 1e-3 * torch.abs(X64[0]).max()
            hit = int(found[supp].sum())
            iters = int(st["outer_iters"][0])
            # the correlation reads the whole dictionary once per outer iteration
            corr_bytes = float(iters) * m * n * (2 if precision == 1 else 4)
            print(json.dumps({
                "big_dictionary": f"{n}x{m}", "k": args.big_k, "rho": args.big_rho, "omega": omega,
                "path": "mixed" if precision == 1 else "plain", "lam": float(lam[0]),
                "ms_per_solve": float(np.median(ms)), "ms_all": [round(v, 3) for v in ms],
                "status": int(st["status"][0]), "outer_iters": iters,
                "active_size": int(st["active_size"][0]), "nnz": int(st["nnz"][0]),
                "rel_err_vs_planted": err, "planted_found": hit, "support_size": int(found.sum()),
                "phase_ms": {k: round(float(ph[k]), 3) for k in ("correlation", "selection", "gram", "finish",
                                                                 "master", "residual")},
                "correlation_gbs": corr_bytes / (ph["correlation"] / 1e3) / 1e9 if ph["correlation"] > 0 else None,
                "generate_s": gen_s}), flush=True)
            s.close()
            del X, X64


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--config", default="c3")
    ap.add_argument("--path", default="mixed", choices=["plain", "mixed"],
                    help="path reported as value; the other one is timed alongside for comparison")
    ap.add_argument("--no-warm", action="store_true", help="report the reported path without the learned warm start")
    ap.add_argument("--train-signals", type=int, default=None)
    ap.add_argument("--train-epochs", type=int, default=4)
    ap.add_argument("--no-compare", action="store_true", help="skip the comparison path")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default route and handshake cadence")
    ap.add_argument("--tune", default=None, metavar="QROUTE,SYNC[,QGRAM]",
                    help="fix the tuned settings instead of running the autotuner (profiling runs)")
    ap.add_argument("--ref-signals", type=int, default=None)
    ap.add_argument("--cpu-signals", type=int, default=ERR_SIGNALS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--corr-shape", type=int, nargs=3, metavar=("N", "M", "P"), default=None,
                    help="profile the correlation GEMM alone on this shape instead of the benchmark")
    ap.add_argument("--gemm-tile", type=int, default=256, choices=[64, 128, 256],
                    help="signals per tile of the BF16 GEMM in the correlation microbenchmark")
    ap.add_argument("--omp-compare", type=int, default=0, metavar="P",
                    help="lambda = 0 on the 4096 x 16384, k 400-600 shape for P signals: rho = 1 (batch "
                         "OMP) against multi-atom growth, instead of the benchmark")
    ap.add_argument("--no-c5", action="store_true", help="skip the streaming warm-vs-cold measurement")
    ap.add_argument("--c5-only", action="store_true", help="only the streaming warm-vs-cold measurement")
    ap.add_argument("--c5-train", type=int, default=None, help="training signals of the streaming measurement")
    ap.add_argument("--big-dict", action="store_true",
                    help="single-signal MPL / SMPL on the paper's 2^12 x 2^20 big dictionary instead of the benchmark")
    ap.add_argument("--big-shape", type=int, nargs=2, default=[4096, 1 << 20], metavar=("N", "M"))
    ap.add_argument("--big-k", type=int, default=600)
    ap.add_argument("--big-rho", type=int, default=50)
    ap.add_argument("--solve-once", default=None, metavar="CFG",
                    help="profiling target: --warmup solves, then one solve of workload CFG")
    ap.add_argument("--solve-p", type=int, default=None, help="signals of the --solve-once workload")
    ap.add_argument("--solve-qgram", type=int, default=1)
    ap.add_argument("--solve-graph", type=int, default=1)
    ap.add_argument("--solve-sync", type=int, default=4)
    ap.add_argument("--solve-qroute", type=int, default=0, help="identity route bound of the --solve-once run")
    ap.add_argument("--solve-omega", type=int, default=1, help="Algorithm 2's omega of the --solve-once run")
    ap.add_argument("--solve-train", type=int, default=0, metavar="EPOCHS",
                    help="after the --solve-once solve, train the proposal network on it for this many epochs")
    ap.add_argument("--solve-reentry", type=int, default=0, choices=[0, 1],
                    help="MPL_OPT_REENTRY of the --solve-once run (1: the same launches on every run, e.g. "
                         "for a launch list whose skip count comes from a run without the profiler)")
    args = ap.parse_args()
    if args.solve_once:
        solve_once(args)
        return
    if args.big_dict:
        big_dictionary_run(args)
        return
    if args.c5_only:
        import torch
        from paper_1302_5010_gb300 import mpl
        print(json.dumps(streaming_warm_vs_cold(args, mpl, torch, torch.device("cuda", 0))), flush=True)
        return
    if args.corr_shape:
        correlation_microbench(args)
        return
    if args.omp_compare:
        omp_compare(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_1302_5010_gb300 import mpl, synth

    assert torch.cuda.is_available(), "bench.py needs a CUDA device"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    # each rank its own batch of independent signals (weak scaling)
    P = rank_problem(synth, args.config, rank)
    smax = SMAX.get(args.config)
    precision = 1 if args.path == "mixed" else 0
    warm = not args.no_warm
    # disjoint training stream for the proposal network (same generator, other signal seed)
    ntrain = args.train_signals or TRAIN_SIGNALS.get(args.config, 8192)
    P_train = rank_problem(synth, args.config, rank, p=ntrain, seed_shift=9000) if warm else None
    n_err = min(P.p, args.cpu_signals) if (rank == 0 and not args.no_cpu_baseline) else 0
    main_run = timed_path(args, mpl, torch, P, dev, precision, world, dist, local, warm=warm, P_train=P_train,
                          smax=smax, want_x64=n_err)
    names = {1: "mixed-bf16", 0: "plain-fp32"}
    line = {"metric": METRIC, "value": main_run["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main_run["tot_ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if precision == 0 else "bf16+f32", "data": "synthetic",
            "config": workload_desc(args.config, P, names[precision] + ("+warm-start" if warm else "")),
            "certified_all": main_run["certified"], "e2e": main_run["e2e"],
            "gpu_launches": int(main_run["launches"]), "clocks": main_run["clocks"],
            "roofline": main_run["roofline"], "correlation_gemm": main_run["gemm"],
            "kernels": main_run["kernels"],
            "outer_iters_mean": main_run["outer_iters_mean"], "active_size_mean": main_run["active_size_mean"],
            "warm_start_training": main_run["training"], "autotune": main_run["autotune"]}
    line["config"]["smax"] = smax
    if not args.no_compare:
        # the comparison path: the other precision without the warm start, everything else equal
        # (same batch, capacity and autotuner candidates)
        other = timed_path(args, mpl, torch, P, dev, 1 - precision, world, dist, local, smax=smax)
        line[names[1 - precision].replace("-", "_")] = {
            "value": other["value"], "ms_per_step": other["tot_ms"] / args.steps, "e2e": other["e2e"]["value"],
            "certified_all": other["certified"], "roofline": other["roofline"],
            "outer_iters_mean": other["outer_iters_mean"], "correlation_gemm": other["gemm"],
            "kernels": other["kernels"], "clocks": other["clocks"], "autotune": other["autotune"],
            "warm_start": False}
        line["speedup_vs_" + names[1 - precision].replace("-", "_")] = main_run["value"] / other["value"]
    if rank == 0 and not args.no_c5 and args.config != "c5":
        # the streaming workload's warm start against the cold solve (extra keys, rank 0 only)
        line["c5_streaming"] = streaming_warm_vs_cold(args, mpl, torch, dev)
    if n_err:
        cb, Xo = cpu_baseline(args.config, P, n_err)
        line["cpu_baseline"] = cb
        line["error_vs_oracle"] = error_vs_oracle(P, main_run["X64"], Xo)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
