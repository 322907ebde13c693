"""Benchmark of the rank-2 Galerkin ROM leapfrog on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

Workload (one bench "step" = one full rom_run_rank2 call over it): K = Kv = Ks
= 512 reduced operators (Asv ~ N(0, 1/K), Avs = -Asv^T), M = 256 Ricker
realizations (T_m = u_m dt, u_m ~ U[30, 60)), 10000 leapfrog steps, R = 64
receiver rows recorded every r = 10 steps, FP32 with Kahan-compensated
state.  Each timed step starts from zero state with L2 flushed (a 256 MB
write between steps, outside the timed events).

Metric: sample-steps/s = M * nsteps / t (one sample-step advances one
realization by one full leapfrog step), whole job over all ranks.  Useful
FLOP/s = (4 Kv Ks M + 2 R Kv M / r) per leapfrog step.

Multi-GPU: every rank integrates its own M realizations (replicas by
realization, no data-path collective); `value` sums over ranks and the time is
the max over ranks.  Rank 0 prints one JSON line.

`--impl reference` times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload.
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

WORKLOAD = dict(name="rank2-fp32-K512-M256-N10000-R64-r10", K=512, M=256, nsteps=10000, R=64,
                r=10, prec="fp32", seed=0)
# The split-precision tensor-core workload (selected with --workload 2).
WORKLOAD2 = dict(name="rank2-split-K1024-M1024-N20000-R64-r10", K=1024, M=1024, nsteps=20000,
                 R=64, r=10, prec="tf32x3", seed=0)
# Nominal dense tensor-core rates relative to BF16 (profiling recipe table).
TC_RATIO = {"tf32x3": 1.1 / 2.25, "bf16x3": 1.0, "bf16": 1.0, "bf16s": 1.0}
TC_PRODUCTS = {"tf32x3": 3, "bf16x3": 5, "bf16": 1, "bf16s": 6}
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (Blackwell)


METRIC = "rank-2 ROM sample-steps/s (FP32 leapfrog, rel err <= 1e-4)"


def bench_config(W, world):
    """The `config` object of the headline line (both arms)."""
    return {"workload": W["name"], "K": W["K"], "M": W["M"], "nsteps": W["nsteps"], "R": W["R"],
            "r": W["r"], "prec": W["prec"], "parallelism": f"replicas-by-realization x{world}",
            "l2": "flushed (256 MB write) before every timed step"}


def useful_flops(K, M, N, R, r):
    return (4.0 * K * K * M + (2.0 * R * K * M / r if r else 0.0)) * N


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def measured_pipe_peaks(rom):
    """The roofline denominators measured live on this device by the library's
    microbenchmarks (rom_measure_peak): FP32 / FP64 FMA and TF32 / BF16 tensor
    TFLOP/s, L2 read GB/s.  A kind that fails is left out."""
    out = {}
    for kind in ("fp32", "fp64", "tf32", "bf16", "l2"):
        try:
            out[kind] = rom.measure_peak(kind)[0]
        except Exception as exc:  # a failed probe leaves that denominator to the nominal basis
            out[kind + "_error"] = str(exc)
    return out


def fp32_roofline(rom, tflops):
    """The FP32 FMA roofline of a secondary workload: the achieved useful
    rate against the FP32 peak measured live (rom_measure_peak)."""
    try:
        pk = rom.measure_peak("fp32")[0]
    except Exception as exc:  # no denominator: report the rate alone
        return {"bound": "alu", "achieved": tflops, "unit": "TFLOP/s", "peak_error": str(exc)}
    return {"bound": "alu", "achieved": tflops, "peak": pk, "unit": "TFLOP/s", "frac": tflops / pk,
            "peak_kind": "FP32 FMA microbenchmark (rom_measure_peak), this run"}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

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
        self.t.join(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- reference --
def run_reference(args):
    """The FP64 CPU oracle on a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2009_11742_gb300 import inputs
    p = inputs.make_problem(WORKLOAD["K"], WORKLOAD["K"], WORKLOAD["M"], WORKLOAD["R"],
                            seed=WORKLOAD["seed"])
    cores = oracle.max_threads()
    ncol = min(WORKLOAD["M"], 2 * cores)
    cols = np.linspace(0, WORKLOAD["M"] - 1, ncol).astype(int)
    # calibrate so that each step is a few seconds of CPU work
    t0 = time.perf_counter()
    oracle.problem_forward(p, nsteps=50, r=WORKLOAD["r"], columns=cols)
    per_step = (time.perf_counter() - t0) / 50
    nst = int(max(100, min(WORKLOAD["nsteps"], 3.0 / max(per_step, 1e-9))))
    nst -= nst % WORKLOAD["r"]
    for _ in range(args.warmup):
        oracle.problem_forward(p, nsteps=max(WORKLOAD["r"], nst // 10), r=WORKLOAD["r"],
                               columns=cols)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.problem_forward(p, nsteps=nst, r=WORKLOAD["r"], columns=cols)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = ncol * nst * args.steps / tot
    sample = f"{ncol} of {WORKLOAD['M']} columns x {nst} of {WORKLOAD['nsteps']} steps per step"
    line = {
        "impl": "reference", "metric": METRIC,
        "value": value, "unit": "sample-steps/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": bench_config(WORKLOAD, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": "sample-steps/s", "cores": cores,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "sample-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(p, target_s=16.0):
    """Oracle throughput on a bounded sample (all host cores)."""
    import oracle
    cores = oracle.max_threads()
    ncol = min(WORKLOAD["M"], 2 * cores)
    cols = np.linspace(0, WORKLOAD["M"] - 1, ncol).astype(int)
    oracle.problem_forward(p, nsteps=WORKLOAD["r"], r=WORKLOAD["r"], columns=cols)  # threads up
    # long enough that the call's fixed cost (buffers, thread start) is small
    ncal = min(WORKLOAD["nsteps"], 1000)
    t0 = time.perf_counter()
    oracle.problem_forward(p, nsteps=ncal, r=WORKLOAD["r"], columns=cols)
    per_step = (time.perf_counter() - t0) / ncal
    full = per_step * WORKLOAD["nsteps"]
    if full < target_s and ncol < WORKLOAD["M"]:
        # every step fits: widen the column sample (whole multiples of the cores)
        ncol0 = ncol
        ncol = min(WORKLOAD["M"], max(ncol0, int(ncol0 * target_s / max(full, 1e-9)) // cores * cores))
        cols = np.linspace(0, WORKLOAD["M"] - 1, ncol).astype(int)
        per_step *= ncol / ncol0
    nst = int(max(100, min(WORKLOAD["nsteps"], target_s / max(per_step, 1e-9))))
    nst -= nst % WORKLOAD["r"]
    t0 = time.perf_counter()
    oracle.problem_forward(p, nsteps=nst, r=WORKLOAD["r"], columns=cols)
    dt = time.perf_counter() - t0
    # the same oracle on one thread (a few columns, a few seconds)
    c1 = cols[:2]
    oracle.problem_forward(p, nsteps=WORKLOAD["r"], r=WORKLOAD["r"], columns=c1, threads=1)
    t0 = time.perf_counter()
    oracle.problem_forward(p, nsteps=100, r=WORKLOAD["r"], columns=c1, threads=1)
    per1 = (time.perf_counter() - t0) / 100
    n1 = int(max(100, min(WORKLOAD["nsteps"], 4.0 / max(per1, 1e-9))))
    n1 -= n1 % WORKLOAD["r"]
    t0 = time.perf_counter()
    oracle.problem_forward(p, nsteps=n1, r=WORKLOAD["r"], columns=c1, threads=1)
    dt1 = time.perf_counter() - t0
    return {"value": ncol * nst / dt, "unit": "sample-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{ncol} of {WORKLOAD['M']} columns x {nst} of {WORKLOAD['nsteps']} "
                      f"steps ({dt:.1f} s, OpenMP over columns)",
            "one_thread": {"value": len(c1) * n1 / dt1, "unit": "sample-steps/s",
                           "sample": f"{len(c1)} columns x {n1} steps ({dt1:.1f} s)"}}


def rank_periods(T_all, rank, world):
    """Periods of the realizations one rank integrates: an ensemble of
    world * M realizations split into contiguous shards of M (replicas by
    realization, no data-path exchange)."""
    M = len(T_all) // world
    return T_all[rank * M:(rank + 1) * M]


def max_over_ranks(t, dist, device):
    """Job time = the slowest rank's time (every rank's value when dist is None)."""
    if dist is None:
        return t
    import torch
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def profiled_traffic(kname, nsteps):
    """DRAM bytes (read + write) of one full-size launch, from the committed
    ncu summary of that kernel on this workload, or None."""
    import re
    stem = ("rank2_split_and_stream_kernels" if "rank2_stream_kernel" in kname
            else kname.split("<")[0])
    prof = os.path.join(ROOT, "profiles", f"{stem}_fp32_K512_M256_N{nsteps}.md")
    try:
        m = re.search(r"^dram_bytes_per_launch:\s*(\d+)", open(prof).read(), re.M)
    except OSError:
        return None
    return int(m.group(1)) if m else None


# ------------------------------------------------------------------- gb300 --
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true", help="skip the sampled oracle error check")
    ap.add_argument("--nsteps", type=int, default=None,
                    help="leapfrog steps per run (default: the workload's 10000; profiling only)")
    ap.add_argument("--only-rank2", action="store_true",
                    help="time the rank-2 runs only (no e2e, rank-1, oracle legs; profiling only)")
    ap.add_argument("--workload", type=int, default=1, choices=[0, 1, 2, 3, 4, 5, 6, 7],
                    help="0: K=128 M=16 N=1000 FP64; 1: K=512 FP32 (default, the headline); "
                         "2: K=1024 split precision; 3: 64 batched ROMs; 4: adjoint K=512 M=128 N=4000 c=64; "
                         "5: many-query UQ run (Kv=436, Ks=417, M=512, 20000 steps) with ensemble statistics; "
                         "6: rank-3 (16 operators x 16 forcings, K=256, 10000 steps) in one launch; "
                         "7: rank-2 full-order model (512 x 2048 grid, 3.14 M unknowns, M=32, 1000 steps)")
    ap.add_argument("--prec", default=None, help="override the workload's precision")
    ap.add_argument("--tc-cols", type=int, default=0, help="tensor-core columns per block")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2009_11742_gb300 import build as rbuild
    rbuild.build()
    from paper_2009_11742_gb300 import inputs, rom

    if args.workload == 0:
        return bench_fp64(args, torch, dev, inputs, rom)
    if args.workload == 5:
        return bench_uq(args, torch, dev, inputs, rom)
    if args.workload == 3:
        return bench_batched(args, torch, dev, inputs, rom)
    if args.workload == 4:
        return bench_adjoint(args, torch, dev, inputs, rom)
    if args.workload == 6:
        return bench_rank3(args, torch, dev, inputs, rom)
    if args.workload == 7:
        return bench_fom(args, torch, dev, inputs, rom)

    W = dict(WORKLOAD if args.workload == 1 else WORKLOAD2)
    if args.nsteps:
        W["nsteps"] = args.nsteps
    if args.prec:
        W["prec"] = args.prec
    prec = W["prec"]
    K, M, N, R, r = W["K"], W["M"], W["nsteps"], W["R"], W["r"]
    p = inputs.make_problem(K, K, M * world, R, seed=W["seed"])
    p.T = rank_periods(p.T, rank, world)
    h = rom.Rom.from_problem(p)
    if args.tc_cols:
        rom.rom_set_tc_columns(h.h, args.tc_cols)
    V = rom.Rom.new_state(K, M, "fp32", device=dev)
    S = rom.Rom.new_state(K, M, "fp32", device=dev)
    T = torch.as_tensor(p.T, dtype=torch.float32, device=dev)
    nrec = N // r
    tr = torch.zeros((nrec, M, R), dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.Stream(device=dev)

    def one_run():
        h.run_rank2(V, S, T, N, r=r, traces=tr, prec=prec, stream=stream)

    def reset():
        V.zero_()
        S.zero_()
        flush.fill_(1.0)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            reset()
            one_run()
    torch.cuda.synchronize()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    sampler = ClockSampler(local) if rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            reset()
            evs[i][0].record(stream)
            one_run()
            evs[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    st = h.sync_status()
    if st != 0:
        raise RuntimeError(f"device status {rom.status_string(st)}")
    per = [a.elapsed_time(b) * 1e-3 for a, b in evs]
    t_dev = max_over_ranks(sum(per), dist, dev)
    value = world * M * N * args.steps / t_dev
    ms_per_step = 1e3 * t_dev / args.steps
    flops = useful_flops(K, M, N, R, r)

    if args.only_rank2 or args.workload != 1:
        if rank == 0:
            out = {"only_rank2": True, "workload": W["name"], "prec": prec, "value": value,
                   "unit": "sample-steps/s", "ms_per_step": ms_per_step, "nsteps": N,
                   "tflops_useful": world * flops * args.steps / t_dev / 1e12, "clocks": clocks}
            if prec == "fp32":
                out["roofline"] = fp32_roofline(rom, out["tflops_useful"])
                out["plan"] = h.plan(M)
            if prec in TC_RATIO:
                pk, pk_kind = peaks()
                mp = measured_pipe_peaks(rom)
                ach = TC_PRODUCTS[prec] * 4.0 * K * K * M * N / (t_dev / args.steps) / 1e12
                if prec == "tf32x3" and "tf32" in mp:
                    # TF32 products against the TF32 pipe's own measured rate
                    peak, basis = mp["tf32"], "tf32 tcgen05 microbenchmark (rom_measure_peak), this run"
                else:
                    peak = pk.get("bf16_tflops", 1900.0) * TC_RATIO[prec]
                    basis = f"bf16 cuBLAS {pk_kind}" + (f" x {TC_RATIO[prec]:.3f}" if TC_RATIO[prec] != 1.0 else "")
                out["roofline_tensor"] = {"bound": "tensor", "achieved": ach, "peak": peak,
                                          "unit": "TFLOP/s", "frac": ach / peak,
                                          "basis": f"{TC_PRODUCTS[prec]} products x 4 K^2 M per step; {basis}",
                                          "measured_pipe_peaks": mp}
            if not args.no_check and args.workload == 2:
                import oracle
                cols = np.array([0, 511, 1023])
                V.zero_(); S.zero_()
                one_run(); torch.cuda.synchronize()
                Vo, So, tro = oracle.problem_forward(p, nsteps=N, r=r, columns=cols)
                Vg = V.cpu().numpy()[:, cols]
                tg = tr.transpose(1, 2).cpu().numpy()[:, :, cols]
                out["rel_err_vs_oracle"] = {
                    "V": float(np.linalg.norm(Vg - Vo) / np.linalg.norm(Vo)),
                    "traces": float(np.linalg.norm(tg - tro) / np.linalg.norm(tro)),
                    "columns": cols.tolist()}
            print(json.dumps(out), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- end-to-end through the C ABI with pinned host buffers
    Vh = torch.zeros((M, K), dtype=torch.float32).pin_memory().numpy().T
    Sh = torch.zeros((M, K), dtype=torch.float32).pin_memory().numpy().T
    Th = torch.as_tensor(p.T, dtype=torch.float32).pin_memory().numpy()
    trh = torch.zeros((nrec, M, R), dtype=torch.float32).pin_memory().numpy()
    h.run_rank2(Vh, Sh, Th, N, r=r, traces=trh, prec="fp32")  # warm the staging buffers
    e2e_times = []
    for _ in range(max(3, args.steps // 2)):
        Vh[...] = 0
        Sh[...] = 0
        t0 = time.perf_counter()
        h.run_rank2(Vh, Sh, Th, N, r=r, traces=trh, prec="fp32")
        e2e_times.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(sum(e2e_times) / len(e2e_times), dist, dev)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # ---- rank-1 baselines on the same operator (fewer steps; throughput is per sample-step)
    N1 = 2000
    v1 = torch.zeros(K, dtype=torch.float32, device=dev)
    s1 = torch.zeros(K, dtype=torch.float32, device=dev)
    for _ in range(2):
        h.run_rank1(v1, s1, float(p.T[0]), N1, prec="fp32", stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.run_rank1(v1, s1, float(p.T[0]), N1, prec="fp32", stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    r1_single = N1 / (e0.elapsed_time(e1) * 1e-3)
    Ve = rom.Rom.new_state(K, M, "fp32", device=dev)
    Se = rom.Rom.new_state(K, M, "fp32", device=dev)
    h.run_rank1_ensemble(Ve, Se, T, N1 // 10, prec="fp32", stream=stream)
    e0.record(stream)
    h.run_rank1_ensemble(Ve, Se, T, N1, prec="fp32", stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    r1_ens = M * N1 / (e0.elapsed_time(e1) * 1e-3)
    rank1_best = max(r1_single, r1_ens)

    # ---- accuracy on sampled columns against the FP64 oracle (full 10000 steps)
    err = None
    if not args.no_check:
        import oracle
        V.zero_()
        S.zero_()
        one_run()
        torch.cuda.synchronize()
        cols = np.array([0, 85, 170, 255])
        Vo, So, tro = oracle.problem_forward(p, nsteps=N, r=r, columns=cols)
        Vg = V.cpu().numpy()[:, cols]
        Sg = S.cpu().numpy()[:, cols]
        tg = tr.transpose(1, 2).cpu().numpy()[:, :, cols]

        def rel(a, b):
            return float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))

        err = {"V": rel(Vg, Vo), "S": rel(Sg, So), "traces": rel(tg, tro),
               "columns": cols.tolist()}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline_sample(p)

    pk, pk_kind = peaks()
    sm_clock_max = float(pk.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_nominal = nsm * FP32_LANES_PER_SM * 2 * sm_clock_max * 1e6 / 1e12  # TFLOP/s
    mp = measured_pipe_peaks(rom)
    achieved = flops / (t_dev / args.steps) / 1e12
    plan = h.plan(M, "fp32")
    kname = ("rank2_split_kernel<8>" if plan["variant"] == 2
             else "rank2_split_kernel<8> + rank2_stream_kernel<8,4>" if plan["variant"] == 4
             else "rank2_simt_kernel<float,8,8,true>")
    traffic = profiled_traffic(kname, N) if (K, M, R, r) == (512, 256, 64, 10) else None
    if "fp32" in mp:
        fp32_peak = mp["fp32"]
        basis = ("measured: FP32 FMA microbenchmark over all SMs (rom_measure_peak), this run; "
                 f"nominal {nsm} SMs x {FP32_LANES_PER_SM} lanes x 2 x {sm_clock_max:.0f} MHz = "
                 f"{fp32_nominal:.1f}")
    else:
        fp32_peak = fp32_nominal
        basis = (f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 FMA lanes x 2 x "
                 f"{sm_clock_max:.0f} MHz (max SM clock, {pk_kind})")
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": traffic,
            "kernel": kname, "plan": plan, "peak_basis": basis,
            "peak_nominal": fp32_nominal, "frac_of_nominal": achieved / fp32_nominal,
            "measured_pipe_peaks": mp}

    es = 4
    h2d = (2 * K * M + M) * es
    d2h = (2 * K * M + nrec * R * M) * es
    line = {
        "metric": METRIC,
        "value": value, "unit": "sample-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(W, world),
        "tflops_useful": world * flops * args.steps / t_dev / 1e12,
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": world * M * N / e2e_t, "unit": "sample-steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # one split-kernel launch per step, plus its companion when the plan has one
        "gpu_launches": args.steps * (2 if plan.get("variant") == 4 else 1),
        "clocks": clocks,
        "wall_s_timed_region": wall,
        "rank1": {"single_sample_steps_s": r1_single, "ensemble_sample_steps_s": r1_ens,
                  "rank2_speedup_vs_best_rank1": value / world / rank1_best,
                  # operator bytes per sample-step: both K x K FP32 operators (2 MB at
                  # K = 512, L2-resident, so L2 rather than HBM is the ceiling)
                  "single_operator_gbs": r1_single * 8.0 * K * K / 1e9,
                  "ensemble_operator_gbs": r1_ens * 8.0 * K * K / 1e9,
                  "hbm_gbs_measured": pk.get("hbm_gbs"),
                  "l2_gbs_measured": mp.get("l2"),
                  "ensemble_frac_of_l2": (r1_ens * 8.0 * K * K / 1e9 / mp["l2"]) if mp.get("l2") else None},
        "rel_err_vs_oracle": err,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    h.close()
    return 0


def bench_uq(args, torch, dev, inputs, rom):
    """Workload 5: the many-query UQ run of Sec. 4.5.2 on synthetic operators
    (Kv = 436, Ks = 417, 512 realizations of T ~ U(31, 69) steps, 20000
    steps, 64 receivers every 10 steps), then the per-receiver ensemble mean
    and 5/50/95 % bands on the device.  Reports both times, the rank-2 vs
    rank-1 ensemble throughput ratio and sampled accuracy."""
    c = inputs.WORKLOADS[5]
    p = inputs.workload(5)
    N = args.nsteps or c["steps"]
    r, M, R, Kv, Ks = c["r"], p.M, p.R, p.Kv, p.Ks
    h = rom.Rom.from_problem(p)
    V = rom.Rom.new_state(Kv, M, "fp32", device=dev)
    S = rom.Rom.new_state(Ks, M, "fp32", device=dev)
    T = torch.as_tensor(p.T, dtype=torch.float32, device=dev)
    tr = torch.zeros((N // r, M, R), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def one():
        V.zero_(); S.zero_()
        h.run_rank2(V, S, T, N, r=r, traces=tr, prec="fp32", stream=stream)

    for _ in range(max(1, args.warmup)):
        one()
        with torch.cuda.stream(stream):
            rom.trace_stats(tr, c["probs"], stream=stream)
    torch.cuda.synchronize()
    t_run, t_stats = [], []
    for _ in range(args.steps):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        V.zero_(); S.zero_()
        torch.cuda.synchronize()
        e0.record(stream)
        h.run_rank2(V, S, T, N, r=r, traces=tr, prec="fp32", stream=stream)
        e1.record(stream)
        with torch.cuda.stream(stream):
            mean, q = rom.trace_stats(tr, c["probs"], stream=stream)
        e2.record(stream)
        torch.cuda.synchronize()
        t_run.append(e0.elapsed_time(e1) * 1e-3)
        t_stats.append(e1.elapsed_time(e2) * 1e-3)
    tr_run, tr_stats = sum(t_run) / len(t_run), sum(t_stats) / len(t_stats)
    # rank-1 ensemble (one realization per CTA, operators streamed) on 2000 steps
    N1 = min(N, 2000)
    Ve = rom.Rom.new_state(Kv, M, "fp32", device=dev)
    Se = rom.Rom.new_state(Ks, M, "fp32", device=dev)
    h.run_rank1_ensemble(Ve, Se, T, 200, prec="fp32", stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.run_rank1_ensemble(Ve, Se, T, N1, prec="fp32", stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    r1 = M * N1 / (e0.elapsed_time(e1) * 1e-3)
    # accuracy: 4 sampled realizations over the first 2000 steps
    import oracle
    Na = min(N, 2000)
    V.zero_(); S.zero_()
    tra = torch.zeros((Na // r, M, R), dtype=torch.float32, device=dev)
    h.run_rank2(V, S, T, Na, r=r, traces=tra, prec="fp32", stream=stream)
    torch.cuda.synchronize()
    cols = np.array([0, 170, 341, 511])
    _, _, tro = oracle.problem_forward(p, nsteps=Na, r=r, columns=cols)
    tg = tra.transpose(1, 2).cpu().numpy()[:, :, cols]
    err = float(np.linalg.norm(tg - tro) / np.linalg.norm(tro))
    print(json.dumps({"only_rank2": True, "workload": c["name"], "nsteps": N,
                      "value": M * N / tr_run, "unit": "sample-steps/s",
                      "run_ms": 1e3 * tr_run, "stats_ms": 1e3 * tr_stats,
                      "stats": {"records": N // r, "receivers": R, "realizations": M,
                                "probs": list(c["probs"])},
                      "rank1_ensemble_sample_steps_s": r1,
                      "rank2_over_rank1_ensemble": (M * N / tr_run) / r1,
                      "tflops_useful": 4.0 * Kv * Ks * M * N / tr_run / 1e12,
                      "roofline": fp32_roofline(rom, 4.0 * Kv * Ks * M * N / tr_run / 1e12),
                      "plan": h.plan(M),
                      "rel_err_traces_vs_oracle": {"value": err, "columns": cols.tolist(), "steps": Na}}),
          flush=True)
    return 0


def bench_fp64(args, torch, dev, inputs, rom):
    """Workload 0: the FP64 check path (K = 128, M = 16, 1000 steps, no traces):
    achieved FP64 rate against the FP64 rate measured by the library's
    microbenchmark (and the 1.25 TFLOP/s nominal), the FP64
    rank-1 paths on the same operator, and the error against the FP64
    oracle."""
    p = inputs.workload(0)
    K, M, N = 128, 16, args.nsteps or 1000
    h = rom.Rom.from_problem(p)
    V = rom.Rom.new_state(K, M, "fp64", device=dev)
    S = rom.Rom.new_state(K, M, "fp64", device=dev)
    T = torch.as_tensor(p.T, dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(device=dev)
    for _ in range(args.warmup):
        V.zero_(); S.zero_()
        h.run_rank2(V, S, T, N, prec="fp64", stream=stream)
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        V.zero_(); S.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h.run_rank2(V, S, T, N, prec="fp64", stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e-3)
    t = sum(ts) / len(ts)
    # rank-1 FP64 baselines on the same operator: one realization at a time,
    # and the M realizations as independent GEMV solves
    v1 = torch.zeros(K, dtype=torch.float64, device=dev)
    s1 = torch.zeros(K, dtype=torch.float64, device=dev)
    Ve = rom.Rom.new_state(K, M, "fp64", device=dev)
    Se = rom.Rom.new_state(K, M, "fp64", device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h.run_rank1(v1, s1, float(p.T[0]), N, prec="fp64", stream=stream)
    e0.record(stream)
    h.run_rank1(v1, s1, float(p.T[0]), N, prec="fp64", stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    r1_single = N / (e0.elapsed_time(e1) * 1e-3)
    h.run_rank1_ensemble(Ve, Se, T, N, prec="fp64", stream=stream)
    e0.record(stream)
    h.run_rank1_ensemble(Ve, Se, T, N, prec="fp64", stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    r1_ens = M * N / (e0.elapsed_time(e1) * 1e-3)
    mp = measured_pipe_peaks(rom)
    import oracle
    Vo, So, _ = oracle.problem_forward(p, nsteps=N, r=0)
    Vg, Sg = V.cpu().numpy(), S.cpu().numpy()
    flops = 4.0 * K * K * M * N
    print(json.dumps({"only_rank2": True, "workload": "rank2-fp64-K128-M16-N1000", "nsteps": N,
                      "value": M * N / t, "unit": "sample-steps/s", "ms_per_step": 1e3 * t,
                      "us_per_leapfrog_step": 1e6 * t / N,
                      "gflops_fp64": flops / t / 1e9, "frac_of_fp64_nominal_1250_gflops": flops / t / 1.25e12,
                      "fp64_peak_measured_tflops": mp.get("fp64"),
                      "frac_of_fp64_measured": (flops / t / 1e12 / mp["fp64"]) if mp.get("fp64") else None,
                      "bound": "FP64 units and cluster barriers (1 MFLOP per leapfrog step)",
                      "plan": h.plan(M, "fp64"),
                      "rank1_fp64": {"single_sample_steps_s": r1_single, "ensemble_sample_steps_s": r1_ens,
                                     "rank2_speedup_vs_best_rank1": (M * N / t) / max(r1_single, r1_ens)},
                      "rel_err_vs_oracle": {"V": float(np.linalg.norm(Vg - Vo) / np.linalg.norm(Vo)),
                                            "S": float(np.linalg.norm(Sg - So) / np.linalg.norm(So))}}),
          flush=True)
    return 0


def bench_adjoint(args, torch, dev, inputs, rom):
    """Workload 4: gradients of the trace misfit (K = 512, M = 128, 4000 steps,
    R = 64, checkpoints every 64 steps) against the forward run with every
    trace recorded; reports the time ratio adjoint / forward."""
    p = inputs.workload(4)
    K, M, R = 512, 128, 64
    N = args.nsteps or 4000
    h = rom.Rom.from_problem(p)
    V0 = rom.Rom.new_state(K, M, "fp32", device=dev)
    S0 = rom.Rom.new_state(K, M, "fp32", device=dev)
    T = torch.as_tensor(p.T, dtype=torch.float32, device=dev)
    g = torch.Generator(device="cpu").manual_seed(0)
    ys = (0.01 * torch.randn((N, M, R), generator=g)).to(dev)  # synthetic targets (timing only)
    tr = torch.zeros((N, M, R), dtype=torch.float32, device=dev)
    V = rom.Rom.new_state(K, M, "fp32", device=dev)
    S = rom.Rom.new_state(K, M, "fp32", device=dev)
    ws = torch.empty(rom.rom_adjoint_workspace_size(h.h, M, N, 64, rom.ROM_FP32), dtype=torch.uint8,
                     device=dev)
    gV = rom.Rom.new_state(K, M, "fp32", device=dev)
    gS = rom.Rom.new_state(K, M, "fp32", device=dev)
    gT = torch.zeros(M, dtype=torch.float32, device=dev)

    def fwd():
        V.zero_(); S.zero_()
        h.run_rank2(V, S, T, N, r=1, traces=tr, prec="fp32")

    # every trace kept (one segment, no recompute): the memory-for-time trade
    ws0 = torch.empty(rom.rom_adjoint_workspace_size(h.h, M, N, 0, rom.ROM_FP32), dtype=torch.uint8,
                      device=dev)

    def adj(ckpt=64):
        w = ws if ckpt else ws0
        st, _ = rom.rom_adjoint(h.h, V0.data_ptr(), S0.data_ptr(), T.data_ptr(), M, N,
                                ys.data_ptr(), ckpt, gV.data_ptr(), gS.data_ptr(), gT.data_ptr(),
                                w.data_ptr(), w.numel(), rom.ROM_FP32, None)
        assert st == 0

    for _ in range(args.warmup):
        fwd(); adj(); adj(0)
    torch.cuda.synchronize()

    def timed(fn):
        ts = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return sum(ts) / len(ts)
    tf = timed(fwd)
    ta = timed(adj)
    ta0 = timed(lambda: adj(0))
    print(json.dumps({"only_rank2": True, "workload": "adjoint-K512-M128-N4000-R64-r1-c64",
                      "nsteps": N, "forward_ms": 1e3 * tf, "adjoint_ms": 1e3 * ta,
                      "adjoint_over_forward": ta / tf,
                      "adjoint_sample_steps_per_s": M * N / ta, "unit": "sample-steps/s",
                      "all_traces_kept": {"adjoint_ms": 1e3 * ta0, "adjoint_over_forward": ta0 / tf,
                                          "workspace_bytes": ws0.numel(), "c64_workspace_bytes": ws.numel()}}),
          flush=True)
    return 0


def bench_batched(args, torch, dev, inputs, rom):
    """Workload 3: 64 independent ROMs (K_i in {64..768}, M_i in [4, 256]),
    5000 steps each, one graph launch per bench step; timed with the
    proportional SM shares, then again after rom_autotune_batched has
    measured the schedule (the tuning probe is outside the timed region)."""
    probs = inputs.batched_problems()
    N = args.nsteps or 5000
    prec = args.prec or "fp32"
    items = []
    for p in probs:
        h = rom.Rom.from_problem(p)
        items.append((h, rom.Rom.new_state(p.Kv, p.M, "fp32", device=dev),
                      rom.Rom.new_state(p.Ks, p.M, "fp32", device=dev),
                      torch.as_tensor(p.T, dtype=torch.float32, device=dev), None))
    stream = torch.cuda.Stream(device=dev)

    def timed():
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                rom.run_batched(items, N, prec=prec, stream=stream)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                for (_, V, S, _, _) in items:
                    V.zero_()
                    S.zero_()
                evs[i][0].record(stream)
                rom.run_batched(items, N, prec=prec, stream=stream)
                evs[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) * 1e-3 / args.steps

    t0 = timed()
    probe_us = rom.autotune_batched(items, prec=prec, probe_steps=200, stream=stream)
    t = timed()
    ss = sum(p.M for p in probs) * N
    fl = sum(4.0 * p.Kv * p.Ks * p.M for p in probs) * N
    print(json.dumps({"only_rank2": True, "workload": "batched-64roms-K64..768-M4..256-N5000", "prec": prec,
                      "nsteps": N, "value": ss / t, "unit": "sample-steps/s",
                      "ms_per_step": 1e3 * t, "tflops_useful": fl / t / 1e12,
                      "untuned": {"value": ss / t0, "ms_per_step": 1e3 * t0},
                      "autotune_probe_us_per_step": probe_us,
                      "columns_total": sum(p.M for p in probs),
                      **({"roofline": fp32_roofline(rom, fl / t / 1e12)} if prec == "fp32" else {})}),
          flush=True)
    return 0


def bench_fom(args, torch, dev, inputs, rom):
    """Workload 7: the rank-2 full-order model of Sec. 3 at one of the
    paper's FOM sizes (3,143,168 unknowns in App. B; here a 512 x 2048 grid,
    3,141,633 unknowns) with the App. A setup: homogeneous layer, rho 2500,
    vs 5000, dt 0.05 s, a source 640 km deep next to the axis, the first
    derivative of a Gaussian with periods drawn in (60, 80) s, 1000 steps
    from rest with the forcing clock starting at step 1500 (75 s), so that
    the pulse peaks (1.5 T = 90-120 s) fall inside the run, 64 surface
    receivers every 10 steps.  M = 32 realizations in one run,
    beside the rank-1 FOM (M = 1) on the same grid.  The roofline is HBM:
    8 M bytes per unknown per step in FP32 (16 M in FP64), every state value
    read and written once."""
    import numpy as np
    Nr, Nt, M = 512, 2048, 32
    N = args.nsteps or 1000
    prec = args.prec or "fp32"
    es = 8 if prec == "fp64" else 4
    tdt = torch.float64 if prec == "fp64" else torch.float32
    f = rom.Fom(Nr, Nt)
    src = f.source_index(640e3, j=1)
    recv = torch.tensor([f.vindex(Nr - 1, j) for j in np.linspace(1, Nt - 1, 64).astype(int)],
                        dtype=torch.int32, device=dev)
    rng = np.random.default_rng(7)
    nun = f.nv + f.n1 + f.n2
    stream = torch.cuda.Stream(device=dev)

    def timed(Mx):
        V, S1, S2 = f.new_state(Mx, prec, device=dev)
        T = torch.as_tensor(rng.uniform(60.0, 80.0, Mx), dtype=tdt, device=dev)
        tr = torch.zeros((N // 10, recv.numel(), Mx), dtype=tdt, device=dev)

        def one():
            f.run(V, S1, S2, N, src=src, T=T, recv=recv, r=10, traces=tr, prec=prec, stream=stream,
                  n0=1500)

        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                one()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                for x in (V, S1, S2):
                    x.zero_()
                evs[i][0].record(stream)
                one()
                evs[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) * 1e-3 / args.steps

    t = timed(M)
    t1 = timed(1)
    # the algorithmic minimum of a step: every state value read once and written once
    byts = 2.0 * es * nun * M * N
    pk, pk_kind = peaks()
    hbm = pk.get("hbm_gbs")
    out = {"only_rank2": True, "workload": f"fom-{Nr}x{Nt}-{nun}unknowns-M{M}-N{N}-{prec}",
           "nsteps": N, "value": M * N / t, "unit": "sample-steps/s", "ms_per_step": 1e3 * t / N,
           "unknown_updates_per_s": nun * M * N / t,
           "roofline": {"bound": "hbm", "achieved": byts / t / 1e9, "peak": hbm, "unit": "GB/s",
                        "frac": (byts / t / 1e9 / hbm) if hbm else None, "peak_kind": pk_kind,
                        "basis": f"{2 * es} B per unknown per realization per step "
                                 "(every state value read once and written once; the fused pass)"},
           "rank1": {"value": N / t1, "ms_per_step": 1e3 * t1 / N,
                     "achieved_gbs": 2.0 * es * nun * N / t1 / 1e9},
           "rank2_over_rank1_per_realization": (M * N / t) / (N / t1)}
    print(json.dumps(out), flush=True)
    return 0


def bench_rank3(args, torch, dev, inputs, rom):
    """Workload 6: the rank-3 outlook (Sec. 5).  16 operators (K = 256, one
    shared dt) times 16 forcings each, 10000 FP32 steps with traces every 10
    steps, in one launch (rom_run_rank3).  Beside it, the same work as a
    batched graph of 16 rank-2 runs and as 16 rank-2 runs one after another."""
    import numpy as np
    nops, K, M, R, r = 16, 256, 16, 64, 10
    N = args.nsteps or 10000
    probs = inputs.rank3_problems(nops, K, K, M, R, seed=600)
    roms = [rom.Rom.from_problem(p) for p in probs]
    Mt = nops * M
    V = rom.Rom.new_state(K, Mt, "fp32", device=dev)
    S = rom.Rom.new_state(K, Mt, "fp32", device=dev)
    T = torch.as_tensor(np.concatenate([p.T for p in probs]), dtype=torch.float32, device=dev)
    tr = torch.zeros(((N // r) * Mt * R,), dtype=torch.float32, device=dev)
    # per-operator column slices (contiguous: the state is column-major)
    Vs = [V[:, i * M:(i + 1) * M] for i in range(nops)]
    Ss = [S[:, i * M:(i + 1) * M] for i in range(nops)]
    Ts = [T[i * M:(i + 1) * M] for i in range(nops)]
    trs = [torch.zeros(((N // r) * M * R,), dtype=torch.float32, device=dev) for _ in range(nops)]
    stream = torch.cuda.Stream(device=dev)

    def rank3():
        rom.run_rank3(roms, V, S, T, N, r=r, traces=tr, prec="fp32", stream=stream)

    def batched():
        rom.run_batched([(roms[i], Vs[i], Ss[i], Ts[i], trs[i]) for i in range(nops)], N, r=r,
                        prec="fp32", stream=stream)

    def sequential():
        for i in range(nops):
            roms[i].run_rank2(Vs[i], Ss[i], Ts[i], N, r=r, traces=trs[i], prec="fp32", stream=stream)

    def timed(fn):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                V.zero_()
                S.zero_()
                fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                V.zero_()
                S.zero_()
                evs[i][0].record(stream)
                fn()
                evs[i][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) * 1e-3 / args.steps

    t_b = timed(batched)
    t_s = timed(sequential)
    t3 = timed(rank3)  # last, so that V and the traces hold the rank-3 result
    ss = Mt * N
    out = {"only_rank2": True, "workload": f"rank3-{nops}ops-K{K}-M{M}-N{N}-R{R}-r{r}", "nsteps": N,
           "value": ss / t3, "unit": "sample-steps/s", "ms_per_step": 1e3 * t3,
           "tflops_useful": 4.0 * K * K * Mt * N / t3 / 1e12,
           "batched_graph": {"value": ss / t_b, "ms_per_step": 1e3 * t_b},
           "sequential_rank2": {"value": ss / t_s, "ms_per_step": 1e3 * t_s}}
    if not args.no_check:
        import oracle
        Vg = V.cpu().numpy()
        trg = tr.cpu().numpy().reshape(N // r, Mt, R)
        errs = []
        for i, m in ((0, 0), (nops // 2, M // 2), (nops - 1, M - 1)):
            p = probs[i]
            z = np.zeros((K, 1))
            Vo, _, tro = oracle.forward(p.Avs, p.Asv, p.g, p.C, p.dt, z, z, N, T=p.T[m:m + 1], r=r)
            c = i * M + m
            errs.append(max(float(np.linalg.norm(Vg[:, c] - Vo[:, 0]) / np.linalg.norm(Vo[:, 0])),
                            float(np.linalg.norm(trg[:, c, :] - tro[:, :, 0]) / np.linalg.norm(tro[:, :, 0]))))
        out["rel_err_vs_oracle"] = {"value": max(errs), "columns": "3 sampled (operator, forcing) pairs"}
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
