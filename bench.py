"""Benchmark: cascaded biquad filtering throughput (GS/s) on one GB300.

Workload (headline): order-16 Butterworth low-pass (8 sections) at 0.05 of Nyquist, one float32
signal of 2^28 N(0,1) samples from seed 1 -- the plain single-signal kernel at full size.
A step is one pass of the whole hot path over the signal: one sos_filter_run call (all 8
sections, one kernel launch).  Inputs (1 GiB) and outputs (1 GiB) are both larger than the
129 MB L2, so no flush is needed between steps.

The same JSON line also carries the other measured targets, each timed with CUDA events on the
launching stream: the order-2 plateau (2^29 and 2^30 samples), the order-2 workload at 2^20
samples over a rotating pool of buffers larger than L2, the cyclic-reduction solver at orders 16
and 2, the batched mix (per call and replayed from a CUDA graph, with its ratio to the plain
kernel and per-signal accuracy) and the serving mix (capacity, p50/p99 latency at 80 % load and
the ratio to the plain kernel).  ``--quick`` prints the headline alone.

Prints one JSON line (rank 0).  ``--impl reference`` times the float64 CPU oracle instead,
on a bounded sample of the same workload.
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

WORKLOAD = "order-16 Butterworth lowpass (8 SOS) at 0.05 Nyquist, 1 float32 signal of 2^28 N(0,1) samples, seed 1"
N_SAMPLES = 1 << 28
ORDER = 16
WN = 0.05
SEED = 1
BYTES_PER_SAMPLE = 8  # 4 B read + 4 B written: the algorithmic traffic of the filter (Sec. IV-C, Eq. 28)
CPU_SAMPLE = 1 << 24  # oracle sample per step of the reference arm
# DRAM bytes (read + write) of one launch of the timed kernel on the 2^28 workload, per (solver, N):
# an ncu capture of the same kernel on 2^26 samples scaled by 4.  An entry must be re-captured (or
# removed) whenever its kernel changes.
SOLVER_CR, SOLVER_PH, SOLVER_DTCR, SOLVER_TC = 1, 2, 3, 4
TRAFFIC_BYTES_2P28 = {
    # sos_lane_kernel<8, 64, 7> at 2^26 samples: 268,859,904 B read + 211,708,672 B written
    (SOLVER_PH, 64): 4 * (268859904 + 211708672),
    # sos_tc_kernel<8> at 2^26 samples: 269,061,632 B read + 213,409,792 B written
    (SOLVER_TC, 64): 4 * (269061632 + 213409792),
}
PH_GROUPS_PER_BLOCK = 7
CR_GROUPS_PER_BLOCK = {32: 8, 64: 4}


def kernel_name(solver: int, N: int, K: int, W: int = 0) -> str:
    """The kernel a run launches, by solver, samples per lane, sections per pass and groups per tile."""
    k = min(K, 8)
    if solver == SOLVER_PH:
        w = W or PH_GROUPS_PER_BLOCK
        return (f"sos_lane_kernel<{k}, {N}, {w}> (PH factorization, {k} sections, N = {N} samples per lane, "
                f"{w} groups per block)")
    if solver == SOLVER_DTCR:
        return (f"sos_dtcr_kernel<{k}, 64> (double-thread-group cyclic reduction, {k} sections, N = 64 samples per "
                "lane, 4 groups of two warps per block)")
    if solver == SOLVER_TC:
        return (f"sos_tc_kernel<{k}> (PH factorization on the tensor cores: tcgen05 TF32 products split three "
                f"ways, TMA staging; {k} sections, N = 64 samples per lane, 8 groups per block)")
    return (f"sos_cascade_kernel<{k}, {N}> (cyclic reduction, {k} sections, N = {N} samples per lane, "
            f"{CR_GROUPS_PER_BLOCK.get(N, '?')} groups per block)")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = max(smax, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The largest of every rank's value (the job's time is its slowest replica's); no-op at one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(samples_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job GS/s of `world` independent replicas (weak scaling): all samples over the slowest time."""
    return samples_per_rank * world / (ms_max * 1e-3) / 1e9


def bench_reference(args):
    """The float64 CPU oracle on the host cores, bounded sample of the same workload."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    import workloads
    from workloads import designs
    sos = designs.butter_lowpass(ORDER, WN)
    x = workloads.normal_f32(SEED, CPU_SAMPLE)
    oracle.sosfilt(sos, x[:4096])  # build/load
    times = []
    for _ in range(args.warmup):  # untimed steps, the same work as a timed one
        oracle.sosfilt(sos, x)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sosfilt(sos, x)
        times.append(time.perf_counter() - t0)
    per = float(np.mean(times))
    gss = CPU_SAMPLE / per / 1e9
    line = {"impl": "reference", "metric": "GS/s", "value": gss, "unit": "GS/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"first 2^{int(np.log2(CPU_SAMPLE))} samples per step"},
            "cpu_baseline": {"value": gss, "unit": "GS/s", "cores": 1, "kind": "oracle",
                             "sample": f"first 2^{int(np.log2(CPU_SAMPLE))} samples of the workload, 1 core"},
            "e2e": {"value": gss, "unit": "GS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_leg(sos, x_host, y_dev=None, chunk: int = 1 << 24):
    """The float64 oracle over the whole workload on one host core.

    It runs in chunks of ``chunk`` samples with the state carried between them (bit-identical to one
    pass), and only the oracle calls are timed.  Given the device output ``y_dev`` of the timed run
    (a tensor), the same pass also yields the accuracy measure of Sec. IV-F over every sample,
    max|y - y_ref| / max|y_ref|, against the design's bound, and (untimed) the same measure against
    the oracle run on the coefficients rounded to float32, which leaves out the part of the error
    that the rounding of the coefficients alone causes.  Returns (baseline, accuracy or None).
    """
    import oracle
    from workloads import designs
    oracle.sosfilt(sos, x_host[:1024])  # load the oracle outside the timed calls
    n = x_host.shape[0]
    keep = y_dev is not None
    sos32 = np.asarray(sos, dtype=np.float32).astype(np.float64)
    z = np.zeros((sos.shape[0], 2))
    z32 = np.zeros((sos.shape[0], 2))
    dt = num = den = num32 = den32 = 0.0
    for a in range(0, n, chunk):
        t0 = time.perf_counter()
        ref, z = oracle.sosfilt(sos, x_host[a:a + chunk], zi=z, return_state=True, keep_output=keep)
        dt += time.perf_counter() - t0
        if keep:
            got = y_dev[a:a + chunk].cpu().numpy().astype(np.float64)
            num = max(num, float(np.abs(got - ref).max()))
            den = max(den, float(np.abs(ref).max()))
            ref32, z32 = oracle.sosfilt(sos32, x_host[a:a + chunk], zi=z32, return_state=True)
            num32 = max(num32, float(np.abs(got - ref32).max()))
            den32 = max(den32, float(np.abs(ref32).max()))
    base = {"value": n / dt / 1e9, "unit": "GS/s", "cores": 1, "kind": "oracle",
            "sample": f"the whole workload (2^{int(np.log2(n))} samples) once on one host core, {dt:.1f} s"}
    acc = None
    if keep:
        acc = {"max_rel_error": num / den if den > 0 else num, "bound": designs.tolerance_for(sos),
               "measure": "max|y - y_oracle| / max|y_oracle| over every sample of the timed run's output",
               "max_rel_error_vs_f32_coefficients": num32 / den32 if den32 > 0 else num32}
    return base, acc


def cpu_wavefront_leg(x_host):
    """The float64 oracle run as the multi-core wavefront of Sec. III-A on the host cores (one thread
    per section at most: more would only wait), over a bounded sample of the workload; its output is
    bit-identical to the one-core oracle's."""
    import oracle
    from workloads import designs
    sos = designs.butter_lowpass(ORDER, WN)
    threads = max(1, min(_cores(), ORDER // 2))
    n = min(x_host.shape[0], 1 << 24)
    oracle.sosfilt_wavefront(sos, x_host[:4096], threads=threads, block=8192)
    t0 = time.perf_counter()
    oracle.sosfilt_wavefront(sos, x_host[:n], threads=threads, block=8192, keep_output=False)
    dt = time.perf_counter() - t0
    return {"value": n / dt / 1e9, "unit": "GS/s", "cores": threads, "kind": "oracle, multi-core wavefront",
            "sample": f"first 2^{int(np.log2(n))} samples, groups of 8192 samples, {threads} threads, {dt:.2f} s"}


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_launches(torch, fn, steps: int, stream) -> float:
    """Mean ms per call of fn() over `steps` calls, CUDA events on `stream`, synchronized on both
    sides."""
    e0, e1 = _events(torch)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(steps):
        fn(i)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def hbm_roofline(samples: int, ms: float, kernel: str, traffic=None):
    """The roofline object of a launch over `samples` samples taking `ms`: 8 algorithmic bytes per
    sample against the measured copy bandwidth."""
    peak, kind = _peaks()
    achieved = BYTES_PER_SAMPLE * samples / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": kind, "kernel": kernel}


def fp32_fma_roof(torch, dev, sm_max_mhz):
    """Peak FP32 FMA rate of the device: SMs x 128 FP32 lanes x the maximum SM clock (one FMA per lane
    per cycle), in TFMA/s, with how it was derived."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(sm_max_mhz) if sm_max_mhz else 2070.0
    return sms * 128 * mhz * 1e6 / 1e12, f"derived: {sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz (max SM clock)"


def tc_tensor_roofline(K: int, n: int, ms: float) -> dict:
    """Tensor-core roofline of the PH kernel on the tensor cores.  Per 128-row unit (8192 samples) it
    issues 24 TF32 MMAs of 128 x 80 x 8 (the Toeplitz and state-response products, three ways) and 6
    (2K <= 8: 3) of 128 x 64 x 8 (the correction), i.e. 576 (528) flops per sample; the peak is the
    measured bf16 burst rate times the nominal TF32 / bf16 ratio 1.1 / 2.25."""
    corr = 6 if K > 4 else 3
    flops_per_sample = (24 * 2 * 128 * 80 * 8 + corr * 2 * 128 * 64 * 8) / 8192
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        bf16, kind = 1900.0, "fallback"
    peak = bf16 * 1.1 / 2.25
    achieved = flops_per_sample * n / (ms * 1e-3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "flops_per_sample": flops_per_sample, "peak_kind": kind,
            "peak_how": "bf16 dense burst (MEASURED_PEAKS.json) x nominal TF32/bf16 ratio 1.1/2.25"}


def chosen_kernel(K: int, n: int):
    """(solver, N, groups per tile) that a default-tuned filter of K sections runs on n samples: the
    autotuner's choice when it has run in this process, else the library default (PH at N = 64, 7)."""
    from paper_2607_23763_gb300 import autotune_choice
    c = autotune_choice(K, n, with_groups=True)
    return tuple(c) if c[:2] != (0, 0) else (SOLVER_PH, 64, PH_GROUPS_PER_BLOCK)


def plain_rate(torch, sos, x, y, steps: int, warmup: int, tuning=None) -> float:
    """ms per sos_filter_run of one filter over all of x (both larger than L2)."""
    from paper_2607_23763_gb300 import SosFilter
    f = SosFilter(sos, tuning=tuning)
    for _ in range(warmup):
        f.run(x, y)
    ms = time_launches(torch, lambda i: f.run(x, y), steps, torch.cuda.current_stream())
    assert f.sync_status() == 0
    f.close()
    return ms


def order2_plateau_leg(torch, dev, steps: int, warmup: int):
    """The order-2 workload's filter (Butterworth at 0.2 Nyquist) over 2^29 and 2^30 samples; the
    plateau is the mean of the two rates (the paper's plateau protocol, Sec. IV-F, at GB300 sizes)."""
    import workloads
    from workloads import designs
    sos = designs.butter_lowpass(2, 0.2)
    n_max = 1 << 30
    x = torch.from_numpy(workloads.normal_f32(0, n_max)).to(dev)
    y = torch.empty_like(x)
    pts = {}
    for lg in (29, 30):
        n = 1 << lg
        ms = plain_rate(torch, sos, x[:n], y[:n], steps, warmup)
        pts[f"2^{lg}"] = {"value": n / ms / 1e6, "ms_per_launch": ms}
    del x, y
    ms_mean = 0.5 * (pts["2^29"]["ms_per_launch"] / 2 + pts["2^30"]["ms_per_launch"] / 4)  # per 2^28 samples
    value = 0.5 * (pts["2^29"]["value"] + pts["2^30"]["value"])
    sv, nv, wv = chosen_kernel(1, 1 << 30)
    roof = hbm_roofline(1 << 28, ms_mean, kernel_name(sv, nv, 1, wv))
    roof["achieved"] = value * BYTES_PER_SAMPLE  # mean of the two points' GB/s
    roof["frac"] = roof["achieved"] / roof["peak"]
    return {"workload": "order-2 Butterworth lowpass (1 SOS) at 0.2 Nyquist, 1 float32 signal of N(0,1) samples, "
                        "seed 0, 2^29 and 2^30 samples", "value": value, "unit": "GS/s", "points": pts,
            "roofline": roof, "target_frac": 0.70}


def config1_leg(torch, dev, launches: int = 256, pool: int = 64):
    """Order-2 Butterworth at 0.2 Nyquist on 2^20 samples (seed 0, zero state): one launch per step,
    cycling through `pool` input/output pairs (pool x 8 MiB, more than 4x L2) so that no launch finds
    its input in L2.  Accuracy over the whole output of the first pair."""
    import oracle
    import workloads
    from workloads import designs
    from paper_2607_23763_gb300 import SosFilter
    sos = designs.butter_lowpass(2, 0.2)
    n = 1 << 20
    xh = workloads.normal_f32(0, n)
    xs = torch.from_numpy(xh).to(dev).repeat(pool, 1)  # pool copies of the same signal
    ys = torch.empty_like(xs)
    f = SosFilter(sos)
    for i in range(2 * pool):
        f.run(xs[i % pool], ys[i % pool])
    ms = time_launches(torch, lambda i: f.run(xs[i % pool], ys[i % pool]), launches, torch.cuda.current_stream())
    assert f.sync_status() == 0
    # the paper's protocol: the launches captured into a CUDA graph (one launch per pool pair) and
    # the graph replayed, so that no host work stands between launches
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            for i in range(pool):
                f.run(xs[i], ys[i], stream=side)
    torch.cuda.synchronize()
    graph.replay()
    reps = max(1, launches // pool)
    g_ms = time_launches(torch, lambda i: graph.replay(), reps, torch.cuda.current_stream()) / pool
    assert f.sync_status() == 0
    del graph
    err = oracle.rel_err(ys[0].cpu().numpy(), oracle.sosfilt(sos, xh))
    f.close()
    return {"workload": "order-2 Butterworth lowpass (1 SOS) at 0.2 Nyquist, 1 float32 signal of 2^20 N(0,1) "
                        "samples, seed 0, zero state",
            "value": n / g_ms / 1e6, "unit": "GS/s", "ms_per_launch": g_ms,
            "how": f"{pool} launches (one per pool pair) captured into a CUDA graph, replayed {reps} times",
            "eager": {"value": n / ms / 1e6, "ms_per_launch": ms,
                      "how": f"{launches} sos_filter_run calls back to back on the stream"},
            "l2": f"{pool} input/output pairs of 2^20 samples cycled ({pool * 8} MiB, more than 4x L2)",
            "launches": launches, "roofline": hbm_roofline(n, g_ms, kernel_name(*chosen_kernel(1, n)[:2], 1, chosen_kernel(1, n)[2])),
            "accuracy": {"max_rel_error": err, "bound": designs.tolerance_for(sos)}}


def cr_solver_leg(torch, dev, x16, y16, steps: int, warmup: int, fma_peak):
    """The divide-and-conquer cyclic-reduction solver (Sec. II-D/E) on the order-16 workload and on
    the order-2 filter, 2^28 samples each, at its default N, single-warp (STCR) and double-thread-group
    (DTCR, Sec. IV-E)."""
    import workloads
    from workloads import designs
    out = {}
    for order, wn, x, y in ((16, WN, x16, y16), (2, 0.2, None, None)):
        sos = designs.butter_lowpass(order, wn)
        if x is None:
            x = torch.from_numpy(workloads.normal_f32(0, 1 << 28)).to(dev)
            y = torch.empty_like(x)
        K = order // 2
        N = 64 if K == 1 else 32  # the library's default N of cyclic reduction
        n = x.numel()
        fma = 10 * K
        for solver, tag, NN in ((SOLVER_CR, "", N), (SOLVER_DTCR, "dtcr_", 64)):
            ms = plain_rate(torch, sos, x, y, steps, warmup, tuning={"solver": solver})
            out[f"{tag}order{order}"] = {
                "value": n / ms / 1e6, "unit": "GS/s", "ms_per_launch": ms, "N": NN,
                "roofline": hbm_roofline(n, ms, kernel_name(solver, NN, K)),
                "roofline_alu": {"bound": "alu", "achieved": fma * n / (ms * 1e-3) / 1e12, "peak": fma_peak,
                                 "unit": "TFMA/s", "frac": fma * n / (ms * 1e-3) / 1e12 / fma_peak,
                                 "fma_per_sample": fma}}
    return out


def _leg(name, fn, line, *a, **kw):
    """Run one extra measurement into line[name]; a failure is recorded there and the rest goes on."""
    t0 = time.perf_counter()
    try:
        line[name] = fn(*a, **kw)
    except Exception as e:  # a failed leg must not cost the headline
        line[name] = {"error": f"{type(e).__name__}: {e}"}
    if isinstance(line[name], dict):
        line[name]["wall_s"] = round(time.perf_counter() - t0, 1)


def bench_ours(args):
    import torch
    import torch.distributed as dist

    import workloads
    from workloads import designs
    from paper_2607_23763_gb300 import SosFilter

    t_start = time.perf_counter()
    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    sos = designs.butter_lowpass(ORDER, WN)
    x_host = workloads.normal_f32(SEED, N_SAMPLES)
    choice = None
    if not args.no_autotune and not (args.N or args.carry or args.solver or args.lbw or args.deterministic or
                                     args.groups):
        # the library's autotuner picks the launch configuration per order and length (outside the
        # timed region); the filter below, with default tuning, then runs its choice
        from paper_2607_23763_gb300 import autotune, autotune_choice
        autotune()
        choice = autotune_choice(ORDER // 2, N_SAMPLES, with_groups=True)
        if choice[:2] == (0, 0):
            choice = None
    tuning = {}
    if args.N:
        tuning["N"] = args.N
    if args.lbw:
        tuning["lookback_width"] = args.lbw
    if args.carry:
        tuning["carry"] = args.carry
    if args.solver:
        tuning["solver"] = args.solver
    if args.deterministic:
        tuning["deterministic"] = 1
    if args.groups:
        tuning["groups_per_cta"] = args.groups
    tuning = tuning or None
    f = SosFilter(sos, tuning=tuning)
    x = torch.from_numpy(x_host).to(dev)
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        f.run(x, y)
    barrier()
    assert f.sync_status() == 0
    start, stop = _events(torch)
    with ClockSampler(local) as clk:
        barrier()
        start.record(stream)
        for _ in range(args.steps):
            f.run(x, y)
        stop.record(stream)
        barrier()
    ms = max_over_ranks(start.elapsed_time(stop), world, dev)
    ms_step = ms / args.steps
    gss = replica_rate(N_SAMPLES, world, ms_step)
    assert f.sync_status() == 0

    # end to end through the C ABI with host buffers: sos_filter_run_host copies the pinned input
    # in, filters and copies the output back in overlapping chunks, every step
    xh = torch.from_numpy(x_host).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    for _ in range(2):
        f.run_host(xh, yh)
    barrier()
    e_steps = max(3, min(args.steps, 10))
    t0 = time.perf_counter()
    for _ in range(e_steps):
        f.run_host(xh, yh)
    barrier()
    e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / e_steps, world, dev)
    e_gss = replica_rate(N_SAMPLES, world, e_ms)
    # the same through the direct mode: the kernels read and write the pinned buffers in place
    e_direct = None
    try:
        from paper_2607_23763_gb300._binding import HOST_DIRECT
        for _ in range(2):
            f.run_host(xh, yh, chunk=HOST_DIRECT)
        barrier()
        t0 = time.perf_counter()
        for _ in range(e_steps):
            f.run_host(xh, yh, chunk=HOST_DIRECT)
        barrier()
        d_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / e_steps, world, dev)
        e_direct = {"value": replica_rate(N_SAMPLES, world, d_ms), "unit": "GS/s", "ms_per_step": d_ms,
                    "h2d_bytes_per_step": 4 * N_SAMPLES, "d2h_bytes_per_step": 4 * N_SAMPLES,
                    "how": "sos_filter_run_host(..., SOS_HOST_DIRECT): the kernel reads the pinned input and "
                           "writes the pinned output over the CPU-GPU link, no staging"}
    except Exception as e:  # recorded, the staged number stands
        e_direct = {"error": f"{type(e).__name__}: {e}"}
    staged = {"value": e_gss, "unit": "GS/s", "ms_per_step": e_ms,
              "how": "sos_filter_run_host, staged: chunks of 2^24 samples copied in, filtered and copied out on "
                     "three overlapping streams"}
    use_direct = e_direct.get("value", 0.0) > e_gss
    del xh, yh

    # the kernel that ran: the autotuner's choice, else the tuning's (the library default is PH at
    # N = 64; a carry scheme or lookback width selects cyclic reduction, by default at N = 32)
    if choice:
        kid = tuple(choice)
    elif args.solver:
        kid = (args.solver, args.N or (64 if args.solver in (SOLVER_PH, SOLVER_DTCR, SOLVER_TC) else 32), args.groups)
    elif args.carry or args.lbw:
        kid = (SOLVER_CR, args.N or 32, 0)
    else:
        kid = (SOLVER_PH, args.N or 64, args.groups)
    K = ORDER // 2
    clocks = clk.summary()
    # the FP32 roof the method meets first at high order: its FMAs per sample (PH: 4K for the
    # particular pass with b0 = 1 plus 2K for the correction; cyclic reduction: 8K + 2K, Sec. IV-C)
    fma_per_sample = 6 * K if kid[0] == SOLVER_PH else 10 * K
    fma_peak, fma_kind = fp32_fma_roof(torch, dev, clocks.get("sm_max_mhz"))
    alu_achieved = fma_per_sample * N_SAMPLES / (ms_step * 1e-3) / 1e12
    traffic = (TRAFFIC_BYTES_2P28.get(kid[:2]) if (N_SAMPLES == 1 << 28 and ORDER == 16 and not args.lbw
                                               and args.carry != 2) else None)
    line = {
        "metric": "GS/s", "value": gss, "unit": "GS/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "samples": N_SAMPLES, "sections": K,
                   "N": kid[1], "L": 32, "groups_per_cta": kid[2] or None,
                   "solver": {SOLVER_PH: "PH", SOLVER_CR: "CR", SOLVER_DTCR: "DTCR", SOLVER_TC: "PH-TC"}[kid[0]],
                   "deterministic": bool(args.deterministic),
                   "autotuned": choice is not None,
                   "l2": "inputs and outputs larger than L2 (1 GiB each)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": hbm_roofline(N_SAMPLES, ms_step, kernel_name(kid[0], kid[1], K, kid[2]), traffic),
        "roofline_alu": {"bound": "alu", "achieved": alu_achieved, "peak": fma_peak, "unit": "TFMA/s",
                         "frac": alu_achieved / fma_peak, "fma_per_sample": fma_per_sample, "peak_kind": fma_kind},
        "e2e": {"value": e_direct["value"] if use_direct else e_gss, "unit": "GS/s",
                "h2d_bytes_per_step": 4 * N_SAMPLES, "d2h_bytes_per_step": 4 * N_SAMPLES,
                "mode": "direct" if use_direct else "staged", "staged": staged, "direct": e_direct},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if kid[0] == SOLVER_TC:
        # the products run on the tensor cores, not the FP32 pipe: their TF32 rate instead
        line.pop("roofline_alu")
        line["roofline_tensor"] = tc_tensor_roofline(K, N_SAMPLES, ms_step)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"], line["accuracy"] = cpu_baseline_leg(sos, x_host, y)
        line["cpu_wavefront"] = cpu_wavefront_leg(x_host)
    f.close()
    if rank == 0 and not args.quick:
        # the other targets, measured on this GPU in the same run (rank 0 only)
        steps, warm = 10, 3
        _leg("cr_solver", cr_solver_leg, line, torch, dev, x, y, steps, warm, fma_peak)
        del x, y
        torch.cuda.empty_cache()
        _leg("order2_plateau", order2_plateau_leg, line, torch, dev, steps, warm)
        torch.cuda.empty_cache()
        _leg("config1_2p20", config1_leg, line, torch, dev)
        torch.cuda.empty_cache()
        plain = {}
        _leg("batched", batched_leg, line, torch, dev, steps=5, warmup=3, no_cpu=args.no_cpu, plain=plain,
             autotune=not args.no_autotune)
        torch.cuda.empty_cache()
        _leg("serving", serving_leg, line, torch, dev, n_streams=args.streams, per_stream=args.chunks_per_stream,
             n_open=args.serving_open_requests, plain=plain, autotune=not args.no_autotune)
    line["wall_s"] = round(time.perf_counter() - t_start, 1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batch_sample_leg(specs, xs, ys, n_sample: int = 64):
    """The float64 oracle over the first `n_sample` signals of a batched mix (one host core): its
    rate, and each signal's error max|y - y_oracle| / max|y_oracle| against the bound the GPU tests
    apply to random mixes (the plain bound, widened where float32 arithmetic itself cannot reach it:
    tests/_tol.py).  `xs` are the host inputs, `ys` the outputs of the timed run (tensors)."""
    import oracle
    from tests import _tol
    errs, within, dt, total = [], 0, 0.0, 0
    for (sos, n, _), x, y in zip(specs[:n_sample], xs[:n_sample], ys[:n_sample]):
        t0 = time.perf_counter()
        ref = oracle.sosfilt(sos, x)
        dt += time.perf_counter() - t0
        total += n
        err = oracle.rel_err(y.cpu().numpy(), ref)
        errs.append(err)
        within += err < _tol.bound(sos, x, ref, random_mix=True)
    base = {"value": total / dt / 1e9, "unit": "GS/s", "cores": 1, "kind": "oracle",
            "sample": f"the first {len(errs)} signals of the mix ({total} samples), one host core, {dt:.1f} s"}
    acc = {"signals": len(errs), "within_bound": int(within), "max_rel_error": float(max(errs)),
           "median_rel_error": float(np.median(errs)),
           "measure": "per signal max|y - y_oracle| / max|y_oracle|, bound as in the GPU tests for random mixes"}
    return base, acc


def plain_rates_by_sections(torch, dev, plain: dict, steps: int = 5, warmup: int = 3) -> dict:
    """The plain single-signal kernel's GS/s on 2^28 samples for 1, 2, 4 and 8 random sections (the
    orders of the mixes), cached in `plain`."""
    if plain:
        return plain
    import workloads
    from workloads import designs
    x = torch.from_numpy(workloads.normal_f32(1, 1 << 28)).to(dev)
    y = torch.empty_like(x)
    for K in (1, 2, 4, 8):
        sos = designs.random_sections(workloads.uniform_f64(7, 3 * K, stream=1).reshape(K, 3))
        plain[K] = (1 << 28) / plain_rate(torch, sos, x, y, steps, warmup) / 1e6
    return plain


def batched_leg(torch, dev, steps: int = 5, warmup: int = 3, no_cpu: bool = False, plain=None,
                autotune: bool = True, n_sig: int = 4096):
    """Batched mix: 4096 signals (orders 2/4/8/16, lengths 2^10..2^22) in one sos_filter_run_batch call
    per step; GS/s of the whole batch, the same batch as a prepared plan replayed from a CUDA graph,
    and both as a fraction of the plain kernel's time for the same signals at each signal's order.
    With `autotune`, the batch autotuner first picks each signal's tile geometry (N = 64 or 32 samples
    per lane) by section count and length (outside the timed region)."""
    import workloads
    from paper_2607_23763_gb300 import (SosFilter, run_batch, batch_sync_status, BatchPlan, autotune_batch,
                                        autotune_batch_choice)

    specs = [workloads.batched_signal(i) for i in range(n_sig)]
    tune_gss = autotune_batch() if autotune else None
    geom = [autotune_batch_choice(sos.shape[0], n) or 64 for sos, n, _ in specs]
    fs = [SosFilter(sos) for sos, _, _ in specs]
    xs, xs_host = [], []  # host copies kept only for the CPU leg's sample
    for i, (_, n, seed) in enumerate(specs):
        x = workloads.normal_f32(seed, n)
        xs.append(torch.from_numpy(x).to(dev))
        if i < 64:
            xs_host.append(x)
    ys = [torch.empty_like(x) for x in xs]
    total = sum(n for _, n, _ in specs)
    for _ in range(warmup):
        run_batch(fs, xs, ys)
    torch.cuda.synchronize()
    assert batch_sync_status(0) == 0
    stream = torch.cuda.current_stream()
    with ClockSampler(dev.index or 0) as clk:
        ms = time_launches(torch, lambda i: run_batch(fs, xs, ys), steps, stream)
    assert batch_sync_status(0) == 0
    # the same call through the C ABI with the caller's host arrays built once (as a C caller keeps
    # them): the library's per-call cost without the Python binding's marshalling of 4096 tensors
    import ctypes
    from paper_2607_23763_gb300 import load_library
    lib = load_library()
    arr = lambda vals, t=ctypes.c_void_p: (t * n_sig)(*vals)
    hf, hx, hy = arr([f.handle for f in fs]), arr([x.data_ptr() for x in xs]), arr([y.data_ptr() for y in ys])
    hn = arr([x.numel() for x in xs], ctypes.c_int64)
    sh = ctypes.c_void_p(stream.cuda_stream)
    c_call = lambda i: lib.sos_filter_run_batch(n_sig, ctypes.addressof(hf), ctypes.addressof(hx), ctypes.addressof(hy),
                                                ctypes.addressof(hn), sh)
    for _ in range(warmup):
        c_call(0)
    c_ms = time_launches(torch, c_call, steps, stream)
    assert batch_sync_status(0) == 0
    # the same batch as a prepared plan captured into a CUDA graph, replayed
    plan = BatchPlan(fs, xs, ys)
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        plan.launch(side)
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.launch()
    for _ in range(warmup):
        graph.replay()
    with ClockSampler(dev.index or 0) as clk_graph:
        graph_ms = time_launches(torch, lambda i: graph.replay(), steps, stream)
    assert plan.status() == 0
    plan.close()
    del graph
    rate = plain_rates_by_sections(torch, dev, plain if plain is not None else {})
    plain_ms = sum(n / rate[sos.shape[0]] / 1e6 for sos, n, _ in specs)
    out = {"workload": f"batched mix: {n_sig} float32 signals, lengths round(2^U), U~U[10,22], orders uniform over "
                       "{2,4,8,16}, random stable sections, N(0,1) input, seeds 1000+i",
           "samples": total, "l2": "inputs and outputs larger than L2",
           # the workload's configuration: one persistent launch, captured into a CUDA graph
           "value": total / graph_ms / 1e6, "unit": "GS/s", "ms_per_step": graph_ms, "steps": steps,
           "vs_plain_kernel": plain_ms / graph_ms,
           "how": "prepared batch plan (one persistent launch over every class) captured into a CUDA graph, "
                  "replayed once per step",
           "per_call": {
               "c_abi": {"value": total / c_ms / 1e6, "ms_per_step": c_ms, "vs_plain_kernel": plain_ms / c_ms,
                         "how": "sos_filter_run_batch per step, host arrays built once"},
               "python_binding": {"value": total / ms / 1e6, "ms_per_step": ms, "vs_plain_kernel": plain_ms / ms,
                                  "how": "run_batch per step: the binding marshals 4096 tensors per call",
                                  "clocks": clk.summary()}},
           "plain_gss_by_order": {str(2 * k): v for k, v in rate.items()},
           "target_vs_plain": 0.60, "clocks": clk_graph.summary(),
           "tile_geometry": {
               "autotuned": tune_gss is not None, "L": 32, "groups_per_tile": 7,
               "signals_N32": sum(g == 32 for g in geom),
               "samples_N32": sum(n for (_, n, _), g in zip(specs, geom) if g == 32),
               "autotune_gss": None if tune_gss is None else {
                   "layout": "[sections 1..8][signal length 2^12, 2^15, 2^18, 2^21][N = 64, N = 32]",
                   "value": np.round(tune_gss, 1).tolist()}}}
    if not no_cpu:
        out["cpu_baseline"], out["accuracy"] = batch_sample_leg(specs, xs_host, ys)
    for f in fs:
        f.close()
    return out


def _autotune_plain(args):
    """The library's autotuner, so that the plain kernel the mixes are compared with is the fastest
    configuration per order (as in the default run)."""
    if not args.no_autotune:
        from paper_2607_23763_gb300 import autotune
        autotune()


def bench_batched(args):
    import torch
    torch.cuda.set_device(0)
    _autotune_plain(args)
    leg = batched_leg(torch, torch.device("cuda", 0), args.steps, args.warmup, args.no_cpu,
                      autotune=not args.no_autotune, n_sig=args.batch_signals)
    line = {"metric": "GS/s", "value": leg["value"], "unit": "GS/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": leg["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": leg["workload"], "samples": leg["samples"], "l2": leg["l2"]},
            "gpu_launches": args.steps}
    line.update({k: v for k, v in leg.items() if k not in line and k not in ("workload", "samples", "l2")})
    print(json.dumps(line), flush=True)


def serving_leg(torch, dev, n_streams: int = 10000, per_stream: int = 10, n_open: int = 110000, plain=None,
                autotune: bool = True):
    """Serving mix: streams with orders 2/4/8/16 at 40/30/20/10 %, chunks of U[4096, 65536] samples.
    Capacity = closed loop (every chunk queued at t = 0); then Poisson arrivals at 80 % of capacity;
    latency = completion - scheduled arrival; p50/p99 over the requests after a 10 % warm-up.  The
    capacity is also given as a fraction of the plain kernel's rate for the same chunks (each chunk
    at the plain 2^28-sample rate of its order)."""
    import workloads
    from paper_2607_23763_gb300 import SosServer, autotune_batch, autotune_batch_choice

    if autotune and autotune_batch_choice(1, 1 << 15) == 0:
        autotune_batch()  # each chunk's tile geometry by order and length (outside the timed region)
    srv = SosServer(budget_bytes=16 << 30)
    t0 = time.perf_counter()
    soss = [workloads.serving_stream(s) for s in range(n_streams)]
    sids = [srv.add_stream(sos) for sos in soss]
    t_setup = time.perf_counter() - t0
    hi = 65536
    pool = torch.from_numpy(workloads.normal_f32(77, 1 << 24)).to(dev)  # chunk inputs are windows of this pool
    out = torch.empty(n_streams * hi, device=dev)
    rng = np.random.default_rng(5)

    def requests(n_req, arrivals):
        sid = rng.integers(0, n_streams, n_req)
        lens = np.array([workloads.serving_chunk_len(int(s), int(c)) for s, c in
                         zip(sid, rng.integers(0, 1 << 20, n_req))], dtype=np.int64)
        off = rng.integers(0, pool.numel() - hi, n_req) // 4 * 4  # chunks start on 16-byte boundaries
        xp = pool.data_ptr() + 4 * off
        yp = out.data_ptr() + 4 * (sid * hi)
        lat = srv.replay([sids[s] for s in sid], xp, yp, lens, arrivals)
        return sid, lens, lat

    # closed loop: capacity
    n_cap = n_streams * per_stream
    sid_c, lens_c, lat_c = requests(n_cap, np.zeros(n_cap))
    capacity = lens_c.sum() / lat_c.max() / 1e9
    # open loop: Poisson arrivals at 80 % of capacity
    mean_len = (4096 + hi) / 2
    rate = 0.8 * capacity * 1e9 / mean_len
    n_open = max(n_open, 1000)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_open))
    _, lens, lat = requests(n_open, arrivals)
    keep = slice(n_open // 10, None)
    p50, p99 = np.percentile(lat[keep] * 1e3, [50, 99])
    wall = arrivals[-1] + lat[-1]
    st = srv.stats()
    srv.close()
    res = {"workload": f"serving mix: {n_streams} streams, orders 2/4/8/16 at 40/30/20/10 %, chunks U[4096, 65536] "
                       "float32 samples, Poisson arrivals at 80 % of measured capacity, 16 GiB budget, state "
                       "resident on the device",
           "value": lens.sum() / wall / 1e9, "unit": "GS/s", "open_loop_requests": n_open,
           "closed_loop_requests": n_cap, "capacity_gss": capacity, "offered_gss": 0.8 * capacity,
           "latency_ms": {"p50": p50, "p99": p99, "max": float(lat.max() * 1e3)},
           "batches": st["batches"], "max_batch": st["max_batch_seen"], "setup_s": t_setup}
    if plain is not None:
        rates = plain_rates_by_sections(torch, dev, plain)
        plain_s = sum(int(n) / rates[soss[int(s)].shape[0]] / 1e9 for s, n in zip(sid_c, lens_c))
        res["capacity_vs_plain_kernel"] = plain_s / lat_c.max()
        res["target_vs_plain"] = 0.60
    res["one_batch"] = serving_batch_probe(torch, dev, soss, pool)
    return res


def serving_batch_probe(torch, dev, soss, pool, m: int = 4096, reps: int = 3):
    """Where a serving batch's time goes: one sos_filter_run_batch_ex call over m chunks shaped like
    the serving mix (the first m streams' filters, chunk lengths U[4096, 65536], states carried), timed
    on the host (the call itself: planning and launches) and on the device (CUDA events)."""
    import workloads
    from paper_2607_23763_gb300 import SosFilter, run_batch, batch_sync_status
    fs = [SosFilter(sos) for sos in soss[:m]]
    lens = [workloads.serving_chunk_len(i, 0) for i in range(m)]
    xs, off = [], 0
    for n in lens:
        xs.append(pool[off:off + n])
        off = (off + n + 3) // 4 * 4
        if off + 65536 > pool.numel():
            off = 0
    ys = [torch.empty(n, device=dev) for n in lens]
    zs = [torch.zeros(f.K, 2, device=dev) for f in fs]
    zf = [torch.zeros(f.K, 2, device=dev) for f in fs]
    from paper_2607_23763_gb300 import BatchPlan
    for _ in range(2):
        run_batch(fs, xs, ys, zis=zs, zfs=zf)
    torch.cuda.synchronize()
    host = []
    for _ in range(reps):  # fewer calls than the library's scratch sets: no call waits for the device
        t0 = time.perf_counter()
        run_batch(fs, xs, ys, zis=zs, zfs=zf)
        host.append(time.perf_counter() - t0)
    torch.cuda.synchronize()
    assert batch_sync_status(dev.index or 0) == 0
    # the device's share: the same batch as a prepared plan, whose launches enqueue no host work
    plan = BatchPlan(fs, xs, ys, zis=zs, zfs=zf)
    plan.launch()
    dev_ms = time_launches(torch, lambda i: plan.launch(), reps, torch.cuda.current_stream())
    assert plan.status() == 0
    plan.close()
    for f in fs:
        f.close()
    return {"chunks": m, "samples": int(sum(lens)), "host_ms_per_call": 1e3 * float(np.median(host)),
            "device_ms_per_call": dev_ms, "device_gss": sum(lens) / dev_ms / 1e6}


def bench_serving(args):
    import torch
    torch.cuda.set_device(0)
    _autotune_plain(args)
    leg = serving_leg(torch, torch.device("cuda", 0), args.streams, args.chunks_per_stream, args.open_requests, {},
                      autotune=not args.no_autotune)
    line = {"metric": "GS/s", "value": leg["value"], "unit": "GS/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": leg["workload"], "open_loop_requests": leg["open_loop_requests"],
                       "closed_loop_requests": leg["closed_loop_requests"]}}
    line.update({k: v for k, v in leg.items() if k not in line and k != "workload"})
    print(json.dumps(line), flush=True)


def bench_precision(args):
    """Precision stress: order-16 resonator bank at pole radius 0.999, 2^30 samples (N(0,1) plus a unit
    sinusoid at 0.32 pi, seed 4): GS/s and, from the CPU-baseline leg's oracle pass, the error against
    the float64 oracle over every sample."""
    import numpy as np
    import torch

    import workloads
    from workloads import designs
    from paper_2607_23763_gb300 import SosFilter

    torch.cuda.set_device(0)
    sos = designs.resonator_bank()
    n = 1 << 30
    x_host = workloads.normal_f32(4, n, sin_amp=1.0, sin_omega=0.32 * np.pi)
    f = SosFilter(sos)
    x = torch.from_numpy(x_host).cuda()
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        f.run(x, y)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        f.run(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    assert f.sync_status() == 0
    ms = e0.elapsed_time(e1) / args.steps
    del x
    base, acc = cpu_baseline_leg(sos, x_host, y)
    line = {"metric": "GS/s", "value": n / ms / 1e6, "unit": "GS/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "precision stress: order-16 resonator bank, 8 sections with poles at radius "
                                   "0.999, angles evenly spaced in [0.30 pi, 0.34 pi]; 2^30 float32 samples of "
                                   "N(0,1) plus sin(0.32 pi n), seed 4", "carry": "float32"},
            "max_rel_error": acc["max_rel_error"], "bound": acc["bound"], "accuracy": acc, "cpu_baseline": base}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="plain", choices=["plain", "batched", "serving", "precision"],
                    help="plain = the order-16 single-signal workload (default); batched / serving mixes")
    ap.add_argument("--streams", type=int, default=10000, help="serving: streams")
    ap.add_argument("--batch-signals", type=int, default=4096,
                    help="batched: the first M signals of the mix (4096 = the workload; fewer for profiling captures)")
    ap.add_argument("--chunks-per-stream", type=int, default=10, help="serving: closed-loop chunks per stream")
    ap.add_argument("--open-requests", type=int, default=110000, help="serving: open-loop requests")
    ap.add_argument("--serving-open-requests", type=int, default=30000,
                    help="open-loop requests of the serving measurement inside the default line")
    ap.add_argument("--quick", action="store_true", help="the headline alone (no extra measurements)")
    ap.add_argument("--N", type=int, default=0, help="samples per thread (16/32/64); 0 = library default")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline leg")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (profiling runs: a fixed sequence of launches)")
    ap.add_argument("--carry", type=int, default=0, help="1 = one carry per tile for the cascade, 2 = per section")
    ap.add_argument("--solver", type=int, default=0,
                    help="1 = cyclic reduction, 2 = PH factorization, 3 = DTCR, 4 = PH on the tensor cores; 0 = default")
    ap.add_argument("--deterministic", action="store_true",
                    help="fixed lookback composition (bit-reproducible outputs; PH solver)")
    ap.add_argument("--lbw", type=int, default=0, help="lookback width (predecessor blocks per round / 32); 0 = default")
    ap.add_argument("--groups", type=int, default=0, help="PH groups per tile (7, or 10 at N = 64); 0 = default")
    ap.add_argument("--order", type=int, default=16, help="filter order (16 = the workload; others for sweeps)")
    ap.add_argument("--log2n", type=int, default=28,
                    help="signal length 2^log2n (28 = the workload; smaller only for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    global N_SAMPLES, WORKLOAD, ORDER
    if args.order != 16:
        ORDER = args.order
        WORKLOAD = WORKLOAD.replace("order-16", f"order-{ORDER}").replace("(8 SOS)", f"({ORDER // 2} SOS)")
    if args.log2n != 28:
        N_SAMPLES = 1 << args.log2n
        WORKLOAD = WORKLOAD.replace("2^28", f"2^{args.log2n}")
    if args.impl == "reference":
        bench_reference(args)
    elif args.workload == "batched":
        bench_batched(args)
    elif args.workload == "serving":
        bench_serving(args)
    elif args.workload == "precision":
        bench_precision(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
