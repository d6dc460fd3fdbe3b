#!/usr/bin/env python
"""Throughput of the split-step method (SSM) on GB300: particle-steps/s.

Workload: the coupled 3-d McKean-Vlasov system with an implicit pairwise drift,
N = 2^18 particles, d = 3, h = 2^-8, T = 1, seed 2 (X_0 ~ N(0, I_3), synthetic).
One "step" is one whole SSM step (§2.3): Philox Brownian increments, the
implicit step solved for all particles (O(N^2) pair sums per pass), the O(N^2)
pairwise drift, and the fused explicit update with FP64 moments.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica (its own seed); value is the units of all ranks over the slowest rank's
time ("weak" scaling).  ``--impl reference`` times the FP64 CPU oracle on the
host cores on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_PART, DIM, H, T_END, SEED = 1 << 18, 3, 2.0 ** -8, 1.0, 2
FP32_LANES_PER_SM = 128
# Algorithmic FP32 flops per pair interaction (FFMA = 2, the special-function op not
# counted), the counts of the method's direct formulas: step-1 residual pair
# (x_j - y)/(1 + |x_j - y|^2): 3 differences, |d|^2 + 1 as 3 FFMA = 6, the weighted
# accumulation 3 FFMA = 6, i.e. 15 (plus the weight sum 1: 16 with it); drift pair
# (y_j - y) exp(-|d|^2/2): 3 differences, |d|^2 as 1 FMUL + 2 FFMA = 5, scaled exponent
# argument 1, 3 FFMA = 6, i.e. 15.
FLOPS_PAIR = {0: 15.0, 1: 15.0}          # 0: step-1 pair sums, 1: step-2 drift
FLOPS_PAIR_WITH_WSUM = 16.0              # step-1 count including the weight sum
# FP32 flops the centred-expansion kernels execute per pair (same sums, fewer
# operations): step 1: 1 + 3 x 2 (q) + 3 x 2 + 1 = 14; drift: 3 x 2 + 3 x 2 + 1 = 13.
FLOPS_PAIR_EXPANDED = {0: 14.0, 1: 13.0}
FORM_NAMES = {0: "scalar", 1: "packed difference form", 2: "packed centred expansion"}
# DRAM bytes (read + write) of one step-1 pair launch of the centred-expansion kernel
# k_pair2x<PK_NEWTON3, threads, rpt> at N = 2^18, from one ncu capture each
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by (threads, targets per
# thread, source chunks) for the shapes and chunk counts the autotuner picks among
# (the partial sums written grow with the chunks); valid only for the kernel sources
# they were measured on (the tile code and its launchers, SHA-256 below), otherwise
# the roofline's traffic is null.
MEASURED_TRAFFIC = {"kernel": ("k_pair2x", 0, 1 << 18),
                    "bytes": {(128, 4, 13): 14148096 + 50406656,
                              (128, 4, 19): 13293568 + 99668480,
                              (128, 4, 26): 16857600 + 159375104,
                              (128, 4, 32): 16656128 + 209221888,
                              (128, 8, 7): 13107456 + 2366464,
                              (128, 8, 10): 13922816 + 25005312,
                              (128, 8, 14): 13753344 + 57894144,
                              (128, 8, 17): 14568192 + 82809088},
                    "sources": ("paper_2105_09688_gb300/csrc/pair_tile.cuh", "paper_2105_09688_gb300/csrc/k_pair.cu"),
                    "sha256": "c9553bd4d11365f463499e3a028266f900b5a19d59551615d0fe122f59e8e401"}


def measured_traffic(kernel, kind, threads, rpt, n, chunks):
    """The ncu DRAM bytes per launch of this kernel if they were measured on the
    current sources, else None."""
    import hashlib
    m = MEASURED_TRAFFIC
    if (kernel, kind, n) != m["kernel"] or (threads, rpt, chunks) not in m["bytes"]:
        return None
    h = hashlib.sha256()
    for f in m["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return m["bytes"][(threads, rpt, chunks)] if h.hexdigest() == m["sha256"] else None
METRIC = "particle-steps/s, N=2^18 d=3: learned+FP32 vs plain FP64 SSM at stated error"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--fp64-steps", type=int, default=1, help="timed steps of the plain FP64 comparison (0 = skip)")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--batched", type=int, default=1, help="also time the 64-ensemble batched form (1/0)")
    p.add_argument("--o-n", type=int, default=1, help="also time the O(N) kernels at N=2^26 against HBM (1/0)")
    p.add_argument("--full-run", type=int, default=1, help="also time one ssm_run over the whole horizon (1/0)")
    p.add_argument("--fixed-passes", type=int, default=0, choices=[0, 1],
                   help="step graphs with a fixed sequence of step-1 pass launches instead of the device-driven "
                        "loop (for profilers that do not follow conditional graph nodes)")
    p.add_argument("--profile-o-n", type=int, default=0, metavar="LOG2N",
                   help="profiling driver: 4 steps of the O(N) coefficient set --profile-set at N = 2^LOG2N in "
                        "the form of --precision, and exit")
    p.add_argument("--profile-set", default="ou", choices=["ou", "gl1", "gl2", "poly", "cs"],
                   help="--profile-o-n: OU (d = 3) or one of the moment-interaction examples")
    p.add_argument("--profile-kernels", type=int, default=0, metavar="LOG2N",
                   help="profiling driver: one SSM step at N = 2^LOG2N, then one step-1 pair pass and one drift "
                        "pair pass (13 + 2 launches of k_pair), and exit")
    p.add_argument("--chunks", type=int, default=0,
                   help="--profile-kernels: source chunks of both pair kinds (0 = planned)")
    p.add_argument("--measure-y", type=int, default=0, choices=[0, 1],
                   help="--profile-kernels: step 1 against mu^Y (one step, no isolated passes)")
    p.add_argument("--profile-batched", type=int, default=0, metavar="K",
                   help="profiling driver: the 64-ensemble batched workload over T = 2^-K (FP32C, one graph "
                        "launch), and exit")
    p.add_argument("--precision", default="fp32c", choices=["fp32c", "fp64"], help="form for --profile-kernels")
    p.add_argument("--packed", type=int, default=0, choices=[0, 1, 2],
                   help="--profile-kernels: pair-kernel form (0 scalar, 1 packed difference form, 2 packed "
                        "centred expansion)")
    p.add_argument("--rpt", type=int, default=4, choices=[4, 8],
                   help="--profile-kernels: targets per thread of the packed kernels (128 threads)")
    return p.parse_args()


def profile_kernels(args):
    """Small, self-terminating case for ncu: the pair kernels of one step plus one
    isolated pass of each kind (nothing is timed or printed as a result)."""
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    prec = S.SSM_FP32C if args.precision == "fp32c" else S.SSM_FP64
    s = S.SSM(d=DIM, N=1 << args.profile_kernels, h=H, T=T_END, coef=S.SSM_COEF_COUPLED3D, seed=SEED, precision=prec,
              fixed_pass_launches=args.fixed_passes,
              measure_y=args.measure_y, tile_chunks=args.chunks)
    if args.packed:
        s.set_plan(0, args.packed, 128, args.rpt)
        s.set_plan(1, args.packed, 128, args.rpt)
    s.step()
    if not args.measure_y:
        s.pair_pass(0)
        s.pair_pass(1)
    s.sync()
    s.close()


def profile_batched(args):
    """Small, self-terminating case for ncu: the batched workload's 64 ensembles over
    a shortened horizon T = 2^-K (their own N and h), one graph launch."""
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    from paper_2105_09688_gb300.convergence import mixed_ensembles
    T = 2.0 ** -args.profile_batched
    descs = [dict(d, T=T) for d in mixed_ensembles() if d["h"] <= T]
    b = S.Batch(descs, precision=S.SSM_FP32C)
    b.run()
    b.sync()
    b.close()


def profile_o_n(args):
    """Small, self-terminating case for ncu: four steps of the O(N) kernels."""
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S
    prec = S.SSM_FP32C if args.precision == "fp32c" else S.SSM_FP64
    if args.profile_set == "ou":
        d, coef, p, m0, s0 = ON_D, S.SSM_COEF_OU, (-1.0, 0.5, 0.5), 1.0, 0.5
    else:
        d, cname, p, m0, s0 = MOMENT_MODELS[args.profile_set]
        coef = getattr(S, cname)
    s = S.SSM(d=d, N=1 << args.profile_o_n, h=2.0 ** -6, T=1.0, coef=coef, seed=7, precision=prec,
              coef_params=p, x0_mean=m0, x0_std=s0)
    s.run_steps(4)
    s.sync()
    s.close()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(seconds):
    """The FP64 oracle on the host cores, one step of the workload restricted to a
    bounded sample of target particles (each target does its full O(N) work)."""
    import oracle as O
    P = O.problem(d=DIM, coef=O.COEF_COUPLED3D, N=N_PART, h=H, seed=SEED)
    x = O.init_x0(P)
    nth = O.num_threads()
    n = max(nth, 8)
    t0 = time.perf_counter()
    O.sample_step(P, x, np.arange(n), 0)
    dt = time.perf_counter() - t0
    n2 = int(max(n, min(N_PART, n * seconds / max(dt, 1e-3))))
    n2 = (n2 + nth - 1) // nth * nth
    idx = np.random.default_rng(0).choice(N_PART, size=min(n2, N_PART), replace=False)
    t0 = time.perf_counter()
    O.sample_step(P, x, idx, 0)
    dt = time.perf_counter() - t0
    return {"value": idx.size / dt, "unit": "particle-steps/s", "cores": nth, "kind": "oracle",
            "sample": "step 0 of N=2^18 d=3 h=2^-8 restricted to %d random target particles (each: FP64 Newton "
                      "implicit solve against all N particles + pairwise drift against all N), %.1f s" %
                      (idx.size, dt)}


def run_reference(args, world, rank):
    if rank != 0:
        return
    cb = cpu_baseline(max(2.0, args.cpu_seconds))
    steps_s = []
    import oracle as O
    P = O.problem(d=DIM, coef=O.COEF_COUPLED3D, N=N_PART, h=H, seed=SEED)
    x = O.init_x0(P)
    # each step a bounded sample: the K + W steps together take about --cpu-seconds
    per = max(O.num_threads(), int(cb["value"] * max(1.0, args.cpu_seconds) / max(1, args.steps + args.warmup)))
    rng = np.random.default_rng(1)
    for k in range(args.warmup + args.steps):
        idx = rng.choice(N_PART, size=min(per, N_PART), replace=False)
        t0 = time.perf_counter()
        O.sample_step(P, x, idx, k)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            steps_s.append(idx.size / dt)
    v = statistics.median(steps_s)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * N_PART / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: X_0 ~ N(0, I_3) from Philox4x32-10 seed 2",
            "config": {"workload": "coupled3d N=2^18 d=3 h=2^-8 T=1 seed=2 (FP64 oracle, sampled targets)",
                       "sample_targets_per_step": per, "l2": "n/a (CPU)"},
            "sampled": "each step times %d of the N targets (each with its full O(N) work); value is targets/s, "
                       "ms_per_step is N / value, an extrapolation to the whole step" % per,
            "cpu_baseline": dict(cb, value=v, sample="%d random targets per step, full O(N) work each" % per),
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def bench_batched(torch, S, stream, carry=1):
    """The 64-ensemble batched workload in one graph launch (FP32C), from the carried
    start of step 1 (ssm_opts.carry_start) or, carry=0, from the plain start."""
    from paper_2105_09688_gb300.convergence import mixed_ensembles
    descs = mixed_ensembles()      # 64 ensembles, N_e log-uniform in [2^10, 2^16], d = 1 and 3
    b = S.Batch(descs, stream=stream, precision=S.SSM_FP32C, carry_start=carry)
    best = b.autotune()
    units = sum(d["N"] * round(d["T"] / d["h"]) for d in descs)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream.synchronize()
    e0.record(stream)
    b.run()                                  # one graph launch: every ensemble to T
    e1.record(stream)
    e1.synchronize()
    b.sync()
    dt = e0.elapsed_time(e1) / 1e3
    st = b.stats()
    res = {"value": units / dt, "unit": "particle-steps/s", "seconds": dt, "ensembles": len(descs),
           "particle_steps": units, "N_range": [min(d["N"] for d in descs), max(d["N"] for d in descs)],
           "batch_steps": st["batch_steps"], "newton_rows": st["newton_rows"], "plan": b.plan(),
           "tuned_pass_ms": best, "graph_launches": 1, "start": "carried" if carry else "plain"}
    b.close()
    return res


ON_LOG2N, ON_D = 26, 3
# The paper's moment-interaction examples timed beside OU: name -> (d, coefficient set,
# parameters, X_0 mean, X_0 standard deviation).
MOMENT_MODELS = {"gl1": (1, "SSM_COEF_GL1", (1.5, 0.5), 1.0, 0.0),
                 "gl2": (1, "SSM_COEF_GL2", (1.5, 0.5), 1.0, 0.0),
                 "poly": (1, "SSM_COEF_POLY", (-1.0,), 1.0, 0.0),
                 "cs": (2, "SSM_COEF_CS", (2.0, 4.0), 1.0, 2.0 ** 0.5)}
# Algorithmic FP64 bytes per particle-step and component of the O(N) step.  OU and
# the polynomial drift take step 1 inside step 2's kernel (X read, the stage Y and
# the new X written: 3 x 8 bytes); the cubic sets run step 1 as its own kernel (X
# read, Y written; then Y read, X written: 4 x 8 bytes).
FUSED_STEP1 = ("SSM_COEF_OU", "SSM_COEF_POLY")


def o_n_bytes(cname, d):
    return (3 if cname in FUSED_STEP1 else 4) * 8 * d


ON_BYTES_PER_PARTICLE_STEP = o_n_bytes("SSM_COEF_OU", ON_D)


def measured_peaks():
    """The generated MEASURED_PEAKS.json of this GPU type ({} if absent)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def fp32_peak(torch, dev):
    """FP32 CUDA-core peak in TFLOP/s: SMs (as the device reports them) x 128 FP32
    lanes x 2 flops (FFMA) x the maximum SM clock (MEASURED_PEAKS.json's sm_max_mhz,
    else the 2070 MHz nominal maximum); returns (TFLOP/s, basis, SMs, MHz)."""
    sms = int(torch.cuda.get_device_properties(dev).multi_processor_count)
    mhz = measured_peaks().get("sm_max_mhz")
    src = "MEASURED_PEAKS.json sm_max_mhz"
    if not mhz:
        mhz, src = 2070.0, "nominal maximum SM clock"
    mhz = float(mhz)
    tf = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    basis = ("FP32 CUDA-core: %d SMs (cudaDevAttrMultiProcessorCount via torch) x %d lanes x 2 flop x %.0f MHz (%s)"
             % (sms, FP32_LANES_PER_SM, mhz, src))
    return tf, basis, sms, mhz


def hbm_peak_gbs():
    """Measured HBM copy bandwidth of this GPU type (generated file), else the
    fallback figure; returns (GB/s, basis)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = json.load(f).get("hbm_gbs")
        if v:
            return float(v), "measured"
    except (OSError, ValueError):
        pass
    return 6800.0, "fallback"


def bench_o_n(torch, S, stream, steps=5, warmup=3):
    """The O(N) kernels against the HBM roofline: the OU coefficient set (both steps
    per particle: step 1 is linear in the particle, so it runs inside step 2's kernel
    with the mean of Y from the moments of X_n), d = 3, N = 2^26 (state 1.6 GB per
    array, far beyond L2), FP64 and FP32C forms.  Algorithmic bytes per
    particle-step: X read, the stage Y and the new X written (FP64 SoA)."""
    peak, basis = hbm_peak_gbs()
    N = 1 << ON_LOG2N
    out = {"workload": "OU d=3 N=2^26 h=2^-6 (one k_euler per step, step 1 fused)",
           "bytes_per_particle_step": ON_BYTES_PER_PARTICLE_STEP, "peak_gbs": peak, "peak_basis": basis}
    for name, prec in (("fp64", S.SSM_FP64), ("fp32c", S.SSM_FP32C)):
        try:
            s = S.SSM(d=ON_D, N=N, h=2.0 ** -6, T=1.0, coef=S.SSM_COEF_OU, seed=7, stream=stream, precision=prec,
                      coef_params=(-1.0, 0.5, 0.5), x0_mean=1.0, x0_std=0.5)
        except S.SSMError as e:
            out[name] = {"error": str(e)}
            continue
        s.run_steps(warmup)
        s.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        s.run_steps(steps)
        ev[1].record(stream)
        ev[1].synchronize()
        dt = ev[0].elapsed_time(ev[1]) / 1e3 / steps
        gbs = N * ON_BYTES_PER_PARTICLE_STEP / dt / 1e9
        out[name] = {"particle_steps_per_s": N / dt, "ms_per_step": dt * 1e3, "achieved_gbs": gbs, "frac": gbs / peak}
        s.close()
    # the paper's moment-interaction examples, FP32C, same N (o_n_bytes per particle-step)
    models = {}
    for name, (d, cname, p, m0, s0) in MOMENT_MODELS.items():
        coef = getattr(S, cname)
        s = S.SSM(d=d, N=N, h=2.0 ** -6, T=1.0, coef=coef, seed=7, stream=stream, precision=S.SSM_FP32C,
                  coef_params=p, x0_mean=m0, x0_std=s0)
        s.run_steps(warmup)
        s.sync()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        s.run_steps(steps)
        ev[1].record(stream)
        ev[1].synchronize()
        dt = ev[0].elapsed_time(ev[1]) / 1e3 / steps
        gbs = N * o_n_bytes(cname, d) / dt / 1e9
        models[name] = {"d": d, "particle_steps_per_s": N / dt, "ms_per_step": dt * 1e3,
                        "bytes_per_particle_step": o_n_bytes(cname, d), "achieved_gbs": gbs, "frac": gbs / peak,
                        "kernels": "k_euler (step 1 fused)" if cname in FUSED_STEP1 else "k_mm_implicit + k_euler"}
        s.close()
    out["fp32c_moment_models"] = models
    return out


def aggregate_replicas(torch, world, local_seconds, local_units, device):
    """Whole-job throughput of independent replicas: every rank's units over the
    slowest rank's time (all-reduce MAX of the time; ranks hold equal work)."""
    total = float(local_seconds)
    if world > 1:
        t = torch.tensor([total], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total = float(t.item())
    return total, world * local_units / total


def time_spread_steps(torch, s, stream, flush, K, M, nvtx=False):
    """Time K single SSM steps spread evenly over the rest of the run (the learned
    start's cost depends on the step index: its carried error needs a few steps to
    settle), with untimed steps in between and an L2 flush before each timed step.
    Each timed step is bracketed by CUDA events on the context's stream.  Returns the
    step times (s) and the step-1 passes and pair rows of the timed steps."""
    x_entry, n_entry = s.get_state()
    n = n_entry
    stride = max(1, (M - n) // K)
    times, passes, rows = [], [], []
    mid = None
    for k in range(K):
        if k == K // 2:
            mid = s.get_state()            # the state at the middle of the timed sample (untimed)
        if n + stride > M:                  # more timed steps than the run has left: go back to the entry state
            s.set_state(x_entry, n_entry)
            n = n_entry
        if stride > 1:
            s.run_steps(stride - 1)         # untimed
        s.sync()
        st0 = s.stats()
        with torch.cuda.stream(stream):
            flush.zero_()                   # L2 flush (not timed)
        ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        if nvtx:
            torch.cuda.nvtx.range_push("timed_steps")   # lets a profiler select exactly the timed steps
        ev[0].record(stream)
        s.run_steps(1)
        ev[1].record(stream)
        if nvtx:
            torch.cuda.nvtx.range_pop()
        ev[1].synchronize()
        st1 = s.stats()
        times.append(ev[0].elapsed_time(ev[1]) / 1e3)
        passes.append(st1["newton_passes"] - st0["newton_passes"])
        rows.append(st1["newton_rows"] - st0["newton_rows"])
        n += stride
    return times, passes, rows, stride, mid


def time_kernel(torch, S, s, stream, which, reps):
    """Average duration of one full pair pass (CUDA events on the context's stream)."""
    s.pair_pass(which)   # warm
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    stream.synchronize()
    ev[0].record(stream)
    for _ in range(reps):
        s.pair_pass(which)
    ev[1].record(stream)
    ev[1].synchronize()
    return ev[0].elapsed_time(ev[1]) / 1e3 / reps


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.profile_kernels:
        profile_kernels(args)
        return
    if args.profile_o_n:
        profile_o_n(args)
        return
    if args.profile_batched:
        profile_batched(args)
        return
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return
    from paper_2105_09688_gb300 import build as B
    B.build()
    import paper_2105_09688_gb300 as S

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    seed = SEED + 1000 * rank
    prec = S.SSM_FP32C
    form = "fp32c"
    if os.path.exists(os.path.join(ROOT, "paper_2105_09688_gb300", "ws_weights.bin")) and hasattr(S, "load_ws"):
        prec, form = S.SSM_FP32C_LEARNED, "learned+fp32c"
    s = S.SSM(d=DIM, N=N_PART, h=H, T=T_END, coef=S.SSM_COEF_COUPLED3D, seed=seed, stream=stream, precision=prec,
              fixed_pass_launches=args.fixed_passes)
    if prec == S.SSM_FP32C_LEARNED:
        S.load_ws(s)
    s.run_steps(1)
    tuned_ms = s.autotune()                    # launch shapes, tuned outside the timed region
    plans = {"step1_pairs": s.plan(0), "drift_pairs": s.plan(1),
             "tuned_pass_ms": [float(v) for v in tuned_ms]}
    for _ in range(args.warmup):
        s.run_steps(1)
    s.sync()
    M_STEPS = int(round(T_END / H))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)   # > 129 MB L2
    st0 = s.stats()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    step_s, step_passes, step_rows, stride, mid_state = time_spread_steps(torch, s, stream, flush, args.steps,
                                                                          M_STEPS, nvtx=True)
    torch.cuda.synchronize()
    clocks = clk.stop()
    s.sync()
    st1 = s.stats()
    total, value = aggregate_replicas(torch, world, float(sum(step_s)), N_PART * args.steps, dev)
    newton_passes = sum(step_passes) / args.steps
    newton_rows = sum(step_rows) / args.steps

    # dominant kernel in isolation (same stream, CUDA events)
    t_newton = time_kernel(torch, S, s, stream, 0, 3)
    t_drift = time_kernel(torch, S, s, stream, 1, 3)
    share_newton = newton_rows / N_PART * t_newton
    dom = 0 if share_newton >= t_drift else 1
    t_dom = t_newton if dom == 0 else t_drift
    flops = FLOPS_PAIR[dom] * N_PART * N_PART
    peak, peak_basis, n_sms, sm_mhz = fp32_peak(torch, dev)
    achieved = flops / t_dom / 1e12
    dom_plan = plans["step1_pairs" if dom == 0 else "drift_pairs"]
    dom_form = dom_plan["form"]
    executed = (FLOPS_PAIR_EXPANDED if dom_form == 2 else FLOPS_PAIR)[dom] * N_PART * N_PART / t_dom / 1e12
    traffic = measured_traffic(("k_pair", "k_pair2", "k_pair2x")[dom_form], dom, dom_plan["threads"],
                               dom_plan["targets_per_thread"], N_PART, dom_plan["chunks"])
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)",
                "kernel": "%s<%s> (%s)" % (("k_pair", "k_pair2", "k_pair2x")[dom_form],
                                           "PK_NEWTON3" if dom == 0 else "PK_DRIFT3", FORM_NAMES[dom_form]),
                "flops_per_pair": FLOPS_PAIR[dom],
                "flops_basis": "algorithmic count of the direct pair formula: residual-only step-1 pair 15 flops, "
                               "drift pair 15 (FFMA = 2, the special-function op not counted)",
                "frac_with_weight_sum": (FLOPS_PAIR_WITH_WSUM * N_PART * N_PART / t_dom / 1e12 / peak
                                         if dom == 0 else None),
                "executed_tflops": executed, "executed_frac": executed / peak,
                "executed_flops_per_pair": (FLOPS_PAIR_EXPANDED if dom_form == 2 else FLOPS_PAIR)[dom],
                "peak_basis": peak_basis, "sms": n_sms, "sm_max_mhz": sm_mhz,
                "kernel_ms": t_dom * 1e3, "other_pair_kernel_ms": (t_drift if dom == 0 else t_newton) * 1e3,
                "other_pair_kernel_frac": FLOPS_PAIR[1 - dom] * N_PART * N_PART
                / (t_drift if dom == 0 else t_newton) / 1e12 / peak}
    # the FP32 pipes measured on this device (ssm_pipe_probe), and the FMA-pipe
    # occupancy of the dominant kernel against the measured packed-FFMA2 rate: the
    # centred expansion issues 8 FMA lane operations a pair (step 1: q in 4, the
    # weighted sums in 4; drift: 3 + 4) as FFMA2
    try:
        pipes = S.ssm_pipe_probe()
        fma_ops = {0: 8.0, 1: 7.0}[dom] if dom_form == 2 else None
        cap = pipes["ffma2"] * n_sms * pipes["clock_ghz"] * 1e9
        roofline["measured_pipes"] = dict(pipes, unit="FP32 lane operations per clock per SM")
        roofline["measured_ffma2_tflops"] = 2.0 * cap / 1e12
        roofline["fma_pipe_frac_of_measured_ffma2"] = (fma_ops * N_PART * N_PART / t_dom / cap) if fma_ops else None
    except S.SSMError as e:
        roofline["measured_pipes"] = {"error": str(e)}

    # end to end through the C ABI, from the middle of the timed sample: every step puts
    # the state in from pinned host memory, takes the step and reads the new state
    # back into pinned host memory (each step's output is the next step's input)
    xh = torch.empty((N_PART, DIM), dtype=torch.float64, pin_memory=True).numpy()
    e2e_steps = max(1, min(args.steps, 5))
    x_mid, n_mid = mid_state
    n_mid = min(n_mid, int(round(T_END / H)) - e2e_steps - 1)
    s.set_state(x_mid, n_mid)
    s.run_steps(1)                                     # untimed: the learned start's carried error is rebuilt
    _, n_e = s.get_state(out=xh)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        s.set_state(xh, n_e)
        s.run_steps(1)
        _, n_e = s.get_state(out=xh)
    e2e_dt = time.perf_counter() - t0
    e2e = {"value": N_PART * e2e_steps / e2e_dt * world, "unit": "particle-steps/s",
           "h2d_bytes_per_step": N_PART * DIM * 8, "d2h_bytes_per_step": N_PART * DIM * 8,
           "steps": e2e_steps}
    s.close()

    # the whole horizon as a user runs it: one ssm_run of M = T/h = 256 steps from X_0,
    # wall time from the first enqueue to the final stream sync (context creation,
    # X_0 and tuning excluded; the shapes tuned above), one run
    full_run = None
    if args.full_run:
        r = S.SSM(d=DIM, N=N_PART, h=H, T=T_END, coef=S.SSM_COEF_COUPLED3D, seed=seed, stream=stream,
                  precision=prec)
        if prec == S.SSM_FP32C_LEARNED:
            S.load_ws(r)
        for w in (0, 1):
            pl = plans["step1_pairs" if w == 0 else "drift_pairs"]
            r.set_plan(w, pl["form"], pl["threads"], pl["targets_per_thread"])
        r.sync()
        torch.cuda.synchronize()
        fev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        t0 = time.perf_counter()
        fev[0].record(stream)
        r.run()
        fev[1].record(stream)
        r.sync()
        wall = time.perf_counter() - t0
        rst = r.stats()
        M = rst["steps"]
        full_run = {"value": N_PART * M / wall, "unit": "particle-steps/s", "steps": M, "wall_s": wall,
                    "device_s": fev[0].elapsed_time(fev[1]) / 1e3, "runs": 1,
                    "timing": "host wall clock from the first enqueue of ssm_run to the final stream sync; "
                              "no L2 flush between steps",
                    "newton_passes_per_step": rst["newton_passes"] / M,
                    "newton_rows_per_step": rst["newton_rows"] / M, "max_passes": rst["max_passes"],
                    "fallbacks": rst["fallbacks"], "floor_accepts": rst["floor_accepts"]}
        r.close()

    # the learned start alone, its network forward on the tensor cores (mma.sync, BF16)
    # and on the CUDA cores (FFMA, FP32), on the same state (the faster is the default)
    ws_forward = None
    if form.startswith("learned"):
        ws_forward = {}
        for fwd, name in ((0, "mma_sync_bf16"), (1, "ffma_fp32")):
            q = S.SSM(d=DIM, N=N_PART, h=H, T=T_END, coef=S.SSM_COEF_COUPLED3D, seed=seed, stream=stream,
                      precision=S.SSM_FP32C_LEARNED, ws_forward=fwd)
            S.load_ws(q)
            q.run_steps(1)
            q.pair_pass(2)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            stream.synchronize()
            ev[0].record(stream)
            for _ in range(5):
                q.pair_pass(2)
            ev[1].record(stream)
            ev[1].synchronize()
            ws_forward[name + "_ms"] = ev[0].elapsed_time(ev[1]) / 5
            q.close()
        ws_forward["default"] = "mma_sync_bf16"

    # the same FP32C form without the learned start (same launch shapes, same timing)
    # the FP32C form without the learned start, from the plain start Y = X and from the
    # carried start (ssm_opts.carry_start: the previous step's converged pair sums), on
    # the tuned shapes and chunk counts, timed like the headline
    def fp32c_form(carry):
        q = S.SSM(d=DIM, N=N_PART, h=H, T=T_END, coef=S.SSM_COEF_COUPLED3D, seed=seed, stream=stream,
                  precision=S.SSM_FP32C, carry_start=carry)
        for w in (0, 1):
            pl = plans["step1_pairs" if w == 0 else "drift_pairs"]
            q.set_plan(w, pl["form"], pl["threads"], pl["targets_per_thread"], chunks=pl["chunks"])
        for _ in range(args.warmup + 1):
            q.run_steps(1)
        q.sync()
        qt_s, _, qrows, _, _ = time_spread_steps(torch, q, stream, flush, args.steps, int(round(T_END / H)))
        qt = sum(qt_s)
        q.close()
        return {"value": N_PART * args.steps / qt, "unit": "particle-steps/s", "ms_per_step": 1e3 * qt / args.steps,
                "newton_rows_per_step": sum(qrows) / args.steps}

    fp32c_plain = fp32c_carried = None
    if form.startswith("learned"):
        fp32c_plain = fp32c_form(0)
        fp32c_carried = fp32c_form(1)

    # plain FP64 GPU SSM on the same workload (comparison of the metric): its own
    # launch shapes (tuned on the same workload at N = 2^16, where a pass takes 1/16 of
    # the time, and applied at 2^18), one untimed warm-up step, then the timed steps
    fp64 = None
    if args.fp64_steps > 0:
        tq = S.SSM(d=DIM, N=1 << 16, h=H, T=T_END, coef=S.SSM_COEF_COUPLED3D, seed=seed, stream=stream,
                   precision=S.SSM_FP64)
        tq.run_steps(1)
        tq.autotune()
        fplans = [tq.plan(0), tq.plan(1)]
        tq.close()
        p = S.SSM(d=DIM, N=N_PART, h=H, T=T_END, coef=S.SSM_COEF_COUPLED3D, seed=seed, stream=stream,
                  precision=S.SSM_FP64)
        for w in (0, 1):
            p.set_plan(w, fplans[w]["form"], fplans[w]["threads"], fplans[w]["targets_per_thread"])
        p.run_steps(1)                      # warm-up step (untimed)
        p.sync()
        pst0 = p.stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        p.run_steps(args.fp64_steps)
        e1.record(stream)
        e1.synchronize()
        dt = e0.elapsed_time(e1) / 1e3
        pst = p.stats()
        fp64 = {"value": N_PART * args.fp64_steps / dt, "unit": "particle-steps/s", "steps": args.fp64_steps,
                "warmup": 1, "ms_per_step": dt * 1e3 / args.fp64_steps,
                "plans": {"step1_pairs": fplans[0], "drift_pairs": fplans[1]},
                "timing": "CUDA events around %d step(s) after one warm-up step; shapes tuned at N=2^16"
                          % args.fp64_steps,
                "newton_passes_per_step": (pst["newton_passes"] - pst0["newton_passes"]) / args.fp64_steps}
        p.close()

    batched = None
    if args.batched:
        batched = bench_batched(torch, S, stream, carry=1)
        plain = bench_batched(torch, S, stream, carry=0)
        batched["plain_start"] = {k: plain[k] for k in ("value", "seconds", "newton_rows")}

    # step 1 against mu^Y (the joint system of the earlier implicit scheme), same workload, FP32C
    my = S.SSM(d=DIM, N=N_PART, h=H, T=T_END, coef=S.SSM_COEF_COUPLED3D, seed=seed, stream=stream,
               precision=S.SSM_FP32C, measure_y=1)
    for w in (0, 1):
        pl = plans["step1_pairs" if w == 0 else "drift_pairs"]
        my.set_plan(w, pl["form"], pl["threads"], pl["targets_per_thread"])
    my.run_steps(1)
    my.sync()
    ms0 = my.stats()
    mev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    mev[0].record(stream)
    my.run_steps(3)
    mev[1].record(stream)
    mev[1].synchronize()
    ms1 = my.stats()
    mdt = mev[0].elapsed_time(mev[1]) / 1e3 / 3
    measure_y = {"value": N_PART / mdt, "unit": "particle-steps/s", "ms_per_step": mdt * 1e3, "steps": 3,
                 "passes_per_step": (ms1["newton_passes"] - ms0["newton_passes"]) / 3}
    my.close()
    o_n = bench_o_n(torch, S, stream) if args.o_n else None

    # kernels of one step: k_newton_begin, the learned start (learned form), a pair-sum
    # and an update launch per step-1 pass (a device-driven loop runs only the passes
    # with work), k_step_stats, the drift pair sums, k_euler, k_advance
    launches_per_step = (1 + (1 if form.startswith("learned") else 0) + 4
                         + 2 * (S.ssm_opts_default().newton_kmax if args.fixed_passes else newton_passes))
    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic: X_0 ~ N(0, I_3) from Philox4x32-10 (seed 2 + 1000 rank)",
            "config": {"workload": "coupled3d N=2^18 d=3 h=2^-8 T=1 seed=2", "form": form,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed between timed steps (512 MB write, untimed)",
                       "timed_steps": "%d single steps spread over the run, every %d-th step after %d warm-up steps "
                                      "(untimed steps in between)" % (args.steps, stride, args.warmup + 1),
                       "newton_passes_per_step": newton_passes, "newton_rows_per_step": newton_rows,
                       "plans": plans},
            "roofline": roofline, "e2e": e2e, "clocks": clocks, "gpu_launches": int(round(launches_per_step * args.steps)),
            "fp32c_without_learned_start": fp32c_plain,
            "fp32c_carried_start": fp32c_carried,
            "fallbacks_per_step": (st1["fallbacks"] - st0["fallbacks"]) / max(1, st1["steps"] - st0["steps"]),
            "plain_fp64": fp64,
            "batched_form": batched,
            "measure_y_form": measure_y,
            "o_n_kernels": o_n,
            "full_run": full_run,
            "learned_start_forward": ws_forward,
            "floor_accepts_per_step": (st1["floor_accepts"] - st0["floor_accepts"]) / max(1, st1["steps"] - st0["steps"]),
            "speedup_vs_plain_fp64": (value / world / fp64["value"]) if fp64 else None}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
