"""Benchmark: particle-timeslices/s of the path action + adjoint gradient.

One step = one whole-path Metropolis-adjusted Langevin update of every chain
(proposal from the path gradient -> action and adjoint gradient of the proposal
-> FP64 Metropolis-Hastings test -> accept/commit), i.e. every stage of the hot
path.  A step evaluates the action and gradient once per chain, so it processes
N * T particle-timeslices per chain.

  python bench.py [--gpus N] [--steps K] [--warmup W]
                  [--config lj500|ho3d|lj108|ragged|ho1d|ho_pamd]
                  [--impl ours|reference]

--impl reference times the CPU oracle (the slow plain FP64 program the GPU path
is checked against) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "particle-timeslices/s for path action+adjoint gradient, batched vs plain GPU"
UNIT = "particle-timeslices/s"
# Algorithmic flop count of the LJ action + adjoint (FMA = 2, rsqrt/rint = 1):
# per unordered in-cutoff pair 44 for the force and 31 for the Hessian-vector
# product; per particle-timeslice 23 for residual, |r|^2 and gradient assembly.
FLOPS_PER_PAIR = 75
FLOPS_PER_UNIT = 23
# Harmonic action + gradient: read x once, write g once per coordinate.


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="lj500")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--h", type=float, default=0.0, help="MALA step (0: per-config default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--T", type=int, default=0, help="override steps per chain (profiling)")
    ap.add_argument("--chains", type=int, default=0, help="override chains per system (profiling)")
    ap.add_argument("--only-kernel", action="store_true",
                    help="time only the action+gradient call (small profiling runs)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default LJ launch shape instead of autotuning it")
    return ap.parse_args()


DEFAULT_H = {"lj500": 2e-7, "lj108": 5e-7, "ragged": 2e-7, "ho3d": 1e-5, "ho1d": 1e-4}


def workload_desc(w):
    import pamd_inputs as inputs  # noqa: F401
    s = w.systems
    if w.name == "ragged":
        return (f"ragged: {len(s)} LJ systems, N in [{min(x.N for x in s)},{max(x.N for x in s)}], "
                f"T in [{min(x.T for x in s)},{max(x.T for x in s)}], rho=0.85, T*=1, rc=min(2.5,L/2), "
                f"D=1, dt={w.dt}, EM start paths")
    x = s[0]
    if x.kind == "lj":
        return (f"{w.name}: LJ liquid N={x.N}, rho=0.85, T*=1, rc={x.rc_eff:g}, box={x.box:.4f}, "
                f"T={x.T} steps, {x.n_chains} chains, D=1, dt={w.dt}, FCC + Euler-Maruyama start path")
    return (f"{w.name}: {x.d}D harmonic oscillator k=1, T={x.T} steps, {x.n_chains} chains, "
            f"D=1, beta=1, dt={w.dt}, start path {w.init}")


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


#: Sources that define each profiled kernel (with the shared header).
KERNEL_SOURCES = {
    "lj_action_kernel": ("lj_kernels.cu", "pamd_internal.cuh"),
    "lj_paired_kernel": ("lj_paired.cu", "pamd_internal.cuh"),
    "ho_vec_kernel": ("ho_kernels.cu", "pamd_internal.cuh"),
    "fragment_line_kernel": ("fragment_kernels.cu", "fragment.cuh", "pamd_internal.cuh"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1907_09529_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(config, kernel):
    """DRAM bytes per launch recorded from an ncu capture of the current kernel source
    (profiles/traffic.json), or None if the kernel's sources changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    ent = rec.get(config, {})
    if ent.get("kernel") != kernel or ent.get("source_hash") != kernel_source_hash(kernel):
        return None
    return ent.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ CPU oracle leg
def oracle_sample(w, budget_s=12.0, single_core=False):
    """Time the CPU oracle's action+gradient on a bounded sample of the workload:
    one chain of the (first) system, slices grown until ~budget_s of CPU work.
    single_core: also time the same oracle on one thread (bit-identical results)
    on a proportionally shorter sample."""
    import oracle
    import pamd_inputs as inputs
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    spec = w.systems[0]
    if w.name == "ragged":
        spec = max(w.systems, key=lambda s: s.N)
    pot = (oracle.lennard_jones(spec.box, spec.rc_eff) if spec.kind == "lj"
           else oracle.harmonic(spec.k))
    nth = oracle.max_threads()

    def run(T, threads=None):
        T = min(T, spec.T)
        s1 = inputs.SystemSpec(spec.kind, spec.N, spec.d, T, 1)
        if spec.kind == "lj":
            x0 = inputs.initial_positions(s1, 1)
            xi = inputs.euler_noise(s1, 2)
            path = oracle.euler_batch(pot, x0, xi, w.D, w.beta, w.dt, store_f32=True)[0]
        else:
            path = inputs.gaussian_path(3, 1, T, spec.d, spec.N, 1.0)[0]
        t0 = time.perf_counter()
        oracle.action_grad(pot, path, w.D, w.beta, w.dt, nthreads=threads or nth)
        return T, time.perf_counter() - t0

    T, dtm = run(8 if spec.kind == "lj" else 4096)
    while dtm < budget_s / 8 and T < spec.T:
        T, dtm = run(min(spec.T, int(T * max(2.0, budget_s / max(dtm, 1e-3) / 4))))
    if dtm < budget_s / 3 and T < spec.T:
        T, dtm = run(min(spec.T, int(T * budget_s / max(dtm, 1e-3))))
    # a whole chain is cheap (oscillator): repeat whole chains up to the budget
    reps, total = 1, dtm
    while total < budget_s / 2 and reps < spec.n_chains:
        total += run(T)[1]
        reps += 1
    units = spec.N * T * reps
    res = {"value": units / total, "unit": UNIT, "cores": nth, "kind": "oracle",
           "sample": f"{reps} chain(s) of {spec.kind} N={spec.N}, {T} of {spec.T} steps each, "
                     f"action+gradient ({total:.1f} s, OpenMP over slices)"}
    if single_core:
        T1, d1 = run(max(2, T // max(1, nth)), threads=1)
        r1 = 1
        while d1 < budget_s / 4 and r1 < 64:
            d1 += run(T1, threads=1)[1]
            r1 += 1
        res["single_core"] = {"value": spec.N * T1 * r1 / d1, "unit": UNIT, "cores": 1,
                              "sample": f"{r1} chain(s), {T1} steps each ({d1:.1f} s, one thread)"}
    return res


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times, res = [], None
    for i in range(args.warmup + args.steps):
        res = oracle_sample(w, budget_s=max(2.0, 60.0 / max(1, args.steps + args.warmup)))
        if i >= args.warmup:
            times.append(1.0 / res["value"])
    v = 1.0 / statistics.mean(times)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload_desc(w)},
           "cpu_baseline": {**res, "value": v},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------ GPU leg
def measure_fp32_peak(dev, stream, target_ms=60.0):
    """FP32 FMA throughput of this GPU, measured with the library's probe kernel
    (8 independent dependent FMA chains per thread, two 1024-thread CTAs per SM;
    scalar fma.rn.f32 and packed fma.rn.f32x2).  Best of 3 timed launches after a
    warm-up, CUDA events on the launching stream, SM clocks sampled meanwhile."""
    import ctypes
    import torch
    from paper_1907_09529_gb300 import _lib
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 2 * sms, 1024
    out = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    res = {"sms": sms, "blocks": blocks, "threads": threads}
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    for packed in (0, 1):
        iters = 20000
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        # size the launch to about target_ms
        e0.record(stream)
        _lib.pamd_fp32_fma_probe(packed, blocks, threads, iters, ctypes.c_void_p(out.data_ptr()), sp)
        e1.record(stream)
        torch.cuda.synchronize()
        iters = max(1000, int(iters * target_ms / max(e0.elapsed_time(e1), 1e-3)))
        best = 0.0
        for _ in range(4):
            e0.record(stream)
            fl = _lib.pamd_fp32_fma_probe(packed, blocks, threads, iters,
                                          ctypes.c_void_p(out.data_ptr()), sp)
            e1.record(stream)
            torch.cuda.synchronize()
            best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        res["packed_tflops" if packed else "scalar_tflops"] = best
    clk = clocks.stop()
    res["sm_mhz"] = clk.get("sm_mhz")
    res["peak_tflops"] = max(res["scalar_tflops"], res["packed_tflops"])
    return res


def measure_fp64_peak(dev, stream, target_ms=40.0):
    """FP64 FMA throughput of this GPU (the library's fma.rn.f64 probe: 8 independent
    dependent chains per thread, two 1024-thread CTAs per SM), best of 3 timed
    launches after a sizing launch, CUDA events on the launching stream."""
    import ctypes
    import torch
    from paper_1907_09529_gb300 import _lib
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 2 * sms, 1024
    out = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = 200
    e0.record(stream)
    _lib.pamd_fp64_fma_probe(blocks, threads, iters, ctypes.c_void_p(out.data_ptr()), sp)
    e1.record(stream)
    torch.cuda.synchronize()
    iters = max(50, int(iters * target_ms / max(e0.elapsed_time(e1), 1e-3)))
    best = 0.0
    for _ in range(3):
        e0.record(stream)
        fl = _lib.pamd_fp64_fma_probe(blocks, threads, iters, ctypes.c_void_p(out.data_ptr()), sp)
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return {"sms": sms, "blocks": blocks, "threads": threads, "fp64_tflops": best}


def host_facts():
    """CPU placement of this process (the host side of the end-to-end copies)."""
    facts = {"cpus": os.cpu_count()}
    try:
        facts["cpus_allowed"] = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        pass
    try:
        facts["numa_nodes"] = len([d for d in os.listdir("/sys/devices/system/node")
                                   if d.startswith("node") and d[4:].isdigit()])
    except OSError:
        pass
    return facts


def rank_seed(w, rank: int) -> int:
    """Every rank draws its own chains: the workload is replicated with a
    rank-dependent seed (weak scaling, no data exchanged between ranks)."""
    return w.seed * 100 + rank


def aggregate(units_per_rank: int, world: int, steps: int, ms_max: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return units_per_rank * world * steps / (ms_max * 1e-3)


def max_over_ranks(ms: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_sampler(args, w, pamd, prob, dev, rank, world):
    """PAMD integration (Fig. 2) with the multilevel sampler: one step = one
    shifting event of every chain (n_sample MC steps + shift/regenerate)."""
    import torch
    from paper_1907_09529_gb300.integrator import PamdIntegrator
    spec = w.systems[0]
    n_shift, n_sample, l_min, l_max = 64, 1, 4, 8
    if spec.T < 4096:
        n_shift, l_min, l_max = 16, 2, 4
    pos = prob.empty(dev)
    g = torch.Generator(device=dev)
    g.manual_seed(rank_seed(w, rank))
    prob.view(pos, 0).copy_(torch.randn(prob.view(pos, 0).shape, generator=g, device=dev))
    integ = PamdIntegrator(prob, n_shift, n_sample, l_min, l_max, seed=rank_seed(w, rank))
    integ.run(pos, max(1, args.warmup))
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    integ.run(pos, args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    clk = clocks.stop()
    units = spec.N * spec.T * spec.n_chains * n_sample
    value = aggregate(units, world, args.steps, ms)
    # one-line paths that fit one CTA run the event as n_sample launches, the last
    # of which also shifts and regrows the path: every MC step reads the path once
    # and writes it once (accepted interiors, or the shifted path)
    nbytes = spec.n_chains * (spec.T + 1) * 4 * 2 * n_sample
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    achieved = nbytes / (ms / args.steps * 1e-3) / 1e9
    peak = float(peaks.get("hbm_gbs", 6800.0))
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import numpy as np
        import oracle
        T = spec.T
        pot = oracle.harmonic(spec.k)
        x = np.random.default_rng(1).standard_normal((T + 1, 1, 1))
        rng = np.random.default_rng(2)
        t0, n = time.perf_counter(), 0
        while time.perf_counter() - t0 < 10.0:
            l = int(rng.integers(l_min, l_max + 1))
            o = int(rng.integers(0, 1 << l))
            z = rng.standard_normal(x.shape)
            lu = np.log(rng.random(oracle.n_fragments(T, l, o)))
            oracle.fragment_step(pot, x, l, o, z, lu, w.D, w.beta, w.dt, exact_ho=True)
            n += 1
        dtm = time.perf_counter() - t0
        cpu = {"value": n * T / dtm, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} multilevel MC steps of one chain (T={T}), {dtm:.1f} s"}
    if rank == 0:
        out = {"metric": "particle-timeslices/s sampled by the PAMD loop (multilevel MC + shift)",
               "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": (f"ho_pamd: 1D harmonic oscillator, PAMD loop (Fig. 2) with "
                                       f"the multilevel sampler (Sec. III), exact propagator, "
                                       f"straight-line regeneration, dt={w.dt}, "
                                       f"N_path={spec.T}, N_sample={n_sample}, N_shift={n_shift}, "
                                       f"levels {l_min}..{l_max}, {spec.n_chains} chains"),
                          "units": "MD force evaluations of the sampler (N_sample * N_path per "
                                   "chain per shifting event)",
                          "l2": "inputs larger than L2" if nbytes / 2 > 129e6 else "L2-resident"},
               "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak,
                            "traffic": profiled_traffic("ho_pamd", "fragment_line_kernel"),
                            "kernel": "fragment_line_kernel<float> (MC step + fused shift)",
                            "peak_note": "of measured; algorithmic bytes = 8 per slice per MC "
                                         "step (read + write); the kernel is issue-bound on "
                                         "the Philox normals and scans, not on HBM"},
               "cpu_baseline": cpu, "e2e": None,
               "gpu_launches": args.steps * n_sample,
               "clocks": clk,
               "accept_rate": float(integ.n_accepted.sum()) / max(1.0, float(integ.n_proposed.sum()))}
        print(json.dumps(out), flush=True)


def launches_per_update(prob):
    """Kernels of one path update: propose, one action launch per harmonic system,
    one LJ launch per block-size class (two when a single-precision batch mixes
    N <= 512 and N > 512), finalize S, reverse, finalize q_fwd and q_rev, accept,
    commit."""
    n_ho = sum(1 for s in prob.systems if s.kind == "harmonic")
    lj = [s.N for s in prob.systems if s.kind == "lj"]
    n_lj = 0
    if lj:
        mixed = min(lj) <= 512 < max(lj) and prob.precision == "fp32"
        n_lj = 2 if mixed else 1
    return 1 + n_ho + n_lj + 1 + 1 + 2 + 1 + 1


def main():
    args = parse()
    import dataclasses
    import pamd_inputs as inputs
    w = inputs.workload(args.config)
    if args.T or args.chains:
        w = dataclasses.replace(w, systems=[dataclasses.replace(
            s, T=args.T or s.T, n_chains=args.chains or s.n_chains) for s in w.systems])
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    import torch.distributed as dist
    import __graft_entry__
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    __graft_entry__.build()
    import paper_1907_09529_gb300 as pamd

    systems = []
    for s in w.systems:
        if s.kind == "lj":
            systems.append(pamd.System("lj", s.N, s.d, s.T, s.n_chains, box=s.box, rc=s.rc_eff))
        else:
            systems.append(pamd.System("harmonic", s.N, s.d, s.T, s.n_chains, k=s.k))
    if w.name == "ho_pamd":
        # the paper's Simulation 3 as validated: exact oscillator propagator,
        # straight-line regeneration
        prob = pamd.Problem(systems, w.D, w.beta, w.dt, "fp32", ho_exact_propagator=True,
                            regenerate_flat=True)
    else:
        prob = pamd.Problem(systems, w.D, w.beta, w.dt, "fp32")
    stream = torch.cuda.current_stream(dev)
    if w.name == "ho_pamd":
        run_sampler(args, w, pamd, prob, dev, rank, world)
        if world > 1:
            dist.destroy_process_group()
        return

    # Start paths, built on the device: Gaussian slices or Euler-Maruyama from FCC / 0.
    seed = rank_seed(w, rank)
    pos = prob.empty(dev)
    for q, s in enumerate(w.systems):
        v = prob.view(pos, q)
        if w.init == "gaussian":
            g = torch.Generator(device=dev)
            g.manual_seed(seed + q)
            v.copy_(torch.randn(v.shape, generator=g, device=dev) / math.sqrt(w.beta * s.k))
        else:
            v[:, 0].copy_(torch.from_numpy(inputs.initial_positions(s, seed)).to(dev))
    if w.init != "gaussian":
        pamd.euler_reference(prob, pos, seed=seed, counter=0)
    tuned = None
    if any(s.kind == "lj" for s in w.systems) and not args.no_autotune and not args.only_kernel:
        from paper_1907_09529_gb300 import autotune as at
        shapes = list(at.candidates(tiles=(8, 16, 32, 64, 96, 128, 160, 192, 224, 256),
                                    windows=(8, 12, 16, 24)))
        best, timings = at.autotune(prob, pos, shapes, reps=2, cache=None)
        tuned = {"tile_steps": best[0], "window_steps": best[4],
                 "ms_per_call": round(timings[json.dumps(best)], 4),
                 "candidates": len(shapes)}
    S, grad = pamd.action_grad(prob, pos)
    torch.cuda.synchronize()
    h = args.h if args.h > 0 else DEFAULT_H.get(w.name, 1e-6)
    nacc = torch.zeros(prob.n_chains, dtype=torch.int32, device=dev)
    units_rank = prob.units

    def step(i):
        pamd.path_update(prob, pos, grad, S, h, 1, seed=seed, counter=1000 + i, n_accepted=nacc)

    if args.only_kernel:
        for _ in range(args.warmup):
            pamd.action_grad(prob, pos, S, grad)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            pamd.action_grad(prob, pos, S, grad)
        e1.record(stream)
        torch.cuda.synchronize()
        if rank == 0:
            ms = e0.elapsed_time(e1) / max(1, args.steps)
            print(json.dumps({"only_kernel": True, "workload": workload_desc(w), "ms_per_call": ms,
                              "units_per_call": units_rank,
                              "units_per_s": units_rank / (ms * 1e-3)}), flush=True)
        return

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    n_acc_steps = float(nacc.sum().item())  # accepted proposals of the warm-up and timed steps
    ms_max = max_over_ranks(ms, dev)
    value = aggregate(units_rank, world, args.steps, ms_max)

    # End to end through the C ABI with host buffers (right after the timed steps,
    # before the long plain-FP64 leg): every step copies the path,
    # its cached gradient and action to the device and the updated ones back.
    e2e = None
    if not args.no_e2e:
        hpos = pos.cpu().pin_memory()
        hgrad = grad.cpu().pin_memory()
        hS = S.cpu().pin_memory()
        hacc = torch.zeros(prob.n_chains, dtype=torch.int32).pin_memory()
        pamd.path_update(prob, hpos, hgrad, hS, h, 1, seed=seed, counter=5, n_accepted=hacc)
        ne = max(3, args.steps)  # the same number of steps as the device-timed region
        # pinned copy rates of this host link, measured on the same buffers (they vary
        # between machines and bound the end-to-end time)
        scratch = torch.empty_like(pos)
        hscratch = torch.empty_like(hpos).pin_memory()
        ce0, ce1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ce0.record(stream)
        scratch.copy_(hpos, non_blocking=True)
        ce1.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = hpos.numel() * hpos.element_size() / (ce0.elapsed_time(ce1) * 1e-3) / 1e9
        ce0.record(stream)
        hscratch.copy_(scratch, non_blocking=True)
        ce1.record(stream)
        torch.cuda.synchronize()
        d2h_gbs = hpos.numel() * hpos.element_size() / (ce0.elapsed_time(ce1) * 1e-3) / 1e9
        del scratch, hscratch
        e2e_clocks = ClockSampler(local)
        e2e_clocks.start()
        step_ms = []
        t0 = time.perf_counter()
        for i in range(ne):
            t1 = time.perf_counter()
            pamd.path_update(prob, hpos, hgrad, hS, h, 1, seed=seed, counter=6 + i, n_accepted=hacc)
            step_ms.append((time.perf_counter() - t1) * 1e3)
        t_e2e = (time.perf_counter() - t0) / ne
        e2e_clk = e2e_clocks.stop()
        nbuf = prob.span * 4
        from paper_1907_09529_gb300 import _lib
        total_ms, chunks = _lib.pamd_pipeline_timeline()
        e2e = {"value": units_rank * world / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": 2 * nbuf + 8 * prob.n_chains + 4 * prob.n_chains,
               "d2h_bytes_per_step": 2 * nbuf + 8 * prob.n_chains + 4 * prob.n_chains,
               "ms_per_step": t_e2e * 1e3,
               "step_ms": [round(v, 2) for v in step_ms],
               "median_ms_per_step": round(statistics.median(step_ms), 3),
               "sm_mhz": e2e_clk.get("sm_mhz"),
               "pinned_copy_gbs": {"h2d": round(h2d_gbs, 1), "d2h": round(d2h_gbs, 1)},
               "pipeline": {"lanes": int(os.environ.get("PAMD_PIPE_LANES", "3")),
                            "last_step_device_ms": round(total_ms, 3),
                            "chunks_ms_in_updated_out": [[round(v, 3) for v in c] for c in chunks]},
               "host": host_facts()}

    # The ragged workload's full path-sampling loop: 100 updates in one call, which
    # the library captures once into a CUDA graph and then replays.
    graph_loop = None
    if w.name == "ragged" and rank == 0:
        nup = 100
        pamd.action_grad(prob, pos, S, grad)  # the cached action and gradient of pos
        pamd.path_update(prob, pos, grad, S, h, nup, seed=seed, counter=50000, n_accepted=nacc)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        pamd.path_update(prob, pos, grad, S, h, nup, seed=seed, counter=60000, n_accepted=nacc)
        g1.record(stream)
        torch.cuda.synchronize()
        gms = g0.elapsed_time(g1)
        graph_loop = {"updates_per_call": nup, "ms_per_call": gms, "ms_per_update": gms / nup,
                      "value": units_rank * nup / (gms * 1e-3), "unit": UNIT,
                      "note": "one pamd_path_update call of 100 updates, replayed from its captured CUDA graph"}

    # Dominant kernel: the action + adjoint kernel alone (one launch per LJ system
    # + a tiny finalize), timed with events on its stream over the same data.
    nk = 10
    gk = torch.empty_like(pos)
    Sk = torch.empty_like(S)
    pamd.action_grad(prob, pos, Sk, gk)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nk):
        pamd.action_grad(prob, pos, Sk, gk)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_kernel = e0.elapsed_time(e1) / nk

    has_lj = any(s.kind == "lj" for s in w.systems)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = json.load(fh)
    except (OSError, ValueError):
        pass
    if has_lj:
        counts = pamd.lj_pair_counts(prob, pos)
        pairs = 0
        off = 0
        for s in w.systems:
            nsl = s.n_chains * (s.T + 1)
            c = counts[off:off + nsl].view(s.n_chains, s.T + 1)[:, :s.T]
            pairs += int(c.sum().item()) // 2
            off += nsl
        flops = FLOPS_PER_PAIR * pairs + FLOPS_PER_UNIT * units_rank
        achieved = flops / (ms_kernel * 1e-3) / 1e12
        probe = measure_fp32_peak(dev, stream)
        peak = probe["peak_tflops"]
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": profiled_traffic(args.config, "lj_paired_kernel"),
                "kernel": "lj_paired_kernel<GRAD=1,512>",
                "peak_note": ("of measured: FP32 FMA throughput probe in this run "
                              f"({probe['sms']} SMs, FMA = 2 flops; scalar "
                              f"{probe['scalar_tflops']:.1f}, packed f32x2 "
                              f"{probe['packed_tflops']:.1f} TFLOP/s at a median "
                              f"{probe['sm_mhz']} MHz; peak = the larger)"),
                "fp32_probe": probe,
                "pairs_per_launch": pairs, "flops_per_launch": flops, "kernel_ms": ms_kernel}
    else:
        nbytes = sum(s.n_chains * (s.T + 1) * s.d * s.N for s in w.systems) * 4 * 2
        achieved = nbytes / (ms_kernel * 1e-3) / 1e9
        peak = float(peaks.get("hbm_gbs", 6800.0))
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": profiled_traffic(args.config, "ho_vec_kernel"),
                "kernel": "ho_vec_kernel<s,true>", "peak_note":
                "of measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)",
                "bytes_per_launch": nbytes, "kernel_ms": ms_kernel}

    # Plain single-path FP64 form of the same action + gradient (one chain per launch),
    # with the library's automatic launch shape (not the shape tuned for the batched
    # single-precision kernel above).
    plain = None
    if not args.no_plain and rank == 0:
        pamd.tune()
        p64 = pamd.Problem(systems, w.D, w.beta, w.dt, "fp64", one_chain_per_launch=True)
        pos64 = pos.double()
        S64, g64 = pamd.action_grad(p64, pos64)
        torch.cuda.synchronize()
        reps = 2
        e0.record(stream)
        for _ in range(reps):
            pamd.action_grad(p64, pos64, S64, g64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / reps
        relS = float(((S64 - Sk).abs() / S64.abs()).max().item())
        relG = float(((g64.float() - gk).norm() / g64.norm()).item())
        plain = {"value": units_rank / (ms64 * 1e-3), "unit": UNIT, "ms_per_call": ms64,
                 "batched_fp32_ms_per_call": ms_kernel,
                 "speedup_batched_vs_plain": ms64 / ms_kernel,
                 "fp32_vs_fp64_rel_err_S": relS, "fp32_vs_fp64_rel_err_grad": relG}
        if has_lj:  # the plain form against the measured FP64 rate (same algorithmic flops)
            p64peak = measure_fp64_peak(dev, stream)
            a64 = flops / (ms64 * 1e-3) / 1e12
            plain["roofline"] = {"bound": "fp64", "achieved": a64,
                                 "peak": p64peak["fp64_tflops"], "unit": "TFLOP/s",
                                 "frac": a64 / p64peak["fp64_tflops"],
                                 "peak_note": "of measured: FP64 FMA probe in this run"}
        del pos64, S64, g64

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(w, single_core=True)

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(w), "precision": "FP32 data, FP64 accumulation",
                       "units_per_step_per_gpu": units_rank, "mala_h": h,
                       "l2": "inputs larger than L2 (no flush needed)"
                       if prob.span * 4 * 4 > 129e6 else "inputs smaller than L2",
                       "parallelism": f"chains sharded over {world} GPU(s), no collective",
                       "lj_launch_shape": tuned or "default"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "plain_fp64": plain,
            "gpu_launches": args.steps * (launches_per_update(prob)) + 1 * args.steps,
            "clocks": clk, "graph_loop": graph_loop, "accept_rate": n_acc_steps / max(
                1, prob.n_chains * (args.steps + args.warmup)),
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
