"""Benchmark of the GB300 THC-RR-CCSD residual library.

One step = one evaluation of the projected residual (Algs. 1-10: T1 dressing,
fused Cholesky-slab pass, Algs. 6 and 7, Algs. 9-10) plus the energy, through
thc_residual, on the synthetic system o=40, v=200, P=400, G=1200, K=600
(seed 1).  The state (Zc, t1) is the solver's iterate after two Jacobi steps
from zero.  Default arithmetic: float64 throughout, with the products run on
the tensor cores as exact integer slices combined in float64 (agreeing with
the float64 CUDA-core products to float64 rounding); --precision fp64 keeps
every product on the CUDA cores, --precision mixed is the float32 + bf16x3
policy.

  value      residual evaluations / s with inputs resident in HBM (device
             pointers), CUDA events on the library's stream, max over ranks
  e2e        the same through host (pinned) buffers: H2D of (Zc, t1) and D2H
             of (sigma, Omega1, E) inside every step
  roofline   dominant kernel: algorithmic flops per launch / average launch
             time, from the library's per-step CUDA-event profile
  cpu_baseline  the FP64 CPU oracle, one full residual on the same system
  solve      solves from zero of the same system: float64 to |r| < 1e-8 (its
             energy is the reference), mixed precision, and mixed precision
             with the learned preconditioner (trained on the GPU on pairs
             from six small systems of the same family); for each the wall
             time until the energy is within 1e-6 Eh of the reference

Multi-GPU (torchrun): every rank evaluates residuals of its own system
(independent problems, weak scaling, no collective in the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "o40_v200_P400_G1200_K600"
WORKLOAD = WORKLOAD_NAME = METRIC = None


def set_workload(name):
    """Select one of synth.CONFIGS (named by size) as the benchmarked system."""
    global WORKLOAD, WORKLOAD_NAME, METRIC
    from synth import CONFIGS
    o, v, P, G, K, seed = CONFIGS[name]
    WORKLOAD = dict(o=o, v=v, P=P, G=G, K=K, seed=seed)
    WORKLOAD_NAME = f"THC-RR-CCSD o={o} v={v} P={P} G={G} K={K} seed={seed}"
    METRIC = f"residual evals/s (THC-RR-CCSD, o={o} v={v} P={P} G={G} K={K})"


set_workload(DEFAULT_WORKLOAD)
UNIT = "residual evals/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# Float64 and float32 CUDA-core peaks of one GB300 at the maximum SM clock:
# 152 SMs x (FMA lanes per SM) x 2 flops x 2.07 GHz (64-bit: 2 lanes per SM,
# 32-bit: 128); `bench.py --peaks` measures them with thc_probe_alu.
FP64_ALU_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# float32 operations issued per (I, X, Y, Z) term by each triangle kernel:
# float64 kernel 3.5 float64 flops (t shared by the mirror outputs); float32
# kernel over X pairs (P a multiple of 4) 2 FMA-pipe lane operations (one
# packed multiply and three packed FMAs per pair of X and pair of mirror
# outputs), 3 for the unpaired float32 kernel; float-pair kernel 43 float32
# operations per pair of mirror outputs (19 for t, 12 per accumulation).
TRI_ISSUED = {"fp64": 3.5, "mixed": 2.0, "fp64tc": 21.5}
TRI_KERNEL = {"fp64": "k_triangle_sym64", "mixed": "k_triangle_pair", "fp64tc": "k_triangle_df"}


def _mixed_triangle_unpaired():
    """The paired float32 triangle needs P % 4 == 0 and P <= 28000."""
    return WORKLOAD is not None and not (WORKLOAD["P"] % 4 == 0 and WORKLOAD["P"] <= 28000)

# DRAM bytes (read + write) of one triangle launch at o=40, v=200, P=400,
# G=1200, from one ncu capture of the kernel that runs at that precision
# (None: not captured since the kernel last changed).
TRIANGLE_TRAFFIC_BYTES = {"fp64": 97.58e9 + 0.52e9, "fp64tc": 36.653e9 + 0.517e9,
                          "mixed": 12.702e9 + 0.249e9}


def triangle_roofline(precision, flops, ms, launches, share):
    """Roofline of the triangle kernel from its per-step CUDA-event time.
    flops: the algorithmic count, 5 per (I, X, Y, Z) term."""
    achieved = (flops / launches) / (ms / launches * 1e-3) / 1e12     # TFLOP/s
    terms_per_s = achieved * 1e12 / 5.0
    n_issued = TRI_ISSUED[precision]
    kernel = TRI_KERNEL[precision]
    if precision == "mixed" and _mixed_triangle_unpaired():
        n_issued, kernel = 3.0, "k_triangle_f32"
    if precision == "fp64":
        pipe = FP64_ALU_TFLOPS * 1e12 / 2.0        # float64 FMA-lane operations / s
        issued = terms_per_s * TRI_ISSUED["fp64"] / 2.0
        unit_peak, src = FP64_ALU_TFLOPS, "derived: 152 SMs x 2 fp64 FMA lanes x 2 x 2.07 GHz"
    else:
        pipe = FP32_ALU_TFLOPS * 1e12 / 2.0        # float32 lane operations / s
        issued = terms_per_s * n_issued
        unit_peak, src = FP32_ALU_TFLOPS, "derived: 152 SMs x 128 fp32 lanes x 2 x 2.07 GHz"
    peak = pipe / n_issued * 5.0 / 1e12 if precision != "fp64" else unit_peak
    out = {"kernel": kernel + " (Alg. 6 line 11)",
           "bound": "alu", "achieved": achieved, "unit": "TFLOP/s",
           "achieved_counts": "algorithmic flops, 5 per (I, X, Y, Z) term",
           "frac_issued": issued / pipe,
           "frac_issued_counts": "operations the kernel issues per term (%g) / pipe rate"
                                 % n_issued,
           "frac_algorithmic": achieved / unit_peak,
           "frac_algorithmic_peak": unit_peak,
           "traffic": TRIANGLE_TRAFFIC_BYTES[precision] if WORKLOAD_NAME.startswith(
               "THC-RR-CCSD o=40 v=200 P=400 G=1200") else None,
           "traffic_unit": "bytes per launch (ncu dram__bytes_read + write)",
           "share_of_step": share}
    if precision == "fp64tc":
        # float64 result from float32 pairs: the bound is the FP32 pipe at
        # 21.5 operations per term
        out.update({"peak": peak, "frac": achieved / peak,
                    "peak_source": src + "; / 21.5 float32 operations per term x 5 flops",
                    "frac_of_fp64_alu_peak": achieved / FP64_ALU_TFLOPS})
    else:
        out.update({"peak": unit_peak, "frac": achieved / unit_peak, "peak_source": src})
    return out


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        self.proc.wait()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, flag in zip(names, parts[5:9]):
                    if flag.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, dist, device):
    """The largest per-rank value (a time) over all ranks; x itself at N = 1."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, ms_max):
    """Residual evaluations per second of the whole job: every rank evaluates
    one residual of its own system per step, and the slowest rank sets the
    step time."""
    return world * 1e3 / ms_max


# Systems whose float64 Cholesky vectors exceed this many bytes are generated
# on the GPU and handed to the library a slab at a time.
HOST_L_LIMIT = 64e9


def _system(seed_offset=0, device=None):
    from synth import make_device_system, make_system
    w = WORKLOAD
    args = (w["o"], w["v"], w["P"], w["G"], w["K"], w["seed"] + seed_offset)
    if 8.0 * w["K"] * (w["o"] + w["v"]) ** 2 > HOST_L_LIMIT:
        return make_device_system(*args, device=device)
    return make_system(*args)


def _context(pkg, s, dev=None, **kw):
    """A library context for s: from its Cholesky array, or (device-generated
    systems) from its slabs through thc_load_cholesky."""
    import torch
    if s.L is not None:
        if dev is None:
            return pkg.Context(s.eps_o, s.eps_v, s.Y, s.L, s.x, s.z, **kw)
        tens = [torch.from_numpy(a).to(dev) for a in (s.eps_o, s.eps_v, s.Y, s.L, s.x, s.z)]
        return pkg.Context(*tens, **kw)
    ctx = pkg.Context(s.eps_o, s.eps_v, s.Y, None, s.x, s.z, n_k=s.K, **kw)
    lo, hi = 0, s.K
    if kw.get("shard") is not None:
        from paper_2111_11473_gb300.shard import shard_bounds
        lo, hi = shard_bounds(s.K, *kw["shard"])
    for k0, Lk in s.cholesky_slabs(nk=32, k_lo=lo, k_hi=hi):
        ctx.load_cholesky(k0, Lk)
        del Lk
    torch.cuda.empty_cache()
    ctx.finish_init()
    return ctx


def oracle_residual_seconds(s, Zc, t1):
    """Time one full FP64 oracle residual (+ energy) on the host cores."""
    from oracle import closed_shell as cs, solver as osolver, thc
    H = cs.Hamiltonian.from_inputs(s.eps_o, s.eps_v, s.L, s.x, s.z)
    t0 = time.perf_counter()
    osolver.projected_residual(H, s.Y, Zc, t1)
    cs.energy(H, t1, thc.amplitudes(s.Y, Zc, s.o))
    return time.perf_counter() - t0


def _threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return max(n)
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args):
    """The oracle arm: FP64 CPU oracle on the host cores, same system and metric."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    if args.workload != DEFAULT_WORKLOAD:
        # The oracle forms the 4-index amplitudes and integrals (o^2 v^2 and
        # v^4 doubles): beyond the default size they do not fit host memory.
        print(json.dumps({"impl": "reference", "unavailable":
                          "the FP64 oracle forms 4-index tensors that do not fit host memory "
                          "at this size"}), flush=True)
        return 0
    import numpy as np
    from synth import random_amplitudes
    s = _system()
    Zc, t1 = random_amplitudes(s.P, s.o, s.v, 3, t2_scale=0.01, t1_scale=0.01)
    # One oracle residual at this size takes about a minute; the arm runs at
    # most one untimed and two timed evaluations so that it ends in minutes.
    warm = min(args.warmup, 0)
    steps = max(1, min(args.steps, 2))
    for _ in range(warm):
        oracle_residual_seconds(s, Zc, t1)
    times = [oracle_residual_seconds(s, Zc, t1) for _ in range(steps)]
    sec = sum(times) / len(times)
    value = 1.0 / sec
    sample = "one full FP64 oracle residual + energy of the bench system per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus, "steps": steps, "warmup": warm, "ms_per_step": 1e3 * sec,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD_NAME, "oracle": "numpy FP64"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def serial_shard_check(pkg, s, dev, stream, ctx, args):
    """The float64 residual (tensor-core products) at the mixed solve's
    converged point, evaluated as the sum of `args.fp64_check_shards` shard
    contexts made one after another on this GPU, so that only a part of the
    float64 Cholesky vectors is on the device at a time; compared with the
    mixed residual and energy at the same point."""
    import numpy as np
    import torch
    hist = []
    Zc, t1, rep = ctx.solve(r_tol=args.solve_rtol, e_tol=1e-8, max_iter=args.max_iter,
                            history=hist, raise_on_failure=False)
    mixed = ctx.residual(Zc, t1)
    ctx.close()   # the float64 shard contexts need the device memory
    n = args.fp64_check_shards
    parts, shards = [], []
    for i in range(n):
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        c = _context(pkg, s, dev, precision=pkg.THC_PREC_FP64_TC, stream=stream, shard=(i, n))
        init_s = time.perf_counter() - t0
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        parts.append(c.residual(Zc, t1))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        shards.append({"init_s": init_s, "residual_ms": e0.elapsed_time(e1),
                       "device_gb_in_use": torch.cuda.mem_get_info(dev)[1] / 1e9 -
                                           torch.cuda.mem_get_info(dev)[0] / 1e9})
        c.close()
    sig = sum(p[0] for p in parts)
    sig1 = sum(p[1] for p in parts)
    E = sum(p[2] for p in parts)
    return {"mixed_solve": {"iters": rep.iters, "status": rep.status, "energy": rep.energy,
                            "r_norm": rep.r_norm, "wall_s": rep.wall_s},
            "fp64_residual_ms": sum(x["residual_ms"] for x in shards),
            "shards": shards,
            "energy_fp64": E, "energy_mixed": mixed[2], "dE_mixed_minus_fp64": mixed[2] - E,
            "max_abs_dsigma": float(np.abs(mixed[0] - sig).max()),
            "max_abs_sigma_fp64": float(np.abs(sig).max()),
            "norm_dsigma1": float(np.linalg.norm(mixed[1] - sig1)),
            "norm_sigma1_fp64": float(np.linalg.norm(sig1))}


def run_sharded(args, pkg, dev, stream, dist, world, rank):
    """One system split over the ranks: every step evaluates each rank's
    shard of the residual and sums the parts (sigma, Omega1, energy) with one
    NCCL all-reduce; the state is a generic one at amplitude scale 0.01
    (a residual's cost does not depend on the values)."""
    import torch
    from synth import random_amplitudes
    s = _system(device=dev)
    prec = {"fp64": pkg.THC_PREC_FP64, "fp64tc": pkg.THC_PREC_FP64_TC,
            "mixed": pkg.THC_PREC_MIXED}[args.precision]
    ctx = _context(pkg, s, dev, precision=prec, stream=stream, shard=(rank, world))
    Zc0, t10 = random_amplitudes(s.P, s.o, s.v, 7, t2_scale=0.01, t1_scale=0.01)
    Zc = torch.from_numpy(Zc0).to(dev)
    t1 = torch.from_numpy(t10).to(dev)
    sig = torch.empty((s.P, s.P), dtype=torch.float64, device=dev)
    sig1 = torch.empty((s.o, s.v), dtype=torch.float64, device=dev)
    flat = torch.empty(s.P * s.P + s.o * s.v + 1, dtype=torch.float64, device=dev)

    def step():
        _, _, e = ctx.residual(Zc, t1, out=(sig, sig1))
        flat[:s.P * s.P].copy_(sig.reshape(-1))
        flat[s.P * s.P:-1].copy_(sig1.reshape(-1))
        flat[-1] = e
        dist.all_reduce(flat)

    for _ in range(max(3, args.warmup)):
        step()
    sampler = ClockSampler(dev.index)
    sampler.start()
    dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, dev)
    energy = float(flat[-1])
    ctx.close()
    if rank == 0:
        line = {"metric": METRIC, "value": 1e3 / ms, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f64" if args.precision != "mixed" else "f32+bf16x3",
                "data": "synthetic",
                "config": {"workload": WORKLOAD_NAME, "precision": args.precision,
                           "parallelism": f"one system in {world} shards (Cholesky vectors, "
                                          "Alg. 6 rows; Alg. 7 on the last), NCCL all-reduce "
                                          "of sigma, Omega1, energy per step",
                           "state": "generic, amplitude scale 0.01"},
                "energy": energy, "clocks": clocks}
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()
    return 0


def run_peaks():
    """Roofline denominators and product rates measured through the library:
    float64 / float32 / packed-pair FMA throughput, and one 4096^3 product
    per tensor-core mode (CUDA events, milliseconds per product)."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_2111_11473_gb300 import binding as b
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(0)
    sampler.start()
    out = {"fp64_fma_tflops": b.probe_alu(0, stream), "fp32_fma_tflops": b.probe_alu(1, stream),
           "fp32x2_fma_tflops": b.probe_alu(2, stream),
           "derived": {"fp64_alu_tflops": FP64_ALU_TFLOPS, "fp32_alu_tflops": FP32_ALU_TFLOPS}}
    n = 4096
    bf16 = _peaks().get("bf16_tflops")
    gemm = {}
    for mode, name, nprod in ((0, "bf16x3", 3), (1, "bf16x3_with_pack", 3), (2, "bf16x1", 1),
                              (3, "float64_slices", 36)):
        ms = b.probe_gemm(mode, n, n, n, 10 if mode < 3 else 3, stream)
        alg = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
        gemm[name] = {"ms": ms, "algorithmic_tflops": alg, "bf16_product_tflops": alg * nprod,
                      "frac_of_measured_bf16": (alg * nprod / bf16) if bf16 else None}
    out["gemm_4096"] = gemm
    out["clocks"] = sampler.stop()
    print(json.dumps(out), flush=True)
    return 0


def _rate(ctx, Zc, t1, sig, sig1, stream, dev, steps=5, warmup=3):
    """Residual evaluations per second (CUDA events on the library's stream)."""
    import torch
    for _ in range(warmup):
        ctx.residual(Zc, t1, out=(sig, sig1))
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        ctx.residual(Zc, t1, out=(sig, sig1))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return 1e3 * steps / e0.elapsed_time(e1)


PRODUCT_STEPS = ["dress", "fock", "alg1", "alg2_8", "post", "alg6_gemm", "alg6_post", "alg7",
                 "energy"]


def policy_scan(pkg, s, dev, stream, args):
    """Per-step error of the mixed policy at the float64 converged point:
    for every step with products, that step in bf16 (hi*hi) and the rest in
    bf16x3, against the float64 residual and energy at the same (Zc, t1);
    the residual time of each policy; then solves of the uniform bf16x3
    policy and of the candidate policy (bf16 in every step whose error stays
    below 1e-9 Eh and 1e-7 of max|sigma|) to the float64 energy."""
    import numpy as np
    import torch
    from paper_2111_11473_gb300 import precond
    out = {}
    with _context(pkg, s, precision=pkg.THC_PREC_FP64_TC, stream=stream) as c:
        hist = []
        Zc, t1, rep = c.solve(r_tol=args.fp64_rtol, max_iter=args.max_iter, history=hist,
                              raise_on_failure=False)
        ref = c.residual(Zc, t1)
    f = {"energy": rep.energy, "iters": rep.iters, "wall_s": rep.wall_s, "r_norm": rep.r_norm,
         "time_to_e_tol_s": precond.time_to(hist, rep.energy, 1e-6)[1]}
    out["fp64"] = f
    Zd = torch.from_numpy(Zc).to(dev)
    td = torch.from_numpy(t1).to(dev)
    sig = torch.empty((s.P, s.P), dtype=torch.float64, device=dev)
    sig1 = torch.empty((s.o, s.v), dtype=torch.float64, device=dev)
    scale = float(np.abs(ref[0]).max())

    def measure(policy):
        with _context(pkg, s, precision=pkg.THC_PREC_MIXED, stream=stream, policy=policy) as c:
            r = c.residual(Zc, t1)
            rate = _rate(c, Zd, td, sig, sig1, stream, dev)
        d = r[0] - ref[0]
        return {"max_abs_dsigma": float(np.abs(d).max()), "norm_dsigma": float(np.linalg.norm(d)),
                "norm_dsigma1": float(np.linalg.norm(r[1] - ref[1])), "dE": r[2] - ref[2],
                "ms": 1e3 / rate}

    rows = {"bf16x3": measure(None)}
    for step in PRODUCT_STEPS:
        rows[step + "=bf16"] = measure({step: "bf16"})
    out["residual_at_fp64_solution"] = rows
    base = rows["bf16x3"]
    cheap = [st for st in PRODUCT_STEPS
             if abs(rows[st + "=bf16"]["dE"] - base["dE"]) < 1e-9 and
             rows[st + "=bf16"]["max_abs_dsigma"] < base["max_abs_dsigma"] + 1e-7 * scale]
    cand = {st: "bf16" for st in cheap}
    out["candidate"] = {"steps_bf16": cheap, **measure(cand)}
    for name, pol in (("bf16x3", None), ("candidate", cand)):
        with _context(pkg, s, precision=pkg.THC_PREC_MIXED, stream=stream, policy=pol) as c:
            m = precond.run_solve(c, f["energy"], None, r_tol=args.solve_rtol,
                                  max_iter=args.max_iter, stop_de=1e-8)
        out["solve_" + name] = {"energy": m["energy"], "energy_minus_fp64": m["energy"] - f["energy"],
                                "iters": m["iters"], "wall_s": m["wall_s"],
                                "time_to_e_tol_s": m["time_to_e_tol_s"]}
    return out


def fp64_vs_mixed_iterations(pkg, s, stream, n_iter):
    """Energy of the float64 and of the mixed-precision solve from zero,
    iteration by iteration (each on its own trajectory), and their difference."""
    out = {}
    for name, prec in (("fp64", pkg.THC_PREC_FP64), ("mixed", pkg.THC_PREC_MIXED)):
        with _context(pkg, s, precision=prec, stream=stream) as c:
            hist = []
            c.solve(r_tol=0.0, max_iter=n_iter, history=hist, raise_on_failure=False)
            out[name] = [h[0] for h in hist]
            out[name + "_seconds"] = [h[2] for h in hist]
    out["energy_diff_per_iteration"] = [m - f for f, m in zip(out["fp64"], out["mixed"])]
    return out


def solve_variants(pkg, s, dev, stream, ctx, args, prec, rate=None):
    """Solves from zero: float64, mixed precision, and mixed precision with the
    learned preconditioner; time to 1e-6 Eh of the float64 converged energy
    (of the plain mixed solve's converged energy when the float64 solve is
    skipped, at sizes where it would take too long).  ``rate`` is the mixed
    residual rate when ctx is the mixed context and it was measured already."""
    import numpy as np
    import torch
    from paper_2111_11473_gb300 import precond
    from synth import make_system
    out = {}
    f = None
    if not args.skip_fp64_solve:
        # the float64 solve runs on the float64 policy benchmarked (CUDA-core
        # or tensor-core products), the CUDA-core one when mixed is benchmarked
        fprec = prec if prec != pkg.THC_PREC_MIXED else pkg.THC_PREC_FP64
        fp64_ctx = ctx if prec == fprec else _context(pkg, s, precision=fprec, stream=stream)
        f = precond.run_solve(fp64_ctx, None, None, r_tol=args.fp64_rtol,
                              max_iter=args.max_iter)
        f["evals_per_s"] = None
        out["fp64"] = f
        if fp64_ctx is not ctx:
            fp64_ctx.close()
    # Mixed precision: residual rate on the bench state, then solves.
    mctx = ctx if prec == pkg.THC_PREC_MIXED else _context(
        pkg, s, precision=pkg.THC_PREC_MIXED, stream=stream)
    if rate is not None and mctx is ctx:
        mrate = rate
    else:
        Zc0, t10, _ = mctx.solve(max_iter=3, diis_n=0, raise_on_failure=False)
        Zc = torch.from_numpy(Zc0).to(dev)
        t1 = torch.from_numpy(t10).to(dev)
        sig = torch.empty((s.P, s.P), dtype=torch.float64, device=dev)
        sig1 = torch.empty((s.o, s.v), dtype=torch.float64, device=dev)
        mrate = _rate(mctx, Zc, t1, sig, sig1, stream, dev)
    e_ref = f["energy"] if f is not None else None
    # The mixed-precision residual has a floor near 5e-6 at o=40 (the bf16x3
    # products' rounding): the mixed solves stop at |r| < solve_rtol (1e-5)
    # once the energy changes by less than 1e-8 Eh per iteration.
    m = precond.run_solve(mctx, e_ref, None, r_tol=args.solve_rtol, max_iter=args.max_iter,
                          stop_de=1e-8)
    m["evals_per_s"] = mrate
    if e_ref is None:
        e_ref = m["energy"]
    out["mixed"] = m
    # Learned preconditioner: pairs from small systems of the same family
    # (v = 5o, P = 10o, G = 30o, K = 15o), trained on the GPU.
    t0 = time.perf_counter()
    Xs, js, ts = [], [], []
    for k, o in enumerate((8, 10, 12, 14, 16, 18)):
        ss = make_system(o, 5 * o, 10 * o, 30 * o, 15 * o, 100 + k)
        with _context(pkg, ss, precision=pkg.THC_PREC_MIXED, stream=stream) as c:
            X, j, t, _ = precond.collect_pairs(c, seed=k)
        Xs.append(X)
        js.append(j)
        ts.append(t)
    X, j, t = (np.concatenate(a) for a in (Xs, js, ts))
    net, loss, jacobi = precond.train(X, j, t, epochs=20)
    train_s = time.perf_counter() - t0
    lrn = precond.run_solve(mctx, e_ref, net, r_tol=args.solve_rtol, max_iter=args.max_iter,
                            stop_de=1e-8)
    lrn["evals_per_s"] = mrate
    lrn["training"] = {"systems": "o = 8..18, v = 5o, P = 10o, G = 30o, K = 15o, seeds 100-105",
                       "pairs": int(len(j)), "loss": loss, "loss_plain_jacobi": jacobi,
                       "seconds": train_s, "hidden": 256, "weights": "bf16"}
    out["mixed+learned"] = lrn
    net.close()
    if mctx is not ctx:
        mctx.close()
    t_ref = f["time_to_e_tol_s"] if f is not None else None
    out["e_ref"] = e_ref
    out["e_ref_source"] = "float64 solve" if f is not None else "plain mixed-precision solve"
    out["speedup_time_to_1e-6_Eh_vs_fp64"] = {
        k: (t_ref / out[k]["time_to_e_tol_s"]
            if t_ref and out[k]["time_to_e_tol_s"] else None)
        for k in ("mixed", "mixed+learned")}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64tc", choices=["fp64", "fp64tc", "mixed"],
                    help="fp64tc (default): float64, the products as exact integer slices on "
                         "the tensor cores combined in float64; fp64: float64 on the CUDA "
                         "cores; mixed: float32 + bf16x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    help="system from synth.CONFIGS (named by size)")
    ap.add_argument("--skip-fp64-solve", action="store_true",
                    help="no float64 solve (sizes where it takes too long)")
    ap.add_argument("--fp64-rtol", type=float, default=1e-8,
                    help="residual tolerance of the float64 reference solve")
    ap.add_argument("--solve-rtol", type=float, default=1e-5,
                    help="residual tolerance of the mixed-precision solves")
    ap.add_argument("--max-iter", type=int, default=60, help="iteration cap of every solve")
    ap.add_argument("--t2sq-route", type=int, default=0, choices=[0, 1, 2],
                    help="Eqs. 32-33: 0 automatic, 1 Alg. 6 (O(N^4)), 2 Algs. 4-5 (O(N^5))")
    ap.add_argument("--fp64-iters", type=int, default=0,
                    help="also run this many float64 and mixed iterations from zero "
                         "and report their energy difference per iteration")
    ap.add_argument("--policy-scan", action="store_true",
                    help="per-step error and time of the mixed policy at the float64 "
                         "solution, and solves of the candidate per-step policy")
    ap.add_argument("--sharded", action="store_true",
                    help="under torchrun: one system split over the ranks (thc_config "
                         "shard_index / shard_count), the parts summed by one NCCL "
                         "all-reduce per step (strong scaling)")
    ap.add_argument("--fp64-check-shards", type=int, default=0,
                    help="with --precision mixed: evaluate the float64 residual at the mixed "
                         "solve's converged point as the sum of this many shard contexts made "
                         "one after another (systems whose float64 Cholesky vectors do not fit)")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the CUDA-core FMA rates and time 4096^3 tensor-core "
                         "products (thc_probe_alu, thc_probe_gemm), print one JSON line")
    args = ap.parse_args()
    set_workload(args.workload)
    if args.impl == "reference":
        return run_reference(args)
    if args.peaks:
        return run_peaks()

    import numpy as np
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as g
    if rank == 0:
        g.build()
    if dist is not None:
        dist.barrier()
    g.build()
    import paper_2111_11473_gb300 as pkg

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.sharded and world > 1:
        return run_sharded(args, pkg, dev, stream, dist, world, rank)
    s = _system(seed_offset=rank, device=dev)
    prec = {"fp64": pkg.THC_PREC_FP64, "fp64tc": pkg.THC_PREC_FP64_TC,
            "mixed": pkg.THC_PREC_MIXED}[args.precision]
    t_init = time.perf_counter()
    ctx = _context(pkg, s, dev, precision=prec, stream=stream, t2sq_route=args.t2sq_route)
    init_s = time.perf_counter() - t_init
    # State: two Jacobi steps from zero (projected MP1 and one more step).
    Zc0, t10, _ = ctx.solve(max_iter=3, diis_n=0, raise_on_failure=False)
    Zc = torch.from_numpy(Zc0).to(dev)
    t1 = torch.from_numpy(t10).to(dev)
    sig = torch.empty((s.P, s.P), dtype=torch.float64, device=dev)
    sig1 = torch.empty((s.o, s.v), dtype=torch.float64, device=dev)

    for _ in range(max(3, args.warmup)):
        ctx.residual(Zc, t1, out=(sig, sig1))
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local)
    sampler.start()
    ctx.profile(True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    energy = None
    for _ in range(args.steps):
        _, _, energy = ctx.residual(Zc, t1, out=(sig, sig1))
    e1.record(stream)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = max_over_ranks(ms, dist, dev)
    value = whole_job_rate(world, ms_max)

    # App. II density matrices of the bench state (one call, device buffers).
    Doo = torch.empty((s.o, s.o), dtype=torch.float64, device=dev)
    Dvv = torch.empty((s.v, s.v), dtype=torch.float64, device=dev)
    ctx.mp2_density(Zc, out=(Doo, Dvv))
    torch.cuda.synchronize(dev)
    d0 = torch.cuda.Event(enable_timing=True)
    d1 = torch.cuda.Event(enable_timing=True)
    d0.record(stream)
    ctx.mp2_density(Zc, out=(Doo, Dvv))
    d1.record(stream)
    torch.cuda.synchronize(dev)
    density_ms = d0.elapsed_time(d1)

    # End to end through the public API with pinned host buffers.
    Zh = torch.from_numpy(Zc0).pin_memory()
    t1h = torch.from_numpy(t10).pin_memory()
    sh = torch.empty((s.P, s.P), dtype=torch.float64).pin_memory()
    s1h = torch.empty((s.o, s.v), dtype=torch.float64).pin_memory()
    ctx.residual(Zh, t1h, out=(sh, s1h))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.residual(Zh, t1h, out=(sh, s1h))
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, dist, dev)
    h2d = (s.P * s.P + s.o * s.v) * 8
    d2h = (s.P * s.P + s.o * s.v + 1) * 8

    # Dominant kernel and its roofline.
    steps = {k: {"ms_per_residual": v[0] / max(1, prof["residuals"]),
                 "gflop_per_residual": v[1] / 1e9 / max(1, prof["residuals"]),
                 "launches": v[2]}
             for k, v in prof.items() if k not in ("residuals", "kernel_launches")}
    dom = max((k for k in steps), key=lambda k: steps[k]["ms_per_residual"])
    tri_ms, tri_fl, tri_n = prof["triangle"]
    fp64 = args.precision != "mixed"
    total_ms = max(1e-9, sum(v["ms_per_residual"] for v in steps.values()) *
                   max(1, prof["residuals"]))
    if tri_n > 0:
        roofline = triangle_roofline(args.precision, tri_fl, tri_ms, tri_n, tri_ms / total_ms)
    else:
        # Algs. 4-5 route: the dominant step is a group of batched products.
        ms_d, fl_d, n_d = prof[dom]
        achieved = fl_d / (ms_d * 1e-3) / 1e12
        if args.precision == "fp64tc":
            # 36 bf16 products per float64 multiply-add (8 slices a side)
            peak = _peaks().get("bf16_tflops", 1931.0) / 36.0
            bound, src = "tensor", "measured bf16 burst peak / 36 (slice products)"
        elif fp64:
            peak, bound, src = FP64_ALU_TFLOPS, "alu", "derived: 152 SMs x 2 fp64 FMA lanes x 2 x 2.07 GHz"
        else:
            # bf16x3: three bf16 products per algorithmic multiply-add
            peak = _peaks().get("bf16_tflops", 1931.0) / 3.0
            bound, src = "tensor", "measured bf16 burst peak / 3 (bf16x3 products)"
        roofline = {"kernel": f"{dom} step (batched products)", "bound": bound,
                    "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": None, "peak_source": src,
                    "share_of_step": ms_d / total_ms}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if fp64 else "f32+bf16x3",
        "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME, "precision": args.precision,
                   "products": {"fp64tc": "float64 by 8 exact 7-bit integer slices per operand "
                                          "row on the tensor cores, combined in float64",
                                "fp64": "float64 on the CUDA cores",
                                "mixed": "float32 operands, bf16 hi/lo on the tensor cores"}[
                                    args.precision],
                   "t2sq_route": args.t2sq_route,
                   "state": "solver iterate after two Jacobi steps from zero",
                   "l2": "inputs larger than L2 (Cholesky blocks %.3g GB)" % (
                       s.K * (s.o * s.o + s.o * s.v + s.v * (s.v + 1) / 2) *
                       (8 if fp64 else 4) / 1e9),
                   "parallelism": f"{world} independent system(s), one per GPU"},
        "energy": energy,
        "e2e": {"value": whole_job_rate(world, 1e3 * e2e_s), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": prof["kernel_launches"],
        "mp2_density_ms": density_ms,
        "clocks": clocks,
        "roofline": roofline,
        "dominant_step": dom,
        "steps_breakdown": steps,
    }

    line["init_s"] = init_s
    if not args.no_solve:
        line["solve"] = solve_variants(pkg, s, dev, stream, ctx, args, prec, rate=1e3 / ms)
    if args.fp64_iters > 0:
        line["fp64_vs_mixed"] = fp64_vs_mixed_iterations(pkg, s, stream, args.fp64_iters)
    if args.policy_scan:
        line["policy_scan"] = policy_scan(pkg, s, dev, stream, args)
    if args.fp64_check_shards > 0:
        line["fp64_check"] = serial_shard_check(pkg, s, dev, stream, ctx, args)
    ctx.close()

    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == DEFAULT_WORKLOAD:
        sec = oracle_residual_seconds(s, Zc0, t10)
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": UNIT, "cores": _threads(),
                                "kind": "oracle",
                                "sample": "one full FP64 oracle residual + energy of the "
                                          "bench system (about a minute of host time)"}
    if dist is not None:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
