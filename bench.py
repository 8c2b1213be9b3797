"""Benchmark: boundary-MPS contraction of a synthetic PEPS (implicit randomized
SVD einsumsvd, two-layer zip-up) on one or more GB300s.

One step = one full contraction <psi|psi> of the workload's PEPS (every row,
every einsumsvd of Algorithms 2-4), inputs resident in HBM.  The default
workload is the 16 x 16, D = 8 (double-layer bond 64), m = 256, p = 16, q = 2
complex64 norm on the mixed-precision tensor-core path.  Prints one JSON line
(rank 0).  ``--impl reference`` times the CPU oracle instead (the reference
arm of this repository: a plain FP64 NumPy replay of the paper's algorithms)
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

import synth  # noqa: E402

METRIC = "PEPS contraction s & einsumsvd TFLOP/s, mixed vs plain FP32 at 1e-5 rel err"
L2_BYTES = 129 * 2 ** 20


def algorithmic_flops(shapes, q, cplx):
    """Algorithmic flops of one contraction from its einsumsvd step shapes,
    counting the work the schedule executes.

    Per step (complex MAC = 8 flops, real MAC = 2):
      (2q+2) implicit products, each l*(b d D^6-type site stages + the two
      m^2 stages) as counted by the plan (Table 2's two-layer terms);
      q+1 orthogonalisations of the M x l block at 2 M l^2
      (Householder-equivalent), and q of the N x l block at 2 N l^2 when the
      step runs them (s["orth_n"]; the tensor-core schedule feeds A^H P to the
      next product directly and skips them); the R factor of the N x l block
      of P^H A (N l^2); U = P U~ (M l k) and W = U~^H B (k l N).
    """
    mult = 8.0 if cplx else 2.0
    tot = 0.0
    for s in shapes:
        M, N, ell, k, prod = s["M"], s["N"], s["ell"], s["k"], s["prod_macs"]
        macs = (2 * q + 2) * prod + (q + 1) * 2 * M * ell ** 2
        if s.get("orth_n", True):
            macs += q * 2 * N * ell ** 2
        macs += N * ell ** 2 + M * ell * k + k * ell * N
        tot += mult * macs
    return tot


def tc_eligible(d, Dl, Du, Dx, De, DL, DU, DX, DE, a, b, M, cplx, double=False):
    """Whether the library runs a step on the tensor cores: every contracted
    extent of its stage GEMMs keeps TMA rows 16-byte aligned (a multiple of 2
    complex or 4 real single-precision values); FP64 data never do."""
    if double:
        return False
    align = 2 if cplx else 4
    P1, Q1, P2, Q2 = Dl * Du, Dx * De, DL * DU, DX * DE
    ks = (Q1, d * Q2, Du * DU * b, a * Dl * DL, M, a, P2, d * P1)
    return all(k % align == 0 for k in ks)


def mark_schedule(shapes, prec_plain, orth_q=False):
    """Record per step whether the N-side orthogonalisations run (plain
    schedule, or a step that falls back to it, or an explicit request)."""
    for s in shapes:
        s["orth_n"] = bool(prec_plain or orth_q or not s.get("tc", False))
    return shapes


def step_shapes(cfg):
    """Shapes of every einsumsvd step of the sweep (same rule as the library)."""
    nrow, ncol, d, D, m, p = cfg.nrow, cfg.ncol, cfg.d, cfg.D, cfg.m, cfg.p
    two = cfg.two_layer
    dims = [[synth.site_shape(nrow, ncol, r, c, d, D) for c in range(ncol)] for r in range(nrow)]
    bra = (lambda r, c: dims[r][c]) if two else (lambda r, c: (1, 1, 1, 1, 1))
    bound = [(dims[0][c][1] * bra(0, c)[1], dims[0][c][3] * bra(0, c)[3], dims[0][c][4] * bra(0, c)[4])
             for c in range(ncol)]
    out = []
    for r in range(1, nrow):
        new = [None] * ncol
        kprev = 1
        for i in range(1, ncol):
            kp, bp = dims[r][i - 1], bra(r, i - 1)
            kc, bc = dims[r][i], bra(r, i)
            a, v, b = bound[i]
            t = kp[3] * bp[3]
            M = kprev * t
            N = kc[3] * bc[3] * b * kc[4] * bc[4]
            k = min(m, M, N)
            ell = min(k + p, M, N)
            h = kc[1] * bc[1]
            dd = kc[0]
            P1, Q1, P2, Q2 = kc[1] * kc[2], kc[3] * kc[4], bc[1] * bc[2], bc[3] * bc[4]
            prod = ell * (b * dd * (P1 * Q1 * Q2 + P1 * Q2 * P2) + a * h * v * b + M * a * h)
            tc = tc_eligible(dd, kc[1], kc[2], kc[3], kc[4], bc[1], bc[2], bc[3], bc[4], a, b, M,
                             cfg.dtype.startswith("c"), cfg.dtype in ("f64", "c128"))
            out.append(dict(M=M, N=N, ell=ell, k=k, prod_macs=prod, row=r, col=i, tc=tc))
            new[i - 1] = (kprev, t, k)
            kprev = k
        kl, bl = dims[r][ncol - 1], bra(r, ncol - 1)
        new[ncol - 1] = (kprev, kl[3] * bl[3], 1)
        bound = new
    return out


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- multi-rank host logic (weak scaling: every rank its own work, no data-path collective) ----

def replica_seed(cfg, rank):
    """Seed of rank `rank`'s replica of the workload's PEPS."""
    return cfg.seed + 1000 * rank


def rank_instance_ids(rank, n):
    """Instance ids of rank `rank`'s batch of n instances (disjoint across ranks)."""
    return [rank * n + i for i in range(n)]


def max_over_ranks(value, world, device="cpu"):
    """The largest per-rank value over all ranks (the slowest rank's step time)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def lpt_shard(costs, world):
    """Longest-processing-time-first partition of one batch over `world` ranks
    (the natural sharding of independent einsumsvd instances): instances in
    order of decreasing cost, each to the rank with the least load so far
    (ties to the lower rank).  Returns every rank's instance indices, sorted."""
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda r: (load[r], r))
        load[r] += costs[i]
        parts[r].append(i)
    return [sorted(p) for p in parts]


def whole_job_value(world, flops_per_rank, ms_step):
    """Whole-job throughput in TFLOP/s: the work of every rank over the slowest rank's time."""
    return world * flops_per_rank / (ms_step * 1e-3) / 1e12


TUNE_DIR = os.path.join(ROOT, "paper_2006_15234_gb300", "tuning")


def load_tune(workload):
    """The stored tensor-core tile table of a workload (tuning/<workload>.txt)."""
    path = os.path.join(TUNE_DIR, workload + ".txt")
    if not os.path.exists(path):
        return None
    return {"source": os.path.relpath(path, ROOT), "table": open(path).read()}


# DRAM traffic of the tensor-core GEMM family on the 16 x 16 mixed contraction:
# ncu dram__bytes_read.sum + dram__bytes_write.sum summed over every tc_gemm
# launch of one contraction (a one-pass capture of the full workload, tile
# table applied), divided by the launch count.  It stands only while the
# kernel's sources hash to the value it was taken with.
TC_GEMM_TRAFFIC = {"workload": "c5_16x16_norm_c64_D8_m256", "launches": 8526, "read_gb": 21795.914,
                   "write_gb": 9270.977, "bytes_per_launch": 3.6438e9, "sources_sha": "258729a8e9e5e73f"}


def tc_gemm_sources_sha():
    import hashlib
    parts = []
    for f in ("tcgemm.cu", "tcgemm.h", "tc_host.cu"):
        with open(os.path.join(ROOT, "paper_2006_15234_gb300", "csrc", f), "rb") as fh:
            parts.append(hashlib.sha256(fh.read()).hexdigest())
    return hashlib.sha256("".join(parts).encode()).hexdigest()[:16]


def tc_gemm_traffic(workload, kname):
    """Per-launch DRAM bytes of tc_gemm for this workload, or None when it was
    not captured for it or the kernel changed since."""
    t = TC_GEMM_TRAFFIC
    if kname != "tc_gemm" or workload != t["workload"] or tc_gemm_sources_sha() != t["sources_sha"]:
        return None
    return t["bytes_per_launch"]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def run_ours(args, cfg):
    import torch
    import torch.distributed as dist
    from paper_2006_15234_gb300 import libpeps

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tdt = {"c64": torch.complex64, "f32": torch.float32, "f64": torch.float64}[cfg.dtype]
    # weak scaling: every rank contracts its own PEPS (replicas of the workload)
    ket = synth.random_peps(cfg.nrow, cfg.ncol, cfg.d, cfg.D, cfg.dtype, cfg.dist, replica_seed(cfg, rank))
    kt = [[torch.tensor(T, dtype=tdt, device=dev) for T in row] for row in ket]
    prec = {"plain": libpeps.PREC_PLAIN, "mixed": libpeps.PREC_MIXED, "fast": libpeps.PREC_FAST}[args.prec]
    flags = libpeps.FLAG_FP64_SMALL if args.fp64_small else 0
    opts = libpeps.make_opts(cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=prec, flags=flags)
    plan = libpeps.ContractPlan(kt, kt if cfg.two_layer else None, opts)
    launches = plan.launches()
    nlaunch = len(launches)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up: the first execute uploads the descriptors; with a CUDA graph the
    # remaining warm-up steps replay the captured sweep
    plan.execute()
    la, ph = plan.result()
    tune = None
    if not args.no_autotune and prec != libpeps.PREC_PLAIN:
        # MMA widths per tensor-core GEMM shape: the stored table of this
        # workload if there is one, else timed here (before the graph capture)
        tune = load_tune(cfg.name)
        if tune is None:
            t0 = time.perf_counter()
            plan.autotune(reps=3)
            tune = {"source": "tuned in this run", "seconds": round(time.perf_counter() - t0, 3),
                    "table": plan.tune_table()}
        else:
            plan.set_tune_table(tune["table"])
        plan.execute()
        la_t, _ = plan.result()
        assert la_t == la, (la_t, la)
    if args.launch_list:
        # one more contraction, bracketed for an external launch-list capture
        # (ncu --profile-from-start off), then stop
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        plan.execute()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"launch_list": cfg.name, "kernel_launches": plan.kernel_launches()}), flush=True)
        return
    run = plan.execute
    graph = None
    if not args.no_graph:
        # the whole sweep as one CUDA graph (descriptors are already resident)
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                plan.execute()
        stream.wait_stream(side)
        run = graph.replay
    for _ in range(max(0, args.warmup - 1)):
        run()
    if args.warmup > 1:
        la_g, _ = plan.result()
        assert abs(la_g - la) <= 1e-6 * abs(la), (la_g, la)
    barrier()
    times = []
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.add_(1.0)                       # evict L2 between steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            times.append((e0, e1))
        barrier()
        t_wall = time.perf_counter() - t_wall
    ms = [a.elapsed_time(b) for a, b in times]
    ms_step = max_over_ranks(float(np.mean(ms)), world, dev)

    # end-to-end through the public API with host buffers: H2D of every site,
    # the contraction, D2H of the result, every step inside the timed region
    host = [[torch.tensor(T, dtype=tdt).pin_memory() for T in row] for row in ket]
    h2d = sum(T.numel() * T.element_size() for row in host for T in row)
    e2e = []
    for _ in range(min(args.steps, 5)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for r, row in enumerate(host):
            for c, T in enumerate(row):
                kt[r][c].copy_(T, non_blocking=True)
        run()
        la2, _ = plan.result()
        e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(float(np.median(e2e)), world, dev)

    # per-launch device times of one more execute (CUDA events on the stream)
    prof = plan.profile()
    kern = plan.kernels()
    by_tag, by_kern = {}, {}
    for (tag, fl, by), kname, t in zip(launches, kern, prof):
        d = by_tag.setdefault(tag, [0.0, 0.0, 0.0, 0])
        d[0] += t; d[1] += fl; d[2] += by; d[3] += 1
        d = by_kern.setdefault(kname, [0.0, 0.0, 0.0, 0])
        d[0] += t; d[1] += fl; d[2] += by; d[3] += 1
    shapes = mark_schedule(step_shapes(cfg), prec == libpeps.PREC_PLAIN)
    flops = algorithmic_flops(shapes, cfg.q, cfg.dtype == "c64")
    value = whole_job_value(world, flops, ms_step)
    peaks, peak_src = measured_peaks()
    # the dominant kernel: the family with the largest device time
    kname, (dt_ms, dfl, dby, dn) = max(by_kern.items(), key=lambda kv: kv[1][0])
    if kname == "tc_gemm":
        bound, unit = "tensor", "TFLOP/s"
        achieved = dfl / (dt_ms * 1e-3) / 1e12
        tf32 = peaks.get("bf16_tflops_sustained", 1700.0) / 2.0      # TF32 = half the bf16 rate
        if prec == libpeps.PREC_FAST:
            peak, peak_note = tf32, f"TF32 dense = bf16 sustained x 1/2 ({peak_src})"
        else:
            peak = tf32 / 3.0
            peak_note = (f"FP32-level products as 3 TF32 MMAs: bf16 sustained x 1/2 x 1/3 ({peak_src}); "
                         f"algorithmic FP32 flops counted once")
    elif dfl / max(dby, 1) > 12:
        bound, unit = "alu", "TFLOP/s"
        achieved = dfl / (dt_ms * 1e-3) / 1e12
        clk_max = peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * clk_max * 1e6 / 1e12                  # FP32 FMA lanes x 2 x clock
        peak_note = "FP32 SIMT: 152 SMs x 128 lanes x 2 flop x max SM clock"
    else:
        bound, unit = "hbm", "GB/s"
        achieved = dby / (dt_ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        peak_note = f"HBM copy bandwidth ({peak_src})"
    plain = None
    if not args.no_compare_plain and prec != libpeps.PREC_PLAIN:
        # the plain FP32 CUDA-core path on the same PEPS: one contraction after
        # one untimed execute (descriptor upload), CUDA events on the stream
        pplan = libpeps.ContractPlan(kt, kt if cfg.two_layer else None,
                                     libpeps.make_opts(cfg.m, cfg.p, cfg.q, cfg.omega_seed,
                                                       prec=libpeps.PREC_PLAIN, flags=flags))
        pplan.execute()
        torch.cuda.synchronize()
        flush.add_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pplan.execute()
        e1.record(stream)
        torch.cuda.synchronize()
        plain_s = e0.elapsed_time(e1) / 1e3
        plain_la, _ = pplan.result()
        pflops = algorithmic_flops(mark_schedule(step_shapes(cfg), True), cfg.q, cfg.dtype == "c64")
        plain = {"contraction_s": round(plain_s, 4), "tflops": round(pflops / plain_s / 1e12, 4),
                 "log_norm": plain_la, "mixed_speedup": round(plain_s / (ms_step / 1e3), 3)}
        del pplan
    # the contracted log-norm against the FP64 oracle's stored value (rank 0's
    # PEPS is the stored workload's): |d log|v|| and the relative error on v
    parity = None
    gold = load_golden(f"{cfg.name.split('_')[0]}_sweep.json") if rank == 0 else None
    if gold is not None and "log_norm" in gold:
        def err(x):
            d = abs(x - gold["log_norm"])
            return {"dlog": d, "rel_v": float(np.expm1(d)), "rel_log": d / abs(gold["log_norm"])}
        parity = {"oracle_log_norm": gold["log_norm"], args.prec: err(la)}
        if plain is not None:
            parity["plain"] = err(plain["log_norm"])
    c3 = None
    if args.config == "c5" and not args.no_c3 and world == 1:
        c3 = batched_subrecord(dev)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": cfg.dtype,
        "data": "synthetic (seeded Gaussian PEPS, shapes of the workload)",
        "config": {"workload": cfg.name, "nrow": cfg.nrow, "ncol": cfg.ncol, "d": cfg.d,
                   "bond": cfg.D, "m": cfg.m, "p": cfg.p, "q": cfg.q, "precision": args.prec,
                   "small_factorisations": "fp64" if args.fp64_small else "single (R_B factor fp64)",
                   "contraction_s": round(ms_step / 1e3, 6), "einsumsvd_steps": len(shapes),
                   "algorithmic_tflop_per_step": round(flops / 1e12, 6),
                   "l2": "flushed between steps (2x L2 write outside the timed events)",
                   "parallelism": f"replicas x{world}", "log_norm": la,
                   "cuda_graph": graph is not None},
        "gpu_launches": plan.kernel_launches() * args.steps,
        "e2e": {"value": round(world * flops / e2e_s / 1e12, 4), "unit": "TFLOP/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 16},
        "roofline": {"bound": bound, "kernel": kname, "achieved": round(achieved, 3),
                     "peak": round(peak, 1), "unit": unit, "frac": round(achieved / peak, 4),
                     "traffic": tc_gemm_traffic(cfg.name, kname) if prec == libpeps.PREC_MIXED else None,
                     "algorithmic_bytes_per_launch": round(dby / dn, 1), "launches_per_step": dn,
                     "avg_launch_ms": round(dt_ms / dn, 5), "peak_source": peak_note,
                     "algorithmic_per_launch": round((dfl if unit == "TFLOP/s" else dby) / dn, 1),
                     "share_of_step": round(dt_ms / max(sum(v[0] for v in by_kern.values()), 1e-9), 4)},
        "kernel_ms": {k: round(v[0], 4) for k, v in sorted(by_kern.items(), key=lambda kv: -kv[1][0])},
        "stage_ms": {k: round(v[0], 4) for k, v in sorted(by_tag.items(), key=lambda kv: -kv[1][0])},
    }
    if tune is not None:
        line["config"]["tile_table"] = {"source": tune["source"],
                                        "shapes": len([x for x in tune["table"].splitlines() if x]),
                                        **({"tune_s": tune["seconds"]} if "seconds" in tune else {})}
        if rank == 0 and "seconds" in tune and args.tune_out:
            with open(args.tune_out, "w") as f:
                f.write(tune["table"])
    if plain is not None:
        line["plain_fp32"] = plain
    if parity is not None:
        line["parity_vs_oracle"] = parity
    if c3 is not None:
        line["batched_c3"] = c3
    clk = clk.summary()
    if clk:
        line["clocks"] = clk
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batched_shapes(cfg, rank=0):
    """(shape tuple, algorithmic flops, tensor-core eligible) of every
    instance of the batched workload: one zip-up step per instance,
    kL = a = b = m, t = h = D^2, rank k = m (the paper's per-step einsumsvd
    with its own m)."""
    out = []
    for m, D in synth.batched_dims(cfg):
        R = D * D
        M, N = m * R, m * R * R
        k = min(m, M, N)
        ell = min(k + cfg.p, M, N)
        prod = ell * (m * cfg.d * (R * R * R + R * R * R) + m * R * R * m + M * m * R)
        # single-precision instances all run on the tensor cores in the mixed
        # schedule: aligned ones as they are, the rest through a zero-padded copy
        aligned = tc_eligible(cfg.d, D, D, D, D, D, D, D, D, m, m, M, False)
        shp = dict(M=M, N=N, ell=ell, k=k, prod_macs=prod, tc=True, aligned=aligned)
        out.append(((m, R, m, m, cfg.d, D, D, D, D, D, D, D, D, m), shp))
    return out


GOLDEN = os.path.join(ROOT, "tests", "golden")


def load_golden(name):
    try:
        with open(os.path.join(GOLDEN, name)) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def batched_costs(cfg, plain):
    """Executed algorithmic flops of every instance of the batch."""
    return [algorithmic_flops(mark_schedule([dict(x)], plain), cfg.q, False) for _, x in batched_shapes(cfg)]


def measure_batched(cfg, prec, steps, warmup, dev, rank=0, world=1, use_graph=True, e2e=False, clock=None,
                    tune_branches=True):
    """One plan over this rank's LPT share of the 512 instances, replayed as
    one CUDA graph; returns the device time per batch, the executed
    algorithmic flops, every instance's singular values and the plan's
    kernel ledger."""
    import torch
    from paper_2006_15234_gb300 import libpeps
    plain = prec == libpeps.PREC_PLAIN
    costs = batched_costs(cfg, plain)
    ids = lpt_shard(costs, world)[rank]
    shp = [batched_shapes(cfg)[i] for i in ids]
    n = len(shp)
    flops = sum(costs[i] for i in ids)
    host, io = [], []
    plan = libpeps.EinsumsvdPlan(torch.float32, [s for s, _ in shp],
                                 libpeps.make_opts(128, cfg.p, cfg.q, cfg.omega_seed, prec=prec),
                                 instance_ids=ids, device=dev)
    for i, (s, _) in enumerate(shp):
        m, D = s[0], s[5]
        inst = synth.batched_instance(cfg, ids[i], m, D)
        h = [torch.from_numpy(np.ascontiguousarray(inst[k], dtype=np.float32)).pin_memory()
             for k in ("V", "S", "ket", "bra")]
        host.append(h)
        k = plan.ranks[i]
        U = torch.empty((s[0] * s[1], k), dtype=torch.float32, device=dev)
        W = torch.empty((k, s[7] * s[11] * s[3] * s[8] * s[12]), dtype=torch.float32, device=dev)
        sg = torch.empty(k, dtype=torch.float64, device=dev)
        lg = torch.empty(1, dtype=torch.float64, device=dev)
        io.append(tuple(x.to(dev) for x in h) + (U, W, sg, lg))
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    branches = None
    if not plain and tune_branches:
        # side streams of the tensor-core chains: the fastest of a few counts
        best = None
        for nb in (8, 16, 32, 64):
            plan.set_branches(nb, dev)
            plan.execute(io)              # descriptor upload
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                plan.execute(io)
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 2
            if best is None or t < best[1]:
                best = (nb, t)
        branches = best[0]
        plan.set_branches(branches, dev)
    plan.execute(io)                      # descriptor upload
    torch.cuda.synchronize()
    run = lambda: plan.execute(io)        # noqa: E731
    graph = None
    if use_graph:
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(graph, stream=side):
                plan.execute(io)
        stream.wait_stream(side)
        run = graph.replay
    for _ in range(max(0, warmup - 1)):
        run()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    times = []
    import contextlib
    with (clock if clock is not None else contextlib.nullcontext()):
        for _ in range(steps):
            flush.add_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            times.append((e0, e1))
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in times]))
    sig = [x[6].cpu().numpy() for x in io]
    out = {"ms": ms, "flops": flops, "sig": sig, "ids": ids, "plan": plan, "io": io, "host": host, "run": run,
           "graph": graph is not None, "n": n, "tc_instances": 0 if plain else n, "branches": branches,
           "padded_instances": 0 if plain else sum(1 for _, x in shp if not x["aligned"])}
    if e2e:
        # end to end: H2D of every instance's operands, the batch, D2H of all singular values
        out["h2d"] = sum(x.numel() * x.element_size() for h in host for x in h)
        out["d2h"] = sum(x[6].numel() * 8 for x in io)
        sig_host = [torch.empty(x[6].numel(), dtype=torch.float64).pin_memory() for x in io]
        t = []
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for h, x in zip(host, io):
                for a, b in zip(h, x[:4]):
                    b.copy_(a, non_blocking=True)
            run()
            for hs, x in zip(sig_host, io):
                hs.copy_(x[6], non_blocking=True)
            torch.cuda.synchronize()
            t.append(time.perf_counter() - t0)
        out["e2e_s"] = float(np.median(t))
    return out


def batched_sigma_error(sig, gold, ids=None):
    """Largest normwise singular-value error max_i |s_i - s_i^ref| / s_1^ref
    over the instances against the oracle's stored values (None without them)."""
    if gold is None:
        return None
    worst = 0.0
    refs = gold["instances"] if ids is None else [gold["instances"][i] for i in ids]
    for g, ref in zip(sig, refs):
        r = np.asarray(ref["sigma"])
        worst = max(worst, float(np.max(np.abs(g[: len(r)] - r)) / max(r[0], 1e-300)))
    return worst


def batched_subrecord(dev, steps=3, warmup=3):
    """The 512-instance batched einsumsvd in both precisions (one CUDA graph
    per batch): device seconds per batch, executed algorithmic TFLOP/s and
    the largest singular-value error against the oracle's stored values."""
    import torch
    from paper_2006_15234_gb300 import libpeps
    cfg = synth.config("c3")
    gold = load_golden("c3_sigma.json")
    out = {"workload": cfg.name}
    for name, prec in (("mixed", libpeps.PREC_MIXED), ("plain", libpeps.PREC_PLAIN)):
        r = measure_batched(cfg, prec, steps, warmup, dev)
        out[name] = {"batch_s": round(r["ms"] / 1e3, 5), "tflops": round(r["flops"] / (r["ms"] * 1e-3) / 1e12, 4),
                     "sigma_err_vs_oracle": batched_sigma_error(r["sig"], gold),
                     "kernel_launches": r["plan"].kernel_launches()}
        if name == "mixed":
            out["tensor_core_instances"] = r["tc_instances"]
            out["padded_instances"] = r["padded_instances"]
            out["branches"] = r["branches"]
        del r
        torch.cuda.empty_cache()
    out["mixed_speedup"] = round(out["plain"]["batch_s"] / out["mixed"]["batch_s"], 3)
    return out


def run_batched(args, cfg):
    """Batched einsumsvd: 512 independent instances in one plan, replayed as
    one CUDA graph (a step = all instances once)."""
    import torch
    import torch.distributed as dist
    from paper_2006_15234_gb300 import libpeps
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    prec = {"plain": libpeps.PREC_PLAIN, "mixed": libpeps.PREC_MIXED, "fast": libpeps.PREC_FAST}[args.prec]
    # weak scaling: every rank its own 512 instances (instance seeds offset by rank)
    clk = ClockSampler(local)
    r = measure_batched(cfg, prec, args.steps, args.warmup, dev, rank, world, not args.no_graph, e2e=True,
                        clock=clk)
    ms_step = max_over_ranks(r["ms"], world, dev)
    e2e_s = max_over_ranks(r["e2e_s"], world, dev)
    flops, plan, n = r["flops"], r["plan"], r["n"]
    launches = plan.launches()
    prof = plan.profile()
    kern = plan.kernels()
    by_kern = {}
    for (tag, fl, by), kname, t in zip(launches, kern, prof):
        d = by_kern.setdefault(kname, [0.0, 0.0, 0.0, 0])
        d[0] += t; d[1] += fl; d[2] += by; d[3] += 1
    # the roofline is taken on the family with the most time among those with
    # an algorithmic count (the small Cholesky / Jacobi factorisations have
    # none: they are latency-bound); the family with the most time overall is
    # named beside it
    top_time = max(by_kern.items(), key=lambda kv: kv[1][0])[0]
    small = ("chol", "jacobi", "finalize", "zero")
    counted = {k: v for k, v in by_kern.items() if k not in small and (v[1] > 0 or v[2] > 0)} or by_kern
    kname, (dt_ms, dfl, dby, dn) = max(counted.items(), key=lambda kv: kv[1][0])
    peaks, peak_src = measured_peaks()
    if kname == "tc_gemm" or dfl / max(dby, 1) > 12:
        bound, unit = ("tensor", "TFLOP/s") if kname == "tc_gemm" else ("alu", "TFLOP/s")
        achieved = dfl / (dt_ms * 1e-3) / 1e12
        if kname == "tc_gemm":
            peak = peaks.get("bf16_tflops_sustained", 1700.0) / 2.0 / 3.0
            peak_note = f"FP32-level products as 3 TF32 MMAs: bf16 sustained x 1/2 x 1/3 ({peak_src})"
        else:
            peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            peak_note = "FP32 SIMT: 152 SMs x 128 lanes x 2 flop x max SM clock"
    else:
        bound, unit = "hbm", "GB/s"
        achieved = dby / (dt_ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        peak_note = f"HBM copy bandwidth ({peak_src})"
    err = batched_sigma_error(r["sig"], load_golden("c3_sigma.json"), r["ids"])
    if world > 1:
        errs = [None] * world
        dist.all_gather_object(errs, err)
        err = None if any(e is None for e in errs) else max(errs)
    flops_all = sum(batched_costs(cfg, prec == libpeps.PREC_PLAIN))
    line = {
        "metric": METRIC, "value": round(flops_all / (ms_step * 1e-3) / 1e12, 4), "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded N(0,1) operands, instance sizes of the workload)",
        "config": {"workload": cfg.name, "instances": n, "m_range": cfg.extra["m_range"],
                   "D_range": cfg.extra["D_range"], "p": cfg.p, "q": cfg.q, "rank": "k = m per instance",
                   "precision": args.prec, "algorithmic_tflop_per_step": round(flops_all / 1e12, 6),
                   "tensor_core_instances": r["tc_instances"], "padded_instances": r["padded_instances"],
                   "branches": r["branches"], "sigma_err_vs_oracle": err,
                   "l2": "flushed between steps (2x L2 write outside the timed events)",
                   "parallelism": f"one batch split by LPT over {world} rank(s)", "cuda_graph": r["graph"]},
        "gpu_launches": plan.kernel_launches() * args.steps,
        "e2e": {"value": round(flops_all / e2e_s / 1e12, 4), "unit": "TFLOP/s",
                "h2d_bytes_per_step": r["h2d"], "d2h_bytes_per_step": r["d2h"]},
        "roofline": {"bound": bound, "kernel": kname, "achieved": round(achieved, 3), "peak": round(peak, 1),
                     "unit": unit, "frac": round(achieved / peak, 4), "traffic": None,
                     "launches_per_step": dn, "avg_launch_ms": round(dt_ms / dn, 5), "peak_source": peak_note,
                     "share_of_step": round(dt_ms / max(sum(v[0] for v in by_kern.values()), 1e-9), 4),
                     "dominant_by_time": top_time,
                     "dominant_share": round(by_kern[top_time][0] / max(sum(v[0] for v in by_kern.values()),
                                                                         1e-9), 4)},
        "kernel_ms": {k: round(v[0], 4) for k, v in sorted(by_kern.items(), key=lambda kv: -kv[1][0])},
    }
    clk = clk.summary()
    if clk:
        line["clocks"] = clk
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_expect_cache(args, cfg):
    """Expectation value <psi|H|psi>/<psi|psi> of the transverse-field Ising
    Hamiltonian (one-site X on every site, ZZ on every bond) on the 12 x 12,
    D = 4 PEPS with the cached environments of Sec. IV-B (two sweeps per
    lattice, then one strip per term) and without them (fresh sweeps for the
    environments of every row that holds a term): device seconds of each, the
    speed-up, and the energies of both schedules."""
    import torch
    from paper_2006_15234_gb300 import libpeps
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    prec = {"plain": libpeps.PREC_PLAIN, "mixed": libpeps.PREC_MIXED, "fast": libpeps.PREC_FAST}[args.prec]
    ket = synth.peps_for(cfg)
    kt = [[torch.tensor(T, dtype=torch.complex64, device=dev) for T in row] for row in ket]
    terms = synth.tfi_terms(cfg.nrow, cfg.ncol, cfg.extra["J"], cfg.extra["h"])
    opts = libpeps.make_opts(cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=prec)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    with ClockSampler(0) as clk:
        for name, cache in (("cached", True), ("uncached", False)):
            plan = libpeps.ExpectationPlan(kt, terms, opts, use_cache=cache)
            for _ in range(max(1, args.warmup)):
                plan.execute()
            torch.cuda.synchronize()
            run = plan.execute
            graph = None
            if not args.no_graph:
                graph = libpeps.cuda_graph(plan.execute)
                run = graph.replay
                run()
                torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                flush.add_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            e, lnorm, _ = plan.result()
            fl = sum(f for _, f, _ in plan.launches())
            # per-launch device times of one more execute, by kernel family
            kms = {}
            for kname, dt in zip(plan.kernels(), plan.profile()):
                kms[kname] = kms.get(kname, 0.0) + dt
            out[name] = {"seconds": round(float(np.mean(ms)) / 1e3, 5), "energy": e, "log_norm": lnorm,
                         "launch_flops_tflop": round(fl / 1e12, 4), "kernel_launches": plan.kernel_launches(),
                         "workspace_gb": round(plan.workspace_bytes / 1e9, 3), "cuda_graph": graph is not None,
                         "kernel_ms": {k: round(v, 3) for k, v in sorted(kms.items(), key=lambda kv: -kv[1])}}
            del graph, plan
    t_c = out["cached"]["seconds"]
    line = {
        "metric": METRIC, "value": round(out["cached"]["launch_flops_tflop"] / t_c, 4), "unit": "TFLOP/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t_c, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": cfg.dtype,
        "data": "synthetic (seeded Gaussian PEPS, shapes of the workload)",
        "config": {"workload": cfg.name, "nrow": cfg.nrow, "ncol": cfg.ncol, "bond": cfg.D, "m": cfg.m,
                   "p": cfg.p, "q": cfg.q, "precision": args.prec, "terms": len(terms),
                   "cache_speedup": round(out["uncached"]["seconds"] / t_c, 3),
                   "l2": "flushed between steps (2x L2 write outside the timed events)"},
        "cache": out,
    }
    clk = clk.summary()
    if clk:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)


def run_onelayer(args, cfg):
    """One-layer boundary contraction (Algorithm 2 with the one-layer zip-up)
    of an 8 x 8 PEPS without physical index, the contraction bond equal to
    the initial bond, D = m = 2, 4, 8 (the supported range of the one-layer
    site stages), and D = 8 with m = 64: device seconds per contraction as a
    replayed CUDA graph, and the contracted log|v|."""
    import torch
    from paper_2006_15234_gb300 import libpeps
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    prec = {"plain": libpeps.PREC_PLAIN, "mixed": libpeps.PREC_MIXED, "fast": libpeps.PREC_FAST}[args.prec]
    stream = torch.cuda.current_stream()
    points = []
    with ClockSampler(0) as clk:
        for D, m in ((2, 2), (4, 4), (8, 8), (8, 64)):
            ket = synth.random_peps(cfg.nrow, cfg.ncol, 1, D, "f32", cfg.dist, cfg.seed + D)
            kt = [[torch.tensor(T, dtype=torch.float32, device=dev) for T in row] for row in ket]
            plan = libpeps.ContractPlan(kt, None, libpeps.make_opts(m, cfg.p, cfg.q, cfg.omega_seed, prec=prec))
            plan.execute()
            torch.cuda.synchronize()
            run = plan.execute if args.no_graph else libpeps.cuda_graph(plan.execute).replay
            for _ in range(max(1, args.warmup)):
                run()
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            la, _ = plan.result()
            points.append({"D": D, "m": m, "contraction_ms": round(float(np.mean(ms)), 4), "log_abs": la,
                           "kernel_launches": plan.kernel_launches()})
            del plan
    t = points[2]["contraction_ms"]
    line = {
        "metric": METRIC, "value": round(t / 1e3, 6), "unit": "s per contraction (D = m = 8)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded N(0,1)/2 PEPS without physical index)",
        "config": {"workload": cfg.name, "nrow": cfg.nrow, "ncol": cfg.ncol, "precision": args.prec,
                   "p": cfg.p, "q": cfg.q, "points": points, "cuda_graph": not args.no_graph},
    }
    clk = clk.summary()
    if clk:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)


def run_ite(args, cfg):
    """Imaginary-time evolution of the transverse-field Ising model on the
    8 x 8, D = 4 PEPS (Sec. II-D): an ITE step is one TEBD layer of
    exp(-tau H_j) (one-site operators, then Algorithm 1 on every bond,
    normalised bonds), timed as a replayed CUDA graph; the Rayleigh quotient
    (Eq. 6, cached environments), which the paper evaluates for the final
    state, is timed separately (one replayed graph of the expectation plan).
    Energies before and after the timed steps."""
    import torch
    from paper_2006_15234_gb300 import libpeps
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    prec = {"plain": libpeps.PREC_PLAIN, "mixed": libpeps.PREC_MIXED, "fast": libpeps.PREC_FAST}[args.prec]
    ket = synth.peps_for(cfg)
    kt = [[torch.tensor(T, dtype=torch.complex64, device=dev) for T in row] for row in ket]
    terms = synth.tfi_terms(cfg.nrow, cfg.ncol, cfg.extra["J"], cfg.extra["h"])
    Gb, Gs = synth.tfi_ite_gates(cfg.extra["J"], cfg.extra["h"], cfg.extra["tau"])
    drv = libpeps.IteDriver(kt, Gb, Gs, terms, libpeps.make_opts(cfg.m, cfg.p, cfg.q, cfg.omega_seed, prec=prec),
                            cfg.seed)
    fl_layer = sum(f for _, f, _ in drv.tebd.launches())
    stream = torch.cuda.current_stream()
    warm = max(3, args.warmup)
    e_start = drv.run(warm, every=warm)[-1]      # evolution, energy of the state reached
    torch.cuda.synchronize()
    layer, energy = drv.tebd.execute, drv.expect.execute
    if not args.no_graph:
        layer = libpeps.cuda_graph(drv.tebd.execute).replay
        energy = libpeps.cuda_graph(drv.expect.execute).replay
        torch.cuda.synchronize()

    def timed(fn, n):
        out = []
        for _ in range(n):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return float(np.mean(out))
    with ClockSampler(0) as clk:
        t_layer = timed(layer, args.steps)
        t_energy = timed(energy, 3)
    e_end = drv.expect.result()[0]
    line = {
        "metric": METRIC, "value": round(fl_layer / (t_layer * 1e-3) / 1e12, 4), "unit": "TFLOP/s",
        "n_gpus": 1, "steps": args.steps, "warmup": warm, "ms_per_step": round(t_layer, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": cfg.dtype,
        "data": "synthetic (seeded Gaussian PEPS start, exp(-tau H_j) of the TFI model)",
        "config": {"workload": cfg.name, "nrow": cfg.nrow, "ncol": cfg.ncol, "bond": cfg.D, "m": cfg.m,
                   "p": cfg.p, "q": cfg.q, "tau": cfg.extra["tau"], "precision_energy": args.prec,
                   "ite_steps_per_s": round(1e3 / t_layer, 2), "layer_ms": round(t_layer, 4),
                   "energy_eval_ms": round(t_energy, 4),
                   "energy_per_site_after_warmup": round(e_start / (cfg.nrow * cfg.ncol), 6),
                   "energy_per_site_after_timed_steps": round(e_end / (cfg.nrow * cfg.ncol), 6),
                   "cuda_graph": not args.no_graph,
                   "l2": "not flushed: each step reads what the previous one wrote"},
        "gpu_launches": drv.tebd.kernel_launches() * args.steps + drv.expect.kernel_launches() * 3,
    }
    clk = clk.summary()
    if clk:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)


def run_tebd(args, cfg):
    """One TEBD layer (Algorithm 1 on every nearest-neighbour bond, four
    passes of disjoint bonds) of the imaginary-time TFI gate on the 16 x 16,
    D = 8 complex64 PEPS, in place: device seconds per layer (each step
    evolves the state by one more layer) and the algorithmic flops of the
    site QR factorisations and the N = Q R~ products."""
    import torch
    from paper_2006_15234_gb300 import libpeps
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ket = synth.peps_for(cfg)
    kt = [[torch.tensor(T, dtype=torch.complex64, device=dev) for T in row] for row in ket]
    G = synth.tfi_bond_gate(cfg.extra["J"], cfg.extra["h"], cfg.extra["tau"])
    plan = libpeps.TebdPlan(kt, G, cfg.omega_seed)
    nbonds = cfg.nrow * (cfg.ncol - 1) + (cfg.nrow - 1) * cfg.ncol
    flops = sum(f for _, f, _ in plan.launches())
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(max(1, args.warmup)):
        plan.execute()
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            flush.add_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.execute()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    t = float(np.mean(ms))
    finite = all(bool(torch.isfinite(T).all()) for row in kt for T in row)
    # per-launch device times of one more layer (CUDA events on the stream)
    prof = plan.profile()
    by_tag, by_kern = {}, {}
    for (tag, fl, _), kname, dt in zip(plan.launches(), plan.kernels(), prof):
        by_tag[tag] = by_tag.get(tag, 0.0) + dt
        by_kern[kname] = by_kern.get(kname, 0.0) + dt
    line = {
        "metric": METRIC, "value": round(flops / (t * 1e-3) / 1e12, 4), "unit": "TFLOP/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": cfg.dtype,
        "data": "synthetic (seeded Gaussian PEPS, imaginary-time TFI gate)",
        "config": {"workload": cfg.name, "nrow": cfg.nrow, "ncol": cfg.ncol, "bond": cfg.D, "bonds": nbonds,
                   "tau": cfg.extra["tau"], "layer_s": round(t / 1e3, 6), "us_per_bond": round(1e3 * t / nbonds, 3),
                   "ledger_entries": plan.launch_count(), "launch_flops_gflop": round(flops / 1e9, 3),
                   "sites_finite": finite,
                   "l2": "flushed between steps (2x L2 write outside the timed events)"},
        "gpu_launches": plan.kernel_launches() * args.steps,
        "kernel_ms": {k: round(v, 4) for k, v in sorted(by_kern.items(), key=lambda kv: -kv[1])},
        "stage_ms": {k: round(v, 4) for k, v in sorted(by_tag.items(), key=lambda kv: -kv[1])},
    }
    clk = clk.summary()
    if clk:
        line["clocks"] = clk
    print(json.dumps(line), flush=True)


def cpu_baseline(cfg, args):
    """The oracle as it stands, on a bounded sample of the workload."""
    from oracle import bmps, rsvd
    cores = os.cpu_count()
    if cfg.name.startswith("c3"):
        # instances in order until about 15 s of oracle time
        fl, dt, cnt = 0.0, 0.0, 0
        for i, ((s, x), (m, D)) in enumerate(zip(batched_shapes(cfg), synth.batched_dims(cfg))):
            f = algorithmic_flops([dict(x, orth_n=True)], cfg.q, False)
            inst = synth.batched_instance(cfg, i, m, D)
            t0 = time.perf_counter()
            rsvd.einsumsvd(inst["V"], inst["S"], inst["ket"], inst["bra"], m, cfg.p, cfg.q, cfg.omega_seed, i)
            dt += time.perf_counter() - t0
            fl += f
            cnt += 1
            if dt > 15.0:
                break
        return {"value": round(fl / dt / 1e12, 6), "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                "sample": f"the first {cnt} of the 512 instances", "seconds": round(dt, 3)}
    ket = synth.peps_for(cfg)
    shapes = step_shapes(cfg)
    if cfg.nrow * cfg.ncol <= 64:
        t0 = time.perf_counter()
        bmps.contract(ket, ket if cfg.two_layer else None, cfg.m, cfg.p, cfg.q, cfg.omega_seed)
        dt = time.perf_counter() - t0
        fl = algorithmic_flops(shapes, cfg.q, cfg.dtype == "c64")
        sample = "one full contraction"
    else:
        # one implicit product A X of the largest einsumsvd step (the operation
        # that carries most of the flops), on all of its l sketch columns
        from oracle.implicit import ImplicitOp
        big = max(shapes, key=lambda s: s["prod_macs"])
        rng = np.random.default_rng(0)
        R = cfg.D ** 2
        kL = big["M"] // R
        a = b = cfg.m

        def cg(shape):
            z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
            return synth.round_to(z / np.linalg.norm(z), cfg.dtype)
        V, S = cg((kL, R, a, R)), cg((a, R, b))
        K = cg((cfg.d, cfg.D, cfg.D, cfg.D, cfg.D))
        op = ImplicitOp(V, S, K, K)
        cols = big["ell"]
        X = rng.standard_normal((op.N, cols)) + 1j * rng.standard_normal((op.N, cols))
        t0 = time.perf_counter()
        op.matvec(X)
        dt = time.perf_counter() - t0
        fl = 8.0 * big["prod_macs"] * cols / big["ell"]
        sample = (f"one implicit product A X of the largest einsumsvd step (M={big['M']}, N={big['N']}) "
                  f"on {cols} of its {big['ell']} sketch columns")
    return {"value": round(fl / dt / 1e12, 6), "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": sample, "seconds": round(dt, 3)}


def run_reference(args, cfg):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import bmps  # noqa: F401
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(cfg, args)
    t_all = []
    for _ in range(args.steps):
        r = cpu_baseline(cfg, args)
        vals.append(r["value"])
        t_all.append(r["seconds"])
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": "TFLOP/s",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * float(np.median(t_all)), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded Gaussian PEPS, shapes of the workload)",
            "config": {"workload": cfg.name, "precision": "fp64 oracle"},
            "cpu_baseline": {"value": round(v, 6), "unit": "TFLOP/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": round(v, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_step_profile(args, cfg):
    """One einsumsvd step of the workload's middle-step shape (kL = m, t = D^2,
    a = m, every bond D, complex64) with the right boundary bond b reduced to
    32 so that the step fits a few GB: per-stage and per-launch times from the
    plan's own event ledger, then a second execute bracketed by
    cudaProfilerStart / Stop for an ncu capture of single kernels
    (ncu --profile-from-start off -k regex:<kernel> -s <n> -c <k>)."""
    import numpy as np
    import torch
    from paper_2006_15234_gb300 import libpeps

    D, m, d = cfg.D, cfg.m, cfg.d
    shape = (m, D * D, m, 32, d) + (D,) * 8
    kL, t, a, b = shape[:4]
    prec = {"plain": libpeps.PREC_PLAIN, "mixed": libpeps.PREC_MIXED, "fast": libpeps.PREC_FAST}[args.prec]
    opts = libpeps.make_opts(m, cfg.p, cfg.q, cfg.omega_seed, prec=prec)
    plan = libpeps.EinsumsvdPlan(torch.complex64, [shape], opts)
    g = torch.Generator(device="cuda").manual_seed(1)

    def rnd(*sh):
        return torch.randn(*sh, dtype=torch.complex64, device="cuda", generator=g) / np.sqrt(np.prod(sh[1:]))

    V = rnd(kL, t, a, D * D)
    S = rnd(a, D * D, b)
    K = rnd(d, D, D, D, D)
    Kb = rnd(d, D, D, D, D)
    k = plan.ranks[0]
    M, N = kL * t, D * D * b * D * D
    U = torch.empty(M, k, dtype=torch.complex64, device="cuda")
    W = torch.empty(k, N, dtype=torch.complex64, device="cuda")
    sig = torch.empty(k, dtype=torch.float64, device="cuda")
    ls = torch.empty(1, dtype=torch.float64, device="cuda")
    io = [(V, S, K, Kb, U, W, sig, ls)]
    plan.execute(io)
    torch.cuda.synchronize()
    ms = plan.profile()
    launches = plan.launches()
    tags = {}
    for (tag, fl, by), t_ in zip(launches, ms):
        x = tags.setdefault(tag, [0.0, 0.0])
        x[0] += t_
        x[1] += fl
    stages = {tag: {"ms": round(t_, 4), "tflops": round(fl / max(t_, 1e-9) / 1e9, 2)}
              for tag, (t_, fl) in sorted(tags.items(), key=lambda kv: -kv[1][0])}
    per = [{"i": i, "tag": tag, "ms": round(t_, 4), "tflops": round(fl / max(t_, 1e-9) / 1e9, 2),
            "gbs": round(by / max(t_, 1e-9) / 1e6, 1)} for i, ((tag, fl, by), t_) in enumerate(zip(launches, ms))]
    torch.cuda.profiler.start()
    plan.execute(io)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"step_profile": {"shape": shape, "workspace_gb": round(plan.workspace_bytes / 1e9, 3),
                                       "stages": stages, "launches": per}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c5", choices=["c2", "c5", "c4", "c3", "f1", "f2", "f3", "f4"])
    ap.add_argument("--prec", default="mixed", choices=["plain", "mixed", "fast"])
    ap.add_argument("--no-compare-plain", action="store_true",
                    help="skip the plain FP32 contraction timed beside the mixed one")
    ap.add_argument("--fp64-small", action="store_true",
                    help="CholeskyQR2 factorisations and the Jacobi SVD in FP64 (PEPS_FLAG_FP64_SMALL)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the rule-based MMA widths (no stored or live tile table)")
    ap.add_argument("--tune-out", default=None, help="write a freshly tuned tile table to this file")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the batched-einsumsvd sub-record of the default run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--launch-list", action="store_true",
                    help="warm up, run one more contraction and exit (for an ncu launch list)")
    ap.add_argument("--step-profile", action="store_true",
                    help="one middle einsumsvd step (b = 32): stage ledger, then one execute for ncu")
    args = ap.parse_args()
    cfg = synth.config(args.config)
    if args.step_profile:
        run_step_profile(args, cfg)
    elif args.impl == "reference":
        run_reference(args, cfg)
    elif args.config == "c3":
        run_batched(args, cfg)
    elif args.config == "f2":
        run_expect_cache(args, cfg)
    elif args.config == "f1":
        run_tebd(args, cfg)
    elif args.config == "f3":
        run_ite(args, cfg)
    elif args.config == "f4":
        run_onelayer(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
