"""Benchmark: out-of-core GEMM effective TFLOP/s including host transfers.

Workload (default): plain FP64 C = 1.5*A*B + 0.5*C, M = N = K = 32768, entries
i.i.d. N(0,1) from the seeded Philox generator, A, B, C in pinned host memory
(3 x 8 GiB), device budget 4 GiB.  One step is one ooc_dgemm call through the
C ABI: every slice/block H2D, every tile kernel and every block D2H.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--config fp64-32768] [--n 32768] [--budget-gib 4]

value      = 2*M*N*K per step / device time of the step (CUDA events the library
             records on its own streams, first H2D start to last D2H end).
e2e        = the same metric on host wall time of the public call (argument
             checks, planning, arena allocation and release included).
roofline   = the dominant kernel (FP64 tile contraction): algorithmic FLOP per
             launch / mean launch time (CUDA events around each launch on the
             compute stream), against the FP64 peak.
cpu_baseline / --impl reference: the CPU oracle, as it stands, on sampled C
             blocks of the same problem, scaled to TFLOP/s.
Multi-GPU: the path is run as independent replicas (one per rank, weak scaling).
"""
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

import numpy as np  # noqa: E402

import synth  # noqa: E402

CONFIGS = {
    # name: (form, M, N, K, alpha, beta, budget bytes, distribution)
    "fp64-32768": ("fp64", 32768, 32768, 32768, 1.5, 0.5, 4 << 30, synth.NORMAL),
    "fp64-1024": ("fp64", 1024, 1024, 1024, 1.0, 0.0, 4 << 20, synth.UNIFORM),
    "ozaki-65536": ("ozaki", 65536, 65536, 16384, 1.0, 0.0, 16 << 30, synth.LOGSPREAD),
    "bf16x3-65536": ("bf16x3", 65536, 65536, 65536, 1.0, 1.0, 8 << 30, synth.UNIFORM),
    # 256 uneven FP64 problems, M, N, K log-uniform in [512, 32768], ~64 GiB host in total
    "batched-256": ("batched", 256, 512, 32768, 1.0, 0.0, 8 << 30, synth.NORMAL),
    # level-3 operations on the same pipeline (M = order, N = right-hand sides / K = inner dimension)
    "syrk-32768": ("syrk", 32768, 32768, 16384, 1.0, 0.5, 4 << 30, synth.NORMAL),
    "trsm-32768": ("trsm", 32768, 32768, 0, 1.0, 0.0, 4 << 30, synth.UNIFORM),
    "potrf-32768": ("potrf", 32768, 32768, 0, 1.0, 0.0, 4 << 30, synth.NORMAL),
    "getrf-32768": ("getrf", 32768, 32768, 0, 1.0, 0.0, 4 << 30, synth.NORMAL),
    # Section IV nsteps: 4 SUMMA-style calls with 4096-wide panels into one 65536^2 C, Ozaki form, C resident in HBM
    "summa-65536": ("summa", 65536, 65536, 16384, 1.0, 0.5, 48 << 30, synth.NORMAL),
    # the out-of-core GEMM written in the pipeline-description language, beside the built-in schedule
    "pipe-16384": ("pipe", 16384, 16384, 16384, 1.5, 0.5, 4 << 30, synth.NORMAL),
}
LEVEL3 = ("syrk", "trsm", "potrf", "getrf")
# per form: (element dtype name, relative Frobenius tolerance, products per logical product, dtype tag)
FORMS = {"fp64": ("float64", 1e-13, 1, "f64"), "ozaki": ("float64", 1e-12, 36, "f64 (bf16 digit planes)"),
         "bf16x3": ("float32", 1e-6, 6, "f32 (bf16x3 pieces)"), "batched": ("float64", 1e-13, 1, "f64"),
         "syrk": ("float64", 1e-13, 1, "f64"), "trsm": ("float64", 1e-12, 1, "f64"),
         "potrf": ("float64", 1e-12, 1, "f64"), "getrf": ("float64", 1e-12, 1, "f64"), "summa": ("float64", 1e-12, 36, "f64 (bf16 digit planes)"),
         "pipe": ("float64", 1e-13, 1, "f64")}


def batch_shapes(seed, count, lo, hi, cap=64 << 30, es=8):
    """Seeded (M, N, K) triples, each dimension log-uniform in [lo, hi]; a draw is
    kept only while the running host footprint stays within its pro-rata share
    of `cap` (count problems in about `cap` bytes of host memory)."""
    rng = np.random.default_rng(seed)
    out, used = [], 0
    while len(out) < count:
        m, n, k = (int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(3))
        fp = (m * k + k * n + m * n) * es
        if used + fp <= cap * (len(out) + 1) / count:
            out.append((m, n, k))
            used += fp
    return out
NOMINAL_FP64_TF, NOMINAL_BF16_TF = 1.25, 2250.0
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the
# dominant kernel, from one ncu capture of the configuration's plan (the summary
# under profiles/ named for the kernel); reported only when a run uses that plan.
TRAFFIC = {"fp64-32768": {"plan": (2048, 8192, 8192), "bytes": 2.624778e9 + 135.795456e6,
                          "profile": "profiles/fp64_tile_kernel_traffic_32768.md"},
           "ozaki-65536": {"plan": (1024, 21888, 16384), "bytes": 11.501296128e9 + 199.416576e6,
                           "profile": "profiles/tc_terms_kernel_traffic_65536.md"},
           "bf16x3-65536": {"plan": (1024, 7296, 65536), "bytes": 4.110287616e9 + 27.162880e6,
                            "profile": "profiles/tc_terms_kernel_traffic_65536.md"}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="fp64-32768", choices=sorted(CONFIGS))
    ap.add_argument("--n", type=int, default=0, help="override M = N = K (smaller runs)")
    ap.add_argument("--budget-gib", type=float, default=0.0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--form", default="", choices=["", "fp64", "ozaki"],
                    help="GEMM form of the level-3 configurations' updates (default FP64)")
    ap.add_argument("--repeat-ci", type=float, default=0.0, metavar="F",
                    help="GEMM configurations, one process: Section V's rule instead of exactly --steps timed "
                         "steps: at least max(3, steps), then more until the Student-t 95%% confidence "
                         "half-width of the step time is within F of its mean (the paper: 0.025)")
    ap.add_argument("--repeat-max-s", type=float, default=600.0,
                    help="cap on the timed seconds under --repeat-ci")
    return ap.parse_args()


# two-sided 95 % Student-t quantiles t(0.975, df); between entries the smaller df's (larger) value
T975 = ((1, 12.706), (2, 4.303), (3, 3.182), (4, 2.776), (5, 2.571), (6, 2.447), (7, 2.365), (8, 2.306),
        (9, 2.262), (10, 2.228), (12, 2.179), (15, 2.131), (20, 2.086), (25, 2.060), (30, 2.042),
        (40, 2.021), (60, 2.000), (120, 1.980))


def t975(df):
    try:
        from scipy import stats
        return float(stats.t.ppf(0.975, df))
    except ImportError:
        return [t for d, t in T975 if d <= df][-1]


def ci95(xs):
    """Mean and Student-t 95 % confidence half-width of independent observations (Section V)."""
    n = len(xs)
    if n < 2:
        return None
    mean = statistics.fmean(xs)
    hw = t975(n - 1) * statistics.stdev(xs) / n ** 0.5
    return {"n": n, "mean_s": mean, "half_width_s": hw, "frac": hw / mean if mean > 0 else None}


def run_timed(step, args, seconds_of, world):
    """The timed steps: exactly --steps, or with --repeat-ci F Section V's rule -- at least
    max(3, --steps), then one more at a time until the 95 % confidence half-width of the step
    time is within F of its mean or the timed steps reach --repeat-max-s seconds."""
    out = [step() for _ in range(args.steps)]
    if args.repeat_ci <= 0:
        return out, None
    if world > 1:
        raise SystemExit("--repeat-ci runs one process (the stopping rule is per process)")
    while len(out) < 3:
        out.append(step())
    while True:
        c = ci95([seconds_of(o) for o in out])
        spent = sum(seconds_of(o) for o in out)
        if c["frac"] is not None and c["frac"] <= args.repeat_ci or spent >= args.repeat_max_s:
            break
        out.append(step())
    c["rule"] = "Section V: repeat until the Student-t 95%% half-width <= %.3f of the mean (min 3, cap %.0f s)" % (
        args.repeat_ci, args.repeat_max_s)
    c["met"] = c["frac"] is not None and c["frac"] <= args.repeat_ci
    return out, c


def workload(args):
    form, M, N, K, alpha, beta, budget, dist = CONFIGS[args.config]
    if args.n and form != "batched":
        K = max(1, K * args.n // M)
        M = N = args.n
    if args.budget_gib:
        budget = int(args.budget_gib * (1 << 30))
    return dict(form=form, M=M, N=N, K=K, alpha=alpha, beta=beta, budget=budget, dist=dist)


def config_json(w, l2_note):
    dist = {synth.NORMAL: "N(0,1)", synth.UNIFORM: "U[-1,1]", synth.LOGSPREAD: "sign*10^U(-4,4)"}[w["dist"]]
    es = 4 if w["form"] == "bf16x3" else 8
    host = (w["M"] * w["K"] + w["K"] * w["N"] + w["M"] * w["N"]) * es
    return {"workload": "out-of-core %s GEMM M=%d N=%d K=%d, alpha=%g beta=%g, %s, host pinned %.0f GiB, "
                        "device budget %.2f GiB" % (w["form"].upper(), w["M"], w["N"], w["K"], w["alpha"], w["beta"],
                                                    dist, host / 2 ** 30, w["budget"] / 2 ** 30),
            "M": w["M"], "N": w["N"], "K": w["K"], "alpha": w["alpha"], "beta": w["beta"],
            "device_budget_bytes": w["budget"], "form": w["form"], "l2": l2_note}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def fp64_peak(P, local, no_clocks):
    """The device's FP64 peak measured by the library's probe (mma.sync f64 from registers,
    the instruction the FP64 tile kernel runs), with the SM clock sampled while it runs:
    (TFLOP/s, median SM MHz or None)."""
    clk = ClockSampler(local, enabled=not no_clocks)
    tf = P.ooc_query_fp64_peak(1.5)
    c = clk.stop()
    return tf, (c or {}).get("sm_mhz")


def fp64_roof_fields(pk, pk_src, probe, achieved, run_mhz):
    """Roofline fields of an FP64 kernel: the measured probe peak as the denominator, the bf16-derived
    figure beside it as context, and the fraction normalised by the SM clocks of both measurements."""
    tf, probe_mhz = probe
    derived = pk["bf16_tflops_sustained"] * NOMINAL_FP64_TF / NOMINAL_BF16_TF
    out = {"peak": tf, "frac": achieved / tf if achieved and tf else None,
           "peak_source": "measured: FP64 mma.sync probe (ooc_query_fp64_peak) in this run at %s MHz" % (
               "%.0f" % probe_mhz if probe_mhz else "unsampled"),
           "peak_derived_tflops": derived,
           "peak_derived_source": "%s bf16 sustained %.1f TF x nominal FP64/BF16 ratio %.2f/%.0f" % (
               pk_src, pk["bf16_tflops_sustained"], NOMINAL_FP64_TF, NOMINAL_BF16_TF),
           "probe_sm_mhz": probe_mhz, "run_sm_mhz": run_mhz}
    if achieved and tf and probe_mhz and run_mhz:
        out["frac_clock_normalised"] = (achieved / run_mhz) / (tf / probe_mhz)
    return out


def sample_blocks(w, count, r, seed=12345):
    rng = np.random.default_rng(seed)
    i0 = rng.integers(0, max(1, w["M"] - r + 1), size=count)
    j0 = rng.integers(0, max(1, w["N"] - r + 1), size=count)
    return list(zip(i0.tolist(), j0.tolist()))


def oracle_sample(w, A, B, Cold_blocks, blocks, r, nthreads):
    """Oracle values of the sampled blocks; returns (list of arrays, seconds, threads)."""
    import oracle
    out, t0, used = [], time.perf_counter(), 1
    for (i0, j0), cold in zip(blocks, Cold_blocks):
        v, used = oracle.gemm_block("N", "N", i0, j0, r, r, w["K"], w["alpha"], A, B, w["beta"],
                                    cold if w["beta"] != 0 else None, nthreads=nthreads)
        out.append(v)
    return out, time.perf_counter() - t0, used


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def calibrate_sample(w, A, B, C, target_s, r, nthreads):
    """Number of r x r blocks the oracle computes in about target_s seconds (at least 2)."""
    blocks = sample_blocks(w, 1, r, seed=999)
    cold = [C[i:i + r, j:j + r].numpy().astype(np.float64) for i, j in blocks]
    _, dt, _ = oracle_sample(w, A, B, cold, blocks, r, nthreads)
    return max(2, min(256, int(target_s / max(dt, 1e-3))))


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, enabled=True):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        if not enabled:
            return
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r[2] > 250.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in load for k in range(4) if r[3][1 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "samples_under_load": len(load),
                "reasons": reasons}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(values, pg):
    """Element-wise maximum of this rank's timings over all ranks (the values themselves alone)."""
    if not pg:
        return list(values)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().tolist()


def run_reference(args, w, world, rank, pg):
    """--impl reference: the CPU oracle on a bounded sample of the same workload."""
    if rank != 0:
        return
    import torch
    r = 64
    cores = host_cores()
    dt = getattr(torch, FORMS[w["form"]][0])
    A = torch.empty((w["M"], w["K"]), dtype=dt)
    B = torch.empty((w["K"], w["N"]), dtype=dt)
    C = torch.empty((w["M"], w["N"]), dtype=dt)
    for t, s in ((A, 0), (B, 1), (C, 2)):
        synth.fill(t, 1, s, w["dist"])
    per_step = max(1, calibrate_sample(w, A, B, C, args.cpu_seconds / max(1, args.steps + args.warmup), r, cores))
    blocks = sample_blocks(w, per_step, r)
    cold = [C[i:i + r, j:j + r].numpy().astype(np.float64) for i, j in blocks]
    for _ in range(args.warmup):
        oracle_sample(w, A, B, cold, blocks, r, cores)
    times = []
    for _ in range(args.steps):
        _, dt, used = oracle_sample(w, A, B, cold, blocks, r, cores)
        times.append(dt)
    flops = 2.0 * r * r * w["K"] * per_step
    value = flops * len(times) / sum(times) / 1e12
    sample = "%d seeded %dx%d blocks of C per step, K=%d (full problem extrapolated at this rate)" % (
        per_step, r, r, w["K"])
    line = {"impl": "reference", "metric": "out-of-core GEMM effective TFLOP/s incl. transfers",
            "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": FORMS[w["form"]][3], "data": "synthetic (seeded Philox)",
            "config": config_json(w, "CPU oracle"),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, w, world, rank, local, pg):
    import torch
    import paper_1808_05056_gb300 as P

    torch.cuda.set_device(local)
    P.load()
    M, N, K = w["M"], w["N"], w["K"]
    dtname, tol, products, dtag = FORMS[w["form"]]
    dt = getattr(torch, dtname)
    A = torch.empty((M, K), dtype=dt, pin_memory=True)
    B = torch.empty((K, N), dtype=dt, pin_memory=True)
    C = torch.empty((M, N), dtype=dt, pin_memory=True)
    t_fill = time.perf_counter()
    for t, s in ((A, 0), (B, 1), (C, 2)):
        synth.fill(t, 1 + rank, s, w["dist"])
    t_fill = time.perf_counter() - t_fill
    form_id = {"fp64": P.OOC_FORM_FP64, "ozaki": P.OOC_FORM_OZAKI, "bf16x3": P.OOC_FORM_BF16X3}[w["form"]]
    opts = P.make_opts(form=form_id)
    call = P.ooc_sgemm if w["form"] == "bf16x3" else P.ooc_dgemm

    def step():
        st = P.ooc_stats()
        t0 = time.perf_counter()
        rc = call("N", "N", M, N, K, w["alpha"], A, K, B, N, w["beta"], C, N, w["budget"], opts, st)
        wall = time.perf_counter() - t0
        if rc != 0:
            raise RuntimeError("ooc_dgemm failed: %s: %s" % (P.ooc_strerror(rc), P.ooc_last_error()))
        return st, wall

    # warm-up; the last one is checked against the oracle on sampled blocks
    r = 64
    cores = host_cores()
    n_blocks = calibrate_sample(w, A, B, C, args.cpu_seconds, r, cores) if rank == 0 else 0
    blocks = sample_blocks(w, n_blocks, r)
    for k in range(max(0, args.warmup - 1)):
        step()
    cold = [C[i:i + r, j:j + r].numpy().astype(np.float64) for i, j in blocks]
    step()
    parity = None
    cpu = None
    if rank == 0:
        ref, dt, used = oracle_sample(w, A, B, cold, blocks, r, cores)
        errs = []
        for (i, j), rv in zip(blocks, ref):
            got = C[i:i + r, j:j + r].numpy()
            errs.append(float(np.linalg.norm(got - rv) / np.linalg.norm(rv)))
        parity = {"max_rel_fro": max(errs), "tolerance": tol, "blocks": len(blocks), "block": r,
                  "pass": max(errs) <= tol}
        cpu = {"value": 2.0 * r * r * K * len(blocks) / dt / 1e12, "unit": "TFLOP/s", "cores": used,
               "kind": "oracle",
               "sample": "%d seeded %dx%d blocks of C, K=%d, %.1f s (full problem extrapolated at this rate)" % (
                   len(blocks), r, r, K, dt)}

    # live FP64 reference rate of the device (cuBLAS DGEMM), context for the peak
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    torch.matmul(a, a)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        torch.matmul(a, a)
    e1.record()
    torch.cuda.synchronize()
    cublas_tf = 3 * 2 * 4096 ** 3 / (e0.elapsed_time(e1) / 1e3) / 1e12
    del a
    probe = fp64_peak(P, local, args.no_clocks) if w["form"] == "fp64" else (None, None)

    clk = ClockSampler(local, enabled=not args.no_clocks)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    stats, repeat = run_timed(step, args, lambda o: o[0].device_seconds, world)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.stop()
    n_steps = len(stats)

    dev_s = sum(s.device_seconds for s, _ in stats)
    wall_s = sum(wl for _, wl in stats)
    ker_s = sum(s.kernel_seconds for s, _ in stats)
    split_s = sum(s.split_seconds for s, _ in stats)
    launches = sum(s.kernel_launches for s, _ in stats)
    dev_s, wall_s = max_over_ranks([dev_s, wall_s], pg)
    if rank != 0:
        return
    flops = 2.0 * M * N * K
    value = world * flops * n_steps / dev_s / 1e12
    e2e = world * flops * n_steps / wall_s / 1e12
    pk, pk_src = peaks()
    s0 = stats[0][0]
    link_h2d, link_d2h = P.ooc_query_device()[1:]
    b_alg = s0.h2d_bytes + s0.d2h_bytes
    tr = TRAFFIC.get(args.config)
    traffic = tr["bytes"] if tr and not args.n and (s0.mb, s0.nb, s0.kb) == tr["plan"] else None
    if w["form"] == "fp64":
        achieved = flops * n_steps / ker_s / 1e12
        roof = {"bound": "tensor", "kernel": "fp64_tile_kernel (FP64 mma.sync, TMA-fed)",
                "achieved": achieved, "unit": "TFLOP/s", "traffic": traffic,
                "traffic_alg_bytes": 8.0 * (s0.mb * s0.kb + s0.kb * s0.nb + 2 * s0.mb * s0.nb),
                "traffic_source": tr["profile"] if traffic else None,
                "fp64_cublas_measured_tflops": cublas_tf, "frac_of_cublas_dgemm": achieved / cublas_tf,
                "launches_per_step": s0.steps}
        roof.update(fp64_roof_fields(pk, pk_src, probe, achieved, (clocks or {}).get("sm_mhz")))
        compute_peak = roof["peak"]
    else:
        peak = pk["bf16_tflops_sustained"]
        # the contraction alone: its launches' event time minus the split kernels before them
        achieved = flops * s0.products * n_steps / (ker_s - split_s) / 1e12
        roof = {"bound": "tensor",
                "kernel": "tc_terms_kernel (tcgen05 bf16 x bf16 -> f32 TMEM, TMA)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                "split_kernels_s_per_step": split_s / n_steps,
                "with_split_kernels": flops * s0.products * n_steps / ker_s / 1e12,
                "traffic_alg_bytes": (s0.slices if w["form"] == "ozaki" else 3) * 2.0 * (s0.mb + s0.nb) * s0.kb +
                                     (2.0 if w["beta"] != 0 else 1.0) * s0.mb * s0.nb * (4 if w["form"] == "bf16x3" else 8),
                "traffic_source": tr["profile"] if traffic else None,
                "flop_count": "2*M*N*K x %d bf16 products per logical product" % s0.products,
                "peak_source": "%s bf16 sustained (cuBLAS) %.1f TF" % (pk_src, peak),
                "logical_tflops": flops * n_steps / (ker_s - split_s) / 1e12, "launches_per_step": s0.steps}
        compute_peak = peak / s0.products
    t_roof = max(flops / (compute_peak * 1e12), s0.h2d_bytes / (link_h2d * 1e9), s0.d2h_bytes / (link_d2h * 1e9))
    host_gib = (M * K + K * N + M * N) * (4 if w["form"] == "bf16x3" else 8) / 2 ** 30
    line = {
        "metric": "out-of-core GEMM effective TFLOP/s incl. transfers",
        "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": n_steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dev_s / n_steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtag, "data": "synthetic (seeded Philox, pinned host)",
        "config": config_json(w, "inputs larger than L2: %.0f GiB host operands streamed through a %.2f GiB "
                                 "device budget each step" % (host_gib, w["budget"] / 2 ** 30)),
        "roofline": roof,
        "ooc_roofline": {"t_roof_s": t_roof, "t_step_s": dev_s / n_steps, "frac": t_roof / (dev_s / n_steps),
                         "compute_peak_logical_tflops": compute_peak, "h2d_gbps": link_h2d, "d2h_gbps": link_d2h,
                         "h2d_bytes": s0.h2d_bytes, "d2h_bytes": s0.d2h_bytes, "bytes_alg": b_alg},
        "plan": {"mb": s0.mb, "nb": s0.nb, "kb": s0.kb, "depth": s0.depth, "b_buffers": s0.b_buffers,
                 "c_buffers": s0.c_buffers, "blocks": s0.blocks, "device_bytes": s0.device_bytes},
        "e2e": {"value": e2e, "unit": "TFLOP/s", "h2d_bytes_per_step": s0.h2d_bytes,
                "d2h_bytes_per_step": s0.d2h_bytes},
        "gpu_launches": launches,
        "fp64_cublas_measured_tflops": cublas_tf,
        "parity": parity,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "setup_fill_s": t_fill,
        "repeat": repeat if repeat else ci95([st.device_seconds for st, _ in stats]),
    }
    print(json.dumps(line), flush=True)


def run_batched_bench(args, w, world, rank, local, pg):
    """Batched configuration: one ooc_dgemm_batched call over all problems per step
    (--impl reference: the oracle on sampled blocks of the same problems)."""
    import torch
    count, lo, hi = w["M"], w["N"], w["K"]
    if args.n:  # smaller runs: fewer, smaller problems
        count, hi = max(4, args.n // 128), max(lo, min(hi, args.n))
    shapes = batch_shapes(1234, count, lo, hi)
    flops = sum(2.0 * m * n * k for m, n, k in shapes)
    r = 32
    cores = host_cores()
    if args.impl == "reference":
        if rank != 0:
            return
        picks = list(range(0, len(shapes), max(1, len(shapes) // 8)))[:8]
        per = []
        for q in picks:
            m, n, k = shapes[q]
            A = torch.empty((m, k), dtype=torch.float64); B = torch.empty((k, n), dtype=torch.float64)
            synth.fill(A, 100 + q, 0, w["dist"]); synth.fill(B, 100 + q, 1, w["dist"])
            per.append((q, A, B))
        times = []
        for it in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            for q, A, B in per:
                m, n, k = shapes[q]
                wq = dict(w, M=m, N=n, K=k, beta=0.0)
                oracle_sample(wq, A, B, [None], sample_blocks(wq, 1, r, seed=q), r, cores)
            if it >= args.warmup:
                times.append(time.perf_counter() - t0)
        fl = sum(2.0 * r * r * shapes[q][2] for q, _, _ in per)
        value = fl * len(times) / sum(times) / 1e12
        line = {"impl": "reference", "metric": "out-of-core GEMM effective TFLOP/s incl. transfers", "value": value,
                "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Philox)",
                "config": {"workload": "%d uneven FP64 GEMMs, M,N,K log-uniform [%d, %d]" % (len(shapes), lo, hi)},
                "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                                 "sample": "one %dx%d block of C in each of %d of the problems per step" % (r, r, len(per))},
                "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import paper_1808_05056_gb300 as P
    torch.cuda.set_device(local)
    P.load()
    ops = []
    t_fill = time.perf_counter()
    for q, (m, n, k) in enumerate(shapes):
        A = torch.empty((m, k), dtype=torch.float64, pin_memory=True)
        B = torch.empty((k, n), dtype=torch.float64, pin_memory=True)
        C = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
        synth.fill(A, 100 + q + 1000 * rank, 0, w["dist"])
        synth.fill(B, 100 + q + 1000 * rank, 1, w["dist"])
        ops.append((A, B, C))
    t_fill = time.perf_counter() - t_fill
    descs = [P.gemm_desc("N", "N", A, B, C, w["alpha"], w["beta"]) for A, B, C in ops]
    # CUDA-graph capture of the whole batched pipeline: measured faster (1.041 vs 1.031 TFLOP/s), the default
    graph = os.environ.get("OOC_BENCH_GRAPH", "1") == "1"
    # plans from the learned cost model when its file is present (else the analytic planner)
    from paper_1808_05056_gb300 import tune
    planner = "analytic"
    flags = P.OOC_BATCH_GRAPH if graph else 0
    if os.environ.get("OOC_BENCH_PLANNER", "model") == "model" and os.path.exists(tune.DEFAULT_MODEL):
        tune.install()
        flags |= P.OOC_PLAN_MODEL
        planner = "learned cost model (%s)" % os.path.basename(tune.DEFAULT_MODEL)
    opts = P.make_opts(form=P.OOC_FORM_FP64, flags=flags)

    def step():
        st = P.ooc_stats()
        t0 = time.perf_counter()
        rc = P.ooc_dgemm_batched(descs, w["budget"], opts, st)
        wall = time.perf_counter() - t0
        if rc != 0:
            raise RuntimeError("ooc_dgemm_batched: %s: %s" % (P.ooc_strerror(rc), P.ooc_last_error()))
        return st, wall

    for _ in range(args.warmup):
        step()
    # parity on one sampled block of a spread of problems (beta = 0: C is recomputed each step)
    parity = None
    cpu = None
    if rank == 0:
        errs, t_or, fl = [], 0.0, 0.0
        for q in range(0, len(shapes), max(1, len(shapes) // 8)):
            m, n, k = shapes[q]
            A, B, C = ops[q]
            wq = dict(w, M=m, N=n, K=k)
            blk = sample_blocks(wq, 1, r, seed=q)
            ref, dt, used = oracle_sample(wq, A, B, [None], blk, r, cores)
            t_or += dt
            fl += 2.0 * r * r * k
            i, j = blk[0]
            got = C[i:i + r, j:j + r].numpy()
            errs.append(float(np.linalg.norm(got - ref[0]) / np.linalg.norm(ref[0])))
        parity = {"max_rel_fro": max(errs), "tolerance": 1e-13, "problems_checked": len(errs), "block": r,
                  "pass": max(errs) <= 1e-13}
        cpu = {"value": fl / t_or / 1e12, "unit": "TFLOP/s", "cores": used, "kind": "oracle",
               "sample": "one %dx%d block of C in each of %d problems, %.1f s" % (r, r, len(errs), t_or)}
    probe = fp64_peak(P, local, args.no_clocks)
    clk = ClockSampler(local, enabled=not args.no_clocks)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    stats, repeat = run_timed(step, args, lambda o: o[0].device_seconds, world)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.stop()
    n_steps = len(stats)
    dev_s = sum(st.device_seconds for st, _ in stats)
    wall_s = sum(wl for _, wl in stats)
    ker_s = sum(st.kernel_seconds for st, _ in stats)
    dev_s, wall_s = max_over_ranks([dev_s, wall_s], pg)
    if rank != 0:
        return
    s0 = stats[0][0]
    if s0.mb == 0:  # grouped path: problems multiplied whole, nothing planned
        planner = "none: every problem fits whole in half the budget, grouped (%d groups)" % s0.steps
    pk, pk_src = peaks()
    # the two halves' kernels overlap, so the summed kernel time over-counts: device time instead
    achieved = flops * n_steps / dev_s / 1e12 if dev_s > 0 else None
    roof = {"bound": "tensor", "kernel": "fp64_tile_kernel (FP64 mma.sync, TMA-fed)", "achieved": achieved,
            "unit": "TFLOP/s", "traffic": None}
    roof.update(fp64_roof_fields(pk, pk_src, probe, achieved, (clocks or {}).get("sm_mhz")))
    line = {
        "metric": "out-of-core GEMM effective TFLOP/s incl. transfers",
        "value": world * flops * n_steps / dev_s / 1e12, "unit": "TFLOP/s", "n_gpus": world,
        "steps": n_steps, "warmup": args.warmup, "ms_per_step": 1e3 * dev_s / n_steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Philox N(0,1), pinned host)",
        "config": {"workload": "%d uneven FP64 GEMMs, M,N,K log-uniform in [%d, %d] (seed 1234), %.1f GiB host, "
                               "device budget %.2f GiB, one ooc_dgemm_batched call per step%s" % (
                                   len(shapes), lo, hi,
                                   sum((m * k + k * n + m * n) * 8 for m, n, k in shapes) / 2 ** 30,
                                   w["budget"] / 2 ** 30, " (CUDA graph)" if graph else ""),
                   "problems": len(shapes), "total_flop": flops, "planner": planner,
                   "l2": "inputs larger than L2 (tens of GiB of host operands per step)"},
        "roofline": roof,
        "e2e": {"value": world * flops * n_steps / wall_s / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": s0.h2d_bytes, "d2h_bytes_per_step": s0.d2h_bytes},
        "gpu_launches": sum(st.kernel_launches for st, _ in stats),
        "parity": parity, "cpu_baseline": cpu, "clocks": clocks, "setup_fill_s": t_fill,
        "repeat": repeat if repeat else ci95([st.device_seconds for st, _ in stats]),
    }
    print(json.dumps(line), flush=True)


def level3_flops(w):
    n = w["M"]
    if w["form"] == "syrk":
        return float(n) * (n + 1) * w["K"]
    if w["form"] == "trsm":
        return float(n) * n * w["N"]
    if w["form"] == "getrf":
        return 2.0 * float(n) ** 3 / 3.0
    return float(n) ** 3 / 3.0


def level3_inputs(w, rank, torch):
    """Pinned host operands of a level-3 configuration (and pristine copies of what the call overwrites)."""
    n, N, K = w["M"], w["N"], w["K"]
    seed = 300 + rank
    if w["form"] == "syrk":
        A = torch.empty((n, K), dtype=torch.float64, pin_memory=True)
        C = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        synth.fill(A, seed, 0, w["dist"])
        synth.fill(C, seed, 2, w["dist"])
        return dict(A=A, C=C)
    if w["form"] == "trsm":
        # lower triangular, diagonally dominant: off-diagonal U[-1,1] / n, diagonal 2 (well conditioned)
        A = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        synth.fill(A, seed, 0, w["dist"])
        a = A.numpy()
        for r0 in range(0, n, 4096):   # row strips: bounded temporary memory
            blk = a[r0:r0 + 4096]
            blk *= 1.0 / n
            blk[:, r0 + 4096:] = 0.0
            for i in range(blk.shape[0]):
                blk[i, r0 + i + 1:] = 0.0
                blk[i, r0 + i] = 2.0
        B = torch.empty((n, N), dtype=torch.float64, pin_memory=True)
        synth.fill(B, seed, 1, synth.NORMAL)
        B0 = torch.empty_like(B, pin_memory=True)
        B0.copy_(B)
        return dict(A=A, B=B, B0=B0)
    if w["form"] == "getrf":
        A = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
        synth.fill(A, seed, 0, w["dist"])
        A0 = torch.empty_like(A, pin_memory=True)
        A0.copy_(A)
        return dict(A=A, A0=A0, ipiv=np.zeros(n, dtype=np.int64))
    # potrf: symmetric N(0,1) off the diagonal (lower triangle read), diagonal n + N(0,1): SPD, well conditioned
    A = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    synth.fill(A, seed, 0, w["dist"])
    a = A.numpy()
    a[np.diag_indices(n)] += float(n)
    A0 = torch.empty_like(A, pin_memory=True)
    A0.copy_(A)
    return dict(A=A, A0=A0)


def level3_call(P, w, ops, opts, st):
    n, N, K = w["M"], w["N"], w["K"]
    if w["form"] == "syrk":
        return P.ooc_dsyrk("L", "N", n, K, w["alpha"], ops["A"], K, w["beta"], ops["C"], n, w["budget"], opts, st), 0
    if w["form"] == "trsm":
        return P.ooc_dtrsm("L", "L", "N", "N", n, N, w["alpha"], ops["A"], n, ops["B"], N, w["budget"], opts, st), 0
    if w["form"] == "getrf":
        return P.ooc_dgetrf(n, ops["A"], n, ops["ipiv"], w["budget"], opts, st)
    return P.ooc_dpotrf("L", n, ops["A"], n, w["budget"], opts, st)


def level3_restore(w, ops):
    """Put back what the previous call overwrote (outside the timed region)."""
    if w["form"] == "trsm":
        ops["B"].copy_(ops["B0"])
    elif w["form"] in ("potrf", "getrf"):
        ops["A"].copy_(ops["A0"])


def level3_parity(w, ops, before, cores):
    """Oracle check of the last call on a bounded sample; returns (parity dict, cpu_baseline dict)."""
    from oracle import level3 as L3
    import oracle
    n, N, K = w["M"], w["N"], w["K"]
    tol = FORMS[w["form"]][1]
    if w["form"] == "syrk":
        r = 64
        t0 = time.perf_counter()
        errs = []
        for (i, j), c0 in before:
            ref = L3.syrk_block("L", "N", i, j, r, r, w["alpha"], ops["A"].numpy(), w["beta"], c0, nthreads=cores)
            errs.append(oracle.rel_fro(ops["C"].numpy()[i:i + r, j:j + r][L3.tri_mask(r, r, "L", 0, i, j)],
                                       ref[L3.tri_mask(r, r, "L", 0, i, j)]))
        dt = time.perf_counter() - t0
        flops = 2.0 * r * r * K * len(before)
        sample = "%d seeded %dx%d blocks of the lower triangle, K=%d" % (len(before), r, r, K)
    elif w["form"] == "trsm":
        cols = before["cols"]
        t0 = time.perf_counter()
        ref = L3.trsm("L", "L", "N", "N", w["alpha"], ops["A"].numpy(), before["B0"], nthreads=cores)
        dt = time.perf_counter() - t0
        got = ops["B"].numpy()[:, cols]
        errs = [oracle.rel_fro(got, ref)]
        flops = float(n) * n * len(cols)
        sample = "%d seeded right-hand sides (columns of B) of order %d" % (len(cols), n)
    elif w["form"] == "getrf":
        # entries of P A - L U, each scaled by (|L| |U|)_ij: the entrywise backward error
        a, a0, ipiv = ops["A"].numpy(), ops["A0"].numpy(), ops["ipiv"]
        rows = np.arange(n)
        for j, p in enumerate(ipiv):
            rows[j], rows[p] = rows[p], rows[j]
        t0 = time.perf_counter()
        worst, lmax = 0.0, 0.0
        for (i, j) in before["entries"]:
            k = min(i, j)
            l = np.append(a[i, :k], 1.0 if i <= j else a[i, k])   # L[i, 0..k]
            u = a[:k + 1, j].copy()                                 # U[0..k, j]
            if i > j:
                u[k] = a[k, j]
            lu = float(np.dot(l, u))
            scale = float(np.dot(np.abs(l), np.abs(u)))
            worst = max(worst, abs(lu - a0[rows[i], j]) / max(scale, 1e-300))
            lmax = max(lmax, float(np.abs(a[i, :min(i, n)]).max()) if i > 0 else 0.0)
        dt = time.perf_counter() - t0
        errs = [worst] + ([0.0] if lmax <= 1.0 else [float("inf")])
        flops = 2.0 * n * len(before["entries"])
        sample = "%d sampled entries of P A - L U (backward error, scaled by |L||U|) and |L| <= 1 on their rows" % (
            len(before["entries"]))
    else:
        b = before["lead"]
        t0 = time.perf_counter()
        ref, info = L3.potrf("L", before["A0lead"], nthreads=cores)
        dt = time.perf_counter() - t0
        m = L3.tri_mask(b, b, "L")
        errs = [oracle.rel_fro(ops["A"].numpy()[:b, :b][m], ref[m])]
        # sampled entries of L L^T against the input, anywhere in the matrix
        a = ops["A"].numpy()
        worst = 0.0
        for (i, j), aij in before["entries"]:
            k = min(i, j) + 1
            llt = float(np.dot(a[i, :k], a[j, :k]))
            worst = max(worst, abs(llt - aij) / float(n))
        errs.append(worst)
        flops = float(b) ** 3 / 3.0
        sample = "leading %dx%d block factored by the oracle; %d sampled entries of L L^T" % (
            b, b, len(before["entries"]))
    parity = {"max_rel_fro": float(max(errs)), "tolerance": tol, "pass": bool(max(errs) <= tol)}
    cpu = {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
           "sample": sample + ", %.1f s" % dt}
    return parity, cpu


def level3_snapshot(w, ops):
    """What the oracle check needs from the inputs of the next call."""
    n, N = w["M"], w["N"]
    rng = np.random.default_rng(4321)
    if w["form"] == "syrk":
        r = 64
        out = []
        for _ in range(12):
            i = int(rng.integers(0, n - r + 1))
            j = int(rng.integers(0, i + 1)) if i > 0 else 0
            out.append(((i, j), ops["C"].numpy()[i:i + r, j:j + r].copy()))
        out.append(((0, 0), ops["C"].numpy()[:r, :r].copy()))
        out.append(((n - r, n - r), ops["C"].numpy()[n - r:, n - r:].copy()))
        return out
    if w["form"] == "trsm":
        cols = sorted(set(int(c) for c in rng.integers(0, N, size=6)) | {0, N - 1})
        return {"cols": cols, "B0": ops["B"].numpy()[:, cols].copy()}
    if w["form"] == "getrf":
        return {"entries": [(int(rng.integers(0, n)), int(rng.integers(0, n))) for _ in range(64)]}
    b = min(n, 2048)
    ents = []
    for _ in range(64):
        i = int(rng.integers(0, n))
        j = int(rng.integers(0, i + 1))
        ents.append(((i, j), float(ops["A"].numpy()[i, j])))
    return {"lead": b, "A0lead": ops["A"].numpy()[:b, :b].copy(), "entries": ents}


def run_level3_bench(args, w, world, rank, local, pg):
    """SYRK / TRSM / Cholesky configurations: one driver call per step."""
    import torch
    cores = host_cores()
    flops = level3_flops(w)
    metric = "out-of-core %s effective TFLOP/s incl. transfers" % w["form"].upper()
    desc = {"syrk": "SYRK C = A A^T (lower) N=%d K=%d, alpha=%g beta=%g, N(0,1)" % (w["M"], w["K"], w["alpha"],
                                                                                   w["beta"]),
            "trsm": "TRSM L X = B, lower non-unit, M=%d N=%d, diagonally dominant" % (w["M"], w["N"]),
            "potrf": "Cholesky A = L L^T N=%d, SPD (symmetric N(0,1) + N I)" % w["M"],
            "getrf": "LU with partial pivoting P A = L U N=%d, N(0,1)" % w["M"]}[w["form"]]
    cfg = {"workload": "out-of-core " + desc + ", device budget %.2f GiB" % (w["budget"] / 2 ** 30),
           "form": w["form"], "update_form": args.form or "fp64", "device_budget_bytes": w["budget"],
           "l2": "inputs larger than L2: host operands of %d GiB streamed through the device budget" % (
               (8 * w["M"] * (w["M"] + max(w["N"], w["K"]))) >> 30)}
    import torch
    ops = level3_inputs(w, rank, torch)
    if args.impl == "reference":
        if rank != 0:
            return
        times = []
        for it in range(args.warmup + args.steps):
            snap = level3_snapshot(w, ops)
            par, cpu = level3_parity(w, ops, snap, cores)   # the oracle on the sample (parity is vacuous here)
            if it >= args.warmup:
                times.append(cpu)
        value = sum(c["value"] for c in times) / len(times)
        line = {"impl": "reference", "metric": metric, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Philox)",
                "config": cfg, "cpu_baseline": dict(times[-1], value=value),
                "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    import paper_1808_05056_gb300 as P
    torch.cuda.set_device(local)
    P.load()
    opts = P.make_opts(form=P.OOC_FORM_OZAKI if args.form == "ozaki" else P.OOC_FORM_FP64)

    def step():
        st = P.ooc_stats()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, info = level3_call(P, w, ops, opts, st)
        wall = time.perf_counter() - t0
        if rc != 0 or info != 0:
            raise RuntimeError("%s failed: %s (info %d): %s" % (w["form"], P.ooc_strerror(rc), info,
                                                                P.ooc_last_error()))
        return st, wall

    for k in range(max(0, args.warmup - 1)):
        step()
        level3_restore(w, ops)
    snap = level3_snapshot(w, ops) if rank == 0 else None
    step()
    parity = cpu = None
    if rank == 0:
        parity, cpu = level3_parity(w, ops, snap, cores)
    level3_restore(w, ops)
    probe = fp64_peak(P, local, args.no_clocks) if args.form != "ozaki" else (None, None)
    clk = ClockSampler(local, enabled=not args.no_clocks)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    stats = []
    for k in range(args.steps):
        stats.append(step())
        if k + 1 < args.steps:
            level3_restore(w, ops)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.stop()
    wall_s = sum(wl for _, wl in stats)
    ker_s = sum(s.kernel_seconds for s, _ in stats)
    wall_s, = max_over_ranks([wall_s], pg)
    if rank != 0:
        return
    s0 = stats[0][0]
    value = world * flops * args.steps / wall_s / 1e12
    pk, pk_src = peaks()
    achieved = flops * args.steps / wall_s / 1e12
    roof = {"bound": "tensor", "kernel": "pipelined out-of-core GEMM updates (%s tile kernel)" % (
                "tc_terms Ozaki" if args.form == "ozaki" else "fp64_tile"),
            "achieved": achieved, "unit": "TFLOP/s", "traffic": None}
    if args.form != "ozaki":
        roof.update(fp64_roof_fields(pk, pk_src, probe, achieved, (clocks or {}).get("sm_mhz")))
    else:
        nprod = s0.products or 45
        roof.update({"peak": pk["bf16_tflops_sustained"] / nprod, "frac": achieved / (pk["bf16_tflops_sustained"] / nprod),
                     "peak_source": "%s bf16 sustained %.1f TF / %d Ozaki digit products" % (
                         pk_src, pk["bf16_tflops_sustained"], nprod)})
    line = {
        "metric": metric, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Philox, pinned host)",
        "config": cfg,
        "roofline": roof,
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": s0.h2d_bytes,
                "d2h_bytes_per_step": s0.d2h_bytes},
        "gpu_launches": s0.kernel_launches,
        "gemm_calls_per_step": s0.steps, "kernel_seconds_per_step": ker_s / args.steps,
        "parity": parity, "cpu_baseline": cpu, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_summa_bench(args, w, world, rank, local, pg):
    """nsteps configuration: one session (create, 4 calls, finish) per step, against the same
    calls made one by one with ooc_dgemm (every C block crosses the link in every call)."""
    import torch
    M, N, K = w["M"], w["N"], w["K"]
    ks = 4096                      # SUMMA panel width
    nsteps = max(1, K // ks)
    K = ks * nsteps
    cores = host_cores()
    panels = []
    for q in range(nsteps):
        A = torch.empty((M, ks), dtype=torch.float64, pin_memory=True)
        B = torch.empty((ks, N), dtype=torch.float64, pin_memory=True)
        synth.fill(A, 500 + q + 1000 * rank, 0, w["dist"])
        synth.fill(B, 500 + q + 1000 * rank, 1, w["dist"])
        panels.append((A, B, 1.0 if q % 2 == 0 else -0.5))
    C = torch.empty((M, N), dtype=torch.float64, pin_memory=True)
    C0 = torch.empty_like(C, pin_memory=True)
    synth.fill(C0, 500 + 1000 * rank, 2, w["dist"])
    flops = 2.0 * M * N * K
    desc = ("out-of-core C = beta C + sum of %d calls alpha_s A_s B_s (SUMMA-style steps), M=N=%d, K=%d per call, "
            "Ozaki form, beta=%g, N(0,1), device budget %.0f GiB" % (nsteps, M, ks, w["beta"], w["budget"] / 2 ** 30))
    cfg = {"workload": desc, "form": "summa", "M": M, "N": N, "K_per_call": ks, "calls": nsteps,
           "device_budget_bytes": w["budget"],
           "l2": "inputs larger than L2: %.0f GiB of host operands per step" % ((M * N + K * (M + N)) * 8 / 2 ** 30)}
    r = 64
    blocks = sample_blocks(w, 8, r)

    def oracle_blocks():
        import oracle
        out, t0 = [], time.perf_counter()
        for i, j in blocks:
            cur = C0[i:i + r, j:j + r].numpy().astype(np.float64)
            for q, (A, B, alpha) in enumerate(panels):
                b = w["beta"] if q == 0 else 1.0
                cur, _ = oracle.gemm_block("N", "N", i, j, r, r, ks, alpha, A.numpy(), B.numpy(), b, cur,
                                           nthreads=cores)
            out.append(cur)
        return out, time.perf_counter() - t0

    if args.impl == "reference":
        if rank != 0:
            return
        times = []
        for it in range(args.warmup + args.steps):
            _, dt = oracle_blocks()
            if it >= args.warmup:
                times.append(dt)
        value = 2.0 * r * r * K * len(blocks) * len(times) / sum(times) / 1e12
        line = {"impl": "reference", "metric": "out-of-core nsteps GEMM effective TFLOP/s incl. transfers",
                "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Philox)", "config": cfg,
                "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                                 "sample": "%d seeded %dx%d blocks of C through all %d calls" % (
                                     len(blocks), r, r, nsteps)},
                "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    import paper_1808_05056_gb300 as P
    torch.cuda.set_device(local)
    P.load()
    opts = P.make_opts(form=P.OOC_FORM_OZAKI)

    def session_step():
        C.copy_(C0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s = P.Session(M, N, C, N, w["beta"], w["budget"], k_hint=ks, opts=opts)
        if s.rc != 0:
            raise RuntimeError("session: %s" % P.ooc_last_error())
        info = s.query()
        for A, B, alpha in panels:
            if s.step("N", "N", ks, alpha, A, ks, B, N) != 0:
                raise RuntimeError("session step: %s" % P.ooc_last_error())
        st = P.ooc_stats()
        if s.finish(st) != 0:
            raise RuntimeError("session finish: %s" % P.ooc_last_error())
        return time.perf_counter() - t0, st, info

    def plain_step():
        C.copy_(C0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0.0
        for q, (A, B, alpha) in enumerate(panels):
            st = P.ooc_stats()
            rc = P.ooc_dgemm("N", "N", M, N, ks, alpha, A, ks, B, N, w["beta"] if q == 0 else 1.0, C, N,
                             w["budget"], opts, st)
            if rc != 0:
                raise RuntimeError("ooc_dgemm: %s" % P.ooc_last_error())
            h2d += st.h2d_bytes
            d2h += st.d2h_bytes
        return time.perf_counter() - t0, h2d, d2h

    for _ in range(max(0, args.warmup - 1)):
        session_step()
    session_step()
    parity = cpu = None
    if rank == 0:
        ref, dt = oracle_blocks()
        errs = [float(np.linalg.norm(C[i:i + r, j:j + r].numpy() - rv) / np.linalg.norm(rv))
                for (i, j), rv in zip(blocks, ref)]
        parity = {"max_rel_fro": max(errs), "tolerance": FORMS["summa"][1], "blocks": len(blocks), "block": r,
                  "pass": max(errs) <= FORMS["summa"][1]}
        cpu = {"value": 2.0 * r * r * K * len(blocks) / dt / 1e12, "unit": "TFLOP/s", "cores": cores,
               "kind": "oracle", "sample": "%d seeded %dx%d blocks of C through all %d calls, %.1f s" % (
                   len(blocks), r, r, nsteps, dt)}
    clk = ClockSampler(local, enabled=not args.no_clocks)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    runs = [session_step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.stop()
    wall = sum(x[0] for x in runs)
    wall, = max_over_ranks([wall], pg)
    plain_t, plain_h2d, plain_d2h = plain_step()   # comparison, outside the timed region
    if rank != 0:
        return
    _, st, info = runs[0]
    pk, pk_src = peaks()
    value = world * flops * args.steps / wall / 1e12
    peak = pk["bf16_tflops_sustained"]
    line = {
        "metric": "out-of-core nsteps GEMM effective TFLOP/s incl. transfers", "value": value, "unit": "TFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": FORMS["summa"][3],
        "data": "synthetic (seeded Philox, pinned host)", "config": cfg,
        "roofline": {"bound": "tensor", "kernel": "tc_terms_kernel (Ozaki, tcgen05)",
                     "achieved": flops * 36 / (st.kernel_seconds - st.split_seconds) / 1e12, "peak": peak,
                     "unit": "TFLOP/s",
                     "frac": flops * 36 / (st.kernel_seconds - st.split_seconds) / 1e12 / peak, "traffic": None,
                     "peak_source": "%s bf16 sustained (cuBLAS) %.1f TF" % (pk_src, peak)},
        "session": {"resident_blocks": info["resident_blocks"], "blocks": info["blocks"], "mb": info["mb"],
                    "nb": info["nb"], "h2d_bytes": st.h2d_bytes, "d2h_bytes": st.d2h_bytes},
        "without_session": {"value": flops / plain_t / 1e12, "unit": "TFLOP/s", "h2d_bytes": plain_h2d,
                            "d2h_bytes": plain_d2h, "note": "the same %d calls as plain ooc_dgemm" % nsteps},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": st.h2d_bytes,
                "d2h_bytes_per_step": st.d2h_bytes},
        "gpu_launches": st.kernel_launches, "parity": parity, "cpu_baseline": cpu, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_pipe_bench(args, w, world, rank, local, pg):
    """The MMOOC description of the pipeline language, compiled and run by the library, against
    ooc_dgemm forced to the same blocking and rings (one call each per step)."""
    import torch
    M, N, K = w["M"], w["N"], w["K"]
    cores = host_cores()
    A = torch.empty((M, K), dtype=torch.float64, pin_memory=True)
    B = torch.empty((K, N), dtype=torch.float64, pin_memory=True)
    C = torch.empty((M, N), dtype=torch.float64, pin_memory=True)
    for t, s_ in ((A, 0), (B, 1), (C, 2)):
        synth.fill(t, 600 + rank, s_, w["dist"])
    flops = 2.0 * M * N * K
    cfg = config_json(w, "inputs larger than L2: %.0f GiB host operands" % ((M * K + K * N + M * N) * 8 / 2 ** 30))
    cfg["workload"] = "pipeline-language " + cfg["workload"]
    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args, dict(w, form="fp64"), world, rank, pg)
        return
    import paper_1808_05056_gb300 as P
    torch.cuda.set_device(local)
    P.load()
    plan = P.ooc_plan(M, N, K, 8, 1, w["budget"], P.make_opts())
    rings = (plan["depth"], plan["b_buffers"], plan["c_buffers"])
    pipe = P.Pipe(P.MMOOC_PIPELINE)
    for name, v in dict(mb=plan["mb"], nb=plan["nb"], kb=plan["kb"], ra=rings[0], rb=rings[1], rc=rings[2],
                        alpha=w["alpha"], beta=w["beta"], beta_nz=int(w["beta"] != 0.0)).items():
        pipe.set(name, v)
    for name, t in (("A", A), ("B", B), ("C", C)):
        pipe.bind(name, t)
    opts = P.make_opts(mb=plan["mb"], nb=plan["nb"], kb=plan["kb"], depth=rings[0], b_buffers=rings[1],
                       c_buffers=rings[2])

    def step_pipe():
        st = P.ooc_stats()
        t0 = time.perf_counter()
        if pipe.run(w["budget"], st) != 0:
            raise RuntimeError("pipe: %s" % P.ooc_last_error())
        return st, time.perf_counter() - t0

    def step_native():
        st = P.ooc_stats()
        t0 = time.perf_counter()
        if P.ooc_dgemm("N", "N", M, N, K, w["alpha"], A, K, B, N, w["beta"], C, N, w["budget"], opts, st) != 0:
            raise RuntimeError("ooc_dgemm: %s" % P.ooc_last_error())
        return st, time.perf_counter() - t0

    r = 64
    blocks = sample_blocks(w, 8, r)
    for _ in range(max(0, args.warmup - 1)):
        step_pipe()
    cold = [C[i:i + r, j:j + r].numpy().astype(np.float64) for i, j in blocks]
    step_pipe()
    parity = cpu = None
    if rank == 0:
        ref, dt, used = oracle_sample(w, A.numpy(), B.numpy(), cold, blocks, r, cores)
        errs = [float(np.linalg.norm(C[i:i + r, j:j + r].numpy() - rv) / np.linalg.norm(rv))
                for (i, j), rv in zip(blocks, ref)]
        parity = {"max_rel_fro": max(errs), "tolerance": 1e-13, "blocks": len(blocks), "block": r,
                  "pass": max(errs) <= 1e-13}
        cpu = {"value": 2.0 * r * r * K * len(blocks) / dt / 1e12, "unit": "TFLOP/s", "cores": used,
               "kind": "oracle", "sample": "%d seeded %dx%d blocks of C, K=%d, %.1f s" % (len(blocks), r, r, K, dt)}
    probe = fp64_peak(P, local, args.no_clocks)
    clk = ClockSampler(local, enabled=not args.no_clocks)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    runs = [step_pipe() for _ in range(args.steps)]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = clk.stop()
    dev = sum(s_.device_seconds for s_, _ in runs)
    wall = sum(x for _, x in runs)
    dev, wall = max_over_ranks([dev, wall], pg)
    nat = [step_native() for _ in range(max(1, args.steps))]   # comparison, outside the timed region
    if rank != 0:
        return
    s0 = runs[0][0]
    pk, pk_src = peaks()
    achieved = flops * args.steps / sum(s_.kernel_seconds for s_, _ in runs) / 1e12
    roof = {"bound": "tensor", "kernel": "fp64_tile_kernel (FP64 mma.sync, TMA-fed)", "achieved": achieved,
            "unit": "TFLOP/s", "traffic": None}
    roof.update(fp64_roof_fields(pk, pk_src, probe, achieved, (clocks or {}).get("sm_mhz")))
    line = {
        "metric": "out-of-core GEMM effective TFLOP/s incl. transfers (pipeline-language schedule)",
        "value": world * flops * args.steps / dev / 1e12, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dev / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded Philox, pinned host)", "config": cfg,
        "roofline": roof,
        "plan": {"mb": plan["mb"], "nb": plan["nb"], "kb": plan["kb"], "rings": rings},
        "native_same_plan": {"value": flops * len(nat) / sum(s_.device_seconds for s_, _ in nat) / 1e12,
                             "unit": "TFLOP/s", "h2d_bytes": nat[0][0].h2d_bytes, "d2h_bytes": nat[0][0].d2h_bytes},
        "e2e": {"value": world * flops * args.steps / wall / 1e12, "unit": "TFLOP/s",
                "h2d_bytes_per_step": s0.h2d_bytes, "d2h_bytes_per_step": s0.d2h_bytes},
        "gpu_launches": s0.kernel_launches, "parity": parity, "cpu_baseline": cpu, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    w = workload(args)
    world, rank, local, pg = dist_init(args)
    args.gpus = world if world > 1 else args.gpus
    if w["form"] in LEVEL3:
        run_level3_bench(args, w, world, rank, local, pg)
    elif w["form"] == "summa":
        run_summa_bench(args, w, world, rank, local, pg)
    elif w["form"] == "pipe":
        run_pipe_bench(args, w, world, rank, local, pg)
    elif w["form"] == "batched":
        run_batched_bench(args, w, world, rank, local, pg)
    elif args.impl == "reference":
        run_reference(args, w, world, rank, pg)
    else:
        run_ours(args, w, world, rank, local, pg)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
