"""Benchmark of the tensor-train multigroup S_N transport step on GB300.

Workload: the 2-D plane problem -- 128 x 128 cells on [0,1]^2, G = 64 log-spaced groups,
16 polar x 32 azimuthal ordinates (536,870,912 full-grid unknowns), Gaussian-blob density
(8 blobs, contrast 100), kappa_s = 0.1 kappa_a, T linear in x, vacuum boundaries, CFL 0.5,
TT ranks capped at 32, rounding tolerance 1e-6.  One step = transport, round, source,
round (tt_step).  W warm-up steps start from I^0 = epsilon(T); K steps are then timed.

Our arm: CUDA events around each tt_step on the library's stream, L2 flushed (256 MB
write) between timed steps, max over ranks; N > 1 runs independent replicas.
Reference arm (--impl reference): the CPU oracle (naive explicit-sum TT, LAPACK QR+SVD)
on the same workload, on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TT transport steps/s and core-contraction TFLOP/s at fixed tol, FP64 vs mixed"
# Nominal pipe rates (152 SMs at the 2070 MHz maximum SM clock), used only where the in-run probe
# (tt_peak_probe) fails: FP64 FMA 2/clk/SM, FP32 FMA 128/clk/SM, kind::tf32 tensor 1.1 PFLOP/s dense.
NOMINAL_TFLOPS = {"fp64": 152 * 2 * 2 * 2.070e9 / 1e12, "fp32": 152 * 128 * 2 * 2.070e9 / 1e12,
                  "tf32_tensor": 1100.0}
MIXED_LEGS = ("mixed", "mixed_3xtf32")
# DRAM traffic of one launch of the transport-sum TSQR leaf (the dominant kernel), per (precision,
# leaf variant): (bytes read, bytes written, leaves) on the 96 x 96 workload (589,824 rows), from
#   python bench.py --size medium --precision P --start graded --steps 1 --warmup 0 --breakdown-steps 1
#       --tsqr transport=V:L,source=rowsplit:456 --no-gram --no-cpu-baseline --e2e-steps 0 --batch-in-line 0
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none
#       -k regex:"^k_tsqr_leaf$" -c 1 --csv <the same command>
# (first leaf launch = the transport sum of the first step, at full rank).  Reads scale with the rows
# and writes (the leaves' R factors) with the leaves.  Valid only while the leaf kernels' source
# (csrc/bigpass.cuh) is the one captured: its SHA-256 prefix is LEAF_DRAM_SOURCE.
LEAF_DRAM_SOURCE = "2a260ffa11b3c772"
LEAF_DRAM_96 = {("mixed", "column"): (76399616, 28006400, 439),
                ("mixed", "column_dense"): (76594688, 59895296, 595),
                ("fp64", "column"): (201468672, 4627456, 303)}


def leaf_source_sha():
    import hashlib
    path = os.path.join(ROOT, "paper_2602_00290_gb300", "csrc", "bigpass.cuh")
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest()[:16]


def leaf_traffic(precision, variant, leaves, nrows):
    """DRAM bytes of one transport-sum leaf launch at nrows rows and `leaves` leaves, scaled from the
    96 x 96 capture of the same kernel; None when there is none or the kernel source changed since."""
    t = LEAF_DRAM_96.get(("fp64" if precision == "fp64" else "mixed", variant))
    if t is None or LEAF_DRAM_SOURCE is None or leaf_source_sha() != LEAF_DRAM_SOURCE:
        return None
    rd, wr, lm = t
    return rd * nrows / 589824 + wr * leaves / lm
PREC_TEXT = {"fp64": "fp64",
             "mixed": "mixed: f32 passes over the merged core (FP32 FMA), f64 small cores",
             "mixed_3xtf32": "mixed_3xtf32: f32 passes over the merged core, the update GEMM on the tensor cores "
                             "(tcgen05 kind::tf32, split 3xTF32 products, FP32 accumulation), f64 small cores"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="all", choices=["fp64", "mixed", "mixed_3xtf32", "all"])
    ap.add_argument("--size", default="full", choices=["full", "medium", "small"])
    ap.add_argument("--e2e-steps", type=int, default=-1, help="steps of the end-to-end leg (default: --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gram", action="store_true", help="skip the FP64 leg with Gram rounding")
    ap.add_argument("--no-graphs", action="store_true",
                    help="step eagerly instead of replaying the captured step graph")
    ap.add_argument("--breakdown-steps", type=int, default=3,
                    help="instrumented steps (eager, CUDA events per kernel phase) after the timed ones")
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default TSQR kernels instead of the autotuned choice (tt_autotune)")
    ap.add_argument("--tsqr", default="",
                    help="pin the TSQR choice instead of autotuning, e.g. "
                         "'transport=column_dense:608,source=rowsplit:456' (tt_context_set_tsqr)")
    ap.add_argument("--workload", default="plane", choices=["plane", "batched"],
                    help="plane: the 128x128 single-problem step (the headline line); batched: the "
                         "256-problem batch stepped as one CUDA graph (a separate measurement)")
    ap.add_argument("--nprob", type=int, default=256)
    ap.add_argument("--batch-scale", type=int, default=1)
    ap.add_argument("--streams", type=int, default=128)
    ap.add_argument("--start", default="planck", choices=["planck", "graded"],
                    help="initial state: I0 = epsilon(T) (rank 1), or the seeded graded state of rank r_max "
                         "(workloads.graded_state; every pass at full width from the first step, e.g. to profile)")
    ap.add_argument("--batch-in-line", type=int, default=4,
                    help="scale of the batched block of the default line (256 problems, cells and groups "
                         "divided by it; 0 leaves the block out)")
    return ap.parse_args()


def workload(size):
    from paper_2602_00290_gb300.workloads import plane_config1
    if size == "small":
        return plane_config1(nx=32, ny=32, G=16, ntheta=8, nphi=16, rmax=16)
    if size == "medium":  # merged core of 96*96*64 rows x 32: 151 MB in FP64, above the 129 MB L2
        return plane_config1(nx=96, ny=96)
    return plane_config1()


def workload_config(wl, ws=1):
    """The config dict of the JSON line, identical in both arms: the workload, its sizes, and how
    the GPU arm treats the L2 between timed steps (the per-arm precision is under "run")."""
    return {"workload": wl.name, "nx": wl.nx, "ny": wl.ny, "groups": wl.ngroup,
            "ordinates": [wl.ntheta, wl.nphi], "tol": wl.tol, "rmax": wl.rmax,
            "full_grid_unknowns": wl.full_unknowns(), "steps_from": "I0 = epsilon(T)",
            "l2": "GPU arm: flushed between timed steps (256 MB write)",
            "parallelism": "replicas" if ws > 1 else "single"}


def measure_peaks(tt, torch, clocks_index):
    """Peaks of the FP64 and FP32 FMA pipes and of the kind::tf32 tensor pipe on this GPU, each the
    best of 3 probes (tt_peak_probe, CUDA events, about 20-40 ms each), with the SM clock sampled
    while they ran; a failed probe falls back to the nominal rate, named as such."""
    iters = {"fp64": 400_000, "fp32": 4_000_000, "tf32_tensor": 200_000}
    out = {}
    clocks = Clocks(clocks_index)
    for kind, n in iters.items():
        try:
            tt.peak_probe(kind, max(1, n // 50))  # warm: clocks up, module loaded
            best = 0.0
            for _ in range(3):
                flops, ms = tt.peak_probe(kind, n)
                best = max(best, flops / (ms * 1e-3) / 1e12)
            out[kind] = {"tflops": best, "source": "measured"}
        except Exception as e:  # never lose the line over a probe
            out[kind] = {"tflops": NOMINAL_TFLOPS[kind], "source": f"nominal ({e})"}
    clk = clocks.stop()
    out["clocks"] = clk
    out["how"] = ("tt_peak_probe: FP64 / FP32 = 8 independent FMA chains per thread on every SM; tf32_tensor = "
                  "one CTA per SM issuing kind::tf32 MMAs of 128 x 256 x 8 from shared memory; best of 3")
    return out


def counted_flops(N, r_before, r_mid, r_after, nterm=4, nbc=0):
    """Counted core-contraction flops of one step: 2 N (R1^2 + R1 r' + R2^2 + R2 r'') with
    R1 = (n+1) r + n_b (transport sum) and R2 = r' + 1 (source sum)."""
    R1 = (nterm + 1) * r_before + nbc
    R2 = r_mid + 1
    return 2.0 * N * (R1 * R1 + R1 * r_mid + R2 * R2 + R2 * r_after)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        time.sleep(0.1)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_steps_per_s(wl, x_cores, nsteps_max=3, budget_s=20.0):
    """Time the CPU oracle (naive TT step) on the given state; returns (steps/s, steps, seconds,
    the state after the first step, that step's rounding info)."""
    from oracle import naive_tt, problem
    coef = problem.build(wl)
    x = x_cores
    first = None
    info = {}
    t0 = time.perf_counter()
    n = 0
    while n < nsteps_max:
        x = naive_tt.step(x, coef, wl.tol, wl.rmax, info if n == 0 else None)
        if n == 0:
            first = x
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return n / dt, n, dt, first, info


def dense_dof_rate(wl_full, n=32, reps=5):
    """DOF-updates/s of the dense FP64 oracle stepper (OpenMP) on an n x n sample of the workload's
    per-cell structure (same groups and ordinates), the rate the paper quotes for a traditional
    S_N solver (Sec. 3.2, 'speedup'); returns (rate, unknowns of the sample, threads, seconds)."""
    from oracle import dense
    from paper_2602_00290_gb300.workloads import plane_config1
    wl = plane_config1(nx=n, ny=n, G=wl_full.ngroup, ntheta=wl_full.ntheta, nphi=wl_full.nphi,
                       rmax=wl_full.rmax, tol=wl_full.tol)
    S = dense.DenseSolver(wl)
    I = S.initial()
    I = S.step(I)  # warm (page-in, thread start-up)
    t0 = time.perf_counter()
    for _ in range(reps):
        I = S.step(I)
    dt = time.perf_counter() - t0
    unknowns = wl.full_unknowns()
    return reps * unknowns / dt, unknowns, dense.DenseSolver.threads(), dt


def max_over_ranks(x, dist, device):
    """The largest x over all ranks (the job's time is its slowest rank's); x itself alone."""
    if not dist:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import naive_tt, problem
    wl = workload(args.size)
    coef = problem.build(wl)
    x = naive_tt.initial_tt(problem.initial_rows(wl, coef), coef)
    for _ in range(args.warmup):
        x = naive_tt.step(x, coef, wl.tol, wl.rmax)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x = naive_tt.step(x, coef, wl.tol, wl.rmax)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, args.gpus),
            "run": {"precision": "fp64 (the oracle: naive explicit-sum TT, LAPACK QR + SVD, host cores)"},
            "cpu_baseline": {"kind": "oracle", "value": v, "unit": "steps/s", "cores": host_cores(),
                             "sample": f"{args.steps} naive explicit-sum TT steps (LAPACK QR + SVD) after "
                                       f"{args.warmup} warm-up steps from I0"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "ranks": naive_tt.ranks(x)}
    print(json.dumps(line), flush=True)
    return 0


def time_precision(tt, torch, ctx, plan, wl, args, precision, dist, clocks_index, peaks, rounding="tsqr"):
    """W warm-up then K timed tt_step calls for one precision; returns (line fields, state)."""
    ctx.set_rounding(rounding)
    dtype = "f64" if precision == "fp64" else "f32"
    rcap = [wl.rmax, wl.rmax]
    if args.start == "graded":
        from paper_2602_00290_gb300.workloads import graded_state
        x = tt.TT.from_cores(graded_state(wl), rcap=rcap, dtype=dtype)
    else:
        x = tt.initial_state(plan, rcap, dtype)
    stream = ctx.stream
    energy = torch.zeros(4, dtype=torch.float64, device="cuda")
    pinned = None
    if rounding == "tsqr" and args.tsqr:
        # pinned choice (e.g. the autotuner's, to profile the same kernels without timing
        # trials), in force from the first warm-up step on
        ncaps = {"transport": (2 * wl.ndim + 1) * wl.rmax, "source": wl.rmax + 1}
        pinned = {}
        for item in args.tsqr.split(","):
            role, spec = item.split("=")
            variant, leaves = spec.split(":")
            ctx.set_tsqr(precision, ncaps[role], variant, int(leaves))
            pinned[role] = ctx.get_tsqr(precision, ncaps[role])
        pinned["pinned"] = True
    ctx.set_graphs(not args.no_graphs)
    for _ in range(args.warmup):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, precision, energy)
    ctx.sync()
    tune = pinned
    if tune is None and rounding == "tsqr" and not args.no_autotune:
        # TSQR kernels and leaf counts for this state's shape, timed on a copy of it
        tune = ctx.autotune(plan, x, wl.tol, wl.rmax, precision, steps=2)
    # two more untimed steps in every leg (the legs' states stay step for step comparable): the
    # first with the kernels in force runs eagerly, the second captures its step graph, so that
    # every timed step is a replay
    for _ in range(2):
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, precision, energy)
    ctx.sync()
    ranks = [x.ranks()]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    clocks = Clocks(clocks_index)
    ctx.counters(reset=True)
    ctx.diagnostics(reset=True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    rank_hist = torch.zeros(args.steps, 4, dtype=torch.int32, device="cuda")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        evs[i][0].record(stream)
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, precision, energy)
        evs[i][1].record(stream)
        rank_hist[i].copy_(x.rank)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ctx.sync()
    _, klaunch = ctx.counters(reset=True)
    diag = ctx.diagnostics(reset=True)
    clk = clocks.stop()
    # per-phase kernel times: a few more steps, eager, with CUDA events around each kernel phase
    # (the timed steps above replay the step graph, which carries no per-phase events)
    nb = max(1, args.breakdown_steps)
    b_ranks = [x.ranks()]
    ctx.set_timing(True)
    for _ in range(nb):
        flush.zero_()
        tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, precision, energy)
        b_ranks.append(x.ranks())
    ctx.sync()
    ctx.set_timing(False)
    kms, _ = ctx.counters(reset=True)
    ctx.diagnostics(reset=True)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    hist = rank_hist.cpu().numpy()
    r_seq = [ranks[0]] + [list(map(int, h)) for h in hist]
    N = wl.nrow
    flops = 0.0
    leaf_flops = 0.0
    for i in range(args.steps):
        rb, ra = r_seq[i][1], r_seq[i + 1][1]
        flops += counted_flops(N, rb, ra, ra)
    for i in range(nb):
        R1 = 5 * b_ranks[i][1]  # transport-sum columns (Z and its 4 upwind images; vacuum: no inflow columns)
        leaf_flops += 2.0 * N * R1 * R1
    ws = dist.get_world_size() if dist else 1
    out = {"value": ws * args.steps / (total_ms / 1e3), "ms_per_step": total_ms / args.steps,
           "tflops": flops / (total_ms / 1e3) / 1e12,
           "breakdown_ms_per_step": {k: v / nb for k, v in kms.items()},
           "breakdown_steps": nb, "step_graphs": not args.no_graphs,
           "gpu_launches": int(sum(klaunch.values())), "clocks": clk, "ranks": r_seq[-1],
           "rank_history": [r[1:-1] for r in r_seq], "jacobi": diag}
    if tune is not None:
        out["tsqr_autotune"] = tune
    leaf_tf = leaf_flops / (kms["tsqr_leaf"] / 1e3) / 1e12 if kms["tsqr_leaf"] > 0 else None
    pk = peaks["fp64" if precision == "fp64" else "fp32"]
    peak = pk["tflops"]
    variant = tune["transport"][0] if tune is not None else "column"
    kname = {"column": "k_tsqr_leaf", "rowsplit": "k_tsqr_leaf_rs",
             "column_dense": "k_tsqr_leaf (32-row blocks, 4 CTAs/SM)"}[variant]
    out["roofline"] = {"kernel": kname + " over the transport sum (one launch per step, R1 = 5r columns)",
                       "bound": "alu", "achieved": leaf_tf, "peak": peak, "unit": "TFLOP/s",
                       "frac": (leaf_tf / peak) if leaf_tf else None,
                       "traffic": leaf_traffic(precision, variant, int(tune["transport"][1]) if tune else 0, wl.nrow),
                       "traffic_note": ("ncu DRAM bytes (read + written) of this leaf kernel on the 96 x 96 workload, "
                                        "reads scaled by rows and writes by leaves; null when no capture of the kernel "
                                        "source as it stands is recorded"),
                       "flops_per_launch": "2 N_Z R1^2 (R1 = 5 r, r the rank entering the step)",
                       "peak_source": ("FP64" if precision == "fp64" else "FP32") + " FMA pipe, " + pk["source"] +
                                      " in this run (tt_peak_probe)",
                       "share": (kms["tsqr_leaf"] / nb) / (total_ms / args.steps) if total_ms else None}
    # the first update pass (Z_new = Z_sum W over the transport sum, K = R1, N = r'): on the tensor
    # cores in the 3xTF32 leg (three kind::tf32 MMAs per product), FP32 FMA otherwise
    up_flops = 0.0
    for i in range(nb):
        up_flops += 2.0 * N * (5 * b_ranks[i][1]) * b_ranks[i + 1][1]
    if kms["update"] > 0:
        up_alg = up_flops / (kms["update"] / 1e3) / 1e12
        if precision == "mixed_3xtf32":
            tp = peaks["tf32_tensor"]
            out["roofline_update"] = {
                "kernel": "k_update_tc (tcgen05 kind::tf32, 3xTF32, 128-row tiles, one CTA per SM)",
                "bound": "tensor", "achieved": 3.0 * up_alg, "peak": tp["tflops"], "unit": "TFLOP/s",
                "frac": 3.0 * up_alg / tp["tflops"], "algorithmic_tflops": up_alg,
                "flops_per_launch": "3 x 2 N_Z R1 r' tensor-pipe flops (three TF32 products per FP32 product)",
                "peak_source": "kind::tf32 tensor pipe, " + tp["source"] + " in this run (tt_peak_probe)",
                "ms_per_launch": kms["update"] / nb}
        else:
            out["roofline_update"] = {
                "kernel": ("k_update (FP64)" if precision == "fp64" else "k_update_blk (FP32 FMA)"),
                "bound": "alu", "achieved": up_alg, "peak": peak, "unit": "TFLOP/s", "frac": up_alg / peak,
                "flops_per_launch": "2 N_Z R1 r'", "ms_per_launch": kms["update"] / nb}
    ctx.set_rounding("tsqr")
    return out, x, energy


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    from paper_2602_00290_gb300 import _build
    _build.build()
    import paper_2602_00290_gb300 as tt

    wl = workload(args.size)
    ctx = tt.Context()
    plan = tt.Plan(ctx, wl)
    vis = (os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local]
           if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local))
    peaks = measure_peaks(tt, torch, vis)
    precs = ["fp64", "mixed", "mixed_3xtf32"] if args.precision == "all" else [args.precision]
    results, states = {}, {}
    for prec in precs:
        results[prec], states[prec], energy = time_precision(tt, torch, ctx, plan, wl, args, prec, dist, vis, peaks)
    if "fp64" in precs and not args.no_gram:
        results["fp64_gram"], states["fp64_gram"], _ = time_precision(tt, torch, ctx, plan, wl, args, "fp64", dist,
                                                                      vis, peaks, rounding="gram")
        # randomized rounding: Gaussian sketch of r_max + 8 columns (seeded)
        from paper_2602_00290_gb300.workloads import sketch_matrix
        ctx.set_sketch(sketch_matrix(wl.ntheta * wl.nphi, wl.rmax + 8, seed=11))
        results["fp64_randomized"], states["fp64_randomized"], _ = time_precision(
            tt, torch, ctx, plan, wl, args, "fp64", dist, vis, peaks, rounding="randomized")
    # headline: the faster mixed leg (the precision is named in config), else FP64
    mixed_done = [p for p in MIXED_LEGS if p in results]
    head = max(mixed_done, key=lambda p: results[p]["value"]) if mixed_done else "fp64"
    R = results[head]
    x = states[head]
    line = {"metric": METRIC, "value": R["value"], "unit": "steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": R["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if head != "fp64" else "f64",
            "data": "synthetic",
            "config": workload_config(wl, ws),
            "run": {"precision": PREC_TEXT[head], "state_dtype": "f32" if head != "fp64" else "f64",
                    "step": ("replay of the captured step graph" if R["step_graphs"] else "eager launches")},
            "tflops": R["tflops"], "roofline": R["roofline"], "roofline_update": R.get("roofline_update"),
            "peaks_measured": peaks,
            "breakdown_ms_per_step": R["breakdown_ms_per_step"], "breakdown_steps": R["breakdown_steps"],
            "gpu_launches": R["gpu_launches"], "clocks": R["clocks"], "ranks": R["ranks"], "rank_history": R["rank_history"],
            "jacobi": R["jacobi"]}
    if "tsqr_autotune" in R:
        line["tsqr_autotune"] = R["tsqr_autotune"]
    keys = ("value", "ms_per_step", "tflops", "roofline", "roofline_update", "breakdown_ms_per_step",
            "gpu_launches", "ranks", "jacobi", "tsqr_autotune")
    for p in ("fp64",) + MIXED_LEGS:
        if p in results and p != head:
            line[p] = {k: results[p][k] for k in keys if k in results[p]}
    if "fp64" in results and head != "fp64":
        F = results["fp64"]
        line["speedup_mixed_over_fp64"] = R["value"] / F["value"]
        Ed = tt.tt_energy_density(ctx, plan, states["fp64"]).cpu().numpy()
        for p in mixed_done:
            Em = tt.tt_energy_density(ctx, plan, states[p]).cpu().numpy()
            line[f"{p}_vs_fp64_energy_density_rel_err"] = float(np.linalg.norm(Em - Ed) / np.linalg.norm(Ed))
    if "fp64_gram" in results:
        G = results["fp64_gram"]
        line["fp64_gram"] = {k: G[k] for k in ("value", "ms_per_step", "tflops", "breakdown_ms_per_step",
                                               "gpu_launches", "ranks", "jacobi")}
        # the Gram pass over the transport sum (symmetric: N R1 (R1 + 1) flops at R1 = 5r)
        rh = G["rank_history"]
        gflops = sum(2.0 * wl.nrow * (5 * r[0]) * (5 * r[0] + 1) / 2.0 for r in rh[:-1])
        gms = G["breakdown_ms_per_step"]["tsqr_leaf"] * args.steps
        ach = gflops / (gms / 1e3) / 1e12 if gms > 0 else None
        line["fp64_gram"]["roofline"] = {
            "kernel": "k_gram_tiles + k_gram_reduce over the transport sum (FP64 Gram, upper triangle)",
            "bound": "alu", "achieved": ach, "peak": peaks["fp64"]["tflops"], "unit": "TFLOP/s",
            "frac": ach / peaks["fp64"]["tflops"] if ach else None,
            "peak_source": "FP64 FMA pipe, " + peaks["fp64"]["source"] + " in this run (tt_peak_probe)"}
        Eg = tt.tt_energy_density(ctx, plan, states["fp64_gram"]).cpu().numpy()
        Ed = tt.tt_energy_density(ctx, plan, states["fp64"]).cpu().numpy()
        line["fp64_gram"]["energy_density_rel_err_vs_tsqr"] = float(np.linalg.norm(Eg - Ed) / np.linalg.norm(Ed))
    if "fp64_randomized" in results:
        Rr = results["fp64_randomized"]
        line["fp64_randomized"] = {k: Rr[k] for k in ("value", "ms_per_step", "tflops", "breakdown_ms_per_step",
                                                      "gpu_launches", "ranks")}
        line["fp64_randomized"]["sketch_columns"] = wl.rmax + 8
        Er = tt.tt_energy_density(ctx, plan, states["fp64_randomized"]).cpu().numpy()
        Ed = tt.tt_energy_density(ctx, plan, states["fp64"]).cpu().numpy()
        line["fp64_randomized"]["energy_density_rel_err_vs_tsqr"] = float(np.linalg.norm(Er - Ed) / np.linalg.norm(Ed))
    # internal structure of the final state's merged core (Sec. 5.2): delta-ranks at the rounding
    # tolerance and the compression ratios of Eqs. (compression), (rel_compression_nu/_x)
    try:
        t0 = time.time()
        r1, r1x, _, _, ir_st = tt.tt_internal_ranks(ctx, plan, x, wl.tol, with_status=True)
        ir_status = ("ok" if ir_st == tt.TT_OK else
                     "a Jacobi solve reached its sweep cap (TT_ERR_TIMEOUT): ranks of its last sweep")
        r2, r3 = x.ranks()[1], x.ranks()[2]
        nX, nnu, nth, nph = wl.nx * wl.ny * wl.nz, wl.ngroup, wl.ntheta, wl.nphi
        ntt = nX * nnu * r2 + nth * r2 * r3 + nph * r3
        line["internal_ranks"] = {
            "delta": wl.tol, "r1_nu": r1, "r1_x": r1x, "tt_ranks": [r2, r3],
            "compression": nX * nnu * nth * nph / ntt,
            "compression_rel_nu": ntt / (nnu * r1 + nX * r1 * r2 + nth * r2 * r3 + nph * r3),
            "compression_rel_x": ntt / (nX * r1x + nnu * r1x * r2 + nth * r2 * r3 + nph * r3),
            "seconds": time.time() - t0, "status": ir_status}
    except Exception as e:  # the analysis is a report, not part of the timed step
        line["internal_ranks"] = {"error": str(e)}
    # the batched workload (independent problems of uneven shape, one CUDA graph per batch step),
    # at a stated reduced scale so that the default run stays within minutes
    if args.batch_in_line > 0 and rank == 0:
        try:
            line["batched"] = batched_block(tt, torch, ctx, args, 256, args.batch_in_line, "mixed")
        except Exception as e:  # a second measurement, never a reason to lose the line
            line["batched"] = {"error": str(e)}
    # storage factor k_s (App. A, 'Compression'): peak device storage of a step (the state at its
    # rank capacities plus the step's workspace) over the bytes of the rounded TT it leaves
    try:
        ks = {}
        for p in results:
            if p not in ("fp64",) + MIXED_LEGS:
                continue
            st = states[p]
            esz = 8 if st.dtype == "f64" else 4
            r = st.ranks()
            live = esz * (wl.nrow * r[1] + r[1] * wl.ntheta * r[2] + r[2] * wl.nphi)
            cap = sum(c.numel() * c.element_size() for c in st.cores)
            wsb = tt.tt_workspace_query(ctx, plan, st, p)
            ks[p] = {"k_s": (cap + wsb) / live, "workspace_bytes": wsb, "state_capacity_bytes": cap,
                     "rounded_tt_bytes": live}
        line["storage_factor"] = ks
    except Exception as e:  # a report, never a reason to lose the line
        line["storage_factor"] = {"error": str(e)}
    # end-to-end through the C ABI with host buffers (pinned), copies inside the timed region
    e2e_steps = args.steps if args.e2e_steps < 0 else args.e2e_steps
    if e2e_steps > 0:
        stream = ctx.stream
        energy = torch.zeros(4, dtype=torch.float64, device="cuda")
        host = [c.cpu().pin_memory() for c in x.cores]
        host_rank = x.rank.cpu().pin_memory()
        host_energy = torch.zeros(4, dtype=torch.float64).pin_memory()
        h2d = sum(c.numel() * c.element_size() for c in host) + host_rank.numel() * 4
        d2h = h2d + host_energy.numel() * 8
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        # untimed: an eager step and the capture of the step graph for this energy buffer (each
        # timed step starts from the host copy of the state)
        for _ in range(2):
            tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, head, energy)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(e2e_steps):
            with torch.cuda.stream(stream):
                for c, h in zip(x.cores, host):
                    c.copy_(h, non_blocking=True)
                x.rank.copy_(host_rank, non_blocking=True)
            tt.tt_step(ctx, plan, x, wl.tol, wl.rmax, head, energy)
            with torch.cuda.stream(stream):
                for c, h in zip(x.cores, host):
                    h.copy_(c, non_blocking=True)
                host_rank.copy_(x.rank, non_blocking=True)
                host_energy.copy_(energy, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = e0.elapsed_time(e1)
        try:
            ctx.sync()
            e2e_status = "ok"
        except tt.TTError as e:
            e2e_status = str(e)
        line["e2e"] = {"value": ws * e2e_steps / (e2e_ms / 1e3), "unit": "steps/s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "steps": e2e_steps, "precision": head, "status": e2e_status}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        start = states["fp64"] if "fp64" in states else x
        cores = start.to_cores()
        v, n, dt, first, info = oracle_steps_per_s(wl, cores)
        line["cpu_baseline"] = {"value": v, "unit": "steps/s", "cores": host_cores(), "kind": "oracle",
                                "sample": f"{n} naive explicit-sum TT step(s) (numpy, LAPACK QR + SVD) of the "
                                          f"same workload from the GPU state after the timed steps ({dt:.1f} s)"}
        # the error of every leg against the FP64 oracle: one step of each precision from the same
        # state as the oracle's first timed step
        try:
            from oracle import naive_tt, problem
            coef = problem.build(wl)
            Eref = naive_tt.energy_density_rows(first, coef)
            errs, ranks_eq = {}, {}
            for p in ("fp64",) + MIXED_LEGS:
                if p not in results:
                    continue
                y = tt.TT.from_cores(cores, rcap=[wl.rmax, wl.rmax], dtype="f64" if p == "fp64" else "f32")
                tt.tt_step(ctx, plan, y, wl.tol, wl.rmax, p)
                ctx.sync()
                E = tt.tt_energy_density(ctx, plan, y).cpu().numpy()
                errs[p] = float(np.linalg.norm(E - Eref) / np.linalg.norm(Eref))
                ranks_eq[p] = y.ranks() == naive_tt.ranks(first)
            gaps = [b["gap"] for k in ("transport_round", "source_round") for b in info[k]["bonds"]]
            line["error_vs_oracle"] = {
                "energy_density_rel_err": errs, "ranks_equal": ranks_eq, "oracle_min_rank_gap": min(gaps),
                "how": ("one tt_step of each precision and one oracle step from the same FP64 state (the FP64 "
                        "leg's after its timed steps): ||E - E_oracle||_F / ||E_oracle||_F over every merged row")}
            line["mixed_vs_oracle_energy_density_rel_err"] = errs.get(head)
        except Exception as e:  # a report beside the baseline, never a reason to lose the line
            line["error_vs_oracle"] = {"error": str(e)}
        # the paper's speedup S = t_dense / t_TT (Sec. 3.2), against the dense oracle's rate on
        # this host (the paper quotes 3.6-5.0e8 DOF-updates/s on its M3 Ultra; context only)
        try:
            rate, nu, thr, ddt = dense_dof_rate(wl)
            t_dense = wl.full_unknowns() / rate
            line["cpu_baseline"]["dense_oracle"] = {
                "dof_updates_per_s": rate, "threads": thr,
                "sample": f"5 dense FP64 steps of a 32x32-cell, {wl.ngroup}-group, {wl.ntheta}x{wl.nphi}-ordinate "
                          f"grid ({nu} unknowns, {ddt:.1f} s)",
                "dense_step_s_at_workload": t_dense,
                "speedup_tt_gpu_over_dense": t_dense / (line["ms_per_step"] / 1e3)}
        except Exception as e:  # a report beside the baseline, never a reason to lose the line
            line["cpu_baseline"]["dense_oracle"] = {"error": str(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def batched_block(tt, torch, ctx, args, nprob, scale, prec):
    """Problem steps/s of the batched workload (batch_config3, seed 3) through tt_batch_step."""
    from paper_2602_00290_gb300.workloads import batch_config3
    wls = batch_config3(nprob, seed=3, scale=scale)
    plans = [tt.Plan(ctx, wl) for wl in wls]
    dtype = "f64" if prec == "fp64" else "f32"
    states = [tt.initial_state(p, [w.rmax, w.rmax], dtype) for p, w in zip(plans, wls)]
    b = tt.Batch(ctx, plans, states, [w.tol for w in wls], [w.rmax for w in wls], prec, args.streams)
    b.step(3)  # eager step, capture, replay
    b.sync()
    steps = max(3, args.steps // 2)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    b.step(steps)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    st = b.sync()
    ms = e0.elapsed_time(e1)
    info = b.info()
    out = {"problems": len(wls), "scale": scale, "precision": prec, "steps": steps,
           "rows": sum(w.nrow for w in wls), "full_grid_unknowns": sum(w.nrow * w.ntheta * w.nphi for w in wls),
           "batch_steps_per_s": steps / (ms / 1e3), "problem_steps_per_s": len(wls) * steps / (ms / 1e3),
           "ms_per_batch_step": ms / steps, "gpu_launches_per_batch_step": info["launches_per_step"],
           "workspace_gb": info["workspace_bytes"] / 1e9, "all_statuses_ok": all(v == 0 for v in st),
           "workload": ("batch_config3(seed 3): Nx = Ny in {32..192}, G in {16..96}, 8x16..16x32 ordinates, "
                        "r_max 8..48, x- inflow; cells, groups divided by `scale`, ordinates halved")}
    b.close()
    for p in plans:
        p.close()
    del states
    torch.cuda.empty_cache()
    return out


def run_batched(args):
    """Independent problems of uneven shape (Nx = Ny in 32..192, G in 16..96, 8x16..16x32
    ordinates, r_max 8..48, x- inflow) stepped together through tt_batch_step (one CUDA graph per
    step); reports batch steps/s and problem steps/s for the chosen precision(s)."""
    import torch
    torch.cuda.set_device(0)
    from paper_2602_00290_gb300 import _build
    _build.build()
    import paper_2602_00290_gb300 as tt
    from paper_2602_00290_gb300.workloads import batch_config3

    wls = batch_config3(args.nprob, seed=3, scale=args.batch_scale)
    ctx = tt.Context()
    plans = [tt.Plan(ctx, wl) for wl in wls]
    rows = sum(w.nrow for w in wls)
    unknowns = sum(w.nrow * w.ntheta * w.nphi for w in wls)
    # "all" (the default of the single-problem line) runs the three precision levels here too
    precs = ["fp64", "mixed", "mixed_3xtf32"] if args.precision == "all" else [args.precision]
    out = {"metric": "batched TT transport steps/s", "unit": "batch steps/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
           "config": {"workload": f"batch of {len(wls)} independent 2-D problems", "seed": 3,
                      "scale": args.batch_scale, "rows": rows, "full_grid_unknowns": unknowns,
                      "streams": args.streams}}
    for prec in precs:
        dtype = "f64" if prec == "fp64" else "f32"
        states = [tt.initial_state(p, [w.rmax, w.rmax], dtype) for p, w in zip(plans, wls)]
        b = tt.Batch(ctx, plans, states, [w.tol for w in wls], [w.rmax for w in wls], prec, args.streams)
        b.step(max(args.warmup, 1))
        b.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(ctx.stream)
        b.step(args.steps)
        e1.record(ctx.stream)
        torch.cuda.synchronize()
        b.sync()
        ms = e0.elapsed_time(e1)
        info = b.info()
        ranks = [s.ranks()[1:-1] for s in states]
        out[prec] = {"value": args.steps / (ms / 1e3), "ms_per_step": ms / args.steps,
                     "problem_steps_per_s": len(wls) * args.steps / (ms / 1e3),
                     "gpu_launches_per_step": info["launches_per_step"],
                     "workspace_gb": info["workspace_bytes"] / 1e9,
                     "state_gb": sum(c.numel() * c.element_size() for s in states for c in s.cores) / 1e9,
                     "mean_rank": float(sum(r[0] for r in ranks)) / len(ranks)}
        b.close()
        del states
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
