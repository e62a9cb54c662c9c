"""Benchmark: Nystrom PCG solves/sec on the matrix-free ridge workload.

Workload (one "step" = one complete solve, every stage of the hot path):
  X: m = 200000 x n = 4096 FP32, X_ij ~ N(0,1) / (j+1); A = X^T X applied as
  X^T (X v); mu = 1e-3; b = X^T y, y ~ N(0,1); Nystrom sketch with ell = 512
  (Algorithm 1, mixed precision); PCG (Algorithm 3) on FP32 vectors inside
  FP64-residual iterative refinement to ||b - (A + mu I) x|| <= 1e-8 ||b||.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` = solves/sec over all ranks with the
inputs resident in HBM; `e2e` = the same through the C ABI with host inputs
(pinned host -> device copy of X and b, and the solution back, inside the
timed region); `roofline` = the fused ridge matvec kernel (HBM bound)
against the measured copy bandwidth; `cpu_baseline` = the FP64 oracle on a
bounded row sample of the same workload.  X (3.3 GB) is larger than L2, so
no flush is needed between steps.  Under torchrun every rank solves its own
replica (the path has no exchange step); timing is the max over ranks.
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

# the oracle's BLAS runs on exactly the cores this process may use (the
# thread count the CPU baseline reports), unless the caller pinned it
_CORES = len(os.sched_getaffinity(0))
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, str(_CORES))

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N, ELL, MU, TOL = 200_000, 4096, 512, 1e-3, 1e-8
RATED_HBM_GBS = 7900.0  # GB300 HBM3e, rated
INNER_TOL = 1e-4
SEED = 0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--m", type=int, default=M)
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--ell", type=int, default=ELL)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the dense, kernel-ridge, regularisation-path and adjoint "
                         "records that follow the headline")
    ap.add_argument("--solve-only", action="store_true",
                    help="time the solves only (no matvec, launch-count, e2e or CPU legs); "
                         "used for profiler launch lists")
    ap.add_argument("--workload", default="ridge",
                    choices=["ridge", "dense", "krr", "batched", "adjoint", "block", "path"],
                    help="ridge (default): the headline line; the others measure the remaining "
                         "workloads of the hot path (dense FP64; adaptive mixed kernel ridge; "
                         "batched regularisation path; differentiable kernel ridge)")
    ap.add_argument("--matvec-only", action="store_true",
                    help="run only the workload's dominant FP32 matvec (--steps times after "
                         "--warmup); the command behind the ncu summaries in profiles/")
    ap.add_argument("--sketch", default="gaussian", choices=["gaussian", "columns"],
                    help="krr workload: adaptive Gaussian sketch (default) or column-sampling "
                         "Nystrom at --cols sampled points")
    ap.add_argument("--cols", type=int, default=1024)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "f64"],
                    help="krr / batched / adjoint workloads: mixed (FP32 inner solves, FP64-accurate "
                         "residual refinement; the default) or plain FP64 PCG, for comparison")
    ap.add_argument("--pcg-launch", default="graph", choices=["graph", "stream"],
                    help="PCG iterations replayed from a captured CUDA graph (default) or "
                         "launched kernel by kernel on the stream")
    ap.add_argument("--nrhs", type=int, default=4,
                    help="block workload: right-hand sides of the one shifted system")
    ap.add_argument("--block-ell", type=int, default=1024,
                    help="block workload: sketch size of the preconditioner")
    ap.add_argument("--matvec-mode", type=int, default=1, choices=[1, 2],
                    help="--matvec-only: 1 the FP32 product, 2 the FP64-accurate residual "
                         "product (double-FP32 for the ridge and Gaussian operators)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="non-default workloads: multiply the number of points by this factor")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed

def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device="cuda"):
    """Largest value over the ranks (the slowest replica's time); `device` is
    "cuda" under NCCL, "cpu" under gloo."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms_per_step_max, world):
    """Whole-job solves/s for replicas: every rank completes one solve per
    step, and the job's step time is the slowest rank's."""
    return world * 1e3 / ms_per_step_max


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

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
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

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
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if p[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- workload

def make_inputs(m, n):
    from paper_2110_02820_gb300 import workloads as wl
    X = wl.ridge_X(m, n, SEED)
    y = wl.ridge_y(m, SEED)
    return X, y


def rhs_on_device(Xd, y):
    """b = X^T y in FP64 (input preparation, chunked)."""
    import torch
    yd = torch.tensor(y, device=Xd.device)
    b = torch.zeros(Xd.shape[1], dtype=torch.float64, device=Xd.device)
    for r0 in range(0, Xd.shape[0], 16384):
        b += Xd[r0:r0 + 16384].double().t() @ yd[r0:r0 + 16384]
    return b


def solve_once(ny, op, b, ell, seed):
    f = ny.nys_sketch(op, ell, seed=seed, precision=ny.NYS_PREC_MIXED)
    x, res, _ = ny.pcg_solve(op, f, MU, b, tol=TOL, precision=ny.NYS_PREC_MIXED,
                             inner_tol=INNER_TOL, maxit=500, max_refine=20)
    f.free()
    return x, res[0]


def phase_times(ny, op, b, ell, reps=2):
    """Average ms of the sketch (Algorithm 1) and of the refined PCG solve."""
    import torch
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    sk, so = [], []
    for r in range(reps):
        e[0].record()
        f = ny.nys_sketch(op, ell, seed=500 + r, precision=ny.NYS_PREC_MIXED)
        e[1].record()
        ny.pcg_solve(op, f, MU, b, tol=TOL, precision=ny.NYS_PREC_MIXED, inner_tol=INNER_TOL)
        e[2].record()
        torch.cuda.synchronize()
        sk.append(e[0].elapsed_time(e[1]))
        so.append(e[1].elapsed_time(e[2]))
        f.free()
    return {"sketch_ms": statistics.mean(sk), "pcg_ms": statistics.mean(so)}


# ---------------------------------------------------------------- CPU baseline (oracle)

def cpu_baseline(m, n, ell, sample_rows):
    """The FP64 oracle (Algorithm 1 + Algorithm 3 in numpy) on a row sample
    of the workload; cost is linear in the number of rows, so solves/sec at
    full size = 1 / (t_sample * m / sample_rows)."""
    from oracle import nystrom as onys
    from oracle import operators as oops
    from oracle import pcg as opcg
    from paper_2110_02820_gb300 import workloads as wl
    cores = int(os.environ.get("OPENBLAS_NUM_THREADS", len(os.sched_getaffinity(0))))
    Xs = wl.ridge_X(sample_rows, n, SEED + 1)
    ys = wl.ridge_y(sample_rows, SEED + 1)
    X64 = Xs.astype(np.float64)
    b = X64.T @ ys
    Om = wl.omega(n, ell, SEED)
    t0 = time.perf_counter()
    f = onys.rand_nystrom(lambda V: X64.T @ (X64 @ V), Om)
    out = opcg.nys_pcg(lambda v: X64.T @ (X64 @ v), MU, b, None,
                       lambda r: onys.precond_inverse_apply(f["U"], f["lam"], MU, r), TOL, 500)
    t = time.perf_counter() - t0
    t_full = t * m / sample_rows
    return {"value": 1.0 / t_full, "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample_fraction": sample_rows / m, "sample_s": t, "full_solve_s_extrapolated": t_full,
            "sample": f"rows {sample_rows} of {m} (n={n}, ell={ell}), FP64 numpy Algorithm 1 + "
                      f"Algorithm 3 to rel. residual {TOL}: {t:.2f} s, {out['iterations']} "
                      f"iterations; scaled linearly in rows"}


# ---------------------------------------------------------------- arms

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    rows = max(2000, args.m // 4)
    for _ in range(args.warmup):  # untimed
        cpu_baseline(args.m, args.n, args.ell, rows)
    vals = []
    t0 = time.perf_counter()
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(args.m, args.n, args.ell, rows)
        vals.append(1.0 / cb["value"])
    dt = time.perf_counter() - t0
    v = 1.0 / statistics.mean(vals)
    line = {"metric": "PCG solves/sec to rel-residual 1e-8 and kernel-matvec TFLOP/s vs roofline, 1xGB300",
            "impl": "reference", "value": v, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"ridge X {args.m}x{args.n} fp32, ell={args.ell}, mu={MU}, tol={TOL}",
                       "parallelism": "replicas"},
            "cpu_baseline": cb,
            # a step is one solve of a row sample (ms_per_step, what the clock around
            # the run sees); value is solves/s of the full workload, the sample time
            # scaled by m / rows (the oracle's cost is linear in the rows)
            "step": {"kind": "row sample", "rows": rows, "of_rows": args.m,
                     "ms_per_full_solve_extrapolated": 1e3 / v},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def e2e_ridge(ny, torch, X, Xd, b, n, ell, args, world):
    """End-to-end ridge solves through the public API with host inputs: every
    step copies X (3.28 GB) and b from pinned host memory and reads x back.
    Pipelined (the `value`): two device copies of the inputs; while step k
    solves, step k+1's inputs are copied on a second stream (copy engines;
    the copy takes ~1 % of HBM bandwidth), so a step costs max(copy, solve).
    Serial (`serial`): copy, solve, read back, one after the other."""
    Xh = torch.from_numpy(X).pin_memory()
    bh = b.cpu().pin_memory()
    xh = torch.empty(n, dtype=torch.float64).pin_memory()
    Xb = [torch.empty_like(Xd), torch.empty_like(Xd)]
    bb = [torch.empty_like(b), torch.empty_like(b)]
    ops = [ny.gram_operator(Xb[0]), ny.gram_operator(Xb[1])]
    cs = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    free = [torch.cuda.Event(), torch.cuda.Event()]
    main = torch.cuda.current_stream()

    def copy_in(i):
        with torch.cuda.stream(cs):
            cs.wait_event(free[i])          # the solve that last read buffer i is done
            Xb[i].copy_(Xh, non_blocking=True)
            bb[i].copy_(bh, non_blocking=True)
            ready[i].record(cs)

    # warm-up of both buffers' operators
    for i in (0, 1):
        free[i].record(main)
        copy_in(i)
        main.wait_event(ready[i])
        solve_once(ny, ops[i], bb[i], ell, seed=7)
        free[i].record(main)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    copy_in(0)
    for k in range(args.steps):
        i = k % 2
        if k + 1 < args.steps:
            copy_in(1 - i)                  # next step's inputs, behind this solve
        main.wait_event(ready[i])
        xk, _ = solve_once(ny, ops[i], bb[i], ell, seed=k)
        free[i].record(main)
        xh.copy_(xk, non_blocking=True)
        main.synchronize()                  # this step's result is on the host
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    dt = max_over_ranks(dt, world)
    # serial reference: copy, solve, read back
    t0 = time.perf_counter()
    for k in range(args.steps):
        Xb[0].copy_(Xh, non_blocking=True)
        bb[0].copy_(bh, non_blocking=True)
        xk, _ = solve_once(ny, ops[0], bb[0], ell, seed=k)
        xh.copy_(xk, non_blocking=True)
        torch.cuda.synchronize()
    dts = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
    return {"value": world / dt, "unit": "solves/s", "h2d_bytes_per_step": int(X.nbytes + n * 8),
            "d2h_bytes_per_step": int(n * 8),
            "pipeline": "step k+1's H2D copy on a second stream during step k's solve "
                        "(two device copies of X)",
            "serial": {"value": world / dts, "unit": "solves/s"}}


def run_ours(args):
    import torch

    from paper_2110_02820_gb300 import nyspcg as ny
    ny.pcg_graphs(args.pcg_launch == "graph")
    rank, world, local = dist_init(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    m, n, ell = args.m, args.n, args.ell
    X, y = make_inputs(m, n)
    Xd = torch.tensor(X, device=dev)
    b = rhs_on_device(Xd, y)
    op = ny.gram_operator(Xd)
    torch.cuda.synchronize()

    # warm-up (also builds the pools)
    res = None
    for w in range(args.warmup):
        x, res = solve_once(ny, op, b, ell, seed=1000 + w)
    torch.cuda.synchronize()

    # timed region: K complete solves, inputs resident
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    launches0 = ny.kernel_launch_count()
    ev0.record()
    for k in range(args.steps):
        x, res = solve_once(ny, op, b, ell, seed=k)
        iters.append((res.iterations, res.refinements, res.rel_residual, res.status))
    ev1.record()
    torch.cuda.synchronize()
    launches_timed = ny.kernel_launch_count() - launches0
    barrier(world)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms, world)
    bad = [it for it in iters if it[3] != 0]
    if bad:
        # a solve that missed the residual target is not a solve of the metric
        sys.stderr.write(f"bench: {len(bad)} of {len(iters)} timed solves did not converge: {bad[0]}\n")
        sys.exit(3)
    value = job_throughput(ms, world)
    if args.solve_only:
        if rank == 0:
            print(json.dumps({"solve_only": True, "ms_per_step": ms, "value": value,
                              "solve": iters[-1]}), flush=True)
        return

    # dominant kernel: the fused ridge matvec (gram_fused_kernel + its fixed-order
    # reduction), its average duration over the products of two more solves run
    # with CUDA events around each product (kept out of the timed region)
    ny.timing_start(8192)
    for k in range(2):
        solve_once(ny, op, b, ell, seed=k)
    torch.cuda.synchronize()
    mv_total_ms, mv_count = ny.timing_stop()
    mv_ms = mv_total_ms / max(mv_count, 1)
    bytes_mv = float(m) * n * 4  # X read once per matvec
    achieved = bytes_mv / (mv_ms * 1e-3) / 1e9
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peak = json.load(open(peaks_path))["hbm_gbs"]
        peak_src = "measured"
    else:
        peak = 6800.0
        peak_src = "fallback"

    # where a step's time goes
    phases = phase_times(ny, op, b, ell)

    # end to end: host inputs (pinned) -> device, solve, solution -> host
    e2e = None
    if not args.no_e2e:
        e2e = e2e_ridge(ny, torch, X, Xd, b, n, ell, args, world)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_baseline(m, n, ell, max(2000, m // 4))

    # the other workloads, one record each (one GPU, rank 0 only): the dense
    # FP64 solve, kernel ridge regression, the batched regularisation path and
    # the differentiable-KRR step, each with its dominant kernel's roofline
    peaks, legs = None, None
    if rank == 0 and world == 1 and not args.no_legs:
        del Xd, op
        torch.cuda.empty_cache()
        peaks = measured_peaks(ny)
        legs = {}
        for name, st, wu in [("dense", 5, 3), ("krr", 2, 1), ("batched", 1, 1), ("adjoint", 1, 1)]:
            try:
                legs[name] = workload_record(args, name, st, wu, peaks)
            except Exception as e:  # one workload failing does not hide the others
                legs[name] = {"workload": name, "error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()

    if rank == 0:
        line = {
            "metric": "PCG solves/sec to rel-residual 1e-8 and kernel-matvec TFLOP/s vs roofline, 1xGB300",
            "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"ridge X {m}x{n} fp32 (col j scaled 1/(j+1)), A=X^T X, mu={MU}, "
                                   f"ell={ell}, tol={TOL} rel. residual (FP64, refined)",
                       "l2": "inputs larger than L2 (X 3.3 GB)", "parallelism": "replicas"},
            "roofline": {"bound": "hbm", "kernel": "gram_fused_kernel (+reduce)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": peak_src,
                         "peak_note": "peak = measured copy (read + write) bandwidth; this "
                                      "kernel only reads X, so frac can exceed 1",
                         "rated_peak": RATED_HBM_GBS, "frac_of_rated": achieved / RATED_HBM_GBS,
                         "traffic": measured_traffic() if (m, n) == (M, N) else None,
                         "bytes_per_launch": bytes_mv, "ms_per_launch": mv_ms,
                         "launches_timed": int(mv_count)},
            "cpu_baseline": cb,
            "e2e": e2e,
            "gpu_launches": int(launches_timed),
            "pcg_launch": args.pcg_launch,
            "clocks": clk,
            "solve": {"inner_iterations": iters[-1][0], "refinements": iters[-1][1],
                      "rel_residual": iters[-1][2], "status": iters[-1][3]},
            "phases_ms": phases,
            "configs": legs,
            "unit_peaks": peaks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ---------------------------------------------------------------- measured DRAM traffic

PROFILE_RIDGE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "profiles",
                             "gram_fused_kernel_ridge_200000x4096.md")
RIDGE_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2110_02820_gb300",
                         "csrc", "operators.cu")


GRAM_SECTION = "// ============================================================ gram (fused single pass)"


def gram_section(text):
    """The part of operators.cu that holds the fused ridge matvec: from its
    section marker to the next section marker."""
    i = text.find(GRAM_SECTION)
    if i < 0:
        return text
    j = text.find("// ============================================================", i + len(GRAM_SECTION))
    return text[i:j if j > 0 else len(text)]


def measured_traffic():
    """DRAM bytes per ridge-matvec launch from the committed ncu summary, or
    None when the kernel source changed since the counters were taken."""
    import hashlib
    try:
        text = open(PROFILE_RIDGE).read()
        src = hashlib.sha256(gram_section(open(RIDGE_SRC).read()).encode()).hexdigest()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch:", "source_sha256:")):
            k, v = line.strip().split(":", 1)
            vals[k] = v.strip().strip("`")
    if vals.get("source_sha256") != src:
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- other workloads

def _events_ms(fn, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    out = None
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def _events_steps(fn, reps, flush=None):
    """Mean ms per call of fn over reps calls, CUDA events on the current
    stream; `flush` (if given) runs between calls, outside the timed spans."""
    import torch
    tot, out = 0.0, None
    for _ in range(reps):
        if flush is not None:
            flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps, out


class L2Flush:
    """Writes a buffer twice the size of L2 (129 MB on GB300) between timed
    steps whose inputs fit in L2."""

    def __init__(self, device):
        import torch
        self.buf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=device)  # 256 MB

    def __call__(self):
        self.buf.fill_(1.0)


def measured_peaks(ny):
    """Denominators of the roofline fractions: HBM copy bandwidth and BF16
    tensor rate from MEASURED_PEAKS.json (TF32 = BF16 x the nominal 1.1/2.25
    ratio), and the FP64 FMA, FP32 FMA and MUFU ex2 rates measured here by the
    library's unit probes."""
    p = {}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        j = json.load(open(path))
        p.update(hbm_gbs=j["hbm_gbs"], bf16_tflops=j["bf16_tflops"],
                 bf16_tflops_sustained=j.get("bf16_tflops_sustained"), source="measured")
    else:
        p.update(hbm_gbs=6800.0, bf16_tflops=1900.0, bf16_tflops_sustained=1700.0,
                 source="fallback")
    p["tf32_tflops"] = p["bf16_tflops"] * 1.1 / 2.25
    p["tf32_tflops_sustained"] = (p["bf16_tflops_sustained"] or p["bf16_tflops"]) * 1.1 / 2.25
    p["fp64_fma_tflops"] = ny.nys_unit_peak(ny.UNIT_FP64_FMA) / 1e12
    p["fp32_fma_tflops"] = ny.nys_unit_peak(ny.UNIT_FP32_FMA) / 1e12
    p["mufu_ex2_gops"] = ny.nys_unit_peak(ny.UNIT_MUFU_EX2) / 1e9
    return p


def workload_record(args, name, steps, warmup, peaks=None):
    """One record (dict) for the workload `name`: solves/sec (or converged
    systems/sec), per-phase times and the dominant kernel against its
    roofline.  Inputs are resident on the device; between timed steps whose
    inputs fit in L2 a 256 MB buffer is written."""
    import torch

    from paper_2110_02820_gb300 import nyspcg as ny
    from paper_2110_02820_gb300 import workloads as wl
    ny.pcg_graphs(args.pcg_launch == "graph")
    dev = torch.device("cuda", torch.cuda.current_device())
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)  # noqa: E731
    flush = L2Flush(dev)
    line = {"metric": "PCG solves/sec to rel-residual target", "unit": "solves/s",
            "steps": steps, "warmup": warmup, "higher_is_better": True,
            "data": "synthetic", "workload": name, "l2": "256 MB written between timed steps"}
    clocks = ClockSampler(torch.cuda.current_device())
    if name == "dense":
        n, ell, mu, tol = 2048, 64, 1e-4, 1e-10
        A, _ = wl.dense_spd(n, seed=0)
        b = T(wl.rhs(n, seed=0))
        op = ny.dense_operator(T(A))

        phase = {}

        def step(seed):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            f = ny.nys_sketch(op, ell, seed=seed)
            e1.record()
            x, res, _ = ny.pcg_solve(op, f, mu, b, tol=tol)
            e2.record()
            torch.cuda.synchronize()
            phase["sketch_ms"], phase["pcg_ms"] = e0.elapsed_time(e1), e1.elapsed_time(e2)
            f.free()
            return res[0]
        for w in range(warmup):
            step(100 + w)
        clocks.start()
        launches0 = ny.kernel_launch_count()
        # CUDA events around every dense product of the timed solves (recorded
        # on the launching stream, inside the PCG graph as event nodes)
        ny.timing_start(65536)
        ms, res = _events_steps(lambda: step(7), steps, flush)
        mv_total, mv_cnt = ny.timing_stop()
        mv_ms = mv_total / max(mv_cnt, 1)
        line["solve"] = {"iterations": res.iterations, "rel_residual": res.rel_residual,
                         "status": res.status}
        line["phases_ms"] = dict(phase)
        gfl = 2 * n * n / (mv_ms * 1e6)
        line.update({"dtype": "f64", "config": {"workload": f"dense FP64 n={n}, lambda_i=(i+1)^-1.5, "
                                                            f"mu={mu}, ell={ell}, tol={tol}"},
                     "dominant_kernel": {"kernel": "dense_matvec_kernel<double>",
                                         "ms_per_launch": mv_ms, "launches_timed": int(mv_cnt),
                                         "gflops_fp64": gfl, "l2_resident_bytes": n * n * 8}})
        if peaks:
            line["roofline"] = {"bound": "alu", "unit": "TFLOP/s", "achieved": gfl / 1e3,
                                "peak": peaks["fp64_fma_tflops"],
                                "frac": gfl / 1e3 / peaks["fp64_fma_tflops"],
                                "work": "2 n^2 FP64 FLOP per product (A read from L2)",
                                "peak_source": "FP64 FMA pipe measured by nys_unit_peak"}
    elif name in ("krr", "batched"):
        if name == "krr":
            n, d, ell0, ell_max = int(100000 * args.scale), 32, 128, 2048
        else:
            n, d, ell = int(50000 * args.scale), 16, 1024
        P = wl.gmm_points(n, d, seed=0)
        sigma = wl.median_distance(P, seed=0)
        op = ny.rbf_operator(T(P), sigma)
        prec = ny.NYS_PREC_F64 if args.precision == "f64" else ny.NYS_PREC_MIXED
        phase = {}
        if name == "krr":
            mu, tol = 1e-6 * n, 1e-8
            b = T(wl.rhs(n, seed=0))

            def step(seed):
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record()
                if args.sketch == "columns":
                    f = ny.nys_sketch_columns(op, args.cols, seed=seed, precision=prec)
                    info = None
                else:
                    f, info = ny.nys_sketch_adaptive(op, ell0, ell_max, ny.NYS_RULE_RATIO, 40.0, 0,
                                                     mu, seed=seed, precision=prec)
                e1.record()
                x, res, _ = ny.pcg_solve(op, f, mu, b, tol=tol, precision=prec)
                e2.record()
                torch.cuda.synchronize()
                phase["sketch_ms"], phase["pcg_ms"] = e0.elapsed_time(e1), e1.elapsed_time(e2)
                f.free()
                return res[0], info
            sk = (f"column sampling, ell={args.cols} uniform points" if args.sketch == "columns"
                  else f"adaptive ratio rule 40, ell {ell0}->{ell_max}")
            cfg = (f"kernel ridge n={n} d={d} GMM(10), sigma=median dist={sigma:.3f}, mu=1e-6 n, "
                   f"{sk}, {'FP64 PCG' if args.precision == 'f64' else 'mixed + FP64 refinement'}, "
                   f"tol {tol}")
        else:
            mus = list(np.repeat(wl.regularization_path(32, 1e-8 * n, 1e-1 * n), 4))
            B = T(np.tile(wl.rhs(n, seed=0, nrhs=4), (32, 1)))
            tol = 1e-8

            def step(seed):
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record()
                f = ny.nys_sketch(op, ell, seed=seed, precision=prec)
                e1.record()
                x, res, _ = ny.pcg_solve(op, f, mus, B, tol=tol, precision=prec)
                e2.record()
                torch.cuda.synchronize()
                phase["sketch_ms"], phase["pcg_ms"] = e0.elapsed_time(e1), e1.elapsed_time(e2)
                f.free()
                return res, None
            cfg = (f"batched regularisation path n={n} d={d}, 32 shifts log-spaced in "
                   f"[1e-8, 1e-1] n x 4 rhs = 128 systems, ell={ell}, {args.precision}, "
                   f"tol {tol} each")
        for w in range(warmup):
            step(100 + w)
        clocks.start()
        launches0 = ny.kernel_launch_count()
        ny.timing_start(65536)
        ms, (res, info) = _events_steps(lambda: step(7), steps, flush)
        mv_total, mv_cnt = ny.timing_stop()
        mv_ms = mv_total / max(mv_cnt, 1)
        kern = ("rbf_gemv_kernel (tensor-core distances, one vector)" if name == "krr"
                else "rbf_h16_kernel<S,3> (FP16 splits, tensor cores)")
        if args.precision == "f64":
            kern = "rbf_products_kernel (FP64 entries and sums; not event-timed)"
        line.update({"dtype": "f64" if args.precision == "f64" else "f32",
                     "config": {"workload": cfg},
                     "dominant_kernel": {"kernel": kern, "ms_per_launch": mv_ms,
                                         "launches_timed": mv_cnt,
                                         "kernel_entries_per_s":
                                             n * n / (mv_ms * 1e-3) if mv_ms > 0 else None}})
        if name == "krr":
            line["solve"] = {"iterations": res.iterations, "refinements": res.refinements,
                             "rel_residual": res.rel_residual, "status": res.status,
                             "escalated": res.escalated,
                             "ell": info.ell if info else args.cols,
                             "doublings": info.doublings if info else None,
                             "lambda_ell": info.lambda_ell if info else None}
            if peaks and mv_ms > 0 and args.precision != "f64":
                eps = n * n / (mv_ms * 1e-3) / 1e9
                line["roofline"] = {"bound": "alu", "unit": "Gop/s (ex2)", "achieved": eps,
                                    "peak": peaks["mufu_ex2_gops"],
                                    "frac": eps / peaks["mufu_ex2_gops"],
                                    "work": "one MUFU ex2 per kernel entry, n^2 entries per product",
                                    "peak_source": "MUFU ex2 rate measured by nys_unit_peak"}
        else:
            its = [r.iterations for r in res]
            ok = [r.status == 0 for r in res]
            line["solve"] = {"systems": len(res), "converged": int(sum(ok)),
                             "escalated": int(sum(r.escalated for r in res)),
                             "iterations_min": min(its), "iterations_max": max(its),
                             "worst_rel_residual_converged":
                                 max([r.rel_residual for r in res if r.status == 0] or [None]),
                             "status_by_mu": [[float(m), r.status, r.iterations, r.rel_residual]
                                              for m, r in list(zip(mus, res))[::4]]}
            if peaks and args.precision != "f64":
                # the full 128-vector product alone: FP16 splits (kind::f16, three
                # passes of each GEMM) in the tuned shape (vectors per CTA)
                V = T(np.tile(wl.rhs(n, seed=1, nrhs=4), (32, 1)))
                ny.nys_op_matvec(op, 1e-6 * n, V, mode=1)
                pms, _ = _events_steps(lambda: ny.nys_op_matvec(op, 1e-6 * n, V, mode=1), 3)
                npad = (n + 127) // 128 * 128
                code = next((c for k, c in ny.autotune_choices().items()
                             if k.startswith(f"rbf_tc16 passes=3 npad={npad} ")), None)
                S = (128, 64, 32)[code // 8] if code is not None else 128
                cols = -(-V.shape[0] // S)
                alg = 2.0 * n * n * (V.shape[0] + d)
                ks16 = 16 * (-(-d // 16))
                exe = 3.0 * 2.0 * npad * npad * (cols * S + cols * ks16)
                line["dominant_kernel"]["kernel"] = f"rbf_h16_kernel<{S},3> (FP16 splits, tensor cores, " \
                                                    f"{S} systems per CTA)"
                line["roofline"] = {"bound": "tensor", "unit": "TFLOP/s",
                                    "achieved": alg / (pms * 1e-3) / 1e12,
                                    "peak": peaks["bf16_tflops"],
                                    "frac": alg / (pms * 1e-3) / 1e12 / peaks["bf16_tflops"],
                                    "executed_tflops": exe / (pms * 1e-3) / 1e12,
                                    "tensor_pipe_frac": exe / (pms * 1e-3) / 1e12 / peaks["bf16_tflops"],
                                    "ms_per_launch": pms,
                                    "vectors_per_cta": S, "tuned_code": code,
                                    "work": "algorithmic 2 n^2 (nvec + d) FLOP for 128 vectors; "
                                            "executed = 3 FP16 passes of the distance GEMM (K "
                                            "padded to 16) per CTA column and of the "
                                            "kernel-times-vectors GEMM, padded n",
                                    "peak_source": "FP16 dense = measured BF16 rate (same "
                                                   "nominal rate)"}
        line["phases_ms"] = dict(phase)
    elif name == "block":
        # block Nystrom PCG: nrhs right-hand sides of one shifted Gaussian-kernel
        # system, against the same systems solved as independent recurrences
        n, d, ell, nrhs = int(50000 * args.scale), 16, args.block_ell, args.nrhs
        P = wl.gmm_points(n, d, seed=0)
        sigma = wl.median_distance(P, seed=0)
        op = ny.rbf_operator(T(P), sigma)
        mu, tol = 2e-7 * n, 1e-8
        B = T(wl.rhs(n, seed=0, nrhs=nrhs))
        phase = {}

        def step(seed):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            f = ny.nys_sketch(op, ell, seed=seed, precision=ny.NYS_PREC_MIXED)
            e1.record()
            X, res = ny.nys_block_pcg(op, f, mu, B, tol=tol, precision=ny.NYS_PREC_MIXED)
            e2.record()
            torch.cuda.synchronize()
            phase["sketch_ms"], phase["block_pcg_ms"] = e0.elapsed_time(e1), e1.elapsed_time(e2)
            f.free()
            return res, None
        for w in range(warmup):
            step(100 + w)
        clocks.start()
        launches0 = ny.kernel_launch_count()
        ms, (res, _) = _events_steps(lambda: step(7), steps, flush)
        # the same systems as independent recurrences (one kernel pass per step for all)
        f = ny.nys_sketch(op, ell, seed=7, precision=ny.NYS_PREC_MIXED)
        ind_ms, (xi, ri, _) = _events_steps(
            lambda: ny.pcg_solve(op, f, [mu] * nrhs, B, tol=tol, precision=ny.NYS_PREC_MIXED), 1)
        f.free()
        ok = [r.status == 0 for r in res]
        line.update({"dtype": "f32",
                     "config": {"workload": f"block PCG, Gaussian kernel n={n} d={d} "
                                            f"GMM(10), {nrhs} right-hand sides of mu=2e-7 n, "
                                            f"ell={ell}, mixed, tol {tol}"},
                     "solve": {"systems": nrhs, "converged": int(sum(ok)),
                               "block_products": res[0].iterations,
                               "refinements": res[0].refinements,
                               "worst_rel_residual": max(r.rel_residual for r in res)},
                     "independent": {"pcg_ms": ind_ms,
                                     "iterations_max": max(r.iterations for r in ri),
                                     "converged": int(sum(r.status == 0 for r in ri))},
                     "phases_ms": dict(phase)})
    elif name == "path":
        # regularization path on the ridge operator: decreasing shifts, warm
        # starts, factor reuse (err_factor 30, q 5), mixed precision
        X, y = make_inputs(args.m, args.n)
        Xd = T(X)
        b = rhs_on_device(Xd, y)
        op = ny.gram_operator(Xd)
        mus = [10.0 ** e for e in range(1, -4, -1)]
        ell0, ell_max, tol = 128, 2048, 1e-8

        def step(seed):
            Xs, out = ny.nys_reg_path(op, mus, b, ell0, ell_max, 30.0, 5, seed=seed, tol=tol,
                                      precision=ny.NYS_PREC_MIXED)
            return out, None
        for w in range(warmup):
            step(100 + w)
        clocks.start()
        launches0 = ny.kernel_launch_count()
        ms, (out, _) = _events_steps(lambda: step(7), steps)
        ok = [o["status"] == 0 for o in out]
        line.update({"dtype": "f32", "l2": "inputs larger than L2 (X 3.3 GB)",
                     "config": {"workload": f"regularization path, ridge {args.m}x{args.n}, "
                                            f"mu = 10..1e-3 (5 shifts, decreasing), warm starts, "
                                            f"factor kept while estimate <= 30 mu, ell {ell0}->"
                                            f"{ell_max}, mixed, tol {tol}"},
                     "solve": {"systems": len(mus), "converged": int(sum(ok)),
                               "builds": int(sum(o["resketched"] for o in out)),
                               "per_shift": [[m, o["ell"], o["resketched"], o["iterations"],
                                              o["status"]] for m, o in zip(mus, out)]}})
    else:  # adjoint
        from paper_2110_02820_gb300 import krr
        n, nv, d, ell = int(200000 * args.scale), int(10000 * args.scale), 16, 2048
        P = wl.gmm_points(n, d, seed=0)
        V = wl.gmm_points(nv, d, seed=1)
        y, yv = T(wl.krr_targets(P, 0)), T(wl.krr_targets(V, 1))
        sigma0 = wl.median_distance(P, seed=0)
        Pt, Vt = T(P), T(V)

        phase = {}

        def step(seed):
            sg = torch.tensor(sigma0, dtype=torch.float64, device=dev, requires_grad=True)
            m = torch.tensor(1e-6 * n, dtype=torch.float64, device=dev, requires_grad=True)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            L = krr.validation_loss(Pt, y, Vt, yv, sg, m, ell,
                                    precision=ny.NYS_PREC_F64 if args.precision == "f64"
                                    else ny.NYS_PREC_MIXED,
                                    tol=1e-8, seed=seed)
            e1.record()
            L.backward()
            e2.record()
            torch.cuda.synchronize()
            phase["forward_ms"], phase["backward_ms"] = e0.elapsed_time(e1), e1.elapsed_time(e2)
            return float(L.detach()), float(m.grad), float(sg.grad)
        for w in range(warmup):
            step(100 + w)
        clocks.start()
        launches0 = ny.kernel_launch_count()
        ny.timing_start(65536)
        ms, out = _events_steps(lambda: step(7), steps, flush)
        mv_total, mv_cnt = ny.timing_stop()
        mv_ms = mv_total / max(mv_cnt, 1)
        line.update({"dtype": "f64" if args.precision == "f64" else "f32",
                     "config": {"workload": f"differentiable KRR n_train={n} n_val={nv} d={d} "
                                            f"ell={ell} {args.precision}, loss + dL/dmu + dL/dsigma"},
                     "solve": {"loss": out[0], "dL_dmu": out[1], "dL_dsigma": out[2]},
                     "dominant_kernel": {"kernel": "rbf_gemv_kernel (one vector, inside the "
                                                   "forward and adjoint solves)",
                                         "ms_per_launch": mv_ms, "launches_timed": mv_cnt},
                     "phases_ms": dict(phase)})
        if peaks and mv_ms > 0 and args.precision != "f64":
            eps = n * n / (mv_ms * 1e-3) / 1e9
            line["roofline"] = {"bound": "alu", "unit": "Gop/s (ex2)", "achieved": eps,
                                "peak": peaks["mufu_ex2_gops"],
                                "frac": eps / peaks["mufu_ex2_gops"],
                                "work": "one MUFU ex2 per kernel entry, n^2 entries per product",
                                "peak_source": "MUFU ex2 rate measured by nys_unit_peak"}
    line["clocks"] = clocks.stop()
    sol = line.get("solve", {})
    if name in ("batched", "block", "path"):
        line["metric"] = "converged PCG systems/sec (rel-residual 1e-8 each)"
        line["unit"] = "systems/s"
        line["value_note"] = "value = converged systems / solve time"
    line["converged"] = not (sol.get("status", 0) != 0 or
                             sol.get("converged", sol.get("systems", 1)) != sol.get("systems", 1))
    line["ms_per_step"] = ms
    line["value"] = (sol["converged"] if name in ("batched", "block", "path") else 1) * 1e3 / ms
    line["gpu_launches"] = int(ny.kernel_launch_count() - launches0)
    line["pcg_launch"] = args.pcg_launch
    return line


def run_workload(args):
    """One JSON line for a non-default workload."""
    import torch

    from paper_2110_02820_gb300 import nyspcg as ny
    torch.cuda.set_device(0)
    peaks = measured_peaks(ny)
    line = workload_record(args, args.workload, args.steps, args.warmup, peaks)
    line["n_gpus"] = 1
    line["unit_peaks"] = peaks
    if not line["converged"] and line.get("solve", {}).get("converged", 1) == 0:
        sys.stderr.write(f"bench: the {args.workload} solve did not converge: {line['solve']}\n")
        sys.exit(3)
    print(json.dumps(line), flush=True)


def run_matvec_only(args):
    """The dominant FP32 product of a workload, alone: the ridge matvec at
    m x n, or the one-vector Gaussian matvec at n = 100000 scale, d = 32."""
    import torch

    from paper_2110_02820_gb300 import nyspcg as ny
    from paper_2110_02820_gb300 import workloads as wl
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    if args.workload == "ridge":
        X = torch.tensor(wl.ridge_X(args.m, args.n, SEED), device=dev)
        op = ny.gram_operator(X)
        v = torch.tensor(wl.rhs(args.n, SEED), device=dev)
        mu, what = MU, f"ridge matvec {args.m}x{args.n}"
    elif args.workload == "batched":
        n = int(50000 * args.scale)
        P = wl.gmm_points(n, 16, SEED)
        op = ny.rbf_operator(torch.tensor(P, device=dev), wl.median_distance(P, SEED))
        v = torch.tensor(wl.rhs(n, SEED, nrhs=128), device=dev)
        mu, what = 1e-6 * n, f"batched Gaussian matvec n={n} d=16, 128 vectors"
    else:
        n = int(100000 * args.scale)
        P = wl.gmm_points(n, 32, SEED)
        op = ny.rbf_operator(torch.tensor(P, device=dev), wl.median_distance(P, SEED))
        v = torch.tensor(wl.rhs(n, SEED), device=dev)
        mu, what = 1e-6 * n, f"Gaussian matvec n={n} d=32"
    mode = args.matvec_mode
    for _ in range(args.warmup):
        ny.nys_op_matvec(op, mu, v, mode=mode)
    if mode == 1 and v.dim() == 2:
        # many vectors: the call (FP64->FP32 conversions + one tensor-core pass)
        # timed with events on the current stream
        ms, (y,) = _events_ms(lambda: (ny.nys_op_matvec(op, mu, v, mode=mode),), args.steps)
        cnt = args.steps
        ms_per = ms
    elif mode == 1:
        ny.timing_start(max(args.steps, 1))
        for _ in range(args.steps):
            y = ny.nys_op_matvec(op, mu, v, mode=mode)
        ms, cnt = ny.timing_stop()
        ms_per = ms / max(cnt, 1)
    else:
        # the residual product is not among the event-timed FP32 products
        ms_per, y = _events_ms(lambda: ny.nys_op_matvec(op, mu, v, mode=mode), args.steps)
        cnt = args.steps
    print(json.dumps({"matvec_only": what, "mode": mode, "ms_per_matvec": ms_per, "timed": cnt,
                      "checksum": float(y.abs().sum())}), flush=True)


def main():
    args = parse()
    if args.matvec_only:
        run_matvec_only(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload != "ridge":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
