"""Benchmark: factor + PCG wall time to relative residual 1e-10 on the 3D
7-point Laplacian 64^3 (N = 262,144), 10 nested-dissection levels,
eps = 1e-2, b ~ N(0,1) (seed 1); mixed FP32 factor / FP64 PCG against the
plain FP64 form on the same GPU.

One step = spand_factorize + spand_solve (the whole hot path).  The headline
`value` is the mixed form's seconds per step with A's values and b already
resident in HBM; `e2e` is the same metric through the C ABI with host
buffers (H2D of the values and b, D2H of x inside the timed region).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
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

GRID, LEVELS, EPS, SEED = 64, 10, 1e-2, 1
WORKLOAD = "lapl3d_64^3_7pt_L10_eps1e-2"
METRIC = "factor+PCG s to rel-res 1e-10 (3D), mixed/batched vs FP64; % roofline"
# wall-clock budget of the reference arm (full-size oracle steps)
REF_BUDGET_S = 300.0


def workload_config(n, nnz, levels=LEVELS, grid=GRID, world=1) -> dict:
    """The `config` of both arms' lines: the workload only (no precision or
    implementation keys), so that the two lines name the same problem."""
    return {"workload": WORKLOAD if (grid, levels) == (GRID, LEVELS) else f"lapl3d_{grid}^3_7pt_L{levels}_eps1e-2",
            "N": int(n), "nnz": int(nnz), "levels": int(levels), "eps": EPS, "tol": 1e-10, "b_seed": SEED,
            "parallelism": f"replicas x{world}",
            "l2": "256 MB L2 flush between timed GPU steps; factor data > 129 MB"}


_ORACLE_RUN = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
from paper_1901_02971_gb300 import inputs as I
from oracle import spand_oracle as O
p = I.laplacian_3d(%(grid)d); b = I.rhs(p.n, %(seed)d)
t0 = time.perf_counter(); tr = O.analyze(p.n, p.rowptr, p.colind, p.coords, %(levels)d); t_p = time.perf_counter() - t0
print(json.dumps(dict(kind="analysis", t_p=t_p, n=p.n, nnz=p.nnz)), flush=True)
A = O.permuted_matrix(p.rowptr, p.colind, p.vals, tr.perm)
W = %(workers)d
if W > 1:  # the all-core leg: the independent blocks of each level and colour on a spawn pool
    from oracle import spand_parallel as OP
    pool = OP.make_pool(W)
    list(pool.map(abs, range(4 * W)))  # workers started (and the oracle imported) before the clock
    fact = lambda: OP.factorize(p.rowptr, p.colind, p.vals, tr, %(eps)r, pool, W)
else:
    fact = lambda: O.factorize(p.rowptr, p.colind, p.vals, tr, %(eps)r)
start = time.perf_counter(); last = 0.0
for i in range(%(steps)d):
    if i > 0 and time.perf_counter() - start + last > %(budget)r:
        break
    t1 = time.perf_counter()
    F = fact()
    t2 = time.perf_counter()
    x, it, rr = O.pcg(A, b[tr.perm], lambda r: O.apply(F, r))
    t3 = time.perf_counter()
    last = t3 - t1
    print(json.dumps(dict(kind="step", t_f=t2 - t1, t_s=t3 - t2, iters=it, relres=rr,
                          size_top=F.size_top, mem_f=F.mem_f)), flush=True)
"""


def oracle_runs(steps: int = 1, budget_s: float = 1e30, threads: int = 1, grid: int = GRID,
                levels: int = LEVELS, workers: int = 1) -> dict:
    """Times the FP64 oracle on the whole workload in a fresh process
    (started before any CUDA work in this one; its BLAS/LAPACK limited to
    `threads` threads per process): the analysis once, then up to `steps`
    full factorizations + PCG solves, stopping early when the next one would
    run past `budget_s` (at least one always runs).  With workers > 1 the
    factorization is the all-core leg (oracle/spand_parallel.py: the
    independent blocks of each level and colour on a pool of that many
    processes); the PCG stays serial.  Returns t_P and the list of per-step
    t_F, t_S, n_CG."""
    code = _ORACLE_RUN % dict(root=ROOT, grid=grid, seed=SEED, levels=levels, steps=max(1, steps),
                              budget=float(budget_s), eps=EPS, workers=int(workers))
    t = str(int(threads))
    env = dict(os.environ, OPENBLAS_NUM_THREADS=t, OMP_NUM_THREADS=t, MKL_NUM_THREADS=t)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=7200)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed: " + r.stderr[-2000:])
    recs = [json.loads(ln) for ln in r.stdout.splitlines() if ln.startswith("{")]
    ana = [x for x in recs if x["kind"] == "analysis"][0]
    return {"t_p": ana["t_p"], "steps": [x for x in recs if x["kind"] == "step"]}


def oracle_phases(run: dict) -> dict:
    """t_P, and the mean t_F, t_S (s) and the n_CG of the oracle's steps."""
    st = run["steps"]
    return {"t_p_s": round(run["t_p"], 3), "t_f_s": round(statistics.mean(x["t_f"] for x in st), 3),
            "t_s_s": round(statistics.mean(x["t_s"] for x in st), 3), "n_cg": int(st[-1]["iters"]),
            "relres": st[-1]["relres"], "size_top": int(st[-1]["size_top"]), "mem_f": int(st[-1]["mem_f"])}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "_source": "fallback"}


# ALU peaks derived from unit counts and the maximum SM clock (152 SMs,
# 2070 MHz): FP32 = 128 lanes x 2 flops per SM per clock; FP64 as stated for
# GB300 (1.25 TFLOP/s).
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FP64_ALU_TFLOPS = 1.25
# TF32 tensor peak: cuBLAS 8192^3 TF32 GEMM measured on this machine's GB300
# (torch.matmul with TF32 allowed: 1032.7 TFLOP/s; the same probe gave BF16
# 1945 TFLOP/s, in line with the measured bf16 figure, and FP32 SIMT 69.8).
TF32_TENSOR_TFLOPS = 1032.7
HBM_BOUND = {"copy", "apply", "pcg"}


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum, one
# ncu capture of the FP32 form on the 64^3 workload, averaged over the launches
# of one factorization or solve), with the SHA-256 of the kernel source the
# counters were taken on: a changed kernel reports null until re-measured.
# The capture and its command are summarised under profiles/ (DRAM traffic, 64^3).
CPQR_DRAM_BYTES = 583.09e6 + 5.74e6  # read + written by the 265 launches of one factorization
MEASURED_TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum: "cpqr", of all the
    # sparsification launches of one factorization (k_cpqr_cluster,
    # k_cpqr_reg, k_form_q), divided by the family's launch count of the
    # profiled run; "apply", of three applications (one launch each); ncu,
    # one pass
    "cpqr": {"bytes_per_step": CPQR_DRAM_BYTES,
             "src": ["paper_1901_02971_gb300/csrc/cpqr_cluster.cuh", "paper_1901_02971_gb300/csrc/cpqr_reg.cuh"],
             "sha256": ["df1a284e74542b5aa3f39bc25ec90beb14e91cbaa13b15fbeed6c93563a1f421",
                        "f4375f2638107797fe808912ff23db71eba06329efe4f946106ee94aebe58cd8"]},
    "apply": {"bytes_per_launch": (3100.6e6 + 40.1e6) / 3, "src": "paper_1901_02971_gb300/csrc/solve_kernels.cuh",
              "sha256": "6520881e8f0975871035275afc7fec1c110a1adcde70f8a412a4ef8d529d2dcf"},
}


def measured_traffic(fam: str, grid: int, launches: int = 1):
    t = MEASURED_TRAFFIC.get(fam)
    if t is None or grid != GRID:
        return None
    import hashlib
    srcs = t["src"] if isinstance(t["src"], list) else [t["src"]]
    sums = t["sha256"] if isinstance(t["sha256"], list) else [t["sha256"]]
    for src, want in zip(srcs, sums):
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), src)
        try:
            with open(path, "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != want:
                    return None
        except OSError:
            return None
    if "bytes_per_step" in t:
        return t["bytes_per_step"] / max(int(launches), 1)
    return t["bytes_per_launch"]


def make_roofline(prof: dict, peaks: dict, dtype_peak_tflops: float = FP32_ALU_TFLOPS, grid: int = GRID) -> dict:
    """Roofline of the kernel family with the largest device time in one
    profiled factor+solve: achieved = algorithmic flops (or bytes) of its
    launches / their CUDA-event duration."""
    fam = max(prof, key=lambda k: prof[k]["ms"])
    f = prof[fam]
    sec = f["ms"] / 1e3
    traffic = measured_traffic(fam, grid, f["launches"])
    if fam in HBM_BOUND:
        ach = f["bytes"] / sec / 1e9
        pk = float(peaks["hbm_gbs"])
        return {"kernel": fam, "bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s", "frac": ach / pk,
                "traffic": traffic, "peak_source": peaks["_source"], "launches": f["launches"], "ms": f["ms"]}
    ach = f["flops"] / sec / 1e12
    return {"kernel": fam, "bound": "alu", "achieved": ach, "peak": dtype_peak_tflops, "unit": "TFLOP/s",
            "frac": ach / dtype_peak_tflops, "traffic": traffic,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz", "launches": f["launches"],
            "ms": f["ms"]}


def phase_rooflines(prof: dict, peaks: dict, form: str) -> dict:
    """Achieved rate and fraction of its bounding peak for every kernel family
    of one profiled factor+solve: HBM families against the measured copy
    bandwidth; the Schur family of the TF32 / BF16 forms against the tensor
    peak of its operand type; the rest against the FP32 ALU peak."""
    out = {}
    for fam, f in prof.items():
        sec = f["ms"] / 1e3
        if sec <= 0:
            continue
        if fam in HBM_BOUND:
            ach, pk, unit, bound, src = f["bytes"] / sec / 1e9, float(peaks["hbm_gbs"]), "GB/s", "hbm", peaks["_source"]
        elif fam == "schur" and form in ("tf32", "bf16"):
            ach, unit, bound = f["flops"] / sec / 1e12, "TFLOP/s", "tensor"
            pk = TF32_TENSOR_TFLOPS if form == "tf32" else float(peaks["bf16_tflops"])
            src = "measured cuBLAS tf32 probe" if form == "tf32" else peaks["_source"] + " bf16"
        else:
            ach, pk, unit, bound, src = f["flops"] / sec / 1e12, FP32_ALU_TFLOPS, "TFLOP/s", "alu", "derived fp32"
        out[fam] = {"ms": round(f["ms"], 3), "bound": bound, "achieved": round(ach, 3), "peak": pk, "unit": unit,
                    "frac": round(ach / pk, 5), "peak_source": src}
    return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


ORACLE_GOLDEN = os.path.join("tests", "golden", "oracle_lapl3d_64.json")


def x_vs_oracle(xs_by_form: dict) -> dict:
    """Relative error of x against the FP64 oracle's x on the benchmark
    workload, on the 256 sampled entries (and ||x||) that the oracle's run
    stored (written by tests/golden/make_oracle_lapl3d_64.py, which calls
    only the oracle; same problem and right-hand side as this benchmark)."""
    import numpy as np
    with open(os.path.join(ROOT, ORACLE_GOLDEN)) as f:
        g = json.load(f)
    idx = np.asarray(g["sample_idx"], dtype=np.int64)
    ref = np.asarray(g["sample_x"], dtype=np.float64)
    out = {"samples": int(idx.size), "oracle_iters": int(g["iters"]), "source": ORACLE_GOLDEN}
    for name, x in xs_by_form.items():
        x = np.asarray(x, dtype=np.float64)
        out[name] = {"sampled_rel_err": float(np.linalg.norm(x[idx] - ref) / np.linalg.norm(ref)),
                     "norm_rel_err": float(abs(np.linalg.norm(x) - g["x_norm"]) / g["x_norm"])}
    return out


def max_over_ranks(vals, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings over the process group (the
    replicas' whole-job time is the slowest rank's); identity without one."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    import torch
    tt = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return tt.tolist()


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle, as it stands, on the same workload
    and metric.  The analysis runs once (t_P is not part of the metric); then
    full-size factorizations + PCG solves are timed one after another, as
    many of the requested steps as fit in REF_BUDGET_S of wall time (a step
    takes tens of seconds on one host core).  The oracle has nothing to warm
    up (no compilation or caches carried between runs), so no untimed step
    runs; `steps` and `warmup` state what was actually done."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    run = oracle_runs(steps=args.steps, budget_s=args.ref_budget, grid=args.grid, levels=args.levels)
    st = run["steps"]
    times = [x["t_f"] + x["t_s"] for x in st]
    v = statistics.mean(times)
    ph = oracle_phases(run)
    import numpy as np  # noqa: F401  (the oracle's dependency; the reference arm needs no GPU)
    from paper_1901_02971_gb300 import inputs as I
    p = I.laplacian_3d(args.grid)
    sample = (f"the whole workload: FP64 oracle factorization + PCG on the {args.grid}^3 cube (L={args.levels}), "
              f"{len(st)} full-size runs one after another on 1 host core ({cpu_model()}); analysis once "
              f"(t_P {run['t_p']:.1f} s, not in the metric); {len(st)} of the {args.steps} requested steps fit "
              f"in the {args.ref_budget:.0f} s budget")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
           "steps": len(st), "warmup": 0, "steps_requested": args.steps, "warmup_requested": args.warmup,
           "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": workload_config(p.n, p.nnz, levels=args.levels, grid=args.grid, world=args.gpus),
           "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
                            "phases": ph, "step_times_s": [round(t, 3) for t in times]},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def extra_configs(peaks: dict, budget_s: float = 240.0) -> dict:
    """The other workloads of the benchmark family, one factorization + PCG
    each (after one untimed warm-up factorization that allocates the
    device memory), with the paper's metrics: t_F, t_S, n_CG, size_Top,
    mem_F, and the per-phase rooflines of a profiled run.
      * 3D diffusion, a = 10^U(-3,3) per 8^3 block, 128^3 cells, L = 13,
        eps 1e-1 / 1e-2 / 1e-3, FP64 / FP32 / BF16 factors;
      * graph Laplacian of the 10-NN graph of 10^6 random points (+1e-4 I),
        no coordinates, L = 12, eps 1e-2, FP32 factor;
      * the batch of 32 independent 2D diffusion problems (128^2 .. 512^2,
        log-normal a), analyzed together and factorized / solved
        concurrently (one stream each), FP32 factors, with the backward pass
        (adjoint solves and dL/dA) of loss = sum ||x_i - y_i||^2.
    Stops adding workloads once `budget_s` of wall time is spent."""
    import numpy as np
    import torch

    from paper_1901_02971_gb300 import Solver, SpandError, factorize_all, solve_all
    from paper_1901_02971_gb300 import inputs as I
    t_start = time.perf_counter()
    out = {}

    def one(p, coords, tag, **kw):
        s = Solver.from_problem(p, use_coords=coords, tol=1e-10, maxit=500, **kw)
        try:
            b = torch.from_numpy(I.rhs(p.n, SEED)).cuda()
            s.factorize()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.factorize()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            x, it, rr = s.solve(b, check=False)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            st = s.stats()
            s.reset_kernel_profile()
            s.set_profiling(True)
            s.factorize()
            s.solve(b, check=False)
            torch.cuda.synchronize()
            s.set_profiling(False)
            form = kw.get("precision", "fp64")
            pr = phase_rooflines(s.kernel_profile(), peaks, form)
            return {"t_f_s": t1 - t0, "t_s_s": t2 - t1, "n_cg": it, "relres": rr, "size_top": st.size_top,
                    "mem_f": st.mem_f, "t_p_s": st.t_analyze_s, "phase_rooflines": pr}
        except SpandError as e:
            return {"error": str(e)[:200]}
        finally:
            s.close()

    def left():
        return budget_s - (time.perf_counter() - t_start)

    try:
        p = I.diffusion_3d(128, 2)
        c3 = {}
        for eps in (1e-1, 1e-2, 1e-3):
            for form in ("fp64", "fp32", "bf16"):
                if left() <= 0:
                    break
                c3[f"eps{eps:g}_{form}"] = one(p, True, "diff3d_128", levels=13, eps=eps, precision=form)
        out["diff3d_128^3_L13"] = {"N": p.n, "nnz": p.nnz, "runs": c3}
        del p
    except Exception as e:  # reported, never fatal to the headline line
        out["diff3d_128^3_L13"] = {"error": str(e)[:300]}
    try:
        if left() > 0:
            t0 = time.perf_counter()
            p = I.knn_laplacian(1_000_000, 10, 3)
            gen = time.perf_counter() - t0
            r = one(p, False, "knn", levels=12, eps=1e-2, precision="fp32")
            r["generation_s"] = gen
            out["knn_1e6_k10_L12"] = dict(N=p.n, nnz=p.nnz, **r)
            del p
    except Exception as e:
        out["knn_1e6_k10_L12"] = {"error": str(e)[:300]}
    try:
        if left() > 0:
            from paper_1901_02971_gb300.autograd import spand_solve
            items = [I.batch_diffusion_2d(i) for i in range(32)]
            probs = [it[0] for it in items]
            opts = [dict(levels=it[3], eps=1e-2, precision="fp32", tol=1e-10) for it in items]
            t0 = time.perf_counter()
            solvers = Solver.batch(probs, opts)
            t_p = time.perf_counter() - t0
            try:
                bs = [torch.from_numpy(it[2]).cuda() for it in items]
                factorize_all(solvers)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                factorize_all(solvers)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                res = solve_all(solvers, bs)
                torch.cuda.synchronize()
                t3 = time.perf_counter()
                # backward of loss = sum ||x_i - y_i||^2 (adjoint solves + dL/dA), values unchanged
                vals = [torch.from_numpy(p.vals).cuda().requires_grad_(True) for p in probs]
                bv = [b.clone().requires_grad_(True) for b in bs]
                for s, v in zip(solvers, vals):
                    s._vals_version, s._vals_stamp = v, v._version
                ys = [torch.from_numpy(it[1] + 0.01 * I.rhs(p.n, 200 + i)).cuda()
                      for i, (it, p) in enumerate(zip(items, probs))]
                torch.cuda.synchronize()
                t4 = time.perf_counter()
                loss = sum(((spand_solve(v, b, s) - y) ** 2).sum() for v, b, s, y in zip(vals, bv, solvers, ys))
                loss.backward()
                torch.cuda.synchronize()
                t5 = time.perf_counter()
                its = [r[1] for r in res]
                out["batch32_diff2d"] = {"N_total": int(sum(p.n for p in probs)), "t_p_s": t_p, "t_f_s": t2 - t1,
                                         "t_s_s": t3 - t2, "n_cg_max": int(max(its)), "n_cg_mean": float(np.mean(its)),
                                         "relres_max": float(max(r[2] for r in res)),
                                         "forward_backward_s": t5 - t4,
                                         "note": "concurrent factorizations / solves, one CUDA stream per problem; "
                                                 "forward+backward re-solves every problem then runs its adjoint "
                                                 "solve and the sampled dL/dA kernel"}
            finally:
                for s in solvers:
                    s.close()
    except Exception as e:
        out["batch32_diff2d"] = {"error": str(e)[:300]}
    out["wall_s"] = time.perf_counter() - t_start
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra-configs", action="store_true",
                    help="skip the 128^3 diffusion, 10^6-point kNN and 32-problem batch workloads")
    ap.add_argument("--ref-budget", type=float, default=REF_BUDGET_S,
                    help="wall-clock budget (s) of the reference arm's full-size oracle steps")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the skip sweep, the simultaneous order and the other compressions (profiling runs)")
    ap.add_argument("--grid", type=int, default=GRID, help="cube edge (small cases for profiling only)")
    ap.add_argument("--levels", type=int, default=LEVELS)
    ap.add_argument("--form", default="tf32", choices=["fp32", "tf32", "bf16"],
                    help="mixed form that is timed and reported as the headline (FP32 factor; Schur GEMMs on the "
                         "SIMT pipes, or on the tensor cores with TF32 / BF16 operands)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    rank, world, local = dist_env()
    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and (args.grid, args.levels) == (GRID, LEVELS):
        cpu = oracle_runs(steps=1)  # the whole workload, once, 1 thread; before any CUDA work here
        ncores = os.cpu_count() or 1
        try:
            cpu_all = (oracle_runs(steps=1, workers=ncores), ncores) if ncores > 1 else None
        except RuntimeError as e:  # reported, never fatal to the headline line
            cpu_all = ({"error": str(e)[-300:]}, ncores)
    import numpy as np
    import torch

    from paper_1901_02971_gb300 import Solver
    from paper_1901_02971_gb300 import build as B
    from paper_1901_02971_gb300 import inputs as I

    B.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    p = I.laplacian_3d(args.grid)
    b = I.rhs(p.n, SEED)
    levels = args.levels
    workload = WORKLOAD if (args.grid, levels) == (GRID, LEVELS) else f"lapl3d_{args.grid}^3_7pt_L{levels}_eps1e-2"
    if workload != WORKLOAD:
        args.no_cpu_baseline = True
    vals_d = torch.from_numpy(p.vals).cuda()
    b_d = torch.from_numpy(b).cuda()
    x_d = torch.empty_like(b_d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def run_form(precision, steps, warmup, timed_clocks=False, skip=0, order="coloured", **kw):
        s = Solver.from_problem(p, levels=levels, eps=EPS, precision=precision, skip=skip, sparsify_order=order,
                                **kw)
        for _ in range(warmup):
            s.factorize(vals_d)
            s.solve(b_d, x_d)
        times, iters = [], []
        l0 = s.launch_count()
        clk = Clocks(local) if timed_clocks else None
        if clk:
            clk.__enter__()
        barrier()
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            s.factorize(vals_d)
            _, it, rr = s.solve(b_d, x_d)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
            iters.append(it)
        barrier()
        launches = (s.launch_count() - l0) / max(steps, 1)
        if clk:
            clk.__exit__(None, None, None)
        return s, times, iters, rr, (clk.summary() if clk else None), launches

    def kernel_profile(s):
        """One extra factor+solve with per-family CUDA events (not part of the
        timed steps); returns the family table."""
        s.reset_kernel_profile()
        s.set_profiling(True)
        flush.zero_()
        torch.cuda.synchronize()
        s.factorize(vals_d)
        s.solve(b_d, x_d)
        torch.cuda.synchronize()
        s.set_profiling(False)
        return s.kernel_profile()

    s32, t32, it32, rr32, clocks, launches32 = run_form(args.form, args.steps, args.warmup, timed_clocks=True)
    st32 = s32.stats()
    ph32 = s32.phase_times()
    prof32 = kernel_profile(s32)
    s64, t64, it64, rr64, _, _ = run_form("fp64", max(1, args.fp64_steps), 1)
    # skip sweep of the mixed form (a performance knob: no scaling or
    # sparsification for the first `skip` steps)
    sweep = {"0": {"s_per_step": statistics.mean(t32), "iters": it32[-1], "size_top": s32.stats().size_top,
                   "mem_f": s32.stats().mem_f}}
    for sk in (() if args.headline_only else (2, 4)):
        ss, ts, its, _, _, _ = run_form(args.form, 2, 1, skip=sk)
        sst = ss.stats()
        sweep[str(sk)] = {"s_per_step": statistics.mean(ts), "iters": its[-1], "size_top": sst.size_top,
                          "mem_f": sst.mem_f}
        ss.close()
    # the simultaneous sparsification order (an option: every interface of a
    # level compressed from the same scaled matrix in one launch), same form
    try:
        if args.headline_only:
            raise RuntimeError("not run (--headline-only)")
        ssim, tsim, itsim, rrsim, _, _ = run_form(args.form, 2, 1, order="simultaneous")
        phs = ssim.phase_times()
        sim = {"s_per_step": statistics.mean(tsim), "iters": itsim[-1], "relres": rrsim,
               "t_factor_ms_phases": list(phs[:4]), "size_top": ssim.stats().size_top, "mem_f": ssim.stats().mem_f}
        ssim.close()
    except Exception as e:  # reported, never fatal to the headline line
        sim = {"error": str(e)[:300]}
    # the other compressions of the interfaces, same form and workload: the
    # randomized range finder (sketch in place of the QR of A_pn) and the
    # interpolative variants InS / In (Sec. 2.6.2)
    alt = {}
    for name, kw in (() if args.headline_only else
                     (("randomized", {"compression": "randomized", "sketch_seed": 7}),
                      ("InS", {"variant": "InS"}), ("In", {"variant": "In"}))):
        try:
            sa, ta, ita, rra, _, _ = run_form(args.form, 2, 1, **kw)
            pha = sa.phase_times()
            alt[name] = {"s_per_step": statistics.mean(ta), "iters": ita[-1], "relres": rra,
                         "t_factor_ms_phases": list(pha[:4]), "apply_ms": pha[4], "size_top": sa.stats().size_top,
                         "mem_f": sa.stats().mem_f}
            sa.close()
        except Exception as e:  # reported, never fatal to the headline line
            alt[name] = {"error": str(e)[:300]}
    st64 = s64.stats()
    ph64 = s64.phase_times()
    # accuracy of x of each form against each other (FP64 reference on the GPU)
    x32 = s32.solve(b_d)[0].cpu().numpy()
    x64 = s64.solve(b_d)[0].cpu().numpy()
    relres_host = float(np.linalg.norm(b - p.to_scipy() @ x32) / np.linalg.norm(b))
    vs_oracle = None
    if workload == WORKLOAD:
        try:
            vs_oracle = x_vs_oracle({"mixed_" + args.form: x32, "plain_fp64": x64})
        except (OSError, KeyError, ValueError) as e:
            vs_oracle = {"error": str(e)[:200]}
    # end to end through the C ABI with host buffers
    x_h = np.empty(p.n)
    e2e = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s32.factorize(p.vals)
        s32.solve(b, x_h)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e.append(time.perf_counter() - t0)
    v = statistics.mean(t32)
    ve = statistics.mean(e2e)
    v, ve = max_over_ranks([v, ve], dist, "cuda")
    if rank != 0:
        return 0
    peaks = load_peaks()
    roofline = make_roofline(prof32, peaks, grid=args.grid)
    extras = None
    if rank == 0 and not args.no_extra_configs and workload == WORKLOAD:
        s32.close()
        s64.close()
        extras = extra_configs(peaks)
    out = {
        "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32 factor; f64 pivot Cholesky, PCG, SpMV",
                  "tf32": "f32 factor (tf32 Schur operands); f64 pivot Cholesky, PCG, SpMV",
                  "bf16": "f32 factor (bf16 Schur operands); f64 pivot Cholesky, PCG, SpMV"}[args.form],
        "data": "synthetic",
        "config": workload_config(p.n, p.nnz, levels=levels, grid=args.grid, world=world),
        "factor": {"fp32": "fp32 storage, fp32 solves/GEMMs/QR", "tf32": "fp32 storage, Schur GEMMs tf32 on tensor cores",
                   "bf16": "fp32 storage, Schur GEMMs bf16 on tensor cores"}[args.form] +
                  "; pivot and scaling Cholesky fp64; PCG, dots and SpMV fp64",
        "forms": {
            "mixed_" + args.form: {"s_per_step": v, "iters": it32[-1], "relres": rr32, "t_factor_ms_phases": list(ph32[:4]),
                           "apply_ms": ph32[4], "size_top": st32.size_top, "mem_f": st32.mem_f,
                           "factor_gflop": st32.factor_flops / 1e9},
            "plain_fp64": {"s_per_step": statistics.mean(t64), "iters": it64[-1], "relres": rr64,
                           "t_factor_ms_phases": list(ph64[:4]), "apply_ms": ph64[4], "size_top": st64.size_top,
                           "mem_f": st64.mem_f, "factor_gflop": st64.factor_flops / 1e9},
            "speedup_mixed_vs_fp64": statistics.mean(t64) / v,
            "x_rel_diff_mixed_vs_fp64": float(np.linalg.norm(x32 - x64) / np.linalg.norm(x64)),
            "true_relres_host": relres_host,
            "x_vs_fp64_oracle": vs_oracle,
            "skip_sweep_mixed_" + args.form: sweep,
            "mixed_" + args.form + "_simultaneous_order": sim,
            "mixed_" + args.form + "_compressions": alt,
        },
        "e2e": {"value": ve, "unit": "s", "h2d_bytes_per_step": int(p.nnz * 8 + p.n * 8),
                "d2h_bytes_per_step": int(p.n * 8)},
        "clocks": clocks,
        "roofline": roofline,
        "gpu_launches": int(round(launches32)),
        "kernel_families_ms": {k: round(v["ms"], 3) for k, v in prof32.items()},
        "phase_rooflines": phase_rooflines(prof32, peaks, args.form),
        "peaks_source": peaks["_source"],
    }
    if extras is not None:
        out["other_workloads"] = extras
    if cpu is not None:
        ph = oracle_phases(cpu)
        cv = ph["t_f_s"] + ph["t_s_s"]
        out["cpu_baseline"] = {"value": cv, "unit": "s", "cores": 1, "kind": "oracle",
                               "sample": f"the whole workload, once: FP64 oracle factorization + PCG on the 64^3 "
                                         f"cube (L={LEVELS}) on 1 host core ({cpu_model()}), {ph['n_cg']} "
                                         f"iterations; analysis t_P {ph['t_p_s']:.1f} s not in the metric",
                               "phases": ph}
    if cpu_all is not None:
        run_all, ncores = cpu_all
        if "error" in run_all:
            out["cpu_baseline_all_cores"] = {"error": run_all["error"], "cores": ncores}
        else:
            pa = oracle_phases(run_all)
            out["cpu_baseline_all_cores"] = {
                "value": pa["t_f_s"] + pa["t_s_s"], "unit": "s", "cores": ncores, "kind": "oracle",
                "sample": f"the whole workload, once: the oracle's factorization with the independent blocks of "
                          f"each level and colour on a pool of {ncores} processes (spawn; blocks pickled to and "
                          f"from the workers; oracle/spand_parallel.py), then the serial PCG; "
                          f"{pa['n_cg']} iterations; analysis t_P {pa['t_p_s']:.1f} s not in the metric",
                "phases": pa}
    print(json.dumps(out))
    s32.close()
    s64.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
