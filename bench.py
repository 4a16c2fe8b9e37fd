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
# bounded oracle sample: the same family at 32^3 (L = 7 keeps the 8^3 leaves),
# scaled to the 64^3 unit by the N log N factorization cost ratio (Sec. 3.3)
SAMPLE_GRID, SAMPLE_LEVELS = 32, 7


def _nlogn(n):
    return n * math.log2(n)


SAMPLE_SCALE = _nlogn(GRID ** 3) / _nlogn(SAMPLE_GRID ** 3)


def oracle_sample_seconds(threads: int = 1) -> dict:
    """Runs the FP64 oracle once on the bounded sample in a fresh process
    (spawned before any CUDA work) whose BLAS/LAPACK calls use `threads`
    threads; returns its wall time."""
    code = (
        "import os,sys,time,json;sys.path.insert(0,%r)\n"
        "from paper_1901_02971_gb300 import inputs as I\n"
        "from oracle import spand_oracle as O\n"
        "p=I.laplacian_3d(%d);b=I.rhs(p.n,%d)\n"
        "t0=time.perf_counter();tr=O.analyze(p.n,p.rowptr,p.colind,p.coords,%d);t1=time.perf_counter()\n"
        "F=O.factorize(p.rowptr,p.colind,p.vals,tr,%r);t2=time.perf_counter()\n"
        "A=O.permuted_matrix(p.rowptr,p.colind,p.vals,tr.perm)\n"
        "x,it,rr=O.pcg(A,b[tr.perm],lambda r:O.apply(F,r));t3=time.perf_counter()\n"
        "print(json.dumps(dict(t_p=t1-t0,t_f=t2-t1,t_s=t3-t2,iters=it,relres=rr)))\n"
    ) % (ROOT, SAMPLE_GRID, SEED, SAMPLE_LEVELS, EPS)
    t = str(int(threads))
    env = dict(os.environ, OPENBLAS_NUM_THREADS=t, OMP_NUM_THREADS=t, MKL_NUM_THREADS=t)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def sample_phases(r: dict) -> dict:
    """The oracle sample's own phase times and PCG count (unscaled): analysis
    t_P, factorization t_F, PCG t_S (s), iterations n_CG."""
    return {"t_p_s": round(r["t_p"], 4), "t_f_s": round(r["t_f"], 4), "t_s_s": round(r["t_s"], 4),
            "n_cg": int(r["iters"])}


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
MEASURED_TRAFFIC = {
    "cpqr": {"bytes_per_launch": (583.4e6 + 13.8e6) / 212,
             "src": ["paper_1901_02971_gb300/csrc/cpqr_cluster.cuh", "paper_1901_02971_gb300/csrc/cpqr_reg.cuh"],
             "sha256": ["354ec7fda5fb9373049b5f2a1946c215d720f4dd2c38934a2327d32eada75f44",
                        "836df7b7d270b09faac01137e4b748a8b7b66bba747ef1eb9b66b4622ec27290"]},
    "apply": {"bytes_per_launch": (2070.9e6 + 27.7e6) / 2, "src": "paper_1901_02971_gb300/csrc/solve_kernels.cuh",
              "sha256": "d0f0fe613eb473dc7d77d8c65ee86cd5bf0c489ba06b3025e26d980cc3300dda"},
}


def measured_traffic(fam: str, grid: int):
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
    return t["bytes_per_launch"]


def make_roofline(prof: dict, peaks: dict, dtype_peak_tflops: float = FP32_ALU_TFLOPS, grid: int = GRID) -> dict:
    """Roofline of the kernel family with the largest device time in one
    profiled factor+solve: achieved = algorithmic flops (or bytes) of its
    launches / their CUDA-event duration."""
    fam = max(prof, key=lambda k: prof[k]["ms"])
    f = prof[fam]
    sec = f["ms"] / 1e3
    traffic = measured_traffic(fam, grid)
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
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    times, iters, last = [], [], None
    for i in range(args.warmup + args.steps):
        r = oracle_sample_seconds()
        if i >= args.warmup:
            times.append((r["t_f"] + r["t_s"]) * SAMPLE_SCALE)
            iters.append(r["iters"])
            last = r
    v = statistics.mean(times)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "l2": "inputs larger than L2 (factor > 129 MB)"},
           "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                            "sample": f"FP64 oracle factor+PCG on the {SAMPLE_GRID}^3 cube (L={SAMPLE_LEVELS}), "
                                      f"scaled x{SAMPLE_SCALE:.2f} by N log N to 64^3; iters {iters[0]}",
                            "sample_phases": sample_phases(last)},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2)
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
        cpu = oracle_sample_seconds()  # before any CUDA work in this process
        cpu_all = oracle_sample_seconds(os.cpu_count() or 1)
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

    def run_form(precision, steps, warmup, timed_clocks=False, skip=0, order="coloured"):
        s = Solver.from_problem(p, levels=levels, eps=EPS, precision=precision, skip=skip, sparsify_order=order)
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
    for sk in (2, 4):
        ss, ts, its, _, _, _ = run_form(args.form, 2, 1, skip=sk)
        sst = ss.stats()
        sweep[str(sk)] = {"s_per_step": statistics.mean(ts), "iters": its[-1], "size_top": sst.size_top,
                          "mem_f": sst.mem_f}
        ss.close()
    # the simultaneous sparsification order (an option: every interface of a
    # level compressed from the same scaled matrix in one launch), same form
    try:
        ssim, tsim, itsim, rrsim, _, _ = run_form(args.form, 2, 1, order="simultaneous")
        phs = ssim.phase_times()
        sim = {"s_per_step": statistics.mean(tsim), "iters": itsim[-1], "relres": rrsim,
               "t_factor_ms_phases": list(phs[:4]), "size_top": ssim.stats().size_top, "mem_f": ssim.stats().mem_f}
        ssim.close()
    except Exception as e:  # reported, never fatal to the headline line
        sim = {"error": str(e)[:300]}
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
    out = {
        "metric": METRIC, "value": v, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": v * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "f32 (tf32 Schur operands)", "bf16": "f32 (bf16 Schur operands)"}[args.form],
        "data": "synthetic",
        "config": {"workload": workload, "N": p.n, "nnz": p.nnz, "levels": levels, "eps": EPS,
                   "factor": {"fp32": "fp32 (mixed)", "tf32": "fp32, Schur GEMMs tf32 on tensor cores",
                              "bf16": "fp32, Schur GEMMs bf16 on tensor cores"}[args.form] + ", PCG fp64",
                   "parallelism": f"replicas x{world}",
                   "l2": "256 MB L2 flush between timed steps; factor data > 129 MB"},
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
    if cpu is not None:
        cv = (cpu["t_f"] + cpu["t_s"]) * SAMPLE_SCALE
        out["cpu_baseline"] = {"value": cv, "unit": "s", "cores": 1, "kind": "oracle",
                               "sample": f"FP64 oracle factor+PCG on the {SAMPLE_GRID}^3 cube (L={SAMPLE_LEVELS}, "
                                         f"{cpu['t_f'] + cpu['t_s']:.2f} s, {cpu['iters']} iters), scaled "
                                         f"x{SAMPLE_SCALE:.2f} (N log N) to 64^3",
                               "sample_phases": sample_phases(cpu)}
        ca = (cpu_all["t_f"] + cpu_all["t_s"]) * SAMPLE_SCALE
        out["cpu_baseline_all_cores"] = {
            "value": ca, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"the same sample with the oracle's BLAS/LAPACK on all {os.cpu_count()} host cores "
                      f"({cpu_all['t_f'] + cpu_all['t_s']:.2f} s), scaled x{SAMPLE_SCALE:.2f}",
            "sample_phases": sample_phases(cpu_all)}
    print(json.dumps(out))
    s32.close()
    s64.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
