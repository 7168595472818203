"""Benchmark: H-LU of the n = 20480 unit-sphere BEM H-matrix and the solve of
16 right-hand sides to a 1e-10 relative residual on one GB300.

One step = hlu_factor (the whole H-LU task graph) + hlu_solve_refined (solves
with the factors, FP64 residual H-matvec, update, until every column reaches
||b - A_H x|| <= 1e-10 ||b||).  The headline arm stores and computes the
factors in FP32 and runs the SVD of every truncation core (QR of R'^T and the
one-sided Jacobi) in FP64; the FP64 arm and the variant with an FP32 Jacobi
are timed beside it, and the factorisation error E_fac of every arm's factors
is estimated on the device (hlu_factor_error).  Inputs (the H-matrix and
b) are resident in HBM when the timed region starts; the working set (factor
arena >= 4 GB) is far larger than the 129 MB L2, so no L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 runs under torch.distributed.run: one independent replica per GPU (the
factorisation does not shard), barrier + max-over-ranks timing, value = the
model flops of all ranks / that time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "H-LU GFLOP/s & solves/s to 1e-10 residual, FP32-TC+IR vs FP64; p50/p99 latency"
WORKLOAD = "sphere20480"  # icosphere r=5, n=20480, leaf 64, eta=2, eps=1e-4, 16 rhs
TOL = 1e-10
KIND_NAMES = ("getrf", "trsm", "project", "accum", "radd", "split")
GEOMETRY = {3: "unit-sphere surface, kernel 1/(4 pi r),", 2: "circle of radius 1/2, kernel -log(r)/(2 pi),",
            1: "interval [0, 1], kernel -log(r),"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=("native", "reference"))
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison arm")
    ap.add_argument("--solver", default="ir", choices=("ir", "gmres"),
                    help="FP64 iteration preconditioned by the factors: refinement or GMRES(restart)")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--tensor", action="store_true",
                    help="FP32 factors: dense products of the factorisation on the tensor cores (tcgen05)")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the n = 81920 leg (GMRES(30), eps 1e-6, 64 rhs) reported in the sphere20480 line")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the batched (ellipsoids64) and serving (serve64r5) legs reported in the sphere20480 "
                         "line")
    ap.add_argument("--construct", action="store_true",
                    help="time the construction of the workload's H-matrix on the GPU (hlu_bem_build)")
    return ap.parse_args()


class RankOps:
    """Barrier and max / sum over the replicas of a multi-GPU run (one rank per GPU, each rank an
    independent H-LU: no collective on the data path, only these scalar reductions of the timing and
    the work). `device` is where the scalar lives: "cuda" for NCCL, "cpu" for gloo."""

    def __init__(self, world, device):
        self.world, self.device = world, device

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def _reduce(self, v, op):
        if self.world == 1:
            return v
        import torch
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=op)
        return t.item()

    def max(self, v):
        import torch.distributed as dist
        return self._reduce(v, dist.ReduceOp.MAX) if self.world > 1 else v

    def sum(self, v):
        import torch.distributed as dist
        return self._reduce(v, dist.ReduceOp.SUM) if self.world > 1 else v


def aggregate(total_ms_per_rank_max, work_per_rank_sum):
    """Whole-job throughput of weak-scaled replicas: the work of all ranks over the slowest rank's time."""
    return work_per_rank_sum / (total_ms_per_rank_max * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- CPU side
CPU_SAMPLE_N = 5120    # CPU baseline: the leading diagonal block of about this many unknowns
REF_SAMPLE_N = 2560    # reference arm: a smaller block per step (bounded run time)


def sample_level(n, target):
    """Cluster-tree level whose leading block has about `target` unknowns (bisection halves n)."""
    import math
    return max(0, int(round(math.log2(max(n, 1) / target))))


def _oracle_sample_worker(workload, level, reps):
    """Run in a single-threaded subprocess: FP64 oracle H-LU of one diagonal block."""
    import numpy as np
    from bem_inputs import WORKLOADS, build_problem
    from bem_inputs.problem import sub_problem
    from oracle import HLUOracle
    w = WORKLOADS[workload]
    p = build_problem(**w)
    c = int(np.flatnonzero(p.tree.level == level)[0])
    q = sub_problem(p, c)
    times, flops = [], 0.0
    for _ in range(reps):
        t0 = time.perf_counter()
        o = HLUOracle(q, q.eps).factor()
        times.append(time.perf_counter() - t0)
        flops = o.c.total()
    print(json.dumps({"n": q.n, "leaves": q.n_leaves, "times": times, "flops": flops}))


def oracle_sample(workload, level, reps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import sys; sys.path.insert(0, %r); import bench; bench._oracle_sample_worker(%r, %d, %d)"
            % (ROOT, workload, level, reps))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_info():
    """The host CPU as lscpu names it, and the hardware threads."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                if not model.isdigit():
                    break
    except Exception:
        pass
    return {"cpu_model": model, "nproc": os.cpu_count()}


def _oracle_full_worker(workload):
    """Run in a subprocess (its thread count set by the caller): the FP64 oracle's H-LU and solve of a
    whole named workload."""
    from bem_inputs import WORKLOADS, build_problem
    from oracle import HLUOracle
    from oracle.errors import lu_solve
    p = build_problem(**WORKLOADS[workload])
    t0 = time.perf_counter()
    o = HLUOracle(p, p.eps).factor()
    t1 = time.perf_counter()
    lu_solve(o.A, p.b_perm())
    t2 = time.perf_counter()
    print(json.dumps({"n": p.n, "leaves": p.n_leaves, "factor_s": t1 - t0, "solve_s": t2 - t1,
                      "flops": o.c.total()}))


def oracle_full(workload, threads):
    """The whole workload on the oracle: `threads` = 1 (one core) or the host's cores (numpy's BLAS
    on all of them; the oracle's recursion itself is sequential)."""
    t = str(int(threads))
    env = dict(os.environ, OMP_NUM_THREADS=t, OPENBLAS_NUM_THREADS=t, MKL_NUM_THREADS=t, CUDA_VISIBLE_DEVICES="")
    code = "import sys; sys.path.insert(0, %r); import bench; bench._oracle_full_worker(%r)" % (ROOT, workload)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle run failed:\n" + r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    res["threads"] = int(threads)
    res["gflops"] = res["flops"] / (res["factor_s"] + res["solve_s"]) / 1e9
    return res


def workload_config(args, w, p, world):
    """The `config` of a single-problem line (the same for the native and the reference arm)."""
    return {"workload": f"{args.workload}: {GEOMETRY[w.get('dim', 3)]} n={p.n}, leaf {w['leaf']}, "
                        f"eta={w['eta']:g}, eps={w['eps']:g}, {p.nrhs} rhs ~ N(0,1) seed 0, tol 1e-10",
            "n": p.n, "leaves": p.n_leaves, "nrhs": p.nrhs,
            "l2": f"inputs larger than L2 (A_H leaf data {p.data.nbytes / 1e9:.2f} GB)",
            "parallelism": f"replicas x{world}",
            "solver": f"GMRES({args.restart})" if args.solver == "gmres" else "iterative refinement"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    reps = args.warmup + args.steps
    from bem_inputs import WORKLOADS, build_problem
    w = dict(WORKLOADS[args.workload])
    p = build_problem(**w)  # the configuration's H-matrix (cached on disk after the first build)
    level = sample_level(p.n, REF_SAMPLE_N)
    res = oracle_sample(args.workload, level, reps)
    ts = res["times"][args.warmup:]
    step = sum(ts) / len(ts)
    gflops = res["flops"] / step / 1e9
    sample = (f"each step: FP64 oracle H-LU of the leading level-{level} diagonal block (n={res['n']}, "
              f"{res['leaves']} leaves) of this configuration's H-matrix, factor only, 1 thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": gflops, "unit": "GFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, w, p, args.gpus),
        "cpu_baseline": dict({"value": gflops, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": sample},
                             **cpu_info()),
        "e2e": {"value": gflops, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU side
class ClockSampler:
    """nvidia-smi clock and throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        import statistics
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
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
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def recorded_traffic(dom, a_h_bytes, eps, leaf):
    """DRAM bytes per launch of the factorisation kernel from the committed ncu summary
    (profiles/traffic.json), scaled by A_H bytes; None when the kernel source changed since or
    the workload's truncation tolerance or leaf size differs from the captured one."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        rec = json.load(open(os.path.join(here, "profiles", "traffic.json")))
        src = open(os.path.join(here, rec["source"]), "rb").read()
    except (OSError, ValueError, KeyError):
        return None, "no ncu record"
    if dom != "dataflow_factor":
        return None, "ncu record is for the factorisation kernel"
    if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
        return None, "kernel source changed since the ncu capture"
    if eps != rec["captured_eps"] or leaf != rec["captured_leaf"]:
        return None, "ncu record taken at another truncation tolerance or leaf size"
    dram = rec["dram_bytes_read"] + rec["dram_bytes_write"]
    scale = a_h_bytes / rec["captured_a_h_bytes"]
    return dram * scale, (f"ncu dram bytes of one launch on {rec['captured_workload']} x {scale:.3f} "
                          f"(A_H bytes ratio), {rec['summary']}")


def class_roofline(st, prof, nprof, fp32_peak):
    """Per task class of the factorisation: model flops over the summed task time (the rate of one
    worker CTA while it runs that class) against one worker's share of the FP32 FMA peak
    (two worker CTAs per SM)."""
    import torch
    workers = 2 * torch.cuda.get_device_properties(0).multi_processor_count
    per_worker = fp32_peak * 1e12 / workers
    out = {}
    for k, busy in prof["task_busy_ms"].items():
        fl = st["flops_by_kind"].get(k, 0.0)
        if busy <= 0 or fl <= 0:
            continue
        rate = fl / (busy / nprof * 1e-3)
        out[k] = {"model_gflop": fl / 1e9, "busy_ms": busy / nprof, "gflops_per_worker": rate / 1e9,
                  "frac_of_worker_fp32_peak": rate / per_worker}
    return out


def rank_hist(st):
    """Ranks of the low-rank leaves of L and U after the factorisation: {rank: count}, '>32' last."""
    h = list(st.get("rank_hist", []))
    out = {str(k): int(v) for k, v in enumerate(h[:33]) if v}
    if len(h) > 33 and h[33]:
        out[">32"] = int(h[33])
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


FLAGS = 0  # hlu_opts.flags of every handle the bench makes (--tensor sets FLAG_TENSOR)


def make_handle(p, precision, stream):
    from paper_1906_00874_gb300 import HLU
    return HLU.from_problem(p, precision=precision, stream=stream, flags=FLAGS)


_T_START = time.time()


def _pick(d, keys):
    """The entries of d named by keys ("a.b" reaches into a nested dict); missing ones are left out."""
    out = {}
    for k in keys:
        v, ok = d, True
        for part in k.split("."):
            ok = isinstance(v, dict) and part in v
            if not ok:
                break
            v = v[part]
        if ok:
            out[k] = v
    return out


# The batched and serving workloads as they run alone (their own bench lines), summarised into the
# headline line: each is a child process, so that a failure or a hang there cannot cost this line.
EXTRA_LEGS = (
    ("c4_ellipsoids64", ["--workload", "ellipsoids64", "--steps", "2", "--warmup", "3"],
     ("config.workload", "value", "unit", "ms_per_step", "steps", "warmup", "loop_fp64_ms", "speedup_vs_fp64_loop",
      "worst_problem_resid", "efac_stacked_fp32", "factor_model_gflop", "max_rank", "plan", "e2e.value",
      "e2e.ms_per_step", "roofline.frac", "cpu_baseline.value", "cpu_baseline.unit", "cpu_baseline.sample",
      "gpu_launches", "clocks")),
    ("c5_serve64r5", ["--workload", "serve64r5"],
     ("config.workload", "value", "unit", "p50_ms", "p99_ms", "mean_ms", "capacity_rps", "capacity_burst_rps",
      "arrival_rate_rps", "device_overlap.fraction", "server.groups_created", "server.evicted_groups",
      "latency_breakdown.resident", "latency_breakdown.waited_for_admission", "gpu_launches", "clocks")),
)


def extra_legs(budget_s=480.0, leg_cap_s=300.0):
    """Runs EXTRA_LEGS while the whole bench stays within budget_s seconds of wall time."""
    legs = {}
    for key, argv, keys in EXTRA_LEGS:
        left = min(leg_cap_s, budget_s - (time.time() - _T_START))
        if left < 60.0:
            legs[key] = {"skipped": "bench wall-time budget spent"}
            continue
        try:
            t0 = time.time()
            r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + argv, capture_output=True,
                               text=True, timeout=left, cwd=ROOT)
            line = next((ln for ln in reversed(r.stdout.splitlines()) if ln.startswith("{")), None)
            if r.returncode != 0 or line is None:
                legs[key] = {"error": f"exit {r.returncode}: " + " | ".join(r.stderr.strip().splitlines()[-3:])}
            else:
                legs[key] = _pick(json.loads(line), keys)
                legs[key]["wall_s"] = round(time.time() - t0, 1)
        except subprocess.TimeoutExpired:
            legs[key] = {"error": f"timed out after {left:.0f} s"}
        except Exception as e:  # reported, not fatal
            legs[key] = {"error": f"{type(e).__name__}: {e}"}
    return legs


def run_native(args):
    import numpy as np
    import torch

    from bem_inputs import WORKLOADS, build_problem
    from paper_1906_00874_gb300 import HLU_FP32, HLU_FP32_CORE32, HLU_FP64, build
    from paper_1906_00874_gb300.hlu import probe_alu_peaks, to_device_panel

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    w = dict(WORKLOADS[args.workload])
    p = build_problem(**w)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    b = to_device_panel(p.b)
    x = torch.zeros_like(b)

    ranks = RankOps(world, "cuda")
    barrier, max_over_ranks, sum_over_ranks = ranks.barrier, ranks.max, ranks.sum

    def step(h):
        h.factor(p.eps)
        if args.solver == "gmres":
            it, res = h.solve_gmres(b, x, tol=TOL, restart=args.restart, max_iter=300)
        else:
            it, res = h.solve_refined(b, x, tol=TOL, max_iter=30)
        return it, res

    def timed_arm(h, steps, warmup):
        for _ in range(warmup):
            step(h)
        torch.cuda.synchronize()
        launches0 = h.stats()["kernels_launched"]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        iters, resid = [], []
        barrier()
        torch.cuda.synchronize()
        ev[0].record(stream)
        for i in range(steps):
            it, res = step(h)
            ev[i + 1].record(stream)
            iters.append(it)
            resid.append(res)
        torch.cuda.synchronize()
        barrier()
        per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
        total_ms = ev[0].elapsed_time(ev[steps])
        st = h.stats()
        return {"total_ms": total_ms, "per_step_ms": per, "iters": iters, "resid": resid,
                "launches": st["kernels_launched"] - launches0, "stats": st}

    def flops_per_step(h):
        st = h.stats()  # counters of the last step: factor + its solves/products
        return st["model_flops"] + st["solve_flops"], st

    # ---------------- headline arm: FP32 factors + FP64 refinement
    h32 = make_handle(p, HLU_FP32, sptr)
    with ClockSampler(local) as clk:
        arm32 = timed_arm(h32, args.steps, args.warmup)
    f32, st32 = flops_per_step(h32)
    t_ms = max_over_ranks(arm32["total_ms"])
    total_flops = sum_over_ranks(f32 * args.steps)
    value = aggregate(t_ms, total_flops) / 1e9
    per = sorted(arm32["per_step_ms"])

    def pct(a, q):
        return a[min(len(a) - 1, int(round(q * (len(a) - 1))))]

    # ---------------- profiled pass (per-kernel-class time, same steps)
    h32.set_profiling(True)
    for _ in range(max(1, min(args.steps, 3))):
        step(h32)
    torch.cuda.synchronize()
    prof = h32.stats()
    h32.set_profiling(False)
    nprof = max(1, min(args.steps, 3))

    # factorisation error of the headline factors (device power iteration, FP64 sums)
    step(h32)
    torch.cuda.synchronize()
    efac32 = h32.factor_error()[0]

    def side_arm(precision):
        """A comparison arm on its own handle: time to 1e-10 over a few steps, E_fac of its factors."""
        h = make_handle(p, precision, sptr)
        a = timed_arm(h, max(2, args.steps // 3), max(1, args.warmup // 2))
        fl, st = flops_per_step(h)
        k = len(a["per_step_ms"])
        t = max_over_ranks(a["total_ms"]) / k
        out = {"time_to_1e10_ms": t, "gflops": fl / (t * 1e-3) / 1e9, "ir_iters": a["iters"][-1],
               "resid": a["resid"][-1], "factor_model_gflop": st["model_flops"] / 1e9,
               "max_rank": st["max_rank"], "steps": k, "efac": h.factor_error()[0]}
        h.close()
        return out

    # ---------------- FP64 arm, and FP32 factors with an FP32 Jacobi in the truncation cores
    arm64 = None if args.no_fp64 else side_arm(HLU_FP64)
    core32 = side_arm(HLU_FP32_CORE32)

    # ---------------- end to end through the public API with host buffers
    e2e = e2e_arm(p, HLU_FP32, sptr, min(args.steps, 3), f32, args.solver, args.restart)

    # ---------------- roofline of the dominant kernel (profiled pass, CUDA events on the stream)
    fp64_peak, fp32_peak = probe_alu_peaks()
    ms = prof["kernel_ms"]
    dom = max(ms, key=lambda k: ms[k])
    dom_ms = ms[dom] / nprof
    launches = prof["kernel_launches"][dom] / nprof
    if dom == "dataflow_factor":
        # one persistent launch runs the whole factorisation task graph
        dom_flops = st32["model_flops"]
        kname = "k_dataflow<float> (factorisation)"
    elif dom in ("dataflow_solve", "dataflow_matvec"):
        dom_flops = st32["solve_flops"] * ms[dom] / max(1e-9, ms["dataflow_solve"] + ms["dataflow_matvec"])
        kname = "k_dataflow<float> (H-solves)" if dom == "dataflow_solve" else "k_dataflow<double> (H-matvec)"
    else:
        dom_flops = st32["flops_by_kind"][dom]
        kname = f"k_{dom}<float>"
    achieved = dom_flops / (dom_ms * 1e-3) / 1e12 if dom_ms > 0 else 0.0
    # algorithmic bytes of the factorisation: read A_H once (FP64) and write the factors once (FP32)
    alg_bytes = 1.5 * p.data.nbytes if dom == "dataflow_factor" else None
    hbm_peak = measured_peaks().get("hbm_gbs", 6800.0)
    traffic, traffic_note = recorded_traffic(dom, p.data.nbytes, p.eps, w["leaf"])
    roof = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak if fp32_peak else None, "traffic": traffic,
            "traffic_source": traffic_note,
            "peak_source": "measured FP32 FMA probe (hlu_probe_alu_peaks), of measured",
            "model_gflop_per_launch": dom_flops / 1e9 / max(launches, 1e-9),
            "avg_launch_ms": dom_ms / max(launches, 1e-9), "launches_per_step": launches,
            "share_of_kernel_time": ms[dom] / max(1e-9, sum(ms.values())),
            "hbm_view": None if alg_bytes is None else {
                "alg_bytes_per_launch": alg_bytes,
                "achieved_gbs": alg_bytes / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else 0.0,
                "peak_gbs": hbm_peak, "peak_source": "MEASURED_PEAKS.json hbm_gbs (fallback 6800)"},
            "kernel_ms_per_step": {k: v / nprof for k, v in ms.items()},
            "task_busy_ms_per_factor": {k: prof["task_busy_ms"][k] / nprof for k in KIND_NAMES
                                        if prof["task_busy_ms"][k]},
            # summed over the workers of the factorisation launch: lifetime = tasks + waits on empty
            # queue slots + the executor's own work (claims, successor release, barriers)
            "worker_ms_per_factor": {
                "life": prof["worker_life_ms"] / nprof, "queue_wait": prof["worker_wait_ms"] / nprof,
                "tasks": sum(prof["task_busy_ms"][k] for k in KIND_NAMES) / nprof,
                "executor": (prof["worker_life_ms"] - prof["worker_wait_ms"]
                             - sum(prof["task_busy_ms"][k] for k in KIND_NAMES)) / nprof},
            "classes": class_roofline(st32, prof, nprof, fp32_peak),
            "tasks_per_factor": {k: prof["task_count"][k] // nprof for k in KIND_NAMES if prof["task_count"][k]},
            "active_workers": prof["task_count"]["dataflow_solve"] // max(nprof, 1),
            "radd_busy_ms_by_size": {k: round(v / nprof, 1) for k, v in prof["radd_busy_ms"].items() if v},
            "radd_count_by_size": {k: v // nprof for k, v in prof["radd_count"].items() if v},
            "radd_phases_per_factor": {route: {k: (v if k.startswith("mean_") else v / nprof)
                                               for k, v in ph.items()}
                                       for route, ph in prof["radd_phase"].items()}}

    # ---------------- the n = 81920 configuration (leaves built on the GPU), reported as one key
    c3 = None
    if args.workload == WORKLOAD and not args.no_c3:
        try:
            c3 = c3_leg(sptr, fp32_peak, steps=2)
        except Exception as e:  # reported, not fatal
            c3 = {"error": f"{type(e).__name__}: {e}"}

    cpu = None
    if rank == 0:
        try:
            level = sample_level(p.n, CPU_SAMPLE_N)
            res = oracle_sample(args.workload, level, 1)
            cpu = {"value": res["flops"] / res["times"][0] / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                   "sample": (f"FP64 oracle H-LU (factor only) of the leading level-{level} diagonal "
                              f"block, n={res['n']}, {res['leaves']} leaves, of the same H-matrix; "
                              f"{res['times'][0]:.1f} s on 1 host thread")}
            cpu.update(cpu_info())
            if args.workload == WORKLOAD and not args.no_c3:
                # the whole n = 5120 configuration (factor + solve) on one core and on all of them
                full = {}
                for th in (1, os.cpu_count() or 1):
                    r = oracle_full("sphere5120", th)
                    full["threads_%d" % th] = {k: r[k] for k in ("n", "leaves", "factor_s", "solve_s", "gflops")}
                cpu["full_sphere5120"] = full
        except Exception as e:  # reported, not fatal
            cpu = {"value": None, "unit": "GFLOP/s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}

    legs = None
    if rank == 0 and world == 1 and args.workload == WORKLOAD and not args.no_c3 and not args.no_extra:
        legs = extra_legs()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 factors; f64 Jacobi SVD of every truncation core, f64 residual and solution",
            "data": "synthetic",
            "config": workload_config(args, w, p, world),
            "device_gb": st32["device_bytes"] / 1e9,
            "time_to_1e10_ms": t_ms / args.steps, "solves_per_s": p.nrhs * args.steps * world / (t_ms * 1e-3),
            "p50_ms": pct(per, 0.5), "p99_ms": pct(per, 0.99), "ir_iters": arm32["iters"][-1],
            "rank_hist": rank_hist(st32),
            "resid": max(arm32["resid"]), "factor_model_gflop": st32["model_flops"] / 1e9,
            "step_model_gflop": f32 / 1e9, "max_rank": st32["max_rank"],
            "efac_fp32": efac32, "efac_note": "||A_H - L U||_2 / ||A_H||_2 of each arm's factors, device power "
                                                  "iteration (hlu_factor_error), bound 10 eps",
            "fp64_arm": arm64, "fp32_core32_arm": core32, "e2e": e2e, "gpu_launches": arm32["launches"], "clocks": clk.summary(),
            "roofline": roof, "cpu_baseline": cpu, "c3_sphere81920": c3,
            **(legs or {}),
            "alu_peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak},
            "plan": {"tasks": st32["n_tasks"], "waves": st32["n_waves"], "launches_per_factor": st32["n_launches"]},
        }
        print(json.dumps(line), flush=True)
    h32.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def c3_leg(sptr, fp32_peak, steps=2, restart=30):
    """sphere81920: n = 81920, leaf 64, eta 2, eps 1e-6, 64 rhs.  The block structure is planned on
    the host (mesh, Algorithms 1 and 2); the leaf data are computed on the GPU (hlu_bem_build: dense
    leaves, cross approximation and truncation at eps).  One step = FP32 factorisation (FP64 Jacobi
    SVD in every truncation core) + GMRES(30) in FP64 on A_H to a 1e-10 relative residual for all 64
    right-hand sides; CUDA events around the steps."""
    import torch

    from bem_inputs import WORKLOADS, build_structure
    from paper_1906_00874_gb300 import HLU_FP32
    from paper_1906_00874_gb300.hlu import BEMBuild, to_device_panel
    w = dict(WORKLOADS["sphere81920"])
    t0 = time.perf_counter()
    s = build_structure(**w)
    structure_s = time.perf_counter() - t0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = BEMBuild.from_problem(s)
    torch.cuda.synchronize()
    construct_ms = (time.perf_counter() - t0) * 1e3
    h = g.create(precision=HLU_FP32, stream=sptr, flags=FLAGS, temp_reuse=1)
    create = h.stats()["create_ms"]
    b = to_device_panel(s.b)
    x = torch.zeros_like(b)

    def step():
        h.factor(w["eps"])
        return h.solve_gmres(b, x, tol=TOL, restart=restart, max_iter=300)
    step()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    torch.cuda.synchronize()
    ev[0].record(stream)
    out = []
    for i in range(steps):
        out.append(step())
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    st = h.stats()
    fl = st["model_flops"] + st["solve_flops"]
    efac = h.factor_error()[0]
    h.set_profiling(True)
    step()
    torch.cuda.synchronize()
    prof = h.stats()
    h.set_profiling(False)
    res = {"workload": "sphere81920: unit sphere, n=81920, leaf 64, eta 2, eps 1e-6, 64 rhs ~ N(0,1) seed 0, "
                       "GMRES(30) to 1e-10, leaves built on the GPU",
           "time_to_1e10_ms": sum(per) / len(per), "per_step_ms": per,
           "factor_ms": prof["kernel_ms"]["dataflow_factor"],
           "gmres_steps": out[-1][0], "resid": out[-1][1], "efac": efac,
           "model_gflop_per_step": fl / 1e9, "gflops": fl / (sum(per) / len(per) * 1e-3) / 1e9,
           "solves_per_s": 64 * steps / (sum(per) * 1e-3),
           "rank_hist": rank_hist(st), "max_rank": st["max_rank"], "leaves": int(s.n_leaves),
           "tasks": st["n_tasks"], "device_gb": st["device_bytes"] / 1e9,
           "host_structure_s": structure_s, "gpu_construct_ms": construct_ms, "create_ms": create,
           "classes": class_roofline(st, prof, 1, fp32_peak)}
    h.close()
    g.close()
    return res


def e2e_arm(p, precision, sptr, steps, flops_step, solver="ir", restart=30):
    """Public-API end to end: hlu_create from host arrays (H2D of the H-matrix),
    factor, b from pinned host memory, refinement, x back to pinned host memory."""
    import numpy as np
    import torch

    from paper_1906_00874_gb300 import HLU
    b_host = torch.tensor(np.ascontiguousarray(p.b.T)).pin_memory()  # (nrhs, n) row-major = n x nrhs col-major
    x_host = torch.empty_like(b_host).pin_memory()
    t = p.tree
    h2d = (p.data.nbytes + p.row_cl.nbytes + p.col_cl.nbytes + p.kind.nbytes + p.rank.nbytes + p.offset.nbytes
           + t.perm.nbytes + t.begin.nbytes + t.size.nbytes + t.son0.nbytes + t.son1.nbytes + b_host.numel() * 8)
    d2h = x_host.numel() * 8
    times = []
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = HLU(p.n, t.perm, t.begin, t.size, t.son0, t.son1, p.row_cl, p.col_cl, p.kind, p.rank, p.offset, p.data,
                precision=precision, stream=sptr)
        h.factor(p.eps)
        bd = b_host.to("cuda", non_blocking=True).t()
        xd = torch.zeros_like(bd)
        if solver == "gmres":
            h.solve_gmres(bd, xd, tol=TOL, restart=restart, max_iter=300)
        else:
            h.solve_refined(bd, xd, tol=TOL, max_iter=30)
        x_host.copy_(xd.t(), non_blocking=True)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        create = h.stats()["create_ms"]
        h.close()
    ts = times[1:]  # the first call also pays one-time start-up costs
    sec = sum(ts) / len(ts)
    return {"value": flops_step / sec / 1e9, "unit": "GFLOP/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": sec * 1e3, "create_ms_last": create,
            "includes": f"hlu_create (validation, planning, upload) + factor + "
                        f"{'GMRES' if solver == 'gmres' else 'refinement'} + copies"}


def _structure_one(kw):
    from bem_inputs import build_structure
    return build_structure(**kw)


def build_batch(name):
    """The seeded structures of a named batch (geometry, cluster tree, block-tree leaves and
    right-hand sides; no leaf data), built on all host cores by spawned workers before any CUDA
    call.  The leaf data are computed on the GPU afterwards (construct_leaves)."""
    import multiprocessing as mp

    from bem_inputs import BATCHES, batch_specs
    specs = batch_specs(**BATCHES[name])
    with mp.get_context("spawn").Pool(min(len(specs), os.cpu_count() or 1)) as pool:
        return specs, pool.map(_structure_one, specs, chunksize=1)


def construct_leaves(structs):
    """Leaf data of every structure computed on the GPU (hlu_bem_build: dense leaves, cross
    approximation and truncation at the problem's eps) and copied into the problem (host arrays,
    the input layout of hlu_create_batch)."""
    from paper_1906_00874_gb300.hlu import BEMBuild
    for s in structs:
        g = BEMBuild.from_problem(s)
        s.rank, s.offset, s.data = g.rank.copy(), g.offset.copy(), g.data()
        g.close()
    return structs


def _oracle_batch_worker(name, budget_s):
    """Run in a single-threaded subprocess: the FP64 oracle's H-LU and solve of the batch's smallest
    problems (host-built leaves), one after the other, until `budget_s` seconds are used."""
    import numpy as np
    from bem_inputs import BATCHES, batch_specs, build_problem
    from oracle import HLUOracle
    from oracle.errors import lu_solve
    specs = sorted(batch_specs(**BATCHES[name]), key=lambda kw: kw["r"])
    done, t_all, ns = 0, 0.0, []
    for kw in specs:
        p = build_problem(**kw)
        t0 = time.perf_counter()
        o = HLUOracle(p, p.eps).factor()
        lu_solve(o.A, p.b_perm())
        t_all += time.perf_counter() - t0
        done += 1
        ns.append(p.n)
        if t_all >= budget_s:
            break
    print(json.dumps({"problems": done, "seconds": t_all, "n": sorted(set(ns)), "r": int(specs[0]["r"])}))


def _oracle_one_problem(kw):
    """One problem of a batch on the oracle (a process of the all-cores pool): seconds of H-LU + solve."""
    from bem_inputs import build_problem
    from oracle import HLUOracle
    from oracle.errors import lu_solve
    p = build_problem(**kw)
    t0 = time.perf_counter()
    o = HLUOracle(p, p.eps).factor()
    lu_solve(o.A, p.b_perm())
    return time.perf_counter() - t0


def _oracle_batch_pool_worker(name, count):
    """Run in a subprocess: the batch's `count` smallest problems on the oracle, one single-threaded
    process per host core (the problems are independent); prints the wall time of the pool."""
    import multiprocessing as mp
    from bem_inputs import BATCHES, batch_specs, build_problem
    specs = sorted(batch_specs(**BATCHES[name]), key=lambda kw: kw["r"])[:count]
    for kw in specs:  # build (and cache) the inputs first: only the H-LU and solve are timed
        build_problem(**kw)
    procs = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_one_problem, specs[:procs])  # warm the workers' imports
        t0 = time.perf_counter()
        pool.map(_oracle_one_problem, specs, chunksize=1)
        wall = time.perf_counter() - t0
    print(json.dumps({"problems": len(specs), "seconds": wall, "procs": procs}))


def oracle_batch_pool(name, count):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import sys; sys.path.insert(0, %r); import bench; bench._oracle_batch_pool_worker(%r, %d)"
            % (ROOT, name, int(count)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle batch pool failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_batch_sample(name, budget_s=12.0):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import sys; sys.path.insert(0, %r); import bench; bench._oracle_batch_worker(%r, %r)"
            % (ROOT, name, float(budget_s)))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError("oracle batch sample failed:\n" + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _split_balanced(probs, parts):
    """Problem indices in `parts` groups of about equal leaf counts (largest first, each to the
    lightest group), every group in increasing index order."""
    load, groups = [0] * parts, [[] for _ in range(parts)]
    for i in sorted(range(len(probs)), key=lambda i: -probs[i].n_leaves):
        g = load.index(min(load))
        groups[g].append(i)
        load[g] += probs[i].n_leaves
    return [sorted(g) for g in groups if g]


def run_batch(args):
    """Batched H-LU of many independent problems in one handle (hlu_create_batch: the problems
    planned in parallel on the host, one persistent data-flow launch per factorisation) against a
    loop of per-problem FP64 handles.  One step = factorise every problem (its own eps) and solve its
    right-hand side to a 1e-10 relative residual (FP64 refinement of the stacked block-diagonal
    system).  The launch setting (worker count, product path) is chosen by the tuner on a sample of
    the batch.  Metric: problems solved per second."""
    import concurrent.futures

    import numpy as np
    import torch

    from bem_inputs import BATCHES
    from paper_1906_00874_gb300 import HLU, HLU_FP32, HLU_FP64, build
    from paper_1906_00874_gb300.autotune import candidates, structure_key, tune
    from paper_1906_00874_gb300.hlu import HLUError, probe_alu_peaks, to_device_panel

    rank, world, local = dist_env()
    t0 = time.perf_counter()
    specs, probs = build_batch(args.workload)
    structure_s = time.perf_counter() - t0
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    construct_leaves(probs)
    construct_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    B = len(probs)
    eps = [p.eps for p in probs]
    bn = [float(np.linalg.norm(p.b)) for p in probs]
    ranks = RankOps(world, "cuda")
    barrier, max_over_ranks = ranks.barrier, ranks.max
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    class Part:
        """One batched handle over a subset of the problems, with its stacked b and x."""

        def __init__(self, idx, precision, **kw):
            self.idx = idx
            sub = [probs[i] for i in idx]
            self.h = HLU.batch(sub, precision=precision, stream=sptr, nrhs_max=1, **kw)
            self.b = to_device_panel(np.concatenate([p.b for p in sub], axis=0))
            self.x = torch.zeros_like(self.b)
            nb = [bn[i] for i in idx]
            # stacked tolerance that bounds every problem's own relative residual by 1e-10
            self.tol = TOL * min(nb) / float(np.linalg.norm(nb))
            self.eps = [eps[i] for i in idx]

        def step(self):
            self.h.factor(self.eps)
            return self.h.solve_refined(self.b, self.x, tol=self.tol, max_iter=30)

        def worst_resid(self):
            y = torch.empty_like(self.x)
            self.h.matvec(self.x, y)
            r = (self.b - y).cpu().numpy()[:, 0]
            o, worst = 0, 0.0
            for i in self.idx:
                n = probs[i].n
                worst = max(worst, float(np.linalg.norm(r[o:o + n])) / bn[i])
                o += n
            return worst

    def host_available():
        """Bytes of host memory this process may still use (MemAvailable, and the cgroup limit)."""
        avail = None
        try:
            with open("/proc/meminfo") as f:
                for ln in f:
                    if ln.startswith("MemAvailable:"):
                        avail = int(ln.split()[1]) * 1024
        except OSError:
            pass
        try:
            with open("/sys/fs/cgroup/memory.max") as f:
                lim = f.read().strip()
            with open("/sys/fs/cgroup/memory.current") as f:
                cur = int(f.read().strip())
            if lim != "max":
                avail = min(avail or 1 << 62, int(lim) - cur)
        except (OSError, ValueError):
            pass
        return avail

    def make_parts(precision, **kw):
        """The whole batch in one handle; halves (balanced by leaves) while it does not fit the
        device.  Creating one handle holds, on the host, about 350 bytes per task while it plans (at
        most about 95 tasks per leaf at leaf 32) and two copies of its leaf data while it uploads, so
        the first split also keeps that within 70 % of the host memory available."""
        avail = host_available()
        need = sum(350 * 95 * p.n_leaves + 2 * p.data.nbytes for p in probs)
        first = 1
        while avail is not None and first < 8 and need / first > 0.7 * avail:
            first *= 2
        for parts in (1, 2, 4, 8):
            if parts < first:
                continue
            made = []
            try:
                for idx in _split_balanced(probs, parts):
                    made.append(Part(idx, precision, **kw))
                return made
            except HLUError as e:
                for m in made:
                    m.h.close()
                del made
                torch.cuda.empty_cache()
                if e.status != 2:  # HLU_ENOMEM
                    raise
        raise RuntimeError("the batch does not fit the device even in eight handles")

    # launch setting: tuner trials on a sample of the batch (every third problem, at most 32)
    sample_idx = list(range(0, B, max(1, B // 32)))[:32]
    sample = Part(sample_idx, HLU_FP32, temp_reuse=1)
    cands = candidates(sms, tensor=True)
    choice, trials, _ = tune(sample.h, sample.step, structure_key([probs[i] for i in sample_idx], HLU_FP32),
                             cands, reps=2, use_cache=False)
    sample.h.close()
    del sample
    torch.cuda.empty_cache()

    t0 = time.perf_counter()
    parts32 = make_parts(HLU_FP32, temp_reuse=1)
    create_s = time.perf_counter() - t0
    for part in parts32:
        part.h.set_launch(choice["workers"], choice["flags"])

    def step32():
        return [part.step() for part in parts32]

    l0 = sum(part.h.stats()["kernels_launched"] for part in parts32)
    for _ in range(args.warmup):
        step32()
    barrier()
    torch.cuda.synchronize()
    l1 = sum(part.h.stats()["kernels_launched"] for part in parts32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        outs = [step32() for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    t32 = max_over_ranks(e0.elapsed_time(e1)) / args.steps
    launches = (sum(part.h.stats()["kernels_launched"] for part in parts32) - l1) // args.steps
    res32 = max(part.worst_resid() for part in parts32)
    st = [part.h.stats() for part in parts32]
    fl_factor = sum(s["model_flops"] for s in st)
    dev_bytes = sum(s["device_bytes"] for s in st)
    # one profiled factorisation: the data-flow kernel's share and the roofline
    for part in parts32:
        part.h.set_profiling(True)
    step32()
    torch.cuda.synchronize()
    prof = [part.h.stats() for part in parts32]
    for part in parts32:
        part.h.set_profiling(False)
    factor_ms = sum(p_["kernel_ms"]["dataflow_factor"] for p_ in prof)
    efac_stacked = max(part.h.factor_error()[0] for part in parts32)
    plan_ms = [part.h.stats()["create_ms"] for part in parts32]
    its32 = max(o[0] for o in outs[-1])
    for part in parts32:
        part.h.close()
    del parts32
    torch.cuda.empty_cache()

    # the comparison: one FP64 handle per problem, factor + refinement, one after the other; the
    # handles are created ahead on host threads (each on its own stream), and only each problem's
    # factor + refinement is timed (CUDA events on its stream)
    def create64(i):
        torch.cuda.set_device(local)
        s = torch.cuda.Stream()
        h = HLU.from_problem(probs[i], precision=HLU_FP64, stream=s.cuda_stream, nrhs_max=1)
        return s, h

    loop_ms, loop_its, loop_worst = [], 0, 0.0
    tl0 = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(4) as ex:
        ahead = 6
        futs = {i: ex.submit(create64, i) for i in range(min(ahead, B))}
        for i in range(B):
            s, h = futs.pop(i).result()
            if i + ahead < B:
                futs[i + ahead] = ex.submit(create64, i + ahead)
            with torch.cuda.stream(s):
                b = to_device_panel(probs[i].b)
                x = torch.zeros_like(b)
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(s)
                h.factor(probs[i].eps)
                it, res = h.solve_refined(b, x, tol=TOL, max_iter=30)
                a1.record(s)
                a1.synchronize()
            loop_ms.append(a0.elapsed_time(a1))
            loop_its = max(loop_its, it)
            loop_worst = max(loop_worst, res)
            h.close()
    loop_wall_s = time.perf_counter() - tl0
    tloop = sum(loop_ms)

    # end to end through the public API: hlu_create_batch from host arrays (validation, parallel
    # planning, upload), the tuned launch setting, factor, b from pinned host memory, x back
    b_host = torch.tensor(np.ascontiguousarray(np.concatenate([p.b for p in probs], axis=0).T)).pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    h2d = sum(p.data.nbytes + p.row_cl.nbytes + p.col_cl.nbytes + p.kind.nbytes + p.rank.nbytes + p.offset.nbytes
              + p.tree.perm.nbytes + p.tree.begin.nbytes + p.tree.size.nbytes + p.tree.son0.nbytes
              + p.tree.son1.nbytes for p in probs) + b_host.numel() * 8
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    parts = make_parts(HLU_FP32, temp_reuse=1)
    bd = b_host.to("cuda", non_blocking=True).t()
    xd = torch.zeros_like(bd)
    row0 = np.cumsum([0] + [p.n for p in probs])
    for part in parts:
        part.h.set_launch(choice["workers"], choice["flags"])
        part.h.factor(part.eps)
        if len(parts) == 1:
            part.h.solve_refined(bd, xd, tol=part.tol, max_iter=30)
        else:  # a part's stacked rows are its problems' rows, in order
            sel = torch.as_tensor(np.concatenate([np.arange(row0[i], row0[i + 1]) for i in part.idx]), device="cuda")
            bi = bd[sel, 0].reshape(1, -1).t()
            xi = torch.zeros_like(bi)
            part.h.solve_refined(bi, xi, tol=part.tol, max_iter=30)
            xd[sel, 0] = xi[:, 0]
    x_host.copy_(xd.t(), non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - te0
    for part in parts:
        part.h.close()

    fp64_peak, fp32_peak = probe_alu_peaks()
    achieved = fl_factor / (factor_ms * 1e-3) / 1e12 if factor_ms else None
    cpu = None
    if rank == 0:
        try:
            o = oracle_batch_sample(args.workload)
            cpu = {"value": o["problems"] / o["seconds"], "unit": "problems/s", "cores": 1, "kind": "oracle",
                   "sample": f"FP64 oracle H-LU + solve of the batch's {o['problems']} smallest problems "
                             f"(r = {o['r']}, n = {o['n']}, host-built leaves), {o['seconds']:.1f} s on 1 host "
                             f"thread"}
            cpu.update(cpu_info())
            # all host cores: the independent problems spread over one single-threaded process per core
            allc = oracle_batch_pool(args.workload, 2 * (os.cpu_count() or 1))
            cpu["all_cores"] = {"value": allc["problems"] / allc["seconds"], "unit": "problems/s",
                                "cores": allc["procs"], "problems": allc["problems"],
                                "seconds": allc["seconds"]}
        except Exception as e:  # the baseline is context; the line stands without it
            cpu = {"value": None, "unit": "problems/s", "cores": 1, "kind": "oracle", "error": str(e)[-300:]}
    if rank == 0:
        ns = sorted({p.n for p in probs})
        w = BATCHES[args.workload]
        line = {
            "metric": "batched H-LU: problems factorised and solved to 1e-10 per second", "value": B * world / (t32 * 1e-3),
            "unit": "problems/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t32,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 factors; f64 truncation-core SVD, residual and solution", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {B} ellipsoids, refinement {w['levels']} (n in {ns}), "
                                   f"leaf {w['leaf']}, eta {w['eta']}, eps per problem in {sorted(set(eps))}, "
                                   f"axes {w.get('axes_range', '(1, U[0.4,1], U[0.4,1])')}, 1 rhs each, "
                                   f"tol 1e-10 per problem; leaf data built on the GPU",
                       "n_total": int(sum(p.n for p in probs)), "leaves": int(sum(p.n_leaves for p in probs)),
                       "problems_by_n": {str(n): sum(p.n == n for p in probs) for n in ns},
                       "parallelism": f"replicas x{world}", "handles": len(st),
                       "l2": f"inputs larger than L2 (device memory {dev_bytes / 1e9:.1f} GB)"},
            "batched_fp32_ms": t32, "loop_fp64_ms": tloop, "loop_fp64_wall_s": loop_wall_s,
            "speedup_vs_fp64_loop": tloop / t32,
            "ir_iters": {"batched_fp32": its32, "loop_fp64_max": loop_its},
            "worst_problem_resid": {"batched_fp32": res32, "loop_fp64": loop_worst},
            "efac_stacked_fp32": efac_stacked,
            "factor_model_gflop": fl_factor / 1e9, "max_rank": max(s["max_rank"] for s in st),
            "plan": {"tasks": sum(s["n_tasks"] for s in st), "create_ms": plan_ms},
            "tuner": {"sample_problems": len(sample_idx), "choice": choice,
                      "trials": [{"workers": c["workers"], "flags": c["flags"], "s": round(t, 4)} for c, t in trials]},
            "host_structure_s": structure_s, "gpu_construct_s": construct_s, "create_s": create_s,
            "host_mem_available_gb": (host_available() or 0) / 1e9,
            "e2e": {"value": B / e2e_s, "unit": "problems/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(x_host.numel() * 8), "ms_per_step": e2e_s * 1e3,
                    "includes": "hlu_create_batch (validation, parallel planning, upload) + factor + refinement + "
                                "copies, one step"},
            "roofline": {"kernel": "k_dataflow<float> (factorisation)", "bound": "alu", "achieved": achieved,
                         "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak if achieved and fp32_peak else None, "traffic": None,
                         "peak_source": "measured FP32 FMA probe (hlu_probe_alu_peaks), of measured",
                         "factor_kernel_ms": factor_ms},
            "cpu_baseline": cpu,
            "gpu_launches": launches, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_serve(args):
    """Serving loop (paper_1906_00874_gb300.serve) on a seeded Poisson request stream. Calibration:
    a pass with every request arriving at once gives the burst capacity (requests/s), and a pass with
    Poisson arrivals at that rate gives the sustained capacity (requests served per second); the
    timed passes replay the stream with exponential inter-arrival times at 0.8x the sustained
    capacity on the wall clock, each pass on a fresh server (no factors resident at the start).
    Reports throughput and the p50 / p99 latency from arrival to solution on the host."""
    import numpy as np
    import torch

    from bem_inputs import STREAMS, stream_specs
    from paper_1906_00874_gb300 import build
    from paper_1906_00874_gb300.serve import Request, Server

    rank, world, local = dist_env()
    w = dict(STREAMS[args.workload])
    temp_reuse = w.pop("temp_reuse", 0)
    stream, specs = stream_specs(**w)
    # structures on all host cores (before any CUDA call), leaf data on the GPU
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(len(specs), os.cpu_count() or 1)) as pool:
        probs = pool.map(_structure_one, specs, chunksize=1)
    torch.cuda.set_device(local)
    build.build()
    construct_leaves(probs)
    rhs = [np.random.default_rng(sd).standard_normal((probs[k].n, c)) for k, c, sd in stream]

    def pct(a, q):
        return a[min(len(a) - 1, int(round(q * (len(a) - 1))))]

    def replay(arrivals, timeline=False):
        # a stream per group, half the workers per launch, groups of <= 16
        srv = Server(timeline=timeline, temp_reuse=temp_reuse)
        reqs = [Request(k, probs[k], b, arrival=float(t), rid=i)
                for i, ((k, _, _), b, t) in enumerate(zip(stream, rhs, arrivals))]
        torch.cuda.synchronize()
        ref = torch.cuda.Event(enable_timing=True)
        ref.record()
        t0 = time.perf_counter()
        srv.clock = lambda: time.perf_counter() - t0
        srv.serve(reqs)
        makespan = srv.clock()
        torch.cuda.synchronize()
        ov = overlap(srv.events, ref) if timeline else None
        srv.close()  # adds the kernel launches of the handles it releases
        st = dict(srv.stats)
        adm = sorted(srv.admissions, key=lambda a: -(a[2] + a[3]))
        st["slowest_admissions"] = [{"problems": a[0], "n": a[1], "create_s": round(a[2], 3),
                                     "factor_s": round(a[3], 3)} for a in adm[:5]]
        st["admission_create_s"] = round(sum(a[2] for a in adm), 3)
        st["admission_factor_s"] = round(sum(a[3] for a in adm), 3)
        lat = sorted((r.done - r.arrival) * 1e3 for r in reqs)
        return makespan, lat, st, reqs, ov

    def breakdown(reqs):
        """p50 / p99 latency of the requests that waited for a factorisation of their problem and of
        those served from resident factors, and by problem size."""
        out = {}
        groups = {"waited_for_admission": [r for r in reqs if r.waited],
                  "resident": [r for r in reqs if not r.waited]}
        for n in sorted({probs[r.key].n for r in reqs}):
            groups[f"n={n}"] = [r for r in reqs if probs[r.key].n == n]
        for name, rs in groups.items():
            v = sorted((r.done - r.arrival) * 1e3 for r in rs)
            if v:
                out[name] = {"count": len(v), "p50_ms": pct(v, 0.5), "p99_ms": pct(v, 0.99)}
        # where the time goes: arrival -> group resident -> solve start -> solution
        for name, a, b in (("to_resident", "arrival", "resident_at"), ("resident_to_solve", "resident_at", "solve_at"),
                           ("solve", "solve_at", "done")):
            v = sorted((getattr(r, b) - getattr(r, a)) * 1e3 for r in reqs
                       if getattr(r, a) is not None and getattr(r, b) is not None)
            if v:
                out["phase_" + name] = {"p50_ms": pct(v, 0.5), "p99_ms": pct(v, 0.99), "max_ms": v[-1]}
        return out

    def overlap(events, ref):
        """Device time during which a factorisation and a solve of another group were both running,
        over the factorisations' time (event timestamps on the groups' streams)."""
        fac = [(ref.elapsed_time(a), ref.elapsed_time(b), g) for k, g, a, b in events if k == "factor"]
        sol = [(ref.elapsed_time(a), ref.elapsed_time(b), g) for k, g, a, b in events if k == "solve"]
        both = 0.0
        for f0, f1, fg in fac:
            segs = sorted((max(f0, s0), min(f1, s1)) for s0, s1, sg in sol if sg != fg and s0 < f1 and f0 < s1)
            end = f0
            for a, b in segs:
                a = max(a, end)
                if b > a:
                    both += b - a
                    end = b
        tot = sum(f1 - f0 for f0, f1, _ in fac)
        return {"factor_ms": tot, "factor_with_solve_ms": both, "fraction": both / tot if tot else 0.0,
                "factorisations": len(fac), "solves": len(sol)}

    zero = np.zeros(len(stream))
    for _ in range(max(1, args.warmup // 3)):
        cal_t = replay(zero)[0]
    burst = len(stream) / cal_t
    # sustained capacity: the stream with Poisson arrivals at the burst capacity, requests served per
    # second of that pass (a trickle of arrivals is grouped less than a burst)
    g = np.random.default_rng(0)
    arrivals = np.cumsum(g.exponential(1.0 / burst, len(stream)))
    capacity = len(stream) / replay(arrivals - arrivals[0])[0]
    rate = 0.8 * capacity
    runs = []
    with ClockSampler(local) as clk:
        for i in range(max(1, args.steps // 3)):
            arrivals = np.cumsum(g.exponential(1.0 / rate, len(stream)))
            arrivals -= arrivals[0]
            runs.append(replay(arrivals, timeline=(i == 0)))
    lat = sorted(x for r in runs for x in r[1])
    mk = sum(r[0] for r in runs)
    st = runs[-1][2]

    if rank == 0:
        nrhs = sum(c for _, c, _ in stream)
        line = {
            "metric": "H-LU serving: requests solved to 1e-10 per second, p50/p99 latency", "unit": "requests/s",
            "value": len(stream) * len(runs) / mk, "n_gpus": world, "steps": len(runs), "warmup": args.warmup,
            "ms_per_step": mk / len(runs) * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 factors; f64 truncation-core SVD, residual and solution", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {len(stream)} requests, {len(specs)} distinct ellipsoid problems "
                                   f"(n in {sorted({p.n for p in probs})}), {int(100 * w['repeat'])}% repeats, "
                                   f"nrhs uniform in {list(w['nrhs'])} ({nrhs} in all), Poisson arrivals at 0.8x "
                                   f"the measured sustained capacity, 150 GB budget, tol 1e-10 per request",
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2"},
            "capacity_rps": capacity, "capacity_burst_rps": burst, "arrival_rate_rps": rate,
            "p50_ms": pct(lat, 0.5), "p99_ms": pct(lat, 0.99), "mean_ms": float(np.mean(lat)),
            "server": st, "device_overlap": runs[0][4],
            "latency_breakdown": breakdown([r for run in runs for r in run[3]]), "gpu_launches": int(sum(r[2].get("kernels_launched", 0) for r in runs)),
            "e2e": {"value": len(stream) * len(runs) / mk, "unit": "requests/s",
                    "h2d_bytes_per_step": int(sum(b.nbytes for b in rhs) + sum(p.data.nbytes for p in probs)),
                    "d2h_bytes_per_step": int(sum(b.nbytes for b in rhs)),
                    "includes": "host arrays in, handle creation + factorisation of new problems, solves, "
                                "solutions back to host: the serving loop is end to end"},
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)


def run_construct(args):
    """Construction of the workload's H-matrix leaves on the GPU (dense blocks, ACA + truncation of
    the admissible blocks) against the host generator that built the same matrix (Python + NumPy,
    one process). The block tree and the leaf kinds are the host's; the GPU computes the data."""
    import numpy as np
    import torch

    from bem_inputs import WORKLOADS, build_problem
    from paper_1906_00874_gb300 import build
    from paper_1906_00874_gb300.hlu import BEMBuild

    w = dict(WORKLOADS[args.workload])
    p = build_problem(cache=False, **w)
    torch.cuda.set_device(0)
    build.build()
    for _ in range(max(1, args.warmup)):
        BEMBuild.from_problem(p).close()
    times = []
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = BEMBuild.from_problem(p)
        times.append(time.perf_counter() - t0)
    ranks = g.rank[p.kind == 1]
    same = float(np.mean(ranks == p.rank[p.kind == 1]))
    g.close()
    sec = sorted(times)[len(times) // 2]
    print(json.dumps({
        "metric": "H-matrix construction time (leaf data of a given block tree)", "value": sec * 1e3, "unit": "ms",
        "higher_is_better": False, "n_gpus": 1, "steps": len(times), "warmup": args.warmup, "data": "synthetic",
        "config": {"workload": f"{args.workload}: n={p.n}, {p.n_leaves} leaves "
                               f"({int((p.kind == 1).sum())} low rank), eps={p.eps:g}"},
        "host_generator_s": p.build_seconds, "speedup_vs_host_generator": p.build_seconds / sec,
        "low_rank_rank_equal_to_host": same, "data_doubles": int(g.data_len)}), flush=True)


def main():
    global FLAGS
    args = parse()
    if args.tensor:
        from paper_1906_00874_gb300.hlu import FLAG_TENSOR
        FLAGS = FLAG_TENSOR
    if args.construct:
        run_construct(args)
        return
    from bem_inputs import BATCHES, STREAMS
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in BATCHES:
        run_batch(args)
    elif args.workload in STREAMS:
        run_serve(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
