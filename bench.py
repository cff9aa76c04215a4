#!/usr/bin/env python
"""Benchmark of the power-series H-matrix EFIE solve on GB300.

Metric: power-series RHS solves per second on the 2-lambda PEC sphere
(icosphere level 5, 20480 triangles, 30720 RWG unknowns, octree leaves <= 128,
ACA tol 1e-4), 362 monostatic right-hand sides (theta = 0..180 deg step 1,
phi = 0, theta- and phi-polarised plane waves).  One step = one
hm_power_series_solve over the whole RHS batch, inputs resident in HBM.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

N > 1 runs replicas (one independent copy of the system per GPU, RHS batch per
GPU fixed: weak scaling, no collective on the data path).  Prints one JSON
line on rank 0.

Other workloads (--workload): sphere_r0.5_L3 and sphere_r2_L5_1rhs (one RHS),
scatterer_batch (grouped solve of a seeded batch), sphere_scaling (set-up and
solve time against N), sphere_r10_L7 (the 10-lambda sphere in RHS chunks) and
leaf_size_study (series error against leaf size, Sec. V-A).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "power-series RHS solves/s at rel.err ≤1e-4 vs FP64; mixed vs FP64 on 1 GB300"

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# FP64-accurate residual far-field kernels, from one ncu capture of this bench
# (2-lambda sphere, 362 RHS, mixed precision; summary under profiles/).  They
# are reported as the roofline's "traffic" only while the code of the kernel
# and of the schedules it walks (the sources with comments and whitespace
# removed) still hashes to the captured version; any later change turns them
# off (null).
NCU_TRAFFIC_SOURCE = (("paper_2109_04129_gb300/csrc/hm_oz.cu",
                       "paper_2109_04129_gb300/csrc/hm_api.cu"),
                      "f9a9c915837432ae5b089b53f37fb42a08c37953169e90360d9e39aeca1dd399")
NCU_TRAFFIC = {("sphere_r2_L5", "mixed", 362, "far_stage1"): 2.117330944e9 + 1.990641920e9,
               ("sphere_r2_L5", "mixed", 362, "far_stage2"): 30.812379648e9 + 0.183819008e9}


def code_hash(text):
    """sha256 of C/CUDA source with its comments and whitespace removed (the
    kernel sources hold no string literal with a comment marker)."""
    import hashlib
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return hashlib.sha256(" ".join(text.split()).encode()).hexdigest()


def captured_traffic(workload, precision, nrhs, kernel):
    """ncu DRAM bytes per launch of `kernel`, or None when not captured for this
    configuration or when the kernel code changed since the capture."""
    b = NCU_TRAFFIC.get((workload, precision, nrhs, kernel))
    if b is None:
        return None
    text = ""
    for path in NCU_TRAFFIC_SOURCE[0]:
        with open(os.path.join(ROOT, path)) as f:
            text += f.read()
    if code_hash(text) != NCU_TRAFFIC_SOURCE[1]:
        return None
    return b


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="sphere_r2_L5")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the plain FP64 GPU solve measured beside the mixed one")
    ap.add_argument("--ordering", default="nd", choices=["nd", "dfs"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-single-rhs", action="store_true",
                    help="skip the one-RHS (bandwidth-bound) leg")
    ap.add_argument("--split-max", type=int, default=0,
                    help="largest split-K size of the tensor-core sweeps (0: the library's)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-tensor-cores", action="store_true",
                    help="the mixed chain on the CUDA cores (FP32 arithmetic), for comparison")
    ap.add_argument("--cpu-rhs", type=int, default=4, help="RHS in the oracle's timed sample")
    ap.add_argument("--chunk", type=int, default=120,
                    help="RHS per call of --workload sphere_r10_L7")
    ap.add_argument("--fill", default=None, choices=["A", "B"],
                    help="scaling reading: A (full fill; default) or B (near-pattern fill; "
                         "the default of --workload sphere_r10_L7)")
    ap.add_argument("--oracle-check", action="store_true",
                    help="sphere_r10_L7: oracle series on the library's blocks (8 RHS)")
    ap.add_argument("--levels", type=int, nargs="+", default=[3, 4, 5, 6],
                    help="icosphere levels of --workload sphere_scaling")
    ap.add_argument("--batch-count", type=int, default=64,
                    help="scatterers in --workload scatterer_batch")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
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
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "native" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, val, device):
    if ws == 1:
        return val
    import torch
    import torch.distributed as dist
    t = torch.tensor([val], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_desc(w, N, nrhs):
    """The workload named by both arms' config: mesh, size, tree, ACA and the
    incidence sweep of a single-scatterer workload."""
    lam = w.wavelength
    kind = w.mesh[0]
    if kind == "icosphere":
        geo = f"PEC sphere r={w.mesh[2] / lam:g} lambda, icosphere L{w.mesh[1]}"
    elif kind == "plate":
        geo = f"PEC plate {w.mesh[1] / lam:g} x {w.mesh[1] / lam:g} lambda, " \
              f"{w.mesh[2]} x {w.mesh[2]} cells"
    else:
        geo = f"PEC {kind} {w.mesh[1:]}"
    sw = w.sweep
    if sw[0] == "single":
        rhs = f"{nrhs} RHS"
    else:
        pols = "/".join("theta" if p == 0 else "phi" for p in sw[5])
        rhs = (f"{nrhs} monostatic RHS ({sw[0]} {sw[1]:g}..{sw[2]:g} step {sw[3]:g}, "
               f"{pols} pol)")
    aca = f"{w.aca_tol:.0e}".replace("e-0", "e-")
    return f"{w.name}: {geo}, N={N}, leaves<={w.leaf_max}, ACA {aca}, {rhs}"


def job_rate(ws, units_per_rank, t_local, device):
    """Whole-job rate: every rank processed `units_per_rank` units; the job took
    the slowest rank's time.  Returns (time per step of the job, units/s)."""
    t = max_over_ranks(ws, t_local, device)
    return t, ws * units_per_rank / t


def gemm_peak(dev, dtype):
    """ALU denominators: cuBLAS GEMM 4096^3 in the given dtype, best of 5 (TFLOP/s)."""
    import torch
    a = torch.randn(4096, 4096, dtype=dtype, device=dev)
    b = torch.randn(4096, 4096, dtype=dtype, device=dev)
    a @ b
    torch.cuda.synchronize()
    best = 1e30
    for _ in range(5):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2 * 4096 ** 3 / best / 1e12


# ----------------------------------------------------------------- oracle leg
def oracle_setup(w, processes):
    from oracle.efie import EFIE
    from oracle.hmatrix import build_hmatrix
    from oracle.scaling import compute_scaling, nd_order
    v, f = w.build_mesh()
    t0 = time.perf_counter()
    H = build_hmatrix(v, f, w.wavelength, w.leaf_max, w.aca_tol, processes=processes,
                      use_c=True)
    S = compute_scaling(H, "A", nd_order(H.tree, list(H.near.keys())))
    th, ph, po = w.angles()
    B = EFIE(H.rwg, w.wavelength).plane_wave(th, ph, po)
    return H, S, B, time.perf_counter() - t0


def oracle_time(H, S, B, nrhs_sample, reps, refine=True):
    """Oracle solve (plain NumPy FP64) of a bounded RHS sample, timed per
    repetition.  refine=True times the work of the mixed path: the two-term
    series, the FP64 residual and the series of the refinement step
    (oracle.series.refine_once); refine=False the plain two-term series."""
    from oracle.series import refine_once, series_solve
    idx = list(range(0, B.shape[1], max(1, B.shape[1] // nrhs_sample)))[:nrhs_sample]
    Bs = B[:, idx]
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        x2, _ = series_solve(H, S, Bs, 2)
        if refine:
            refine_once(H, S, Bs, x2)
        ts.append(time.perf_counter() - t0)
    return len(idx), ts


def openblas_threads():
    """(set, get) thread-count functions of the OpenBLAS that NumPy loaded
    (found by name among the process's mapped libraries), or None."""
    import ctypes
    try:
        with open("/proc/self/maps") as f:
            paths = sorted({ln.split()[-1] for ln in f
                            if "openblas" in ln.lower() and ".so" in ln})
    except OSError:
        return None
    for path in paths:
        try:
            lib = ctypes.CDLL(path)
        except OSError:
            continue
        for pre, suf in (("scipy_openblas", "64_"), ("openblas", ""), ("openblas", "64_"),
                         ("scipy_openblas", "")):
            st, gt = f"{pre}_set_num_threads{suf}", f"{pre}_get_num_threads{suf}"
            if hasattr(lib, st) and hasattr(lib, gt):
                return getattr(lib, st), getattr(lib, gt)
    return None


def oracle_job(name, processes, nrhs_sample, reps, conn):
    """Oracle set-up, then (on "go") the timed sample, in a separate (spawned)
    process: the series + refinement (like-for-like with the mixed GPU path)
    and the plain series with NumPy's BLAS on all its threads, then the first
    again with that BLAS on one thread.  It reports "ready" after the set-up
    and waits for "go", which the GPU side sends after its own measurements,
    so the two never run at the same time."""
    try:
        from hm_workloads import get_workload
        w = get_workload(name)
        H, S, B, setup_s = oracle_setup(w, processes)
        conn.send({"ready": True})
        if conn.recv() != "go":
            return
        n, ts = oracle_time(H, S, B, nrhs_sample, reps, refine=True)
        _, ts_plain = oracle_time(H, S, B, nrhs_sample, reps, refine=False)
        threads, one = cpu_threads(), None
        ob = openblas_threads()
        if ob is not None:
            set_t, get_t = ob
            threads = int(get_t())
            set_t(1)
            try:
                n1, ts1 = oracle_time(H, S, B, nrhs_sample, 1, refine=True)
            finally:
                set_t(threads)
            one = {"n": n1, "ts": ts1}
        conn.send({"n": n, "ts": ts, "ts_plain": ts_plain, "setup_s": setup_s,
                   "threads": threads, "nrhs": B.shape[1], "one_thread": one})
    except Exception as e:  # reported in the JSON line
        conn.send({"error": repr(e)})
    conn.close()


def one_thread_entry(res):
    """The oracle's rate with NumPy's BLAS on one thread, for cpu_baseline."""
    one = res.get("one_thread")
    if not one:
        return {"value": None, "note": "OpenBLAS thread control not found"}
    return {"value": one["n"] / min(one["ts"]), "unit": "RHS/s", "cores": 1,
            "sample": f"the same {one['n']} RHS, one run"}


def start_oracle(name, nrhs_sample, reps):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    parent, child = ctx.Pipe(duplex=True)
    procs = max(1, min(16, (os.cpu_count() or 2) - 2))
    p = ctx.Process(target=oracle_job, args=(name, procs, nrhs_sample, reps, child))
    p.start()
    o = {"proc": p, "conn": parent, "procs": procs, "error": None, "done": False}
    _ORACLES.append(o)
    return o


_ORACLES = []


def oracle_stop_all():
    """Release oracle processes whose result was never collected (the GPU leg
    failed): they wait for "go" and would keep the interpreter from exiting."""
    for o in _ORACLES:
        if o["done"]:
            continue
        try:
            o["conn"].send("stop")
        except (OSError, ValueError):
            pass
        o["proc"].join(timeout=60)
        if o["proc"].is_alive():
            o["proc"].terminate()
            o["proc"].join(timeout=10)
        o["done"] = True


def oracle_ready(oracle):
    """Block until the oracle process has finished its set-up (before the GPU's
    timed region, so that the set-up's worker processes do not share the host
    with it)."""
    if oracle is None:
        return
    msg = oracle["conn"].recv()
    if "error" in msg:
        oracle["error"] = msg


def oracle_result(oracle, what):
    """Send "go", collect the timed sample and format cpu_baseline."""
    proc, conn, procs = oracle["proc"], oracle["conn"], oracle["procs"]
    res = oracle["error"]
    if res is None:
        conn.send("go")
        res = conn.recv()
    proc.join()
    oracle["done"] = True
    if "error" in res:
        return {"value": None, "unit": "RHS/s", "kind": "oracle", "error": res["error"]}
    t = min(res["ts"])
    return {"value": res["n"] / t, "unit": "RHS/s", "cores": res["threads"], "kind": "oracle",
            "sample": f"{res['n']} of {res['nrhs']} RHS of {what}, oracle FP64 two-term series "
                      f"+ one refinement step (residual and second series: the mixed path's "
                      f"work), best of {len(res['ts'])}; oracle set-up {res['setup_s']:.0f} s "
                      f"untimed ({procs} processes, finished before the GPU's timed region; "
                      f"the sample ran after it)",
            "series_only": {"value": res["n"] / min(res["ts_plain"]), "unit": "RHS/s",
                            "what": "plain two-term series on the same sample"},
            "single_thread": one_thread_entry(res)}


def cpu_threads():
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [1])
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return
    from hm_workloads import get_workload
    w = get_workload(args.workload)
    procs = max(1, min(16, os.cpu_count() or 1))
    H, S, B, setup_s = oracle_setup(w, procs)
    # one step = the mixed path's work on the sample: series + refinement
    n, ts = oracle_time(H, S, B, args.cpu_rhs, args.warmup + args.steps, refine=True)
    ts = ts[args.warmup:]
    t = sum(ts) / len(ts)
    val = n / t
    _, ts_plain = oracle_time(H, S, B, args.cpu_rhs, 1, refine=False)
    threads, one = cpu_threads(), {"one_thread": None}
    ob = openblas_threads()
    if ob is not None:
        threads = int(ob[1]())
        ob[0](1)
        try:
            n1, ts1 = oracle_time(H, S, B, args.cpu_rhs, 1)
        finally:
            ob[0](threads)
        one = {"one_thread": {"n": n1, "ts": ts1}}
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "RHS/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": workload_desc(w, H.N, B.shape[1]),
                   "sample": f"{n} of {B.shape[1]} RHS per step"},
        "cpu_baseline": {"value": val, "unit": "RHS/s", "cores": threads, "kind": "oracle",
                         "sample": f"{n} RHS per step of the {B.shape[1]}-RHS sweep, oracle "
                                   f"FP64 two-term series + one refinement step (the mixed "
                                   f"path's work); oracle set-up {setup_s:.0f} s (not timed, "
                                   f"{procs} processes)",
                         "series_only": {"value": n / min(ts_plain), "unit": "RHS/s",
                                         "what": "plain two-term series on the same sample"},
                         "single_thread": one_thread_entry(one)},
        "e2e": {"value": val, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- native leg
def run_native(args):
    ws, rank, local = dist_setup(args)
    # the oracle leg starts before the first GPU call (spawned, CPU only); its
    # set-up overlaps the GPU set-up, and its timed sample runs after every
    # GPU measurement (oracle_ready / oracle_result)
    oracle = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        oracle = start_oracle(args.workload, args.cpu_rhs, 2)
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2109_04129_gb300 as hp
    from hm_workloads import get_workload
    w = get_workload(args.workload)
    v, f = w.build_mesh()
    prec = hp.HM_MIXED if args.precision == "mixed" else hp.HM_FP64
    t0 = time.perf_counter()
    sol = hp.Solver.build(v, f, wavelength=w.wavelength, leaf_max=w.leaf_max,
                          aca_tol=w.aca_tol,
                          ordering=hp.HM_ORDER_ND if args.ordering == "nd" else hp.HM_ORDER_DFS,
                          precision=prec, refine_steps=1 if prec == hp.HM_MIXED else 0,
                          **engine_kw(args))
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    sol.compute_scaling()
    t_scale = time.perf_counter() - t0
    st = sol.stats()
    th, ph, po = w.angles()
    nrhs = len(th)
    B = torch.empty((nrhs, sol.N), dtype=torch.complex128, device=dev)
    sol.plane_wave(B, th, ph, po)
    X = torch.empty_like(B)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        sol.solve(X, B)
    torch.cuda.synchronize()
    oracle_ready(oracle)
    # ---- timed region: device-resident inputs (alpha/far data > L2: no flush)
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = sol.stats()["kernel_launches"]
    with ClockSampler(local) as clk:
        torch.cuda.nvtx.range_push("hm_timed")
        e0.record(stream)
        for _ in range(args.steps):
            sol.solve(X, B)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    timed_launches = sol.stats()["kernel_launches"] - l0
    barrier(ws)
    t_dev = e0.elapsed_time(e1) / 1e3 / args.steps
    t_dev, value = job_rate(ws, nrhs, t_dev, dev)
    ratio, _ = sol.diagnostics(nrhs)
    # ---- per-kernel timing (same steps, events around every launch)
    sol.profile_enable(True)
    for _ in range(args.steps):
        sol.solve(X, B)
    prof = sol.profile()
    sol.profile_enable(False)
    peaks, peak_kind = measured_peaks()
    kernels = kernel_table(prof, args.steps)
    roof = roofline(prof, nrhs, prec == hp.HM_MIXED, peaks, peak_kind, dev)
    roof["traffic"] = captured_traffic(args.workload, args.precision, nrhs, roof["kernel"])
    if roof["traffic"] is not None:
        roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of this "
                                  "kernel, one capture of this bench on the same kernel source")
    # ---- end to end through the host-buffer C-ABI call
    Bh = torch.empty((nrhs, sol.N), dtype=torch.complex128, pin_memory=True)
    Bh.copy_(B)
    Xh = torch.empty_like(Bh, pin_memory=True)
    bn, xn = Bh.numpy(), Xh.numpy()
    sol.solve_host(xn, bn)
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sol.solve_host(xn, bn)
    t_e2e = (time.perf_counter() - t0) / args.steps
    t_e2e, v_e2e = job_rate(ws, nrhs, t_e2e, dev)
    e2e = {"value": v_e2e, "unit": "RHS/s",
           "h2d_bytes_per_step": int(bn.nbytes), "d2h_bytes_per_step": int(xn.nbytes)}
    line = {
        "metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128" if prec == hp.HM_FP64 else
                 "mixed: c64 chain on tcgen05 (3-way bf16 split, f32 accum), c128 D^-1, "
                 "FP64-accurate residual on tcgen05 (exact 7-bit slicing)",
        "data": "synthetic",
        "config": {"workload": workload_desc(w, sol.N, nrhs),
                   "precision": args.precision, "ordering": args.ordering,
                   "engine": engine_kw(args) or "library defaults",
                   "l2": "inputs larger than L2 (alpha + far factors), no flush",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "alpha_entries": st["alpha_entries"], "far_entries": st["far_entries"],
                   "near_entries": st["near_entries"], "fwd_levels": st["fwd_levels"],
                   "build_s": round(t_build, 2), "scaling_s": round(t_scale, 2),
                   "series_ratio_max": float(np.max(ratio))},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": timed_launches,
        "clocks": clk.summary(),
        "kernels": kernels,
    }
    sol64 = None
    if prec == hp.HM_MIXED and not args.no_fp64_compare:
        # the FP64 GPU chain on the same system: the plain two-term series
        # (rate) and the series plus the same FP64 refinement (the like-for-like
        # accuracy comparator of the mixed solve)
        fp64 = {}
        for refine in (1, 0):
            s64 = hp.Solver.build(v, f, wavelength=w.wavelength, leaf_max=w.leaf_max,
                                  aca_tol=w.aca_tol,
                                  ordering=hp.HM_ORDER_ND if args.ordering == "nd" else hp.HM_ORDER_DFS,
                                  precision=hp.HM_FP64, refine_steps=refine)
            s64.compute_scaling()
            X64 = torch.empty_like(B)
            s64.solve(X64, B)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(2):
                s64.solve(X64, B)
            e1.record(stream)
            torch.cuda.synchronize()
            fp64[refine] = (e0.elapsed_time(e1) / 1e3 / 2, X64)
            if refine == 0:
                sol64 = s64          # kept for the single-RHS leg
            else:
                del s64
        sol.solve(X, B)
        torch.cuda.synchronize()
        Xr = fp64[1][1]
        d = torch.linalg.vector_norm(X - Xr, dim=1) / torch.linalg.vector_norm(Xr, dim=1)
        t64 = fp64[0][0]
        line["fp64_gpu"] = {
            "value": nrhs / t64, "unit": "RHS/s", "ms_per_step": 1e3 * t64, "steps": 2,
            "warmup": 1, "what": "plain FP64 two-term series (FP64 units)",
            "with_refinement_value": nrhs / fp64[1][0],
            "mixed_vs_fp64_refined_rel_err_max": float(d.max().item()),
            "speedup_mixed_over_plain_fp64": value / (nrhs / t64),
            "speedup_mixed_over_fp64_refined": value / (nrhs / fp64[1][0])}
        del fp64
    if not args.no_single_rhs:
        # one RHS (the first of the sweep): the bandwidth-bound form of the
        # same chain, every block read once per sweep (HBM roofline)
        single = {}
        for tag, sh in (("mixed" if prec == hp.HM_MIXED else "fp64", sol), ("fp64", sol64)):
            if sh is None or tag in single:
                continue
            single[tag] = single_rhs_leg(sh, B[:1].contiguous(), max(5, args.steps), peaks,
                                         peak_kind, stream)
        line["single_rhs"] = single
    if oracle is not None:
        line["cpu_baseline"] = oracle_result(oracle, "the same sweep")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def engine_kw(args):
    """Engine switches of the mixed handle from the command line (defaults: the
    library's)."""
    kw = {}
    if args.split_max:
        kw["tc_split_max"] = args.split_max
    if args.no_autotune:
        kw["autotune"] = 0
    if args.no_tensor_cores:
        kw["tensor_cores"] = 0
    return kw


def kernel_table(prof, steps):
    tot_ms = sum(p[1] for p in prof.values())
    kernels = {}
    for cat, (launches, ms, byts, flops) in prof.items():
        if not launches:
            continue
        kernels[cat] = {"ms_per_step": round(ms / steps, 4), "share": round(ms / tot_ms, 4),
                        "launches_per_step": int(launches / steps),
                        "tflops": round(flops / (ms / 1e3) / 1e12, 4),
                        "gbs": round(byts / (ms / 1e3) / 1e9, 2)}
    return kernels


TENSOR_CATS = ("mixed_sweep", "mixed_far")            # complex64 chain on tcgen05
OZ_CATS = ("far_stage1", "far_stage2", "near")         # FP64-accurate residual on tcgen05
FP32_CATS = ("mixed_sweep", "mixed_far")


def roofline(prof, nrhs, mixed, peaks, peak_kind, dev):
    """Roofline of the category with the largest share of the profiled time.
    With 32 or more RHS the mixed handle's products run on the tensor cores:
    algorithmic complex-MAC flops (8 per MAC) against the measured bf16 peak
    (sustained: timed inside a long step).  Below 32 RHS every block is read
    once per launch for a handful of RHS: algorithmic bytes per launch against
    the measured HBM copy bandwidth.  FP64 chains with many RHS: FP64 flops
    against cuBLAS DGEMM measured here."""
    tot_ms = sum(p[1] for p in prof.values())
    name, (launches, ms, byts, flops) = max(prof.items(), key=lambda kv: kv[1][1])
    avg_s = ms / 1e3 / max(1.0, launches)
    share = ms / tot_ms
    tc = mixed and nrhs >= 32
    if flops > 0 and tc and (name in TENSOR_CATS or name in OZ_CATS or name == "dinv"):
        pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        ach = flops / max(launches, 1) / avg_s / 1e12
        # executed bf16 flops per algorithmic flop: 6 slice products (three-way
        # split) or 36 digit products (FP64-accurate slicing)
        xf = 6.0 if name in TENSOR_CATS else 36.0
        return {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": None, "kernel": name,
                "peak_source": f"{peak_kind} bf16_tflops_sustained",
                "note": "achieved counts 8 flops per complex MAC; the kernel executes "
                        + ("48 bf16 flops per complex MAC (3-way split, 6 slice products, "
                           "real-expanded complex)" if name in TENSOR_CATS else
                           "288 bf16 flops per complex MAC (8 digits, 36 slice products)"),
                "executed_tflops": ach * xf, "executed_frac": ach * xf / pk, "share": share}
    if nrhs < 32 or flops <= 0:
        ach = byts / max(launches, 1) / avg_s / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "traffic": None, "kernel": name,
                "peak_source": f"{peak_kind} hbm_gbs",
                "note": "algorithmic bytes per launch (every matrix block once, input and "
                        "output panels once) over the launch's CUDA-event time",
                "share": share}
    import torch
    fp32 = name in FP32_CATS
    pk = gemm_peak(dev, torch.float32 if fp32 else torch.float64)
    ach = flops / max(launches, 1) / avg_s / 1e12
    return {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
            "traffic": None, "kernel": name,
            "peak_source": ("cuBLAS SGEMM" if fp32 else "cuBLAS DGEMM")
                           + " 4096^3 measured in this run", "share": share}


def single_rhs_leg(sol, B1, steps, peaks, peak_kind, stream):
    """Rate of one-RHS solves and the achieved HBM bandwidth of the chain:
    algorithmic bytes of every launch (the library's per-launch counts) over
    the device time of the solve, and the roofline of its dominant category."""
    import torch
    X1 = torch.empty_like(B1)
    for _ in range(3):
        sol.solve(X1, B1)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        sol.solve(X1, B1)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / steps
    # the same solve replayed from a CUDA graph (the grouped entry point with
    # one problem): no host launch overhead between the chain's ~140-280 launches
    import paper_2109_04129_gb300 as hp
    Xg = torch.empty_like(B1)
    for _ in range(3):
        hp.solve_grouped([sol], [Xg], [B1])
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        hp.solve_grouped([sol], [Xg], [B1])
    e1.record(stream)
    torch.cuda.synchronize()
    tg = e0.elapsed_time(e1) / 1e3 / steps
    same = bool(torch.equal(Xg, X1))
    sol.profile_enable(True)
    sol.solve(X1, B1)
    prof = sol.profile()
    sol.profile_enable(False)
    byts = sum(p[2] for p in prof.values())
    launches = int(sum(p[0] for p in prof.values()))
    roof = roofline(prof, 1, sol.params.precision == 1, peaks, peak_kind, None)
    return {"value": 1.0 / t, "unit": "RHS/s", "ms_per_solve": 1e3 * t, "steps": steps,
            "alg_bytes_per_solve": byts, "achieved_gbs": byts / t / 1e9,
            "hbm_frac": byts / t / 1e9 / peaks["hbm_gbs"], "launches_per_solve": launches,
            "graph": {"value": 1.0 / tg, "ms_per_solve": 1e3 * tg,
                      "achieved_gbs": byts / tg / 1e9,
                      "hbm_frac": byts / tg / 1e9 / peaks["hbm_gbs"],
                      "equals_stream_solve": same},
            "roofline": roof, "kernels": kernel_table(prof, 1)}


# ------------------------------------------------------- grouped scatterer batch
BATCH_METRIC = "grouped power-series RHS solves/s over a batch of scatterers, mixed precision"


def run_batch(args):
    """A batch of independent closed scatterers (spheres, prolate ellipsoids,
    closed cylinders; 1920-31098 unknowns, leaf caps 32-256, 91 monostatic RHS
    each), all solved per step by one grouped call (one CUDA-graph launch with
    a branch per scatterer).  Compared with the same solves issued one after
    another on one stream."""
    ws, rank, local = dist_setup(args)
    from hm_workloads import scatterer_batch
    ws_list = scatterer_batch(args.batch_count)
    meshes = [w.build_mesh() for w in ws_list]
    sizes = [len(f) * 3 // 2 for _, f in meshes]
    small = int(min(range(len(sizes)), key=lambda i: sizes[i]))
    oracle = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        oracle = start_oracle(ws_list[small].name, args.cpu_rhs, 2)
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2109_04129_gb300 as hp
    prec = hp.HM_MIXED if args.precision == "mixed" else hp.HM_FP64
    t0 = time.perf_counter()
    sols, Bs = [], []
    for w, (v, f) in zip(ws_list, meshes):
        sol = hp.Solver.build(v, f, wavelength=w.wavelength, leaf_max=w.leaf_max,
                              aca_tol=w.aca_tol,
                              ordering=hp.HM_ORDER_ND if args.ordering == "nd" else hp.HM_ORDER_DFS,
                              precision=prec, refine_steps=1 if prec == hp.HM_MIXED else 0)
        sol.compute_scaling()
        th, ph, po = w.angles()
        B = torch.empty((len(th), sol.N), dtype=torch.complex128, device=dev)
        sol.plane_wave(B, th, ph, po)
        # one solve right away: sizes the work panels and tunes the sweeps, after
        # which the handle drops its complex64 matrix copies (the peak of device
        # memory stays one handle's transient above the batch's steady state)
        sol.solve(torch.empty_like(B), B)
        sols.append(sol)
        Bs.append(B)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    Ns = [s.N for s in sols]
    held_gb = sum(s.stats()["device_bytes"] for s in sols) / 1e9
    free_b, total_b = torch.cuda.mem_get_info(dev)
    nrhs_tot = sum(B.shape[0] for B in Bs)
    Xs = [torch.empty_like(B) for B in Bs]
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        hp.solve_grouped(sols, Xs, Bs)
    torch.cuda.synchronize()
    oracle_ready(oracle)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            hp.solve_grouped(sols, Xs, Bs)
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(ws)
    t_dev, value = job_rate(ws, nrhs_tot, e0.elapsed_time(e1) / 1e3 / args.steps, dev)
    # the same solves one after another on one stream (no graph)
    Ys = [torch.empty_like(B) for B in Bs]
    l0 = sols[0].stats()["kernel_launches"]
    for s, Y, B in zip(sols, Ys, Bs):
        s.solve(Y, B)
    torch.cuda.synchronize()
    launches_per_step = sols[0].stats()["kernel_launches"] - l0
    e0.record(stream)
    for _ in range(args.steps):
        for s, Y, B in zip(sols, Ys, Bs):
            s.solve(Y, B)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq, v_seq = job_rate(ws, nrhs_tot, e0.elapsed_time(e1) / 1e3 / args.steps, dev)
    same = all(torch.equal(X, Y) for X, Y in zip(Xs, Ys))
    ratio_max = max(float(np.max(s.diagnostics(B.shape[0])[0])) for s, B in zip(sols, Bs))
    # per-kernel timing: one profiled pass of the single solves (events around
    # every launch cannot be recorded in the graph)
    tot = {}
    for s, Y, B in zip(sols, Ys, Bs):
        s.profile_enable(True)
        s.solve(Y, B)
        for cat, v in s.profile().items():
            a = tot.setdefault(cat, [0.0, 0.0, 0.0, 0.0])
            for i in range(4):
                a[i] += v[i]
        s.profile_enable(False)
    tot_ms = sum(v[1] for v in tot.values())
    name, (launches, ms, byts, flops) = max(tot.items(), key=lambda kv: kv[1][1])
    peaks, peak_kind = measured_peaks()
    avg_s = ms / 1e3 / max(1.0, launches)
    if prec == hp.HM_MIXED and name in ("mixed_sweep", "mixed_far", "far_stage1", "far_stage2",
                                         "near"):
        pk = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
        ach = flops / max(launches, 1) / avg_s / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": None, "kernel": name,
                "peak_source": f"{peak_kind} bf16_tflops_sustained",
                "note": "per-launch durations from the profiled single solves; achieved "
                        "counts 8 flops per complex MAC", "share": ms / tot_ms}
    else:
        pk = gemm_peak(dev, torch.float64)
        ach = flops / max(launches, 1) / avg_s / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": None, "kernel": name,
                "peak_source": "cuBLAS DGEMM 4096^3 measured in this run", "share": ms / tot_ms}
    kernels = {c: {"ms_per_step": round(v[1], 3), "share": round(v[1] / tot_ms, 4),
                   "launches_per_step": int(v[0])} for c, v in tot.items() if v[0]}
    # end to end: pinned host B in, grouped solve, pinned host X out, every step
    Bh = [torch.empty(B.shape, dtype=B.dtype, pin_memory=True).copy_(B) for B in Bs]
    Xh = [torch.empty(B.shape, dtype=B.dtype, pin_memory=True) for B in Bs]
    Bd = [torch.empty_like(B) for B in Bs]

    def e2e_step():
        for d, h in zip(Bd, Bh):
            d.copy_(h, non_blocking=True)
        hp.solve_grouped(sols, Xs, Bd)
        for h, d in zip(Xh, Xs):
            h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()

    e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    t_e2e, v_e2e = job_rate(ws, nrhs_tot, (time.perf_counter() - t0) / args.steps, dev)
    nbytes = sum(B.numel() * 16 for B in Bs)
    n_handles = len(sols)
    # accuracy last: it closes every mixed handle once its comparator is done
    # (all handles resident leave no room for the FP64 comparators)
    del Ys, Bh, Xh, Bd
    torch.cuda.empty_cache()
    accuracy = batch_accuracy(sols, Xs, Bs, ws_list) if prec == hp.HM_MIXED else None
    line = {
        "metric": BATCH_METRIC, "value": value, "unit": "RHS/s", "n_gpus": ws,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": 1e3 * t_dev,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128" if prec == hp.HM_FP64 else
                 "mixed: c64 chain on tcgen05, c128 D^-1, FP64-accurate residual",
        "data": "synthetic",
        "config": {"workload": f"scatterer_batch: {n_handles} seeded closed scatterers "
                               f"(sphere / prolate ellipsoid / closed cylinder), N "
                               f"{min(Ns)}-{max(Ns)} (total {sum(Ns)}), leaves 32-256, "
                               f"91 monostatic RHS each ({nrhs_tot} total)",
                   "precision": args.precision, "ordering": args.ordering,
                   "l2": "inputs larger than L2 (all scatterers' factors), no flush",
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "setup_s": round(t_setup, 1), "series_ratio_max": ratio_max,
                   "device_gb_held_by_handles_after_set_up": round(held_gb, 1),
                   "device_gb_free_after_set_up": round(free_b / 1e9, 1)},
        "roofline": roof,
        "e2e": {"value": v_e2e, "unit": "RHS/s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
        "gpu_launches": launches_per_step * args.steps,
        "graph_launches": args.steps,
        "clocks": clk.summary(),
        "accuracy": accuracy,
        "sequential": {"value": v_seq, "unit": "RHS/s",
                       "ms_per_step": 1e3 * t_seq,
                       "what": "the same solves issued one after another, no graph",
                       "grouped_equals_sequential": same},
        "kernels": kernels,
    }
    if oracle is not None:
        line["cpu_baseline"] = oracle_result(
            oracle, f"the smallest scatterer ({ws_list[small].name}, N={Ns[small]})")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------- scaling study (set-up / solve vs N)
SCALING_METRIC = "set-up and solve time against N (icospheres at ~10 edges per wavelength)"


def run_scaling(args):
    """Set-up time, memory and solve time against N (the paper's scaling study,
    Sec. IV, Eq. 46-56, Figs. 3 and 5) on icospheres of increasing level at a
    fixed density: level L has radius 0.5 * 2^(L-3) wavelengths (level 5 is the
    2 lambda benchmark sphere), leaf cap 128, ACA 1e-4, nested-dissection
    order, reading A.  Per level: H-matrix build and scaling on the GPU (wall
    time), device bytes, and the device time of the mixed solve (362-RHS sweep
    and one RHS) and of the plain FP64 series (362 RHS and one RHS)."""
    import numpy as np
    import torch
    import paper_2109_04129_gb300 as hp
    from hm_workloads import icosphere, monostatic_angles
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    th, ph, po = monostatic_angles("theta", 0.0, 180.0, 1.0, 0.0, (0, 1))
    rows = []

    def timed(sol, B, steps):
        X = torch.empty_like(B)
        sol.solve(X, B)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            sol.solve(X, B)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / steps

    for L in args.levels:
        v, f = icosphere(L, 0.5 * 2 ** (L - 3))
        row = {"level": L, "radius_lambda": 0.5 * 2 ** (L - 3)}
        for prec in (hp.HM_MIXED, hp.HM_FP64):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sol = hp.Solver.build(v, f, leaf_max=128, aca_tol=1e-4, ordering=hp.HM_ORDER_ND,
                                  fill=hp.HM_FILL_NEAR if args.fill == "B" else hp.HM_FILL_FULL,
                                  precision=prec, refine_steps=1 if prec == hp.HM_MIXED else 0)
            t_build = time.perf_counter() - t0
            t0 = time.perf_counter()
            sol.compute_scaling()
            t_scale = time.perf_counter() - t0
            B = torch.empty((len(th), sol.N), dtype=torch.complex128, device=dev)
            sol.plane_wave(B, th, ph, po)
            t_many = timed(sol, B, max(2, args.steps // 2))
            t_one = timed(sol, B[:1].contiguous(), max(3, args.steps))
            st = sol.stats()
            tag = "mixed" if prec == hp.HM_MIXED else "fp64"
            row.update({"N": sol.N, "leaves": st["leaves"], "alpha_entries": st["alpha_entries"],
                        "near_entries": st["near_entries"], "far_entries": st["far_entries"],
                        f"{tag}_build_s": round(t_build, 2), f"{tag}_scaling_s": round(t_scale, 2),
                        f"{tag}_device_gb": round(st["device_bytes"] / 1e9, 2),
                        f"{tag}_ms_362rhs": round(1e3 * t_many, 3),
                        f"{tag}_rhs_per_s_362": round(len(th) / t_many, 1),
                        f"{tag}_ms_1rhs": round(1e3 * t_one, 3)})
            del sol, B
            torch.cuda.empty_cache()
        rows.append(row)
        print(json.dumps({"partial": row}), file=sys.stderr, flush=True)
    line = {"metric": SCALING_METRIC, "value": rows[-1]["mixed_rhs_per_s_362"], "unit": "RHS/s",
            "n_gpus": ws, "steps": args.steps, "warmup": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "mixed and c128", "data": "synthetic",
            "config": {"workload": "icospheres L" + ",".join(str(L) for L in args.levels) +
                       ", radius 0.5*2^(L-3) lambda, leaves<=128, ACA 1e-4, ND order, reading "
                       + ("B" if args.fill == "B" else "A") + ", 362 monostatic RHS and one RHS",
                       "value_is": "mixed RHS/s at the largest level"},
            "levels": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)


LEAF_STUDY = (  # (icosphere level, radius in wavelengths, leaf caps, eta, reference)
    (4, 1.0, (32, 64, 128, 256, 512, 1024), 0.0, "own"),
    (4, 1.0, (64, 256), 1.0, "own"),
    (5, 2.0, (128, 256, 512), 0.0, "first"),
    (5, 2.0, (256,), 1.0, "first"),
)


def run_leaf_study(args):
    """Accuracy of the power series against the leaf size (Sec. V-A, Fig. 4)
    on the GPU: for each sphere, leaf cap and admissibility constant of
    LEAF_STUDY, hm_build (ND order, reading A) and hm_compute_scaling, then
    the x-polarised theta = 0 plane wave solved by the FP64 series with 2, 3
    and 5 terms (the handle saved and loaded with each n_terms), the Eq. 45
    ratio, and the relative L2 error against the direct solution of the
    assembled H-matrix: Z applied to the identity in column chunks through
    hm_apply (FP64-accurate products of a mixed handle; Z = Z^T) and solved by
    a dense LU (torch.linalg.solve, the study's reference only).  "own": each
    cap's own matrix; "first": the first cap's matrix for every cap of the
    sphere (one LU; the matrices differ by the ACA tolerance)."""
    import tempfile
    import numpy as np
    import torch
    import paper_2109_04129_gb300 as hp
    from hm_workloads import icosphere
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rows = []
    d = tempfile.mkdtemp()
    path = os.path.join(d, "leaf.hmps")

    def dense_z(sol, chunk=2048):
        Zd = torch.empty((sol.N, sol.N), dtype=torch.complex128, device=dev)
        for c0 in range(0, sol.N, chunk):
            c = min(chunk, sol.N - c0)
            E = torch.zeros((c, sol.N), dtype=torch.complex128, device=dev)
            E[torch.arange(c, device=dev), torch.arange(c0, c0 + c, device=dev)] = 1.0
            sol.apply("Z", Zd[c0:c0 + c], E)      # rows of Z^T = columns of Z
            del E
        torch.cuda.synchronize()
        return Zd

    try:
        for level, radius, caps, eta, ref_kind in LEAF_STUDY:
            v, f = icosphere(level, radius)
            x_ref = None
            for cap in caps:
                t0 = time.perf_counter()
                sol = hp.Solver.build(v, f, wavelength=1.0, leaf_max=cap, aca_tol=1e-4,
                                      ordering=hp.HM_ORDER_ND, precision=hp.HM_MIXED,
                                      refine_steps=1, eta=eta)
                sol.compute_scaling()
                t_setup = time.perf_counter() - t0
                st = sol.stats()
                b = torch.empty((1, sol.N), dtype=torch.complex128, device=dev)
                sol.plane_wave(b, np.zeros(1), np.zeros(1), np.zeros(1, dtype=np.int32))
                if x_ref is None or ref_kind == "own":
                    Zd = dense_z(sol)
                    x_ref = torch.linalg.solve(Zd, b[0].unsqueeze(1))[:, 0]
                    resid = float((torch.linalg.vector_norm(Zd @ x_ref - b[0]) /
                                   torch.linalg.vector_norm(b[0])).item())
                    del Zd
                    torch.cuda.empty_cache()
                sol.save(path)
                sol.close()
                del sol
                errs, ratio = {}, None
                for nt in (2, 3, 5):
                    s2 = hp.Solver.load(path, precision=hp.HM_FP64, n_terms=nt)
                    X = torch.empty_like(b)
                    s2.solve(X, b)
                    if ratio is None:
                        ratio = float(s2.diagnostics(1)[0][0])
                    errs[f"err_{nt}_terms"] = float(
                        (torch.linalg.vector_norm(X[0] - x_ref) /
                         torch.linalg.vector_norm(x_ref)).item())
                    s2.close()
                os.unlink(path)
                row = {"level": level, "radius_lambda": radius, "N": st["N"],
                       "leaf_cap": cap, "eta": eta,
                       "leaves": st["leaves"], "reference": ref_kind,
                       "lu_residual": resid, "ratio_eq45": ratio, **errs,
                       "setup_s": round(t_setup, 2)}
                rows.append(row)
                print(json.dumps({"partial": row}), file=sys.stderr, flush=True)
                torch.cuda.empty_cache()
    finally:
        import shutil
        shutil.rmtree(d, ignore_errors=True)
    line = {"metric": "relative L2 error of the power-series solution against the direct "
                      "solution vs leaf size (Sec. V-A, Fig. 4)",
            "value": None, "unit": "relative L2 error", "n_gpus": ws, "steps": 1, "warmup": 0,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic",
            "config": {"workload": "icospheres 1 lambda (L4) and 2 lambda (L5), x-polarised "
                                   "theta=0 plane wave, ACA 1e-4, ND order, reading A",
                       "reference": "dense LU of the assembled H-matrix (torch.linalg.solve)"},
            "rows": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)


def batch_accuracy(sols, Xs, Bs, ws_list, bar=1e-4):
    """Each scatterer's grouped mixed result against the FP64 chain with the
    same refinement on the same set-up: the mixed handle is saved (H-matrix,
    scaling and supernodes, FP64 values), closed, and loaded as an FP64
    handle, one scatterer at a time (the mixed handles are closed here, so
    this comes last).  Returns the largest relative L2 error over all RHS and
    the scatterers whose error exceeds the bar."""
    import tempfile
    import numpy as np
    import torch
    import paper_2109_04129_gb300 as hp
    worst, over, per = 0.0, [], []
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "s.hmps")
        for i, (sol, X, B) in enumerate(zip(sols, Xs, Bs)):
            ratio = float(np.max(sol.diagnostics(B.shape[0])[0]))
            n = sol.N
            sol.save(path)
            sol.close()
            torch.cuda.empty_cache()
            ref = hp.Solver.load(path, precision=hp.HM_FP64, refine_steps=1)
            Xr = torch.empty_like(B)
            ref.solve(Xr, B)
            torch.cuda.synchronize()
            e = float((torch.linalg.vector_norm(X - Xr, dim=1) /
                       torch.linalg.vector_norm(Xr, dim=1)).max().item())
            per.append(round(e, 9))
            worst = max(worst, e)
            if e > bar:
                over.append({"scatterer": ws_list[i].name, "N": n, "rel_err": e,
                             "series_ratio_max": ratio})
            ref.close()
            del Xr
            os.unlink(path)
    return {"rel_err_max": worst, "bar": bar, "over_bar": over, "per_scatterer": per,
            "what": "grouped mixed solve vs FP64 chain + same refinement, same set-up"}


# ------------------------------------------------------- the 10 lambda sphere (RHS in chunks)
def run_large(args):
    """The 10 lambda sphere (icosphere level 7, N = 491520, leaves <= 256, ACA
    1e-4, 720 monostatic RHS theta = 0..179.75 step 0.25): H-matrix fill and
    scaling on the GPU, then the mixed series with one refinement over the
    720 RHS in chunks of --chunk RHS per call (the stage-1 far-field panels
    grow as 2 (sum of far ranks) x nrhs, which bounds one call's batch on one
    GPU).  Accuracy on the 8 sampled RHS 0, 90, ..., 630: against the library's
    FP64 chain with the same refinement on the same set-up (the mixed handle
    saved and loaded as FP64) and, with --oracle-check, against the CPU
    oracle's series + refinement on the library's own blocks (imported), which
    also gives the CPU baseline."""
    import tempfile
    import numpy as np
    import torch
    import paper_2109_04129_gb300 as hp
    from hm_workloads import get_workload
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    w = get_workload(args.workload)
    v, f = w.build_mesh()
    fill = hp.HM_FILL_FULL if args.fill == "A" else hp.HM_FILL_NEAR
    t0 = time.perf_counter()
    sol = hp.Solver.build(v, f, wavelength=w.wavelength, leaf_max=w.leaf_max, aca_tol=w.aca_tol,
                          ordering=hp.HM_ORDER_ND, fill=fill, precision=hp.HM_MIXED,
                          refine_steps=1, **engine_kw(args))
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    sol.compute_scaling()
    t_scale = time.perf_counter() - t0
    st = sol.stats()
    th, ph, po = w.angles()
    nrhs = len(th)
    B = torch.empty((nrhs, sol.N), dtype=torch.complex128, device=dev)
    sol.plane_wave(B, th, ph, po)
    X = torch.empty_like(B)
    c = max(1, min(args.chunk, nrhs))
    chunks = [(r, min(nrhs, r + c)) for r in range(0, nrhs, c)]

    def sweep():
        for a, b in chunks:
            sol.solve(X[a:b], B[a:b])

    sol.solve(X[:c], B[:c])                     # sizes the work panels
    torch.cuda.synchronize()
    free_b, total_b = torch.cuda.mem_get_info(dev)
    for _ in range(max(0, args.warmup - 1)):
        sweep()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = sol.stats()["kernel_launches"]
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            sweep()
        e1.record(stream)
        torch.cuda.synchronize()
    launches = sol.stats()["kernel_launches"] - l0
    t_dev = e0.elapsed_time(e1) / 1e3 / args.steps
    ratio = np.concatenate([sol.diagnostics(b - a)[0] for a, b in chunks[-1:]])
    sol.profile_enable(True)
    sol.solve(X[:c], B[:c])
    prof = sol.profile()
    sol.profile_enable(False)
    peaks, peak_kind = measured_peaks()
    roof = roofline(prof, c, True, peaks, peak_kind, dev)
    # end to end: pinned host chunks in and out through the host-buffer call
    Bh = torch.empty((nrhs, sol.N), dtype=torch.complex128, pin_memory=True)
    Bh.copy_(B)
    Xh = torch.empty_like(Bh, pin_memory=True)
    bn, xn = Bh.numpy(), Xh.numpy()
    t0 = time.perf_counter()
    for a, b in chunks:
        sol.solve_host(xn[a:b], bn[a:b])
    t_e2e = time.perf_counter() - t0
    idx = list(range(0, nrhs, 90))[:8]
    xm = X[idx].cpu().numpy().T.copy()
    bs = B[idx].cpu().numpy().T.copy()
    acc = {"sampled_rhs": idx}
    cpu = None
    import shutil
    import tempfile
    d = tempfile.mkdtemp()
    path = os.path.join(d, "s10.hmps")
    try:
        saved = False
        try:
            sol.save(path)
            saved = True
        except Exception as e:      # reported in the JSON line (e.g. no room for the file)
            acc["error"] = "save: " + repr(e)
        sol.close()
        del sol, X, Bh, Xh
        torch.cuda.empty_cache()
        x64 = None
        if saved:
            try:
                ref = hp.Solver.load(path, precision=hp.HM_FP64, refine_steps=1)
                Bs = torch.from_numpy(np.ascontiguousarray(bs.T)).to(dev)
                Xr = torch.empty_like(Bs)
                ref.solve(Xr, Bs)
                x64 = Xr.cpu().numpy().T
                e = np.linalg.norm(xm - x64, axis=0) / np.linalg.norm(x64, axis=0)
                acc["mixed_vs_gpu_fp64_refined_rel_err"] = [float(x) for x in e]
                ref.close()
            except Exception as e:
                acc["error"] = "fp64 comparator: " + repr(e)
        if saved and args.oracle_check:
            try:
                from oracle.export import load_blocks
                from oracle.series import refine_once, series_solve
                H, S = load_blocks(path)
                t0 = time.perf_counter()
                x2, _ = series_solve(H, S, bs, 2)
                xo = refine_once(H, S, bs, x2)
                t_or = time.perf_counter() - t0
                acc["mixed_vs_oracle_rel_err"] = [
                    float(x) for x in np.linalg.norm(xm - xo, axis=0) / np.linalg.norm(xo, axis=0)]
                if x64 is not None:
                    acc["gpu_fp64_vs_oracle_rel_err"] = [
                        float(x) for x in
                        np.linalg.norm(x64 - xo, axis=0) / np.linalg.norm(xo, axis=0)]
                cpu = {"value": len(idx) / t_or, "unit": "RHS/s", "cores": cpu_threads(),
                       "kind": "oracle",
                       "sample": f"the {len(idx)} sampled RHS, oracle FP64 series + one "
                                 "refinement step on the library's blocks (imported), one run"}
            except Exception as e:
                acc["oracle_error"] = repr(e)
    finally:
        shutil.rmtree(d, ignore_errors=True)
    acc["bar"] = 1e-4
    line = {
        "metric": METRIC, "value": nrhs / t_dev, "unit": "RHS/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "mixed: c64 chain on tcgen05 (3-way bf16 split, f32 accum), c128 D^-1, "
                 "FP64-accurate residual on tcgen05 (exact 7-bit slicing)",
        "data": "synthetic",
        "config": {"workload": workload_desc(w, st["N"], nrhs),
                   "precision": "mixed", "ordering": "nd",
                   "fill": "reading B (near-pattern fill)" if fill == hp.HM_FILL_NEAR
                           else "reading A (full fill)",
                   "rhs_per_call": c, "calls_per_step": len(chunks),
                   "l2": "inputs larger than L2, no flush", "parallelism": "single GPU",
                   "alpha_entries": st["alpha_entries"], "far_entries": st["far_entries"],
                   "near_entries": st["near_entries"], "leaves": st["leaves"],
                   "build_s": round(t_build, 1), "scaling_s": round(t_scale, 1),
                   "device_gb_held": round(st["device_bytes"] / 1e9, 1),
                   "device_gb_free_after_first_solve": round(free_b / 1e9, 1),
                   "series_ratio_max_last_chunk": float(np.max(ratio))},
        "roofline": roof, "accuracy": acc,
        "e2e": {"value": nrhs / t_e2e, "unit": "RHS/s", "h2d_bytes_per_step": int(bn.nbytes),
                "d2h_bytes_per_step": int(xn.nbytes)},
        "gpu_launches": launches, "clocks": clk.summary(), "kernels": kernel_table(prof, 1),
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    try:
        dispatch(args)
    finally:
        oracle_stop_all()


def dispatch(args):
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "sphere_r10_L7":
        run_large(args)
    elif args.workload == "sphere_scaling":
        run_scaling(args)
    elif args.workload == "leaf_size_study":
        run_leaf_study(args)
    elif args.workload == "scatterer_batch":
        run_batch(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
