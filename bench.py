#!/usr/bin/env python
"""Benchmark of the matrix-element hot path: pairs/s of H_ij, S_ij on one GB300.

A step is one tnqe_matrix_elements call over all M(M+1)/2 pairs of the
workload (rotation of every off-diagonal pair + transfer contraction of every
pair), with the states already resident in HBM.  Default workload: N = 14
spatial orbitals, 7 + 7 electrons, L = 28, M = 16 states at chi = 128
(136 pairs), seeded synthetic inputs.  Default form: the FP64 contraction in
particle-number charge blocks.  The line also times, on the same workload,
the plain (dense) FP64 GPU form and the sliced-BF16 tensor-core form, and
compares every form's H, S and lowest energy with the stored oracle values
(tests/golden/, written by the oracle alone).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica of the workload (the pairs of one workload need no exchange); value is
the units of all ranks over the slowest rank's time.
"""
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

import numpy as np

METRIC = "pair matrix elements/s at N=14, chi=128 vs plain FP64 GPU; |dE| (Ha) vs oracle"
UNIT = "pairs/s"
PREC = {"fp64": 0, "tf32x3": 1, "bf16x3": 2, "bf16x6": 3, "bf16x10": 4, "bf16x15": 5}
DTYPE = {"fp64": "f64", "tf32x3": "tf32x3", "bf16x3": "bf16x3", "bf16x6": "bf16x6", "bf16x10": "bf16x10",
         "bf16x15": "bf16x15"}
PRODUCTS = {"bf16x3": 3, "bf16x6": 6, "bf16x10": 10, "bf16x15": 15}   # BF16 slice products per GEMM
FORMS = {"blocks": 0, "dense": 1}                                      # FP64 contraction form


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples (clocks, throttle reasons) while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
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
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if n_gpus > 1 else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def blas_info():
    """Name and version of the BLAS numpy uses, and the host's core count."""
    try:
        d = np.show_config(mode="dicts")["Build Dependencies"]["blas"]
        name = f"{d.get('name')} {d.get('version')}"
    except Exception:
        name = "unknown"
    threads = os.environ.get("OPENBLAS_NUM_THREADS") or os.environ.get("OMP_NUM_THREADS")
    return name, int(threads) if threads else os.cpu_count()


def oracle_pair_times(w, sample):
    """Seconds per pair of the CPU oracle as it stands; the MPOs of the sample's bras
    are built outside the timed region (host planning, as tnqe_add_mps does)."""
    from oracle import mps as om
    o = om.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff)
    for m in w.mps:
        o.add_mps(m.tensors, m.U)
    for i in sorted({i for i, _ in sample}):
        o.mpo(i)
    out = []
    for p in sample:
        t0 = time.perf_counter()
        o.pair(*p)
        out.append(time.perf_counter() - t0)
    return out


def oracle_single_thread(workload, pair):
    """The same oracle pair on one BLAS thread, in a fresh interpreter (the thread count of a
    BLAS already loaded cannot be lowered)."""
    code = ("import sys, json, time; sys.path.insert(0, %r); import bench; "
            "from paper_2404_10223_gb300 import inputs; w = inputs.workload(%r); "
            "print(json.dumps(bench.oracle_pair_times(w, [%r])))") % (ROOT, workload, tuple(pair))
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])[0]


def cpu_baseline(w, pairs, single_thread=True):
    """The oracle on a bounded sample of the workload: one rotated pair (0, 1) and one
    unrotated pair (1, 1), each timed once, weighted by the workload's mix of rotated and
    unrotated pairs into the time of one whole step (an extrapolation, labelled as such)."""
    n_rot = sum(1 for i, j in pairs if i != j)
    n_unrot = len(pairs) - n_rot
    t_rot, t_unrot = oracle_pair_times(w, [(0, 1), (1, 1)])
    step_s = n_rot * t_rot + n_unrot * t_unrot
    blas, threads = blas_info()
    out = {"value": len(pairs) / step_s, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": (f"pairs (0,1) rotated {t_rot:.1f} s and (1,1) unrotated {t_unrot:.1f} s of {w.name}, "
                      f"MPOs of bases 0 and 1 built outside the timed region; value extrapolated to the "
                      f"step's {n_rot} rotated + {n_unrot} unrotated pairs ({step_s:.0f} s per step)"),
           "extrapolated": True, "nproc": os.cpu_count(), "blas": blas, "blas_threads": threads,
           "seconds_per_pair": {"rotated": t_rot, "unrotated": t_unrot}}
    if single_thread:
        t1 = oracle_single_thread(w.name, (1, 1))
        if t1 is not None:
            out["single_thread"] = {"pair": [1, 1], "seconds": t1, "speedup_of_all_cores": t1 / t_unrot}
    return out


def reference_cycle(w, k):
    """Pair of reference step k: bra 0 (one MPO, built before the timed steps) against the
    other states, with the unrotated pair (0, 0) in the workload's share of the steps."""
    pairs = w.all_pairs()
    frac = sum(1 for i, j in pairs if i == j) / len(pairs)
    if math.floor((k + 1) * frac) > math.floor(k * frac):
        return (0, 0)
    return (0, 1 + k % (w.M - 1))


def run_reference(args):
    from oracle import mps as om
    from paper_2404_10223_gb300 import inputs
    rank, world, local = dist_init(args.gpus)
    if rank != 0:
        return
    w = inputs.workload(args.workload)
    o = om.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff)
    for m in w.mps:
        o.add_mps(m.tensors, m.U)
    o.mpo(0)                                   # host planning, outside the timed steps
    for k in range(args.warmup):
        o.pair(*reference_cycle(w, k))
    times, done = [], []
    for k in range(args.steps):
        p = reference_cycle(w, k)
        t0 = time.perf_counter()
        o.pair(*p)
        times.append(time.perf_counter() - t0)
        done.append(p)
    ms = 1000.0 * statistics.mean(times)
    value = 1000.0 / ms
    blas, threads = blas_info()
    n_unrot = sum(1 for p in done if p[0] == p[1])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, "fp64"),
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": threads, "nproc": os.cpu_count(),
                             "blas": blas,
                             "sample": (f"one pair of {w.name} per step ({args.steps - n_unrot} rotated, {n_unrot} "
                                        "unrotated, the workload's mix), bra 0 whose MPO is built before the "
                                        "timed steps; value = pairs / time of those steps")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(w, prec):
    return {"workload": w.name, "N": w.N, "n_alpha": w.n_alpha, "n_beta": w.n_beta, "M": w.M,
            "pairs": len(w.all_pairs()), "chi": sorted(set(m.chi for m in w.mps)), "seed": w.seed,
            "cutoff": w.cutoff, "precision": prec, "l2": "flushed between steps (256 MiB write)"}


def golden(name):
    path = os.path.join(ROOT, "tests", "golden", f"{name}_oracle.npz")
    return dict(np.load(path)) if os.path.exists(path) else None


def measure_fp64_peak(torch):
    """FP64 rate of this GPU: cuBLAS DGEMM through torch.matmul (4096^3, best of 3)."""
    n = 4096
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def run_native(args):
    import torch
    from paper_2404_10223_gb300 import build as B
    from paper_2404_10223_gb300 import inputs, tnqe
    rank, world, local = dist_init(args.gpus)
    torch.cuda.set_device(local)
    if not os.path.exists(B.LIB):
        if rank == 0:
            B.build()
        barrier(world)
    tnqe.load()
    w = inputs.workload(args.workload)
    pairs = w.all_pairs()
    if args.states:                       # only the pairs among these states (profiling captures)
        keep = {int(x) for x in args.states.split(",")}
        pairs = [(i, j) for i, j in pairs if i in keep and j in keep]
    if args.max_pairs > 0:                # a smaller case of the same workload (profiling captures)
        pairs = pairs[:args.max_pairs]
    npairs = len(pairs)
    gold = golden(w.name)
    fp64_peak = measure_fp64_peak(torch) if not args.no_fp64_peak else None
    stream = torch.cuda.Stream()
    form = FORMS[args.form]
    g = tnqe.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff, precision=PREC[args.precision],
                     contraction_form=form, cuda_stream=stream.cuda_stream, device=local)
    for m in w.mps:
        g.add_mps(m.tensors, m.U)
    tuned = None
    if args.shapes:
        tuned = [int(x) for x in args.shapes.split(",")]
        g.set_tuning(*tuned)
    elif (args.precision.startswith("bf16") or (args.precision == "fp64" and args.form == "blocks")) \
            and not args.no_autotune:
        tuned, _ = g.autotune(pairs)      # launch shapes, chosen outside the timed region
    Hd = torch.zeros(npairs, dtype=torch.float64, device="cuda")
    Sd = torch.zeros(npairs, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        g.matrix_elements(pairs, Hd.data_ptr(), Sd.data_ptr())

    def timed(K, prof=None):
        out = []
        for _ in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
            if prof is not None:
                prof += g.last_profile()
        return out

    def energy(Hv, Sv):
        Hm, Sm = np.zeros((w.M, w.M)), np.zeros((w.M, w.M))
        for (i, j), h, s_ in zip(pairs, Hv, Sv):
            Hm[i, j] = Hm[j, i] = h
            Sm[i, j] = Sm[j, i] = s_
        return g.solve(Hm, Sm)[0][0]

    def vs_oracle(Hv, Sv):
        """Element-wise against the stored oracle pairs present in this call; |dE| when all are."""
        if gold is None:
            return None
        where = {(int(i), int(j)): k for k, (i, j) in enumerate(gold["pairs"])}
        idx = [(p, where[pr]) for p, pr in enumerate(pairs) if pr in where]
        if not idx:
            return None
        a = np.array([p for p, _ in idx])
        b = np.array([k for _, k in idx])
        out = {"pairs_compared": len(idx), "max_dH": float(np.abs(Hv[a] - gold["H"][b]).max()),
               "max_dS": float(np.abs(Sv[a] - gold["S"][b]).max())}
        if "E" in gold and len(idx) == len(pairs) == len(w.all_pairs()):
            out["dE_Ha"] = abs(energy(Hv, Sv) - float(gold["E"][0]))
            out["E_oracle"] = float(gold["E"][0])
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    prof = np.zeros(tnqe.TNQE_PROFILE_LEN)
    barrier(world)
    torch.cuda.synchronize()
    step_ms = timed(args.steps, prof)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    replayed = g.graph_count() > 0
    ms = statistics.mean(step_ms)
    ms_max = max_over_ranks(ms, world)
    value = npairs * world / (ms_max / 1000.0)
    K = args.steps
    Hh = Hd.cpu().numpy().copy()
    Sh = Sd.cpu().numpy().copy()
    peaks, peak_src = load_peaks()
    alu_peak = fp64_peak if fp64_peak else peaks["bf16_tflops"] * (1.25 / 2250.0)
    alu_src = ("measured FP64 rate of this GPU: cuBLAS DGEMM (torch.matmul 4096^3, best of 3) before the timed steps"
               if fp64_peak else "FP64 = measured bf16 burst x 1.25/2250 (nominal ratio)")
    rot = ("rotate_pairs_kernel", (prof[0] / K, prof[4] / K, "alu", alu_peak, "TFLOP/s"))
    if args.precision == "fp64" and form == FORMS["blocks"]:
        kern = dict([rot,
                     ("bs_stage1_kernel", (prof[1] / K, prof[5] / K, "alu", alu_peak, "TFLOP/s")),
                     ("bs_stage2_kernel", (prof[2] / K, prof[8] / K, "alu", alu_peak, "TFLOP/s")),
                     ("bs_stage3_kernel", (prof[3] / K, prof[7] / K, "alu", alu_peak, "TFLOP/s"))])
    elif args.precision == "fp64":
        kern = dict([rot,
                     ("gemm_f64_grouped(stage1)", (prof[1] / K, prof[5] / K, "alu", alu_peak, "TFLOP/s")),
                     ("spmm_f64_grouped", (prof[2] / K, prof[6] / K, "hbm", peaks["hbm_gbs"], "GB/s")),
                     ("gemm_f64_grouped(stage3)", (prof[3] / K, prof[7] / K, "alu", alu_peak, "TFLOP/s"))])
    elif args.precision == "tf32x3":
        tf32_eff = peaks["bf16_tflops"] * (1.1 / 2.25) / 3.0
        kern = dict([rot,
                     ("gemm_tf32x3_kernel(stage1)", (prof[1] / K, prof[5] / K, "tensor", tf32_eff, "TFLOP/s")),
                     ("spmm_t_f32_kernel", (prof[2] / K, prof[6] / K, "hbm", peaks["hbm_gbs"], "GB/s")),
                     ("gemm_tf32x3_kernel(stage3)", (prof[3] / K, prof[7] / K, "tensor", tf32_eff, "TFLOP/s"))])
    else:
        npr = PRODUCTS[args.precision]
        kern = dict([rot,
                     ("gemm_bf16s_kernel(stage1)", (prof[1] / K, npr * prof[5] / K, "tensor", peaks["bf16_tflops"], "TFLOP/s")),
                     ("spmm_df_kernel", (prof[2] / K, prof[6] / K, "hbm", peaks["hbm_gbs"], "GB/s")),
                     ("gemm_bf16s_kernel(stage3)", (prof[3] / K, npr * prof[7] / K, "tensor", peaks["bf16_tflops"], "TFLOP/s")),
                     ("slice_rows/cols/sites_kernel", (prof[10] / K, prof[11] / K, "hbm", peaks["hbm_gbs"], "GB/s"))])
    top = max(kern, key=lambda k: kern[k][0])
    # DRAM bytes per launch from an ncu capture of the current kernel (profiles/), scaled from the
    # captured case to this launch by the units it processes; None where no capture exists.
    n_rot = sum(1 for i, j in pairs if i != j)
    # rotate_pairs_kernel (1024-thread CTAs, 12-warp lead team): 10.58 MB read + 0.57 MB written by
    # a launch of 2 rotated pairs of n14_chi128 (profiles/rotate_pairs_n14_small.md)
    traffic_table = {("n14_chi128", "rotate_pairs_kernel"): 11.154e6 / 2 * n_rot}
    traffic = traffic_table.get((w.name, top))
    t_ms, work, bound, peak, unit = kern[top]
    achieved = (work / (t_ms / 1e3)) / (1e12 if unit == "TFLOP/s" else 1e9) if t_ms > 0 else 0.0
    roof = {"kernel": top, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak if peak else None, "traffic": traffic,
            "peak_source": {"alu": alu_src,
                            "tensor": ("TF32x3 useful = measured bf16 burst x 1.1/2.25 / 3"
                                       if args.precision == "tf32x3" else
                                       "measured bf16 burst; achieved counts every issued slice product"),
                            "hbm": f"hbm_gbs ({peak_src})"}[bound],
            "ms_per_step": t_ms, "work_per_step": work,
            "work_definition": ("rotation: per gate 2 dL dM dR (two-site blocks) + 8 m n (gate) + 4 m n^2 + "
                                "8 n^3 per m x n charge block (LAPACK-SVD-equivalent), counted in the kernel"
                                if top == "rotate_pairs_kernel" else "algorithmic FLOPs of the blocks computed"),
            "breakdown_ms": {k: v[0] for k, v in kern.items()},
            "kernels": {k: {"ms_per_step": v[0], "work_per_step": v[1], "bound": v[2], "unit": v[4],
                            "achieved": ((v[1] / (v[0] / 1e3)) / (1e12 if v[4] == "TFLOP/s" else 1e9)) if v[0] > 0 else 0.0,
                            "frac": (((v[1] / (v[0] / 1e3)) / (1e12 if v[4] == "TFLOP/s" else 1e9)) / v[3])
                            if v[0] > 0 and v[3] else None}
                        for k, v in kern.items()},
            "breakdown_scope": ("kernels of the main stream; in the sliced and charge-block forms the (i, i) "
                                "pairs, which need no rotation, contract on a second stream beside the "
                                "rotation kernel and are not in the breakdown")}
    # the other forms on the same workload: the plain (dense) FP64 GPU form and the sliced BF16 form
    others = {}
    if args.compare_steps > 0:
        cfgs = [("plain_fp64_gpu", "fp64", "dense"), ("mixed_precision_bf16x15", "bf16x15", "dense")]
        for key, prec, fm in cfgs:
            if (prec, fm) == (args.precision, args.form) or args.compare_steps <= 0:
                continue
            g.set_precision(PREC[prec])
            g.set_form(FORMS[fm])
            if prec.startswith("bf16") and not args.no_autotune:
                g.autotune(pairs)
            step()
            step()                         # the second identical call captures the graph
            torch.cuda.synchronize()
            f_ms = statistics.mean(timed(args.compare_steps))
            f_max = max_over_ranks(f_ms, world)
            Hx, Sx = Hd.cpu().numpy().copy(), Sd.cpu().numpy().copy()
            others[key] = {"value": npairs * world / (f_max / 1000.0), "unit": UNIT, "ms_per_step": f_ms,
                           "steps": args.compare_steps, "precision": prec, "form": fm,
                           "headline_speedup": f_max / ms_max, "vs_oracle": vs_oracle(Hx, Sx)}
        g.set_precision(PREC[args.precision])
        g.set_form(form)
        if args.shapes:
            g.set_tuning(*tuned)
        elif args.precision.startswith("bf16") and not args.no_autotune:
            g.autotune(pairs)
    # end to end through host buffers: H2D of every state, D2H of H and S
    pinned = []
    h2d = 0
    for m in w.mps:
        ts = [torch.from_numpy(np.ascontiguousarray(t)).pin_memory() for t in m.tensors]
        U = torch.from_numpy(np.ascontiguousarray(m.U)).pin_memory()
        pinned.append((ts, U))
        h2d += sum(t.numel() * 8 for t in ts) + U.numel() * 8
    e2e_ms = []
    for it in range(0 if args.no_e2e else max(1, min(args.steps, 3)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.reset_mps()
        for ts, U in pinned:
            g.add_mps([t.numpy() for t in ts], U.numpy())
        He, Se = g.matrix_elements(pairs)
        torch.cuda.synchronize()
        if it > 0:
            e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    e2e_v = npairs * world / (max_over_ranks(statistics.mean(e2e_ms), world) / 1000.0) if e2e_ms else None
    launches = int(prof[9])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {**config_of(w, args.precision), "pairs": npairs, "form": args.form},
            "clocks": clk, "gpu_launches": launches,
            "graph": {"replayed": replayed, "tuned_shapes": tuned},
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 16 * npairs},
            "roofline": roof, "vs_oracle": vs_oracle(Hh, Sh), **others}
    if "plain_fp64_gpu" in others:
        line["speedup_vs_plain_fp64_gpu"] = others["plain_fp64_gpu"]["headline_speedup"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, pairs, single_thread=not args.no_single_thread)
    g.close()
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="n14_chi128")
    ap.add_argument("--precision", default="fp64", choices=list(PREC))
    ap.add_argument("--form", default="blocks", choices=list(FORMS),
                    help="FP64 contraction in charge blocks (default) or dense")
    ap.add_argument("--compare-steps", type=int, default=2,
                    help="timed steps of the plain FP64 and sliced-BF16 forms (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-single-thread", action="store_true", help="skip the one-thread oracle leg")
    ap.add_argument("--no-fp64-peak", action="store_true", help="skip the DGEMM probe of the FP64 peak")
    ap.add_argument("--max-pairs", type=int, default=0, help="use only the first K pairs (profiling on a small case)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes (profiling)")
    ap.add_argument("--shapes", default="", help="bn1,bn3,spmm_bw launch shapes instead of autotuning")
    ap.add_argument("--states", default="", help="comma-separated state ids: only pairs among them (profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
