#!/usr/bin/env python
"""Benchmark of the matrix-element hot path: pairs/s of H_ij, S_ij on one GB300.

A step is one tnqe_matrix_elements call over all M(M+1)/2 pairs of the
workload (rotation of every off-diagonal pair + transfer contraction of every
pair), with the states already resident in HBM.  Default workload: N = 14
spatial orbitals, 7 + 7 electrons, L = 28, M = 16 states at chi = 128
(136 pairs), seeded synthetic inputs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent
replica of the workload (the pairs of one workload need no exchange); value is
the units of all ranks over the slowest rank's time.
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

import numpy as np

METRIC = "pair matrix elements/s at N=14, chi=128 vs plain FP64 GPU; |dE| (Ha) vs oracle"
UNIT = "pairs/s"
PREC = {"fp64": 0, "tf32x3": 1, "bf16x3": 2, "bf16x6": 3, "bf16x10": 4, "bf16x15": 5}
DTYPE = {"fp64": "f64", "tf32x3": "tf32x3", "bf16x3": "bf16x3", "bf16x6": "bf16x6", "bf16x10": "bf16x10",
         "bf16x15": "bf16x15"}
PRODUCTS = {"bf16x3": 3, "bf16x6": 6, "bf16x10": 10, "bf16x15": 15}   # BF16 slice products per GEMM


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


def oracle_sample(w, seconds_cap=40.0):
    """The CPU oracle as it stands on a bounded sample of the workload's pairs."""
    from oracle import mps as om
    o = om.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff)
    for m in w.mps:
        o.add_mps(m.tensors, m.U)
    o.mpo(0)                      # basis-0 operator built outside the timed region (host planning)
    sample = [(0, 1), (0, 0)]
    done, t0 = [], time.time()
    for p in sample:
        o.pair(*p)
        done.append(p)
        if time.time() - t0 > seconds_cap:
            break
    el = time.time() - t0
    return len(done) / el, el, done


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args):
    from paper_2404_10223_gb300 import inputs
    rank, world, local = dist_init(args.gpus)
    if rank != 0:
        return
    w = inputs.workload(args.workload)
    times = []
    for _ in range(args.warmup):
        oracle_sample(w, 5.0)
    for _ in range(args.steps):
        v, el, done = oracle_sample(w, 20.0)
        times.append(el / len(done))
    value = 1.0 / statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(times) * len(w.all_pairs()),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, "fp64"),
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": cpu_threads(),
                             "sample": "pairs (0,1) and (0,0) of the workload per step, MPO of basis 0 prebuilt"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(w, prec):
    return {"workload": w.name, "N": w.N, "n_alpha": w.n_alpha, "n_beta": w.n_beta, "M": w.M,
            "pairs": len(w.all_pairs()), "chi": sorted(set(m.chi for m in w.mps)), "seed": w.seed,
            "cutoff": w.cutoff, "precision": prec, "l2": "flushed between steps (256 MiB write)"}


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
    stream = torch.cuda.Stream()
    g = tnqe.Context(w.h1, w.eri, w.N, w.n_alpha, w.n_beta, cutoff=w.cutoff, precision=PREC[args.precision],
                     cuda_stream=stream.cuda_stream, device=local)
    for m in w.mps:
        g.add_mps(m.tensors, m.U)
    tuned = None
    if args.shapes:
        tuned = [int(x) for x in args.shapes.split(",")]
        g.set_tuning(*tuned)
    elif args.precision.startswith("bf16") and not args.no_autotune:
        tuned, _ = g.autotune(pairs)      # launch shapes, chosen outside the timed region
    Hd = torch.zeros(npairs, dtype=torch.float64, device="cuda")
    Sd = torch.zeros(npairs, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        g.matrix_elements(pairs, Hd.data_ptr(), Sd.data_ptr())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    step_ms, prof = [], np.zeros(tnqe.TNQE_PROFILE_LEN)
    barrier(world)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        prof += g.last_profile()
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    replayed = g.graph_count() > 0
    ms = statistics.mean(step_ms)
    ms_max = max_over_ranks(ms, world)
    value = npairs * world / (ms_max / 1000.0)
    K = args.steps
    peaks, peak_src = load_peaks()
    fp64_peak = peaks["bf16_tflops"] * (1.25 / 2250.0)          # nominal FP64 : BF16 dense ratio
    if args.precision == "fp64":
        kern = {
            "rotate_pairs_kernel": (prof[0] / K, prof[4] / K, "alu", fp64_peak, "TFLOP/s"),
            "gemm_f64_grouped(stage1)": (prof[1] / K, prof[5] / K, "alu", fp64_peak, "TFLOP/s"),
            "spmm_f64_grouped": (prof[2] / K, prof[6] / K, "hbm", peaks["hbm_gbs"], "GB/s"),
            "gemm_f64_grouped(stage3)": (prof[3] / K, prof[7] / K, "alu", fp64_peak, "TFLOP/s"),
        }
    elif args.precision == "tf32x3":
        # TF32x3: three TF32 MMAs per product; useful FLOPs against the TF32 dense peak
        # (measured BF16 burst x nominal TF32:BF16 = 1.1 : 2.25) divided by 3
        tf32_eff = peaks["bf16_tflops"] * (1.1 / 2.25) / 3.0
        kern = {
            "rotate_pairs_kernel": (prof[0] / K, prof[4] / K, "alu", fp64_peak, "TFLOP/s"),
            "gemm_tf32x3_kernel(stage1)": (prof[1] / K, prof[5] / K, "tensor", tf32_eff, "TFLOP/s"),
            "spmm_t_f32_kernel": (prof[2] / K, prof[6] / K, "hbm", peaks["hbm_gbs"], "GB/s"),
            "gemm_tf32x3_kernel(stage3)": (prof[3] / K, prof[7] / K, "tensor", tf32_eff, "TFLOP/s"),
        }
    else:
        # sliced BF16: issued MMA FLOPs (useful x slice products) against the measured BF16 burst peak
        npr = PRODUCTS[args.precision]
        kern = {
            "rotate_pairs_kernel": (prof[0] / K, prof[4] / K, "alu", fp64_peak, "TFLOP/s"),
            "gemm_bf16s_kernel(stage1)": (prof[1] / K, npr * prof[5] / K, "tensor", peaks["bf16_tflops"], "TFLOP/s"),
            "spmm_df_kernel": (prof[2] / K, prof[6] / K, "hbm", peaks["hbm_gbs"], "GB/s"),
            "gemm_bf16s_kernel(stage3)": (prof[3] / K, npr * prof[7] / K, "tensor", peaks["bf16_tflops"], "TFLOP/s"),
            "slice_rows/cols/sites_kernel": (prof[10] / K, prof[11] / K, "hbm", peaks["hbm_gbs"], "GB/s"),
        }
    top = max(kern, key=lambda k: kern[k][0])
    # DRAM bytes per launch from the ncu captures in profiles/ (read + write), scaled from the
    # captured case to this launch by the units it processes; None where no capture of the
    # current kernel exists for this workload.
    n_rot = sum(1 for i, j in pairs if i != j)
    # rotate_pairs_kernel: 10.63 MB read + 0.76 MB written by a launch of 2 rotated pairs
    traffic_table = {("n14_chi128", "rotate_pairs_kernel"): 11.39e6 / 2 * n_rot}
    traffic = traffic_table.get((w.name, top))
    t_ms, work, bound, peak, unit = kern[top]
    achieved = (work / (t_ms / 1e3)) / (1e12 if unit == "TFLOP/s" else 1e9) if t_ms > 0 else 0.0
    roof = {"kernel": top, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak if peak else None, "traffic": traffic,
            "peak_source": ({"alu": "FP64 = measured bf16 burst x 1.25/2250 (nominal ratio)",
                             "tensor": ("TF32x3 useful = measured bf16 burst x 1.1/2.25 / 3"
                                        if args.precision == "tf32x3" else
                                        "measured bf16 burst; achieved counts every issued slice product"),
                             "hbm": f"hbm_gbs ({peak_src})"}[bound]),
            "ms_per_step": t_ms, "work_per_step": work,
            "breakdown_ms": {k: v[0] for k, v in kern.items()},
            "breakdown_scope": ("kernels of the main stream; with the sliced path the (i, i) pairs, which "
                                "need no rotation, contract on a second stream beside the rotation kernel "
                                "and are not in the breakdown")}
    # the plain FP64 form on the same workload, and |dE| of this precision against it
    Hh = Hd.cpu().numpy().copy()
    Sh = Sd.cpu().numpy().copy()
    fp64 = None
    if args.precision != "fp64" and args.fp64_steps > 0:
        g.set_precision(0)
        step()
        torch.cuda.synchronize()
        f_ms = []
        for _ in range(args.fp64_steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize()
            f_ms.append(e0.elapsed_time(e1))
        H64 = Hd.cpu().numpy().copy()
        S64 = Sd.cpu().numpy().copy()
        g.set_precision(PREC[args.precision])

        def energy(Hv, Sv):
            Mm = w.M
            Hm, Sm = np.zeros((Mm, Mm)), np.zeros((Mm, Mm))
            for (i, j), h, s in zip(pairs, Hv, Sv):
                Hm[i, j] = Hm[j, i] = h
                Sm[i, j] = Sm[j, i] = s
            return g.solve(Hm, Sm)[0][0]
        e_fast, e_64 = energy(Hh, Sh), energy(H64, S64)
        f_mean = statistics.mean(f_ms)
        fp64 = {"value": npairs * world / (max_over_ranks(f_mean, world) / 1000.0), "unit": UNIT,
                "ms_per_step": f_mean, "steps": args.fp64_steps,
                "speedup": (max_over_ranks(f_mean, world) / ms_max),
                "dE_Ha": abs(e_fast - e_64), "E_fp64": e_64,
                "max_dH": float(np.abs(Hh - H64).max()), "max_dS": float(np.abs(Sh - S64).max())}
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
        Hh, Sh = g.matrix_elements(pairs)
        torch.cuda.synchronize()
        if it > 0:
            e2e_ms.append(1000.0 * (time.perf_counter() - t0))
    e2e_v = npairs * world / (max_over_ranks(statistics.mean(e2e_ms), world) / 1000.0) if e2e_ms else None
    launches = int(prof[9])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {**config_of(w, args.precision), "pairs": npairs},
            "clocks": clk, "gpu_launches": launches,
            "graph": {"replayed": replayed, "tuned_shapes": tuned},
            "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 16 * npairs},
            "roofline": roof, "plain_fp64_gpu": fp64}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, el, done = oracle_sample(w, 30.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                                "sample": f"{len(done)} pairs {done} of the workload in {el:.1f} s "
                                          "(basis-0 MPO built outside the timed region)"}
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
    ap.add_argument("--precision", default="bf16x15", choices=list(PREC))
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed steps of the plain FP64 form (0 = skip)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
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
