#!/usr/bin/env python3
"""Benchmark: conjugate-gradient time to relative residual 1e-10 on the largest
single-GPU system -- the 256^3 synthetic FEM stiffness matrix (16.4M rows,
244M non-zeros, four high-contrast inclusions) in symmetric storage (upper
triangle and diagonal, 130M stored entries) -- with mixed precision against
plain FP64 CG on the same GPU, the SpMV HBM bandwidth of each storage format,
and the CPU oracle timed beside it.

One step = one solve from x0 = 0 to a true relative residual <= 1e-10 with the
headline method: single-precision CG iterations on single-precision values,
refined by double-precision reliable updates (the correction is accumulated
in double and the residual replaced by the double-precision b - A x, with the
double-precision values, every decade of residual reduction), inputs resident
in HBM.  The JSON line also carries the plain FP64 CG and the restarted
refinement on the same system and storage, full CSR storage at the same size,
the 128^3 system in all three storage formats, the paper-size system, the
batched, differentiation and 2010-structure legs, and the CPU oracle (one
thread and every host core), each solve with its error against the FP64
oracle's solution.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1: every rank solves its own replica of the system (the solve does not
shard without a collective); timing is the max over ranks.  Without torchrun
the script starts the N ranks itself.
"""
from __future__ import annotations

import argparse
import json
import os
import signal
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import femgen  # noqa: E402

METRIC = "CG time-to-1e-10 residual (s) & SpMV HBM GB/s; mixed/batched vs FP64 CG"
GRIDS = {"128": femgen.LARGE, "31": femgen.PAPER_SIZE, "64": femgen.DIFF, "256": femgen.LARGEST}
TOL = 1e-10
# DRAM bytes (read + write) per single-precision iteration of the headline
# kernel on the same system, by (storage, precision, grid): the difference of
# two ncu captures of one launch, 130 and 30 iterations (None until a capture
# of the current kernel exists).
DRAM_BYTES_PER_ITERATION = {("sym", "fp32_ru", "256"): 1_671_218_550}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--grid", default="256", choices=sorted(GRIDS))
    ap.add_argument("--format", default="sym", choices=["sym", "csr", "csc"])
    ap.add_argument("--precision", default="fp32_ru", choices=["fp32_ru", "fp32_ir", "fp64"])
    ap.add_argument("--inner-tol", type=float, default=1e-4)
    ap.add_argument("--no-extras", action="store_true", help="skip the per-format and CPU-baseline legs")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="only run solves capped at this many iterations (small case for ncu captures)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="budget of each CPU-oracle sample")
    ap.add_argument("--e2e-steps", type=int, default=3, help="end-to-end solves (host memory in and out)")
    ap.add_argument("--no-cpu-full-solve", action="store_true",
                    help="skip the complete 128^3 oracle solve on every host core")
    ap.add_argument("--only-batched", action="store_true", help="only run the batched leg")
    ap.add_argument("--only-differentiable", action="store_true", help="only run the differentiation leg")
    ap.add_argument("--only-paper-size", action="store_true", help="only run the paper-size leg")
    ap.add_argument("--only-ablation", action="store_true", help="only run the 2010-structure ablation leg")
    ap.add_argument("--only-largest", action="store_true",
                    help="only run the comparison solves and products of the 256^3 system")
    ap.add_argument("--profile-batched", type=int, default=0,
                    help="only one mixed-precision solve of the first N batch instances (small case for ncu)")
    ap.add_argument("--profile-spmv", action="store_true",
                    help="only run a few products (double then single precision) of --format, for ncu captures")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def spawn_ranks(args):
    """--gpus N > 1 outside torchrun: start N ranks (one per GPU) through
    torch.distributed.run on this node and pass their output through."""
    import socket

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def dist_setup(args):
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


def max_over_ranks(values, pg, device):
    """Element-wise max of a list of floats over all ranks (replica timing:
    the job is as slow as its slowest GPU).  Identity without a process group."""
    if not pg:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def golden(grid_key, fmt="sym"):
    p = os.path.join(ROOT, "tests", "golden", f"oracle_{grid_key}_{fmt}.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def err_vs_oracle(x_np, gold):
    """Relative difference to the FP64 oracle's solution over the golden
    file's seeded sample positions (None without a golden file)."""
    if not gold:
        return None
    idx = np.asarray(gold["sample_index"])
    xo = np.asarray(gold["sample_x"])
    return float(np.linalg.norm(x_np[idx] - xo) / np.linalg.norm(xo))


def oracle_iteration_seconds(fmt, arrays, b, lib, budget_s, min_iters=5, max_iters=5000):
    """Seconds per CG iteration of the oracle build ``lib`` on this system:
    two runs of m0 and m1 iterations, the difference divided by m1 - m0 (the
    set-up and the closing true-residual product cancel)."""
    import oracle

    m0 = 2
    t0 = time.perf_counter()
    oracle.cg(fmt, *arrays, b, tol=0.0, maxit=m0, lib=lib)
    t_small = time.perf_counter() - t0
    probe = 3
    t0 = time.perf_counter()
    oracle.cg(fmt, *arrays, b, tol=0.0, maxit=m0 + probe, lib=lib)
    spi = max((time.perf_counter() - t0 - t_small) / probe, 1e-9)
    m1 = m0 + int(max(min_iters, min(max_iters, budget_s / spi)))
    t0 = time.perf_counter()
    oracle.cg(fmt, *arrays, b, tol=0.0, maxit=m1, lib=lib)
    t_big = time.perf_counter() - t0
    return max(t_big - t_small, 1e-9) / (m1 - m0), m1 - m0, t_small


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (the JSON line carries their summary); GBCG_CLOCKS_DIR
        # keeps them somewhere else than the temporary directory
        self.path = os.path.join(os.environ.get("GBCG_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"gbcg_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
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
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def flush_l2(torch, buf):
    buf.add_(1.0)  # 256 MiB write, larger than the 129 MB L2


# What bounds the headline kernel, by storage, precision and grid, from its
# ncu captures: "hbm" when DRAM throughput is the limiter, "latency" when
# neither DRAM nor any pipe is saturated (barriers and dependent round trips;
# at 128^3 the symmetric iteration's bytes largely stay in L2, 24% DRAM
# throughput, barrier stalls first).
ROOF_BOUND = {("sym", "fp32_ru", "256"): "hbm", ("sym", "fp32_ru", "128"): "latency",
              ("csr", "fp32_ru", "128"): "latency"}


def per_iteration_bytes(stats, precision):
    """Algorithmic bytes of one CG iteration: the product (matrix arrays, ptr,
    x read once, y written once) plus the vector passes x += a p, r -= a q,
    r'r (read p, q, x, r; write x, r) and p = r + b p (read r, p; write p)."""
    n = stats["n"]
    if precision == "fp64":
        return stats["spmv_bytes_fp64"] + 9 * 8 * n
    return stats["spmv_bytes_fp32"] + 9 * 4 * n


# ---------------------------------------------------------------- reference
def workload_config(g, s, args, world):
    """The config object of the timed workload, the same in both arms."""
    nnz_stored = {"sym": (s.nnz + s.n) // 2, "csr": s.nnz, "csc": s.nnz}[args.format]
    return {"workload": f"fem {g.nx}x{g.ny}x{g.nz} P1 stiffness, {g.n_incl} inclusion(s), contrast "
                        f"{g.contrast:g}, {args.format} storage, {args.precision}, tol 1e-10",
            "n": s.n, "nnz": s.nnz, "nnz_stored": int(nnz_stored),
            "l2": ("matrix larger than L2; " if 12 * nnz_stored > 129e6 else "matrix fits L2; ")
                  + "256 MiB L2 flush before every step",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_reference(args):
    """The reference arm: the oracle (its multi-threaded build, which gives
    the single-threaded build's bits) on every host core, on this arm's
    workload.  Each step times a bounded run of CG iterations; the value is
    the seconds per iteration times the oracle's own iteration count to 1e-10
    (tests/golden)."""
    world, rank, local, pg = dist_setup(args)
    if rank != 0:  # rank 0 alone times the oracle; the others exit without work
        if pg:
            pg.destroy_process_group()
        return 0
    import oracle

    g = GRIDS[args.grid]
    s = femgen.build_system(g)
    arrays = s.upper()
    gold = golden(args.grid, "sym")
    cores = os.cpu_count() or 1
    lib = oracle.load_threaded(cores)
    spi, m, setup_s = oracle_iteration_seconds("sym", arrays, s.b, lib, args.cpu_seconds / 3)
    per_step = int(max(5, min(5000, args.cpu_seconds / spi)))
    iters_needed = gold["iterations"] if gold else None
    times = []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.cg("sym", *arrays, s.b, tol=0.0, maxit=per_step, lib=lib)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(max(dt - setup_s, 1e-9) / per_step)
    spi = statistics.median(times)
    value = spi * iters_needed + setup_s if iters_needed else None
    sample = (f"{per_step} CG iterations per step of the double-precision oracle (symmetric storage, the "
              f"oracle's own method) on the {g.nx}x{g.ny}x{g.nz} system, {oracle.threads(lib)} threads, minus its "
              f"set-up, scaled by the oracle's own iteration count to 1e-10 ({iters_needed}, "
              f"tests/golden/oracle_{args.grid}_sym.json) plus one set-up")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.median(times) * per_step,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(g, s, args, world),
            "cpu_baseline": {"value": value, "unit": "s", "cores": oracle.threads(lib), "kind": "oracle",
                             "sample": sample, "seconds_per_iteration": spi},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


# --------------------------------------------------------------------- ours
def run_ours(args):
    import torch

    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    import paper_1010_4639_gb300 as gb

    gb.build()
    dev = torch.device("cuda", local)
    if args.only_batched:
        print(json.dumps({"batched": batched(torch, gb, args)}), flush=True)
        return 0
    if args.only_ablation:
        print(json.dumps({"ablation_2010": ablation(torch, gb, args, femgen.build_system(femgen.LARGE))}),
              flush=True)
        return 0
    if args.only_largest:
        hbm, _ = peaks()
        s = femgen.build_system(femgen.LARGEST)
        print(json.dumps({"largest": extras(torch, gb, s, {"sym": s.upper(), "csr": (s.ptr, s.idx, s.val)}, None,
                                            args, hbm, golden("256", "sym"))}), flush=True)
        return 0
    if args.only_paper_size:
        print(json.dumps({"paper_size": paper_size(torch, gb, args)}), flush=True)
        return 0
    if args.only_differentiable:
        print(json.dumps({"differentiable": differentiable(torch, gb, args)}), flush=True)
        return 0
    if args.profile_batched:
        bs = femgen.build_batch(femgen.batched_instances(256)[:args.profile_batched], nrhs=8)
        with gb.Batch(bs.row_off, bs.ptr, bs.idx, bs.val, nrhs=8, tune=False) as Bt:
            Bt.set_tuning("fp32_ir", 512, 4, [1, 1, 1, 16, 1, 1, 1, 1])
            _, _, rep = Bt.solve(torch.from_numpy(bs.B).to(dev), tol=TOL, maxit=100000, precision="fp32_ir")
            st = Bt.stats()
        print(json.dumps({"profile_batched": args.profile_batched, "n": bs.n, "nnz": bs.nnz, "report": rep,
                          "iter_bytes_fp32": st["iter_bytes_fp32"]}), flush=True)
        return 0
    g = GRIDS[args.grid]
    s = femgen.build_system(g)
    fmt_arrays = {"sym": s.upper(), "csr": (s.ptr, s.idx, s.val)}
    if args.format == "csc":
        fmt_arrays["csc"] = s.csc()
    A = gb.Matrix(args.format, *fmt_arrays[args.format])
    st = A.stats()
    b = torch.from_numpy(s.b).to(dev)
    x = torch.zeros_like(b)
    solve_kw = dict(tol=TOL, precision=args.precision,
                    inner_tol=args.inner_tol if args.precision == "fp32_ir" else 0.0)
    if args.profile_spmv:
        xv = torch.from_numpy(femgen.random_vector(s.n, 7)).to(dev)
        yv = torch.empty_like(xv)
        for _ in range(max(1, args.warmup)):
            A.spmv(xv, yv)
            A.spmv_f32(xv.float(), yv.float())
        torch.cuda.synchronize()
        print(json.dumps({"profile_spmv": args.format, "stats": st}), flush=True)
        return 0
    if args.profile_iters:
        solve_kw.update(maxit=args.profile_iters, raise_on_error=False)
        for _ in range(max(1, args.warmup)):
            x.zero_()
            A.solve(b, x, **solve_kw)
        torch.cuda.synchronize()
        print(json.dumps({"profile_iters": args.profile_iters, "stats": st}), flush=True)
        return 0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        x.zero_()
        A.solve(b, x, **solve_kw)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            x.zero_()
            flush_l2(torch, flush)
            ev[k][0].record(stream)
            _, info = A.solve(b, x, **solve_kw)
            ev[k][1].record(stream)
            infos.append(info)
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    ms = sum(step_ms) / len(step_ms)
    kernel_ms = sum(i.kernel_ms for i in infos) / len(infos)
    kernel_launches = sum(i.kernel_launches for i in infos) / len(infos)
    iters = infos[-1].iterations
    updates = infos[-1].outer
    ms, kernel_ms = max_over_ranks([ms, kernel_ms], pg, dev)
    x_dev = x.clone()
    # end to end through the public API: pinned host b and x, copies inside the call
    bh = torch.from_numpy(s.b).pin_memory()
    xh = torch.zeros(s.n, dtype=torch.float64).pin_memory()
    e2e = []
    for k in range(max(1, min(args.steps, args.e2e_steps))):
        xh.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info_h = A.solve(bh, xh, **solve_kw)
        e2e.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks([statistics.median(e2e)], pg, dev)[0]
    hbm, peak_kind = peaks()
    per_it = per_iteration_bytes(st, args.precision)
    moved = per_it * iters
    if args.precision == "fp32_ru":  # the double-precision updates: product + x, d, b, r passes
        moved += updates * per_iteration_bytes(st, "fp64")
    achieved = moved / (kernel_ms / 1000.0) / 1e9 if kernel_ms > 0 else None
    dram_it = DRAM_BYTES_PER_ITERATION.get((args.format, args.precision, args.grid))
    traffic = dram_it * iters if dram_it else None  # the 10 updates' share (< 0.1%) left out
    x_np = x_dev.cpu().numpy()
    gold = golden(args.grid, "sym")
    kernel_names = {"fp32_ir": "k_cg<float> persistent inner CG", "fp32_ru": "k_cg_ru persistent CG, "
                    "single-precision iterations with double-precision reliable updates",
                    "fp64": "k_cg<double> persistent CG"}
    line = {
        "metric": METRIC, "value": ms / 1000.0, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": workload_config(g, s, args, world),
        "clocks": clk.summary(),
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 16 * s.n, "d2h_bytes_per_step": 8 * s.n},
        "gpu_launches": int(round(sum(i.launches for i in infos) / len(infos))),
        "roofline": {"bound": ROOF_BOUND.get((args.format, args.precision, args.grid), "hbm"), "achieved": achieved,
                     "peak": hbm, "unit": "GB/s", "frac": (achieved / hbm) if achieved else None,
                     "traffic": traffic,
                     "traffic_source": "ncu DRAM bytes per iteration of this kernel on this system (difference "
                                       "of 130- and 30-iteration launches) x iterations" if traffic else None,
                     "frac_dram": (traffic / (kernel_ms / 1000.0) / 1e9 / hbm) if traffic and kernel_ms > 0
                     else None,
                     "kernel": kernel_names[args.precision],
                     "algorithmic_bytes_per_iteration": per_it, "iterations": iters, "updates": updates,
                     "kernel_ms_per_step": kernel_ms, "kernel_launches_per_step": kernel_launches,
                     "peak_kind": f"{peak_kind} HBM copy bandwidth (of {peak_kind})"},
        "solve": {"iterations": iters, "updates_or_restarts": updates, "status": infos[-1].status,
                  "rel_res_true": infos[-1].rel_res_true,
                  "err_vs_fp64_oracle_sampled": err_vs_oracle(x_np, gold),
                  "oracle_iterations": gold["iterations"] if gold else None,
                  "err_vs_xstar": float(np.linalg.norm(x_np - s.xstar) / np.linalg.norm(s.xstar))},
    }
    ru_gold = golden(args.grid, "sym_ru")
    if ru_gold and args.precision == "fp32_ru":
        line["solve"]["oracle_ru_iterations"] = ru_gold["iterations"]
        line["solve"]["oracle_ru_updates"] = ru_gold["restarts"]
    if not args.no_extras and rank == 0:
        line["variants"] = extras(torch, gb, s, fmt_arrays, A, args, hbm, gold)
        A.close()
        del fmt_arrays
        line["large_128"] = large_128(torch, gb, args, hbm)
        line["paper_size"] = paper_size(torch, gb, args)
        line["batched"] = batched(torch, gb, args)
        line["differentiable"] = differentiable(torch, gb, args)
        line["ablation_2010"] = ablation(torch, gb, args, femgen.build_system(femgen.LARGE))
        line["cpu_baseline"] = cpu_baseline(s, args, gold)
    if rank == 0:
        print(json.dumps(line), flush=True)
    A.close()
    if pg:
        pg.barrier()
        pg.destroy_process_group()
    return 0


_FMA_RATE = []


def fp64_roofline(gb, st, ms, hbm):
    """The double-precision product against min(HBM, FP64 FMA rate): its FMAs
    (two per stored off-diagonal entry in symmetric storage, one per entry in
    full storage) over the device's measured FP64 FMA rate, and the bound
    that is reached first."""
    if not _FMA_RATE:
        _FMA_RATE.append(gb.measure_fp64_fma_rate())
    rate = _FMA_RATE[0]
    fmas = 2 * (st["nnz_input"] - st["n"]) + st["n"] if st["format"] == 1 else st["nnz_full"]
    t_hbm = st["spmv_bytes_fp64"] / (hbm * 1e9)
    t_fma = fmas / rate if rate > 0 else 0.0
    t = ms / 1000.0
    return {"spmv_fp64_fmas": int(fmas), "measured_fp64_fma_per_s": rate,
            "spmv_fp64_frac_of_measured_fp64_fma": t_fma / t,
            "spmv_fp64_bound": "fp64_fma" if t_fma > t_hbm else "hbm",
            "spmv_fp64_frac_of_roofline": max(t_hbm, t_fma) / t}


def time_spmv(torch, M, x, y, f32, reps=20):
    stream = torch.cuda.current_stream()
    fn = M.spmv_f32 if f32 else M.spmv
    for _ in range(3):
        fn(x, y)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def time_solve(torch, M, b, prec, args, flush=None):
    """One solve from x0 = 0 after a warm solve, the L2 flushed first: wall
    time by CUDA events on the stream, kernel time by the library's events."""
    itol = args.inner_tol if prec == "fp32_ir" else 0.0
    x = torch.zeros_like(b)
    M.solve(b, x, tol=TOL, precision=prec, inner_tol=itol, raise_on_error=False)  # warm
    x.zero_()
    if flush is not None:
        flush_l2(torch, flush)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, info = M.solve(b, x, tol=TOL, precision=prec, inner_tol=itol, raise_on_error=False)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1000.0, info, x


def extras(torch, gb, s, fmt_arrays, A_head, args, hbm, gold):
    """The comparison on the benchmarked system: SpMV bandwidth of each
    storage format, and the time to 1e-10 of plain FP64 CG, the restarted
    refinement and reliable updates, each with its error against the FP64
    oracle's solution (sampled positions of the golden file)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    b = torch.from_numpy(s.b).to(dev)
    xv = torch.from_numpy(femgen.random_vector(s.n, 7)).to(dev)
    yv = torch.empty_like(xv)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    plan = {"sym": ("fp64", "fp32_ir", "fp32_ru"), "csr": ("fp64", "fp32_ru")}
    out = {}
    for fmt in ("sym", "csr"):
        M = A_head if (A_head is not None and fmt == args.format) else gb.Matrix(fmt, *fmt_arrays[fmt])
        st = M.stats()
        r = {"nnz_stored": int(st["nnz_input"]), "device_bytes": st["device_bytes"],
             "spmv_fp64_ms": time_spmv(torch, M, xv, yv, False),
             "spmv_fp32_ms": time_spmv(torch, M, xv.float(), yv.float(), True)}
        r["spmv_fp64_GBs"] = st["spmv_bytes_fp64"] / r["spmv_fp64_ms"] / 1e6
        r["spmv_fp32_GBs"] = st["spmv_bytes_fp32"] / r["spmv_fp32_ms"] / 1e6
        r["spmv_fp64_frac_of_measured_hbm"] = r["spmv_fp64_GBs"] / hbm
        r["spmv_fp32_frac_of_measured_hbm"] = r["spmv_fp32_GBs"] / hbm
        r.update(fp64_roofline(gb, st, r["spmv_fp64_ms"], hbm))
        for prec in plan[fmt]:
            t, info, x = time_solve(torch, M, b, prec, args, flush)
            per_it = per_iteration_bytes(st, prec)
            r[prec] = {"s": t, "iterations": info.iterations, "outer": info.outer, "status": info.status,
                       "rel_res_true": info.rel_res_true, "kernel_ms": info.kernel_ms,
                       "iter_us": 1000.0 * info.kernel_ms / max(info.iterations, 1),
                       "kernel_GBs": per_it * info.iterations / (info.kernel_ms / 1000.0) / 1e9,
                       "err_vs_fp64_oracle_sampled": err_vs_oracle(x.cpu().numpy(), gold)}
        if "fp32_ir" in r:
            r["restarted_refinement_speedup_vs_fp64"] = r["fp64"]["s"] / r["fp32_ir"]["s"]
        r["reliable_update_speedup_vs_fp64"] = r["fp64"]["s"] / r["fp32_ru"]["s"]
        out[fmt] = r
        if M is not A_head:
            M.close()
    if gold:
        out["oracle_fp64_iterations"] = gold["iterations"]
    return out


def large_128(torch, gb, args, hbm):
    """The 128^3 system (2.0M rows) in all three storage formats: SpMV
    bandwidth and the three solvers, errors against the FP64 oracle."""
    dev = torch.device("cuda", torch.cuda.current_device())
    s = femgen.build_system(femgen.LARGE)
    gold = golden("128", "sym")
    arrays = {"sym": s.upper(), "csr": (s.ptr, s.idx, s.val), "csc": s.csc()}
    b = torch.from_numpy(s.b).to(dev)
    xv = torch.from_numpy(femgen.random_vector(s.n, 7)).to(dev)
    yv = torch.empty_like(xv)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"workload": "fem 128x128x128, 1 inclusion, contrast 1000, tol 1e-10", "n": s.n, "nnz": s.nnz,
           "oracle_fp64_iterations": gold["iterations"] if gold else None}
    for fmt in ("sym", "csr", "csc"):
        with gb.Matrix(fmt, *arrays[fmt]) as M:
            st = M.stats()
            r = {"spmv_fp64_ms": time_spmv(torch, M, xv, yv, False),
                 "spmv_fp32_ms": time_spmv(torch, M, xv.float(), yv.float(), True)}
            r["spmv_fp64_GBs"] = st["spmv_bytes_fp64"] / r["spmv_fp64_ms"] / 1e6
            r["spmv_fp32_GBs"] = st["spmv_bytes_fp32"] / r["spmv_fp32_ms"] / 1e6
            r["spmv_fp64_frac_of_measured_hbm"] = r["spmv_fp64_GBs"] / hbm
            r["spmv_fp32_frac_of_measured_hbm"] = r["spmv_fp32_GBs"] / hbm
            r.update(fp64_roofline(gb, st, r["spmv_fp64_ms"], hbm))
            for prec in ("fp64", "fp32_ir", "fp32_ru"):
                t, info, x = time_solve(torch, M, b, prec, args, flush)
                per_it = per_iteration_bytes(st, prec)
                r[prec] = {"s": t, "iterations": info.iterations, "outer": info.outer, "status": info.status,
                           "rel_res_true": info.rel_res_true,
                           "iter_us": 1000.0 * info.kernel_ms / max(info.iterations, 1),
                           "kernel_GBs": per_it * info.iterations / (info.kernel_ms / 1000.0) / 1e9,
                           "err_vs_fp64_oracle_sampled": err_vs_oracle(x.cpu().numpy(), gold)}
            r["reliable_update_speedup_vs_fp64"] = r["fp64"]["s"] / r["fp32_ru"]["s"]
            out[fmt] = r
    return out


def paper_size(torch, gb, args):
    """The paper's problem size (31x31x32 nodes, 25 230 rows, L2-resident):
    time to 1e-10 and microseconds per iteration, per storage and precision."""
    import oracle

    dev = torch.device("cuda", torch.cuda.current_device())
    s = femgen.build_system(femgen.PAPER_SIZE)
    arrays = {"sym": s.upper(), "csr": (s.ptr, s.idx, s.val), "csc": s.csc()}
    b = torch.from_numpy(s.b).to(dev)
    ref = oracle.cg("sym", *arrays["sym"], s.b, tol=TOL)  # the FP64 oracle's solution
    out = {"workload": "fem 31x31x32, 1 inclusion, contrast 1000", "n": s.n, "nnz": s.nnz,
           "oracle_fp64_iterations": ref.iterations}
    for fmt in ("sym", "csr"):
        with gb.Matrix(fmt, *arrays[fmt]) as M:
            out[fmt] = {"grid_ctas": M.stats()["grid_ctas"]}
            runs = [("fp64", "standard"), ("fp32_ir", "standard"), ("fp32_ru", "standard")]
            if fmt == "csr":
                runs += [("fp64", "pipelined")]
            for prec, variant in runs:
                x = torch.zeros_like(b)
                ts = []
                for k in range(4):
                    x.zero_()
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    _, info = M.solve(b, x, tol=TOL, precision=prec, variant=variant,
                                      inner_tol=args.inner_tol if prec == "fp32_ir" else 0.0)
                    e1.record()
                    torch.cuda.synchronize()
                    if k:
                        ts.append(e0.elapsed_time(e1) / 1000.0)
                t = statistics.median(ts)
                key = prec if variant == "standard" else f"{prec}_pipelined"
                xs = x.cpu().numpy()
                out[fmt][key] = {"s": t, "iterations": info.iterations, "outer": info.outer,
                                 "status": info.status, "rel_res_true": info.rel_res_true,
                                 "iter_us": 1000.0 * info.kernel_ms / max(info.iterations, 1),
                                 "err_vs_fp64_oracle": float(np.linalg.norm(xs - ref.x) / np.linalg.norm(ref.x))}
    return out


def batched(torch, gb, args):
    """256 uneven FEM systems (grid edges 12..40, contrast 10..1e4), eight
    right-hand sides each, one persistent cluster launch per solve under a
    CUDA graph: mixed precision and double precision, against plain FP64 CG
    solving one system and right-hand side at a time on the same GPU."""
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    bs = femgen.build_batch(femgen.batched_instances(256), nrhs=8)
    gen_s = time.perf_counter() - t0
    out = {"workload": "256 fem instances, edges U{12..40}, contrast log-U[10, 1e4], 8 rhs, tol 1e-10",
           "n": bs.n, "nnz": bs.nnz, "generate_s": gen_s}
    b = torch.from_numpy(bs.B).to(dev)
    sizes = np.diff(bs.row_off)
    nnz_i = np.diff(bs.ptr[bs.row_off])
    with gb.Batch(bs.row_off, bs.ptr, bs.idx, bs.val, nrhs=8, tune=False) as Bt:
        t0 = time.perf_counter()
        tune = Bt.autotune("fp32_ir")
        tune["seconds"] = time.perf_counter() - t0
        out["tuning_fp32"] = tune
        for prec, reps in (("fp32_ru", 3), ("fp32_ir", 3), ("fp64", 1)):
            x = torch.zeros_like(b)
            Bt.solve(b, x, tol=TOL, maxit=100000, precision=prec)  # warm (captures the graph)
            ts, reps_out = [], []
            for _ in range(reps):
                x.zero_()
                torch.cuda.synchronize()
                x, infos, rep = Bt.solve(b, x, tol=TOL, maxit=100000, precision=prec)
                ts.append(rep["kernel_ms"] / 1000.0)
                reps_out.append(rep)
            rep = reps_out[-1]
            _, prods, outers = Bt.instance_times()
            per_it = 8 * nnz_i + 4 * (sizes + 1) + 11 * 4 * 8 * sizes if prec != "fp64" else \
                12 * nnz_i + 4 * (sizes + 1) + 11 * 8 * 8 * sizes
            moved = float(np.sum(prods.astype(np.float64) * per_it))
            t = statistics.median(ts)
            out[prec] = {"s": t, "status": rep["status"], "products": int(rep["products"]),
                         "iterations_total": int(rep["iterations"]), "max_iterations": int(rep["max_iterations"]),
                         "max_rel_res_true": float(infos["rel_res_true"].max()),
                         "systems_ok": int(np.sum(infos["status"] == 0)), "systems": int(infos.size),
                         "threads": rep["threads"], "cluster": rep["cluster"], "clusters": rep["clusters"],
                         "groups": rep["groups"], "max_group": rep["max_group"],
                         "busy_fraction": rep["busy_fraction"], "span_ms": rep["span_ms"],
                         "graph": rep["graph"], "launches_per_solve": rep["launches"],
                         "algorithmic_GBs": moved / t / 1e9}
        out["mixed_speedup_vs_batched_fp64"] = out["fp64"]["s"] / out["fp32_ir"]["s"]
        out["reliable_update_speedup_vs_batched_fp64"] = out["fp64"]["s"] / out["fp32_ru"]["s"]
    # plain double-precision CG, one system and right-hand side at a time (all
    # 256 systems, first right-hand side; eight right-hand sides = 8x)
    seq = 0.0
    for i in range(bs.count):
        p, j, v = bs.instance(i)
        with gb.Matrix("csr", p, j, v) as M:
            bi = torch.from_numpy(np.ascontiguousarray(bs.B[bs.row_off[i]:bs.row_off[i + 1], 0])).to(dev)
            xi = torch.zeros_like(bi)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            M.solve(bi, xi, tol=TOL, maxit=100000, precision="fp64")
            e1.record()
            torch.cuda.synchronize()
            seq += e0.elapsed_time(e1) / 1000.0
    out["sequential_fp64_one_rhs_s"] = seq
    out["sequential_fp64_8rhs_s"] = 8 * seq
    out["batched_speedup_vs_sequential_fp64"] = 8 * seq / min(out["fp32_ir"]["s"], out["fp32_ru"]["s"])
    return out


def differentiable(torch, gb, args):
    """64^3 system, L = ||x - x_t||^2 (x_t ~ U(-1, 1) seeded), symmetric
    storage: forward double-precision CG to 1e-10, backward = adjoint CG to
    1e-10 + sampled-outer-product and element-gradient kernels.  Gradient
    error: fourth-order central differences of fixed-iteration solves along
    the configured 32 random directions (11 in b and 11 in the stored values:
    relative white noise, step 1e-6; 10 in the coefficients: random smooth
    fields, step 1e-5), and the 6^3 dense reference."""
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    g = femgen.DIFF
    s = femgen.build_system(g)
    el = femgen.elements(g)
    up, ui, uv = s.upper()
    pos, w = femgen.element_map(el, up, ui, storage="sym")
    tptr, te, tw = femgen.assembly_map(pos, w, len(ui))
    prep_s = time.perf_counter() - t0
    asm = gb.Assembly(pos, w, tptr, te, tw)
    xt = torch.from_numpy(femgen.random_vector(s.n, 79)).to(dev)
    coef0 = torch.from_numpy(el.coef).to(dev)
    vals0 = asm(coef0)
    S = gb.SparseSolve("sym", up, ui, vals0.cpu().numpy(), tol=TOL)
    b0 = torch.from_numpy(s.b).to(dev)
    fw, bw = [], []
    for k in range(4):
        coef = coef0.clone().requires_grad_(True)
        b = b0.clone().requires_grad_(True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize()
        e[0].record()
        x = S(asm(coef), b)
        L = ((x - xt) ** 2).sum()
        e[1].record()
        L.backward()
        e[2].record()
        torch.cuda.synchronize()
        if k:
            fw.append(e[0].elapsed_time(e[1]) / 1000.0)
            bw.append(e[1].elapsed_time(e[2]) / 1000.0)
    out = {"workload": "fem 64^3, 1 inclusion, contrast 1000, symmetric storage, L = ||x - x_t||^2, tol 1e-10",
           "n": s.n, "nnz_stored": int(len(ui)), "elements": el.count, "prepare_s": prep_s,
           "forward_s": statistics.median(fw), "backward_s": statistics.median(bw),
           "forward_iterations": S.last_info.iterations, "adjoint_iterations": S.last_adjoint_info.iterations}
    gb_, gc = b.grad.clone(), coef.grad.clone()
    # finite differences through fixed-iteration solves (a smooth map)
    with gb.Matrix("sym", up, ui, uv) as A:
        _, info = A.solve(b0, tol=1e-13, maxit=100000)
    F = gb.SparseSolve("sym", up, ui, uv, fixed_iterations=info.iterations + 50)
    coef = coef0.clone().requires_grad_(True)
    vals = asm(coef)
    vals.retain_grad()
    b = b0.clone().requires_grad_(True)
    ((F(vals, b) - xt) ** 2).sum().backward()
    gb_, gv, gc = b.grad, vals.grad, coef.grad
    v0 = vals.detach()
    h = 1e-6

    def diff(vp, bp, vm, bm):
        with torch.no_grad():
            xp, xm = F(vp, bp), F(vm, bm)
        return float(((xp - xm) * (xp + xm - 2.0 * xt)).sum())

    def derivative(point, hh=h):
        return (8.0 * diff(*point(hh), *point(-hh)) - diff(*point(2 * hh), *point(-2 * hh))) / (12.0 * hh)

    gen = torch.Generator(device=dev).manual_seed(5)
    errs = {}
    for t in range(32):
        if t < 11:
            d = torch.randn(b0.shape, generator=gen, device=dev, dtype=torch.float64) * b0.abs()
            fd, an, fam = derivative(lambda e: (v0, b0 + e * d)), float(gb_ @ d), "b"
        elif t < 22:
            d = torch.randn(v0.shape, generator=gen, device=dev, dtype=torch.float64) * v0.abs()
            fd, an, fam = derivative(lambda e: (v0 + e * d, b0)), float(gv @ d), "values"
        else:
            ci = torch.arange(el.count, device=dev) // 6
            p = torch.stack([((ci % (g.nx - 1)).double() + 0.5) / (g.nx - 1),
                             (((ci // (g.nx - 1)) % (g.ny - 1)).double() + 0.5) / (g.ny - 1),
                             ((ci // ((g.nx - 1) * (g.ny - 1))).double() + 0.5) / (g.nz - 1)], dim=1)
            f = torch.zeros(el.count, dtype=torch.float64, device=dev)
            for _ in range(3):
                kv = torch.randint(0, 3, (3,), generator=gen, device=dev).double()
                a = torch.randn((), generator=gen, device=dev, dtype=torch.float64)
                ph = 6.283185307179586 * torch.rand((), generator=gen, device=dev, dtype=torch.float64)
                f += a * torch.cos(6.283185307179586 * (p @ kv) + ph)
            d = f * coef0
            with torch.no_grad():
                fd = derivative(lambda e: (asm(coef0 + e * d), b0), 1e-5)  # step 1e-5: see the tests
            an, fam = float(gc @ d), "coefficients"
        errs.setdefault(fam, []).append(abs(fd - an) / abs(fd))
    out["fd_max_rel_error"] = {k: max(v) for k, v in errs.items()}
    out["fd_directions"] = {k: len(v) for k, v in errs.items()}
    S.close()
    F.close()
    # 6^3 dense reference gradient
    g6 = femgen.Grid(6, 6, 6, contrast=50.0, seed_mesh=7, seed_x=8)
    s6 = femgen.build_system(g6)
    el6 = femgen.elements(g6)
    xt6 = femgen.random_vector(s6.n, 77)
    A6 = np.zeros((s6.n, s6.n))
    for i in range(s6.n):
        A6[i, s6.idx[s6.ptr[i]:s6.ptr[i + 1]]] = s6.val[s6.ptr[i]:s6.ptr[i + 1]]
    x6 = np.linalg.solve(A6, s6.b)
    lam6 = np.linalg.solve(A6, 2.0 * (x6 - xt6))
    u6 = s6.upper()
    p6, w6 = femgen.element_map(el6, u6[0], u6[1], storage="sym")
    t6 = femgen.assembly_map(p6, w6, len(u6[1]))
    asm6 = gb.Assembly(p6, w6, *t6)
    c6 = torch.from_numpy(el6.coef).to(dev).requires_grad_(True)
    S6 = gb.SparseSolve("sym", u6[0], u6[1], u6[2], tol=1e-13)
    b6 = torch.from_numpy(s6.b).to(dev).requires_grad_(True)
    ((S6(asm6(c6), b6) - torch.from_numpy(xt6).to(dev)) ** 2).sum().backward()
    S6.close()
    out["dense_6cube_rel_error_grad_b"] = float(np.linalg.norm(b6.grad.cpu().numpy() - lam6) / np.linalg.norm(lam6))
    return out


def ablation(torch, gb, args, big):
    """The paper's 2010 solver structure on this GPU (thread-per-row CSR
    product, SCSR + SCSC with atomics, host-driven CG with a host round trip
    per dot product) against the library, at the paper's size and at 128^3."""
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}
    for name, s in (("paper_size", femgen.build_system(femgen.PAPER_SIZE)), ("128", big)):
        arrays = {"csr": (s.ptr, s.idx, s.val), "sym": s.upper()}
        xv = torch.from_numpy(femgen.random_vector(s.n, 7)).to(dev)
        yv = torch.empty_like(xv)
        b = torch.from_numpy(s.b).to(dev)
        r = {}
        for fmt in ("csr", "sym"):
            Ab = gb.Ablation(fmt, *arrays[fmt])
            ms_ab = time_spmv(torch, Ab, xv, yv, False)
            # the 2010 kernels read int32 indices: 12 bytes per stored entry
            nnz_st = int(arrays[fmt][1].shape[0])
            bytes_2010 = 12 * nnz_st + 4 * (s.n + 1) + 16 * s.n
            with gb.Matrix(fmt, *arrays[fmt]) as M:
                ms_lib = time_spmv(torch, M, xv, yv, False)
                bytes_ = M.stats()["spmv_bytes_fp64"]
                if fmt == "csr":
                    x = torch.zeros_like(b)
                    M.solve(b, x, tol=TOL)
                    x.zero_()
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    _, info = M.solve(b, x, tol=TOL)
                    lib_s = time.perf_counter() - t0
            r[fmt] = {"spmv_2010_kernel": {"csr": "thread-per-row CSR, one launch",
                                           "sym": "SCSR direct half, then SCSC transpose half with FP64 "
                                                  "atomic adds: two launches, as in the paper"}[fmt],
                      "spmv_2010_ms": ms_ab, "spmv_2010_GBs": bytes_2010 / ms_ab / 1e6,
                      "spmv_library_ms": ms_lib, "spmv_library_GBs": bytes_ / ms_lib / 1e6,
                      "spmv_speedup": ms_ab / ms_lib}
            if fmt == "csr":
                x = torch.zeros_like(b)
                Ab.solve(b, x, tol=TOL)
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, iab = Ab.solve(b, x, tol=TOL)
                ab_s = time.perf_counter() - t0
                r["cg_fp64"] = {"s_2010": ab_s, "iterations_2010": iab.iterations, "launches_2010": iab.launches,
                                "s_library": lib_s, "iterations_library": info.iterations,
                                "launches_library": info.launches, "speedup": ab_s / lib_s}
        out[name] = r
    return out


def cpu_baseline(s, args, gold):
    """The oracle as it stands on the host cores: its single-threaded build
    and its multi-threaded build (same bits) on every core, each on a bounded
    run of CG iterations of the benchmarked system (double precision,
    symmetric storage: the oracle's own method), scaled by the oracle's own
    iteration count to 1e-10; and one complete 1e-10 solve of the 128^3
    system on every core."""
    import oracle

    up = s.upper()
    cores = os.cpu_count() or 1
    lib1 = oracle.load()
    libn = oracle.load_threaded(cores)
    iters = gold["iterations"] if gold else None
    spn, mn, setn = oracle_iteration_seconds("sym", up, s.b, libn, args.cpu_seconds)
    sp1, m1, set1 = oracle_iteration_seconds("sym", up, s.b, lib1, args.cpu_seconds)
    out = {"value": spn * iters + setn if iters else None, "unit": "s", "cores": oracle.threads(libn),
           "kind": "oracle",
           "sample": f"{mn} CG iterations of the double-precision oracle (symmetric storage) on the benchmarked "
                     f"system with its multi-threaded build on {oracle.threads(libn)} threads ({spn * 1000:.1f} ms "
                     f"each) and {m1} with its single-threaded build ({sp1 * 1000:.1f} ms each), scaled by the "
                     f"oracle's own {iters} iterations to 1e-10 (tests/golden) plus one set-up",
           "seconds_per_iteration": spn, "single_thread": {"value": sp1 * iters + set1 if iters else None,
                                                            "seconds_per_iteration": sp1, "cores": 1},
           "host_cores": cores}
    if not args.no_cpu_full_solve:
        s128 = femgen.build_system(femgen.LARGE)
        u128 = s128.upper()
        t0 = time.perf_counter()
        r = oracle.cg("sym", *u128, s128.b, tol=TOL, lib=libn)
        g128 = golden("128", "sym")
        out["full_solve_128"] = {"s": time.perf_counter() - t0, "iterations": r.iterations, "status": r.status,
                                 "rel_res_true": r.rel_res_true, "threads": oracle.threads(libn),
                                 "same_as_golden": (g128 is not None and r.iterations == g128["iterations"])}
    return out


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return spawn_ranks(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
