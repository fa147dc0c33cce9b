#!/usr/bin/env python
"""Benchmark: seconds to solve the n = 1,048,576 sparse least-squares problem to a true
normal-equations relative residual of 1e-8 with two-level Schwarz PCG on one GB300.

Workload (synthetic, seed 0): 1024 x 1024 grid of unknowns, m = 4n random rows with 8
nonzeros inside Chebyshev radius 3 of a random centre (N(0,1) values) plus 1e-2 I rows;
256 subdomains of 64 x 64 columns, overlap 1, at most 32 coarse vectors each (tau
automatic).  A step is one complete ls_solve (x_0 = 0 to ||A^T(b - Ax)|| <= 1e-8 ||A^T b||);
setup is timed separately.  The headline form is the mixed one (FP32 local factors
inside an FP64 flexible CG); the plain FP64 form and GMRES with RAS + the deflated
second level run on the same problem beside it (`--forms`).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU: replicas only (every rank solves its own copy; max time over ranks).
"""
from __future__ import annotations

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

METRIC = "n=1M LS solve s to 1e-8 normal-eq rel resid, mixed vs FP64 form; apply HBM GB/s"
# DRAM bytes (read + write) of one k_local_solve launch, measured by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, one launch, one pass) on the workload,
# form and local-solve configuration named in the key; valid while that kernel and
# workload stay as they are (the capture's command and figures are kept with the profile summaries).
LOCAL_SOLVE_TRAFFIC = {("grid1024-r3k8-N256", "f32", 1): 5.81e9 + 8.75e6}
TRAFFIC_SOURCE = ("constant in bench.py from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of "
                  "this kernel, workload, form and configuration (kept with the profile summaries of k_local_solve)")
FALLBACK_HBM_GBS = 6800.0


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f32", choices=["f32", "f64", "bf16"], help="headline form")
    ap.add_argument("--forms", default="f32,f64,f32dg",
                    help="forms to run (comma list of f32, f64, bf16; suffixes: 'b' the balanced second level, "
                         "'d' RAS with the deflated second level, 'l' the LSQR outer solver, 'g' GMRES(100); "
                         "e.g. f32b, f32bl, f32dg)")
    ap.add_argument("--side", type=int, default=1024)
    ap.add_argument("--block", type=int, default=64)
    ap.add_argument("--nev", type=int, default=32)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--sample-side", type=int, default=256, help="grid side of the CPU-oracle sample")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--mode", default="solve",
                    choices=["solve", "nsweep", "precision", "batch", "tausweep", "diff"],
                    help="solve: the timed benchmark line; nsweep: iterations/setup vs subdomain count "
                         "(blocks 128/64/32); precision: errors of every form on the column-scaled workload; "
                         "batch: 64 independent problems x 32 right-hand sides in shared launches; "
                         "tausweep: iterations and n0 against the threshold tau; "
                         "diff: forward + adjoint solves on the n = 262,144 differentiation workload")
    ap.add_argument("--zero-sum", action="store_true",
                    help="nsweep/tausweep on the zero-sum variant of the grid workload (random rows centred to "
                         "sum to zero: a Laplacian-like near null space that one-level Schwarz cannot handle)")
    ap.add_argument("--spmv", type=int, default=0,
                    help="solve mode: force one sparse-product kernel code for A and A^T (0: autotuned)")
    ap.add_argument("--normal-product", type=int, default=0,
                    help="solve mode: form of A^T (A p): 0 timed choice at setup, 1 two products, 2 row tiles")
    ap.add_argument("--normal-kernel", type=int, default=0,
                    help="solve mode: row-tile kernel configuration (0 timed choice, 1-3: 512 threads with that many "
                         "slices per warp, 4: 1,024 threads)")
    ap.add_argument("--local-config", type=int, default=0,
                    help="solve mode: local-solve configuration (0 timed choice at setup, 1 256 threads / 16 KB "
                         "stages, 2 512 threads / 32 KB stages)")
    ap.add_argument("--no-graph", action="store_true",
                    help="solve mode: run the iterations from the host, kernel by kernel (the same kernels; for "
                         "profilers that do not list the kernels inside a conditional graph node)")
    ap.add_argument("--block-kernel", type=int, default=0,
                    help="batch mode: local-solve kernel of the FP32 block path (0 timed choice, 1 TF32 mma.sync, "
                         "2 tcgen05)")
    ap.add_argument("--nprob", type=int, default=64)
    ap.add_argument("--nrhs", type=int, default=32)
    return ap.parse_args()


def replica_env() -> tuple:
    """(world, rank, local rank) from torchrun's environment; (1, 0, 0) when run alone."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Largest value over the replicas (the slowest replica sets the step time).  Works
    on any initialised process group (NCCL with a device tensor, gloo on the CPU)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured copy, burst)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [l.strip().split(",") for l in open(self.f.name) if l.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() in ("active", "1"):
                        reasons.add(nm)
            except Exception:
                continue
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def local_solve_bytes(st: dict, form: str, restrict: bool = True) -> int:
    """Algorithmic bytes of one local-solve launch: the stored factor tiles (off-diagonal
    panels and inverse diagonal tiles) read by the forward and the backward sweep, the
    gather of r and the write of y (index, r value, scale, y per local entry), and the
    fused coarse restriction (Zbar once) when the launch carries it (the additive
    operator; the balanced and deflated operators restrict in a kernel of their own)."""
    es = {"f64": 8, "f32": 4, "bf16": 2}[form]
    fac = 2 * st["fac_elems"] * es
    if form == "bf16":
        fac += 2 * (st["fac_elems"] // 1024) * 4
    gather = st["total_local"] * (4 + 8 + 8 + 8)
    coarse = st["zbar_elems"] * 8 if restrict else 0
    return fac + gather + coarse


def spmv_bytes(m: int, n: int, nnz: int) -> int:
    """Algorithmic bytes of q = A p then w = A^T q with the fused p.w: both index/value
    streams, both pointer arrays, the vectors read once and the results written once."""
    csr = nnz * 12 + (m + 1) * 8 + n * 8 + m * 8
    csc = nnz * 12 + (n + 1) * 8 + m * 8 + n * 8 + n * 8
    return csr + csc


def tile_bytes(n: int, t: dict) -> int:
    """Algorithmic bytes of the row-tile normal product (with the fused p.w): every stored
    entry of both tile copies once (8-byte value, 2-byte index), the slice offsets and
    column ids, the partial windows written and read back, p read once for the windows
    and once for the dot, w written, and the per-tile and per-column-block tables."""
    ent = (t["row_entries"] + t["col_entries"]) * 10
    meta = (t["row_slices"] + t["col_slices"] + 2) * 8 + t["col_slices"] * 32 * 2 + t["tiles"] * 36 + (n // 256 + 1) * 8
    return ent + meta + t["window_sum"] * 16 + n * 24


def host_cores() -> dict:
    """Host cores this process may run on (its affinity set) and the machine's total."""
    try:
        avail = len(os.sched_getaffinity(0))
    except Exception:
        avail = os.cpu_count() or 1
    return {"threads": avail, "cpu_count": os.cpu_count() or avail}


def cpu_oracle_sample(side: int, block: int, nev: int, rtol: float, reps: int = 1) -> dict:
    """Runs the FP64 oracle (banded mode) on a side x side sample of the same workload in a
    subprocess whose BLAS/OpenMP threads are all the host cores this process may use:
    setup once, then `reps` timed solves."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import oracle as O
from workloads import config_scale
P = config_scale(side={side}, block={block})
A = O.schwarz.as_csr(P.m, P.n, P.row_ptr, P.col, P.val)
t = time.time()
M = O.build_two_level(A, P.part, P.nparts, tau=0.0, nev_max={nev}, mode="banded")
ts = time.time() - t
times, iters = [], 0
for _ in range({reps}):
    t = time.time()
    x, info = O.pcg(A, P.b, M.apply, rtol={rtol})
    times.append(time.time() - t)
    iters = info["iters"]
print(json.dumps(dict(n=P.n, m=P.m, nnz=P.nnz, N=P.nparts, setup_s=ts, solve_s=times, iters=iters, n0=M.n0)))
"""
    cores = host_cores()
    nt = str(cores["threads"])
    env = dict(os.environ, OMP_NUM_THREADS=nt, OPENBLAS_NUM_THREADS=nt, MKL_NUM_THREADS=nt,
               CUDA_VISIBLE_DEVICES="")
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if p.returncode != 0:
        raise RuntimeError("oracle sample failed:\n" + p.stderr[-2000:])
    d = json.loads(p.stdout.strip().splitlines()[-1])
    d.update(cores)
    return d


def sample_workload(side: int, block: int, nev: int, d: dict) -> str:
    """Name of the oracle's sample: the benchmark generator on a side x side grid."""
    return (f"grid{side}-r3k8-N{d['N']}: n={d['n']}, m={d['m']}, nnz={d['nnz']}, {d['N']} subdomains "
            f"{block}x{block} (the benchmark's subdomain geometry), nev_max {nev}, tau auto")


def cpu_baseline_entry(args, d: dict, n_full: int, times: list) -> dict:
    """The oracle's solve seconds on the sample, and their extrapolation to the full
    workload by the ratio of unknowns (every step of a solve costs in proportion to n at
    fixed subdomain geometry, and the iteration counts agree: 17 on both)."""
    scale = n_full / d["n"]
    meas = statistics.mean(times)
    return {"value": meas * scale, "unit": "s", "cores": d["threads"], "kind": "oracle",
            "sample_value": meas, "sample_unit": "s per solve of the sample", "scale_by_n": scale,
            "host": {"threads_used": d["threads"], "cpu_count": d["cpu_count"]},
            "sample": (f"oracle (FP64 numpy/scipy, banded LAPACK factors, ARPACK eigensolves, BLAS threads = "
                       f"{d['threads']} of {d['cpu_count']} host cores) on {sample_workload(args.sample_side, args.block, args.nev, d)}; "
                       f"{d['iters']} PCG iterations to {args.rtol:g}, {meas:.3f} s per solve measured "
                       f"(mean of {len(times)}); value = that x {scale:.0f} (n ratio); oracle setup "
                       f"{d['setup_s']:.1f} s not included")}


def solve_config(args, world: int) -> dict:
    """The benchmark workload, identical in both arms: the grid generator with 4 random rows
    of 8 entries per grid point plus one 1e-2 identity row per column, so m = 5 n and
    nnz = 33 n."""
    n = args.side * args.side
    N = (-(-args.side // args.block)) ** 2  # square blocks, the last row and column ragged
    return {"workload": f"grid{args.side}-r3k8-N{N}: n={n}, m={5 * n}, nnz={33 * n}, "
                        f"{N} subdomains {args.block}x{args.block}, overlap 1, nev_max {args.nev}, tau auto",
            "rtol": args.rtol, "l2": "inputs larger than L2 (factors alone exceed 129 MB)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """The reference arm: the paper ships no code, so the oracle is the reference.  Rank 0
    times it on the host cores on a bounded sample of the workload (the sample grid, same
    subdomain geometry), every step one solve of the sample; the value is extrapolated to
    the full workload by the n ratio and the measured sample seconds are kept beside it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_full = args.side * args.side
    d = cpu_oracle_sample(args.sample_side, args.block, args.nev, args.rtol, reps=args.warmup + args.steps)
    times = d["solve_s"][args.warmup:]
    cb = cpu_baseline_entry(args, d, n_full, times)
    val = cb["value"]
    config = solve_config(args, args.gpus)
    config["sample"] = (sample_workload(args.sample_side, args.block, args.nev, d) + f"; each step one solve of it, "
                        f"value scaled by the n ratio {cb['scale_by_n']:.0f}")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1000, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config,
            "form": f"oracle: plain FP64 PCG with the two-level preconditioner (CPU, {d['threads']} threads)",
            "sample_value": cb["sample_value"], "sample_ms_per_step": cb["sample_value"] * 1000,
            "cpu_baseline": cb,
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = replica_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2107_09006_gb300 import Solver, ls_solve
    from workloads import config_scale

    t = time.time()
    P = config_scale(side=args.side, block=args.block)
    log(f"[bench] workload generated in {time.time() - t:.1f}s: m={P.m} n={P.n} nnz={P.nnz} N={P.nparts}")
    if (P.m, P.nnz, P.nparts) != (5 * P.n, 33 * P.n, (-(-args.side // args.block)) ** 2):
        raise RuntimeError("workload sizes differ from the ones the config line states")
    stream = torch.cuda.current_stream(dev)
    hbm_peak, peak_src = peaks()
    forms = [f for f in args.forms.split(",") if f]
    if args.prec not in forms:
        forms.insert(0, args.prec)
    b_dev = torch.as_tensor(P.b, device=dev)
    x_dev = torch.empty(P.n, dtype=torch.float64, device=dev)
    results, clocks, e2e, launches = {}, None, None, 0

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()

    for spec in forms:
        form = spec.rstrip("bdlg")
        suf = spec[len(form):]
        variant = 1 if "b" in suf else 2 if "d" in suf else 0
        solver = 1 if "l" in suf else 2 if "g" in suf else 0
        def make(timed):
            return Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, device=dev, stream=stream,
                          nev_max=args.nev, factor_prec=form, time_kernels=1 if timed else 0, maxit=2000,
                          variant=variant, solver=solver, spmv=args.spmv, use_graph=0 if args.no_graph else 1,
                          normal_product=args.normal_product, normal_kernel=args.normal_kernel,
                          local_config=args.local_config)

        # The timed solves run on a handle without kernel timing (no global-timer stamp
        # kernels in the loop graph); a second handle with kernel timing then gives the
        # per-kernel figures.
        t = time.time()
        S = make(False)
        torch.cuda.synchronize(dev)
        setup_s = time.time() - t
        sinfo = S.info()
        st = S.storage()
        log(f"[bench] {spec}: setup {setup_s:.2f}s (eig {sinfo['t_eig']:.2f}s) n0={sinfo['n0']} "
            f"k in [{sinfo['kmin']},{sinfo['kmax']}] steps<= {sinfo['eig_steps_max']} fac={st['fac_elems']}")
        for _ in range(args.warmup):
            ls_solve(S.h, b_dev, 1, args.rtol, x_dev)
        headline = spec == args.prec
        ck = None
        if headline:
            ck = Clocks(dev.index or 0)
            ck.start()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos = [ls_solve(S.h, b_dev, 1, args.rtol, x_dev) for _ in range(args.steps)]
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1) / args.steps
        if headline:
            clocks = ck.stop()
        ms = max_over_ranks(ms, world, dev)
        timed_choice = {"local_config": infos[-1]["local_config"], "normal_product": infos[-1]["normal_product"],
                        "normal_kernel": S.normal_tiles()["kernel"]}
        if headline:
            launches = sum(i["launches"] for i in infos)
            # end to end through the public call with pinned host buffers
            bh = torch.as_tensor(P.b).pin_memory()
            xh = torch.empty(P.n, dtype=torch.float64).pin_memory()
            ls_solve(S.h, bh, 1, args.rtol, xh)
            barrier()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(args.steps):
                ls_solve(S.h, bh, 1, args.rtol, xh)
            f1.record(stream)
            barrier()
            e2e_ms = f0.elapsed_time(f1) / args.steps
            xerr = float(np.linalg.norm(xh.numpy() - x_dev.cpu().numpy()) / np.linalg.norm(x_dev.cpu().numpy()))
            e2e = {"value": e2e_ms / 1000.0, "unit": "s", "h2d_bytes_per_step": P.m * 8, "d2h_bytes_per_step": P.n * 8,
                   "x_vs_device_run": xerr}
        S.close()
        del S
        torch.cuda.empty_cache()

        St = make(True)
        ls_solve(St.h, b_dev, 1, args.rtol, x_dev)
        tinfos = [ls_solve(St.h, b_dev, 1, args.rtol, x_dev) for _ in range(max(2, args.steps))]
        nl = sum(i["local_launches"] for i in tinfos)
        ms_local = sum(i["ms_local"] for i in tinfos) / max(nl, 1)
        its = sum(i["iters"] for i in tinfos)
        ms_spmv = sum(i["ms_spmv"] for i in tinfos) / max(its, 1)
        lb = local_solve_bytes(st, form, restrict=variant == 0)
        tiles = St.normal_tiles()
        sb = tile_bytes(P.n, tiles) if tinfos[-1]["normal_product"] == 2 else spmv_bytes(P.m, P.n, P.nnz)
        loc_gbs = lb / (ms_local * 1e-3) / 1e9
        spmv_gbs = sb / (ms_spmv * 1e-3) / 1e9
        ms_iter = sum(i["ms_iter"] for i in tinfos) / max(its, 1)
        results[spec] = {
            "value": ms / 1000.0, "iterations": infos[-1]["iters"], "relres_true": infos[-1]["relres_true"],
            "ms_per_iteration_kernels": ms_iter, "lanes": [tinfos[-1]["lanes_csr"], tinfos[-1]["lanes_csc"]],
            "setup_s": setup_s, "eig_s": sinfo["t_eig"], "n0": sinfo["n0"], "kappa_lanczos": infos[-1]["kappa_lanczos"],
            "choices_of_timed_handle": timed_choice,
            "local_solve": {"config": tinfos[-1]["local_config"], "ms_per_launch": ms_local, "bytes_per_launch": lb,
                            "GBps": loc_gbs, "frac": loc_gbs / hbm_peak,
                            "share_of_step": nl * ms_local / (ms * len(tinfos))},
            "normal_product": {"form": "row tiles" if tinfos[-1]["normal_product"] == 2 else "two products",
                               "tiles": tiles["tiles"], "kernel": tiles["kernel"], "setup_ms": tiles["setup_ms"],
                               "ms_per_iter": ms_spmv, "bytes_per_iter": sb, "GBps": spmv_gbs,
                               "frac": spmv_gbs / hbm_peak, "bytes_two_products": spmv_bytes(P.m, P.n, P.nnz)},
        }
        St.close()
        del St
        torch.cuda.empty_cache()

    head = results[args.prec]
    line = {
        "metric": METRIC, "value": head["value"], "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["value"] * 1000, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"f32": "f32", "f64": "f64", "bf16": "bf16"}[args.prec], "data": "synthetic",
        "config": solve_config(args, world),
        "form": {"f32": "mixed: FP32 local factors, FP64 flexible CG", "f64": "plain FP64",
                 "bf16": "mixed: BF16 local factors"}[args.prec],
        "roofline": {"bound": "hbm", "achieved": head["local_solve"]["GBps"], "peak": hbm_peak, "unit": "GB/s",
                     "frac": head["local_solve"]["frac"],
                     "traffic": LOCAL_SOLVE_TRAFFIC.get((P.name, args.prec, head["local_solve"]["config"])),
                     "traffic_source": TRAFFIC_SOURCE if (P.name, args.prec, head["local_solve"]["config"]) in
                     LOCAL_SOLVE_TRAFFIC else None,
                     "kernel": "k_local_solve (batched envelope trisolves, one CTA per subdomain)",
                     "bytes_per_launch": head["local_solve"]["bytes_per_launch"],
                     "ms_per_launch": head["local_solve"]["ms_per_launch"], "peak_source": peak_src},
        "gpu_launches": launches, "clocks": clocks, "e2e": e2e,
        "iterations": head["iterations"], "setup_s": head["setup_s"], "forms": results,
    }
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            d = cpu_oracle_sample(args.sample_side, args.block, args.nev, args.rtol)
            line["cpu_baseline"] = cpu_baseline_entry(args, d, P.n, d["solve_s"])
        except Exception as ex:  # reported, not fatal
            line["cpu_baseline"] = {"value": None, "unit": "s", "cores": host_cores()["threads"], "kind": "oracle",
                                    "sample": str(ex)[:300]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _device_setup():
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    return torch, dev


def run_nsweep(args):
    """Subdomain-count sweep on the n = 1M grid: for blocks of 128, 64 and 32 columns a
    side (N = 64, 256, 1024) the setup split (index sets + factors, eigensolve + coarse),
    n0, iterations to rtol and the solve time of the two-level additive form, plus the
    iterations of the one-level method, of the balanced form and of GMRES with RAS and
    the deflated second level; one JSON line per N and a summary."""
    torch, dev = _device_setup()
    from paper_2107_09006_gb300 import Solver, ls_solve
    from workloads import config_scale
    rows = []

    def iters_of(P, b, x, stream, **kw):
        S = Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, device=dev, stream=stream,
                   factor_prec=args.prec, maxit=5000, **kw)
        info = ls_solve(S.h, b, 1, args.rtol, x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = ls_solve(S.h, b, 1, args.rtol, x)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        S.close()
        torch.cuda.empty_cache()
        return info["iters"], info["kappa_lanczos"], e0.elapsed_time(e1) / 1000.0

    for block in (128, 64, 32):
        P = config_scale(side=args.side, block=block, zero_sum=args.zero_sum)
        b = torch.as_tensor(P.b, device=dev)
        x = torch.empty(P.n, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)
        t = time.time()
        S = Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, device=dev, stream=stream,
                   nev_max=args.nev, factor_prec=args.prec, time_kernels=1, maxit=5000)
        torch.cuda.synchronize(dev)
        setup = time.time() - t
        si = S.info()
        for _ in range(max(args.warmup, 1)):
            ls_solve(S.h, b, 1, args.rtol, x)
        ts, infos = [], []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            infos.append(ls_solve(S.h, b, 1, args.rtol, x))
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(e0.elapsed_time(e1) / 1000.0)
        it = infos[-1]
        row = {"N": P.nparts, "block": block, "n0": si["n0"], "kmin": si["kmin"], "kmax": si["kmax"],
               "tau_used": si["tau_used"], "setup_s": setup, "eig_coarse_s": si["t_eig"],
               "iterations": it["iters"], "relres_true": it["relres_true"], "kappa_lanczos": it["kappa_lanczos"],
               "solve_s": statistics.median(ts), "ms_local": it["ms_local"] / max(it["local_launches"], 1),
               "ms_coarse_per_iter": it["ms_coarse"] / max(it["iters"], 1),
               "ms_spmv_per_iter": it["ms_spmv"] / max(it["iters"], 1), "fac_elems": S.storage()["fac_elems"]}
        S.close()
        del S
        torch.cuda.empty_cache()
        i1, k1, s1 = iters_of(P, b, x, stream, coarse=0, nev_max=0)
        ib, kb, sb = iters_of(P, b, x, stream, nev_max=args.nev, variant=1)
        idg, _, sdg = iters_of(P, b, x, stream, nev_max=args.nev, variant=2, solver=2)
        row.update({"one_level": {"iterations": i1, "kappa_lanczos": k1, "solve_s": s1},
                    "balanced": {"iterations": ib, "kappa_lanczos": kb, "solve_s": sb},
                    "deflated_ras_gmres": {"iterations": idg, "solve_s": sdg}})
        log(f"[nsweep] {json.dumps(row)}")
        rows.append(row)
    its = [r["iterations"] for r in rows]
    print(json.dumps({"report": "nsweep", "workload": f"grid{args.side}-r3k8" + ("-zerosum" if args.zero_sum else "") +
                      f", nev_max {args.nev}, tau auto, form {args.prec}, rtol {args.rtol:g}", "rows": rows,
                      "iterations_max_over_min": max(its) / min(its)}), flush=True)


def run_precision(args):
    """Column-scaled n = 1M workload (columns scaled by 10**U(-3, 3)): the FP64 form run
    to rtol 1e-13 with column equilibration is the reference solution; every factor
    precision, with the paper's construction as written and with equilibration, is
    solved to 1e-8 and 1e-10 and its relative error against the reference reported."""
    torch, dev = _device_setup()
    import numpy as np
    from paper_2107_09006_gb300 import Solver, ls_solve
    from workloads import config_precision
    P = config_precision(side=args.side, block=args.block)
    b = torch.as_tensor(P.b, device=dev)
    stream = torch.cuda.current_stream(dev)

    def make(prec, eq, maxit):
        t = time.time()
        S = Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, device=dev, stream=stream,
                   nev_max=args.nev, factor_prec=prec, maxit=maxit, equilibrate=eq)
        torch.cuda.synchronize(dev)
        return S, time.time() - t

    def solve(S, rtol):
        x = torch.empty(P.n, dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = ls_solve(S.h, b, 1, rtol, x, raise_on_fail=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return x, info, e0.elapsed_time(e1) / 1000.0

    S, _ = make("f64", 1, 2000)
    xref, iref, _ = solve(S, 1e-13)
    S.close()
    nref = float(torch.linalg.norm(xref))
    rows = []
    for eq in (1, 0):
        for prec in ("f64", "f32", "bf16"):
            S, setup = make(prec, eq, 500 if eq else 4000)
            n0 = S.info()["n0"]
            for rtol in (1e-8, 1e-10):
                x, info, sec = solve(S, rtol)
                err = float(torch.linalg.norm(x - xref)) / nref
                row = {"form": prec, "construction": "equilibrated" if eq else "paper", "rtol": rtol,
                       "iterations": info["iters"], "restarts": info["restarts"], "status": info["status"],
                       "relres_true": info["relres_true"], "rel_error_vs_fp64_1e-13": err, "solve_s": sec,
                       "setup_s": setup, "n0": n0}
                log(f"[precision] {json.dumps(row)}")
                rows.append(row)
            S.close()
            del S
            torch.cuda.empty_cache()
    print(json.dumps({"report": "precision", "workload": f"grid{args.side}-r3k8-N{P.nparts} columns scaled by "
                      f"10**U(-3,3), nev_max {args.nev}, tau auto",
                      "reference": {"form": "f64", "construction": "equilibrated", "rtol": 1e-13,
                                    "iterations": iref["iters"], "relres_true": iref["relres_true"]},
                      "rows": rows}), flush=True)


def run_tausweep(args):
    """Threshold sweep on the n = 1M grid (256 subdomains, FP32 factors, at most 64
    vectors per subdomain): the one-level method, then for each tau the coarse dimension
    n0 and the iterations and solve time of the additive and balanced two-level forms
    (the analogue of the paper's iterations / n0 versus tau study)."""
    torch, dev = _device_setup()
    from paper_2107_09006_gb300 import Solver, ls_solve
    from workloads import config_scale
    P = config_scale(side=args.side, block=args.block, zero_sum=args.zero_sum)
    b = torch.as_tensor(P.b, device=dev)
    x = torch.empty(P.n, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows = []

    def run(label, tau_label, **kw):
        t = time.time()
        S = Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, device=dev, stream=stream,
                   factor_prec=args.prec, maxit=3000, **kw)
        torch.cuda.synchronize(dev)
        setup = time.time() - t
        ls_solve(S.h, b, 1, args.rtol, x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        info = ls_solve(S.h, b, 1, args.rtol, x)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        si = S.info()
        row = {"form": label, "tau": tau_label, "n0": si["n0"], "kmax": si["kmax"], "iterations": info["iters"],
               "kappa_lanczos": info["kappa_lanczos"], "solve_s": e0.elapsed_time(e1) / 1000.0, "setup_s": setup}
        log(f"[tausweep] {json.dumps(row)}")
        rows.append(row)
        S.close()
        torch.cuda.empty_cache()

    run("one-level", None, coarse=0, nev_max=0)
    for tau in (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.8):
        for variant, label in ((0, "additive"), (1, "balanced")):
            run(label, tau, tau=tau, nev_max=64, variant=variant)
    print(json.dumps({"report": "tausweep", "workload": f"{P.name}, form {args.prec}, "
                      f"rtol {args.rtol:g}, nev_max 64", "rows": rows}), flush=True)


def run_diff(args):
    """Differentiation workload (512 x 512 grid, n = 262,144, 64 subdomains, x* drawn):
    loss ||x(A, b) - x*||^2; one step is the forward solve plus the adjoint solve that
    gives the gradients with respect to b and the stored values of A (LSSolve's forward
    and backward), each to 1e-10, in the FP64 and the mixed forms; the mixed forms'
    gradients are compared with the FP64 form's."""
    torch, dev = _device_setup()
    import numpy as np
    from paper_2107_09006_gb300 import Solver
    from workloads import config_diff
    P = config_diff()
    stream = torch.cuda.current_stream(dev)
    b = torch.as_tensor(P.b, device=dev)
    xs = torch.as_tensor(P.xstar, device=dev)
    rows, ref = [], None
    for form in ("f64", "f32", "bf16"):
        S = Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, device=dev, stream=stream,
                   nev_max=args.nev, factor_prec=form)

        def step():
            x, fi = S.solve(b, rtol=1e-10)
            gb, gv, bi = S.backward(b, x, 2.0 * (x - xs), rtol=1e-10)
            return x, gb, gv, fi, bi

        for _ in range(max(args.warmup, 1)):
            step()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            x, gb, gv, fi, bi = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        g = (gb.cpu().numpy(), gv.cpu().numpy())
        row = {"form": form, "s_per_step": e0.elapsed_time(e1) / 1000.0 / args.steps,
               "forward_iterations": fi["iters"], "adjoint_iterations": bi["iters"],
               "adjoint_relres_true": bi["relres_true"]}
        if form == "f64":
            ref = g
        else:
            row["grad_b_rel_diff_vs_f64"] = float(np.linalg.norm(g[0] - ref[0]) / np.linalg.norm(ref[0]))
            row["grad_vals_rel_diff_vs_f64"] = float(np.linalg.norm(g[1] - ref[1]) / np.linalg.norm(ref[1]))
        log(f"[diff] {json.dumps(row)}")
        rows.append(row)
        S.close()
        torch.cuda.empty_cache()
    print(json.dumps({"report": "diff", "workload": f"{P.name}: n={P.n}, m={P.m}, nnz={P.nnz}, 64 subdomains, "
                      f"nev_max {args.nev}, rtol 1e-10 forward and adjoint", "rows": rows}), flush=True)


def run_batch(args):
    """Batched workload: 64 independent problems (n log-uniform in [16384, 262144],
    square grids, 4n rows of 6 nonzeros within radius 2 plus 1e-2 I, uneven bisection
    subdomains of at most 8192 columns), 32 right-hand sides each, FP32 local factors
    inside FP64 flexible CG, one CUDA graph per iteration.  A step is one ls_solve of
    all problems and right-hand sides from x = 0 to every pair's own 1e-8 test."""
    torch, dev = _device_setup()
    import numpy as np
    from paper_2107_09006_gb300 import Solver, ls_solve
    from workloads import config_batch
    t = time.time()
    B = config_batch(nprob=args.nprob, nrhs=args.nrhs)
    log(f"[batch] generated in {time.time() - t:.1f}s: m={B.m} n={B.n} nnz={B.nnz} N={B.nparts}")
    stream = torch.cuda.current_stream(dev)
    t = time.time()
    S = Solver(B.m, B.n, B.row_ptr, B.col, B.val, B.part, B.nparts, device=dev, stream=stream,
               problems=(B.m_off, B.n_off), nev_max=args.nev, factor_prec=args.prec, time_kernels=1, maxit=500,
               block_kernel=args.block_kernel)
    torch.cuda.synchronize(dev)
    setup = time.time() - t
    si, st = S.info(), S.storage()
    log(f"[batch] setup {setup:.1f}s (eig+coarse {si['t_eig']:.1f}s) n0={si['n0']} fac={st['fac_elems']}")
    R = args.nrhs
    b_dev = torch.as_tensor(B.b, device=dev)
    x_dev = torch.empty((R, B.n), dtype=torch.float64, device=dev)
    for _ in range(max(args.warmup, 1)):
        ls_solve(S.h, b_dev, R, args.rtol, x_dev)
    ck = Clocks(dev.index or 0)
    ck.start()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [ls_solve(S.h, b_dev, R, args.rtol, x_dev) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = ck.stop()
    sec = e0.elapsed_time(e1) / 1000.0 / args.steps
    its, relres = S.batch_stats(R)
    inf = infos[-1]
    nl = max(inf["local_launches"], 1)
    ms_local = inf["ms_local"] / nl
    es = {"f64": 8, "f32": 4, "bf16": 2}[args.prec]
    ta = 8 if args.prec == "f64" else 4
    fac_bytes = 2 * st["fac_elems"] * es
    local_bytes = fac_bytes + st["total_local"] * R * 16 + st["total_local"] * 12 + \
        2 * st["total_blocks"] * 1024 * ta  # factor twice, R gather + R write, maps, spill
    local_flops = 4.0 * st["fac_elems"] * R  # 2 flops per element per sweep per right-hand side
    # end to end from pinned host b to pinned host x
    bh = torch.as_tensor(B.b).pin_memory()
    xh = torch.empty((R, B.n), dtype=torch.float64).pin_memory()
    ls_solve(S.h, bh, R, args.rtol, xh)
    torch.cuda.synchronize(dev)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        ls_solve(S.h, bh, R, args.rtol, xh)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    e2e = f0.elapsed_time(f1) / 1000.0 / args.steps
    pairs = B.nprob * R
    out = {
        "report": "batch", "metric": "batched LS solves/s to 1e-8 (problem x rhs pairs)",
        "value": pairs / sec, "unit": "solves/s", "s_per_step": sec, "pairs": pairs,
        "e2e": {"value": pairs / e2e, "unit": "solves/s", "h2d_bytes_per_step": int(B.m) * R * 8,
                "d2h_bytes_per_step": int(B.n) * R * 8},
        "workload": {"name": B.name, "nprob": B.nprob, "nrhs": R, "m": int(B.m), "n": int(B.n), "nnz": B.nnz,
                     "subdomains": B.nparts, "nev_max": args.nev, "form": args.prec, "rtol": args.rtol},
        "iterations": {"max": int(its.max()), "min": int(its.min()), "mean": float(its.mean())},
        "relres_true_max": float(relres.max()), "setup_s": setup, "eig_coarse_s": si["t_eig"], "n0": si["n0"],
        "ms_per_iteration_kernels": inf["ms_iter"] / max(inf["iters"], 1),
        "local_solve": {"ms_per_launch": ms_local, "bytes_per_launch": local_bytes,
                        "GBps": local_bytes / (ms_local * 1e-3) / 1e9,
                        "TFLOPs": local_flops / (ms_local * 1e-3) / 1e12},
        "spmm_pair_ms_per_iter": inf["ms_spmv"] / max(inf["iters"], 1),
        "coarse_ms_per_iter": inf["ms_coarse"] / max(inf["iters"], 1),
        "launches_per_step": inf["launches"], "clocks": clocks,
        "local_kernel": {0: "CUDA cores", 1: "TF32 mma.sync", 2: "tcgen05 (TMEM accumulator)"}[inf["local_kernel"]],
    }
    print(json.dumps(out), flush=True)
    S.close()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "nsweep":
        run_nsweep(a)
    elif a.mode == "precision":
        run_precision(a)
    elif a.mode == "batch":
        run_batch(a)
    elif a.mode == "tausweep":
        run_tausweep(a)
    elif a.mode == "diff":
        run_diff(a)
    else:
        run_ours(a)
