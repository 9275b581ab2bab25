#!/usr/bin/env python
"""SP2 density-matrix solves per second on one GB300, through the C ABI.

Workload (default): the random-cube tight-binding Hamiltonian with 2048 sites x
4 orbitals (N = 8192, Nocc = 4096, seed 0), the paper-shaped stand-in for the
dense SP2 benchmarks of arXiv 2401.13772 (§VI), solved in mixed precision: FP16
hi+lo split squarings on the tensor cores between an FP64-accurate prefix and an
FP64-accurate refinement, FP64 traces and decisions. One step = one whole solve:
Gershgorin bounds, X0 map, the SP2 product loop (decided on the device), and
the copy of D. Inputs are resident in HBM; L2 is flushed (256 MiB write) before
every timed step, outside its events.

The JSON line also carries: the same solve with BF16 hi+mid+lo split squarings
(its own rate and D check), the end-to-end rate through the same C ABI with
host buffers (H host->device and D device->host inside the timed region), the
roofline of the product kernels, the plain FP64 SP2 rate on the same GPU, the
element-wise error of every D against one whole solve of the CPU oracle (plain
FP64 SP2), clocks sampled during the timed region, and that oracle solve's time
on the host cores. `--sites 1024 --prec fp64` (or fp32_split) measures the
N = 4096 plain FP64 (or FP32-split) solve with the same checks.

--impl reference times the CPU oracle (plain FP64 SP2, numpy) on the host
cores instead, on a bounded sample of the same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SP2 solves/s & tensor TFLOP/s vs plain FP64 SP2, same GB300, at stated D error"
UNIT = "solves/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
NOMINAL_BF16_TFLOPS = 2250.0
OZ_KERNEL = ("square_oz_kernel (BF16 digit products, tcgen05; time includes digits_kernel, "
             "traffic is square_oz_kernel's)")
# DRAM bytes (read + write) per launch from one ncu capture of the kernel as it
# stands, keyed by (kernel, n); see profiles/.
SPLIT_KERNEL = "square_split_persist_kernel (tcgen05, FP16x2)"
WIDE_KERNEL = "square_wide_kernel (tcgen05, FP16x2, 128 x 256 tiles)"
NCU_TRAFFIC = {("square_fp64_kernel (FP64 DMMA)", 4096): 1101459200,
               ("square_df64_kernel (double-float, FP32 pipe)", 4096): 521512448,
               ("square_split_kernel (tcgen05)", 4096): 155314688,
               (SPLIT_KERNEL, 4096): 143759360,
               (SPLIT_KERNEL, 8192): 1897807872,
               # mean over one mixed solve's 12 launches (8 prefix products of 13
               # digit products, 4 refinement products of 15)
               (OZ_KERNEL, 4096): 570465856,
               (OZ_KERNEL, 8192): 4121248106}
NOMINAL_FP64_TFLOPS = 1.25
# FP64 ceiling of this GPU: cuBLAS DGEMM 8192^3 (torch.matmul, float64) measured
# on GB300 at 1.10 TFLOP/s (best of 5, CUDA events); used for the FP64 roofline
MEASURED_DGEMM_TFLOPS = 1.10
# FP32-class (all split) solves: no tolerance is stated for them. Gate used:
# max |D - D_ref| <= 1e-4 and |Tr D - Nocc| <= 4 n 2^-22 (the split phase stops
# on its round-off floor, about n times the slices' 2^-22 resolution)
FP32_GATE = {"max_abs_err": 1e-4, "trace_err_per_n": 4.0 * 2.0 ** -22}
DF_OPS = 12  # FP32 instructions per double-float multiply-add in square_df64_kernel
# BF16 digit products per FP64-accurate product in square_oz_kernel: all 15 in
# the refinement, 13 in the prefix (the library's default short form)
OZ_PRODUCTS = 15
OZ_PRODUCTS_PREFIX = 13
IMPL_DTYPE = {"double-float": "double-float", "native fp64": "f64",
              "digits": "bf16 digit products (f32 accumulate)"}


def fp64_impl_kind(args):
    """Arithmetic of the FP64-accurate products of the run."""
    if args.prec == "df64":
        return "double-float"
    if args.prec.startswith("mixed"):
        if args.fp64_impl == 0:  # the library default
            return "digits" if 4 * args.sites <= 8192 else "double-float"
        return {1: "native fp64", 2: "double-float", 3: "digits"}[args.fp64_impl]
    return "native fp64"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed_fp16",
                    choices=["fp64", "df64", "fp32_split", "fp32_split_bf16", "mixed_fp16",
                             "mixed_bf16"])
    ap.add_argument("--fp64-impl", type=int, default=0, choices=[0, 1, 2, 3],
                    help="mixed modes, FP64-accurate products: 0 = library default, 1 = native "
                         "FP64, 2 = double-float, 3 = tensor-core digit products")
    ap.add_argument("--sites", type=int, default=2048)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--tol", type=float, default=1e-10)
    ap.add_argument("--fp64-prefix", type=int, default=8)
    ap.add_argument("--split-tile", type=int, default=0, choices=[0, 1, 2],
                    help="tile of the FP16 split products: 0/1 = 128 x 128, 2 = 128 x 256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-bf16-leg", dest="bf16_leg", action="store_false",
                    help="mixed_fp16 runs: skip the same solve with bf16 hi+mid+lo splits")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the torch-side invariants of D (profiling runs)")
    ap.add_argument("--loop-mode", type=int, default=0,
                    help="0: device-driven WHILE graph; 1: plain launches (profilers)")
    ap.add_argument("--workload", default="dense",
                    choices=["dense", "batched", "learned", "graph", "cheb", "sparse"],
                    help="dense: one N = 8192 cube solve per step (headline); batched: 4000 "
                         "parts of 64..768 orbitals per step; learned: predictor training "
                         "and evaluation; graph: graph-based divide and conquer of a chain; "
                         "cheb: finite-temperature Chebyshev expansion of the N = 4096 cube H; "
                         "sparse: thresholded SP2 of a gapped chain")
    ap.add_argument("--graph-n", type=int, default=8192)
    ap.add_argument("--graph-tau", type=float, default=1e-5)
    ap.add_argument("--graph-parts", type=int, default=16)
    ap.add_argument("--graph-mu", type=float, default=0.1,
                    help="chemical potential (inside the chain's gap [-0.4, 0.4]; a cut chain "
                         "segment can hold an edge state at exactly 0)")
    ap.add_argument("--cheb-mu", type=float, default=0.5,
                    help="cheb workload: chemical potential (eV) of the Fermi function")
    ap.add_argument("--cheb-beta", type=float, default=1.0,
                    help="cheb workload: inverse temperature (1/eV)")
    ap.add_argument("--cheb-sites", type=int, default=1024,
                    help="cheb workload: cube sites (x 4 orbitals)")
    ap.add_argument("--cheb-k", type=int, default=16)
    ap.add_argument("--cheb-m", type=int, default=16)
    ap.add_argument("--cheb-prec", default="fp32_split", choices=["fp32_split", "fp32_split_bf16"])
    ap.add_argument("--no-diag-baseline", action="store_true",
                    help="cheb workload: skip the eigh comparator (e.g. under a profiler)")
    ap.add_argument("--sparse-n", type=int, default=16384)
    ap.add_argument("--sparse-tau", type=float, default=1e-6)
    ap.add_argument("--batch", type=int, default=4000)
    ap.add_argument("--batch-prec", default="fp32_split",
                    choices=["fp32_split", "fp32_split_bf16"])
    ap.add_argument("--no-tune", dest="tune", action="store_false",
                    help="batched workload: skip the launch-configuration autotuner")
    ap.add_argument("--train-count", type=int, default=20000)
    ap.add_argument("--eval-count", type=int, default=1000)
    ap.add_argument("--eval-sites", type=int, default=512)
    return ap.parse_args()


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


def workload_name(sites, seed):
    return (f"random-cube tight-binding H, {sites} sites x 4 orbitals (N={4 * sites}), "
            f"Nocc={2 * sites}, seed {seed}")


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.proc = None
        self.path = None
        self.gpu_id = gpu_id

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "200"]
            if self.gpu_id:
                cmd += ["-i", self.gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample)

def time_oracle_products(H, nocc, k_sample):
    """Time the oracle's plain FP64 SP2 (numpy) as it stands: the solve set-up
    (bounds, X0 map, traces) and k_sample products.
    Returns (t_setup, t_per_product) in seconds."""
    import oracle
    t0 = time.perf_counter()
    oracle.sp2_plain(H, nocc, 0.0, stop_after=0)
    t1 = time.perf_counter()
    oracle.sp2_plain(H, nocc, 0.0, stop_after=k_sample)
    t2 = time.perf_counter()
    t_setup = t1 - t0
    return t_setup, max(1e-9, (t2 - t1 - t_setup) / k_sample)


def cpu_cores():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return os.cpu_count() or 1


# ---------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands

def run_reference(args):
    """The CPU oracle as it stands (plain FP64 SP2, numpy) on the host cores.
    Each step is a bounded sample of one solve of the workload: the set-up
    (bounds, X0 map, traces) and `k_sample` products. `ms_per_step` is the
    measured time of one such step; `value` is solves/s, the sample's rate
    scaled to a whole solve by its iteration count."""
    import numpy as np
    import oracle
    from workloads import cube_hamiltonian
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    H, nocc = cube_hamiltonian(args.sites, args.seed)
    n = H.shape[0]
    # iteration count of the full solve, from the oracle's spectral SP2 on the
    # eigenvalues (numpy eigvalsh; not timed) -- only used to scale the sample
    w = np.linalg.eigvalsh(H)
    emin, emax = oracle.gershgorin_bounds(H)
    iters = oracle.spectral_sp2(w, nocc, args.tol, emin, emax)["iters"]
    k_sample = 1 if n >= 6000 else 2
    for _ in range(args.warmup):
        time_oracle_products(H, nocc, 1)
    step_sec, solve_sec = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        ts, tp = time_oracle_products(H, nocc, k_sample)
        step_sec.append(time.perf_counter() - t0)
        solve_sec.append(ts + iters * tp)
    sec = statistics.mean(solve_sec)
    value = 1.0 / sec
    sample = (f"{k_sample} of {iters} SP2 products (+ bounds and X0) per step on N={n}, "
              f"scaled to a whole solve by the iteration count")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(step_sec) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.sites, args.seed), "n": n,
                       "prec": "fp64 (numpy CPU oracle)", "tol": args.tol},
            "solve_ms_extrapolated": sec * 1e3,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm

def run_batched(args):
    """Batched workload: `--batch` cube parts of U{16..192} sites (n = 64..768),
    Nocc = n/2, one persistent launch per step. Under torchrun the parts are
    sharded over the ranks (greedy LPT on n^3, no collective on the data path)
    and the step time is the maximum over ranks."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    import paper_2401_13772_gb300 as pkg
    from paper_2401_13772_gb300.build import build
    from paper_2401_13772_gb300.sharding import max_over_ranks, shard_parts
    from workloads import batch_packed, batch_sizes
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    all_sites = batch_sizes(args.batch, 0)
    mine = np.array(shard_parts(4 * all_sites, world, rank) if world > 1 else
                    range(args.batch), dtype=np.int64)
    sites = all_sites[mine]
    packed, n, offsets, nocc = batch_packed(sites, 1000, index=mine)
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())
    Hh = torch.from_numpy(packed).pin_memory()
    H = Hh.to(dev)
    D = torch.empty_like(H)
    stream = torch.cuda.current_stream()
    tune = None
    if args.tune:
        # the launch-configuration autotuner, on every k-th part in size order
        # (outside the timed region); later launches use its choice
        stride = max(1, args.batch // 600)
        tune = pkg.batched_tune(H, n, offsets, nocc, 1e-10, D_packed=D, prec=args.batch_prec,
                                sample_stride=stride, reps=3)
        tune["sample_stride"] = stride
    for _ in range(max(1, args.warmup)):
        D, iters, status = pkg.sp2_batched(H, n, offsets, nocc, 1e-10, D_packed=D,
                                           prec=args.batch_prec)
    torch.cuda.synchronize()
    K = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
    clocks = ClockSampler()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for i in range(K):
        ev[2 * i].record(stream)
        pkg.sp2_batched(H, n, offsets, nocc, 1e-10, D_packed=D, prec=args.batch_prec)
        ev[2 * i + 1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    sec_local = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(K)) / K / 1e3
    sec = max_over_ranks(sec_local, device=dev)  # the whole job ends with its slowest rank
    # end to end through the C ABI with host buffers (H in, D out), every rank
    Dh_pin = torch.empty_like(Hh).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    H.copy_(Hh, non_blocking=True)
    pkg.sp2_batched(H, n, offsets, nocc, 1e-10, D_packed=D, prec=args.batch_prec)
    Dh_pin.copy_(D, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_sec = max_over_ranks(e0.elapsed_time(e1) / 1e3, device=dev)
    if rank != 0:
        dist.destroy_process_group()
        return
    it = iters.cpu().numpy()
    st = status.cpu().numpy()
    # per-part SM cycles of one more launch, by row blocks of 128 (outside the timing)
    _, _, _, cyc = pkg.sp2_batched(H, n, offsets, nocc, 1e-10, D_packed=D,
                                   prec=args.batch_prec, cycles=True)
    cyc = cyc.cpu().numpy().astype(np.float64)
    blocks = (n + 127) // 128
    by_blocks = {int(b): {"parts": int((blocks == b).sum()),
                          "mean_mcycles": round(float(cyc[blocks == b].mean()) / 1e6, 3),
                          "share_of_cycles": round(float(cyc[blocks == b].sum() / cyc.sum()), 3)}
                 for b in np.unique(blocks)}
    nn = n.astype(np.float64)
    flops = float(np.sum(it * nn * nn * (nn + 1)))  # this GPU's launch
    peaks, src = load_peaks()
    peak = peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"])
    ach = flops / sec_local / 1e12
    if args.no_check:  # profiling runs: the launch alone
        print(json.dumps({"metric": METRIC, "value": args.batch / sec, "unit": UNIT,
                          "ms_per_step": sec * 1e3, "tflops_algorithmic": ach}), flush=True)
        return
    # a loop of plain per-instance solves (dense FP32-split API), subsample
    sub = np.linspace(0, len(n) - 1, 100).astype(int)
    mats = [torch.from_numpy(packed[offsets[i]:offsets[i] + int(n[i]) ** 2].reshape(
        int(n[i]), int(n[i]))).to(dev) for i in sub]
    for m_, i in zip(mats[:3], sub[:3]):
        pkg.sp2_dense_ex(m_, int(nocc[i]), 1e-10, prec="fp32_split")
    torch.cuda.synchronize()
    e0.record(stream)
    for m_, i in zip(mats, sub):
        pkg.sp2_dense_ex(m_, int(nocc[i]), 1e-10, info=False, prec="fp32_split")
    e1.record(stream)
    torch.cuda.synchronize()
    loop_sec = e0.elapsed_time(e1) / 1e3 * args.batch / len(sub) / world
    # the same subsample as plain FP64 SP2 solves (FP64 accuracy), in a loop
    Ds64 = []
    for m_, i in zip(mats[:2], sub[:2]):
        pkg.sp2_dense_ex(m_, int(nocc[i]), 1e-10, prec="fp64")
    torch.cuda.synchronize()
    e0.record(stream)
    for m_, i in zip(mats, sub):
        Ds64.append(pkg.sp2_dense_ex(m_, int(nocc[i]), 1e-10, info=False, prec="fp64"))
    e1.record(stream)
    torch.cuda.synchronize()
    loop64_sec = e0.elapsed_time(e1) / 1e3 * args.batch / len(sub) / world
    # accuracy on a sample against the oracle: the per-part gate of the
    # FP32-class split products is min(0.2 2^-22 / relgap + 1e-6, 1e-2)
    Dh = D.cpu().numpy()
    errs, ratios, errs64 = [], [], []
    for q, i in enumerate(sub):
        if q % 12:
            continue
        k = int(n[i])
        Hi = packed[offsets[i]:offsets[i] + k * k].reshape(k, k)
        ref = oracle.sp2_plain(Hi, int(nocc[i]), 1e-10)
        e = float(np.abs(Dh[offsets[i]:offsets[i] + k * k].reshape(k, k) - ref["D"]).max())
        w = np.linalg.eigvalsh(Hi)
        emin, emax = oracle.gershgorin_bounds(Hi)
        relgap = (w[nocc[i]] - w[nocc[i] - 1]) / (emax - emin)
        errs.append(e)
        ratios.append(e / min(0.2 * 2.0 ** -22 / relgap + 1e-6, 1e-2))
        errs64.append(float(np.abs(Ds64[q].cpu().numpy() - ref["D"]).max()))
    # the oracle on a bounded sample of the batch, scaled to the whole batch
    t0 = time.perf_counter()
    for i in sub[:20]:
        k = int(n[i])
        oracle.sp2_plain(packed[offsets[i]:offsets[i] + k * k].reshape(k, k), int(nocc[i]),
                         1e-10)
    cpu_sec = (time.perf_counter() - t0) * args.batch / 20
    line = {"metric": METRIC, "value": args.batch / sec, "unit": UNIT, "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": sec * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("f16x2 split, f32 accumulate" if args.batch_prec == "fp32_split"
                      else "bf16x3 split, f32 accumulate"),
            "data": "synthetic",
            "config": {"workload": f"{args.batch} random-cube parts, U{{16..192}} sites x 4 "
                                   f"orbitals (n = 64..768), Nocc = n/2, seeds 1000+i",
                       "prec": args.batch_prec, "tol": 1e-10, "parallelism": "one GPU",
                       "l2": "inputs (about 7 GB) far larger than L2"},
            "iters_mean": float(it.mean()), "status_ok": int((st == 0).sum()),
            "tflops_algorithmic": ach,
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "traffic": None, "kernel": "batched_kernel",
                         "peak_source": f"fp16/bf16 dense, {src} burst",
                         "flops_per_launch": flops, "avg_launch_ms": sec_local * 1e3},
            "loop_baseline": {"value": args.batch / loop_sec, "unit": UNIT,
                              "speedup": loop_sec / sec,
                              "what": "per-instance dense FP32-split solves in a loop "
                                      "(100-instance subsample, scaled): the same accuracy "
                                      "class"},
            "loop_baseline_fp64": {"value": args.batch / loop64_sec, "unit": UNIT,
                                   "speedup": loop64_sec / sec,
                                   "max_abs_err_vs_oracle_sample": max(errs64),
                                   "what": "per-instance plain FP64 SP2 solves in a loop "
                                           "(same subsample, scaled): FP64 accuracy"},
            "d_check": {"max_abs_err_vs_oracle_sample": max(errs), "sample": len(errs),
                        "gate": "per part min(0.2 2^-22 / relgap + 1e-6, 1e-2) (FP32-class "
                                "split products)",
                        "max_err_over_gate": max(ratios), "pass": bool(max(ratios) <= 1.0)},
            "cpu_baseline": {"value": args.batch / cpu_sec, "unit": UNIT,
                             "cores": cpu_cores(), "kind": "oracle",
                             "sample": "20 instances of the batch (plain FP64 SP2, numpy), "
                                       "scaled to the batch"},
            "e2e": {"value": args.batch / e2e_sec, "unit": UNIT,
                    "h2d_bytes_per_step": int(packed.nbytes),
                    "d2h_bytes_per_step": int(packed.nbytes)},
            "gpu_launches": K, "clocks": clk,
            "launch_config": tune if tune is not None else "library default",
            "cycles_by_row_blocks": by_blocks}
    if world > 1:
        line["config"]["parallelism"] = f"parts sharded over {world} ranks (LPT on n^3)"
        dist.destroy_process_group()
    print(json.dumps(line), flush=True)


def run_learned(args):
    """Learned workload: train the predictor on `--train-count` cube instances
    (n = 256..2048 in steps of 4, seeds 10000+i) with SP2-derived labels, then
    evaluate on `--eval-count` fresh instances of `--eval-sites` sites (seeds
    50000+i): products per solve, fallback rate and batched solves/s with and
    without the predictions."""
    import numpy as np
    import torch
    from paper_2401_13772_gb300 import learned as L
    from paper_2401_13772_gb300.build import build
    from workloads import batch_packed
    build()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(0)
    train_sites = rng.integers(64, 513, size=args.train_count)
    margin, kmax = 0.02, 80
    chunk = 500

    def chunk_batch(c0):
        s_ = train_sites[c0:c0 + chunk]
        packed_, n_, off_, nocc_ = batch_packed(s_, 10000 + c0)
        b_ = {"H": torch.from_numpy(packed_).to(dev), "n": n_, "offsets": off_,
              "d_n": torch.from_numpy(n_).to(dev), "d_off": torch.from_numpy(off_).to(dev)}
        return b_, nocc_

    # stage 1: bound targets (extremal eigenvalues from SP2 runs)
    labs = []
    t0 = time.perf_counter()
    for c0 in range(0, args.train_count, chunk):
        b, nocc_c = chunk_batch(c0)
        lab = L.label_batch(b, nocc_c, margin, kmax)
        labs.append({k: v for k, v in lab.items()})
        del b
    X = torch.cat([lb["X"] for lb in labs])
    T = torch.cat([lb["T"] for lb in labs])
    M = torch.cat([lb["M"] for lb in labs])
    t_label = time.perf_counter() - t0
    P = L.Predictor(hidden=128, kmax=kmax, seed=0)
    # hold out 10 % of the instances to calibrate the bound margin
    perm = torch.randperm(X.shape[0], generator=torch.Generator().manual_seed(0)).to(X.device)
    n_val = max(1, X.shape[0] // 10)
    val, trn = perm[:n_val], perm[n_val:]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = P.fit(X[trn], T[trn], M[trn], epochs=200, batch=512, lr=2e-3)
    # calibrate on the held-out instances closest in size to the evaluation
    # set (the overshoot grows with n), all of them if too few
    n_train = torch.from_numpy(4 * train_sites).to(X.device)
    near = val[n_train[val] >= int(0.75 * 4 * args.eval_sites)]
    cal = near if near.numel() >= 50 else val
    margin = L.calibrate_margin(P.predict(X[cal]), T[cal])
    # stage 2: branch targets from runs with the predicted bounds
    T2s, M2s = [], []
    for lab, c0 in zip(labs, range(0, args.train_count, chunk)):
        b, nocc_c = chunk_batch(c0)
        T2, M2 = L.branch_labels(P, b, nocc_c, lab, margin)
        T2s.append(T2)
        M2s.append(M2)
        del b
    T2, M2 = torch.cat(T2s), torch.cat(M2s)
    losses += P.fit(X[trn], T2[trn], M2[trn], epochs=200, batch=512, lr=1e-3)
    margin = L.calibrate_margin(P.predict(X[cal]), T[cal])
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    # the margin that serves instances of the evaluation size best, picked on a
    # separate validation set of that size (seeds 60000+i), not on the
    # evaluation set: the calibrated quantile is the smallest candidate
    vpacked, vn, voff, vnocc = batch_packed(np.full(200, args.eval_sites), 60000)
    vb = {"H": torch.from_numpy(vpacked).to(dev), "n": vn, "offsets": voff,
          "d_n": torch.from_numpy(vn).to(dev), "d_off": torch.from_numpy(voff).to(dev)}
    vplain = L.batched_solve(vb, vnocc)
    vY = P.predict(L.features(vb))
    sweep = {}
    for mg in sorted({round(margin, 4), 0.03, 0.05, 0.08}):
        if mg < margin:
            continue
        r = L.batched_solve(vb, vnocc, bounds=L.predicted_bounds(vY, vplain["bounds"], mg))
        sweep[mg] = (r["products"].double().mean().item(), r["fallback"].double().mean().item())
    margin_cal = margin
    margin = min(sweep, key=lambda k: (sweep[k][0], k))
    del vb, vpacked
    packed, n, offsets, nocc = batch_packed(np.full(args.eval_count, args.eval_sites), 50000)
    ev = {"H": torch.from_numpy(packed).to(dev), "n": n, "offsets": offsets,
          "d_n": torch.from_numpy(n).to(dev), "d_off": torch.from_numpy(offsets).to(dev)}
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    plain, t_plain = timed(lambda: L.batched_solve(ev, nocc))
    gersh = plain["bounds"]

    def learned_solve():
        Y = P.predict(L.features(ev))
        return L.batched_solve(ev, nocc, bounds=L.predicted_bounds(Y, gersh, margin))
    lb, t_lb = timed(learned_solve)
    lj, t_lj = timed(lambda: L.solve_learned(P, ev, nocc, gersh, margin, judge_delta=0.5, tau=2.0))
    # D of a sample of evaluation instances against the oracle (plain FP64 SP2):
    # per instance gate min(0.2 2^-22 / relgap + 1e-6, 1e-2) of the FP32-class
    # split products
    import oracle
    dchk = {"sample": 4, "gate": "per instance min(0.2 2^-22 / relgap + 1e-6, 1e-2)"}
    worst = {"plain": 0.0, "predicted_bounds": 0.0, "bounds_and_branches": 0.0}
    ratio = dict(worst)
    outs = {"plain": plain["D"].cpu().numpy(), "predicted_bounds": lb["D"].cpu().numpy(),
            "bounds_and_branches": lj["D"].cpu().numpy()}
    for i in range(4):
        k = int(n[i])
        Hi = packed[offsets[i]:offsets[i] + k * k].reshape(k, k)
        ref = oracle.sp2_plain(Hi, int(nocc[i]), 1e-10)["D"]
        w = np.linalg.eigvalsh(Hi)
        emin, emax = oracle.gershgorin_bounds(Hi)
        g = min(0.2 * 2.0 ** -22 * (emax - emin) / (w[nocc[i]] - w[nocc[i] - 1]) + 1e-6, 1e-2)
        for key, Dk in outs.items():
            e = float(np.abs(Dk[offsets[i]:offsets[i] + k * k].reshape(k, k) - ref).max())
            worst[key] = max(worst[key], e)
            ratio[key] = max(ratio[key], e / g)
    dchk["max_abs_err_vs_oracle_sample"] = worst
    dchk["max_err_over_gate"] = ratio
    dchk["pass"] = bool(max(ratio.values()) <= 1.0)
    line = {"metric": METRIC, "value": args.eval_count / t_lb, "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 1, "ms_per_step": t_lb * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3 split, f32 accumulate",
            "data": "synthetic",
            "config": {"workload": f"learned bounds/branches: train {args.train_count} cube "
                                   f"instances (n 256..2048), eval {args.eval_count} x "
                                   f"n = {4 * args.eval_sites}",
                       "hidden": 128, "kmax": kmax, "judge_delta": 0.5,
                       "margin": margin,
                       "margin_rule": "fewest products on 200 validation instances of the "
                                      "evaluation size (seeds 60000+i) among the calibrated "
                                      "margin (0.97 quantile of the bound overshoot on "
                                      "held-out training instances of n >= 0.75 n_eval) and "
                                      "0.03, 0.05, 0.08",
                       "margin_calibrated": margin_cal,
                       "margin_sweep": {str(k): {"products_mean": v[0], "fallback_rate": v[1]}
                                        for k, v in sweep.items()},
                       "calibration_instances": int(cal.numel()),
                       "products": "per solve, a rejected predicted run included"},
            "plain": {"solves_per_s": args.eval_count / t_plain,
                      "products_mean": plain["products"].double().mean().item()},
            "predicted_bounds": {"solves_per_s": args.eval_count / t_lb,
                                 "products_mean": lb["products"].double().mean().item(),
                                 "fallback_rate": lb["fallback"].double().mean().item()},
            "bounds_and_branches": {"solves_per_s": args.eval_count / t_lj,
                                    "products_mean": lj["products"].double().mean().item(),
                                    "fallback_rate": lj["fallback"].double().mean().item(),
                                    "predicted_prefix_mean":
                                        lj["pred_len"].double().mean().item()},
            "d_check": dchk,
            "training": {"label_s": t_label, "train_s": t_train, "loss_first": losses[0],
                         "loss_last": losses[-1], "samples": args.train_count}}
    print(json.dumps(line), flush=True)


def run_graph(args):
    """Graph-based divide-and-conquer workload (§VIII.B): a gapped dimerized
    chain of `--graph-n` orbitals at its mid-gap chemical potential; the
    auxiliary matrix is a previously computed density matrix (here the dense
    mixed solve of the same H, which is also the reference); `--graph-parts`
    regular-segment cores, threshold `--graph-tau`. One step = one whole-system
    density matrix from the core-halo parts (one batched SP2 launch)."""
    import numpy as np
    import torch
    import oracle
    import paper_2401_13772_gb300 as pkg
    from paper_2401_13772_gb300.build import build
    from workloads import chain_hamiltonian
    build()
    dev = torch.device("cuda", 0)
    H_np, nocc = chain_hamiltonian(args.graph_n, -1.0, -0.6)
    n = H_np.shape[0]
    H = torch.from_numpy(H_np).to(dev)
    # reference and auxiliary matrix: the dense mixed solve (not timed)
    Dref, dinfo = pkg.sp2_dense_ex(H, nocc, 1e-10, prec="mixed_fp16", fp64_prefix=8)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    pkg.sp2_dense_ex(H, nocc, 1e-10, D=torch.empty_like(H), prec="mixed_fp16", fp64_prefix=8,
                     info=False)
    e1.record()
    torch.cuda.synchronize()
    dense_ms = e0.elapsed_time(e1)
    G = Dref.clone()
    D = torch.empty_like(H)
    tau, parts, mu = args.graph_tau, args.graph_parts, args.graph_mu
    for _ in range(max(1, args.warmup)):
        D, ginfo = pkg.sp2_graph(H, G, tau, parts, mu, 1e-10, D=D)
    torch.cuda.synchronize()
    K = args.steps
    clocks = ClockSampler()
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
    for i in range(K):
        ev[2 * i].record()
        pkg.sp2_graph(H, G, tau, parts, mu, 1e-10, D=D)
        ev[2 * i + 1].record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    sec = sum(ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(K)) / K / 1e3
    Dn = D.cpu().numpy()
    Dr = Dref.cpu().numpy()
    err = float(np.abs(Dn - Dr).max())
    # the oracle's graph solve on the host cores (same tau, parts, auxiliary)
    t0 = time.perf_counter()
    P, _ = oracle.graph_density(H_np, Dr, tau, parts, mu, 1e-10)
    cpu_sec = time.perf_counter() - t0
    err_oracle = float(np.abs(Dn - P).max())
    # end to end: H and G in from pinned host memory, D out
    Hh = torch.from_numpy(H_np).pin_memory()
    Gh = G.cpu().pin_memory()
    Dh = torch.empty_like(Hh).pin_memory()
    torch.cuda.synchronize()
    e0.record()
    H.copy_(Hh, non_blocking=True)
    G.copy_(Gh, non_blocking=True)
    pkg.sp2_graph(H, G, tau, parts, mu, 1e-10, D=D)
    Dh.copy_(D, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_sec = e0.elapsed_time(e1) / 1e3
    s_mean = ginfo["mean_part"]
    flops = ginfo["max_iters"] * parts * s_mean ** 3  # upper estimate of the SP2 products
    peaks, src = load_peaks()
    line = {"metric": METRIC, "value": 1.0 / sec, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16x2 split, f32 accumulate",
            "data": "synthetic",
            "config": {"workload": f"graph-based divide and conquer: dimerized chain N={n} "
                                   f"(t1=-1.0, t2=-0.6, gap 0.8), mu={mu}, {parts} regular-segment "
                                   f"cores, tau={tau} on a previous density matrix",
                       "parallelism": "one GPU"},
            "parts": ginfo, "d_check": {"max_abs_err_vs_dense_solve": err,
                                        "max_abs_err_vs_oracle_graph_solve": err_oracle},
            "dense_mixed_solve_ms": dense_ms, "speedup_vs_dense": dense_ms / (sec * 1e3),
            "roofline": {"bound": "tensor", "achieved": flops / sec / 1e12,
                         "peak": peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]),
                         "unit": "TFLOP/s", "traffic": None,
                         "kernel": "batched_kernel (whole graph step timed)",
                         "peak_source": f"fp16/bf16 dense, {src} burst",
                         "flops_per_launch": flops},
            "cpu_baseline": {"value": 1.0 / cpu_sec, "unit": UNIT, "cores": cpu_cores(),
                             "kind": "oracle", "sample": "one whole graph solve (same tau, "
                                                         "parts and auxiliary matrix)"},
            "e2e": {"value": 1.0 / e2e_sec, "unit": UNIT,
                    "h2d_bytes_per_step": int(2 * H_np.nbytes),
                    "d2h_bytes_per_step": int(H_np.nbytes)},
            "gpu_launches": 5 * K, "clocks": clk}
    line["roofline"]["frac"] = line["roofline"]["achieved"] / line["roofline"]["peak"]
    print(json.dumps(line), flush=True)


def run_cheb(args):
    """Chebyshev Fermi-operator workload (§IV.B): the random-cube H of the dense
    workload (`--sites` x 4 orbitals), f(H) at a known chemical potential and
    temperature, L + 1 = k m terms in the Paterson-Stockmeyer form. One step =
    one whole density matrix through the public call (Gershgorin bounds, one
    read-back of them, coefficients on the host, every product on the GPU)."""
    import numpy as np
    import torch
    import oracle
    import paper_2401_13772_gb300 as pkg
    from paper_2401_13772_gb300.build import build
    from workloads import cube_hamiltonian
    build()
    dev = torch.device("cuda", 0)
    H_np, _ = cube_hamiltonian(args.cheb_sites, args.seed)
    n = H_np.shape[0]
    H = torch.from_numpy(H_np).to(dev)
    D = torch.empty_like(H)
    mu, beta, k, m, prec = args.cheb_mu, args.cheb_beta, args.cheb_k, args.cheb_m, args.cheb_prec
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    info = None
    for _ in range(max(1, args.warmup)):
        D, info = pkg.cheb_fermi(H, mu, beta, k, m, prec=prec, D=D)
    torch.cuda.synchronize()
    K = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
    clocks = ClockSampler()
    clocks.start()
    ms = []
    for i in range(K):
        flush.zero_()  # L2 flushed before each step (outside the events)
        ev[2 * i].record()
        pkg.cheb_fermi(H, mu, beta, k, m, prec=prec, D=D)
        ev[2 * i + 1].record()
        torch.cuda.synchronize()
        ms.append(ev[2 * i].elapsed_time(ev[2 * i + 1]))
    clk = clocks.stop()
    sec = sum(ms) / K / 1e3
    Dn = D.cpu().numpy()
    # the oracle's whole solve on the host cores: accuracy and the CPU baseline
    cpu_sec, err = None, None
    if not args.no_cpu_baseline:
        t0 = time.perf_counter()
        ref = oracle.fermi_operator(H_np, mu, beta, k, m)
        cpu_sec = time.perf_counter() - t0
        err = float(np.abs(Dn - ref["D"]).max())
    # diagonalization comparator of the paper's Chebyshev figure: FP64 eigh on
    # the GPU (cuSOLVER through torch) and V f(w) V^T, timed once
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    diag_ms, err_diag = None, None
    if not args.no_diag_baseline:
        torch.cuda.synchronize()
        e0.record()
        w, V = torch.linalg.eigh(H)
        f = 0.5 * (1.0 - torch.tanh(0.5 * beta * (w - mu)))
        Dd = (V * f) @ V.T
        e1.record()
        torch.cuda.synchronize()
        diag_ms = e0.elapsed_time(e1)
        err_diag = float((D - Dd).abs().max())
    # end to end: H in from pinned host memory, D out
    Hh = torch.from_numpy(H_np).pin_memory()
    Dh = torch.empty_like(Hh).pin_memory()
    torch.cuda.synchronize()
    e0.record()
    H.copy_(Hh, non_blocking=True)
    pkg.cheb_fermi(H, mu, beta, k, m, prec=prec, D=D)
    Dh.copy_(D, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_sec = e0.elapsed_time(e1) / 1e3
    products = info["products"]
    # each product of two commuting symmetric matrices is symmetric: the kernel
    # computes the upper triangle, n^2 (n + 1) flops (a GEMM would count 2 n^3)
    flops = float(n) * n * (n + 1) * products
    peaks, src = load_peaks()
    peak = peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"])
    slope = beta * 0.5 * (info["emax"] - info["emin"]) / 4.0
    gate = 8.0 * 2.0 ** -23 * max(1.0, info["growth"]) * max(1.0, slope)
    line = {"metric": METRIC, "value": 1.0 / sec, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f16x2 split, f32 accumulate" if prec == "fp32_split"
                      else "bf16x3 split, f32 accumulate"),
            "data": "synthetic",
            "config": {"workload": f"Chebyshev Fermi operator (Paterson-Stockmeyer): random-cube "
                                   f"tight-binding H, {args.cheb_sites} sites x 4 orbitals (N={n}), "
                                   f"seed {args.seed}, mu={mu} eV, beta={beta}/eV, "
                                   f"L+1={k * m} terms (k={k}, m={m})",
                       "parallelism": "one GPU",
                       "l2": "flushed before each step (256 MiB write, outside events)"},
            "cheb": info, "serial_recursion_products": k * m - 1,
            "d_check": {"max_abs_err_vs_oracle": err, "gate": gate,
                        "max_abs_err_vs_eigh": err_diag,
                        "truncation_last_coefficient": info["coef_last"]},
            "diag_baseline": None if diag_ms is None else {
                "ms": diag_ms, "speedup": diag_ms / (sec * 1e3),
                "what": "torch.linalg.eigh (FP64, cuSOLVER) + V f V^T on the same GPU"},
            "tflops_algorithmic": flops / sec / 1e12,
            "roofline": {"bound": "tensor", "achieved": flops / sec / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "frac": flops / sec / 1e12 / peak, "traffic": None,
                         "kernel": "cheb_product_kernel (whole solve timed: bounds, host "
                                   "coefficients, T_1, S_j pass and trace included)",
                         "peak_source": f"fp16/bf16 dense, {src} burst",
                         "flops_per_step": flops},
            "cpu_baseline": None if cpu_sec is None else {
                "value": 1.0 / cpu_sec, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                "sample": "one whole solve (same H, mu, beta, k, m; numpy FP64)"},
            "e2e": {"value": 1.0 / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": int(H_np.nbytes),
                    "d2h_bytes_per_step": int(H_np.nbytes)},
            "gpu_launches": info["launches"] * K, "clocks": clk}
    print(json.dumps(line), flush=True)


def run_sparse(args):
    """Thresholded SP2 workload (Listing 1's cutoff tau): the gapped dimerized
    chain of `--sparse-n` orbitals (t1 = -1, t2 = -0.6, half filling), whose
    density matrix is exponentially localized, FP32-split products with
    tau = `--sparse-tau`. One step = one whole solve through the public call.
    Accuracy: rows of D against the exact projector of a 512-site periodic chain
    (the same translation-invariant entries to double precision within 256
    sites of the diagonal, and below 1e-30 beyond)."""
    import numpy as np
    import torch
    import oracle
    import paper_2401_13772_gb300 as pkg
    from paper_2401_13772_gb300.build import build
    from workloads import chain_hamiltonian
    build()
    dev = torch.device("cuda", 0)
    n, tau = args.sparse_n, args.sparse_tau
    H_np, nocc = chain_hamiltonian(n, -1.0, -0.6)
    H = torch.from_numpy(H_np).to(dev)
    D = torch.empty_like(H)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    opts = dict(prec="fp32_split", tau=tau, loop_mode=args.loop_mode)
    info = None
    for _ in range(max(1, args.warmup)):
        D, info = pkg.sp2_dense_ex(H, nocc, 1e-9, D=D, **opts)
    torch.cuda.synchronize()
    K = args.steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * K)]
    clocks = ClockSampler()
    clocks.start()
    ms = []
    for i in range(K):
        flush.zero_()
        ev[2 * i].record()
        pkg.sp2_dense_ex(H, nocc, 1e-9, D=D, info=False, **opts)
        ev[2 * i + 1].record()
        torch.cuda.synchronize()
        ms.append(ev[2 * i].elapsed_time(ev[2 * i + 1]))
    clk = clocks.stop()
    sec = sum(ms) / K / 1e3
    # dense FP32-split solve of the same H (tau = 0), timed once
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Dd, dinfo = pkg.sp2_dense_ex(H, nocc, 1e-9, prec="fp32_split")
    torch.cuda.synchronize()
    e0.record()
    pkg.sp2_dense_ex(H, nocc, 1e-9, D=Dd, prec="fp32_split", info=False)
    e1.record()
    torch.cuda.synchronize()
    dense_ms = e0.elapsed_time(e1)
    # accuracy on sampled rows against the 512-site exact projector
    Hs, ns = chain_hamiltonian(512, -1.0, -0.6)
    w, V = oracle.jacobi_eigh(Hs)
    P, _ = oracle.density_projector(w, V, ns)
    rows = np.linspace(0, n - 1, 64).astype(np.int64)
    Dn = D[torch.from_numpy(rows).to(dev)].cpu().numpy()
    err_band, out_max = 0.0, 0.0
    for k, r in enumerate(rows):
        off = (np.arange(n) - r + n // 2) % n - n // 2  # signed distance on the ring
        band = np.abs(off) < 256
        ref = P[r % 2, (r % 2 + off[band]) % 512]
        err_band = max(err_band, float(np.abs(Dn[k, band] - ref).max()))
        out_max = max(out_max, float(np.abs(Dn[k, ~band]).max()) if (~band).any() else 0.0)
    nnz_frac = float((Dn != 0).mean())
    # the oracle (thresholded SP2, numpy FP64, dense products) on a 2048-site
    # chain, scaled by n^3 to this size
    Hc, nc = chain_hamiltonian(2048, -1.0, -0.6)
    t0 = time.perf_counter()
    from oracle import sparse as osp
    osp.sp2_thresholded(Hc, nc, 1e-9, tau)
    cpu_sec = (time.perf_counter() - t0) * (n / 2048.0) ** 3
    # end to end: H in from pinned host memory, D out
    Hh = torch.from_numpy(H_np).pin_memory()
    Dh = torch.empty_like(Hh).pin_memory()
    torch.cuda.synchronize()
    e0.record()
    H.copy_(Hh, non_blocking=True)
    pkg.sp2_dense_ex(H, nocc, 1e-9, D=D, info=False, **opts)
    Dh.copy_(D, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_sec = e0.elapsed_time(e1) / 1e3
    ld = (n + 127) // 128 * 128
    T = ld // 128
    dense_kb = info["iters"] * T * (T + 1) // 2 * (ld // 64)
    flops = float(info["kblocks"]) * 128 * 128 * 64 * 2  # product work actually streamed
    peaks, src = load_peaks()
    peak = peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"])
    line = {"metric": METRIC, "value": 1.0 / sec, "unit": UNIT, "n_gpus": 1, "steps": K,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16x2 split, f32 accumulate",
            "data": "synthetic",
            "config": {"workload": f"thresholded SP2: dimerized chain N={n} (t1=-1.0, t2=-0.6, "
                                   f"gap 0.8), Nocc={nocc}, tau={tau}",
                       "parallelism": "one GPU",
                       "l2": "flushed before each step (256 MiB write, outside events)"},
            "iters": info["iters"], "status": info["status"],
            "kblocks": info["kblocks"], "dense_kblocks": dense_kb,
            "streamed_fraction": info["kblocks"] / dense_kb,
            "d_check": {"max_abs_err_vs_exact_in_band": err_band,
                        "max_abs_outside_band": out_max, "rows_checked": len(rows),
                        "nonzero_fraction_of_rows": nnz_frac,
                        "trace_err": abs(info["trace"] - nocc)},
            "dense_split_solve_ms": dense_ms, "speedup_vs_dense": dense_ms / (sec * 1e3),
            "roofline": {"bound": "tensor", "achieved": flops / sec / 1e12, "peak": peak,
                         "unit": "TFLOP/s", "frac": flops / sec / 1e12 / peak, "traffic": None,
                         "kernel": "square_split_kernel (thresholded; whole solve timed, "
                                   "work = tile steps streamed)",
                         "peak_source": f"fp16/bf16 dense, {src} burst",
                         "flops_per_step": flops},
            "cpu_baseline": {"value": 1.0 / cpu_sec, "unit": UNIT, "cores": cpu_cores(),
                             "kind": "oracle",
                             "sample": "thresholded SP2 oracle (dense numpy FP64 products) on "
                                       "the 2048-site chain, time scaled by (N/2048)^3"},
            "e2e": {"value": 1.0 / e2e_sec, "unit": UNIT, "h2d_bytes_per_step": int(H_np.nbytes),
                    "d2h_bytes_per_step": int(H_np.nbytes)},
            "gpu_launches": (info["iters"] + 5) * K, "clocks": clk}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched":
        run_batched(args)
        return
    if args.workload == "learned":
        run_learned(args)
        return
    if args.workload == "graph":
        run_graph(args)
        return
    if args.workload == "cheb":
        run_cheb(args)
        return
    if args.workload == "sparse":
        run_sparse(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2401_13772_gb300.build import build
    if rank == 0 or world == 1:
        build()
    if world > 1:
        dist.barrier()
    import paper_2401_13772_gb300 as pkg
    from workloads import cube_hamiltonian

    H_np, nocc = cube_hamiltonian(args.sites, args.seed)
    n = H_np.shape[0]
    H = torch.from_numpy(H_np).to(dev)
    D = torch.empty_like(H)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def mk_events(k):
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
        for e in evs:
            e.record()
        return evs

    opts = dict(prec=args.prec, fp64_prefix=args.fp64_prefix, loop_mode=args.loop_mode,
                fp64_impl=args.fp64_impl, split_tile=args.split_tile)
    # warm-up (builds the loop graph) and the iteration count
    info = None
    for _ in range(max(1, args.warmup)):
        _, info = pkg.sp2_dense_ex(H, nocc, args.tol, D=D, **opts)
    iters = info["iters"]
    impl = fp64_impl_kind(args)
    body_kernels = 1 if args.prec in ("fp64", "df64", "fp32_split", "fp32_split_bf16") else \
        (3 if impl == "digits" else 2)
    if args.loop_mode == 0:
        launches_per_solve = 3 + body_kernels * max(iters, 1) + 1
    else:
        launches_per_solve = 3 + body_kernels * (100 + 1) + 1

    K = args.steps
    ev_s, ev_e = mk_events(K), mk_events(K)
    lp_s, lp_e = mk_events(K), mk_events(K)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    gpu_uuid = None
    try:
        gpu_uuid = str(torch.cuda.get_device_properties(dev).uuid)
        if not gpu_uuid.startswith("GPU-"):
            gpu_uuid = "GPU-" + gpu_uuid
    except Exception:
        gpu_uuid = None
    clocks = ClockSampler(gpu_uuid)
    clocks.start()
    torch.cuda.synchronize()
    for i in range(K):
        flush.zero_()
        ev_s[i].record(stream)
        pkg.sp2_dense_ex(H, nocc, args.tol, D=D, info=False, loop_events=(lp_s[i], lp_e[i]),
                         **opts)
        ev_e[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [ev_s[i].elapsed_time(ev_e[i]) for i in range(K)]
    loop_ms = [lp_s[i].elapsed_time(lp_e[i]) for i in range(K)]
    total_ms = sum(step_ms)
    if world > 1:
        from paper_2401_13772_gb300.sharding import max_over_ranks
        total_ms = max_over_ranks(total_ms, device=dev)
    value = world * K / (total_ms / 1e3)
    ms_per_step = total_ms / K

    # per-solve check of the result (status of the last timed solve)
    _, qinfo = pkg.sp2_dense_ex(H, nocc, args.tol, D=D, **opts)
    D_main = D.clone()
    check = {}
    if not args.no_check:
        # accuracy invariants of D (torch FP64 matmul, outside the timed region)
        check = {"idempotency_max": float((D_main @ D_main - D_main).abs().max()),
                 "trace_err": abs(float(torch.trace(D_main)) - nocc),
                 "commutator_max_rel": float((H @ D_main - D_main @ H).abs().max()) /
                 float(H.abs().max())}

    # Product-kernel launch durations. Inside the WHILE graph a launch cannot
    # be bracketed by events, so the loop region is timed per step (events
    # recorded by the library around the loop) and divided by the products.
    # In the mixed modes the two kernels share that region: the split
    # kernel's own average comes from an all-split solve of the same matrix
    # and is subtracted.
    flops_alg = float(n) * n * (n + 1)  # one symmetric square, upper triangle
    peaks, peak_src = load_peaks()
    bf16_peak = peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"])
    fp64_peak = MEASURED_DGEMM_TFLOPS
    loop_mean = statistics.mean(loop_ms)
    phases = qinfo["phase_iters"]
    n_fp64 = phases[0] + phases[2]
    n_split = phases[1]

    def roof(kernel, ms, peak, note, bound="tensor"):
        ach = flops_alg / (ms * 1e-3) / 1e12
        return {"bound": bound, "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": NCU_TRAFFIC.get((kernel, n)), "kernel": kernel,
                "peak_source": note,
                "flops_per_launch": flops_alg, "avg_launch_ms": ms}

    note64 = ("fp64: measured cuBLAS DGEMM 8192^3 on this GPU (1.10 TFLOP/s; the kernel does "
              "the upper triangle, so its algorithmic rate is its FP64 work rate)")
    note16 = f"fp16/bf16 dense, {peak_src} burst"
    # double-float products: FP32 pipe, 152 SMs x 128 lanes x max SM clock,
    # DF_OPS FP32 instructions per double-float multiply-add (2 flops)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    df_peak = 152 * 128 * sm_mhz * 1e6 * 2.0 / DF_OPS / 1e12
    notedf = (f"double-float: 152 SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz x 2 flops / "
              f"{DF_OPS} FP32 instructions per multiply-add")
    if impl == "double-float":
        k64, p64, n64, b64 = ("square_df64_kernel (double-float, FP32 pipe)", df_peak, notedf,
                              "alu")
    elif impl == "digits":
        # mean digit products per FP64-accurate product of this solve
        oz_mean = ((phases[0] * OZ_PRODUCTS_PREFIX + phases[2] * OZ_PRODUCTS) / n_fp64
                   if n_fp64 else float(OZ_PRODUCTS))
        k64, p64, b64 = (OZ_KERNEL, bf16_peak / oz_mean, "tensor")
        n64 = (f"fp16/bf16 dense, {peak_src} burst / {oz_mean:.2f} BF16 digit products per "
               f"FP64-accurate product ({phases[0]} prefix products of {OZ_PRODUCTS_PREFIX}, "
               f"{phases[2]} refinement products of {OZ_PRODUCTS})")
    else:
        k64, p64, n64, b64 = ("square_fp64_kernel (FP64 DMMA)", fp64_peak, note64, "tensor")
    split_kernel = ("square_split_kernel (tcgen05, BF16x3)" if "bf16" in args.prec
                    else WIDE_KERNEL if args.split_tile == 2 else SPLIT_KERNEL)
    split_ms = None
    if n_split > 0:
        if n_fp64 == 0:
            split_ms = loop_mean / n_split
        else:
            sp_s, sp_e = mk_events(1)[0], mk_events(1)[0]
            pkg.sp2_dense_ex(H, nocc, args.tol, D=D, prec="fp32_split", fp64_prefix=0,
                             loop_mode=args.loop_mode, split_tile=args.split_tile)
            _, sinfo = pkg.sp2_dense_ex(H, nocc, args.tol, D=D, prec="fp32_split",
                                        loop_events=(sp_s, sp_e), loop_mode=args.loop_mode,
                                        split_tile=args.split_tile)
            torch.cuda.synchronize()
            split_ms = sp_s.elapsed_time(sp_e) / max(sinfo["iters"], 1)
    fp64_ms = None
    if n_fp64 > 0:
        fp64_ms = (loop_mean - n_split * (split_ms or 0.0)) / n_fp64
    if fp64_ms is not None and (split_ms is None or n_fp64 * fp64_ms >= n_split * split_ms):
        roofline = roof(k64, fp64_ms, p64, n64, b64)
        secondary = roof(split_kernel, split_ms, bf16_peak, note16) \
            if split_ms else None
    else:
        roofline = roof(split_kernel, split_ms, bf16_peak, note16)
        secondary = roof(k64, fp64_ms, p64, n64, b64) if fp64_ms else None
    if secondary is not None:
        roofline["secondary"] = secondary

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "df64": "double-float (f32 pairs)",
                      "fp32_split": "f16x2 split, f32 accumulate, f64 traces",
                      "fp32_split_bf16": "bf16x3 split, f32 accumulate, f64 traces",
                      "mixed_fp16": IMPL_DTYPE[impl] + " prefix/refine + f16x2 split",
                      "mixed_bf16": IMPL_DTYPE[impl] + " prefix/refine + bf16x3 split"}[
                          args.prec],
            "data": "synthetic",
            "config": {"workload": workload_name(args.sites, args.seed), "n": n, "nocc": nocc,
                       "prec": args.prec, "tol": args.tol, "rule": "nearer",
                       "fp64_prefix": args.fp64_prefix,
                       "fp64_accurate_products": impl,
                       **({"split_tile": "128x256"} if args.split_tile == 2 else {}),
                       "parallelism": f"replicas x{world}",
                       "l2": "flushed before each step (256 MiB write, outside events)"},
            "iters": iters, "status": qinfo["status"], "phase_iters": qinfo["phase_iters"],
            "tflops_algorithmic": iters * flops_alg / (ms_per_step * 1e-3) / 1e12,
            "d_check": check,
            "roofline": roofline, "gpu_launches": launches_per_solve * K,
            "clocks": clk}

    # end to end through the C ABI with host buffers
    if not args.no_e2e:
        Hh = torch.from_numpy(H_np).pin_memory()
        Dh = torch.empty((n, n), dtype=torch.float64).pin_memory()
        Hd2 = torch.empty_like(H)
        Dd2 = torch.empty_like(H)
        es, ee = mk_events(K), mk_events(K)
        torch.cuda.synchronize()
        for i in range(K):
            flush.zero_()
            es[i].record(stream)
            Hd2.copy_(Hh, non_blocking=True)
            if args.prec == "fp64" and args.loop_mode == 0:
                pkg.sp2_dense(Hd2, nocc, args.tol, D=Dd2)
            else:
                pkg.sp2_dense_ex(Hd2, nocc, args.tol, D=Dd2, info=False, **opts)
            Dh.copy_(Dd2, non_blocking=True)
            ee[i].record(stream)
        torch.cuda.synchronize()
        e2e_ms = sum(es[i].elapsed_time(ee[i]) for i in range(K))
        if world > 1:
            t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_ms = float(t.item())
        line["e2e"] = {"value": world * K / (e2e_ms / 1e3), "unit": UNIT,
                       "h2d_bytes_per_step": n * n * 8, "d2h_bytes_per_step": n * n * 8}

    # the same solve with bf16 hi+mid+lo split squarings (mixed runs with fp16)
    D_bf16 = None
    if args.prec == "mixed_fp16" and args.bf16_leg:
        bopts = dict(opts, prec="mixed_bf16")
        pkg.sp2_dense_ex(H, nocc, args.tol, D=D, **bopts)  # warm-up (builds its graph)
        kb = min(K, 5)
        bs, be = mk_events(kb), mk_events(kb)
        torch.cuda.synchronize()
        for i in range(kb):
            flush.zero_()
            bs[i].record(stream)
            pkg.sp2_dense_ex(H, nocc, args.tol, D=D, info=False, **bopts)
            be[i].record(stream)
        torch.cuda.synchronize()
        bms = sum(bs[i].elapsed_time(be[i]) for i in range(kb)) / kb
        binfo = pkg.query()
        D_bf16 = D.clone()
        bchk = {}
        if not args.no_check:
            bchk = {"idempotency_max": float((D_bf16 @ D_bf16 - D_bf16).abs().max()),
                    "trace_err": abs(float(torch.trace(D_bf16)) - nocc)}
        line["mixed_bf16"] = {"value": 1e3 / bms, "unit": UNIT, "ms_per_step": bms,
                              "steps": kb, "dtype": IMPL_DTYPE[impl] +
                              " prefix/refine + bf16x3 split",
                              "iters": binfo["iters"], "phase_iters": binfo["phase_iters"],
                              "status": binfo["status"], "d_check": bchk}

    # plain FP64 SP2 on the same GPU (the comparison the metric asks for)
    D_64 = None
    if args.prec != "fp64" and not args.no_fp64_baseline:
        if n < 6000:  # warm-up; at large n one solve takes tens of seconds and
            pkg.sp2_dense_ex(H, nocc, args.tol, D=D, prec="fp64")  # its graph costs ~1 ms
        e0, e1 = mk_events(1)[0], mk_events(1)[0]
        torch.cuda.synchronize()
        flush.zero_()
        e0.record(stream)
        pkg.sp2_dense_ex(H, nocc, args.tol, D=D, info=False, prec="fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1)
        i64 = pkg.query()
        D_64 = D.clone()
        line["fp64_baseline"] = {"value": 1e3 / t64, "unit": UNIT, "iters": i64["iters"],
                                 "status": i64["status"],
                                 "speedup": (value / world) / (1e3 / t64)}
        if "mixed_bf16" in line:
            line["mixed_bf16"]["speedup_vs_fp64"] = line["mixed_bf16"]["value"] / (1e3 / t64)

    # CPU oracle on the host cores (rank 0, N = 1 only): one whole plain FP64
    # SP2 solve (numpy), which is also the reference D of every error check
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        t0 = time.perf_counter()
        ref = oracle.sp2_plain(H_np, nocc, args.tol)
        sec = time.perf_counter() - t0
        Dref = ref["D"]
        mixed_gate = {"max_abs_err": 1e-5, "trace_err": 1e-8}
        gates = {"fp64": {"max_abs_err": 1e-10}, "df64": {"max_abs_err": 1e-10},
                 "mixed_fp16": mixed_gate, "mixed_bf16": mixed_gate,
                 "fp32_split": FP32_GATE, "fp32_split_bf16": FP32_GATE}
        err = float(np.abs(D_main.cpu().numpy() - Dref).max())
        line["d_check"]["max_abs_err_vs_oracle"] = err
        line["d_check"]["gate"] = gates[args.prec]
        line["d_check"]["oracle_iters"] = ref["iters"]
        g = dict(gates[args.prec])
        if "trace_err_per_n" in g:
            g["trace_err"] = g.pop("trace_err_per_n") * n
        line["d_check"]["gate"] = g
        line["d_check"]["pass"] = bool(err <= g["max_abs_err"] and (
            "trace_err" not in g or "trace_err" not in check or
            check["trace_err"] <= g["trace_err"]))
        if D_bf16 is not None:
            e = float(np.abs(D_bf16.cpu().numpy() - Dref).max())
            bc = line["mixed_bf16"]["d_check"]
            bc["max_abs_err_vs_oracle"] = e
            bc["gate"] = mixed_gate
            bc["pass"] = bool(e <= 1e-5 and bc.get("trace_err", 0.0) <= 1e-8)
        if D_64 is not None:
            e = float(np.abs(D_64.cpu().numpy() - Dref).max())
            line["fp64_baseline"]["d_check"] = {"max_abs_err_vs_oracle": e, "gate": 1e-10,
                                                "pass": bool(e <= 1e-10)}
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": UNIT, "cores": cpu_cores(),
                                "kind": "oracle",
                                "sample": f"one whole solve of the same N={n} workload "
                                          f"(plain FP64 SP2, numpy matmul, {ref['iters']} "
                                          f"products); its D is the reference of every "
                                          f"error check in this line"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
