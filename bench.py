#!/usr/bin/env python3
"""Benchmark: pJDS SpMV y = A x on one GB300 (and replicas on N GPUs).

Workload (default): HMEp-like matrix after Sect. 1.3 of the paper, N = 6.2M,
~15 nonzeros per row (7 fixed diagonals at 0, ±1, ±64, ±4096 plus symmetric
random entries within |j-i| <= N/8), fp64 values, pJDS with b = 32. A step is
one y = A x in the original basis (y scattered through the permutation), with
the matrix and x resident in HBM. L2 is flushed (256 MB write) between timed
steps; each step is timed with CUDA events on the launching stream.

Throughput is reported in GB/s of algorithmic traffic, the paper's
code-balance view (Eq. 1 with ideal RHS reuse): 8+4 bytes per nonzero for
val+col, 8 bytes per element for x read once and y written once, 4 bytes per
row for the permutation: 12 nnz + 20 N bytes (fp64). GF/s = 2 nnz / time.

Side measurements in the same run: ELLPACK-R (the paper's baseline), pJDS with
fp32 and bf16 values, the permuted-basis product, and the end-to-end call from
pinned host memory. The CPU baseline is the fp64 oracle on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       (N > 1: launch with torch.distributed.run, one replica per GPU)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pJDS spMVM GB/s (% HBM roofline) & GF/s vs ELLPACK-R; mixed vs FP64 at stated err"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20

# DRAM bytes per launch of the timed pJDS kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), keyed by workload; valid only
# while the kernel's source (spmv_kernels.cuh) hashes to the recorded value and
# the launch configuration is the recorded one.
NCU_TRAFFIC = {
    # profiles/pjds_rows_kernel_hmep6.2M_f64.md section 2: 1,192,336,896 B read + 22,891,008 B written per launch
    ("hmep_f64_pjds", 6_200_000): {"bytes": 1_215_227_904, "src": "a48f132773d1b136",
                                   "cfg": {"rows_per_thread": 1, "threads_per_row": 1, "block_threads": 256,
                                           "unroll": 4, "staged": 0, "index64": 0, "tile_order": 1,
                                           "plan": -1}},
}


def code_hash(text: str) -> str:
    """Hash of C++ source without its // comments and blank lines, so a
    change to the comments alone keeps the hash."""
    lines = []
    for line in text.splitlines():
        code = line.split("//", 1)[0].rstrip()
        if code.strip():
            lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def kernel_source_hash() -> str:
    with open(os.path.join(ROOT, "paper_1112_5588_gb300", "csrc", "spmv_kernels.cuh")) as fh:
        return code_hash(fh.read())


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def alg_bytes(n_rows, n_cols, nnz, val_bytes, vec_bytes, scatter=True):
    """Algorithmic bytes of one y = A x (ideal x reuse, y written once)."""
    return nnz * (val_bytes + 4) + n_cols * vec_bytes + n_rows * vec_bytes + (4 * n_rows if scatter else 0)


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.index = gpu_id
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append((float(parts[1]), float(parts[2]), parts[4:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k + 1].lower() == "active"})
        loaded = [r[0] for r in rows if r[0] > 0.5 * r[1]] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


def gpu_id_for_smi(torch, dev) -> str:
    """nvidia-smi --id for the torch device: its UUID when torch exposes it."""
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev.index or 0)


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "case":
        return run_case(sys.argv[2:])
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=6_200_000, help="rows of the HMEp-like matrix")
    ap.add_argument("--seed", type=int, default=1234)
    ap.add_argument("--no-side", action="store_true", help="skip the side measurements")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--stencil-g", type=int, default=165, help="grid of the precision (stencil) workload")
    ap.add_argument("--lanczos-steps", type=int, default=200)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local_rank)


def synth_vector(n, seed):
    import synth
    return synth.vector(n, seed=seed)


def kernel_name(cfg: dict) -> str:
    """Readable name of the kernel pjds_spmv launches for a resolved config."""
    if cfg.get("plan") == 1:
        return "pjds_plan_kernel (per-tile mapping)"
    order = "tile order" if cfg.get("tile_order") == 1 else "sorted order"
    if cfg.get("threads_per_row", 1) > 1:
        return f"pjds_tpr_kernel T={cfg['threads_per_row']} U={cfg['unroll']} {cfg['block_threads']} thr/CTA, {order}"
    return (f"pjds_rows_kernel R={cfg['rows_per_thread']} U={cfg['unroll']} {cfg['block_threads']} thr/CTA, "
            f"{order}")


def workload_desc(n):
    return (f"HMEp-like (Holstein-Hubbard stand-in, Sect. 1.3): N={n}, diagonals 0,±1,±64,±4096 + symmetric "
            f"random entries within |j-i|<=N/8, ~15 nnz/row; pJDS b=32, fp64, original basis")


def build_matrix(args):
    import synth
    synth.build()
    A = synth.hmep_like(n=args.n, seed=args.seed)
    x = synth.vector(A.n_cols, seed=args.seed)
    return A, x


def run_reference(args, world, rank):
    """The oracle (fp64 CRS, OpenMP on the host cores) as the reference arm."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    A, x = build_matrix(args)
    cores = oracle.max_threads()
    for _ in range(args.warmup):
        oracle.crs_spmv(A, x)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.crs_spmv(A, x)
        times.append(time.perf_counter() - t0)
    nbytes = alg_bytes(A.n_rows, A.n_cols, A.nnz, 8, 8)
    t = sum(times)
    value = nbytes * args.steps / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(A.n_rows), "n_rows": A.n_rows, "nnz": A.nnz,
                       "parallelism": "host OpenMP"},
            "gflops": round(2 * A.nnz * args.steps / t / 1e9, 3),
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"full matrix, one CRS y=Ax per step ({A.nnz} nnz)"},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def time_launches(torch, launch, steps, warmup, flush):
    """Per-launch device time (s) with CUDA events on the current stream; L2
    flushed before every launch (outside the events)."""
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        launch()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        if flush is not None:
            flush.add_(1)
        ev[k][0].record(s)
        launch()
        ev[k][1].record(s)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) * 1e-3 for a, b in ev]


def run_ours(args, world, rank, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1112_5588_gb300 import pjds, replicas

    dist_on = world > 1
    if dist_on:
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    dev = torch.device("cuda", local_rank if dist_on else 0)
    torch.cuda.set_device(dev)

    t_gen = time.perf_counter()
    A, x = build_matrix(args)
    t_gen = time.perf_counter() - t_gen
    t_conv = time.perf_counter()
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64")
    t_conv = time.perf_counter() - t_conv
    D = H.to_device(dev)
    perm_host = H.perm.copy()
    n_stored = H.n_stored
    H.destroy()
    xt = torch.from_numpy(x).to(dev)
    y = torch.empty(A.n_rows, dtype=torch.float64, device=dev)
    y_pat = torch.empty_like(y)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    nbytes = alg_bytes(A.n_rows, A.n_cols, A.nnz, 8, 8)

    def barrier():
        if dist_on:
            dist.barrier()

    # ---------------- main timed region: K pJDS fp64 products
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_id_for_smi(torch, dev)) as clk:
        durs = time_launches(torch, lambda: pjds.pjds_spmv(D, xt, y), args.steps, args.warmup, flush)
        barrier()
        torch.cuda.synchronize()
    gpu_launches = args.steps
    # gather ceiling: the same traversal without the value stream (the
    # pattern product y = S x), timed the same way right after the product
    durs_pat = time_launches(torch, lambda: pjds.pjds_spmv_pattern(D, xt, y_pat), args.steps, args.warmup, flush)
    # replicas: units of all ranks over the slowest rank's time
    total_bytes, t_total, rate = replicas.aggregate(nbytes * args.steps, sum(durs), dev if dist_on else None)
    value = rate / 1e9
    per_launch = t_total / args.steps
    peak, peak_kind = hbm_peak()
    achieved = nbytes / (sum(durs) / len(durs)) / 1e9
    t_pat = sum(durs_pat) / len(durs_pat)
    ceiling_gbs = nbytes / t_pat / 1e9
    y_gpu = y.cpu().numpy()
    y_pat_gpu = y_pat.cpu().numpy()

    side = {}
    prec_gpu = None
    if not args.no_side:
        side = side_measurements(torch, pjds, A, x, D, xt, y, flush, args, dev, nbytes)
        prec_gpu = precision_gpu_leg(torch, pjds, args, dev, flush)
        side["side"]["batching"] = batching_leg(torch, pjds, args, dev, flush)
        side["side"]["small_case"] = small_case_leg(torch, pjds, args, dev, flush)
        side["side"]["tuning"] = tuning_leg(torch, pjds, args, dev)
        side["side"]["spread"] = spread_leg(torch, pjds, args, dev, flush)

    # ---------------- end to end through the C ABI from pinned host memory: K
    # products in one pjds_spmv_host_stream call (each step copies its x in
    # and its y out; the copies overlap the products), and K single
    # pjds_spmv_host calls (copy in, product, copy out, one after the other)
    # four different x vectors in turn, one host y per step; every step's y
    # is compared with the device product of its x afterwards
    n_x = 4
    xhs = [torch.from_numpy(synth_vector(A.n_cols, args.seed + 100 + v)).pin_memory() for v in range(n_x)]
    y_want = []
    for xv in xhs:
        pjds.pjds_spmv(D, xv.to(dev), y)
        y_want.append(y.cpu().numpy().copy())
    yhs = [torch.empty(A.n_rows, dtype=torch.float64).pin_memory() for _ in range(max(args.steps, args.warmup))]
    xd2 = [torch.empty_like(xt) for _ in range(2)]
    yd2 = [torch.empty_like(y) for _ in range(2)]
    # warm-up: every host buffer takes part in a copy once before the timed call
    n_w = max(args.warmup, len(yhs))
    pjds.pjds_spmv_host_stream(D, [xhs[v % n_x] for v in range(n_w)], [yhs[v % len(yhs)] for v in range(n_w)],
                               xd2, yd2)
    for yh in yhs:
        yh.fill_(float("nan"))
    barrier()
    t0 = time.perf_counter()
    pjds.pjds_spmv_host_stream(D, [xhs[v % n_x] for v in range(args.steps)], yhs[:args.steps], xd2, yd2)
    t_stream = time.perf_counter() - t0
    e2e_steps_ok = [bool(np.array_equal(yhs[v].numpy(), y_want[v % n_x])) for v in range(args.steps)]
    e2e_check = all(e2e_steps_ok)
    xh = xhs[0]
    _, _, e2e_rate = replicas.aggregate(nbytes * args.steps, t_stream, dev if dist_on else None)
    e2e_value = e2e_rate / 1e9
    for _ in range(args.warmup):
        pjds.pjds_spmv_host(D, xh, yhs[0], xd2[0], yd2[0])
    barrier()
    e2e_t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        pjds.pjds_spmv_host(D, xh, yhs[0], xd2[0], yd2[0])
        e2e_t.append(time.perf_counter() - t0)
    _, _, e2e_single_rate = replicas.aggregate(nbytes * args.steps, sum(e2e_t), dev if dist_on else None)

    if rank != 0:
        if dist_on:
            dist.destroy_process_group()
        return 0

    # ---------------- CPU baseline: the fp64 oracle on the host cores (rank 0, N = 1)
    cpu = None
    err = None
    pattern_exact = None
    if world == 1:
        import oracle
        oracle.build()
        cores = oracle.max_threads()
        y_ref = oracle.crs_spmv(A, x)
        reps, t_cpu = 0, 0.0
        while t_cpu < args.cpu_seconds and reps < 1000:
            t0 = time.perf_counter()
            y_ref = oracle.crs_spmv(A, x)
            t_cpu += time.perf_counter() - t0
            reps += 1
        cpu = {"value": round(nbytes * reps / t_cpu / 1e9, 3), "unit": "GB/s", "cores": cores, "kind": "oracle",
               "sample": f"full matrix ({A.nnz} nnz), {reps} CRS products in {t_cpu:.1f} s",
               "gflops": round(2 * A.nnz * reps / t_cpu / 1e9, 3)}
        # the same on one core (a few seconds)
        oracle.set_threads(1)
        reps1, t1 = 0, 0.0
        while t1 < max(1.0, args.cpu_seconds / 4) and reps1 < 100:
            t0 = time.perf_counter()
            oracle.crs_spmv(A, x)
            t1 += time.perf_counter() - t0
            reps1 += 1
        oracle.set_threads(cores)
        cpu["one_core"] = {"value": round(nbytes * reps1 / t1 / 1e9, 3), "unit": "GB/s",
                           "gflops": round(2 * A.nnz * reps1 / t1 / 1e9, 3), "products": reps1}
        absax = oracle.crs_absmv(A, x)
        err = float(np.max(np.abs(y_gpu - y_ref)) / np.max(absax))
        # the pattern product against the oracle's product with unit values
        ones = type(A)(A.n_rows, A.n_cols, A.row_ptr, A.col, np.ones(A.nnz))
        pattern_exact = bool(np.array_equal(y_pat_gpu, oracle.crs_spmv(ones, x)))
        if side:
            side["side"] = reduced_precision_oracle_checks(oracle, A, x, y_ref, absax, side["side"])
        if prec_gpu is not None:
            prec_gpu = precision_oracle_checks(oracle, prec_gpu)

    if side:
        side["side"].pop("_reduced_results", None)
    # the paper's model (Eqs. 1-2) with this GPU's measured bandwidths
    from paper_1112_5588_gb300 import perfmodel as pm
    n_nzr = A.nnz / A.n_rows
    t_single = nbytes / e2e_single_rate  # seconds per single-call product
    t_kernel = per_launch
    model = {"n_nzr": round(n_nzr, 3),
             "code_balance_bytes_per_flop": {"alpha_1_over_nnzr": round(pm.code_balance(1 / n_nzr, n_nzr), 3),
                                             "alpha_1": round(pm.code_balance(1.0, n_nzr), 3)},
             "roofline_gflops_at_peak": {"alpha_1_over_nnzr": round(pm.roofline_gflops(peak, 1 / n_nzr, n_nzr), 1),
                                         "alpha_1": round(pm.roofline_gflops(peak, 1.0, n_nzr), 1)},
             "achieved_gflops": round(2 * A.nnz / t_kernel / 1e9, 1),
             "t_mvm_model_us": round(pm.t_mvm(A.n_rows, n_nzr, 1 / n_nzr, peak * 1e9) * 1e6, 1),
             "t_mvm_measured_us": round(t_kernel * 1e6, 1),
             "t_pci_measured_us": round((t_single - t_kernel) * 1e6, 1),
             "b_pci_effective_gbs": round(16 * A.n_rows / (t_single - t_kernel) / 1e9, 1) if t_single > t_kernel else None}
    src_hash = kernel_source_hash()
    launched = pjds.pjds_spmv_resolve(D)
    tr = NCU_TRAFFIC.get(("hmep_f64_pjds", A.n_rows))
    traffic = tr["bytes"] if tr and tr["src"] == src_hash and tr["cfg"] == launched else None
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(per_launch * 1e3, 5),
        "ms_per_step_median": round(statistics.median(durs) * 1e3, 5), "ms_per_step_min": round(min(durs) * 1e3, 5),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(A.n_rows), "n_rows": A.n_rows, "nnz": A.nnz, "n_stored": n_stored,
                   "b": 32, "alg_bytes_per_step": nbytes, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU", "seed": args.seed},
        "gflops": round(value * 2 * A.nnz / nbytes, 3),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "kernel": kernel_name(launched),
                     "peak_kind": peak_kind,
                     "gather_ceiling_gbs": round(ceiling_gbs, 2),
                     "gather_ceiling_us": round(t_pat * 1e6, 2),
                     "frac_of_min_hbm_gather_ceiling": round(achieved / min(peak, ceiling_gbs), 4),
                     "gather_ceiling_kernel": "pattern product (pjds_spmv_pattern): the same traversal, column "
                                              "stream, x gathers and y stores, no value stream",
                     "gather_ceiling_bitwise_equals_oracle": pattern_exact},
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 3), "unit": "GB/s", "h2d_bytes_per_step": 8 * A.n_cols,
                "d2h_bytes_per_step": 8 * A.n_rows, "api": "pjds_spmv_host_stream (K products, copies overlapped)",
                "result_equals_device_product": e2e_check,
                "steps_checked": len(e2e_steps_ok), "distinct_x": n_x,
                "single_call_value": round(e2e_single_rate / 1e9, 3),
                "single_call_api": "pjds_spmv_host (copy in, product, copy out per call)"},
        "gpu_launches": gpu_launches,
        "perf_model": model,
        "clocks": clk.summary(),
        "error_fp64_normwise": err,
        "setup_s": {"generate": round(t_gen, 2), "pjds_create": round(t_conv, 2)},
        "kernel_src": src_hash,
        "kernel_cfg": launched,
        **side,
        "precision": prec_gpu["report"] if prec_gpu else None,
    }
    print(json.dumps(line), flush=True)
    if dist_on:
        dist.destroy_process_group()
    return 0


def side_measurements(torch, pjds, A, x, D, xt, y, flush, args, dev, nbytes):
    """ELLPACK-R, reduced precision, permuted basis and an L2-warm figure."""
    out = {}
    K, W = max(5, args.steps // 2), 3
    med = statistics.median

    t = med(time_launches(torch, lambda: pjds.pjds_spmv(D, xt, y), K, W, None))
    out["pjds_f64_l2_warm"] = {"gbs": round(nbytes / t / 1e9, 1), "us": round(t * 1e6, 2)}

    E = pjds.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype="f64")
    ell_stored = E.n_stored
    ED = E.to_device(dev)
    E.destroy()
    ye = torch.empty_like(y)
    t_e = med(time_launches(torch, lambda: pjds.ellr_spmv(ED, xt, ye), K, W, flush))
    t_p = med(time_launches(torch, lambda: pjds.pjds_spmv(D, xt, y), K, W, flush))
    ell_bytes = alg_bytes(A.n_rows, A.n_cols, A.nnz, 8, 8, scatter=False) + 4 * A.n_rows
    out["ellr_f64"] = {"gbs": round(ell_bytes / t_e / 1e9, 1), "gflops": round(2 * A.nnz / t_e / 1e9, 2),
                       "us": round(t_e * 1e6, 2), "n_stored": ell_stored,
                       "bit_identical_to_pjds": bool(torch.equal(ye, y))}
    out["pjds_f64_median"] = {"gbs": round(nbytes / t_p / 1e9, 1), "gflops": round(2 * A.nnz / t_p / 1e9, 2),
                              "us": round(t_p * 1e6, 2)}
    out["pjds_vs_ellr_speed"] = round(t_e / t_p, 3)
    out["pjds_data_reduction_vs_ellpack"] = round(1 - D.n_stored / ell_stored, 4)
    del ED, ye

    peak = hbm_peak()[0]
    reduced = {}
    for dt in ("f32", "bf16"):
        Hr = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dt)
        Dr = Hr.to_device(dev)
        Hr.destroy()
        xr = xt.float()
        yr = torch.empty(A.n_rows, dtype=torch.float32, device=dev)
        tr = med(time_launches(torch, lambda: pjds.pjds_spmv(Dr, xr, yr), K, W, flush))
        vb = 4 if dt == "f32" else 2
        b_r = alg_bytes(A.n_rows, A.n_cols, A.nnz, vb, 4)
        out[f"pjds_{dt}"] = {"gbs": round(b_r / tr / 1e9, 1), "gflops": round(2 * A.nnz / tr / 1e9, 2),
                             "us": round(tr * 1e6, 2), "frac_of_hbm": round(b_r / tr / 1e9 / peak, 4),
                             "alg_bytes": b_r, "speedup_vs_f64": round(t_p / tr, 3),
                             "kernel": kernel_name(pjds.pjds_spmv_resolve(Dr))}
        reduced[f"pjds_{dt}"] = (dt, yr.cpu().numpy().copy())
        # its gather ceiling: the same launch without the value stream
        yp = torch.empty_like(yr)
        tpat = med(time_launches(torch, lambda: pjds.pjds_spmv_pattern(Dr, xr, yp), K, W, flush))
        out[f"pjds_{dt}"]["gather_ceiling_us"] = round(tpat * 1e6, 2)
        out[f"pjds_{dt}"]["frac_of_min_hbm_gather_ceiling"] = round(
            (b_r / tr) / min(peak * 1e9, b_r / tpat), 4)
        del Dr, xr, yr
    # ELLPACK-R with fp32 values on the same matrix (Table 1's single-precision row)
    E32 = pjds.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype="f32")
    ED32 = E32.to_device(dev)
    E32.destroy()
    x32 = xt.float()
    y32 = torch.empty(A.n_rows, dtype=torch.float32, device=dev)
    t_e32 = med(time_launches(torch, lambda: pjds.ellr_spmv(ED32, x32, y32), K, W, flush))
    b_e32 = alg_bytes(A.n_rows, A.n_cols, A.nnz, 4, 4, scatter=False) + 4 * A.n_rows
    out["ellr_f32"] = {"gbs": round(b_e32 / t_e32 / 1e9, 1), "gflops": round(2 * A.nnz / t_e32 / 1e9, 2),
                       "us": round(t_e32 * 1e6, 2), "frac_of_hbm": round(b_e32 / t_e32 / 1e9 / peak, 4),
                       "pjds_f32_vs_ellr_f32_speed": round(t_e32 * 1e6 / out["pjds_f32"]["us"], 3)}
    reduced["ellr_f32"] = ("f32", y32.cpu().numpy().copy())
    del ED32, x32, y32
    out["_reduced_results"] = reduced

    Hp = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64", permute_cols=True)
    Dp = Hp.to_device(dev)
    Hp.destroy()
    xp = torch.empty_like(xt)
    yp = torch.empty_like(y)
    pjds.pjds_permute(Dp, xt, xp)
    t_pm = med(time_launches(torch, lambda: pjds.pjds_spmv(Dp, xp, yp), K, W, flush))
    b_pm = alg_bytes(A.n_rows, A.n_cols, A.nnz, 8, 8, scatter=False)
    out["pjds_f64_permuted_basis"] = {"gbs": round(b_pm / t_pm / 1e9, 1), "us": round(t_pm * 1e6, 2)}
    del Dp, xp, yp

    for cfg in ({"rows_per_thread": 2}, {"rows_per_thread": 4}, {"threads_per_row": 2}, {"block_threads": 512},
                {"block_threads": 128}, {"staged": 1}, {"tile_order": -1}):
        tc = med(time_launches(torch, lambda: pjds.pjds_spmv_cfg(D, xt, y, **cfg), K, W, flush))
        key = "cfg_" + "_".join(f"{k}{v}" for k, v in cfg.items())
        out[key] = {"gbs": round(nbytes / tc / 1e9, 1), "us": round(tc * 1e6, 2)}
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return {"side": out}


def small_case_leg(torch, pjds, args, dev, flush):
    """The banded N = 20,000 case (~451k nonzeros, 5.8 MB: L2-resident and
    launch bound): per-launch time with L2 warm and flushed, and 1000
    products captured in one CUDA graph, for pJDS and ELLPACK-R."""
    med = statistics.median
    import synth
    A = synth.banded_uniform(n=20_000, seed=args.seed)
    x = torch.from_numpy(synth.vector(A.n_cols, seed=args.seed)).to(dev)
    nbytes = alg_bytes(A.n_rows, A.n_cols, A.nnz, 8, 8)
    ell_bytes = alg_bytes(A.n_rows, A.n_cols, A.nnz, 8, 8, scatter=False) + 4 * A.n_rows
    out = {"matrix": f"banded N={A.n_rows} nnz={A.nnz}", "alg_bytes": nbytes}
    for fmt in ("pjds", "ellr"):
        H = (pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64") if fmt == "pjds"
             else pjds.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype="f64"))
        D = H.to_device(dev)
        H.destroy()
        y = torch.empty(A.n_rows, dtype=torch.float64, device=dev)
        run = (lambda: pjds.pjds_spmv(D, x, y)) if fmt == "pjds" else (lambda: pjds.ellr_spmv(D, x, y))
        nb = nbytes if fmt == "pjds" else ell_bytes
        hot = med(time_launches(torch, run, 200, 10, None))
        cold = med(time_launches(torch, run, 50, 3, flush))
        y_ref = y.clone()
        side_stream = torch.cuda.Stream(device=dev)
        side_stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side_stream):
            run()
        torch.cuda.current_stream().wait_stream(side_stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(1000):
                run()
        y.zero_()
        g.replay()
        torch.cuda.synchronize()
        same = bool(torch.equal(y, y_ref))
        reps = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            reps.append(e0.elapsed_time(e1) * 1e-3 / 1000)
        t_g = med(reps)
        out[fmt] = {"hot_us": round(hot * 1e6, 2), "hot_gbs": round(nb / hot / 1e9, 1),
                    "cold_us": round(cold * 1e6, 2), "cold_gbs": round(nb / cold / 1e9, 1),
                    "graph1000_us_per_product": round(t_g * 1e6, 3), "graph1000_gbs": round(nb / t_g / 1e9, 1),
                    "graph_result_bit_identical": same}
        del g, D, y
    torch.cuda.synchronize()
    return out


def precision_gpu_leg(torch, pjds, args, dev, flush):
    """Mixed precision on the FEM-like stencil (27-point, 165^3, 10% of pairs
    dropped, SPD): pJDS products in fp64/fp32/bf16, 300-step CG in fp64 vs
    fp32/bf16 inner steps with fp64 residual refinement, and 200 Lanczos steps
    in fp64 vs fp32 with an fp64-refined Ritz pair. Everything runs in the
    permuted basis. Results are checked against the oracle in the CPU leg."""
    import synth
    from paper_1112_5588_gb300 import krylov
    S = synth.stencil27(g=args.stencil_g, p_drop=0.1, seed=args.seed)
    n = S.n_rows
    rep = {"matrix": f"stencil27 g={args.stencil_g} (N={n}, nnz={S.nnz}), SPD, permuted basis"}
    devs, perm = {}, None
    for dt in ("f64", "f32", "bf16"):
        H = pjds.pjds_create(S.n_rows, S.n_cols, S.row_ptr, S.col, S.val, b=32, dtype=dt, permute_cols=True)
        if perm is None:
            perm = H.perm.copy()
        devs[dt] = H.to_device(dev)
        H.destroy()
    # kernel-level: the product in each precision
    xs = torch.from_numpy(synth.vector(n, seed=args.seed)[perm]).to(dev)
    for dt, D in devs.items():
        xv = xs.to(D.vec_dtype)
        yv = torch.empty(n, dtype=D.vec_dtype, device=dev)
        vb = {"f64": 8, "f32": 4, "bf16": 2}[dt]
        xb = 8 if dt == "f64" else 4
        nb = alg_bytes(n, n, S.nnz, vb, xb, scatter=False)
        for tag, kw in (("", {}), ("_staged", {"staged": 1}), ("_sorted_order", {"tile_order": -1})):
            t = statistics.median(time_launches(torch, lambda: pjds.pjds_spmv_cfg(D, xv, yv, **kw), 10, 3, flush))
            rep[f"spmv_{dt}{tag}"] = {"gbs": round(nb / t / 1e9, 1), "us": round(t * 1e6, 2),
                                      "frac_of_hbm": round(nb / t / 1e9 / hbm_peak()[0], 4)}
            if not tag:  # the gather ceiling of the default launch
                yq = torch.empty_like(yv)
                tq = statistics.median(time_launches(torch, lambda: pjds.pjds_spmv_pattern(D, xv, yq), 10, 3, flush))
                rep[f"spmv_{dt}"]["gather_ceiling_us"] = round(tq * 1e6, 2)
                rep[f"spmv_{dt}"]["frac_of_min_hbm_gather_ceiling"] = round(
                    (nb / t) / min(hbm_peak()[0] * 1e9, nb / tq), 4)
    # pJDS in the original basis against ELLPACK-R on the same matrix (fp64)
    Ho = pjds.pjds_create(S.n_rows, S.n_cols, S.row_ptr, S.col, S.val, b=32, dtype="f64")
    Do = Ho.to_device(dev)
    Ho.destroy()
    Eo = pjds.ellr_create(S.n_rows, S.n_cols, S.row_ptr, S.col, S.val, dtype="f64")
    ell_stored = Eo.n_stored
    ED = Eo.to_device(dev)
    Eo.destroy()
    xo = torch.from_numpy(synth.vector(n, seed=args.seed)).to(dev)
    yo, ye = torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.float64, device=dev)
    t_po = statistics.median(time_launches(torch, lambda: pjds.pjds_spmv(Do, xo, yo), 10, 3, flush))
    t_eo = statistics.median(time_launches(torch, lambda: pjds.ellr_spmv(ED, xo, ye), 10, 3, flush))
    nb_o = alg_bytes(n, n, S.nnz, 8, 8)
    nb_e = alg_bytes(n, n, S.nnz, 8, 8, scatter=False) + 4 * n
    rep["original_basis_f64"] = {"pjds_gbs": round(nb_o / t_po / 1e9, 1), "pjds_us": round(t_po * 1e6, 2),
                                 "ellr_gbs": round(nb_e / t_eo / 1e9, 1), "ellr_us": round(t_eo * 1e6, 2),
                                 "pjds_vs_ellr_speed": round(t_eo / t_po, 3),
                                 "pjds_data_reduction_vs_ellpack": round(1 - Do.n_stored / ell_stored, 4),
                                 "bit_identical": bool(torch.equal(yo, ye)) if not pjds.pjds_spmv_resolve(Do)[
                                     "threads_per_row"] > 1 else None}
    del Do, ED, xo, yo, ye
    b = synth.vector(n, seed=args.seed + 1)
    bp = torch.from_numpy(b[perm]).to(dev)
    runs = {"cg_fp64": (None, 1, 300), "cg_f32_refined": ("f32", 6, 50), "cg_bf16_refined": ("bf16", 12, 25)}
    xs_out = {}
    for name, (lo, mo, inner) in runs.items():
        Dlo = devs[lo] if lo else None
        work = torch.empty(krylov.cg_workspace_bytes(n, devs["f64"].n_pad, 1 if lo else 0), dtype=torch.uint8,
                           device=dev)
        xp = torch.zeros_like(bp)
        krylov.cg_solve(devs["f64"], Dlo, bp, xp, max_outer=mo, inner_iters=inner, work=work)  # warm-up
        xp.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = krylov.cg_solve(devs["f64"], Dlo, bp, xp, max_outer=mo, inner_iters=inner, work=work)
        torch.cuda.synchronize()
        dt_s = time.perf_counter() - t0
        x = np.empty(n)
        x[perm] = xp.cpu().numpy()
        xs_out[name] = x
        rep[name] = {"outer": r["outer"], "inner_steps": r["inner_total"], "ms": round(dt_s * 1e3, 2),
                     "rel_residual_gpu": r["rel_residual"]}
    # Lanczos: 200 steps fp64 vs fp32 + fp64 Ritz refinement
    v0 = synth.vector(n, seed=args.seed + 2)[perm]
    lan, ys = {}, {}
    for dt in ("f64", "f32"):
        D = devs[dt]
        v0t = torch.from_numpy(v0).to(dev, D.vec_dtype)
        krylov.lanczos(D, v0t, 20)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        alpha, beta, V = krylov.lanczos(D, v0t, args.lanczos_steps, keep_basis=True)
        torch.cuda.synchronize()
        t_l = time.perf_counter() - t0
        th, svec = krylov.tridiag_extreme(alpha, beta)
        yv, th_ref, resid = krylov.ritz_refine(devs["f64"], V, svec)
        y_o = np.empty(n)
        y_o[perm] = yv.cpu().numpy()
        lan[dt] = {"ms_recurrence": round(t_l * 1e3, 2), "theta_T": th, "theta_refined_fp64": th_ref,
                   "rel_residual_gpu": resid}
        ys[dt] = y_o
        del V
        torch.cuda.empty_cache()
    rep["lanczos_steps"] = args.lanczos_steps
    rep["lanczos"] = lan
    if "f64" in lan and "f32" in lan:
        rep["theta_refined_f32_vs_f64_rel"] = abs(lan["f32"]["theta_refined_fp64"] -
                                                  lan["f64"]["theta_refined_fp64"]) / abs(lan["f64"]["theta_refined_fp64"])
    # the fp64 CG once more with the tiles in sorted order (no traversal table)
    Hn = pjds.pjds_create(S.n_rows, S.n_cols, S.row_ptr, S.col, S.val, b=32, dtype="f64", permute_cols=True)
    Dn = Hn.to_device(dev, tile_order=False)
    Hn.destroy()
    xp = torch.zeros_like(bp)
    krylov.cg_solve(Dn, None, bp, xp, max_outer=1, inner_iters=300)
    xp.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    krylov.cg_solve(Dn, None, bp, xp, max_outer=1, inner_iters=300)
    torch.cuda.synchronize()
    rep["cg_fp64_sorted_order_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
    del Dn, xp
    f64 = rep["cg_fp64"]["ms"]
    for name in ("cg_f32_refined", "cg_bf16_refined"):
        rep[name]["speedup_vs_fp64"] = round(f64 / rep[name]["ms"], 3)
    del devs
    torch.cuda.empty_cache()
    return {"S": S, "b": b, "x": xs_out, "ys": ys, "report": rep}


def batching_leg(torch, pjds, args, dev, flush):
    """Block product with k right-hand sides on the DLR-like matrix (dense
    4x4 blocks, 36 block columns within +-5%: N = 280k, 144 nonzeros/row,
    fp32 values and vectors), and 64 uneven matrices (N log-uniform in
    [10k, 500k], Zipf(2) row lengths capped at 512, fp64) in one persistent
    launch replayed as a CUDA graph vs one launch per matrix."""
    import synth
    from paper_1112_5588_gb300 import batch
    out = {}
    A = synth.block_dense(n_brow=70_000, bs=4, nb=36, frac=0.05, seed=args.seed)
    H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f32")
    D = H.to_device(dev)
    H.destroy()
    spmm = {"matrix": f"DLR-like N={A.n_rows} nnz={A.nnz}", "dtype": "f32"}
    peak = hbm_peak()[0]
    for k in (1, 4, 8, 16, 32):
        X = torch.rand(A.n_cols, k, device=dev)
        Y = torch.empty(A.n_rows, k, device=dev)
        t = statistics.median(time_launches(torch, lambda: batch.spmm(D, X, Y), 10, 3, flush))
        nb = A.nnz * 8 + 4 * k * (A.n_cols + A.n_rows) + 4 * A.n_rows
        spmm[f"k{k}"] = {"us": round(t * 1e6, 2), "gbs": round(nb / t / 1e9, 1),
                         "frac_of_hbm": round(nb / t / 1e9 / peak, 4),
                         "gflops": round(2 * A.nnz * k / t / 1e9, 1),
                         "us_per_rhs": round(t * 1e6 / k, 2)}
        # the gather ceiling: the same launch without the value stream (k rows of X
        # gathered per entry, 4 k bytes each, through L1/L2)
        if k == 1:
            tp = statistics.median(time_launches(torch, lambda: pjds.pjds_spmv_pattern(D, X.view(-1), Y.view(-1)),
                                                 10, 3, flush))
        else:
            tp = statistics.median(time_launches(torch, lambda: batch.spmm_pattern(D, X, Y), 10, 3, flush))
        spmm[f"k{k}"]["gather_ceiling_us"] = round(tp * 1e6, 2)
        spmm[f"k{k}"]["frac_of_gather_ceiling"] = round(tp / t, 4)
        spmm[f"k{k}"]["gathered_bytes_per_entry"] = 4 * k
    spmm["ceiling_note"] = ("frac_of_gather_ceiling = pattern-product time / product time: the pattern product "
                            "(pjds_spmm_pattern) is the same launch without reading the values")
    spmm["pair_share"] = D.pair_share
    # bf16 values (fp32 vectors): one thread per pair of rows sharing their columns from k = 8
    Hb = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="bf16")
    Db = Hb.to_device(dev)
    Hb.destroy()
    spmm["bf16"] = {}
    for k in (8, 32):
        X = torch.rand(A.n_cols, k, device=dev)
        Y = torch.empty(A.n_rows, k, device=dev)
        t = statistics.median(time_launches(torch, lambda: batch.spmm(Db, X, Y), 10, 3, flush))
        tp = statistics.median(time_launches(torch, lambda: batch.spmm_pattern(Db, X, Y), 10, 3, flush))
        nb = A.nnz * 6 + 4 * k * (A.n_cols + A.n_rows) + 4 * A.n_rows
        spmm["bf16"][f"k{k}"] = {"us": round(t * 1e6, 2), "gbs": round(nb / t / 1e9, 1),
                                 "gflops": round(2 * A.nnz * k / t / 1e9, 1),
                                 "gather_ceiling_us": round(tp * 1e6, 2), "frac_of_gather_ceiling": round(tp / t, 4)}
    out["spmm"] = spmm
    del D, Db
    rng = np.random.default_rng(args.seed)
    sizes = np.exp(rng.uniform(np.log(10_000), np.log(500_000), 64)).astype(int)
    from paper_1112_5588_gb300 import learned
    model = learned.load()
    cands = [{"b": 32, "dtype": "f64", "rows_per_thread": 0, "threads_per_row": t, "block_threads": 0, "unroll": 0,
              "tile_order": -1} for t in (1, 2, 4, 8)]
    devs, xs, ys, nnz, nbytes, tuned = [], [], [], 0, 0, []
    for m, n in enumerate(sizes):
        M = synth.zipf_rows(int(n), s=2.0, len_max=512, seed=args.seed + m)
        tuned.append(learned.choose(M, cands, model=model)[1]["threads_per_row"])
        Hm = pjds.pjds_create(M.n_rows, M.n_cols, M.row_ptr, M.col, M.val, b=32, dtype="f64")
        devs.append(Hm.to_device(dev))
        Hm.destroy()
        xs.append(torch.from_numpy(synth.vector(M.n_cols, seed=m)).to(dev))
        ys.append(torch.empty(M.n_rows, dtype=torch.float64, device=dev))
        nnz += M.nnz
        nbytes += alg_bytes(M.n_rows, M.n_cols, M.nnz, 8, 8)
    B = batch.Batch(devs, xs, ys)
    t_batch = statistics.median(time_launches(torch, lambda: B.run(use_graph=True), 10, 3, flush))
    t_batch_pat = statistics.median(time_launches(torch, B.run_pattern, 10, 3, flush))
    t_batch_direct = statistics.median(time_launches(torch, lambda: B.run(use_graph=False), 10, 3, flush))

    def separate():
        for Dm, xm, ym in zip(devs, xs, ys):
            pjds.pjds_spmv(Dm, xm, ym)
    t_sep = statistics.median(time_launches(torch, separate, 10, 3, flush))
    # the same 64 launches recorded once into a CUDA graph (no host overhead)
    g = torch.cuda.CUDAGraph()
    side_stream = torch.cuda.Stream()
    side_stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side_stream):
        separate()
    torch.cuda.current_stream().wait_stream(side_stream)
    with torch.cuda.graph(g):
        separate()
    t_sep_graph = statistics.median(time_launches(torch, g.replay, 10, 3, flush))
    out["multi_matrix"] = {"n_mats": 64, "total_rows": int(sizes.sum()), "nnz": int(nnz), **B.info(),
                           "persistent_graph_us": round(t_batch * 1e6, 2),
                           "persistent_graph_gbs": round(nbytes / t_batch / 1e9, 1),
                           "frac_of_hbm": round(nbytes / t_batch / 1e9 / hbm_peak()[0], 4),
                           "persistent_direct_us": round(t_batch_direct * 1e6, 2),
                           "gather_ceiling_us": round(t_batch_pat * 1e6, 2),
                           "frac_of_gather_ceiling": round(t_batch_pat / t_batch_direct, 4),
                           "separate_launches_us": round(t_sep * 1e6, 2),
                           "separate_launches_graph_us": round(t_sep_graph * 1e6, 2),
                           "speedup_vs_separate": round(t_sep / t_batch, 3),
                           "speedup_vs_separate_graph": round(t_sep_graph / t_batch, 3)}
    B.destroy()
    # tiles with the learned tuner's threads per row for each matrix
    Bt = batch.Batch(devs, xs, ys, lanes=tuned)
    t_tuned = statistics.median(time_launches(torch, lambda: Bt.run(use_graph=True), 10, 3, flush))
    out["multi_matrix"]["tuned_lanes_graph_us"] = round(t_tuned * 1e6, 2)
    out["multi_matrix"]["tuned_lanes_histogram"] = {str(t): int(sum(1 for v in tuned if v == t)) for t in (1, 2, 4, 8)}
    Bt.destroy()
    # the batch's own autotuner: exhaustive sweep of block-length tile rules
    best, timings = batch.tune_rule(devs, xs, ys, reps=5)
    Br = batch.Batch(devs, xs, ys, rule=best)
    t_rule = statistics.median(time_launches(torch, lambda: Br.run(use_graph=True), 10, 3, flush))
    Br.destroy()
    out["multi_matrix"]["rule_sweep_us"] = {",".join("-" if v == batch.NEVER else str(v) for v in r): round(u, 1)
                                            for r, u in timings}
    out["multi_matrix"]["tuned_rule"] = list(best)
    out["multi_matrix"]["tuned_rule_graph_us"] = round(t_rule * 1e6, 2)
    del devs, xs, ys
    torch.cuda.empty_cache()
    return out


def tuning_leg(torch, pjds, args, dev):
    """The candidate sweep on the DLR-like matrix (long rows, fp32): the
    exhaustive autotuner's 36 candidates (b in 32..256, T in 1..8, sorted or
    table tile order, the per-tile mapping; rows per thread left to the
    default rule) with the L2 flushed between runs, against the paper's
    mapping (b = 32, one row per thread, sorted order, timed in the same
    sweep), the library's default and the learned picker (pjds_tune_pick: the
    model inside its training range, the sweep outside it)."""
    import synth
    from paper_1112_5588_gb300 import learned, tune, tuner_data
    A = synth.block_dense(n_brow=70_000, bs=4, nb=36, frac=0.05, seed=args.seed)
    cands = tune.default_space(("f32",))
    # the paper's mapping, timed in the same sweep: b = 32, one row per thread, sorted order
    paper_cand = {"b": 32, "dtype": "f32", "rows_per_thread": 1, "threads_per_row": 1, "tile_order": -1, "plan": -1}
    entries, best = tune.sweep(A, cands + [paper_cand], reps=5)
    paper = round(entries[-1]["us"], 2)
    entries = entries[:-1]
    best = min((k for k, e in enumerate(entries) if e["status"] == 0), key=lambda k: entries[k]["us"])
    us = {tune.cand_key(c): round(e["us"], 2) for c, e in zip(cands, entries) if e["status"] == 0}
    pick = learned.pick(A, "f32")
    t_pick = us[tune.cand_key(pick)]
    D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f32").to_device(dev)
    x = torch.rand(A.n_cols, device=dev)
    y = torch.empty(A.n_rows, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    t_def = statistics.median(time_launches(torch, lambda: pjds.pjds_spmv(D, x, y), 10, 3, flush)) * 1e6
    k_def = tuner_data.default_index(cands, A.n_rows, A.nnz, int(np.diff(A.row_ptr).max()), "f32")
    best_key = tune.cand_key(cands[best])
    # candidates leave rows per thread to the default rule: on this block-structured
    # matrix (pair_share 1000) the one-thread-per-row candidates pair rows like the default
    rpt = {tune.cand_key(c): e["rows_per_thread"] for c, e in zip(cands, entries) if e["status"] == 0}
    return {"matrix": f"DLR-like N={A.n_rows} nnz={A.nnz} (144/row), fp32", "sweep_us": us,
            "sweep_rows_per_thread": rpt, "best": best_key, "best_us": us[best_key], "paper_mapping_us": paper,
            "default_mapping": pjds.pjds_spmv_resolve(D), "pair_share": D.pair_share, "default_us": round(t_def, 2),
            "default_vs_sweep_best": round(t_def / us[best_key] - 1, 4),
            "default_in_sweep": tune.cand_key(cands[k_def]) if k_def >= 0 else None,
            "default_regret_in_sweep": round(us[tune.cand_key(cands[k_def])] / us[best_key] - 1, 4)
            if k_def >= 0 else None,
            "picker": {"choice": tune.cand_key(pick), "source": pick["source"], "features_outside": pick["n_outside"],
                       "us": t_pick, "live_regret": round(t_pick / us[best_key] - 1, 4)},
            "best_speedup_over_paper_mapping": round(paper / us[best_key], 3)}


def spread_leg(torch, pjds, args, dev, flush):
    """Widely spread row lengths (sAMG-like: Zipf s = 2, rows of 1 to 512
    entries, 1M rows; fp64 and fp32): the per-tile mapping pjds_spmv takes
    for such a matrix against every uniform threads-per-row count, L2 flushed
    before each launch; and the learned picker's choice against the
    exhaustive sweep of the candidate space."""
    med = statistics.median
    import synth
    from paper_1112_5588_gb300 import learned, tune, tuner_data
    A = synth.zipf_rows(1_000_000, s=2.0, len_max=512, seed=args.seed)
    lens = np.diff(A.row_ptr)
    out = {"matrix": f"Zipf s=2 N={A.n_rows} nnz={A.nnz} (rows up to {int(lens.max())}, mean {lens.mean():.2f})"}
    for dt, vb, xb in (("f64", 8, 8), ("f32", 4, 4)):
        H = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=dt)
        D = H.to_device(dev)
        n_plan = H.n_plan
        H.destroy()
        x = torch.from_numpy(synth.vector(A.n_cols, seed=args.seed)).to(dev, D.vec_dtype)
        y = torch.empty(A.n_rows, dtype=D.vec_dtype, device=dev)
        nb = alg_bytes(A.n_rows, A.n_cols, A.nnz, vb, xb)
        t_def = med(time_launches(torch, lambda: pjds.pjds_spmv(D, x, y), 20, 3, flush))
        t_hot = med(time_launches(torch, lambda: pjds.pjds_spmv(D, x, y), 20, 3, None))
        yp = torch.empty_like(y)
        t_pat = med(time_launches(torch, lambda: pjds.pjds_spmv_pattern(D, x, yp), 20, 3, flush))
        uni = {t: med(time_launches(torch, lambda: pjds.pjds_spmv_cfg(D, x, y, threads_per_row=t, plan=-1), 20, 3, flush))
               for t in (1, 2, 4, 8)}
        best = min(uni, key=uni.get)
        out[dt] = {"default_uses_plan": pjds.pjds_spmv_resolve(D)["plan"] == 1, "plan_tiles": n_plan,
                   "default_us": round(t_def * 1e6, 2), "default_gbs": round(nb / t_def / 1e9, 1),
                   "working_set_mb": round(nb / 1e6, 1), "l2_mb": 129,
                   "default_l2_warm_us": round(t_hot * 1e6, 2),
                   "gather_ceiling_us": round(t_pat * 1e6, 2), "frac_of_gather_ceiling": round(t_pat / t_def, 4),
                   "bound": ("L2-resident working set: measured cold (L2 flushed before each launch) and warm; "
                             "a warm time near the cold one means latency, not DRAM, sets it"),
                   "uniform_us": {f"T{t}": round(v * 1e6, 2) for t, v in uni.items()},
                   "best_uniform": f"T{best}", "speedup_vs_best_uniform": round(uni[best] / t_def, 3)}
        # the learned picker against the exhaustive sweep of the 36 candidates (one sweep, L2 flushed)
        cands = tune.default_space((dt,))
        entries, k_best = tune.sweep(A, cands, reps=5)
        pick = learned.pick(A, dt)
        k_def = tuner_data.default_index(cands, A.n_rows, A.nnz, int(lens.max()), dt)
        t_best = entries[k_best]["us"]
        out[dt]["sweep_best"] = tune.cand_key(cands[k_best])
        out[dt]["sweep_best_us"] = round(t_best, 2)
        out[dt]["picker"] = {"choice": tune.cand_key(pick), "source": pick["source"],
                             "us": round(entries[pick["index"]]["us"], 2),
                             "live_regret": round(entries[pick["index"]]["us"] / t_best - 1, 4)}
        out[dt]["default_regret_in_sweep"] = round(entries[k_def]["us"] / t_best - 1, 4) if k_def >= 0 else None
        del D, x, y
    # against ELLPACK-R (Table 1's comparison on spread row lengths, sAMG-like): a
    # 200k-row Zipf matrix, fp64; ELLPACK-R pads every row to the longest
    Z = synth.zipf_rows(200_000, s=2.0, len_max=512, seed=args.seed + 1)
    Hz = pjds.pjds_create(Z.n_rows, Z.n_cols, Z.row_ptr, Z.col, Z.val, b=32)
    Ez = pjds.ellr_create(Z.n_rows, Z.n_cols, Z.row_ptr, Z.col, Z.val)
    stored = {"pjds": int(Hz.n_stored), "ellr": int(Ez.n_stored)}
    Dz, Dez = Hz.to_device(dev), Ez.to_device(dev)
    Hz.destroy()
    Ez.destroy()
    x = torch.from_numpy(synth.vector(Z.n_cols, seed=args.seed)).to(dev)
    y, ye = torch.empty(Z.n_rows, dtype=torch.float64, device=dev), torch.empty(Z.n_rows, dtype=torch.float64, device=dev)
    t_p = statistics.median(time_launches(torch, lambda: pjds.pjds_spmv(Dz, x, y), 10, 3, flush))
    t_e = statistics.median(time_launches(torch, lambda: pjds.ellr_spmv(Dez, x, ye), 10, 3, flush))
    pjds.pjds_spmv_cfg(Dz, x, y, threads_per_row=1, rows_per_thread=1, tile_order=-1)
    torch.cuda.synchronize()
    out["vs_ellpack_r"] = {"matrix": f"Zipf s=2 N={Z.n_rows} nnz={Z.nnz} (rows up to {int(np.diff(Z.row_ptr).max())}), fp64",
                           "pjds_us": round(t_p * 1e6, 2), "ellr_us": round(t_e * 1e6, 2),
                           "pjds_vs_ellr_speed": round(t_e / t_p, 3), "stored": stored,
                           "pjds_data_reduction_vs_ellpack": round(1 - stored["pjds"] / stored["ellr"], 4),
                           "bit_identical_one_thread_per_row": bool(torch.equal(y, ye))}
    del Dz, Dez, x, y, ye
    torch.cuda.synchronize()
    return out


def reduced_precision_oracle_checks(oracle, A, x, y_ref, absax, side):
    """Errors of the fp32 / bf16 products against the fp64 oracle: normwise
    against the exact (fp64) matrix, and element by element against the
    oracle's product of the rounded values the kernel holds, within the
    fp32-accumulation bound of the parity tests."""
    from tests import parity
    reduced = side.pop("_reduced_results", {})
    lens = np.diff(A.row_ptr)
    x32 = x.astype(np.float32).astype(np.float64)
    for key, (dt, yv) in reduced.items():
        vals = oracle.round_f32(A.val) if dt == "f32" else oracle.round_bf16(A.val)
        Ar = type(A)(A.n_rows, A.n_cols, A.row_ptr, A.col, vals)
        y_r = oracle.crs_spmv(Ar, x32)
        r = parity.check_fp32(yv, y_r, oracle.crs_absmv(Ar, x32), lens)
        side[key]["error_vs_fp64_oracle"] = {
            "normwise_vs_exact_matrix": float(np.max(np.abs(yv - y_ref)) / np.max(absax)),
            "normwise_vs_rounded_matrix": r["normwise"],
            "elementwise_bound_vs_rounded_matrix_ok": r["ok"], "elements_outside_bound": r["n_bad"]}
    return side


def precision_oracle_checks(oracle, pg):
    """CPU leg: fp64 oracle residuals of the GPU solutions and Ritz pairs."""
    S, b, rep = pg["S"], pg["b"], pg["report"]
    bn = float(np.linalg.norm(b))
    for name, x in pg["x"].items():
        rep[name]["rel_residual_oracle"] = float(np.linalg.norm(b - oracle.crs_spmv(S, x)) / bn)
    for dt, y in pg["ys"].items():
        L = rep["lanczos"][dt]
        Ay = oracle.crs_spmv(S, y)
        rq = float(y @ Ay / (y @ y))
        L["theta_oracle_rayleigh"] = rq
        L["rel_residual_oracle"] = float(np.linalg.norm(Ay - rq * y) / np.linalg.norm(y) / abs(rq))
    pg["report"] = rep
    return pg


CASE_DOC = """Run one pJDS product case a few times, for profiling under ncu.

    python bench.py case --matrix stencil --g 100 --dtype f64 --permuted --staged --reps 3

Builds one seeded synthetic matrix, converts it, uploads it and launches the
chosen product `--reps` times (after `--warmup` launches) on the current
stream, then prints one JSON line with the CUDA-event time of each launch.
Matrices: hmep (--n rows), stencil (--g grid), dlr (--n rows, 144/row), zipf
(--n rows). Kinds: spmv (default), pattern (the pattern product), ellr, spmm (--k right-hand sides);
cg (one mixed-precision CG solve of `--reps` inner steps in the permuted
basis, fp64 outer matrix, --dtype inner matrix, no graph) and lanczos
(`--reps` steps, no graph) on the stencil; batch (--mats Zipf matrices with
N log-uniform in [10k, --n], one persistent launch per repetition); mlp (the
learned tuner's cost model trained for `--reps` epochs on the committed
timing data, then inference over the candidates of the held-out matrices).
"""


def run_case(argv) -> int:
    ap = argparse.ArgumentParser(prog="bench.py case", description=CASE_DOC)
    ap.add_argument("--matrix", choices=["hmep", "stencil", "dlr", "zipf"], default="hmep")
    ap.add_argument("--n", type=int, default=2_000_000)
    ap.add_argument("--g", type=int, default=100)
    ap.add_argument("--dtype", choices=["f64", "f32", "bf16"], default="f64")
    ap.add_argument("--kind", choices=["spmv", "pattern", "ellr", "spmm", "spmm_pattern", "cg", "lanczos", "batch",
                                       "mlp"],
                    default="spmv")
    ap.add_argument("--mats", type=int, default=64)
    ap.add_argument("--k", type=int, default=8)
    ap.add_argument("--permuted", action="store_true")
    ap.add_argument("--staged", action="store_true")
    ap.add_argument("--threads-per-row", type=int, default=0)
    ap.add_argument("--rows-per-thread", type=int, default=0)
    ap.add_argument("--tile-order", type=int, default=0)
    ap.add_argument("--plan", type=int, default=0)
    ap.add_argument("--unroll", type=int, default=0)
    ap.add_argument("--block-threads", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--seed", type=int, default=1234)
    a = ap.parse_args(argv)

    import torch

    import synth
    from paper_1112_5588_gb300 import batch, krylov, pjds

    dev = torch.device("cuda")
    if a.kind == "mlp":
        return run_mlp(a, torch)
    if a.kind == "batch":
        return run_batch(a, torch, synth, batch, pjds, dev)
    if a.kind in ("cg", "lanczos"):
        return run_krylov(a, torch, synth, krylov, pjds, dev)
    if a.matrix == "hmep":
        A = synth.hmep_like(n=a.n, seed=a.seed)
    elif a.matrix == "stencil":
        A = synth.stencil27(g=a.g, seed=a.seed)
    elif a.matrix == "dlr":
        A = synth.block_dense(n_brow=max(1, a.n // 4), bs=4, nb=36, frac=0.05, seed=a.seed)
    else:
        A = synth.zipf_rows(a.n, s=2.0, len_max=512, seed=a.seed)
    if a.kind == "ellr":
        D = pjds.ellr_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, dtype=a.dtype).to_device(dev)
    else:
        D = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=a.dtype,
                             permute_cols=a.permuted).to_device(dev)
    if a.kind in ("spmm", "spmm_pattern"):
        X = torch.rand(A.n_cols, a.k, device=dev, dtype=D.vec_dtype)
        Y = torch.empty(A.n_rows, a.k, device=dev, dtype=D.vec_dtype)
        fn = batch.spmm if a.kind == "spmm" else batch.spmm_pattern
        run = lambda: fn(D, X, Y)  # noqa: E731
    else:
        x = torch.from_numpy(synth.vector(A.n_cols, seed=a.seed)).to(dev, D.vec_dtype)
        y = torch.empty(A.n_rows, device=dev, dtype=D.vec_dtype)
        if a.kind == "ellr":
            run = lambda: pjds.ellr_spmv(D, x, y)  # noqa: E731
        else:
            kw = dict(staged=1 if a.staged else 0, threads_per_row=a.threads_per_row,
                      rows_per_thread=a.rows_per_thread, tile_order=a.tile_order, plan=a.plan,
                      unroll=a.unroll, block_threads=a.block_threads)
            run = (lambda: pjds.pjds_spmv_pattern(D, x, y, **kw)) if a.kind == "pattern" else (  # noqa: E731
                lambda: pjds.pjds_spmv_cfg(D, x, y, **kw))
    for _ in range(a.warmup):
        run()
    torch.cuda.synchronize()
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) * 1e3)
    status = pjds.pjds_device_status() if a.staged else 0
    print(json.dumps({"matrix": a.matrix, "n_rows": A.n_rows, "nnz": A.nnz, "dtype": a.dtype, "kind": a.kind,
                      "permuted": a.permuted, "staged": a.staged, "us": [round(t, 2) for t in times],
                      "cfg": pjds.pjds_spmv_resolve(D, **kw) if a.kind in ("spmv", "pattern") else None,
                      "device_status": status}))
    return 0 if status == 0 else 1


def _timed(torch, run, reps, warmup):
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        times.append(round(e0.elapsed_time(e1) * 1e3, 2))
    return times


def run_mlp(a, torch) -> int:
    import os
    import time
    from paper_1112_5588_gb300 import learned, tuner_data
    data = dict(np.load(os.path.join(ROOT, "paper_1112_5588_gb300", "data", "tuner_timings_gb300.npz"),
                        allow_pickle=False))
    X, y = tuner_data.samples(data, range(int(data["n_train"])))
    m = learned.init(1)
    learned.fit_scaling(m, X, y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = learned.train(m, X, y, epochs=a.reps, batch=1024, lr=2e-3, seed=1)
    t_train = time.perf_counter() - t0
    cands = __import__("json").loads(str(data["cands"]))
    rows = range(int(data["n_train"]), len(data["times_us"]))
    enc = np.concatenate([learned.encode(data["features"][i], cands) for i in rows])
    learned.predict(m, enc)
    t0 = time.perf_counter()
    learned.predict(m, enc)
    t_pred = time.perf_counter() - t0
    print(json.dumps({"kind": "mlp", "samples": int(len(y)), "epochs": a.reps, "train_s": round(t_train, 3),
                      "s_per_epoch": round(t_train / max(a.reps, 1), 4), "loss_first": float(hist[0]),
                      "loss_last": float(hist[-1]), "predict_rows": int(len(enc)), "predict_us": round(t_pred * 1e6, 1)}))
    return 0


def run_batch(a, torch, synth, batch, pjds, dev) -> int:
    rng = np.random.default_rng(a.seed)
    sizes = np.exp(rng.uniform(np.log(10_000), np.log(max(a.n, 10_001)), a.mats)).astype(int)
    devs, xs, ys, nnz = [], [], [], 0
    for m, n in enumerate(sizes):
        M = synth.zipf_rows(int(n), s=2.0, len_max=512, seed=a.seed + m)
        nnz += M.nnz
        devs.append(pjds.pjds_create(M.n_rows, M.n_cols, M.row_ptr, M.col, M.val, b=32,
                                     dtype=a.dtype).to_device(dev))
        xs.append(torch.from_numpy(synth.vector(M.n_cols, seed=m)).to(dev, devs[-1].vec_dtype))
        ys.append(torch.empty(M.n_rows, dtype=devs[-1].vec_dtype, device=dev))
    B = batch.Batch(devs, xs, ys)
    times = _timed(torch, lambda: B.run(use_graph=False), a.reps, a.warmup)
    info = B.info()
    B.destroy()
    print(json.dumps({"kind": "batch", "n_mats": a.mats, "total_rows": int(sizes.sum()), "nnz": int(nnz),
                      "dtype": a.dtype, **info, "us": times}))
    return 0


def run_krylov(a, torch, synth, krylov, pjds, dev) -> int:
    A = synth.stencil27(g=a.g, seed=a.seed)
    H64 = pjds.pjds_create(A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype="f64", permute_cols=True)
    D64 = H64.to_device(dev)
    H64.destroy()
    if a.kind == "cg":
        Dlo = D64 if a.dtype == "f64" else pjds.pjds_create(
            A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=a.dtype, permute_cols=True).to_device(dev)
        b = torch.from_numpy(synth.vector(A.n_rows, seed=a.seed)).to(dev)
        x = torch.zeros_like(b)

        def run():
            x.zero_()
            krylov.cg_solve(D64, Dlo, b, x, max_outer=1, inner_iters=a.reps, use_graph=False)
        times = _timed(torch, run, 1, a.warmup)
    else:
        D = D64 if a.dtype == "f64" else pjds.pjds_create(
            A.n_rows, A.n_cols, A.row_ptr, A.col, A.val, b=32, dtype=a.dtype, permute_cols=True).to_device(dev)
        v0 = torch.from_numpy(synth.vector(A.n_rows, seed=a.seed)).to(dev, D.vec_dtype)
        times = _timed(torch, lambda: krylov.lanczos(D, v0, a.reps, use_graph=False), 1, a.warmup)
    print(json.dumps({"kind": a.kind, "matrix": f"stencil g={a.g}", "n_rows": A.n_rows, "nnz": A.nnz,
                      "dtype": a.dtype, "steps": a.reps, "us_total": times}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
