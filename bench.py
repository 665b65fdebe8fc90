"""Benchmark: SpMV over COO / CSR / DIA and FP64 CG on the 27-point HPCG stencil.

Workload (one "step", data resident in HBM): on the 128^3 stencil (n = 2,097,152,
nnz = 55,742,968, FP64 values, int32 indices) one SpMV per format (COO, CSR, DIA)
followed by 50 unpreconditioned FP64 CG iterations on the DIA matrix from x0 = 0 with
b = A 1. Conversion (HPCG's optimisation set-up phase) is done once, untimed, and
reported. Metric: GB/s by the algorithmic byte model (values + indices + x + y per
SpMV; 88 n extra bytes per CG iteration for its vector passes); per-format GB/s, the
DIA kernel against the HBM roofline, and CG time-to-1e-10 in FP64 and mixed precision
(FP32 DIA values with FP64 refinement) are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mspv|reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU (the
path has no exchange step here); timing is the max over ranks after a barrier.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "SpMV GB/s (% of HBM peak) per format; CG time-to-1e-10, FP64 vs mixed"
GRID = 128
CG_ITERS = 50
NDIAGS = 27
# FP64 ALU roofline: 2 FP64 FMA per clock per SM (GB300), 152 SMs, 2070 MHz max SM clock,
# 2 flops per FMA -> 1.2586 TFLOP/s (NVIDIA's nominal FP64 figure for the part is 1.25).
FP64_FMA_PER_CLK_SM = 2
FP64_PEAK_TFLOPS = 2 * FP64_FMA_PER_CLK_SM * 152 * 2.070e9 / 1e12


# DRAM traffic of one spmv_dia_kernel<double, double, false> launch without the CG epilogue,
# from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, one launch, the first DIA
# SpMV of the run) on the 128^3 stencil, the benchmark's own grid; other grids scale it by rows
# (every stream of the kernel grows with n). Reported only while the source of that launch (the
# FP64 value loader, the kernel and the FP64 branch of its launcher) is the one captured.
DIA_TRAFFIC = {"bytes": 469_803_264 + 4_328_448, "rows": 128 ** 3,
               "src_sha256": "a4c7fd0698f8ce4ff5159215953bb280fe3cb8407e0ef26678feeca0fd806dec"}


def dia_source_sha() -> str | None:
    import hashlib
    try:
        src = open(os.path.join(ROOT, "paper_2304_09511_gb300", "csrc", "spmv.cu")).read()
        a = src.index("template <> struct DiaVec<double, double> {")
        b = src.index("\n};\n", a)
        c = src.index("// One thread per RPT consecutive rows")
        d = src.index("\n}\n", c)
        e = src.index("static void launch_dia(")
        f = src.index("\n}\n", e)
        body = src[src.index("constexpr int RPT = DiaVec<VT, T>::RPT;", e):f]   # the strip-kernel launch
        i = body.index("if constexpr (sizeof(T) == 4) {")
        j = body.index("} else {", i)
    except (OSError, ValueError):
        return None
    return hashlib.sha256((src[a:b] + src[c:d] + body[:i] + body[j:]).encode()).hexdigest()


def dia_traffic(n: int) -> int | None:
    if dia_source_sha() != DIA_TRAFFIC["src_sha256"]:
        return None
    return int(round(DIA_TRAFFIC["bytes"] * n / DIA_TRAFFIC["rows"]))


def byte_model(n: int, nnz: int, ndiags: int, vbytes: int = 8) -> dict:
    """Algorithmic bytes of one SpMV per format and of one CG iteration (DIA)."""
    coo = (vbytes + 8) * nnz + 16 * n
    csr = (vbytes + 4) * nnz + 4 * (n + 1) + 16 * n
    dia = vbytes * ndiags * n + 4 * ndiags + 16 * n
    cg_iter = (dia - 16 * n) + 88 * n
    return {"coo": coo, "csr": csr, "dia": dia, "cg_iter": cg_iter}


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def copy_rate_gbs(torch, dev, elems: int = 1 << 30, repeats: int = 10) -> float:
    """Device-to-device copy rate of this GPU: read + write bytes of one copy of `elems` BF16
    values over its CUDA-event time, the fastest of `repeats` (after two untimed copies). The
    STREAM-style figure, measured live beside the HBM peak that the fractions are taken of."""
    a = torch.ones(elems, dtype=torch.bfloat16, device=dev)
    b = torch.empty_like(a)
    s = torch.cuda.current_stream(dev)
    best = float("inf")
    for k in range(repeats + 2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        b.copy_(a)
        e1.record(s)
        e1.synchronize()
        if k >= 2:
            best = min(best, e0.elapsed_time(e1))
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * 2 * elems / (best * 1e-3) / 1e9


def spmv_launch_ms(torch, stream, launch, reps: int = 30, warm: int = 3) -> float:
    """Median device time of one launch among `reps` back-to-back launches (CUDA events on the
    launching stream around each), after `warm` untimed ones."""
    for _ in range(warm):
        launch()
    pairs = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        launch()
        e1.record(stream)
        pairs.append((e0, e1))
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in pairs]))


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def shard(count: int, world: int, rank: int) -> range:
    """Independent units (e.g. the selector's matrices) dealt round-robin to the ranks."""
    return range(rank, count, world)


def gather_records(rec: list, world: int, key: str = "seed") -> list:
    """Every rank's records, concatenated and ordered by `key` (on every rank)."""
    if world <= 1:
        return sorted(rec, key=lambda x: x[key])
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, rec)
    return sorted((x for part in parts for x in part), key=lambda x: x[key])


def max_over_ranks(value: float, world: int) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mspv_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def time_to_solution(mspv, torch, dev, g, perturb_seed, inner_tol, tune=False):
    """Time to a 1e-10 relative residual from x0 = 0 on the g^3 stencil, DIA: FP64 CG against
    FP64-outer mixed precision. Exact values 26 / -1 with b = A 1 (HPCG's right-hand side), or
    the perturbed SPD stencil, whose values FP32 / BF16 do round, with b = A x* for
    x* ~ U[0.5, 1.5) (seed 1): its rows sum to 1, so A 1 = 1 is an eigenvector and b = A 1 would
    converge in one iteration. Each solver runs once untimed, then once timed with CUDA events;
    max |x - x*| is the error against the exact solution. With `tune`, FP64 CG also runs in the
    format the run-first tuner picks (every format built and timed, the fastest kept)."""
    n = g ** 3
    r, c, v = synth.stencil27_torch(g, dev, perturb_seed=perturb_seed)
    A = mspv.Matrix.from_coo(n, n, r, c, v)
    del r, c, v
    tuned = None
    if tune:
        tuned, tune_ms = A.tune_format(reps=10)
        T = None if tuned in ("dia", "coo") else A.convert(tuned)
    D = A.convert("dia")
    D32 = A.convert("dia", "f32")
    D16 = A.convert("dia", "bf16")
    if tuned == "coo":
        T = A
    else:
        A.close()
    if perturb_seed is None:
        xstar = torch.ones(n, dtype=torch.float64, device=dev)
    else:
        xstar = torch.from_numpy(synth.uniform_x(n, 1) + 0.5).to(dev)
    b = D.spmv(xstar)
    stream = torch.cuda.current_stream()
    modes = (
        ("fp64_cg", lambda xx: D.cg(b, x=xx, tol=1e-10, maxit=20000)),
        ("fp64_cg_tuner_format", (lambda xx: T.cg(b, x=xx, tol=1e-10, maxit=20000)) if tune and T is not None
         else None),
        # FP32 values with FP64 arithmetic in the inner CG and its SpMV (FP64 accumulation)
        ("ir_f32_values_fp64_arith", lambda xx: D.cg_ir(D32, b, x=xx, tol=1e-10, inner_tol=1e-5,
                                                        max_outer=40, maxit_inner=20000)),
        # FP32 / BF16 values, restarted refinement around an FP32-arithmetic inner CG
        ("ir_f32_values_fp32_inner", lambda xx: D.cg_ir(D32, b, x=xx, tol=1e-10, inner_tol=inner_tol,
                                                        max_outer=40, maxit_inner=20000, inner_fp32=True)),
        ("ir_bf16_values_fp32_inner", lambda xx: D.cg_ir(D16, b, x=xx, tol=1e-10, inner_tol=inner_tol,
                                                         max_outer=40, maxit_inner=20000, inner_fp32=True)),
        # one FP32-arithmetic CG with reliable FP64 residual updates
        ("ru_f32_values", lambda xx: D.cg_ru(D32, b, x=xx, tol=1e-10, max_updates=400, maxit=20000)),
        ("ru_bf16_values", lambda xx: D.cg_ru(D16, b, x=xx, tol=1e-10, max_updates=400, maxit=20000)),
    )
    os.environ["MSPV_CG_CHECK_EVERY"] = "10"
    out = {}
    if tune:
        out["tuner"] = {"format": tuned,
                        "ms_per_spmv": {k: (round(x, 5) if math.isfinite(x) else None) for k, x in tune_ms.items()}}
    for label, fn in modes:
        if fn is None:
            continue
        xx = torch.zeros(n, dtype=torch.float64, device=dev)
        fn(xx)
        xx.zero_()
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        e0 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        res = fn(xx)
        e0.record(stream)
        torch.cuda.synchronize()
        out[label] = {"ms": round(s0.elapsed_time(e0), 3), "iters": res.iters, "outer": res.outer_iters,
                      "relres": res.relres, "converged": res.converged,
                      "max_abs_err": float((xx - xstar).abs().max().item())}
    base = out["fp64_cg"]["ms"]
    for label, rec in out.items():
        if "ms" in rec:
            rec["speedup_vs_fp64_cg"] = round(base / rec["ms"], 3)
    for M in (D, D32, D16) + ((T,) if tune and T is not None else ()):
        M.close()
    return out


def run_mspv(args, world, rank, local):
    import torch
    import paper_2304_09511_gb300 as mspv

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    os.environ.setdefault("MSPV_CG_CHECK_EVERY", str(CG_ITERS))

    g = args.grid
    n = g ** 3
    rows, cols, vals = synth.stencil27(g)
    nnz = rows.size
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    A = mspv.Matrix.from_coo(n, n, torch.from_numpy(rows).to(dev), torch.from_numpy(cols).to(dev),
                             torch.from_numpy(vals).to(dev))
    torch.cuda.synchronize()
    t_coo = time.perf_counter() - t0
    t0 = time.perf_counter()
    C = A.convert("csr")
    t_csr = time.perf_counter() - t0
    t0 = time.perf_counter()
    D = A.convert("dia")
    t_dia = time.perf_counter() - t0
    D32 = A.convert("dia", "f32")
    D16 = A.convert("dia", "bf16")
    del rows, cols, vals
    ndiags = D.info["ndiags"]
    bm = byte_model(n, nnz, ndiags)

    x = torch.from_numpy(synth.uniform_x(n, 0)).to(dev)
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    b = D.spmv(ones)
    y = {f: torch.empty(n, dtype=torch.float64, device=dev) for f in ("coo", "csr", "dia")}
    xcg = torch.zeros(n, dtype=torch.float64, device=dev)
    mats = {"coo": A, "csr": C, "dia": D}

    def step(events=None):
        if events:
            events[0].record(stream)
        for k, f in enumerate(("coo", "csr", "dia")):
            mats[f].spmv(x, y[f])
            if events:
                events[k + 1].record(stream)
        xcg.zero_()
        D.cg(b, x=xcg, tol=0.0, maxit=args.cg_iters)
        if events:
            events[4].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(K):
        step(evs[k])
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed_ms = max_over_ranks(start.elapsed_time(end), world)

    seg = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(4)] for k in range(K)])
    ms = {"coo": float(seg[:, 0].mean()), "csr": float(seg[:, 1].mean()), "dia": float(seg[:, 2].mean()),
          "cg": float(seg[:, 3].mean())}
    cg_bytes = bm["cg_iter"] * args.cg_iters + bm["dia"] + 32 * n   # init: A x0, r = b - q, p = r
    step_bytes = bm["coo"] + bm["csr"] + bm["dia"] + cg_bytes
    ms_per_step = elapsed_ms / K
    value = world * step_bytes / (ms_per_step * 1e-3) / 1e9
    peaks = load_peaks()
    # Per-format SpMV time: the median of back-to-back launches, timed right after the step loop.
    # Inside the step the COO launch follows the host's return from the previous step's CG
    # (which reads its iteration count back), so its segment also holds the host's launch
    # latency; that segment is reported beside it as ms_in_step.
    per_format = {}
    for f in ("coo", "csr", "dia"):
        t = spmv_launch_ms(torch, stream, lambda: mats[f].spmv(x, y[f]))
        gbs = bm[f] / (t * 1e-3) / 1e9
        per_format[f] = {"ms": round(t, 5), "ms_in_step": round(ms[f], 5), "GB_s": round(gbs, 1),
                         "frac_of_measured_hbm": round(gbs / peaks["hbm_gbs"], 4),
                         "frac_of_nominal_8TBs": round(gbs / 8000.0, 4),
                         "GFLOP_s": round(2 * nnz / (t * 1e-3) / 1e9, 1),
                         "bytes": bm[f]}
    cg_ms_iter = ms["cg"] / args.cg_iters

    # gpu launches of this library inside the timed region
    # COO: the row-block kernel alone (rows of at most 128 entries), else a chunked kernel + fix-up
    inf = A.info
    coo_kernel = os.environ.get("MSPV_COO_KERNEL") or (
        "seg" if inf["row_max"] > 128 else ("rb" if inf["nnz"] >= 4 * inf["nrows"] else "vec"))
    chunk = 512 if coo_kernel == "seg" else 256
    coo_launches = 1 if coo_kernel == "rb" else 1 + (1 if (nnz + chunk - 1) // chunk > 1 else 0)
    # CG: SpMV + init + start + the b = 0 check, then per iteration SpMV (DIA: 1 kernel), alpha,
    # update, beta, p-update
    launches_per_step = coo_launches + 1 + 1 + (4 + 5 * args.cg_iters)

    # end to end through the public API with host buffers: every step copies its x and b from
    # pinned host memory and reads the three SpMV results and the CG solution back, all inside
    # the timed region. The copies run on a second stream: step k+1's inputs are fetched into
    # the other half of a double buffer while step k computes, and each result is read back as
    # soon as it is ready; events order every copy against the kernels that use its buffer.
    x_h = torch.from_numpy(synth.uniform_x(n, 0)).pin_memory()
    b_h = b.cpu().pin_memory()
    outs_h = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in range(4)]
    x_d = [torch.empty_like(x) for _ in range(2)]
    b_d = [torch.empty_like(b) for _ in range(2)]
    xcg_d = [torch.empty_like(xcg) for _ in range(2)]
    copy = torch.cuda.Stream(device=dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_used = [torch.cuda.Event() for _ in range(2)]    # main stream finished with input buffer
    ev_y = {f: torch.cuda.Event() for f in ("coo", "csr", "dia")}
    ev_y_read = {f: torch.cuda.Event() for f in ("coo", "csr", "dia")}
    ev_x = [torch.cuda.Event() for _ in range(2)]
    ev_x_read = [torch.cuda.Event() for _ in range(2)]
    for e in list(ev_used) + list(ev_y_read.values()) + list(ev_x_read):
        e.record(stream)

    def fetch(k):
        j = k % 2
        copy.wait_event(ev_used[j])
        with torch.cuda.stream(copy):
            x_d[j].copy_(x_h, non_blocking=True)
            b_d[j].copy_(b_h, non_blocking=True)
        ev_in[j].record(copy)

    def e2e_step(k, last):
        j = k % 2
        if not last:
            fetch(k + 1)
        stream.wait_event(ev_in[j])
        for i, f in enumerate(("coo", "csr", "dia")):
            stream.wait_event(ev_y_read[f])
            mats[f].spmv(x_d[j], y[f])
            ev_y[f].record(stream)
            copy.wait_event(ev_y[f])
            with torch.cuda.stream(copy):
                outs_h[i].copy_(y[f], non_blocking=True)
            ev_y_read[f].record(copy)
        stream.wait_event(ev_x_read[j])
        xcg_d[j].zero_()
        D.cg(b_d[j], x=xcg_d[j], tol=0.0, maxit=args.cg_iters)
        ev_used[j].record(stream)
        ev_x[j].record(stream)
        copy.wait_event(ev_x[j])
        with torch.cuda.stream(copy):
            outs_h[3].copy_(xcg_d[j], non_blocking=True)
        ev_x_read[j].record(copy)

    def e2e_run(steps):
        fetch(0)
        for k in range(steps):
            e2e_step(k, k == steps - 1)
        stream.wait_stream(copy)

    e2e_run(max(1, args.warmup))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    s2 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    s2.record(stream)
    copy.wait_event(s2)
    e2e_run(K)
    e2.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(s2.elapsed_time(e2), world) / K
    e2e_value = world * step_bytes / (e2e_ms * 1e-3) / 1e9

    # CG time-to-1e-10 (FP64 DIA) and mixed precision (FP32 DIA values, FP64 refinement)
    tt = {}
    modes = (
        ("fp64", lambda xx: D.cg(b, x=xx, tol=1e-10, maxit=5000)),
        # FP32 values, FP64 arithmetic in the inner CG (as the mixed-precision target specifies)
        ("ir_f32_values_fp64_inner", lambda xx: D.cg_ir(D32, b, x=xx, tol=1e-10, inner_tol=1e-5,
                                                        max_outer=20, maxit_inner=5000)),
        # FP32 / BF16 values with an FP32-arithmetic inner CG
        ("ir_f32_values_fp32_inner", lambda xx: D.cg_ir(D32, b, x=xx, tol=1e-10, inner_tol=args.ir_inner_tol,
                                                        max_outer=30, maxit_inner=5000, inner_fp32=True)),
        ("ir_bf16_values_fp32_inner", lambda xx: D.cg_ir(D16, b, x=xx, tol=1e-10, inner_tol=args.ir_inner_tol,
                                                         max_outer=30, maxit_inner=5000, inner_fp32=True)),
        # one FP32-arithmetic CG with reliable FP64 residual updates
        ("ru_f32_values", lambda xx: D.cg_ru(D32, b, x=xx, tol=1e-10, maxit=5000)),
        ("ru_bf16_values", lambda xx: D.cg_ru(D16, b, x=xx, tol=1e-10, maxit=5000)),
    )
    for label, fn in modes:
        os.environ["MSPV_CG_CHECK_EVERY"] = "10"
        xx = torch.zeros(n, dtype=torch.float64, device=dev)
        fn(xx)   # warm
        xx.zero_()
        s3 = torch.cuda.Event(enable_timing=True)
        e3 = torch.cuda.Event(enable_timing=True)
        s3.record(stream)
        res = fn(xx)
        e3.record(stream)
        torch.cuda.synchronize()
        tt[label] = {"ms": round(s3.elapsed_time(e3), 3), "iters": res.iters, "outer": res.outer_iters,
                     "relres": res.relres, "converged": res.converged}

    # time to solution on the larger stencil, exact and perturbed values
    tts = {}
    if args.tts_grid > 0:
        tts["exact"] = time_to_solution(mspv, torch, dev, args.tts_grid, None, args.ir_inner_tol)
        tts["perturbed"] = time_to_solution(mspv, torch, dev, args.tts_grid, 3, args.ir_inner_tol)
    tts_large = {}
    if args.tts_large_grid > 0:
        tts_large["exact"] = time_to_solution(mspv, torch, dev, args.tts_large_grid, None, args.ir_inner_tol,
                                              tune=True)

    # the FP64 FMA rate of this GPU: the peak of the FP64 (ALU-bound) roofline; and its copy rate
    fp64_peak = mspv.fp64_fma_rate()
    copy_gbs = copy_rate_gbs(torch, dev)
    for f in ("coo", "csr", "dia"):
        per_format[f]["frac_of_live_copy"] = round(per_format[f]["GB_s"] / copy_gbs, 4)

    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = float(clk["sm_max_mhz"]) if clk and clk.get("sm_max_mhz") else 2070.0
    derived_peak = 2.0 * FP64_FMA_PER_CLK_SM * sms * sm_mhz * 1e6 / 1e12

    dia_launch_ms = ms["dia"]
    dia_s = dia_launch_ms * 1e-3
    achieved_tf = 2.0 * nnz / dia_s / 1e12          # algorithmic flops (2 per stored nonzero)
    executed_tf = 2.0 * ndiags * n / dia_s / 1e12    # FMAs the kernel issues (incl. padded slots)
    achieved_gbs = bm["dia"] / dia_s / 1e9
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"27-point stencil {g}^3 (n={n}, nnz={nnz}), FP64 values, int32 indices; "
                               f"step = SpMV COO + CSR + DIA, then {args.cg_iters} FP64 CG iterations (DIA)",
                   "l2": "inputs larger than L2 (matrices 486-925 MB per format; no flush)",
                   "parallelism": f"replicas x{world}"},
        "per_format": per_format,
        "hbm_peak": {"GB_s": peaks["hbm_gbs"], "source": peaks["source"], "copy_measured_live": round(copy_gbs, 1)},
        "cg": {"ms_per_iter": round(cg_ms_iter, 5),
               "GB_s": round(bm["cg_iter"] / (cg_ms_iter * 1e-3) / 1e9, 1),
               "time_to_1e-10": tt,
               f"time_to_1e-10_{args.tts_grid}^3": tts,
               f"time_to_1e-10_{args.tts_large_grid}^3": tts_large},
        "convert_s": {"coo_sort_coalesce": round(t_coo, 4), "csr": round(t_csr, 4), "dia": round(t_dia, 4)},
        "roofline": {"kernel": "spmv_dia_kernel<double>", "bound": "alu",
                     "achieved": round(achieved_tf, 4), "peak": round(derived_peak, 4), "unit": "TFLOP/s",
                     "frac": round(achieved_tf / derived_peak, 4),
                     "peak_source": f"derived: {FP64_FMA_PER_CLK_SM} FP64 FMA/clk/SM x {sms} SMs x "
                                    f"{sm_mhz:.0f} MHz (max SM clock, sampled under load) x 2 flop",
                     "executed_fma_frac": round(executed_tf / derived_peak, 4),
                     "fp64_fma_ceiling_measured": round(fp64_peak, 4),
                     "frac_of_measured_ceiling": round(achieved_tf / fp64_peak, 4),
                     "ceiling_source": "mspv_fp64_fma_rate on this GPU: one full wave of independent "
                                       "FP64 FMA chains (4, 8 or 16 per thread), fastest launch",
                     "traffic": dia_traffic(n),
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch "
                                       "on the 128^3 stencil (scaled by rows at other grids)",
                     "flops_per_launch": 2 * nnz, "bytes_per_launch": bm["dia"],
                     "hbm": {"achieved": round(achieved_gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                             "frac": round(achieved_gbs / peaks["hbm_gbs"], 4), "peak_source": peaks["source"],
                             "copy_measured_live": round(copy_gbs, 1),
                             "frac_of_live_copy": round(achieved_gbs / copy_gbs, 4)}},
        "e2e": {"value": round(e2e_value, 1), "unit": "GB/s", "ms_per_step": round(e2e_ms, 4),
                "h2d_bytes_per_step": 16 * n, "d2h_bytes_per_step": 32 * n},
        "gpu_launches": launches_per_step * K,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the host baseline is an N = 1 figure
        out["cpu_baseline"] = cpu_baseline(g, args.cpu_cg_iters)
    if world > 1:
        torch.distributed.destroy_process_group()
    return out if rank == 0 else None


# ---------------------------------------------------------------------------
# format selection: run-first tuner labels, MLP selector, held-out regret
# ---------------------------------------------------------------------------
SELECTOR_METRIC = "format-selector regret on held-out matrices vs the run-first tuner"


def _regret(ms: np.ndarray, picks: np.ndarray) -> dict:
    best = ms.min(axis=1)
    chosen = ms[np.arange(len(picks)), picks]
    slow = chosen / best
    return {"regret": round(float(chosen.sum() / best.sum() - 1.0), 5),
            "geomean_slowdown": round(float(np.exp(np.mean(np.log(slow)))), 5),
            "mean_slowdown": round(float(np.mean(slow)), 5),
            "max_slowdown": round(float(np.max(slow)), 4),
            "within_10pct": round(float(np.mean(slow <= 1.10)), 4),
            "exact": round(float(np.mean(chosen == best)), 4)}


def run_selector(args, world, rank, local):
    """Labels every synthetic matrix with the run-first tuner (time each format, keep the
    fastest), trains the MLP selector on the 4/5 of seeds with seed % 5 != 0, and reports
    its regret on the held-out fifth; then the 256^3 stencil end to end: the selector's
    format with FP32 values and FP64 refinement against FP64 CG in the tuner's format."""
    import torch
    import paper_2304_09511_gb300 as mspv

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    FMT = ("coo", "csr", "dia")
    rec = []
    t_label = time.perf_counter()
    for seed in shard(args.matrices, world, rank):
        fam, n, r, c, v = synth.family_matrix_torch(seed, dev)
        A = mspv.Matrix.from_coo(n, n, r, c, v)
        del r, c, v
        nnz = A.info["nnz"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = A.features()
        t_feat = time.perf_counter() - t0
        t0 = time.perf_counter()
        best, ms = A.tune_format(reps=args.tune_reps)
        t_tune = time.perf_counter() - t0
        A.close()
        rec.append({"seed": seed, "family": fam, "n": n, "nnz": nnz, "features": f.tolist(),
                    "ms": [ms[k] for k in FMT], "best": FMT.index(best), "t_feat": t_feat, "t_tune": t_tune})
    t_label = time.perf_counter() - t_label
    rec = gather_records(rec, world)
    t_label = max_over_ranks(t_label, world)
    out = None
    if rank == 0:
        X = np.array([x["features"] for x in rec], dtype=np.float32)
        y = np.array([x["best"] for x in rec], dtype=np.int32)
        ms = np.array([x["ms"] for x in rec], dtype=np.float64)
        held = np.array([x["seed"] % 5 == 0 for x in rec])
        t0 = time.perf_counter()
        params = mspv.selector_train(X[~held], y[~held], epochs=args.epochs, lr=args.lr, seed=0)
        t_train = time.perf_counter() - t0
        t0 = time.perf_counter()
        pred = mspv.selector_predict(params, X[held])
        t_pred = time.perf_counter() - t0
        # a DIA pick the tuner could not build (inf) counts as CSR, as mspv_select_format does
        pred = np.where(np.isinf(ms[held][np.arange(held.sum()), pred]), 1, pred)
        train_acc = float(np.mean(mspv.selector_predict(params, X[~held]) == y[~held]))
        fams = np.array([x["family"] for x in rec])
        per_family = {}
        for fam in synth.FAMILIES:
            m = fams[held] == fam
            if m.any():
                per_family[fam] = {"n": int(m.sum()), "accuracy": round(float(np.mean(pred[m] == y[held][m])), 4),
                                   "labels": np.bincount(y[held][m], minlength=3).tolist(),
                                   **_regret(ms[held][m], pred[m])}
        sel_stats = _regret(ms[held], pred)
        csr_stats = _regret(ms[held], np.ones(int(held.sum()), dtype=np.int64))
        # The regret above is measured on the timings that made the labels. A second, independent
        # timing run of the held-out matrices judges the same predictions on fresh timings, and
        # shows how often the tuner's own pick repeats (near-ties flip).
        held_seeds = [x["seed"] for x, h in zip(rec, held) if h]
        ms2 = np.zeros((len(held_seeds), 3))
        for k, seed in enumerate(held_seeds):
            fam, n, r, c, v = synth.family_matrix_torch(seed, dev)
            A = mspv.Matrix.from_coo(n, n, r, c, v)
            del r, c, v
            _, t2 = A.tune_format(reps=args.tune_reps)
            A.close()
            ms2[k] = [t2[f] for f in FMT]
        retimed = {**_regret(ms2, pred), "tuner_label_repeats": round(float(np.mean(ms2.argmin(axis=1) ==
                                                                                 y[held])), 4),
                   "always_csr_regret": _regret(ms2, np.ones(len(held_seeds), dtype=np.int64))["regret"]}
        t_feat = np.array([x["t_feat"] for x in rec])
        t_tune = np.array([x["t_tune"] for x in rec])
        out = {
            "metric": SELECTOR_METRIC, "value": sel_stats["regret"], "unit": "fraction",
            "higher_is_better": False, "n_gpus": world, "mode": "selector", "data": "synthetic",
            "dtype": "f32 (MLP), f64 (SpMV timing)",
            "config": {"workload": f"{args.matrices} seeded matrices, 4 families (banded, uniform 8-64/row, "
                                   "power-law rows, 32x32 block-diagonal), n log-uniform in [1e4, 2e6]; "
                                   f"train seed % 5 != 0 ({int((~held).sum())}), held out seed % 5 == 0 "
                                   f"({int(held.sum())}); labels: run-first tuner, {args.tune_reps} timed "
                                   "SpMV per format; MLP 10-64-64-3, Adam",
                       "epochs": args.epochs, "lr": args.lr, "parallelism": f"labels sharded x{world}"},
            "held_out": {**sel_stats, "accuracy": round(float(np.mean(pred == y[held])), 4),
                         "always_csr": csr_stats, "per_family": per_family},
            "held_out_retimed": retimed,
            "train_accuracy": round(train_acc, 4),
            "label_distribution": {FMT[k]: int(v) for k, v in enumerate(np.bincount(y, minlength=3))},
            "cost_ms_per_matrix": {"features": round(float(t_feat.mean() * 1e3), 3),
                                   "predict_batch_total": round(t_pred * 1e3, 3),
                                   "run_first_tuner": round(float(t_tune.mean() * 1e3), 3)},
            "train_s": round(t_train, 3), "label_s": round(t_label, 2),
        }
        if args.e2e_grid > 0:
            out["stencil_e2e"] = _selector_stencil_e2e(mspv, torch, dev, params, args.e2e_grid)
    if world > 1:
        torch.distributed.destroy_process_group()
    return out


def _selector_stencil_e2e(mspv, torch, dev, params, g):
    """Time-to-1e-10 on the g^3 stencil (b = A 1, x0 = 0): FP64 CG in the tuner's format,
    and FP32-value refinement (FP32-arithmetic inner CG) in the selector's format."""
    n = g ** 3
    r, c, v = synth.stencil27_torch(g, dev)
    A = mspv.Matrix.from_coo(n, n, r, c, v)
    del r, c, v
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    pick = A.select_format(params)
    t_select = time.perf_counter() - t0
    t0 = time.perf_counter()
    tuned, tms = A.tune_format(reps=10)
    t_tune = time.perf_counter() - t0
    res = {"grid": g, "n": n, "nnz": A.info["nnz"], "selector_format": pick, "tuner_format": tuned,
           "tuner_ms_per_spmv": {k: round(x, 5) for k, x in tms.items()},
           "select_s": round(t_select, 4), "tune_s": round(t_tune, 3)}
    M64 = {f: (A if f == "coo" else A.convert(f)) for f in {pick, tuned}}
    Mlo = A.convert(pick, "f32")
    ones = torch.ones(n, dtype=torch.float64, device=dev)
    b = M64[tuned].spmv(ones)
    os.environ["MSPV_CG_CHECK_EVERY"] = "10"

    def timed(fn):
        xx = torch.zeros(n, dtype=torch.float64, device=dev)
        fn(xx)
        xx.zero_()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        out = fn(xx)
        e.record(stream)
        torch.cuda.synchronize()
        err = float((xx - 1.0).abs().max().item())
        return {"ms": round(s.elapsed_time(e), 2), "iters": out.iters, "outer": out.outer_iters,
                "relres": out.relres, "converged": out.converged, "max_abs_err_vs_x1": err}

    res["fp64_cg_tuner_format"] = timed(lambda xx: M64[tuned].cg(b, x=xx, tol=1e-10, maxit=20000))
    if pick != tuned:
        res["fp64_cg_selector_format"] = timed(lambda xx: M64[pick].cg(b, x=xx, tol=1e-10, maxit=20000))
    if Mlo is not None:
        res["ir_f32_values_fp32_inner_selector_format"] = timed(
            lambda xx: M64[pick].cg_ir(Mlo, b, x=xx, tol=1e-10, inner_tol=1e-6, max_outer=30,
                                       maxit_inner=20000, inner_fp32=True))
        res["ru_f32_values_selector_format"] = timed(
            lambda xx: M64[pick].cg_ru(Mlo, b, x=xx, tol=1e-10, maxit=20000))
    return res


# ---------------------------------------------------------------------------
# mixed precision on a large stencil: FP64 CG vs iterative refinement
# ---------------------------------------------------------------------------
MIXED_METRIC = "CG time-to-1e-10 on the 27-point stencil, FP64 vs FP32/BF16-value refinement"


def run_mixed(args, world, rank, local):
    """FP64 CG against FP64-outer iterative refinement with FP32 or BF16 stored values (inner
    CG in FP64 arithmetic, and in FP32 arithmetic), CSR and DIA, on the g^3 stencil with
    b = A 1 from x0 = 0, each to a 1e-10 relative residual; error against x = 1 reported."""
    import torch
    import paper_2304_09511_gb300 as mspv

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    g = args.mixed_grid
    n = g ** 3
    r, c, v = synth.stencil27_torch(g, dev)
    A = mspv.Matrix.from_coo(n, n, r, c, v)
    nnz = A.info["nnz"]
    del r, c, v
    stream = torch.cuda.current_stream()
    os.environ["MSPV_CG_CHECK_EVERY"] = "10"
    ones = torch.ones(n, dtype=torch.float64, device=dev)

    only = {e.strip() for e in args.mixed_only.split(",") if e.strip()}

    class Results(dict):   # drops the solvers --mixed-only leaves out
        def __init__(self, fmt):
            super().__init__()
            self.fmt = fmt

        def run(self, label, fn):
            if not only or f"{self.fmt}:{label}" in only:
                self[label] = timed(fn)

    def timed(fn):
        xx = torch.zeros(n, dtype=torch.float64, device=dev)
        fn(xx)
        xx.zero_()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        s0 = torch.cuda.Event(enable_timing=True)
        e0 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        res = fn(xx)
        e0.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(s0.elapsed_time(e0), world)
        return {"ms": round(ms, 2), "iters": res.iters, "outer": res.outer_iters, "relres": res.relres,
                "converged": res.converged, "max_abs_err_vs_x1": float((xx - 1.0).abs().max().item())}

    clocks = ClockSampler(local)
    clocks.start()
    results = {}
    for fmt in ("csr", "dia"):
        if only and not any(e.startswith(fmt + ":") for e in only):
            continue
        M = A.convert(fmt)
        b = M.spmv(ones)
        out = Results(fmt)
        out.run("fp64_cg", lambda xx: M.cg(b, x=xx, tol=1e-10, maxit=20000))
        for vt in ("f32", "bf16"):
            L = A.convert(fmt, vt)
            out.run(f"ir_{vt}_values_fp64_inner",
                    lambda xx: M.cg_ir(L, b, x=xx, tol=1e-10, inner_tol=1e-5, max_outer=30, maxit_inner=20000))
            out.run(f"ir_{vt}_values_fp32_inner",
                    lambda xx: M.cg_ir(L, b, x=xx, tol=1e-10, inner_tol=args.ir_inner_tol, max_outer=30,
                                       maxit_inner=20000, inner_fp32=True))
            out.run(f"ru_{vt}_values", lambda xx: M.cg_ru(L, b, x=xx, tol=1e-10, maxit=20000))
            L.close()
        if fmt == "dia":   # inner tolerance of the restarted solver, update threshold of the reliable one
            L = A.convert(fmt, "bf16")
            for itol in (1e-3, 1e-4, 1e-5, 1e-7):
                out.run(f"ir_bf16_values_fp32_inner_tol{itol:g}",
                        lambda xx: M.cg_ir(L, b, x=xx, tol=1e-10, inner_tol=itol, max_outer=40,
                                           maxit_inner=20000, inner_fp32=True))
            for d in (0.03, 0.3):
                out.run(f"ru_bf16_values_delta{d:g}",
                        lambda xx: M.cg_ru(L, b, x=xx, tol=1e-10, delta=d, max_updates=200, maxit=20000))
            L.close()
            L = A.convert(fmt, "f32")
            for d in (1e-3, 1e-1):
                out.run(f"ru_f32_values_delta{d:g}",
                        lambda xx: M.cg_ru(L, b, x=xx, tol=1e-10, delta=d, max_updates=200, maxit=20000))
            L.close()
        M.close()
        results[fmt] = dict(out)
    clk = clocks.stop()
    best = min((v["ms"], f, k) for f, o in results.items() for k, v in o.items() if v["converged"])
    out = {"metric": MIXED_METRIC, "value": best[0], "unit": "ms", "higher_is_better": False,
           "n_gpus": world, "mode": "mixed", "scaling": "weak", "data": "synthetic",
           "dtype": "f64 outer; f32/bf16 values", "best": {"format": best[1], "solver": best[2]},
           "config": {"workload": f"27-point stencil {g}^3 (n={n}, nnz={nnz}), b = A 1, x0 = 0, to 1e-10 "
                                  "relative residual; CSR and DIA; FP64 CG vs FP64-outer refinement "
                                  "(restarted, or one FP32 CG with reliable updates) with FP32 or BF16 "
                                  "stored values", "parallelism": f"replicas x{world}"},
           "results": results, "clocks": clk}
    if world > 1:
        torch.distributed.destroy_process_group()
    return out if rank == 0 else None


# ---------------------------------------------------------------------------
# local/remote split of one process's HPCG matrix
# ---------------------------------------------------------------------------
SPLIT_METRIC = "SpMV of one HPCG process's matrix: best single format vs local/remote split (ms)"


def run_split(args, world, rank, local):
    """One interior process of a 3 x 3 x 3 block decomposition of the 27-point problem (all 26
    neighbours), as in the paper's distributed HPCG (Sec. VI): its matrix has a structured
    local part and an unstructured ghost part. Times y = A x for the whole matrix in COO and
    CSR (DIA cannot hold the ghost columns), and for every local format (COO, CSR, DIA) with
    every remote format (COO, CSR): y = A_local x_local, then y += A_remote x_ghost. The
    run-first tuner's choice for each part is reported beside the timings."""
    import torch
    import paper_2304_09511_gb300 as mspv

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream()
    reps = max(args.steps, 10)

    def time_ms(fn):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        e0 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for _ in range(reps):
            fn()
        e0.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(s0.elapsed_time(e0) / reps, world)

    out_sizes = []
    for dims in ((48, 64, 64), (128, 128, 128)):
        r, c, v, n, ng = synth.hpcg_rank_matrix(*dims)
        A = mspv.Matrix.from_coo(n, n + ng, torch.from_numpy(r).to(dev), torch.from_numpy(c).to(dev),
                                 torch.from_numpy(v).to(dev))
        nnz = A.info["nnz"]
        del r, c, v
        x = torch.from_numpy(synth.uniform_x(n + ng, 0)).to(dev)
        xl, xg = x[:n].contiguous(), x[n:].contiguous()
        y = torch.empty(n, dtype=torch.float64, device=dev)
        whole = {"coo": A, "csr": A.convert("csr")}
        res = {"local_block": list(dims), "n": n, "ghosts": ng, "nnz": nnz}
        res["whole_ms"] = {f: round(time_ms(lambda M=M: M.spmv(x, y)), 5) for f, M in whole.items()}
        L0, R0 = A.split_columns(n)
        res["local_nnz"], res["remote_nnz"] = L0.info["nnz"], R0.info["nnz"]
        Ls = {"coo": L0, "csr": L0.convert("csr"), "dia": L0.convert("dia")}
        Rs = {"coo": R0, "csr": R0.convert("csr")}
        split = {}
        for lf, L in Ls.items():
            for rf, R in Rs.items():
                def fn(L=L, R=R):
                    L.spmv(xl, y)
                    R.spmv_add(xg, y)
                split[f"{lf}+{rf}"] = round(time_ms(fn), 5)
        res["split_ms"] = split
        lbest, lms = L0.tune_format(reps=20)
        rbest, rms = R0.tune_format(reps=20)
        res["tuner"] = {"local": lbest, "remote": rbest,
                        "local_ms": {k: round(t, 5) for k, t in lms.items()},
                        "remote_ms": {k: round(t, 5) for k, t in rms.items() if k != "dia"}}
        best_whole = min(res["whole_ms"].items(), key=lambda kv: kv[1])
        best_split = min(split.items(), key=lambda kv: kv[1])
        res["best_whole"] = {"format": best_whole[0], "ms": best_whole[1]}
        res["best_split"] = {"formats": best_split[0], "ms": best_split[1]}
        res["tuned_split_ms"] = split[f"{lbest}+{rbest}"]
        res["speedup_split_vs_whole"] = round(best_whole[1] / best_split[1], 3)
        out_sizes.append(res)
        for M in list(Ls.values()) + list(Rs.values()) + list(whole.values()):
            M.close()
    big = out_sizes[-1]
    out = {"metric": SPLIT_METRIC, "value": big["tuned_split_ms"], "unit": "ms", "higher_is_better": False,
           "n_gpus": world, "mode": "split", "scaling": "weak", "data": "synthetic", "dtype": "f64",
           "config": {"workload": "one interior process (26 neighbours) of a 3x3x3 block decomposition of the "
                                  "27-point problem, local blocks 48x64x64 and 128x128x128; value = tuned "
                                  "local+remote SpMV on the 128^3 block", "reps": reps,
                      "parallelism": f"replicas x{world}"},
           "sizes": out_sizes}
    if world > 1:
        torch.distributed.destroy_process_group()
    return out if rank == 0 else None


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_workload(g):
    import oracle
    n = g ** 3
    rows, cols, vals = synth.stencil27(g)
    # the generator emits canonical COO already (sorted by (row, col), no duplicates)
    O = oracle.Matrix(oracle.COO, n, n, rows.size, ai=rows, aj=cols, av=vals)
    return oracle, n, {"coo": O, "csr": oracle.coo_to_csr(O), "dia": oracle.coo_to_dia(O)}


def oracle_sample(oracle, n, mats, cg_iters):
    """One bounded sample: one SpMV per format and `cg_iters` CG iterations (DIA)."""
    x = synth.uniform_x(n, 0)
    t = {}
    for f in ("coo", "csr", "dia"):
        t0 = time.perf_counter()
        oracle.spmv(mats[f], x)
        t[f] = time.perf_counter() - t0
    b = oracle.spmv(mats["dia"], np.ones(n))
    t0 = time.perf_counter()
    oracle.cg(mats["dia"], b, tol=0.0, maxit=cg_iters)
    t["cg"] = time.perf_counter() - t0
    return t


def cpu_baseline(g, cg_iters):
    """The oracle timed on this host's cores: the parity build on one core, and its OpenMP
    timing copy (-O3; CSR / DIA SpMV rows and CG's vector loops across all cores, COO SpMV
    serial) on every core. The headline value is the all-cores leg."""
    oracle, n, mats = oracle_workload(g)
    nnz = mats["coo"].nnz
    bm = byte_model(n, nnz, mats["dia"].ndiags)
    byts = bm["coo"] + bm["csr"] + bm["dia"] + bm["cg_iter"] * cg_iters + bm["dia"] + 32 * n
    sample = f"{g}^3 stencil: one SpMV per format + {cg_iters} CG iterations (DIA)"

    def leg(t, cores, build):
        secs = sum(t.values())
        return {"value": round(byts / secs / 1e9, 3), "unit": "GB/s", "cores": cores, "build": build,
                "seconds": round(secs, 3),
                "per_format_GB_s": {f: round(bm[f] / t[f] / 1e9, 3) for f in ("coo", "csr", "dia")},
                "cg_ms_per_iter": round(t["cg"] / cg_iters * 1e3, 3)}

    serial = leg(oracle_sample(oracle, n, mats, cg_iters), 1, "parity build: gcc -O2, serial C")
    with oracle.timing_build():
        cores = oracle.threads()
        oracle_sample(oracle, n, mats, 2)   # start the thread team
        all_cores = leg(oracle_sample(oracle, n, mats, cg_iters), cores,
                        "timing copy: gcc -O3 -fopenmp, no -march (one build for x86-64 and AArch64)")
    return {"value": all_cores["value"], "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": sample + f"; all-cores leg ({cores} threads) is the value, serial leg beside it",
            "serial": serial, "all_cores": all_cores}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    oracle, n, mats = oracle_workload(args.grid)
    nnz = mats["coo"].nnz
    bm = byte_model(n, nnz, mats["dia"].ndiags)
    byts = bm["coo"] + bm["csr"] + bm["dia"] + bm["cg_iter"] * args.ref_cg_iters + bm["dia"] + 32 * n
    for _ in range(args.warmup):
        oracle_sample(oracle, n, mats, args.ref_cg_iters)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_sample(oracle, n, mats, args.ref_cg_iters)
    secs = time.perf_counter() - t0
    value = byts * args.steps / secs / 1e9
    sample = (f"{args.grid}^3 stencil: one SpMV per format + {args.ref_cg_iters} CG iterations (DIA) "
              "per step, serial C oracle")
    return {"metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": f"27-point stencil {args.grid}^3 (n={n}, nnz={nnz}), FP64 values, int32 indices; "
                                   "bounded sample of the GPU step (SpMV per format + CG iterations)",
                       "parallelism": "cpu serial"},
            "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["mspv", "reference"], default="mspv")
    ap.add_argument("--grid", type=int, default=GRID)
    ap.add_argument("--cg-iters", type=int, default=CG_ITERS)
    ap.add_argument("--cpu-cg-iters", type=int, default=100,
                    help="CG iterations in the CPU-baseline sample (GPU arm)")
    ap.add_argument("--ir-inner-tol", type=float, default=1e-6,
                    help="inner tolerance of the FP32-arithmetic refinement")
    ap.add_argument("--ref-cg-iters", type=int, default=1,
                    help="CG iterations per step of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tts-large-grid", type=int, default=256,
                    help="step mode: stencil grid of the second time-to-1e-10 block, exact values, FP64 "
                         "CG also in the run-first tuner's format (0 skips it)")
    ap.add_argument("--tts-grid", type=int, default=192,
                    help="step mode: stencil grid of the time-to-1e-10 block, exact and perturbed "
                         "values (0 skips it)")
    ap.add_argument("--mode", choices=["step", "selector", "mixed", "split"], default="step",
                    help="step: the SpMV + CG step (default); selector: tuner labels, MLP "
                         "training and held-out regret, then the stencil end to end; mixed: FP64 "
                         "CG vs FP32/BF16-value refinement on a large stencil; split: one HPCG "
                         "process's matrix, whole vs local/remote formats")
    ap.add_argument("--mixed-grid", type=int, default=192, help="mixed mode: stencil grid")
    ap.add_argument("--mixed-only", default="",
                    help="mixed mode: comma-separated format:solver entries to run (default all), "
                         "e.g. dia:ru_bf16_values")
    ap.add_argument("--matrices", type=int, default=2000, help="selector mode: synthetic matrices")
    ap.add_argument("--tune-reps", type=int, default=10, help="selector mode: timed SpMV per format")
    ap.add_argument("--epochs", type=int, default=300, help="selector mode: training epochs")
    ap.add_argument("--lr", type=float, default=1e-3, help="selector mode: Adam step size")
    ap.add_argument("--e2e-grid", type=int, default=256,
                    help="selector mode: stencil grid of the end-to-end solve (0 skips it)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "mspv":
        args.warmup = 3
    world, rank, local = dist_env()
    if args.impl == "reference":
        out = run_reference(args, world, rank)
    elif args.mode == "selector":
        out = run_selector(args, world, rank, local)
    elif args.mode == "mixed":
        out = run_mixed(args, world, rank, local)
    elif args.mode == "split":
        out = run_split(args, world, rank, local)
    else:
        out = run_mspv(args, world, rank, local)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
