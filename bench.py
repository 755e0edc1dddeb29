"""Benchmark: local stencils/sec of the stencil setup (steps a1-a7) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload helm2d_n1024]
                    [--policy local] [--mode fp64] [--impl ours|reference] [--detail FILE]

One step = one pass of the whole hot path over the workload's potential, resident in HBM:
lsp_set_potential (a1: device copy + v_min/v_max/mean) and lsp_build_stencils (a2-a7: shift
list, per-shift kernel vectors, Gram matrix, near-null vector, and the Q, C, P rows of every
point). The value is points / second (one stencil = the finished Q, C, P rows of one point).
L2 is flushed (256 MiB write) before every timed step, outside the step's events.

The last stdout line is the compact result line (a few KB at most). It carries the headline
(2D n = 1024, per-point shifts, FP64), its roofline, the end-to-end serving loop through the
C ABI with host buffers, the oracle timed on the host cores (one core and all cores), the
clocks seen during the timed region, and one summary per form of the metric (FP64, mixed,
learned at 2D n = 1024 and 3D n = 64). Per-kernel tables, the paper-policy and multi-t
variants and the preconditioner solve go to the --detail file when one is named.

Under torchrun each rank builds the stencils of its own potential (a different seed): the
per-point problems are independent, so ranks share nothing (weak scaling, no collective on
the data path); the step time is the maximum over ranks.

--impl reference times the CPU oracle (numpy/scipy FP64, as it stands) on a bounded sample of
the same workload on all host cores and extrapolates to the whole workload.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "local stencils/sec (Q, C, P rows of every grid point, steps a1-a7)"
LINE_LIMIT = 4096  # bytes of the result line

WORKLOAD_TEXT = {
    "helm2d_n1024": "2D Helmholtz n=1024 (1,048,576 points), 3x3 neighbourhoods, omega=2*pi*256, "
                    "c(x)=1+sum of 64 seeded Gaussians (seed 3)",
    "helm2d_n256": "2D Helmholtz n=256 (65,536 points), 3x3 neighbourhoods, omega=2*pi*64, "
                   "c(x)=1+sum of 16 seeded Gaussians (seed 2)",
    "schr3d_n64": "3D Schroedinger-type n=64 (262,144 points), 3x3x3 neighbourhoods, 8 seeded "
                  "Gaussian wells (seed 4), max|v|h^2=0.6",
    "helm2d_n32": "2D Helmholtz n=32 (1,024 points), 3x3 neighbourhoods, omega=2*pi*8, "
                  "one centred Gaussian bump",
}

# GB300 unit counts for the ALU-bound kernels (152 SMs, 2070 MHz maximum SM clock): the nominal
# FP64 rate, 1.25 TFLOP/s, is 2 FP64 FMA per SM per clock (4 flop); FP32 is 128 FMA lanes per SM
# per clock (256 flop).
SMS, SM_MAX_MHZ = 152, 2070.0
FP64_FLOP_PER_SM_CLK, FP32_FLOP_PER_SM_CLK = 4, 256

# DRAM bytes (read + write) per launch from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum), keyed by (kernel, workload, mode); null where no capture of the
# current kernel exists. The profile named beside each figure holds the command.
TRAFFIC = {
    # profiles/stencil_build_fp64_helm2d_n1024.md: k_stage<1, 3, double, double, 1>, four
    # launches at 2D n = 1024 (per-point shifts): 11.1-11.3 MB read, 0 written
    ("stage1", "helm2d_n1024", "fp64"): 11.2e6,
}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_seed(rank: int):
    """Each rank builds the stencils of its own potential: the workload's seed on rank 0,
    seed 1000 + rank elsewhere (independent problems, no data exchange)."""
    return None if rank == 0 else 1000 + rank


def max_over_ranks(value: float, device: str = "cpu") -> float:
    """The slowest rank's time (the job's time); identity without torch.distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank: int, steps: int, world: int, total_ms: float) -> float:
    """Whole-job stencils/s: all ranks' points over the slowest rank's time."""
    return points_per_rank * steps * world / (total_ms * 1e-3)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return p, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def alu_peak_tflops(fp: str) -> float:
    """FP64 / FP32 peak from the unit counts at the maximum SM clock (TFLOP/s)."""
    per = FP64_FLOP_PER_SM_CLK if fp == "fp64" else FP32_FLOP_PER_SM_CLK
    return per * SMS * SM_MAX_MHZ * 1e6 / 1e12


class Clocks:
    """nvidia-smi samples every 50 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names[1:], parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


def lattice_domain_sizes(m_list: np.ndarray, n: int, d: int) -> list[int]:
    """|E_k| of the lattice-separable stages (host recomputation from the shift list)."""
    p2 = (np.arange(n // 2 + 1, dtype=np.int64)) ** 2
    sizes = [len(m_list)]
    cur = np.asarray(m_list, dtype=np.int64)
    for _ in range(d - 1):
        lo, hi = int(cur.min()), int(cur.max() + p2[-1])
        flags = np.zeros(hi - lo + 1, dtype=bool)
        for p in p2:
            flags[cur + p - lo] = True
        cur = np.nonzero(flags)[0].astype(np.int64) + lo
        sizes.append(len(cur))
    return sizes  # [|E_d| = shifts, |E_{d-1}|, ..., |E_1|]


def kernel_work(name: str, n: int, d: int, N: int, mu: int, sizes: list[int],
                mode: str = "fp64"):
    """Algorithmic (amount, kind) of one launch of a kernel, or None.

    kind: "flop" (FP64 ALU), "tensor_flop" (BF16 tensor cores), "byte" (HBM) or "l2_byte"
    (gathers served by L2: the FP32 stages of the mixed mode)."""
    P = n // 2 + 1
    ncls = {1: 3, 2: 6, 3: 10}
    if name.startswith("stage"):
        if not sizes:
            return None
        k = int(name[-1])
        # stage k runs over E_k; sizes lists E_d, E_{d-1}, ..., so E_k = sizes[d - k]
        count = sizes[d - k]
        if mode == "dword":
            # double-word stages: FP32 operations as written (a double-word multiply-add is
            # 10, a double-word add or subtract 11, a renormalisation 3, every fourth step)
            if k == 1:
                per = (n // 4) * (4 * 11 + 6 * 10 + 6 * 3 / 4) + 2 * 3 * 10
                return count * per, "fp32_op"
            ncls_k = ncls[k]
            return count * P * ncls_k * 2 * (10 + 3 / 4), "fp32_op"
        if mode == "mixed":
            # FP32 stages, counted in FP32 operations as written: stage 1 per mirror pair two
            # squarings, four additions and six fused multiply-adds; later stages one fused
            # multiply-add per class, function and frequency. They are latency-bound on their
            # gathers (ncu), so this fraction is low by nature
            if k == 1:
                return count * ((n // 4) * 12 + 6), "fp32_op"
            return count * P * ncls[k] * 2, "fp32_op"
        if k == 1:
            # mirror-paired: per pair 4 add/sub + 6 FMA (16 flops), plus the middle term (12)
            return count * ((n // 4) * 16 + 12), "flop"
        return count * P * 2 * 2 * ncls[k], "flop"  # 2 functions x one FMA per class
    if name == "rows":
        return N * (8 + 3 * mu * 8), "byte"
    if name == "stats":
        return N * 8, "byte"
    if name == "mlp_rows":
        # the network's dense contractions: (5^d + 1) -> 256 -> 256 -> 256 -> 2|mu|
        nf = 5 ** d + 1
        return N * 2 * (nf * 256 + 2 * 256 * 256 + 256 * 2 * mu), "tensor_flop"
    if name == "mlp_inputs":
        # read the bf16 feature of every point, write the bf16 input tiles (K0 = 32 / 128)
        return N * (2 + (32 if d == 2 else 128) * 2), "byte"
    return None


def roofline(name: str, ms_per_launch: float, work, mode: str, peaks: dict,
             traffic_key=None) -> dict | None:
    """The roofline object of one kernel: algorithmic work per launch over its mean launch
    time, against the peak of the unit that bounds it."""
    if not work or ms_per_launch <= 0:
        return None
    amount, kind = work
    rate = amount / (ms_per_launch * 1e-3)
    if kind == "tensor_flop":
        bound, unit, ach, peak = "tensor", "TFLOP/s", rate / 1e12, peaks["bf16_tflops"]
        src = "bf16_tflops (burst) of measured peaks"
    elif kind == "flop":
        bound, unit, ach, peak = "alu", "TFLOP/s", rate / 1e12, alu_peak_tflops("fp64")
        src = (f"FP64 peak from unit counts: {FP64_FLOP_PER_SM_CLK} flop/SM/clk x {SMS} SMs x "
               f"{SM_MAX_MHZ:.0f} MHz")
    elif kind == "fp32_op":
        bound, unit, ach, peak = "alu", "Top/s", rate / 1e12, FP32_FLOP_PER_SM_CLK / 2 * SMS * SM_MAX_MHZ * 1e6 / 1e12
        src = (f"FP32 issue rate from unit counts: 128 lanes/SM/clk x {SMS} SMs x "
               f"{SM_MAX_MHZ:.0f} MHz")
    elif kind == "l2_byte":
        bound, unit, ach, peak = "l2", "GB/s", rate / 1e9, peaks.get("l2_gbs") or float("nan")
        src = "L2-resident copy (48 MiB, read + write bytes) measured in this run"
    else:
        bound, unit, ach, peak = "hbm", "GB/s", rate / 1e9, peaks["hbm_gbs"]
        src = "hbm_gbs of measured peaks"
    return {"bound": bound, "kernel": name, "achieved": round(ach, 4), "peak": round(peak, 4),
            "unit": unit, "frac": round(ach / peak, 4),
            "traffic": TRAFFIC.get(traffic_key) if traffic_key else None,
            "work_per_launch": amount, "ms_per_launch": round(ms_per_launch, 5),
            "peak_source": src}


def dominant_roofline(ktimes: dict, n: int, d: int, N: int, mu: int, sizes, mode: str,
                      peaks: dict, workload: str):
    """Roofline of the kernel with the largest total time among those with a work count."""
    best = None
    for name, (ms, cnt) in ktimes.items():
        w = kernel_work(name, n, d, N, mu, sizes, mode)
        if w is None:
            continue
        if best is None or ms > best[1]:
            best = (name, ms, cnt, w)
    if best is None:
        return None
    name, ms, cnt, w = best
    return roofline(name, ms / max(cnt, 1), w, mode, peaks, (name, workload, mode))


def measure_l2_gbs(torch) -> float:
    """Copy bandwidth of an L2-resident buffer (48 MiB read + 48 MiB written, best of 20)."""
    a = torch.empty(48 << 20, dtype=torch.uint8, device="cuda").fill_(1)
    b = torch.empty_like(a)
    best = 0.0
    for _ in range(23):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2 * a.numel() / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def measure_fp64_gemm(torch) -> float:
    """FP64 GEMM throughput (TFLOP/s) of the library matmul, best of 5, 4096^3 (context)."""
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    best = 0.0
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        best = max(best, 2 * 4096 ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def run_ours(args):
    import torch

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from lsp_inputs import make_workload
    from paper_1607_02560_gb300 import Context
    from paper_1607_02560_gb300 import build as B

    B.build()
    v_host = make_workload(args.workload, seed=rank_seed(rank), n=args.n)
    d, n = v_host.ndim, v_host.shape[0]
    N = v_host.size
    stream = torch.cuda.Stream()
    ctx = Context(d, n, stream=stream)
    ctx.set_autotune(not args.no_autotune)  # shapes tuned in the first (warm-up) build
    mu = ctx.mu
    v_dev = torch.from_numpy(v_host).to("cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    mlps = {}
    train_info = {}
    if args.mode == "learned" or not args.no_forms:
        for dd in ((d,) if args.mode == "learned" and args.no_forms else (2, 3)):
            mlps[dd], train_info[dd] = train_for(torch, dd, args.learned_steps, stream)
    if args.mode == "learned":
        if args.mlp_schedule is not None:
            mlps[d].set_schedule(args.mlp_schedule)
        ctx.set_mlp(mlps[d])

    def step():
        ctx.set_potential(v_dev)
        ctx.build_stencils(policy=args.policy, mode=args.mode, use_graph=True)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
        ctx.synchronize()
        if ctx.mode_used() == "learned":  # no shift table: the network replaces a2-a6
            ns, m_list = None, None
        else:
            tab = ctx.get_shift_table(with_sidx=False)
            ns = len(tab["s"])
            m_list = np.round((tab["s"] / (np.pi ** 2) - 2) / 4).astype(np.int64)

        # ---- timed region: K steps, graph replay, L2 flushed before each ----
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(local)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            step()
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        total_ms = float(np.sum(step_ms))
        if ws > 1:
            import torch.distributed as dist
            total_ms = max_over_ranks(total_ms, device="cuda")
            dist.barrier()

        # ---- per-kernel timing over K more steps (events around every launch) ----
        ctx.kernel_timing(True)
        for k in range(args.steps):
            flush.zero_()
            step()
        ctx.synchronize()
        ktimes = ctx.kernel_times()
        ctx.kernel_timing(False)

        # ---- end to end through the public API with host buffers ----
        v_pin = torch.empty(v_host.shape, dtype=torch.float64, pin_memory=True)
        v_pin.copy_(torch.from_numpy(v_host))
        outs = [[torch.empty((N, mu), dtype=torch.float64, pin_memory=True).numpy()
                 for _ in range(3)] for _ in range(2)]
        e2e_steps = max(3, args.steps // 2)
        # (a) one step at a time: v in, build, the three row blocks out, waited for
        e2e_ms = []
        for k in range(e2e_steps + 1):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            ctx.set_potential(v_pin.numpy())
            ctx.build_stencils(policy=args.policy, mode=args.mode, use_graph=True)
            for which, o in zip("QCP", outs[0]):
                ctx.get_rows(which, o)
            e2e_ms.append((time.perf_counter() - t1) * 1e3)
        e2e_ms = e2e_ms[1:]

        # (b) serving loop: step k's rows go to the host (get_rows_async, the library's copy
        # stream) while step k + 1 builds; two host buffer sets alternate. The L2 flush runs
        # inside the timed region, and the region ends when the last step's rows have landed.
        def serve(k):
            flush.zero_()
            ctx.set_potential(v_pin.numpy())
            ctx.build_stencils(policy=args.policy, mode=args.mode, use_graph=True)
            for which, o in zip("QCP", outs[k & 1]):
                ctx.get_rows_async(which, o)
        serve(0)
        serve(1)
        ctx.wait_rows()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for k in range(e2e_steps):
            serve(k)
        ctx.wait_rows()
        torch.cuda.synchronize()
        serve_ms = (time.perf_counter() - t1) * 1e3 / e2e_steps

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    value = job_throughput(N, args.steps, ws, total_ms)
    peaks, peak_src = load_peaks()
    peaks = dict(peaks, l2_gbs=measure_l2_gbs(torch))
    sizes = lattice_domain_sizes(m_list, n, d) if m_list is not None else []
    launches = int(sum(c for _, c in ktimes.values()))
    kern = {}
    for name, (ms, cnt) in ktimes.items():
        kern[name] = {"ms_per_launch": ms / max(cnt, 1), "launches": cnt}
        r = roofline(name, ms / max(cnt, 1), kernel_work(name, n, d, N, mu, sizes, args.mode),
                     args.mode, peaks)
        if r:
            kern[name].update(achieved=r["achieved"], unit=r["unit"], frac=r["frac"])
    roof = dominant_roofline(ktimes, n, d, N, mu, sizes, args.mode, peaks, args.workload)
    rows_k = ktimes.get("rows")
    rows_roof = (roofline("rows", rows_k[0] / max(rows_k[1], 1),
                          kernel_work("rows", n, d, N, mu, sizes), args.mode, peaks,
                          ("rows", args.workload, args.mode)) if rows_k else None)
    used = ctx.mode_used()
    tun = ctx.tuning()
    ctx.close()
    res = {
        "metric": METRIC,
        "value": value, "unit": "stencils/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "dword": "f32x2+f64", "mixed": "f32+f64",
                  "learned": "bf16+f32"}[args.mode],
        "data": "synthetic",
        "config": {"workload": args.workload, "policy": args.policy, "mode": args.mode,
                   "mode_used": used, "d": d, "n": n, "points": N, "shifts": ns,
                   "l2": "flushed before every timed step (256 MiB write), outside the step events",
                   "parallelism": f"replicas x{ws} (independent potentials)",
                   "autotune": tuning_summary(tun)},
        "roofline": roof,
        "rows_roofline": rows_roof,
        "gpu_launches": launches,
        "wall_s_timed_region": round(wall, 4),
        "clocks": clk,
        "e2e": {"value": N / (serve_ms * 1e-3), "unit": "stencils/s",
                "h2d_bytes_per_step": int(N * 8), "d2h_bytes_per_step": int(3 * N * mu * 8),
                "ms_per_step": serve_ms,
                "loop": "set_potential from pinned host v, build, get_rows_async of Q, C, P "
                        "into pinned host memory overlapping the next build; ends when the "
                        "last rows land",
                "one_step_at_a_time": {"value": N / (float(np.median(e2e_ms)) * 1e-3),
                                       "ms_per_step": float(np.median(e2e_ms))}},
    }
    detail = {"kernels": kern, "lattice_domains": sizes, "peak_source": peak_src, "tuning": tun,
              "workload_text": WORKLOAD_TEXT.get(args.workload, "")}
    if train_info:
        detail["training"] = {str(k): v for k, v in train_info.items()}
    if ws == 1 and not args.no_forms:
        res["forms"], detail["forms"] = forms_block(args, torch, mlps, peaks)
    if ws == 1 and args.detail:
        fp64_gemm = measure_fp64_gemm(torch)
        detail["fp64_gemm_tflops"] = fp64_gemm
        detail["variants"] = variants(args, torch, peaks)
        if not args.no_solve:
            detail["nd_solve"] = solve_block(args, torch, fp64_gemm, peaks["hbm_gbs"])
    for m in mlps.values():
        m.close()
    if ws == 1 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_baseline(args.workload, args.policy, args.cpu_budget)
    if args.detail:
        detail["result"] = res
        with open(args.detail, "w") as fh:
            json.dump(detail, fh, indent=1)
        res["detail"] = os.path.basename(args.detail)
    print(contract_line(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def tuning_summary(tun: dict) -> dict:
    """{kernel: "threads x CTAs/SM, gain"} for the tuned kernels that take at least 10 us."""
    out = {}
    for key, (th, ps, md, mb) in tun.items():
        if md >= 0.01:
            out[key.split("/")[0]] = f"{th}x{ps} {md / mb:.2f}x"
    return out


def _r(x, nd=4):
    """Round to nd significant digits (keeps the result line short)."""
    if x is None or not isinstance(x, (int, float)) or x == 0 or not np.isfinite(x):
        return x
    return float(f"{x:.{nd}g}")


def contract_line(res: dict) -> str:
    """The one-line JSON result: the contract keys, compact, below LINE_LIMIT bytes."""
    keep_roof = ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic", "peak_source")
    out = {k: res[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup",
                               "ms_per_step", "higher_is_better", "scaling", "vs_baseline",
                               "dtype", "data", "config") if k in res}
    out["value"] = _r(out.get("value"), 6)
    out["ms_per_step"] = _r(out.get("ms_per_step"), 6)
    if res.get("roofline"):
        out["roofline"] = {k: (_r(v) if isinstance(v, float) else v)
                           for k, v in res["roofline"].items() if k in keep_roof}
    if res.get("rows_roofline"):
        r = res["rows_roofline"]
        out["rows_roofline"] = {k: _r(r[k]) for k in ("achieved", "peak", "frac")} | {
            "unit": r["unit"], "traffic": r.get("traffic")}
    for k in ("gpu_launches", "clocks"):
        if k in res:
            out[k] = res[k]
    if "e2e" in res:
        e = res["e2e"]
        out["e2e"] = {"value": _r(e["value"], 6), "unit": e["unit"],
                      "h2d_bytes_per_step": e["h2d_bytes_per_step"],
                      "d2h_bytes_per_step": e["d2h_bytes_per_step"],
                      "ms_per_step": _r(e["ms_per_step"]), "loop": e.get("loop", "")[:160]}
        if "one_step_at_a_time" in e:
            out["e2e"]["one_step_at_a_time"] = _r(e["one_step_at_a_time"]["value"])
    if "cpu_baseline" in res:
        c = res["cpu_baseline"]
        out["cpu_baseline"] = {"value": _r(c["value"]), "unit": c["unit"], "cores": c["cores"],
                               "kind": c["kind"], "sample": c["sample"][:240]}
        if c.get("single_core"):
            s = c["single_core"]
            out["cpu_baseline"]["single_core"] = {"value": _r(s["value"]), "cores": s["cores"]}
    if res.get("forms"):
        out["forms"] = [{k: (_r(v) if isinstance(v, float) else v) for k, v in f.items()}
                        for f in res["forms"]]
    for k in ("detail", "impl"):
        if k in res:
            out[k] = res[k]
    line = json.dumps(out, separators=(",", ":"))
    if len(line.encode()) > LINE_LIMIT:  # drop the optional parts, never the contract keys
        for k in ("forms", "rows_roofline"):
            out.pop(k, None)
            line = json.dumps(out, separators=(",", ":"))
            if len(line.encode()) <= LINE_LIMIT:
                break
    return line


FORMS = [("helm2d_n1024", "fp64"), ("helm2d_n1024", "dword"), ("helm2d_n1024", "mixed"),
         ("helm2d_n1024", "learned"),
         ("schr3d_n64", "fp64"), ("schr3d_n64", "mixed"), ("schr3d_n64", "learned")]


def forms_block(args, torch, mlps, peaks):
    """stencils/s and the dominant kernel's roofline fraction of FP64, mixed and learned at
    2D n = 1024 and 3D n = 64 (per-point shifts), on the same GPU, same step definition."""
    short, full = [], []
    for wl, mode in FORMS:
        d = 2 if wl.startswith("helm2d") else 3
        try:
            r = time_config(torch, wl, args.policy, mode, steps=20, warmup=3, peaks=peaks,
                            mlp=mlps.get(d) if mode == "learned" else None)
        except Exception as exc:  # a form must not hide the main line
            short.append({"workload": wl, "mode": mode, "error": str(exc)[:120]})
            full.append(short[-1])
            continue
        full.append(r)
        roof = r.get("roofline") or {}
        s = {"workload": wl, "mode": mode, "mode_used": r["mode_used"], "value": r["value"],
             "ms": r["ms_per_step"], "kernel": roof.get("kernel"), "bound": roof.get("bound"),
             "frac": roof.get("frac")}
        if "quality" in r:
            s.update(r["quality"])
        short.append(s)
    return short, full


def time_config(torch, workload: str, policy: str, mode: str, steps: int, warmup: int,
                mlp=None, stream=None, t: int = 1, nd_leaf: int = 0, peaks=None,
                gmres: bool = True, autotune: bool = True):
    """stencils/s of one configuration (same step, L2 flush and events as the main line)."""
    from lsp_inputs import make_workload
    from paper_1607_02560_gb300 import Context

    v = make_workload(workload)
    d, n, N = v.ndim, v.shape[0], v.size
    stream = stream or torch.cuda.Stream()
    ctx = Context(d, n, stream=stream)
    ctx.set_autotune(autotune)
    if mlp is not None:
        ctx.set_mlp(mlp)
    v_dev = torch.from_numpy(v).to("cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    kw = dict(policy=policy, mode=mode, use_graph=True, t=t, nd_leaf=nd_leaf)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            ctx.set_potential(v_dev)
            ctx.build_stencils(**kw)
        ctx.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.set_potential(v_dev)
            ctx.build_stencils(**kw)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        used = ctx.mode_used()
        m_list, ns = None, None
        if used != "learned":
            s = ctx.get_shift_table(with_sidx=False)["s"]
            ns = len(s)
            m_list = np.round((s / (np.pi ** 2) - 2) / 4).astype(np.int64)
        out = {"workload": workload, "policy": policy, "mode": mode, "mode_used": used, "t": t,
               "nd_leaf": nd_leaf, "value": N * steps / (tot * 1e-3), "unit": "stencils/s",
               "ms_per_step": tot / steps, "shifts": ns}
        if used == "learned":
            out["quality"] = learned_quality(torch, ctx, v, v_dev, policy, flush, stream, gmres)
            ctx.build_stencils(**kw)
        ctx.kernel_timing(True)
        for _ in range(5):
            flush.zero_()
            ctx.set_potential(v_dev)
            ctx.build_stencils(**kw)
        ctx.synchronize()
        kt = ctx.kernel_times()
        ctx.kernel_timing(False)
    out["tuning"] = ctx.tuning()
    ctx.close()
    mu = (2 * t + 1) ** d
    out["kernel_ms_per_launch"] = {k: round(ms / max(cnt, 1), 4) for k, (ms, cnt) in kt.items()}
    if peaks is not None and t == 1:
        sizes = lattice_domain_sizes(m_list, n, d) if m_list is not None else []
        out["roofline"] = dominant_roofline(kt, n, d, N, mu, sizes, used, peaks, workload)
    return out


GATE_TAU = 1.003  # residual ratio above which a learned stencil takes the eigen path's rows


def learned_quality(torch, ctx, v, v_dev, policy: str, flush, stream, gmres: bool = True) -> dict:
    """What the learned stencils are worth against the eigen path, on this potential:
    |d alpha| per point against the FP64 build; the per-point residual gate at tau = GATE_TAU
    (its build time, the fraction of points sent back to the eigen path, and the residual
    ratio rho = ||alpha^T G[mu, mu^c]|| / sigma_min of the network's stencils); and the GMRES
    count (the library's nested-dissection factorisation of P and GMRES(40), rtol 1e-6, on a
    Gaussian point source) with the ungated, gated and FP64 rows."""
    from lsp_inputs import gaussian_source

    N = v.size
    ctx.build_stencils(policy=policy, mode="learned")
    q_learned = ctx.get_rows("Q").copy()
    ctx.build_stencils(policy=policy, mode="fp64")
    err = np.abs(q_learned - ctx.get_rows("Q")).max(axis=1)  # per point
    out = {"dalpha_p50": float(np.percentile(err, 50)), "dalpha_p99": float(np.percentile(err, 99)),
           "dalpha_max": float(err.max()), "gate_tau": GATE_TAU}
    kw = dict(policy=policy, mode="learned", learned_gate=GATE_TAU, use_graph=True)
    for _ in range(3):
        ctx.build_stencils(**kw)
    ctx.synchronize()
    tot, reps = 0.0, 10
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.set_potential(v_dev)
        ctx.build_stencils(**kw)
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    nfall, rho = ctx.gate_stats()
    out.update({"gated_value": N * reps / (tot * 1e-3), "gated_ms": tot / reps,
                "fallback_frac": nfall / N, "rho_p50": float(np.percentile(rho, 50)),
                "rho_p99": float(np.percentile(rho, 99)), "rho_max": float(rho.max())})
    if gmres:
        f = gaussian_source(v.shape[0], v.ndim, 2.0).reshape(-1)
        its = {}
        for tag, bkw in (("gmres_gated", kw), ("gmres_learned", dict(policy=policy, mode="learned")),
                         ("gmres_fp64", dict(policy=policy, mode="fp64"))):
            try:
                ctx.build_stencils(**bkw)
                ctx.nd_factor()
                _, res = ctx.gmres(f, max_cycles=25)
                its[tag] = int(res["iterations"]) if res["converged"] else -int(res["iterations"])
            except Exception as exc:  # the solve must not hide the timing
                its[tag] = str(exc)[:80]
        out.update(its)
    return out


def train_for(torch, d: int, steps: int, stream):
    """Train the surrogate on training potentials that none of the timed workloads uses: in 2D
    8 seeds (100-107) of the n = 256 generator and 8 seeds (108-115) of the n = 1024 one, in 3D
    16 seeds (100-115) of the n = 64 generator."""
    from lsp_inputs import make_workload
    from paper_1607_02560_gb300.learned import train_surrogate

    if d == 2:
        pots = ([make_workload("helm2d_n256", seed=s) for s in range(100, 108)]
                + [make_workload("helm2d_n1024", seed=s) for s in range(108, 116)])
        seeds = "helm2d_n256 100-107 + helm2d_n1024 108-115"
    else:
        pots = [make_workload("schr3d_n64", seed=s) for s in range(100, 116)]
        seeds = "schr3d_n64 100-115"
    t0 = time.time()
    with torch.cuda.stream(stream):
        mlp, losses = train_surrogate(d, pots, samples_per_potential=65536, steps=steps,
                                      batch=4096, lr=2e-3, stream=stream)
    torch.cuda.synchronize()
    info = {"potentials": len(pots), "seeds": seeds, "pairs": len(pots) * 65536,
            "steps": steps, "batch": 4096, "seconds": round(time.time() - t0, 2),
            "final_loss": float(np.mean(losses[-50:]))}
    return mlp, info


def solve_variant(torch, n: int, policy: str = "paper", fp64_peak: float | None = None,
                  hbm_peak: float | None = None, d: int = 2):
    """Applying the preconditioner (Sec. 5 tables): nested-dissection setup T_NDsetup, one
    application T_NDapp, and the GMRES(40) solve to rtol 1e-6 (T_NDsolve, N_iter). 2D: the
    velocity field of a Gaussian profile at the centre, 4 points per wavelength, n x n grid;
    3D: the Schroedinger-type potential of randomly placed Gaussian wells, n^3 grid."""
    from lsp_inputs import gaussian_source, make_workload
    from paper_1607_02560_gb300 import Context

    wl = "helm2d_n32" if d == 2 else "schr3d_n64"
    v = make_workload(wl, n=n)
    f = gaussian_source(n, d, 2.0).reshape(-1)
    stream = torch.cuda.Stream()
    ctx = Context(d, n, stream=stream)
    text = f"(omega/2pi = {n // 4})" if d == 2 else "(max|v| h^2 = 0.6)"
    out = {"workload": f"{wl} rescaled to n={n} {text}", "policy": policy, "d": d, "n": n}
    with torch.cuda.stream(stream):
        ctx.set_potential(v)
        ctx.build_stencils(policy=policy)
        t0 = time.perf_counter()
        ctx.nd_factor()  # plans the dissection on the host, then factorises
        out["nd_setup_first_call_s"] = time.perf_counter() - t0
        reps = 3 if out["nd_setup_first_call_s"] < 2.0 else 1
        setup = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.nd_factor()
            setup.append(time.perf_counter() - t0)
        info = ctx.nd_info()
        y = torch.from_numpy(np.random.default_rng(0).standard_normal(v.size)).cuda()
        x = torch.empty_like(y)
        torch.cuda.synchronize()
        for _ in range(3):
            ctx.nd_solve(y, x)
        ctx.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(20)]
        for a, b in evs:
            a.record(stream)
            ctx.nd_solve(y, x)
            b.record(stream)
        torch.cuda.synchronize()
        app_ms = float(np.median([a.elapsed_time(b) for a, b in evs]))
        ctx.kernel_timing(True)
        if reps > 1:
            ctx.nd_factor()
        for _ in range(5):
            ctx.nd_solve(y, x)
        ctx.synchronize()
        kt = {k: {"ms": round(ms, 4), "launches": cnt} for k, (ms, cnt) in ctx.kernel_times().items()}
        ctx.kernel_timing(False)
        fd = torch.from_numpy(f).cuda()
        torch.cuda.synchronize()
        ctx.gmres(fd)  # warm
        gm = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ud, res = ctx.gmres(fd)
            gm.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        _, res_h = ctx.gmres(f)  # host buffers in and out
        e2e = time.perf_counter() - t0
    ctx.close()
    setup_s = float(np.median(setup))
    out.update({
        "T_NDsetup_s": setup_s, "T_NDapp_ms": app_ms, "N_iter": res["iterations"],
        "T_NDsolve_s": float(np.median(gm)), "T_NDsolve_host_buffers_s": e2e,
        "converged": res["converged"], "resid_true": res["resid_true"],
        "fronts": info["fronts"], "levels": info["levels"], "max_front": info["max_front"],
        "front_bytes": info["front_bytes"], "flops_lu": info["flops_lu"],
        "flops_issued": info["flops"], "solve_bytes": info["solve_bytes"],
        "kernel_ms": kt})
    if fp64_peak:
        ach = info["flops_lu"] / setup_s / 1e12
        out["setup_roofline"] = {"bound": "fp64", "achieved": ach, "peak": fp64_peak,
                                 "unit": "TFLOP/s", "frac": ach / fp64_peak,
                                 "work": "multifrontal LU count 2/3 s^3 + 2 s^2 r + 2 s r^2 per front"}
    if hbm_peak:
        ach = info["solve_bytes"] / (app_ms * 1e-3) / 1e9
        out["solve_roofline"] = {"bound": "hbm", "achieved": ach, "peak": hbm_peak,
                                 "unit": "GB/s", "frac": ach / hbm_peak,
                                 "work": "front bytes read per solve, (f s + s r) * 8 per front"}
    return out


def solve_block(args, torch, fp64_peak, hbm_peak):
    """The nested-dissection / GMRES measurements at the 2D and 3D sizes asked for."""
    res = []
    for d, sizes in ((2, args.solve_n), (3, args.solve_n3)):
        for n in (int(x) for x in sizes.split(",") if x):
            try:
                res.append(solve_variant(torch, n, "paper", fp64_peak, hbm_peak, d=d))
            except Exception as exc:  # must not hide the main line
                res.append({"d": d, "n": n, "error": str(exc)[:300]})
    return res


def run_solve_only(args):
    """The nested-dissection / GMRES block alone (one JSON line), for profiling runs."""
    import torch
    from paper_1607_02560_gb300 import build as B

    B.build()
    torch.cuda.set_device(0)
    peaks, _ = load_peaks()
    fp64_peak = measure_fp64_gemm(torch)
    out = {"metric": "nested dissection setup / solve", "n_gpus": 1,
           "nd_solve": solve_block(args, torch, fp64_peak, peaks["hbm_gbs"])}
    print(json.dumps(out))


def variants(args, torch, peaks):
    """The paper's shift policy and multi-t builds on the same GPU (detail file only)."""
    out = []
    for wl, pol, mode in [("helm2d_n1024", "paper", "fp64"), ("helm2d_n1024", "paper", "mixed"),
                          ("schr3d_n64", "paper", "fp64")]:
        try:
            out.append(time_config(torch, wl, pol, mode, steps=20, warmup=3, peaks=peaks))
        except Exception as exc:  # a variant must not hide the main line
            out.append({"workload": wl, "policy": pol, "mode": mode, "error": str(exc)[:200]})
    # multi-t (Sec. 4.2): t_j from a nested dissection with leaf boxes of width 8, t_max = 2
    for wl, pol in (("helm2d_n1024", "paper"), ("helm2d_n256", "local"), ("schr3d_n64", "local")):
        try:
            out.append(time_config(torch, wl, pol, "fp64", steps=20, warmup=3, t=2, nd_leaf=8))
        except Exception as exc:
            out.append({"workload": wl, "policy": pol, "t": 2, "error": str(exc)[:200]})
    return out


# ---- the oracle on the host cores ----------------------------------------------------------

def _oracle_shifts(job):
    """Worker task: the oracle's per-shift stencil (a3-a6) for each shift of the job."""
    n, d, shifts = job
    import oracle as O

    t0 = time.perf_counter()
    for s in shifts:
        O.stencil_for_shift(n, d, float(s))
    return time.perf_counter() - t0


class OracleSampler:
    """The oracle, as it stands, timed on `threads` host processes on a bounded sample.

    The shift list, the per-point shift assignment and the row assembly of every point (the
    oracle's build_stencils with no shift solved but one) run once in this process; the
    per-shift solves of a seeded sample of shifts run on `threads` worker processes (started
    with spawn, one numpy/BLAS thread each), and the wall time per shift extrapolates to the
    whole shift list."""

    def __init__(self, workload: str, policy: str, threads: int):
        import concurrent.futures as cf
        import multiprocessing as mp

        self.workload, self.policy, self.threads = workload, policy, threads
        self.ex = None
        if threads > 1:
            self.ex = cf.ProcessPoolExecutor(max_workers=threads,
                                             mp_context=mp.get_context("spawn"))

    def close(self):
        if self.ex is not None:
            self.ex.shutdown()

    def sample(self, budget_s: float, seed: int = 0) -> dict:
        import oracle as O
        from lsp_inputs import make_workload

        v = make_workload(self.workload)
        n, d = v.shape[0], v.ndim
        t0 = time.perf_counter()
        st = O.build_stencils(v, self.policy, shift_subset=[0])  # shift list + s_j + rows
        t_rows = time.perf_counter() - t0
        S = st["S"]
        ns = len(S)
        order = np.random.default_rng(100 + seed).permutation(ns)
        done, wall = 0, 0.0
        if self.ex is None:
            while done < ns and (done == 0 or wall + t_rows < budget_s):
                wall += _oracle_shifts((n, d, [S[order[done]]]))
                done += 1
        else:
            per = 2  # shifts per task
            if seed == 0 or not getattr(self, "_warm", False):  # import the oracle in workers
                list(self.ex.map(_oracle_shifts, [(n, d, [S[order[0]]])] * self.threads))
                self._warm = True
            while done < ns and (done == 0 or wall + t_rows < budget_s):
                batch = order[done:done + self.threads * per]
                jobs = [(n, d, [S[i] for i in batch[k:k + per]]) for k in range(0, len(batch), per)]
                t1 = time.perf_counter()
                list(self.ex.map(_oracle_shifts, jobs))
                wall += time.perf_counter() - t1
                done += len(batch)
        per_shift = wall / max(done, 1)
        total = t_rows + per_shift * ns
        return {"value": v.size / total, "unit": "stencils/s", "cores": self.threads,
                "kind": "oracle", "seconds": wall + t_rows,
                "sample": f"{done} of {ns} seeded shifts on {self.threads} process(es), "
                          f"{per_shift * 1e3:.1f} ms wall per shift, + shift assignment and row "
                          f"assembly of all {v.size} points ({t_rows:.2f} s, one core); "
                          + ("all shifts" if done == ns else "extrapolated to all shifts")}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def thread_env(threads: int = 1) -> dict:
    """Environment that fixes the numpy/BLAS thread count of a fresh interpreter."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
              "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS"):
        env[k] = str(threads)
    return env


def cpu_baseline(workload: str, policy: str, budget_s: float = 15.0) -> dict:
    """The oracle on one host core and on all host cores, each in a fresh interpreter whose
    numpy/BLAS thread count is fixed before numpy loads."""
    res = {}
    for label, procs in (("single_core", 1), ("all", host_cores())):
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-only",
               "--workload", workload, "--policy", policy, "--cpu-procs", str(procs),
               "--cpu-budget", str(budget_s)]
        p = subprocess.run(cmd, env=thread_env(1), capture_output=True, text=True,
                           timeout=budget_s * 6 + 120)
        lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
        if p.returncode != 0 or not lines:
            res[label] = {"error": (p.stderr or "no output")[-200:]}
            continue
        res[label] = json.loads(lines[-1])
    main = res.get("all", {})
    if "value" not in main:
        main = res.get("single_core", {})
    out = dict(main)
    if "value" in res.get("single_core", {}) and res["single_core"] is not main:
        out["single_core"] = res["single_core"]
    return out


def run_cpu_only(args):
    s = OracleSampler(args.workload, args.policy, args.cpu_procs)
    try:
        r = s.sample(args.cpu_budget)
    finally:
        s.close()
    print(json.dumps(r))


def run_reference(args):
    """The reference arm: the oracle as it stands on all host cores, one bounded sample of the
    workload per step; rank 0 alone runs and prints."""
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    if os.environ.get("OMP_NUM_THREADS") != "1":
        # fix numpy/BLAS threads before numpy loads: re-run this arm in a fresh interpreter
        p = subprocess.run([sys.executable, *sys.argv], env=thread_env(1))
        sys.exit(p.returncode)
    procs = args.cpu_procs or host_cores()
    sampler = OracleSampler(args.workload, args.policy, procs)
    vals = []
    try:
        for k in range(args.warmup + args.steps):
            cb = sampler.sample(max(0.2, args.ref_step_s), seed=k)
            if k >= args.warmup:
                vals.append(cb)
    finally:
        sampler.close()
    value = float(np.median([c["value"] for c in vals]))
    out = {"impl": "reference", "metric": METRIC,
           "value": value, "unit": "stencils/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup,
           "ms_per_step": float(np.mean([c["seconds"] for c in vals])) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "policy": args.policy, "mode": "fp64"},
           "cpu_baseline": {"value": value, "unit": "stencils/s", "cores": procs,
                            "kind": "oracle", "sample": "per step: " + vals[-1]["sample"]},
           "e2e": {"value": value, "unit": "stencils/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out, separators=(",", ":")))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="helm2d_n1024")
    ap.add_argument("--policy", default="local", choices=["local", "paper", "mean"])
    ap.add_argument("--mode", default="fp64", choices=["fp64", "dword", "mixed", "learned"])
    ap.add_argument("--learned-steps", type=int, default=3000,
                    help="training steps of the surrogate (learned mode and forms)")
    ap.add_argument("--mlp-schedule", type=int, default=None, choices=[0, 1, 2],
                    help="2D network kernel: 1 = two tiles in flight (default), 0 = one tile, "
                         "2 = two 256-row tiles on a CTA pair")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the FP64 / mixed / learned summaries at 2D n=1024 and 3D n=64")
    ap.add_argument("--detail", default="",
                    help="write per-kernel tables, variants and the preconditioner solve here")
    ap.add_argument("--no-solve", action="store_true",
                    help="skip the nested-dissection / GMRES measurements of --detail")
    ap.add_argument("--solve-n", default="256,512,1024",
                    help="grid sizes of the nested-dissection / GMRES measurements")
    ap.add_argument("--solve-n3", default="16,32",
                    help="3D grid sizes of the nested-dissection / GMRES measurements")
    ap.add_argument("--solve-only", action="store_true",
                    help="print only the nested-dissection / GMRES measurements (profiling)")
    ap.add_argument("--n", type=int, default=None, help="rescale the workload's grid (small cases)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (no tuning pass in the warm-up)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cpu-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-procs", type=int, default=0, help="host processes of the oracle")
    ap.add_argument("--ref-step-s", type=float, default=3.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.cpu_only:
        args.cpu_procs = max(1, args.cpu_procs)
        run_cpu_only(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.solve_only:
        run_solve_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
