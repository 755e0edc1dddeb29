"""Benchmark: local stencils/sec of the stencil setup (steps a1-a7) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload helm2d_n1024]
                    [--policy local] [--impl ours|reference]

One step = one pass of the whole hot path over the workload's potential, resident in HBM:
lsp_set_potential (a1: device copy + v_min/v_max/mean) and lsp_build_stencils (a2-a7: shift
list, per-shift kernel vectors, Gram matrix, near-null vector, and the Q, C, P rows of every
point). The value is points / second (one stencil = the finished Q, C, P rows of one point).
L2 is flushed (256 MiB write) before every timed step, outside the step's events.

Under torchrun each rank builds the stencils of its own potential (a different seed): the
per-point problems are independent, so ranks share nothing (weak scaling, no collective on
the data path); the step time is the maximum over ranks.

--impl reference times the CPU oracle (numpy/scipy FP64) on a bounded sample of the same
workload on the host cores and extrapolates to the whole workload.
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


def kernel_work(name: str, n: int, d: int, N: int, mu: int, sizes: list[int]):
    """Algorithmic (flops or bytes, unit) of one launch of a kernel, or None."""
    P = n // 2 + 1
    ncls = {1: 3, 2: 6, 3: 10}
    if name.startswith("stage"):
        k = int(name[-1])
        # stage k runs over E_k; sizes lists E_d, E_{d-1}, ..., so E_k = sizes[d - k]
        count = sizes[d - k]
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


def measure_fp64_peak(torch) -> float:
    """FP64 GEMM throughput (TFLOP/s) of the library matmul, best of 5, 4096^3."""
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
    mu = ctx.mu
    v_dev = torch.from_numpy(v_host).to("cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    mlp = None
    train_info = None
    if args.mode == "learned":
        mlp, train_info = train_for(torch, args.workload, args.learned_steps, stream)
        ctx.set_mlp(mlp)

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
    sizes = lattice_domain_sizes(m_list, n, d) if m_list is not None else []
    launches = int(sum(c for _, c in ktimes.values()))
    kern = {}
    for name, (ms, cnt) in ktimes.items():
        w = kernel_work(name, n, d, N, mu, sizes)
        kern[name] = {"ms_per_launch": ms / max(cnt, 1), "launches": cnt}
        if w:
            per = w[0] / (ms / max(cnt, 1) * 1e-3)
            flops = w[1] in ("flop", "tensor_flop")
            kern[name]["achieved"] = per / (1e12 if flops else 1e9)
            kern[name]["unit"] = "TFLOP/s" if flops else "GB/s"
    dom = max(ktimes.items(), key=lambda kv: kv[1][0])[0]
    fp64_peak = measure_fp64_peak(torch)
    w = kernel_work(dom, n, d, N, mu, sizes)
    if w and w[1] == "tensor_flop":
        roof = {"bound": "tensor", "kernel": dom, "achieved": kern[dom]["achieved"],
                "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
                "frac": kern[dom]["achieved"] / peaks["bf16_tflops"], "traffic": None,
                "peak_source": f"MEASURED_PEAKS.json bf16_tflops, burst ({peak_src})",
                "work_per_launch": w[0]}
    elif w and w[1] == "flop":
        roof = {"bound": "alu", "kernel": dom, "achieved": kern[dom]["achieved"],
                "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": kern[dom]["achieved"] / fp64_peak, "traffic": None,
                "peak_source": "FP64 DGEMM (torch.matmul 4096^3, best of 6) measured in this "
                               "run; FP64 ALU, nominal 1.25 TFLOP/s on GB300",
                "work_per_launch": w[0]}
    elif w:
        roof = {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["achieved"],
                "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": kern[dom]["achieved"] / peaks["hbm_gbs"], "traffic": None,
                "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                "work_per_launch": w[0]}
    else:
        roof = None
    rows_k = kern.get("rows")
    out = {
        "metric": METRIC,
        "value": value, "unit": "stencils/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "mixed": "f32+f64", "learned": "bf16+f32"}[args.mode],
        "data": "synthetic",
        "config": {"workload": args.workload, "text": WORKLOAD_TEXT.get(args.workload, ""),
                   "policy": args.policy, "mode": args.mode, "d": d, "n": n, "points": N,
                   "shifts": ns, "lattice_domains": sizes, "mode_used": ctx.mode_used(),
                   "l2": "flushed before every timed step (256 MiB write), outside the step events",
                   "parallelism": f"replicas x{ws} (independent potentials)"},
        "roofline": roof,
        "hbm_roofline_rows": ({"achieved": rows_k["achieved"], "peak": peaks["hbm_gbs"],
                               "frac": rows_k["achieved"] / peaks["hbm_gbs"], "unit": "GB/s"}
                              if rows_k and "achieved" in rows_k else None),
        "kernels": kern,
        "gpu_launches": launches,
        "wall_s_timed_region": wall,
        "clocks": clk,
        "e2e": {"value": N / (serve_ms * 1e-3), "unit": "stencils/s",
                "h2d_bytes_per_step": int(N * 8), "d2h_bytes_per_step": int(3 * N * mu * 8),
                "ms_per_step": serve_ms,
                "loop": "set_potential from pinned host memory, build, get_rows_async of Q, C, "
                        "P into pinned host memory (step k's copies overlap step k + 1's "
                        "build); L2 flush inside the region; ends after the last copy landed",
                "one_step_at_a_time": {"value": N / (float(np.median(e2e_ms)) * 1e-3),
                                       "ms_per_step": float(np.median(e2e_ms)),
                                       "loop": "each step's host copies waited for before "
                                               "the next step starts (get_rows)"}},
    }
    if train_info is not None:
        out["config"]["training"] = train_info
    if not args.no_variants:
        out["variants"] = variants(args, torch)
    if not args.no_solve:
        out["nd_solve"] = solve_block(args, torch, fp64_peak, peaks["hbm_gbs"])
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, args.policy, budget_s=args.cpu_budget)
    print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def time_config(torch, workload: str, policy: str, mode: str, steps: int, warmup: int,
                mlp=None, stream=None, t: int = 1, nd_leaf: int = 0):
    """stencils/s of one configuration (same step, L2 flush and events as the main line)."""
    from lsp_inputs import make_workload
    from paper_1607_02560_gb300 import Context

    v = make_workload(workload)
    stream = stream or torch.cuda.Stream()
    ctx = Context(v.ndim, v.shape[0], stream=stream)
    if mlp is not None:
        ctx.set_mlp(mlp)
    v_dev = torch.from_numpy(v).to("cuda")
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            ctx.set_potential(v_dev)
            ctx.build_stencils(policy=policy, mode=mode, use_graph=True, t=t, nd_leaf=nd_leaf)
        ctx.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.set_potential(v_dev)
            ctx.build_stencils(policy=policy, mode=mode, use_graph=True, t=t, nd_leaf=nd_leaf)
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        used = ctx.mode_used()
        ns = len(ctx.get_shift_table(with_sidx=False)["s"]) if used != "learned" else None
        extra = {}
        if used == "learned":
            q_learned = ctx.get_rows("Q").copy()
            ctx.build_stencils(policy=policy, mode="fp64")
            err = np.abs(q_learned - ctx.get_rows("Q")).max(axis=1)  # per point
            extra["max_abs_dalpha_vs_fp64"] = float(err.max())
            extra["dalpha_vs_fp64_per_point"] = {
                "p50": float(np.percentile(err, 50)), "p99": float(np.percentile(err, 99)),
                "p99.9": float(np.percentile(err, 99.9)), "max": float(err.max()),
                "frac_above_1e-2": float(np.mean(err > 1e-2))}
            ctx.build_stencils(policy=policy, mode=mode, use_graph=True, t=t, nd_leaf=nd_leaf)
        ctx.kernel_timing(True)
        for _ in range(5):
            flush.zero_()
            ctx.set_potential(v_dev)
            ctx.build_stencils(policy=policy, mode=mode, use_graph=True, t=t, nd_leaf=nd_leaf)
        ctx.synchronize()
        kt = {k: round(ms / max(cnt, 1), 4) for k, (ms, cnt) in ctx.kernel_times().items()}
        ctx.kernel_timing(False)
    ctx.close()
    out = {"workload": workload, "policy": policy, "mode": mode, "mode_used": used, "t": t,
           "nd_leaf": nd_leaf,
           "value": v.size * steps / (tot * 1e-3), "unit": "stencils/s",
           "ms_per_step": tot / steps, "shifts": ns, "kernel_ms_per_launch": kt}
    out.update(extra)
    return out


def train_for(torch, workload: str, steps: int, stream):
    """Train the surrogate on 16 other seeds (100-115) of the workload."""
    from lsp_inputs import make_workload
    from paper_1607_02560_gb300.learned import train_surrogate

    pots = [make_workload(workload, seed=s) for s in range(100, 116)]
    t0 = time.time()
    with torch.cuda.stream(stream):
        mlp, losses = train_surrogate(pots[0].ndim, pots, samples_per_potential=65536,
                                      steps=steps, batch=4096, lr=2e-3, stream=stream)
    torch.cuda.synchronize()
    info = {"potentials": len(pots), "seeds": "100-115", "pairs": 16 * 65536, "steps": steps,
            "batch": 4096, "seconds": round(time.time() - t0, 2),
            "final_loss": float(np.mean(losses[-50:]))}
    return mlp, info


def learned_variant(torch, workload: str, steps: int = 3000):
    """Train the surrogate on 16 other seeds of the workload, then time the learned build."""
    stream = torch.cuda.Stream()
    mlp, info = train_for(torch, workload, steps, stream)
    out = time_config(torch, workload, "local", "learned", steps=20, warmup=3, mlp=mlp,
                      stream=stream)
    out["training"] = info
    mlp.close()
    return out


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
    fp64_peak = measure_fp64_peak(torch)
    out = {"metric": "nested dissection setup / solve", "n_gpus": 1,
           "nd_solve": solve_block(args, torch, fp64_peak, peaks["hbm_gbs"])}
    print(json.dumps(out))


def variants(args, torch):
    """The metric's other forms on the same GPU: FP64 vs mixed, 2D n=1024 vs 3D n=64, and the
    paper's shift policy."""
    out = []
    for wl, pol, mode in [("helm2d_n1024", "local", "mixed"), ("schr3d_n64", "local", "fp64"),
                          ("schr3d_n64", "local", "mixed"), ("helm2d_n1024", "paper", "fp64"),
                          ("helm2d_n1024", "paper", "mixed")]:
        if (wl, pol, mode) == (args.workload, args.policy, args.mode):
            continue
        try:
            out.append(time_config(torch, wl, pol, mode, steps=20, warmup=3))
        except Exception as exc:  # a variant must not hide the main line
            out.append({"workload": wl, "policy": pol, "mode": mode, "error": str(exc)[:200]})
    # multi-t (Sec. 4.2): t_j from a nested dissection with leaf boxes of width 8, t_max = 2
    for wl, pol in (("helm2d_n1024", "paper"), ("helm2d_n256", "local"), ("schr3d_n64", "local")):
        try:
            out.append(time_config(torch, wl, pol, "fp64", steps=20, warmup=3, t=2, nd_leaf=8))
        except Exception as exc:
            out.append({"workload": wl, "policy": pol, "t": 2, "error": str(exc)[:200]})
    if not args.no_learned:
        for wl in ("helm2d_n1024", "schr3d_n64"):
            try:
                out.append(learned_variant(torch, wl, args.learned_steps))
            except Exception as exc:
                out.append({"workload": wl, "mode": "learned", "error": str(exc)[:300]})
    return out


def cpu_baseline(workload: str, policy: str, budget_s: float = 20.0, step_index: int = 0):
    """The oracle, as it stands, on the host cores: a sample of shifts plus the row assembly
    of every point, extrapolated to the workload's full shift list."""
    import oracle as O
    from lsp_inputs import make_workload

    v = make_workload(workload)
    n, d = v.shape[0], v.ndim
    t0 = time.perf_counter()
    st = O.build_stencils(v, policy, shift_subset=[0])  # shift list + s_j + row assembly
    t_rows = time.perf_counter() - t0
    ns = len(st["S"])
    rng = np.random.default_rng(100 + step_index)
    order = rng.permutation(ns)
    done, t_sh = 0, 0.0
    while done < ns and (t_sh + t_rows) < budget_s:
        t1 = time.perf_counter()
        O.stencil_for_shift(n, d, float(st["S"][order[done]]))
        t_sh += time.perf_counter() - t1
        done += 1
    per_shift = t_sh / max(done, 1)
    total = t_rows + per_shift * ns
    return {"value": v.size / total, "unit": "stencils/s", "cores": 1, "kind": "oracle",
            "sample": f"{done} of {ns} shifts (seeded) timed at {per_shift:.3f} s each + "
                      f"shift assignment and row assembly of all {v.size} points "
                      f"({t_rows:.2f} s); extrapolated to all shifts"
                      + ("" if done == ns else " (extrapolated)"),
            "seconds": t_sh + t_rows}


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    vals = []
    budget = max(2.0, args.ref_step_s)
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(args.workload, args.policy, budget_s=budget, step_index=k)
        if k >= args.warmup:
            vals.append(cb)
    value = float(np.median([c["value"] for c in vals]))
    last = vals[-1]
    out = {"impl": "reference", "metric": METRIC,
           "value": value, "unit": "stencils/s", "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": float(np.mean([c["seconds"] for c in vals])) * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "text": WORKLOAD_TEXT.get(args.workload, ""),
                      "policy": args.policy, "mode": "fp64"},
           "cpu_baseline": {"value": value, "unit": "stencils/s", "cores": 1, "kind": "oracle",
                            "sample": "per step: " + last["sample"]},
           "e2e": {"value": value, "unit": "stencils/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="helm2d_n1024")
    ap.add_argument("--policy", default="local", choices=["local", "paper", "mean"])
    ap.add_argument("--mode", default="fp64", choices=["fp64", "mixed", "learned"])
    ap.add_argument("--learned-steps", type=int, default=3000,
                    help="training steps of the surrogate (learned mode and variants)")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-solve", action="store_true",
                    help="skip the nested-dissection / GMRES measurements")
    ap.add_argument("--solve-n", default="256,512,1024",
                    help="grid sizes of the nested-dissection / GMRES measurements")
    ap.add_argument("--solve-n3", default="16,32",
                    help="3D grid sizes of the nested-dissection / GMRES measurements")
    ap.add_argument("--solve-only", action="store_true",
                    help="print only the nested-dissection / GMRES measurements (profiling)")
    ap.add_argument("--no-learned", action="store_true", help="skip training the surrogate")
    ap.add_argument("--n", type=int, default=None, help="rescale the workload's grid (small cases)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--ref-step-s", type=float, default=4.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.solve_only:
        run_solve_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
