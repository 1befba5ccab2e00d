"""Benchmark of the surrogate ILU(0) smoother on GB300.

Workload (one step = one smoother sweep = residual + forward + backward over
the whole interior): one macro-tetrahedron at level 7 (333,375 interior
points), reference tetrahedron with every coordinate moved by U(-0.1, 0.1)
(seed 3), kappa = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z), surrogate degree
6, MIXED precision (FP32 substitutions and surrogate evaluation, FP64 residual
and update), b ~ U(-1, 1) (seed 4), x0 = 0.  Inputs are smaller than L2, so a
256 MiB buffer is written between timed steps (L2 flush).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.

Further workloads print a line of the same form (not the default run):
  --workload level9  one macro-tet at level 9 (22.1M interior DoF), kappa = 1,
                     degree 6, F32 sweeps (band kernels) and, in the line's
                     "f64" entry, FP64 sweeps; against the HBM roofline at
                     24 (F32) and 56 (F64) algorithmic bytes per DoF.
  --workload batch   256 macro-tets of a jittered 4x4x3 cube mesh (aspect
                     ratio <= 3), levels U{5..8}, degrees U{4..6}, FP32,
                     kappa = 1; one step = one sweep of the whole batch (one
                     CUDA-graph replay, autotuned partition).
  --workload serve   the request loop: Poisson arrivals (mean gap --gap-ms,
                     0.5 ms by default) of interior solves on macro-tets of
                     that mesh, mixed coefficients, to 1e-8: by default
                     V(3,3) multigrid on levels 5-8 (--method pcg: PCG on
                     levels 5-8; --method richardson: smoothed Richardson on
                     levels 5-6); solves/s and p50/p99 latency, beside the
                     same requests solved one after another with FP64 sweeps.
  --workload smoothers  iteration counts of the surrogate ILU(0) smoother
                     against the surrogate symmetric Gauss-Seidel smoother,
                     both as Richardson smoothers and as CG preconditioners,
                     to a relative residual of 1e-8: on the default level-7
                     tet, on macro-tets of the mesh above (level 6), and on
                     trirectangular tets whose top vertex sinks to height h
                     (level 6, all 24 vertex orders for ILU).
  --workload mg      geometric multigrid (V(3,3)-cycle, levels 2..L, exact
                     solve on level 2) on the default tet: V-cycle time and
                     solves to 1e-8 by V-cycle iteration and by V-cycle
                     preconditioned CG at levels 5-9, and the convergence
                     factors of the paper's Table 2 shapes measured on the GPU.
  --workload packed  one tet at --level (default 8) on the packed kernels,
                     FP32: ms per sweep, schedule steps and cycles per step.
  --workload boundary  convergence factors of the V(3,3)-cycle (levels 2..6)
                     with boundary variants V1 and V2 across surrogate
                     degrees: the trirectangular unit tet with kappa_i =
                     1 + 10(x^i + y^i + z^i), i = 0..3, and a tet of height
                     0.1 with kappa = 1, isotropic degrees and (0, 0, d).
"""
import argparse
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

import seeded_inputs as si  # noqa: E402

LEVEL, DEG, TET_SEED, RHS_SEED = 7, 6, 3, 4
COEFF = ("sinprod", 1.0, 0.5, 0)
METRIC = "smoother DoF-sweeps/s (MIXED: FP32 sweeps, FP64 residual/update)"
UNIT = "DoF-sweeps/s"
WORKLOAD = "surrogate ILU(0) smoother sweep, single macro-tet L7 (333375 interior DoF), kappa=1+0.5sin sin sin, deg 6"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


WORKLOAD_TAG = "L7-MIXED-deg6-sinprod"


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from a committed ncu summary under
    profiles/, if it was taken on this workload from the current wavefront
    source (its first 16 hex digits of sha256 match); else None."""
    import glob
    import hashlib
    src = os.path.join(ROOT, "paper_2210_15280_gb300", "csrc", "wavefront.cu")
    try:
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(f):
            kv = dict(t.split("=", 1) for t in line.split() if "=" in t)
            if (kv.get("kernel") == kernel and kv.get("workload") == WORKLOAD_TAG
                    and kv.get("wavefront_sha256_16") == sha and "dram_bytes" in kv):
                return int(kv["dram_bytes"])
    return None


# FP64 pipe of GB300: 152 SMs x 2 DFMA/clk x 2 FLOP x 2.07 GHz (max SM clock)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def interior(level):
    n = 2 ** level
    return (n - 1) * (n - 2) * (n - 3) // 6


def rows(level):
    n = 2 ** level
    return (n - 3) * (n - 2) // 2


def algorithmic(level, deg):
    """Per-launch algorithmic bytes / FLOPs of the three kernels (MIXED,
    variable coefficient): each vector element moved once, tables once."""
    nint, nr = interior(level), rows(level)
    return {
        # x, b, kappa read (8 B each), r written (4 B)
        "residual": {"bytes": nint * 28, "flops": nint * 242},
        # r read, w written (4 B each) + forward table (7 functions x (deg+1) floats per row)
        "forward": {"bytes": nint * 8 + nr * 7 * (deg + 1) * 4, "flops": nint * (14 * deg + 14)},
        # w read, x read + written, backward table (8 functions)
        "backward": {"bytes": nint * 20 + nr * 8 * (deg + 1) * 4, "flops": nint * (16 * deg + 17)},
    }


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.proc, self.path = gpu, None, None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))
        return out


def max_over_ranks(ms, dist, device):
    """The slowest rank's time: every rank gets the maximum (one MAX
    all-reduce; `dist` None for a single process)."""
    if not dist:
        return ms
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, dof_per_rank, steps, total_ms):
    """Whole-job throughput of `world` replicas that each swept `dof_per_rank`
    interior points `steps` times, over the slowest rank's time."""
    return world * dof_per_rank * steps / (total_ms / 1e3)


def cpu_oracle_sample(steps=8, warmup=0):
    """The oracle, as it stands, on the same workload: set-up (untimed), then
    `warmup` untimed and `steps` timed matrix-free sweeps, each = evaluate the
    surrogates at every interior point + one Alg. 2 sweep.  Single-threaded."""
    from oracle import oracle as O
    N = 2 ** LEVEL
    P = si.macro_tet(TET_SEED)
    pr = O.Problem(P, LEVEL, O.Coeff(*COEFF), deg=DEG)
    b = si.rhs(LEVEL, RHS_SEED)
    x = np.zeros(O.num_nodes(N))
    for _ in range(warmup):
        Ls, Dinv = O.eval_surrogates(N, pr.deg, pr.coefs)
        O.smooth(pr.A, N, Ls, Dinv, x, b, 1)
    t0 = time.perf_counter()
    for _ in range(steps):
        Ls, Dinv = O.eval_surrogates(N, pr.deg, pr.coefs)
        O.smooth(pr.A, N, Ls, Dinv, x, b, 1)
    dt = time.perf_counter() - t0
    return {"value": interior(LEVEL) * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"L7 workload, {steps} sweeps, each re-evaluating the eight surrogates at all "
                      f"{interior(LEVEL)} interior points (FP64, 1 thread), {dt:.1f} s"}


def run_reference(args, rank):
    if rank != 0:
        return
    # bounded sample: at most 8 timed and 2 warm-up sweeps of about 0.9 s each
    steps = max(1, min(args.steps, 8))
    warm = max(0, min(args.warmup, 2))
    cb = cpu_oracle_sample(steps, warm)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * interior(LEVEL) / cb["value"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "level": LEVEL, "degree": DEG,
                                            "precision": "F64 (oracle)"},
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def shard_of(levels, rank, world, g):
    """The tets rank `rank` of `world` GPUs sweeps: the library's split of the
    batch by tet (ilu_partition, longest processing time first on the
    interior point counts).  Tets are independent, so no exchange follows."""
    if world <= 1:
        return list(range(len(levels)))
    rank_of, _ = g.partition([interior(int(L)) for L in levels], world)
    return [i for i in range(len(levels)) if rank_of[i] == rank]


def sharded_oracle_sweeps(rank, world, dist, n=10):
    """The sharded run without a GPU: `n` small tets of the batch mesh split
    over `world` ranks as the batch workload splits them; each rank sweeps its
    own tets once (the CPU oracle stands in for the GPU batch) and rank 0
    gathers (tet, x) pairs over the host, in tet order (others get None)."""
    import paper_2210_15280_gb300 as g
    from oracle import oracle as O
    mesh = si.macro_mesh(6, n_tets=n)
    levels = si.batch_levels(7, n, 2, 4)
    out = []
    for i in shard_of(levels, rank, world, g):
        L = int(levels[i])
        pr = O.Problem(mesh[i], L, O.Coeff("const"), deg=[2, 2, 2])
        Ls, Dinv = pr.surrogate_factors()
        x = O.smooth(pr.A, 2 ** L, Ls, Dinv, si.boundary_data(L, 300 + i), si.rhs(L, 400 + i), 1)
        out.append((i, x))
    if dist is None:
        return out
    parts = [None] * world if rank == 0 else None
    dist.gather_object(out, parts, dst=0)
    if rank != 0:
        return None
    return sorted((p for part in parts for p in part), key=lambda p: p[0])


def batch_workload(args, g, torch, rank=0, world=1, dist=None, compact=False):
    """256 tets, one batch, one graph replay per step.  On several GPUs each
    rank sweeps its share of the tets (shard_of) and the line reports all
    ranks' points over the slowest rank's time.  Beside it (one GPU): the same
    tets swept one handle after another, in FP32 and in plain FP64.
    `compact`: at most 20 steps, the sub-object of the default line."""
    from concurrent.futures import ThreadPoolExecutor
    n = 256
    mesh = si.macro_mesh(6, n_tets=n)
    levels_all = si.batch_levels(7, n, 5, 8)
    degs_all = 4 + (si.splitmix64(9, n) % 3).astype(int)
    if not compact and getattr(args, "tets", 0) and 0 < args.tets < n:  # the first tets of the same batch
        n = args.tets
        mesh, levels_all, degs_all = mesh[:n], levels_all[:n], degs_all[:n]
    mine = shard_of(levels_all, rank, world, g)
    levels, degs = [levels_all[i] for i in mine], [degs_all[i] for i in mine]
    with ThreadPoolExecutor(8) as ex:
        tets = list(ex.map(lambda k: g.Tet(mesh[mine[k]], int(levels[k]), coeff=g.make_coeff("const"),
                                           poly_degree=int(degs[k]), precision=g.F32, kernel=g.KERNEL_PACKED,
                                           device=torch.cuda.current_device()), range(len(mine))))
    idof_all = sum(interior(int(L)) for L in levels_all)
    idof = sum(interior(int(L)) for L in levels)
    xs = [torch.zeros(si.num_nodes(int(L)), dtype=torch.float32, device="cuda") for L in levels]
    bh = [si.rhs(int(L), 100 + i).astype(np.float32) for i, L in enumerate(levels)]
    bs = [torch.tensor(v, device="cuda") for v in bh]
    B = g.Batch(tets)
    W, K = max(3, args.warmup), max(1, args.steps)
    if compact:
        K = min(K, 20)
    for _ in range(W):
        B.smooth(xs, bs, 1)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stream = torch.cuda.current_stream()
    for k in range(K):  # inputs (~4 GB) exceed L2: no flush needed
        ev[k][0].record(stream)
        B.smooth(xs, bs, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(a.elapsed_time(b2) for a, b2 in ev), dist, "cuda")
    value = idof_all * K / (total_ms / 1e3)  # every rank's points over the slowest rank's time
    # end to end: host vectors copied in and the result copied out every step
    xh = [np.zeros(v.numel(), dtype=np.float32) for v in xs]
    bhp = [torch.from_numpy(v).pin_memory() for v in bh]
    xhp = [torch.from_numpy(v).pin_memory() for v in xh]
    E = max(2, min(K, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(E):
        for d, h in zip(xs, xhp):
            d.copy_(h, non_blocking=True)
        for d, h in zip(bs, bhp):
            d.copy_(h, non_blocking=True)
        B.smooth(xs, bs, 1)
        for d, h in zip(xs, xhp):
            h.copy_(d, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e = idof_all * E / e2e_s
    nbytes = sum(v.numel() for v in xs) * 4
    achieved = idof * 24 / (total_ms / K / 1e3) / 1e9  # F32 sweep: 24 algorithmic bytes per DoF (this rank)
    hbm, src = peaks()
    launches = B.launches_per_sweep() * K
    per_tet = None
    if world == 1:
        per_tet = one_by_one(g, torch, tets, xs, bs, mesh, levels, degs, W, min(K, 5))
        per_tet["batch_speedup_vs_f32_one_by_one"] = per_tet["f32_ms_per_sweep"] / (total_ms / K)
        per_tet["batch_speedup_vs_f64_one_by_one"] = per_tet["f64_ms_per_sweep"] / (total_ms / K)
    B.close()
    for t in tets:
        t.close()
    if compact:
        return {"value": value, "unit": UNIT, "ms_per_step": total_ms / K, "steps": K, "dtype": "f32",
                "workload": f"batch of {n} macro-tets, levels 5-8, degrees 4-6, {idof_all} interior DoF, "
                            "packed kernels, one graph replay per sweep",
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "kernel": "whole sweep at 24 B/DoF", "peak_source": src},
                "depth": {"note": "the level-8 tets' packed substitutions bound the batch (two SMs each)"},
                "one_by_one": per_tet,
                "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": nbytes}}
    return {"metric": f"smoother DoF-sweeps/s (batch of {n} macro-tets, FP32 sweeps)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batch of {n} macro-tets, levels 5-8, degrees 4-6, {idof_all} interior DoF",
                       "tuned": "packed kernels, longest tets first", "l2": "inputs larger than L2",
                       "parallelism": f"tets sharded over {world} GPU(s), no exchange"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 2 * nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                         "traffic": None, "kernel": "whole sweep (residual + forward + backward)", "peak_source": src},
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                       "samples": clk["samples"]},
            "one_by_one": per_tet}


def one_by_one(g, torch, tets, xs, bs, mesh, levels, degs, W, K):
    """The batch's tets swept one handle after another (one ilu_smooth call
    per tet, same stream): with the batch's FP32 handles, and with plain FP64
    handles (default kernels, matrix-free)."""
    from concurrent.futures import ThreadPoolExecutor

    def run(ts, xv, bv):
        for _ in range(W):
            for t, x, b in zip(ts, xv, bv):
                t.smooth(x, b, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(K):
            for t, x, b in zip(ts, xv, bv):
                t.smooth(x, b, 1)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K

    f32 = run(tets, xs, bs)
    with ThreadPoolExecutor(8) as ex:
        t64 = list(ex.map(lambda k: g.Tet(mesh[k], int(levels[k]), coeff=g.make_coeff("const"),
                                          poly_degree=int(degs[k]), precision=g.F64,
                                          stencil=g.STENCIL_ON_THE_FLY, values=g.VALUES_ON_THE_FLY,
                                          device=torch.cuda.current_device()), range(len(tets))))
    x64 = [torch.zeros(x.numel(), dtype=torch.float64, device="cuda") for x in xs]
    b64 = [b.double() for b in bs]
    f64 = run(t64, x64, b64)
    for t in t64:
        t.close()
    return {"f32_ms_per_sweep": f32, "f64_ms_per_sweep": f64, "sweeps": K,
            "how": "one ilu_smooth per tet, all tets in turn on one stream"}


def level9_workload(args, g, torch, compact=False):
    """Single level-9 tet (22.1M interior DoF), kappa = 1, degree 6: F32 and
    F64 sweeps, both matrix-free (constant stencil, surrogates evaluated in
    the sweep), against the HBM roofline at 24 (F32) and 56 (F64) algorithmic
    bytes per DoF; the F32 and MIXED results against the F64 result after
    two sweeps from the same start with the same polynomials.  `compact`:
    without the level scan, the sub-object of the default line."""
    level = 9
    nint = interior(level)
    P = si.macro_tet(5)
    out = {}
    hbm, src = peaks()
    W, K = max(3, args.warmup), max(1, min(args.steps, 20))
    mf = dict(stencil=g.STENCIL_ON_THE_FLY, values=g.VALUES_ON_THE_FLY)
    coefs = None
    x0 = si.boundary_data(level, 7)
    b_h = si.rhs(level, 6)
    two = {}
    for name, prec, dt, bpd in [("F64", g.F64, torch.float64, 56), ("F32", g.F32, torch.float32, 24),
                                ("MIXED", g.MIXED, torch.float64, 24)]:
        t = g.Tet(P, level, coeff=g.make_coeff("const"), poly_degree=6, precision=prec, **mf)
        if coefs is None:
            coefs = t.export_surrogate()
        else:
            t.import_surrogate(coefs)
        xe = torch.tensor(x0, dtype=dt, device="cuda")
        b = torch.tensor(b_h, dtype=dt, device="cuda")
        t.smooth(xe, b, 2)
        two[name] = xe.double().cpu().numpy()
        del xe
        if name == "MIXED":
            t.close()
            break
        x = torch.zeros_like(b)
        t.smooth(x, b, W)
        torch.cuda.synchronize()
        t.profile(True)
        t.profile_read()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        t.smooth(x, b, K)  # vectors of 90-180 MB each exceed L2
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / K
        kms, launches = t.profile_read()
        achieved = nint * bpd / (ms / 1e3) / 1e9
        out[name] = {"value": nint / (ms / 1e3), "ms_per_step": ms, "achieved_gbs": achieved,
                     "frac": achieved / hbm, "kernel_ms_per_launch": [round(v / K, 4) for v in kms],
                     "launches_per_step": launches / K}
        t.close()
    ref = two["F64"]
    scale = np.abs(ref).max()
    err = {f"{nm}_vs_F64_after_2_sweeps": float(np.abs(two[nm] - ref).max() / scale) for nm in ("F32", "MIXED")}
    f, d = out["F32"], out["F64"]
    sm_mhz = 2070.0
    levels = 3 * 2 ** level - 11
    cyc = g.step_floor(32, 4096)
    depth = {"steps_per_substitution": levels, "floor_cycles_per_step_one_warp": round(cyc, 1),
             "us_per_sweep_at_max_clock": round(2 * levels * cyc / (sm_mhz * 1e6) * 1e6, 1)}
    if compact:
        return {"value": f["value"], "unit": UNIT, "ms_per_step": f["ms_per_step"], "steps": K, "dtype": "f32",
                "workload": f"single macro-tet L9 ({nint} interior DoF), kappa=1, deg 6, band kernels, matrix-free",
                "roofline": {"bound": "hbm", "achieved": f["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                             "frac": f["frac"], "kernel": "whole sweep at 24 B/DoF", "peak_source": src,
                             "kernel_ms_per_launch": f["kernel_ms_per_launch"]},
                "depth": depth,
                "F64": {"value": d["value"], "ms_per_step": d["ms_per_step"], "achieved_gbs": d["achieved_gbs"],
                        "frac": d["frac"], "bytes_per_dof": 56, "kernel_ms_per_launch": d["kernel_ms_per_launch"]},
                "error": err}
    # bandwidth scaling: the same F32 sweep at levels 6-8 (slab kernels) and 9 (band kernels)
    scaling = {}
    for lv in [6, 7, 8]:
        t = g.Tet(P, lv, coeff=g.make_coeff("const"), poly_degree=6, precision=g.F32, **mf)
        b = torch.tensor(si.rhs(lv, 6), dtype=torch.float32, device="cuda")
        x = torch.zeros_like(b)
        t.smooth(x, b, W)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        tot = 0.0
        for k in range(K):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            t.smooth(x, b, 1)
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        ms = tot / K
        scaling[f"L{lv}"] = {"interior_dof": interior(lv), "ms_per_step": round(ms, 4),
                             "value": interior(lv) / (ms / 1e3)}
        t.close()
        del flush
    scaling["L9"] = {"interior_dof": nint, "ms_per_step": round(f["ms_per_step"], 4), "value": f["value"]}
    return {"metric": "smoother DoF-sweeps/s (single macro-tet, level 9, FP32 sweeps)", "value": f["value"],
            "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": f["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"single macro-tet L9 ({nint} interior DoF), kappa=1, deg 6",
                       "kernels": "band (automatic choice at level 9)", "l2": "inputs larger than L2",
                       "operator": "constant stencil", "surrogates": "evaluated on the fly",
                       "parallelism": "replicas x1"},
            "roofline": {"bound": "hbm", "achieved": f["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                         "frac": f["frac"], "traffic": None, "kernel": "whole sweep at 24 B/DoF",
                         "peak_source": src, "kernel_ms_per_launch": f["kernel_ms_per_launch"]},
            "depth": depth,
            "f64": {"value": d["value"], "ms_per_step": d["ms_per_step"], "achieved_gbs": d["achieved_gbs"],
                    "frac": d["frac"], "kernel_ms_per_launch": d["kernel_ms_per_launch"]},
            "error": err,
            "f32_level_scaling": scaling,
            "gpu_launches": int(round(f["launches_per_step"] * K))}


def serve_workload(args, g, torch):
    """Poisson stream of interior solves through the request loop, against the
    same requests solved one after another with FP64 sweeps."""
    pcg = args.method == "pcg"
    mg = args.method == "mg"
    nreq = args.requests
    pool = si.macro_mesh(6, n_tets=32)
    lo, hi = (5, 8) if (pcg or mg) else (5, 6)
    levels = si.batch_levels(11, nreq, lo, hi)
    kinds = [("const", 1.0, 0.0, 0), ("sinprod", 1.0, 0.5, 0), ("kappa_i", 0.0, 0.0, 2)]
    which = si.splitmix64(12, nreq) % len(pool)
    arrivals = si.poisson_arrivals(13, nreq, args.gap_ms * 1e-3)  # seconds from the first submit
    method = g.PCG if pcg else (g.MG_VCYCLE if mg else g.RICHARDSON)
    reqs = []
    for i in range(nreq):
        L = int(levels[i])
        reqs.append(dict(P=pool[int(which[i])], level=L, co=kinds[int(which[i]) % 3], b=si.rhs(L, 1000 + i)))
    # every distinct tet set up once before the timed stream (resident afterwards)
    warm = {}
    for r in reqs:
        warm.setdefault((id(r["P"]), r["level"], r["co"]), r)
    s = g.Server(precision=g.MIXED, max_slots=64, max_cluster=args.max_cluster)
    for tk in [s.submit(r["P"], r["level"], r["b"], coeff=g.make_coeff(*r["co"]), poly_degree=5, method=method)
               for r in warm.values()]:
        s.wait(tk)
    t0 = time.perf_counter()
    tks = []
    for i, r in enumerate(reqs):
        target = t0 + float(arrivals[i])
        while time.perf_counter() < target:
            pass
        tks.append(s.submit(r["P"], r["level"], r["b"], coeff=g.make_coeff(*r["co"]), poly_degree=5, method=method))
    lat, ok = [], 0
    for tk in tks:
        res = s.wait(tk)
        ok += res["status"] == g.ILU_OK
        lat.append(res["latency_ms"])
    wall = time.perf_counter() - t0
    st = s.stats()
    s.close()
    lat = np.sort(np.array(lat))
    # the same requests, one after another, FP64 sweeps, tets set up beforehand
    seq = {}
    for r in reqs:
        key = (id(r["P"]), r["level"], r["co"])
        if key not in seq:
            make = g.Multigrid if mg else g.Tet
            seq[key] = make(r["P"], r["level"], coeff=g.make_coeff(*r["co"]), poly_degree=5, precision=g.F64)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for r in reqs:
        t = seq[(id(r["P"]), r["level"], r["co"])]
        x = torch.zeros(si.num_nodes(r["level"]), dtype=torch.float64, device="cuda")
        b = torch.tensor(r["b"], dtype=torch.float64, device="cuda")
        t.solve(x, b, g.RICHARDSON if mg else method, 1e-8, 100000)
        x.cpu()
    seq_rate = nreq / (time.perf_counter() - t1)
    q = lambda p: float(lat[min(len(lat) - 1, max(0, int(np.ceil(p * len(lat))) - 1))])
    return {"metric": "served interior solves/s (request loop, p50/p99 latency)", "value": nreq / wall,
            "unit": "solves/s", "n_gpus": 1, "steps": nreq, "warmup": len(warm), "ms_per_step": 1e3 * wall / nreq,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"max_cluster": args.max_cluster,
                       "workload": f"{nreq} Poisson-arrival requests (mean gap {args.gap_ms:g} ms), levels {lo}-{hi}, "
                                   f"{'PCG' if pcg else ('V(3,3) multigrid' if mg else 'Richardson')} to 1e-8, "
                                   "MIXED, 32 macro-tets x 3 kappa",
                       "parallelism": "replicas x1"},
            "p50_ms": q(0.5), "p99_ms": q(0.99), "completed": ok, "max_concurrent": st["max_concurrent"],
            "sequential_f64_solves_per_s": seq_rate,
            "e2e": {"value": nreq / wall, "unit": "solves/s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": None}}


def smoothers_workload(args, g, torch):
    """Iterations to a relative residual of 1e-8 for ILU(0) and SGS surrogates
    on the same tets; log(rho_ILU)/log(rho_SGS) = it_SGS/it_ILU for Richardson
    (the measure of the height sweep of Sec. 4.2, here for the single-level
    smoother)."""
    import itertools
    t_start = time.time()
    rtol, cap = 1e-8, 20000
    co = g.make_coeff(*COEFF[:3])

    def iters(P, level, deg, method, factor, coeff=co, seed=RHS_SEED, limit=cap):
        try:
            t = g.Tet(P, level, coeff=coeff, poly_degree=deg, precision=g.MIXED, factor=factor)
        except g.IluError as e:
            return {"error": str(e)}
        b = torch.tensor(si.rhs(level, seed), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        it, rel, ok = t.solve(x, b, method, rtol, limit)
        t.close()
        return it if ok else {"not_converged": it, "rel": rel}

    def pair(P, level, deg, coeff=co):
        out = {}
        for mname, m in [("richardson", g.RICHARDSON), ("pcg", g.PCG)]:
            for fname, f in [("ilu", g.FACTOR_ILU0), ("sgs", g.FACTOR_SGS)]:
                out[f"{mname}_{fname}"] = iters(P, level, deg, m, f, coeff)
        return out

    c2 = pair(si.macro_tet(TET_SEED), LEVEL, DEG)
    mesh = [pair(P, 6, 5, g.make_coeff("const")) for P in si.macro_mesh(6)[:4]]
    heights = []
    for h in [1.0, 0.5, 0.25, 0.125, 0.0625]:
        P = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, h]], float)
        row = {"h": h}
        row.update(pair(P, 6, 6, g.make_coeff("const")))
        best = None
        for perm in itertools.permutations(range(4)):
            it = iters(P[list(perm)], 6, 6, g.RICHARDSON, g.FACTOR_ILU0, g.make_coeff("const"),
                       limit=best[0] if best else cap)
            if isinstance(it, int) and (best is None or it < best[0]):
                best = (it, list(perm))
        row["richardson_ilu_best_order"] = best
        sg = row["richardson_sgs"]
        if best and isinstance(sg, int):
            row["log_rho_ratio_best"] = sg / best[0]
        heights.append(row)
    ri, rs = c2["richardson_ilu"], c2["richardson_sgs"]
    return {"metric": "Richardson iterations to relative residual 1e-8, surrogate ILU(0) smoother",
            "value": ri, "unit": "iterations", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": (time.time() - t_start) * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + ", Richardson and PCG to 1e-8 from x0 = 0, ILU(0) and SGS",
                       "precision": "MIXED", "parallelism": "replicas x1"},
            "sgs_value": rs, "ratio_sgs_over_ilu": (rs / ri) if isinstance(ri, int) and isinstance(rs, int) else None,
            "l7_tet": c2, "mesh_tets_l6_deg5_kappa1": mesh, "trirectangular_l6_deg6_kappa1": heights}


TABLE2 = {  # vertex lists of the shapes (Table SM1; Spindle y read as 10) and the printed ILU rates
    "spindle": ([[0, 0, 0.5], [0, 0, -0.5], [0.5, 10, 0], [-0.5, 10, 0]], {"1234": 0.65, "1324": 0.39, "1423": 0.35}),
    "cap": ([[0, 0, 0], [1, 0, 0], [0.5, 0.866, 0], [0.5, 0.288, 0.093]],
            {"1234": 0.010, "1243": 0.43, "1342": 0.43, "2341": 0.0096}),
    "spade": ([[0, 0, 0], [1, -0.666, 0], [1, 0.666, 0], [1, 0, 0.443]],
              {"1234": 0.084, "1243": 0.053, "1342": 0.060, "2134": 0.014, "2143": 0.14, "2341": 0.028}),
    "regular": ([[0, 0, 0], [1, 0, 0], [0.5, 3 ** 0.5 / 2, 0], [0.5, 3 ** 0.5 / 6, (2 / 3) ** 0.5]], {"1234": 0.025}),
}


def mg_workload(args, g, torch):
    """Multigrid solves on the default tet and Table 2 rates on the GPU."""
    co = g.make_coeff(*COEFF[:3])
    levels = []
    for level, prec in [(5, g.MIXED), (6, g.MIXED), (7, g.MIXED), (8, g.MIXED), (9, g.F32)]:
        t0 = time.time()
        m = g.Multigrid(si.macro_tet(TET_SEED), level, coeff=co, poly_degree=DEG, nu=3, precision=prec)
        setup_s = time.time() - t0
        dt = torch.float32 if prec == g.F32 else torch.float64
        rtol = 1e-5 if prec == g.F32 else 1e-8
        b = torch.tensor(si.rhs(level, RHS_SEED), dtype=dt, device="cuda")
        x = torch.zeros_like(b)
        m.cycle(x, b, 2)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        K = 5
        e0.record()
        m.cycle(x, b, K)
        e1.record()
        torch.cuda.synchronize()
        vms = e0.elapsed_time(e1) / K
        row = {"level": level, "precision": {g.MIXED: "MIXED", g.F32: "F32"}[prec], "interior_dof": interior(level),
               "setup_s": round(setup_s, 3), "vcycle_ms": round(vms, 3), "rtol": rtol}
        for name, meth in [("richardson", g.RICHARDSON), ("pcg", g.PCG)]:
            x.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            it, rel, ok = m.solve(x, b, meth, rtol, 100)
            torch.cuda.synchronize()
            row[name] = {"iters": it, "rel": rel, "ok": ok, "ms": round((time.perf_counter() - t0) * 1e3, 3)}
        levels.append(row)
        m.close()
    rates = []
    for name, (V, cols) in TABLE2.items():
        V = np.array(V, float)
        for pi, paper in cols.items():
            P = np.zeros_like(V)
            for i, c in enumerate(pi):
                P[int(c) - 1] = V[i]
            m = g.Multigrid(P, 6, poly_degree=7, nu=3, precision=g.F64)
            e = torch.tensor(si.interior_error(6, 9), dtype=torch.float64, device="cuda")
            rho, _ = m.rate(e, 20)
            m.close()
            rates.append({"shape": name, "pi": pi, "rho_ilu_gpu": round(rho, 4), "rho_ilu_paper": paper})
    l7 = [r for r in levels if r["level"] == LEVEL][0]
    solve_ms = l7["richardson"]["ms"]
    return {"metric": "multigrid solves to 1e-8: interior DoF solved per second (V-cycle iteration, L7 MIXED)",
            "value": interior(LEVEL) / (solve_ms / 1e3), "unit": "DoF/s", "n_gpus": 1, "steps": 1, "warmup": 2,
            "ms_per_step": solve_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD + ", multigrid V(3,3) levels 2..7, solve to 1e-8 from x0 = 0",
                       "precision": "MIXED", "parallelism": "replicas x1"},
            "levels": levels, "table2_rates_deg7_f64": rates}


def packed_workload(args, g, torch):
    """One tet at --level (8 by default) on the packed kernels, FP32 sweeps,
    kappa = 1 + 0.5 sin sin sin, degree 6: ms per sweep, the schedule's steps
    per substitution and the SM cycles per step (at the sampled clock), beside
    the depth floor of a 384-thread CTA step from ilu_step_floor."""
    level = args.level or 8
    P = si.macro_tet(TET_SEED)
    W, K = max(3, args.warmup), max(1, min(args.steps, 50))
    t = g.Tet(P, level, coeff=g.make_coeff(*COEFF), poly_degree=DEG, precision=g.F32, kernel=g.KERNEL_PACKED)
    b = torch.tensor(si.rhs(level, RHS_SEED), dtype=torch.float32, device="cuda")
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    t.smooth(x, b, W)
    torch.cuda.synchronize()
    t.profile(True)
    t.profile_read()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ms = statistics.median(time_steps(t, x, b, K, flush, torch.cuda.current_stream(), torch))
    clk = clocks.stop()
    kms, launches = t.profile_read()
    t.close()
    T, _, _, _ = g.packed_schedule(level, True)
    mhz = clk["sm_mhz"] or 2070.0
    sub_ms = kms[1] / K  # the packed launch: both substitutions
    floor = g.step_floor(384, 4096)
    return {"metric": f"smoother DoF-sweeps/s (single macro-tet, level {level}, packed kernels, FP32)",
            "value": interior(level) / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": K, "warmup": W,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"single macro-tet L{level} ({interior(level)} interior DoF), kappa=1+0.5sin sin sin, "
                                   "deg 6, KERNEL_PACKED", "l2": "flushed between steps (256 MiB write)"},
            "kernel_ms_per_launch": {"residual": round(kms[0] / K, 5), "packed (both passes)": round(sub_ms, 5),
                                     "update": round(kms[2] / K, 5)},
            "schedule_steps_per_pass": T, "start_quantum": 1 if level <= 6 else (2 if level == 7 else 4),
            "cycles_per_step": round(sub_ms * 1e-3 * mhz * 1e6 / (2 * T)),
            "floor_cycles_per_step_384_threads": round(floor, 1),
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]}}


def boundary_workload(args, g, torch):
    """Rates of the surrogate-ILU V-cycle with boundary variants V1 and V2
    against the surrogate degree (Sec. 4.2, the studies on kappa_i and on a
    flat tet)."""
    t_start = time.time()
    e = torch.tensor(si.interior_error(6, 9), dtype=torch.float64, device="cuda")

    def rho(P, coeff, deg, bnd):
        try:
            m = g.Multigrid(P, 6, coeff=coeff, poly_degree=0, nu=3, precision=g.F64, deg=deg, boundary=bnd)
        except g.IluError as err:  # e.g. a low-degree surrogate of 1/D that is not positive
            return str(err)
        r, _ = m.rate(e.clone(), 20)
        m.close()
        return round(r, 4)

    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    kappa = {}
    for i in range(4):
        co = g.make_coeff("kappa_i", 0.0, 0.0, i)
        kappa[f"kappa_{i}"] = {f"deg{d}": {"V1": rho(tri, co, d, g.BOUNDARY_V1), "V2": rho(tri, co, d, g.BOUNDARY_V2)}
                               for d in range(0, 7)}
    flat = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 0.1]], float)
    one = g.make_coeff("const")
    flat_iso = {f"deg{d}": {"V1": rho(flat, one, d, g.BOUNDARY_V1), "V2": rho(flat, one, d, g.BOUNDARY_V2)}
                for d in range(0, 7)}
    flat_z = {f"deg(0,0,{d})": {"V1": rho(flat, one, [0, 0, d], g.BOUNDARY_V1),
                                "V2": rho(flat, one, [0, 0, d], g.BOUNDARY_V2)} for d in range(0, 9, 2)}
    v = kappa["kappa_3"]["deg3"]
    return {"metric": "V(3,3)-cycle convergence factor, surrogate ILU(0), boundary variant V1 (kappa_3, degree 3)",
            "value": v["V1"], "unit": "rho", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": (time.time() - t_start) * 1e3, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "trirectangular unit tet and a tet of height 0.1, multigrid levels 2..6, "
                                   "20-step power iteration, F64", "parallelism": "replicas x1"},
            "v2_value": v["V2"], "trirectangular_kappa_i": kappa, "height_0.1_isotropic": flat_iso,
            "height_0.1_z_only": flat_z}



def time_steps(t, x, b, K, flush, stream, torch):
    """K sweeps, each bracketed by CUDA events on `stream`, the L2 flushed
    (256 MiB write) before each; returns the per-step milliseconds."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for k in range(K):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        t.smooth(x, b, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(e) for a, e in ev]


def sweep_variant(g, torch, P, flush, stream, W, K, level=None, prec=None, coeff=COEFF, **opts):
    """ms per sweep and DoF-sweeps/s of one set-up variant of the default tet,
    with its per-kernel split (CUDA events around each launch)."""
    level = LEVEL if level is None else level
    prec = g.MIXED if prec is None else prec
    dt = torch.float32 if prec == g.F32 else torch.float64
    t = g.Tet(P, level, coeff=g.make_coeff(*coeff), poly_degree=DEG, precision=prec,
              device=torch.cuda.current_device(), **opts)
    b = torch.tensor(si.rhs(level, RHS_SEED), dtype=dt, device="cuda")
    x = torch.zeros_like(b)
    t.smooth(x, b, W)
    torch.cuda.synchronize()
    t.profile(True)
    t.profile_read()
    ms = statistics.median(time_steps(t, x, b, K, flush, stream, torch))
    kms, launches = t.profile_read()
    t.close()
    return {"ms_per_step": round(ms, 5), "value": interior(level) / (ms / 1e3),
            "kernel_ms_per_launch": {nm: round(v / K, 5) for nm, v in zip(["residual", "forward", "backward"], kms)}}


def depth_bound(g, levels, threads, sm_mhz):
    """The dependency-depth bound of the substitutions: `levels` barrier
    steps per substitution (two substitutions per sweep) at the measured
    cycles of the shortest step body (ilu_step_floor, CTAs of `threads`)."""
    cyc = g.step_floor(threads, 4096)
    return {"steps_per_substitution": levels, "floor_cycles_per_step": round(cyc, 1), "floor_threads": threads,
            "us_per_sweep": round(2 * levels * cyc / (sm_mhz * 1e6) * 1e6, 2)}


def error_report(g, torch, P):
    """Errors of the measured configuration against FP64 references.  Two
    sweeps of the default tet from the same start in MIXED and in F64
    (matrix-free, as timed) against the oracle's two sweeps with the same
    polynomials (the oracle's own fit, imported); then PCG to a relative
    residual of 1e-8 in MIXED and in F64: iterations, final residuals and the
    difference of the two solutions."""
    from oracle import oracle as O
    N = 2 ** LEVEL
    pr = O.Problem(P, LEVEL, O.Coeff(*COEFF), deg=DEG)
    x0 = si.boundary_data(LEVEL, 21)
    b = si.rhs(LEVEL, RHS_SEED)
    want = O.smooth(pr.A, N, pr.Ls, pr.Dinv_s, x0.copy(), b, 2)
    scale = np.abs(want).max()
    out = {"sweeps_vs_oracle": {}, "tolerance": {"F64": 1e-12, "MIXED": "1e-5 relative per sweep"}}
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    sol = {}
    for name, prec in [("MIXED", g.MIXED), ("F64", g.F64)]:
        t = g.Tet(P, LEVEL, coeff=g.make_coeff(*COEFF), poly_degree=DEG, precision=prec,
                  stencil=g.STENCIL_ON_THE_FLY, values=g.VALUES_ON_THE_FLY, device=torch.cuda.current_device())
        t.import_surrogate(pr.coefs)
        xd = torch.tensor(x0, dtype=torch.float64, device="cuda")
        t.smooth(xd, bd, 2)
        out["sweeps_vs_oracle"][f"{name}_after_2_sweeps"] = float(np.abs(xd.cpu().numpy() - want).max() / scale)
        x = torch.zeros(g.num_nodes(LEVEL), dtype=torch.float64, device="cuda")
        it, rel, ok = t.solve(x, bd, g.PCG, 1e-8, 2000)
        sol[name] = (it, rel, bool(ok), x.cpu().numpy())
        t.close()
    ref = sol["F64"][3]
    out["pcg_to_1e-8"] = {nm: {"iterations": v[0], "relative_residual": v[1], "converged": v[2]}
                          for nm, v in sol.items()}
    out["pcg_MIXED_vs_F64_solution"] = float(np.abs(sol["MIXED"][3] - ref).max() / np.abs(ref).max())
    return out


def single_workload(args, g, torch, rank, world, dist, local):
    """The default line: the matrix-free MIXED sweep of the level-7 tet (the
    operator assembled and the surrogates evaluated on the fly), its roofline
    and depth bound, the other precisions and the stored variants as labelled
    extras, then the level-9, batch and error keys."""
    W = max(3, args.warmup)
    K = max(1, args.steps)
    P = si.macro_tet(TET_SEED)
    mf = dict(stencil=g.STENCIL_ON_THE_FLY, values=g.VALUES_ON_THE_FLY)
    t = g.Tet(P, LEVEL, coeff=g.make_coeff(*COEFF), poly_degree=DEG, precision=g.MIXED, device=local, **mf)
    nn = g.num_nodes(LEVEL)
    b_h = si.rhs(LEVEL, RHS_SEED)
    b = torch.tensor(b_h, dtype=torch.float64, device="cuda")
    x = torch.zeros(nn, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(W):
        t.smooth(x, b, 1)
    torch.cuda.synchronize()
    t.profile(True)
    t.profile_read()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ms_steps = time_steps(t, x, b, K, flush, stream, torch)
    if dist:
        dist.barrier()
    clk = clocks.stop()
    total_ms = sum(ms_steps)
    kms, launches = t.profile_read()
    t.profile(False)
    total_ms = max_over_ranks(total_ms, dist, "cuda")
    value = whole_job_rate(world, interior(LEVEL), K, total_ms)

    # end to end through the host-buffer entry point (copies inside the timed region)
    xh = np.zeros(nn)
    t.smooth_host(xh, b_h, 1)
    E = max(3, min(K, 50))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(E):
        t.smooth_host(xh, b_h, 1)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = world * interior(LEVEL) * E / e2e_s

    # roofline of the dominant kernel (HBM) and the sweep's depth bound
    alg = algorithmic(LEVEL, DEG)
    names = ["residual", "forward", "backward"]
    per_launch = {nm: kms[i] / K for i, nm in enumerate(names)}
    dom = max(["forward", "backward"], key=lambda nm: per_launch[nm])
    hbm, src = peaks()
    achieved = alg[dom]["bytes"] / (per_launch[dom] / 1e3) / 1e9
    sm_mhz = clk["sm_mhz"] or 2070.0
    levels = 3 * 2 ** LEVEL - 11
    depth = depth_bound(g, levels, 128, sm_mhz)  # slab CTAs: four compute warps per level step
    hbm_us = 1e6 * sum(alg[nm]["bytes"] for nm in names) / (hbm * 1e9)
    sweep_us = 1e3 * total_ms / K
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": profiled_traffic(dom), "kernel": f"{dom}_kernel", "peak_source": src,
            "algorithmic_bytes": alg[dom]["bytes"],
            "kernel_ms_per_launch": {nm: round(v, 5) for nm, v in per_launch.items()},
            "sweep": {"algorithmic_bytes": sum(alg[nm]["bytes"] for nm in names), "hbm_time_us": round(hbm_us, 2),
                      "depth_time_us": depth["us_per_sweep"], "measured_us": round(sweep_us, 2),
                      "frac_of_binding_bound": round(max(hbm_us, depth["us_per_sweep"]) / sweep_us, 4),
                      "binding": "depth" if depth["us_per_sweep"] > hbm_us else "hbm"},
            "depth": dict(depth, cycles_per_level_measured=round(
                (per_launch["forward"] + per_launch["backward"]) / 2 * 1e-3 / levels * sm_mhz * 1e6))}

    # the same sweep in the other precisions (matrix-free), and the stored variants as labelled extras
    Kp = max(3, min(K, 50))
    prec = {"F32": sweep_variant(g, torch, P, flush, stream, W, Kp, prec=g.F32, **mf),
            "F64": sweep_variant(g, torch, P, flush, stream, W, Kp, prec=g.F64, **mf)}
    nint = interior(LEVEL)
    stored = {
        "MIXED_stored_stencils": dict(sweep_variant(g, torch, P, flush, stream, W, Kp, prec=g.MIXED,
                                                    stencil=g.STENCIL_STORED, values=g.VALUES_ON_THE_FLY),
                                      stored_bytes_per_dof=112, note="14 FP64 coefficients per point, read by "
                                                                     "the residual: 132 instead of 28 B/DoF"),
        "F64_tabulated_values": dict(sweep_variant(g, torch, P, flush, stream, W, Kp, prec=g.F64,
                                                   stencil=g.STENCIL_ON_THE_FLY, values=g.VALUES_TABULATED),
                                     stored_bytes_per_dof=128, note="16 FP64 surrogate values per point, read by "
                                                                    "the substitutions instead of evaluated"),
    }
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "level": LEVEL, "degree": DEG, "precision": "MIXED",
                       "operator": "assembled on the fly", "surrogates": "evaluated on the fly",
                       "l2": "flushed between steps (256 MiB write)", "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * nn * 8,
                    "d2h_bytes_per_step": nn * 8},
            "gpu_launches": int(launches),
            "roofline": roof,
            "other_precisions": prec,
            "stored_variants": stored,
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                       "samples": clk["samples"]}}
    t.close()
    if rank == 0 and not args.no_extras:
        line["level9"] = level9_workload(args, g, torch, compact=True)
        line["batch"] = batch_workload(args, g, torch, compact=True)
        line["error"] = error_report(g, torch, P)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(8)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="default line without the level9/batch/error keys")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batch", "serve", "level9", "smoothers", "mg", "boundary", "packed"])
    ap.add_argument("--level", type=int, default=0, help="packed: the tet's level (8 by default)")
    ap.add_argument("--tets", type=int, default=0, help="batch: sweep only the first N of its 256 tets")
    ap.add_argument("--method", default="mg", choices=["richardson", "pcg", "mg"], help="serve: the requests' method")
    ap.add_argument("--requests", type=int, default=300)
    ap.add_argument("--gap-ms", type=float, default=0.5, help="mean gap of the Poisson arrivals (serve)")
    ap.add_argument("--max-cluster", type=int, default=0, help="CTAs per cluster cap of the served set-ups")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    import paper_2210_15280_gb300 as g
    torch.cuda.set_device(local)
    if args.workload == "batch" and world > 1:  # tets sharded over the ranks
        import torch.distributed as dist
        dist.init_process_group("nccl")
        line = batch_workload(args, g, torch, rank, world, dist)
        if rank == 0:
            print(json.dumps(line), flush=True)
        dist.destroy_process_group()
        return
    if args.workload != "single":
        if rank == 0:
            line = {"batch": batch_workload, "serve": serve_workload, "level9": level9_workload,
                    "smoothers": smoothers_workload, "mg": mg_workload,
                    "boundary": boundary_workload, "packed": packed_workload}[args.workload](
                args, g, torch)
            print(json.dumps(line), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    line = single_workload(args, g, torch, rank, world, dist, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
