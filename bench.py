"""Benchmark: DOF/s of the multigrid-preconditioned CG solve to relative residual 1e-8.

Workload (one "step" = one whole solve from x0 = 0, every hot-path step included):
3-D Poisson on the unit cube minus 20 seeded spheres (r ~ U(0.05, 0.15)), 128^3 background
grid, quadratic open B-splines (1,965,303 active functions), 5 levels, depth-2 octree cut-cell
quadrature, symmetric Nitsche on the immersed boundary, additive Schwarz smoothing.  The
headline value is the plain FP64 V-cycle solve (--precision fp64, default); the FP32
V-cycle inside the FP64 flexible CG ("mixed") and the FP64-finest hybrid are timed beside
it on the same problem, with their speed-up at the same 1e-8 residual.  The 512x512 2-D
workload, the batched solves and the learned stage are reported as sub-objects.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank solves its own seeded
geometry (independent problems, no collective on the data path: weak scaling); the
timed region is bracketed by barriers and the maximum over ranks is taken.
The CPU legs (cpu_baseline, and the reference arm) time the FP64 CPU oracle, the only
other place this script runs it, on a 32^3 instance of the same 20-sphere geometry.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF/s to rel. residual 1e-8 (PCG+MG) vs plain FP64 GPU; HBM GB/s of roofline"
PRESET = "spheres20_128_p2"
WORKLOADS = ("spheres20_128_p2", "discs10_512_p2", "discs10_512_p1", "discs10_512_p3", "disc1_32_p2", "box_256_p2")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one finest-level FP64 apply
# launch with p^T A p, per workload, from one ncu capture of the current kernel (null when
# none has been taken since the kernel last changed)
APPLY_TRAFFIC_BYTES = {
    # dram__bytes_read.sum 238.9 MB + dram__bytes_write.sum 18.6 MB (mean of two launches)
    "poisson3d-128x128x128-20spheres-bspline-p2-5levels-depth2-nitsche": 2.575e8,
}
APPLY_TRAFFIC_SOURCE = {
    "poisson3d-128x128x128-20spheres-bspline-p2-5levels-depth2-nitsche":
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of this kernel in this launch configuration "
        "(profiles/k_apply_zm3d_fp64_poisson3d_128_p2.md)",
}


def workload_name(pr) -> str:
    holes = {"disc1": "1disc", "discs10": "10discs", "spheres20": "20spheres", "none3": "noholes"}[pr.layout]
    size = "x".join([str(pr.n)] * pr.dim)
    basis = "bspline" if pr.basis == 0 else "lagrange"
    return f"poisson{pr.dim}d-{size}-{holes}-{basis}-p{pr.degree}-{pr.levels}levels-depth{pr.depth}-nitsche"


RTOL = 1e-8
# learned stage: training geometries of the workload's hole layout at LEARN_N^3, pairs per
# geometry, Adam steps, pairs per step, step size
LEARN_GEOMS, LEARN_N, LEARN_PAIRS, LEARN_STEPS, LEARN_BATCH, LEARN_LR = 4, 64, 8, 800, 4, 1e-3
LEARN_FCG = 5             # directions kept by the flexible CG that runs the learned stage
FP32_PEAK_NOTE = "152 SMs x 128 FP32 FMA/clk x 2 flop x 2070 MHz"
MAXIT = 2000
FP64_PEAK_NOTE = "152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz"
# CPU oracle sample: the workload's geometry (same hole layout and seed) on a 32^3 grid
# with 4 levels (coarsest 4^3, as the workload's 8^3 at 128^3 with 5 levels is one level
# below 16^3); depth-0 cut-cell quadrature, since the oracle's depth-2 assembly of that
# grid alone takes ~20 min (the solve phase, which is what is timed, does not depend on
# the quadrature depth: same rows, blocks and levels)
CPU_SAMPLE = {"n": 32, "levels": 4, "depth": 0}


def fp64_peak_tflops(sm_mhz: float = 2070.0) -> float:
    return 152 * 2 * 2 * sm_mhz * 1e6 / 1e12


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ CPU oracle legs
# Build once (one process, single-threaded), pickle the assembled system and hierarchy,
# then time solves in fresh processes: one alone (single thread) and one per host core
# at the same time (each an independent copy of the same solve: the oracle's sparse
# products are single-threaded, so the machine's throughput is that of parallel solves).
_ORACLE_BUILD = r"""
import pickle, sys, time
sys.path.insert(0, {root!r})
from oracle import discretize as D, geometry as G, multigrid as MG
from synthetic import config_layout, preset
pr = preset({preset!r}, n={n}, levels={levels}, depth={depth})
lay = config_layout(pr.layout, {seed})
t0 = time.perf_counter()
d = D.Discretization(G.Balls(lay.centers, lay.radii), pr.basis, pr.degree, pr.n, pr.depth, pr.bc)
H = MG.Hierarchy(d, pr.levels)
with open({path!r}, "wb") as f:
    pickle.dump({{"A": d.A, "b": d.b, "H": H, "n_active": int(d.n_active),
                 "build_s": time.perf_counter() - t0}}, f)
"""

_ORACLE_SOLVE = r"""
import json, pickle, sys, time
sys.path.insert(0, {root!r})
from oracle import multigrid as MG
o = pickle.load(open({path!r}, "rb"))
while time.time() < {start}:
    time.sleep(0.01)
times, its = [], []
for k in range({reps}):
    t0 = time.perf_counter()
    x, it, hist = MG.pcg(o["A"], o["b"], o["H"].precondition, rtol={rtol}, maxit={maxit})
    times.append(time.perf_counter() - t0)
    its.append(it)
print(json.dumps({{"n_active": o["n_active"], "times": times, "iterations": its, "rel": hist[-1],
                  "build_s": o["build_s"]}}))
"""

_ONE_THREAD = dict(OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


# the other workloads the oracle solves in full beside the sample (2-D: its assembly takes
# seconds for 32^2 and ~3 min for 512^2): name -> (preset, n, levels, depth)
CPU_FULL = {"disc1_32_p2": ("disc1_32_p2", 32, 3, 3), "discs10_512_p2": ("discs10_512_p2", 512, 6, 0)}


def oracle_build_start(seed: int = 0, preset: str = PRESET, sample: dict | None = None):
    """Starts the oracle's assembly of a CPU system in the background (the 3-D sample by default);
    returns (process, path)."""
    path = os.path.join(tempfile.mkdtemp(prefix="imgm_oracle_"), "system.pkl")
    code = _ORACLE_BUILD.format(root=ROOT, preset=preset, seed=seed, path=path, **(sample or CPU_SAMPLE))
    proc = subprocess.Popen([sys.executable, "-c", code], env=dict(os.environ, **_ONE_THREAD),
                            stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
    return proc, path


def oracle_build_wait(proc, path):
    _, err = proc.communicate(timeout=3600)
    if proc.returncode != 0:
        raise RuntimeError("oracle build failed: " + err[-2000:])
    return path


def oracle_solves(path: str, procs: int, reps: int):
    """Runs `procs` single-threaded solve processes at once, each timing `reps` solves of the
    pickled system; returns their JSON results."""
    start = time.time() + 2.0 + 0.05 * procs          # all start together after loading
    code = _ORACLE_SOLVE.format(root=ROOT, path=path, start=start, reps=reps, rtol=RTOL, maxit=MAXIT)
    ps = [subprocess.Popen([sys.executable, "-c", code], env=dict(os.environ, **_ONE_THREAD),
                           stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True) for _ in range(procs)]
    out = []
    for p in ps:
        o, e = p.communicate(timeout=3600)
        if p.returncode != 0:
            raise RuntimeError("oracle solve failed: " + e[-2000:])
        out.append(json.loads(o.strip().splitlines()[-1]))
    return out


def sample_text(o, procs: int, reps: int) -> str:
    return (f"FP64 CPU oracle (numpy/scipy) CG solve to 1e-8 of the 20-sphere workload geometry at "
            f"{CPU_SAMPLE['n']}^3 ({CPU_SAMPLE['levels']} levels, depth-{CPU_SAMPLE['depth']} cut-cell "
            f"quadrature, {o['n_active']} DOFs, {o['iterations'][0]} iterations), setup excluded; "
            f"{procs} single-threaded process{'es' if procs > 1 else ''} at once, {reps} solves each")


def cpu_full_entry(path: str, name: str, reps: int = 3):
    """Oracle throughput on a whole 2-D workload: one single-threaded solve process, and one per
    host core at once."""
    one = oracle_solves(path, 1, reps)[0]
    t1 = statistics.median(one["times"])
    ncpu = os.cpu_count() or 1
    many = oracle_solves(path, ncpu, 1)
    t_all = max(sum(o["times"]) for o in many)
    return {"workload": name, "n_active": one["n_active"], "iterations": one["iterations"][0],
            "single_thread": {"value": one["n_active"] / t1, "unit": "DOF/s", "cores": 1, "median_s": t1},
            "all_cores": {"value": ncpu * one["n_active"] / t_all, "unit": "DOF/s", "cores": ncpu,
                          "solves": ncpu},
            "oracle_build_s": one["build_s"], "kind": "oracle", "sample": "the whole workload"}


def cpu_baseline_entry(path: str, reps: int = 3):
    """Single-thread and all-cores throughput of the oracle solve on the CPU sample."""
    one = oracle_solves(path, 1, reps)[0]
    t1 = statistics.median(one["times"])
    ncpu = os.cpu_count() or 1
    many = oracle_solves(path, ncpu, reps)
    t_all = max(sum(o["times"]) for o in many)
    value_all = ncpu * reps * many[0]["n_active"] / t_all
    return {"value": value_all, "unit": "DOF/s", "cores": ncpu, "kind": "oracle",
            "sample": sample_text(many[0], ncpu, reps), "host_cpus": ncpu,
            "single_thread": {"value": one["n_active"] / t1, "unit": "DOF/s", "cores": 1,
                              "median_s": t1, "times_s": one["times"]},
            "oracle_build_s": one["build_s"]}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9 and f[1].isdigit():
                    rows.append(f)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [int(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() in ("active", "1")})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": int(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace('.', '', 1).isdigit())
                if any(r[3].replace('.', '', 1).isdigit() for r in rows) else None}


# ------------------------------------------------------------------ GPU arm
# The uneven batch: 16 seeded geometries, half 2-D (64^2 - 1024^2, 1-30 discs) and half 3-D
# (32^3 - 96^3, 1-30 spheres, depth-1 cut cells), p = 1-3, each with 1-8 right-hand sides
# (the first the manufactured one, the others random normal), solved by one graph launch
# in the mixed-precision form.  (The configuration names 64 geometries; 16 keep the host
# setup of the default run near a minute.)
BATCH_GEOMS, BATCH_SEED = 16, 2024


def batch_spec():
    """[(dim, n, holes, degree, levels, depth, nrhs, seed)] of the batch (seeded)."""
    import numpy as np
    rng = np.random.default_rng(BATCH_SEED)
    out = []
    for g in range(BATCH_GEOMS):
        dim = 2 if g % 2 == 0 else 3
        if dim == 2:
            n = int(rng.choice([64, 128, 256, 512, 1024]))
            levels, depth = int(np.log2(n)) - 3, 0                # coarsest 16^2
            deg = int(rng.integers(1, 4))
        else:
            n = int(rng.choice([32, 48, 64, 96]))
            levels = {32: 3, 48: 4, 64: 4, 96: 5}[n]               # coarsest 8^3 or 6^3
            depth = 1
            deg = int(rng.integers(1, 3)) if n > 48 else int(rng.integers(1, 4))
        out.append((dim, n, int(rng.integers(1, 31)), deg, levels, depth, int(rng.integers(1, 9)), 100 + g))
    return out


def run_batched(lib, torch, steps, warmup):
    """Aggregate DOF/s of the batch solved by one graph launch, and of the same solves one
    after the other (each through its own graph)."""
    from synthetic import random_holes
    ctxs, bs = [], []
    spec = batch_spec()
    for k, (dim, n, holes, deg, levels, depth, nrhs, seed) in enumerate(spec):
        r_lo, r_hi = (0.03, 0.1) if dim == 2 else (0.03, 0.08)
        lay = random_holes(dim, holes, r_lo, r_hi, seed)
        # 3-D members keep their finest level in FP64: random-normal right-hand sides put O(1)
        # entries on functions with sliver cut supports, whose Jacobi scale 1/sqrt(A_ii) would
        # carry them out of the FP32 range in an all-FP32 V-cycle
        S = lib.Solver(dim, lay.centers, lay.radii, n, deg, levels, depth, 1, basis=0, precision=1 if dim == 2 else 2)
        mask = torch.as_tensor(S.active_mask(), dtype=torch.float64, device="cuda")
        gen = torch.Generator(device="cuda").manual_seed(1000 + k)
        for j in range(nrhs):
            ctxs.append(S if j == 0 else S.clone())
            bs.append(S.rhs() if j == 0 else torch.randn(S.n_grid(), dtype=torch.float64, device="cuda",
                                                         generator=gen) * mask)
    dofs = sum(c.level_info(c.L)["n_active"] for c in ctxs)
    B = lib.Batch(ctxs)
    xs = [torch.zeros_like(b) for b in bs]
    for _ in range(warmup):
        B.solve(bs, [x.zero_() for x in xs], rtol=RTOL, maxit=MAXIT)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        _, res = B.solve(bs, [x.zero_() for x in xs], rtol=RTOL, maxit=MAXIT)
    e1.record()
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3 / steps
    for c, b, x in zip(ctxs, bs, xs):
        c.pcg_solve(b, x.zero_(), rtol=RTOL, maxit=MAXIT)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        for c, b, x in zip(ctxs, bs, xs):
            c.pcg_solve(b, x.zero_(), rtol=RTOL, maxit=MAXIT)
    e1.record()
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3 / steps
    B.close()
    for c in reversed(ctxs):
        c.close()
    return {"value": dofs / t_batch, "unit": "DOF/s", "ms_per_step": 1e3 * t_batch, "solves": len(ctxs),
            "problems": len(spec), "dofs_per_step": dofs, "sequential_value": dofs / t_seq,
            "speedup_vs_sequential": t_seq / t_batch, "max_iterations": max(r["iterations"] for r in res),
            "all_converged": all(r["status"] == 0 for r in res),
            "workload": "; ".join(f"{n}^{d} {h} {'discs' if d == 2 else 'spheres'} p{p} x{r} rhs"
                                  for d, n, h, p, _, _, r, _ in spec),
            "precision": "mixed: 2-D FP32 V-cycle, 3-D FP64 finest level and FP32 below, in FP64 flexible CG",
            "launch": "one CUDA graph: every solve a branch with its own device-side CG loop"}


def smoother_bandwidth(S, torch, stream):
    """The finest level's FP64 additive Schwarz smoothing (imgm_smooth: the one-function blocks'
    diagonal scaling and the stored blocks), timed from a captured CUDA graph of 50, against its
    algorithmic bytes: the inverses (sum n_j^2 x 8 B), per (block, function) pair its index (4 B),
    block id (4 B), gathered residual (8 B) and atomic update of z (2 x 8 B), and the diagonal pass
    over the level (r in, z out, 1/A_ii: 24 B per row)."""
    info = S.level_info(S.L)
    _, npairs, nvals = S.host_block_sizes(S.L)  # sum n_j (pairs), sum n_j^2 (inverse entries)
    r = S.rhs()
    z = torch.empty_like(r)
    reps = 50
    g = torch.cuda.CUDAGraph()
    try:
        with torch.cuda.graph(g):
            for _ in range(reps):
                S.smooth(r, z)
        g.replay()
        torch.cuda.synchronize()
    except Exception:
        g = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    if g is not None:
        g.replay()
    else:
        for _ in range(reps):
            S.smooth(r, z)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    nbytes = 8 * nvals + 32 * npairs + 24 * info["n_grid"]
    peak = measured_peaks().get("hbm_gbs")
    gbs = nbytes / t / 1e9
    return {"us": 1e6 * t, "algorithmic_bytes": nbytes, "achieved_gbs": gbs, "hbm_peak_gbs": peak,
            "frac_of_hbm": gbs / peak if peak else None, "blocks": info["n_blocks"], "block_pairs": npairs,
            "block_entries": nvals,
            "kernels": "k_scale_diag + k_blocks_pairs (finest level, FP64)"}


def vcycle_bandwidth(S, torch, stream, mixed):
    """One V-cycle (imgm_apply_preconditioner) timed from a captured CUDA graph of 20, with
    its algorithmic vector traffic: per level (13 + 2/2^d) s N_l bytes (pre-smoothing 2,
    residual 3, restriction 1 + 2^-d, prolongation and residual update 4 + 2^-d, post-
    smoothing 3 passes over vectors of s = 4 (FP32) or 8 bytes and N_l rows), against the
    measured HBM copy bandwidth (the V-cycle's vectors exceed L2 only on large grids)."""
    d = S.dim
    s_bytes = 4 if mixed else 8
    nbytes = sum((13 + 2 / 2 ** d) * s_bytes * S.level_info(l)["n_grid"] for l in range(2, S.L + 1))
    # the tables the V-cycle reads as well: each level's stored rows ((2p+1)^d coefficients, read by
    # its two residual applies) and its Schwarz block inverses (sum n_j^2, read by its two smoothings)
    ncoef = (2 * S.p + 1) ** d
    tbytes = sum(2 * s_bytes * (S.level_info(l)["n_band"] * ncoef + S.level_info(l)["block_entries"])
                 for l in range(2, S.L + 1))
    r = S.rhs()
    z = torch.empty_like(r)
    reps = 20
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(reps):
                S.apply_preconditioner(r, z)
        g.replay()
        torch.cuda.synchronize()
    except Exception:
        g = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    if g is not None:
        g.replay()
    else:
        for _ in range(reps):
            S.apply_preconditioner(r, z)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    peak = measured_peaks().get("hbm_gbs")
    gbs = nbytes / t / 1e9
    gbt = (nbytes + tbytes) / t / 1e9
    return {"us": 1e6 * t, "algorithmic_bytes": nbytes, "achieved_gbs": gbs, "hbm_peak_gbs": peak,
            "frac_of_hbm": gbs / peak if peak else None,
            "table_bytes": tbytes, "achieved_gbs_with_tables": gbt,
            "frac_of_hbm_with_tables": gbt / peak if peak else None,
            "note": "algorithmic_bytes: vector passes; table_bytes: stored operator rows and block inverses "
                    "read by the two residual applies and two smoothings of every level"}


def reduce_replicas(dist, device, times, units):
    """Whole-job figures of N independent replicas: each time is the maximum over ranks
    (the job ends with its slowest rank) and the work is the sum of every rank's units
    (the ranks solve different seeded geometries, so their DOF counts differ)."""
    import torch
    if dist is None:
        return list(times), float(units)
    t = torch.tensor(list(times), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.tolist()], float(u.item())


def apply_flops(S) -> float:
    """Algorithmic FP64 flops of one finest-level operator apply: 8(2p+1) per tensor row
    (sum factorisation) + 2 (2p+1)^d per stored row."""
    info = S.level_info(S.L)
    p, d = S.p, S.dim
    tensor_rows = info["n_active"] - info["n_band"]
    return (8 * (2 * p + 1) if d == 2 else 16 * (2 * p + 1)) * tensor_rows + 2 * (2 * p + 1) ** d * info["n_band"]


def run_learned(args, lib, torch, pr, S64, timed_solves, total_units, t64, res64):
    """The learned stage on a 3-D workload: train the network on the V-cycle's own
    residual/error pairs of LEARN_GEOMS seeded geometries of the same hole layout at
    LEARN_N^3 (one level fewer), then time the FP64 solve of the workload with the stage
    against the plain FP64 solve (same solver, same right-hand side, same tolerance)."""
    from synthetic import config_layout, initial_weights, preset, random_error
    tr = preset(args.workload, n=LEARN_N, levels=pr.levels - 1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pairs, shape = [], None
    rms = torch.zeros(LEARN_GEOMS * LEARN_PAIRS, dtype=torch.float64, device="cuda")
    for g in range(LEARN_GEOMS):
        lay_g = config_layout(tr.layout, 1000 + g)
        Sg = lib.Solver(tr.dim, lay_g.centers, lay_g.radii, tr.n, tr.degree, tr.levels, tr.depth, tr.bc,
                        basis=tr.basis, precision=0)
        m = Sg.level_info(Sg.L)["m"]
        shape = (m, m, m)
        mask_h = Sg.active_mask()
        mask = torch.as_tensor(mask_h, device="cuda")
        for k in range(LEARN_PAIRS):
            e0 = torch.as_tensor(random_error(mask_h.size, 10_000 * g + k) * mask_h, device="cuda")
            j = g * LEARN_PAIRS + k
            r1, e1 = Sg.learned_pair(e0, r_rms=rms[j:j + 1])
            pairs.append((r1, e1, mask))
        torch.cuda.synchronize()
        Sg.close()
    t_pairs = time.perf_counter() - t0
    net = lib.Net(initial_weights(args.seed))
    t1 = time.perf_counter()
    sigma = 1.0 / float(rms.mean().item())          # the set's input scale
    losses = lib.train_net(net, pairs, shape, steps=LEARN_STEPS, lr=LEARN_LR, batch=LEARN_BATCH,
                           in_scale=sigma).cpu().numpy()
    t_train = time.perf_counter() - t1
    # the network's forward pass on the workload's grid alone (20 launches after warm-up)
    info = S64.level_info(S64.L)
    m = info["m"]
    mask_w = torch.as_tensor(S64.active_mask(), device="cuda")
    xin = torch.randn(info["n_grid"], dtype=torch.float64, device="cuda") * mask_w
    yout = torch.empty_like(xin)
    for _ in range(3):
        net.forward(xin, (m, m, m), mask=mask_w, out=yout)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    torch.cuda.nvtx.range_push("learned_forward")          # lets ncu select these launches
    f0.record(stream)
    for _ in range(20):
        net.forward(xin, (m, m, m), mask=mask_w, out=yout)
    f1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    fwd_ms = f0.elapsed_time(f1) / 20
    fwd_flops = 2.0 * m ** 3 * 27 * (16 + 16 * 16 + 16)
    S64.set_net(net)
    S64.set_fcg(LEARN_FCG)
    t_l, res_l = timed_solves(S64, args.steps, args.warmup, "solve_learned")
    S64.set_fcg(0)
    S64.set_net(None)
    net.close()
    return {
        "value": total_units / t_l, "unit": "DOF/s", "ms_per_step": 1e3 * t_l / args.steps,
        "iterations": res_l[0]["iterations"], "true_rel_residual": res_l[-1]["true_rel_residual"],
        "gpu_launches_per_solve": int(res_l[0]["kernel_launches"]),
        "plain_fp64": {"value": total_units / t64, "ms_per_step": 1e3 * t64 / args.steps,
                       "iterations": res64[0]["iterations"],
                       "gpu_launches_per_solve": int(res64[0]["kernel_launches"])},
        "speedup_vs_plain_fp64": t64 / t_l,
        "training": {"geometries": LEARN_GEOMS, "n": LEARN_N, "levels": tr.levels, "pairs": len(pairs),
                     "steps": LEARN_STEPS, "batch": LEARN_BATCH, "lr": LEARN_LR, "input_scale": sigma,
                     "pairs_s": t_pairs,
                     "train_s": t_train, "loss_first": float(losses[:4].mean()),
                     "loss_last": float(losses[-20:].mean())},
        "stage": f"z += omega N(r - A z) after every FP64 V-cycle, truncated flexible CG FCG({LEARN_FCG})",
        "forward": {"ms": fwd_ms, "flops": fwd_flops, "achieved_tflops": fwd_flops / (fwd_ms * 1e-3) / 1e12,
                    "tensor_flops": 2.0 * m ** 3 * 27 * 256,
                    "bf16_peak_tflops": measured_peaks().get("bf16_tflops"),
                    "peak_source": "measured bf16 burst (MEASURED_PEAKS.json); tensor_flops are the 16->16 "
                                   "layer's (89 % of the algorithmic flops; all three layers run on the tensor cores)",
                    "frac_of_bf16_peak": (fwd_flops / (fwd_ms * 1e-3) / 1e12) / measured_peaks()["bf16_tflops"]
                    if measured_peaks().get("bf16_tflops") else None,
                    "kernels": forward_kernels(),
                    "timing": "20 stream launches of the whole forward, CUDA events"},
    }


def forward_kernels():
    """The network's forward kernels for the IMGM_NET_TC setting the library reads."""
    mode = os.environ.get("IMGM_NET_TC", "")
    if mode.startswith("0"):
        return "k_pack, then k_conv for the three layers (FP32 FMA on the CUDA cores)"
    if mode == "48":
        return ("k_pack, then k_conv_tcz for the 1->16, 16->16 and 16->1 layers (tcgen05 bf16 MMAs of N = 48 "
                "with the z taps folded in, FP32 accumulators sliding along z in tensor memory; channels "
                "zero-padded to 16)")
    return ("k_pack, then k_conv16_tc for the 1->16, 16->16 and 16->1 layers (implicit GEMM on tcgen05: an "
            "8 x 16 voxel patch (M = 128) x 16 output channels per MMA, K = 16 input channels per tap, 27 taps "
            "into one FP32 accumulator in tensor memory; input planes staged by cp.async in a 4-plane ring; "
            "channels zero-padded to 16)")


def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1903_10977_gb300 as lib
    from synthetic import config_layout, preset

    # the oracle's CPU sample is assembled on one host core while the GPU legs run
    oracle, oracle_full = None, {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        oracle = oracle_build_start(args.seed)
        if args.workload == PRESET and not args.quick:
            for name, (pname, n, levels, depth) in CPU_FULL.items():
                oracle_full[name] = oracle_build_start(args.seed, pname, {"n": n, "levels": levels, "depth": depth})
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    pr = preset(args.workload)
    lay = config_layout(pr.layout, args.seed + rank)
    code = {"fp64": 0, "mixed": 1, "hybrid": 2}[args.precision]
    headline = args.workload == PRESET

    def make(precision, smoother=0, p=pr, l=lay):
        return lib.Solver(p.dim, l.centers, l.radii, p.n, p.degree, p.levels, p.depth, p.bc, basis=p.basis,
                          lo=l.lo, hi=l.hi, precision=precision, smoother=smoother)

    t0 = time.perf_counter()
    S = make(code)
    setup_s = time.perf_counter() - t0
    info = S.level_info(S.L)
    n_active, n_grid = info["n_active"], info["n_grid"]
    b = S.rhs()
    x = torch.zeros_like(b)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > 129 MB L2
    stream = torch.cuda.current_stream()

    def timed_solves(solver, steps, warmup, label, rhs=None):
        """Device time of `steps` whole solves, each after an L2 flush (flush outside the events).
        The timed solves sit in the NVTX range `label` (lets ncu select their launches)."""
        bb = b if rhs is None else rhs
        xx = x if rhs is None else torch.zeros_like(rhs)
        for _ in range(warmup):
            xx.zero_()
            solver.pcg_solve(bb, xx, rtol=RTOL, maxit=MAXIT)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        res = []
        barrier()
        torch.cuda.nvtx.range_push(label)
        for k in range(steps):
            flush.fill_(float(k))
            xx.zero_()
            ev[k][0].record(stream)
            _, r, _ = solver.pcg_solve(bb, xx, rtol=RTOL, maxit=MAXIT)
            ev[k][1].record(stream)
            res.append(r)
        torch.cuda.nvtx.range_pop()
        barrier()
        return sum(a.elapsed_time(c) for a, c in ev) / 1e3, res

    def form(t, res, units, t_ref=None):
        out = {"value": units / t, "unit": "DOF/s", "ms_per_step": 1e3 * t / len(res),
               "iterations": res[0]["iterations"], "true_rel_residual": max(r["true_rel_residual"] for r in res),
               "gpu_launches_per_solve": int(res[0]["kernel_launches"])}
        if t_ref is not None:
            out["speedup_vs_fp64"] = t_ref / t
        return out

    with ClockSampler(local_rank) as clk:
        t_dev, results = timed_solves(S, args.steps, args.warmup, f"solve_{args.precision}")
    clocks = clk.summary()
    units = n_active * args.steps
    # the other V-cycle precisions on the same problem, each against the FP64 solve
    t64, res64, S64 = (t_dev, results, S) if code == 0 else (None, None, None)
    forms = {}
    wanted = [f for f in ("fp64", "mixed", "hybrid") if f != args.precision and (f == "fp64" or not args.quick)]
    for f in wanted:
        Sf = make({"fp64": 0, "mixed": 1, "hybrid": 2}[f])
        tf, rf = timed_solves(Sf, args.steps, args.warmup, f"solve_{f}")
        if f == "fp64":
            t64, res64, S64 = tf, rf, Sf
        else:
            forms[f] = (tf, rf)
            Sf.close()
    learned = None
    if pr.dim == 3 and not args.no_learned:
        learned = run_learned(args, lib, torch, pr, S64, timed_solves, units, t64, res64)

    # end to end: host (pinned) b in, host x out, through the C-ABI
    bh = torch.empty(n_grid, dtype=torch.float64, pin_memory=True)
    bh.copy_(b.cpu())
    xh = torch.empty(n_grid, dtype=torch.float64, pin_memory=True)
    for _ in range(max(1, args.warmup // 2)):
        S.pcg_solve_host_ptr(bh.data_ptr(), xh.data_ptr(), rtol=RTOL, maxit=MAXIT)
    barrier()
    e0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        S.pcg_solve_host_ptr(bh.data_ptr(), xh.data_ptr(), rtol=RTOL, maxit=MAXIT)
    barrier()
    t_e2e = time.perf_counter() - e0

    apply_ms, apply_graph = time_finest_apply(S, torch, stream, n_grid)
    vcycle = vcycle_bandwidth(S, torch, stream, code == 1)
    smoother = smoother_bandwidth(S64 if S64 is not None else S, torch, stream)
    # the 2-D 512x512 workload and the batch beside the 3-D headline
    poisson2d = run_2d(args, lib, torch, timed_solves) if headline and not args.quick else None
    batched = run_batched(lib, torch, max(1, args.steps // 2), 1) if headline and not args.quick else None

    times = [t_dev, t64, t_e2e] + [forms[f][0] for f in sorted(forms)]
    times, total_units = reduce_replicas(dist, "cuda", times, units)
    t_dev, t64, t_e2e = times[:3]
    if dist is not None:
        dist.destroy_process_group()
    if rank != 0:
        return None
    value = total_units / t_dev
    flops = apply_flops(S)
    achieved = flops / (apply_ms * 1e-3) / 1e12
    peak = fp64_peak_tflops()
    wl = workload_name(pr)
    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if code == 0 else "f64+f32", "data": "synthetic",
        "config": {"workload": wl, "dim": pr.dim, "n": pr.n,
                   "basis": "bspline" if pr.basis == 0 else "lagrange", "degree": pr.degree,
                   "levels": pr.levels, "holes": lay.n_holes, "depth": pr.depth, "bc": "nitsche", "rtol": RTOL,
                   "n_active": n_active, "n_grid": n_grid, "seed": args.seed, "parallelism": f"replicas{world}",
                   "vcycle": {0: "fp64", 1: "fp32 (Jacobi-scaled) in fp64 flexible CG",
                              2: "fp64 finest level, fp32 (Jacobi-scaled) below, in fp64 flexible CG"}[code],
                   "smoother": "additive Schwarz",
                   "l2": "flushed (256 MiB write) before every timed solve, flush outside the events",
                   "iterations": results[0]["iterations"],
                   "true_rel_residual": max(r["true_rel_residual"] for r in results), "setup_s": setup_s},
    }
    if code != 0:
        line["fp64"] = form(t64, res64, total_units)
        line["speedup_vs_fp64"] = t64 / t_dev
    for k, f in enumerate(sorted(forms)):
        line[f] = form(times[3 + k], forms[f][1], total_units, t64)
    line.update({
        "poisson2d_512": poisson2d,
        "batched": batched,
        "learned": learned,
        "vcycle": vcycle,
        "smoother": smoother,
        "e2e": {"value": total_units / t_e2e, "unit": "DOF/s", "h2d_bytes_per_step": 8 * n_grid,
                "d2h_bytes_per_step": 8 * n_grid},
        "gpu_launches": sum(int(r["kernel_launches"]) for r in results),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": APPLY_TRAFFIC_BYTES.get(wl),
                     "traffic_source": APPLY_TRAFFIC_SOURCE.get(wl, "no capture of the current kernel"),
                     "kernel": ("k_apply_tile2d<double>" if pr.dim == 2 else "k_apply_zm3d<double>")
                               + " (finest-level FP64 operator apply, imgm_apply_operator)",
                     "peak_source": "derived: " + FP64_PEAK_NOTE, "flops_per_launch": flops,
                     "launch_ms": apply_ms,
                     "timing": "200 launches replayed from a CUDA graph" if apply_graph
                               else "200 stream launches"},
        "clocks": clocks,
    })
    if oracle is not None:
        try:
            line["cpu_baseline"] = cpu_baseline_entry(oracle_build_wait(*oracle))
        except Exception as e:  # the GPU number stands without it
            line["cpu_baseline"] = {"error": str(e)[:200]}
        if not headline:
            line["cpu_baseline_note"] = "cpu_baseline is measured on the 3-D 20-sphere workload's 32^3 sample"
        full = {}
        for name, proc in oracle_full.items():
            try:
                full[name] = cpu_full_entry(oracle_build_wait(*proc), workload_name(preset(name)))
            except Exception as e:
                full[name] = {"error": str(e)[:200]}
        if full:
            line["cpu_oracle_2d"] = full
    if S64 is not S and S64 is not None:
        S64.close()
    S.close()
    return line


def time_finest_apply(S, torch, stream, n_grid):
    """Per-launch time of the finest-level FP64 operator apply (run once per CG iteration in
    every form and three times per FP64 iteration), 200 launches replayed from a captured
    CUDA graph so that host launch gaps do not enter (stream launches as the fallback)."""
    xs = torch.randn(n_grid, dtype=torch.float64, device="cuda") * torch.as_tensor(
        S.active_mask(), dtype=torch.float64, device="cuda")
    ys = torch.empty_like(xs)
    for _ in range(5):
        S.apply_operator(xs, ys)
    reps = 200
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    graph = None
    try:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for _ in range(reps):
                S.apply_operator(xs, ys)
        graph.replay()
        torch.cuda.synchronize()
    except Exception:
        graph = None
    torch.cuda.nvtx.range_push("finest_apply_timing")      # lets ncu select these launches
    k0.record(stream)
    if graph is not None:
        graph.replay()
    else:
        for _ in range(reps):
            S.apply_operator(xs, ys)
    k1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    return k0.elapsed_time(k1) / reps, graph is not None


def run_2d(args, lib, torch, timed_solves):
    """The 2-D 512x512 quadratic B-spline workload (10 discs, 6 levels): FP64, mixed and the
    coloured multiplicative smoother (same precision as the mixed form)."""
    from synthetic import config_layout, preset
    pr = preset("discs10_512_p2")
    lay = config_layout(pr.layout, args.seed)
    out = {"workload": workload_name(pr)}
    t64 = None
    for name, prec, sm in (("fp64", 0, 0), ("mixed", 1, 0), ("multiplicative_mixed", 1, 1)):
        S = lib.Solver(pr.dim, lay.centers, lay.radii, pr.n, pr.degree, pr.levels, pr.depth, pr.bc,
                       basis=pr.basis, lo=lay.lo, hi=lay.hi, precision=prec, smoother=sm)
        units = S.level_info(S.L)["n_active"] * args.steps
        t, res = timed_solves(S, args.steps, args.warmup, f"solve2d_{name}", rhs=S.rhs())
        t64 = t if name == "fp64" else t64
        out[name] = {"value": units / t, "unit": "DOF/s", "ms_per_step": 1e3 * t / args.steps,
                     "iterations": res[0]["iterations"],
                     "true_rel_residual": max(r["true_rel_residual"] for r in res),
                     "gpu_launches_per_solve": int(res[0]["kernel_launches"]), "speedup_vs_fp64": t64 / t}
        out["n_active"] = S.level_info(S.L)["n_active"]
        S.close()
    return out


def run_reference(args, rank):
    """The oracle on the CPU sample: one single-threaded solve process per host core, each
    doing warmup + steps solves; value = DOFs of the timed solves of all processes over the
    longest process's timed span."""
    if rank != 0:
        return None
    path = oracle_build_wait(*oracle_build_start(args.seed))
    ncpu = os.cpu_count() or 1
    outs = oracle_solves(path, ncpu, args.warmup + args.steps)
    t = max(sum(o["times"][args.warmup:]) for o in outs)
    n_act = outs[0]["n_active"]
    value = ncpu * args.steps * n_act / t
    from synthetic import preset
    pr = preset(PRESET)
    return {"metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(pr), "cpu_sample": f"{CPU_SAMPLE['n']}^3 instance of the same "
                       f"geometry, {CPU_SAMPLE['levels']} levels, depth {CPU_SAMPLE['depth']}", "rtol": RTOL,
                       "n_active": n_act, "iterations": outs[0]["iterations"][0]},
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": ncpu, "kind": "oracle",
                             "sample": sample_text(outs[0], ncpu, args.warmup + args.steps)
                                       + f" (the first {args.warmup} of each untimed)",
                             "host_cpus": ncpu, "oracle_build_s": outs[0]["build_s"]},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=PRESET, choices=WORKLOADS,
                    help="the headline is the 3-D 128^3 20-sphere quadratic B-spline workload; the others are "
                         "the other configurations of the same study")
    ap.add_argument("--no-learned", action="store_true",
                    help="3-D workloads: skip training the learned stage and timing the FP64 solve with it")
    ap.add_argument("--quick", action="store_true",
                    help="time the chosen precision (and FP64) only: no other forms, 2-D workload or batch")
    ap.add_argument("--precision", default="fp64", choices=["mixed", "fp64", "hybrid"],
                    help="V-cycle arithmetic of the headline solves (the others are timed beside it)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        line = run_ours(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
