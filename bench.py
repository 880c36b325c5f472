#!/usr/bin/env python
"""CTMRG moves/s on one GB300: Hermitian Z2 path vs the dense path, same GPU.

Workload: real C4v iPEPS, d=2, D=6 (double-layer legs 36 = 21 even + 15 odd),
chi=144, seeded N(0,1) tensor (seed 1159600+3), D4-symmetrised, max|A|=1.
One step = one C4v CTMRG move (enlarged corner, projector, truncation,
renormalisation, normalisation). L2 (129 MB) is flushed between timed moves
by writing a 512 MB buffer outside the timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints ONE JSON line (rank 0). `value` is the Z2 path (TF32x3 block GEMMs,
subspace eigensolver) over the K moves after W warm-up moves. Beside it:
the same moves split into the transient (the first four timed moves, while
the environment still changes) and a steady state (ten moves after move 50);
a table of moves/s and |dE| for {Z2, dense basis} x {FP64 GEMM + FP64 syevd,
TF32x3 GEMM + FP64 syevd, FP64 GEMM + subspace eigensolver, TF32x3 GEMM +
subspace eigensolver}, with the Z2/dense ratio at equal arithmetic; HOTRG steps/s (Z2 vs dense) with the odd
sector fraction; the complex workload; the batched workload.
With torchrun (N>1) every rank runs an independent replica ("replicas only":
the method has no exchange step) and the value is the sum of moves over
ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CTMRG moves/s Z2-Hermitian vs dense (same GB300), D=6 χ=144, |ΔE|≤1e-7"
WORKLOAD = 3
FLUSH_BYTES = 512 << 20

# DRAM traffic per launch of the roofline kernel from one ncu capture, valid only
# while the kernel source is unchanged (sha256 of the file, first 16 hex digits).
NCU_TRAFFIC = {
    # FP64 block GEMM, one ncu capture of a D=6 chi=144 move: mean of its G3/G4/G5 launches
    "gemm_f64": {"bytes_per_launch": 143.3e6, "source_sha": "ac07f1d8a4d24d63"},
    # tensor-core GEMM, one ncu capture of two steady-state D=6 chi=144 moves: mean over its launches
    "gemm_tc_tf32x3": {"bytes_per_launch": 56.6e6, "source_sha": "c3b7279478e6ad5a"},
    # the same capture, mean over its split-output launches (G2-G5, the dominant kernel)
    "gemm_tc_split_tf32x3": {"bytes_per_launch": 131.5e6, "source_sha": "c3b7279478e6ad5a"},
}

EIG_LABEL = {"f64": "FP64 syevd per parity block", "f32p": "FP32 syevd + FP64 Loewdin and projection",
             "subspace": "warm-started subspace iteration (tcgen05 products, FP32 Rayleigh-Ritz), FP64 projection",
             "adaptive": "warm-started subspace iteration, residual tolerance following the change of the kept "
                         "spectrum per move (1e-3 .. 1e-5), FP64 projection"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", default="tf32x3", choices=["f64", "tf32x3", "tf32", "bf16x3"])
    p.add_argument("--eig", default="subspace", choices=["f64", "f32p", "subspace", "adaptive"])
    p.add_argument("--no-table", action="store_true", help="skip the {Z2, dense} x arithmetic table")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-check", action="store_true", help="skip the |dE| run to 50 moves and the steady state")
    p.add_argument("--no-complex", action="store_true", help="skip the complex workload (D=5, chi=100)")
    p.add_argument("--no-dtypes", action="store_true", help="skip the per-dtype |dE| / rho errors (50 moves each)")
    p.add_argument("--no-batched", action="store_true", help="skip the batched workload (32 instances)")
    p.add_argument("--no-hotrg", action="store_true", help="skip the HOTRG line")
    p.add_argument("--no-directional", action="store_true", help="skip the directional (non-C4v) CTMRG line")
    p.add_argument("--profile-region", action="store_true",
                   help="profiling runs only: W warm-up moves, then K moves inside cudaProfilerStart/Stop "
                        "(for ncu --profile-from-start off); prints a short JSON line, no bench line")
    p.add_argument("--profile-directional", action="store_true",
                   help="profiling runs only: the directional CTMRG (D=4, chi=64, seeded asymmetric tensor, "
                        "polar SVD), two sweeps, then one sweep inside cudaProfilerStart/Stop")
    p.add_argument("--basis", default="hermitian", choices=["hermitian", "dense"],
                   help="profiling runs only: the basis of the profiled moves")
    p.add_argument("--workload", type=int, default=WORKLOAD,
                   help="smaller workloads (1, 2) are for profiling runs, not bench lines")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def emit(obj):
    print(json.dumps(obj), flush=True)


def replica_throughput(sec: float, steps: int, world: int, device) -> tuple[float, float]:
    """Whole-job moves/s of `world` independent replicas (one per GPU, no exchange between them):
    world * steps moves in the slowest rank's time, taken as the max over ranks after the timed
    region. Returns (moves/s, seconds)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([sec], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        sec = float(t.item())
    return world * steps / sec, sec


def golden_snapshot(moves: int, k: int | None = None):
    path = os.path.join(ROOT, "tests", "golden", f"ctmrg_w{WORKLOAD if k is None else k}.json")
    try:
        with open(path) as f:
            return json.load(f)["checkpoints"].get(str(moves))
    except OSError:
        return None


def golden_energy(moves: int, k: int | None = None):
    snap = golden_snapshot(moves, k)
    return None if snap is None else snap["energy"]


def workload_name(k: int) -> str:
    """The config.workload string of real workload k, the same on both arms."""
    from paper_2410_11596_gb300 import inputs
    w = inputs.WORKLOADS[k]
    D = w["D"]
    return (f"real C4v iPEPS d={w['d']} D={D} chi={w['chi']} (q={D * D}: {D * (D + 1) // 2} even/"
            f"{D * (D - 1) // 2} odd), seeded N(0,1), D4-symmetrised, max|A|=1")


def r3(x):
    """Rounded for the JSON line (3 significant digits)."""
    if x is None:
        return None
    return float(f"{x:.3g}")


# ---------------------------------------------------------------------------
# CPU side: the oracle (reference arm and cpu_baseline)


def oracle_setup():
    from oracle import ctmrg as oc, doublelayer as odl
    from paper_2410_11596_gb300 import inputs
    w = inputs.WORKLOADS[WORKLOAD]
    A = inputs.workload_tensor(WORKLOAD)
    a = odl.double_layer(A)
    C, T = oc.init_environment(a)
    C, T = C / np.abs(C).max(), T / np.abs(T).max()
    C, T, _ = oc.move(C, T, a, w["chi"])   # the first move starts from chi0 = D^2 (cheap)
    return oc, a, C, T, w["chi"]


def oracle_moves(n: int, state=None):
    """Time n full-size oracle moves; returns (seconds per move list, state)."""
    oc, a, C, T, chi = state or oracle_setup()
    ts = []
    for _ in range(n):
        t0 = time.perf_counter()
        C, T, _ = oc.move(C, T, a, chi)
        ts.append(time.perf_counter() - t0)
    return ts, (oc, a, C, T, chi)


def oracle_sample(n: int, warmup: int) -> str:
    from paper_2410_11596_gb300 import inputs
    w = inputs.WORKLOADS[WORKLOAD]
    n_c = w["chi"] * w["D"] ** 2
    return (f"{n} full-size oracle moves (D={w['D']}, chi={w['chi']}, C' {n_c}x{n_c} numpy eigh) after an "
            f"untimed traced-boundary init, first move and {warmup} warm-up moves; numpy BLAS with its default "
            "thread count")


def cpu_baseline(n: int = 3):
    ts, _ = oracle_moves(n)
    return {"value": n / float(np.sum(ts)), "unit": "moves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": oracle_sample(n, 0)}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    # a full-size oracle move takes a few seconds on the host cores; K and W
    # are bounded so that the run ends within a few minutes
    steps, warmup = min(args.steps, 40), min(args.warmup, 10)
    state = None
    if warmup:
        _, state = oracle_moves(warmup, state)
    ts, _ = oracle_moves(steps, state)
    sec = float(np.sum(ts))
    val = steps / sec
    cores = os.cpu_count()
    emit({"impl": "reference", "metric": METRIC, "value": val, "unit": "moves/s", "n_gpus": args.gpus,
          "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * sec / steps,
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
          "data": "synthetic",
          "config": {"workload": workload_name(WORKLOAD), "basis": "dense (the oracle works in the plain basis)",
                     "path": "dense FP64 oracle (numpy eigh, tensordot) on host cores"},
          "cpu_baseline": {"value": val, "unit": "moves/s", "cores": cores, "kind": "oracle",
                           "sample": oracle_sample(steps, warmup)},
          "e2e": {"value": val, "unit": "moves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})


# ---------------------------------------------------------------------------
# GPU side


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples: $HS_CLOCKS_DIR if set, else the temporary directory
        self.path = os.path.join(os.environ.get("HS_CLOCKS_DIR") or tempfile.gettempdir(), f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def fp64_peak_tflops(torch, dev):
    """cuBLAS DGEMM 4096^3, best of 4 (the FP64 pipe's measured rate on this GPU)."""
    a = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    b = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
    best = 1e9
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        a @ b
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2 * 4096 ** 3 / (best * 1e-3) / 1e12


def measured_bf16_tflops():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"   # profiling recipe fallback (bf16 burst)


def source_sha(rel):
    with open(os.path.join(ROOT, rel), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def timed_moves(torch, c, ctx, n, flush):
    """n moves, each bracketed by CUDA events on the context stream; L2 flushed between."""
    s = ctx.stream
    ms = []
    for _ in range(n):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        c.move()
        e1.record(s)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def run_profile_directional(args):
    """One directional sweep (four moves) inside cudaProfilerStart/Stop, for ncu --profile-from-start off."""
    import torch
    from paper_2410_11596_gb300 import build, inputs, _lib as L
    from paper_2410_11596_gb300.api import Context, DirectionalCTMRG
    if not os.path.exists(L.LIB_PATH):
        build.build()
    ctx = Context(0)
    A = inputs.asymmetric_ipeps(2, 4, inputs.SEED_BASE + 5204)
    c = DirectionalCTMRG(ctx, A, 64, basis=args.basis, svd="polar")
    c.run(2)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    c.sweep()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    emit({"profile_directional": True, "D": 4, "chi": 64, "basis": args.basis, "svd": "polar",
          "bonds": [c.bond(b) for b in range(4)]})


def run_profile_region(args):
    """W warm-up moves, then K moves bracketed by cudaProfilerStart/Stop."""
    import torch
    from paper_2410_11596_gb300 import _lib as L, build, inputs
    from paper_2410_11596_gb300.api import CTMRG, Context
    if not os.path.exists(L.LIB_PATH):
        build.build()
    w = inputs.WORKLOADS[WORKLOAD]
    ctx = Context(0)
    c = CTMRG(ctx, inputs.workload_tensor(WORKLOAD), w["chi"], basis=args.basis, precision=args.precision,
              backend="own", eig=args.eig)
    c.run(args.warmup)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    infos = c.run(args.steps)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    emit({"profile_region": True, "workload": WORKLOAD, "basis": args.basis, "warmup": args.warmup,
          "steps": args.steps, "subspace_converged": sum(1 for i in infos if i["flags"] & 2)})


def arm(torch, ctx, A, chi, flush, basis, precision, eig, nwarm, ntimed, check_move, h):
    """moves/s of one {basis, arithmetic} combination (ntimed moves after nwarm), and |dE| against
    the oracle at move check_move (run on to it if needed)."""
    from paper_2410_11596_gb300.api import CTMRG
    c = CTMRG(ctx, A, chi, basis=basis, precision=precision, backend="own", eig=eig)
    c.run(nwarm)
    ms = timed_moves(torch, c, ctx, ntimed, flush)
    done = nwarm + ntimed
    dE = None
    ref = golden_energy(check_move)
    if ref is not None and check_move >= done:
        c.run(check_move - done)
        dE = abs(c.energy(h) - ref)
    conv = sum(1 for i in c.infos[nwarm:nwarm + ntimed] if i.get("flags", 0) & 2)
    del c
    return {"moves_per_s": r3(ntimed / (np.sum(ms) / 1e3)), "abs_dE": r3(dE), "moves": f"{nwarm + 1}-{done}",
            "dE_at": check_move, **({"subspace_converged": conv} if eig in ("subspace", "adaptive") else {})}


def hotrg_line(torch, ctx):
    """HOTRG steps/s, Z2 vs dense basis, with FP64 and with TF32x3 block GEMMs (FP64 Gram eig
    in both), and the odd fraction of the kept states per step (Z2, TF32x3)."""
    from paper_2410_11596_gb300 import inputs
    from paper_2410_11596_gb300.api import HOTRG
    out = []
    for D, chi in ((2, 16), (2, 32), (4, 16), (4, 24), (4, 32)):
        A = inputs.random_ipeps(2, D, inputs.SEED_BASE + 40 + D)
        row = {"D": D, "chi": chi}
        for prec in ("f64", "tf32x3"):
            for basis in ("hermitian", "dense"):
                hg = HOTRG(ctx, A, chi, basis=basis, precision=prec)
                hg.run(4)                      # the tensor reaches chi on every leg
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                n = 6
                infos = hg.run(n)
                torch.cuda.synchronize()
                row[f"{'z2' if basis == 'hermitian' else 'dense'}_{prec}"] = r3(n / (time.perf_counter() - t0))
                if basis == "hermitian" and prec == "tf32x3":
                    row["odd_fraction"] = [round(i["h_odd"] / (i["h_even"] + i["h_odd"]), 3) for i in infos]
                del hg
            row[f"speedup_{prec}"] = r3(row[f"z2_{prec}"] / row[f"dense_{prec}"])
        out.append(row)
    return {"unit": "steps/s", "rows": out}


def directional_line(torch, ctx):
    """Directional CTMRG (four corners and edges, no lattice symmetry) on seeded asymmetric
    tensors: directional moves/s in the Z2 and the plain basis (FP64 GEMMs and FP64 Jacobi SVD in
    both), after two warm-up sweeps, and the odd fraction of the kept states."""
    from paper_2410_11596_gb300 import inputs
    from paper_2410_11596_gb300.api import DirectionalCTMRG
    rows = []
    for D, chi in ((3, 36), (4, 64), (5, 100)):
        A = inputs.asymmetric_ipeps(2, D, inputs.SEED_BASE + 5200 + D)
        row = {"D": D, "chi": chi}
        for svd in (("jacobi", "polar") if D < 5 else ("polar",)):   # the Jacobi SVD takes ~9 s per dense move at D=5
            for basis in ("hermitian", "dense"):
                c = DirectionalCTMRG(ctx, A, chi, basis=basis, svd=svd)
                c.run(2)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                infos = c.run(1)[-4:]
                torch.cuda.synchronize()
                key = ("z2" if basis == "hermitian" else "dense") + "_" + svd
                row[f"{key}_moves_per_s"] = r3(4 / (time.perf_counter() - t0))
                if svd == "jacobi":
                    row[f"{key.split('_')[0]}_gflop_per_move"] = r3(sum(i["gemm_flops"] for i in infos) / 4 / 1e9)
                if basis == "hermitian" and svd == "jacobi":
                    row["odd_fraction"] = r3(float(np.mean([i["chi_odd"] / (i["chi_even"] + i["chi_odd"])
                                                            for i in infos])))
                del c
            row[f"speedup_{svd}"] = r3(row[f"z2_{svd}_moves_per_s"] / row[f"dense_{svd}_moves_per_s"])
        rows.append(row)
    return {"unit": "directional moves/s (one side each), moves 9-12",
            "arith": "f64 GEMM + f64 SVD (jacobi: gesvdj; polar: Xgesvdp)", "rows": rows}


def run_ours(args):
    import torch
    from paper_2410_11596_gb300 import _lib as L, build, inputs
    from paper_2410_11596_gb300.api import CTMRG, Context

    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if not os.path.exists(L.LIB_PATH):
        build.build()
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    w = inputs.WORKLOADS[WORKLOAD]
    chi = w["chi"]
    A = inputs.workload_tensor(WORKLOAD)
    h = inputs.heisenberg_bond()
    ctx = Context(local)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # ---- the headline: W warm-up moves, K timed moves ----
    c = CTMRG(ctx, A, chi, basis="hermitian", precision=args.precision, backend="own", eig=args.eig)
    c.run(args.warmup)
    # the timed moves carry no events (they would sit between the kernels of a
    # move): the counters only (launches, algorithmic flops); the tensor-core
    # kernel's own time comes from a replica of these moves below
    L.hs_profile_enable(ctx.handle, True)
    L.hs_profile_phases(ctx.handle, ())
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        t_wall = time.perf_counter()
        ms = timed_moves(torch, c, ctx, args.steps, flush)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    prof = L.hs_profile_read(ctx.handle)
    L.hs_profile_enable(ctx.handle, False)
    value, sec = replica_throughput(float(np.sum(ms)) / 1e3, args.steps, world, dev)
    ntr = min(4, args.steps)
    transient = ntr / (np.sum(ms[:ntr]) / 1e3)
    conv_timed = sum(1 for i in c.infos[args.warmup:] if i.get("flags", 0) & 2)

    # |dE| against the oracle after 50 moves, then the steady state (ten moves
    # after move 50, every warm start in place) and its phase split
    dE = None
    steady = None
    if not args.no_check:
        done = args.warmup + args.steps
        if done < 50:
            c.run(50 - done)
        ref = golden_energy(50)
        dE = abs(c.energy(h) - ref) if ref is not None else None
        nst = 10
        first = len(c.infos) + 1
        mss = timed_moves(torch, c, ctx, nst, flush)
        conv = int(sum(1 for i in c.infos[-nst:] if i.get("flags", 0) & 2))
        # the phase split from the next moves: the events between phases
        # cost time of their own, so they stay out of the timed moves above
        L.hs_profile_phases(ctx.handle, None)
        L.hs_profile_enable(ctx.handle, True)
        msp = timed_moves(torch, c, ctx, nst, flush)
        ps = L.hs_profile_read(ctx.handle)
        L.hs_profile_enable(ctx.handle, False)
        steady = {"moves": "%d-%d" % (first, first + nst - 1), "moves_per_s": r3(nst / (np.sum(mss) / 1e3)),
                  "subspace_converged": conv,
                  "phase_ms": {k: r3(v / nst) for k, v in ps["phase_ms"].items() if v > 0},
                  "phase_moves_ms": r3(float(np.mean(msp)))}
    del c

    # the same W + K moves again (deterministic: the same kernels on the same
    # data), now with events around each block GEMM launch: the roofline
    # kernel's device time and flops over the timed moves
    cr = CTMRG(ctx, A, chi, basis="hermitian", precision=args.precision, backend="own", eig=args.eig)
    cr.run(args.warmup)
    L.hs_profile_enable(ctx.handle, True)
    L.hs_profile_phases(ctx.handle, ("gemm", "gemm_tc", "gemm_tc_split"))
    ms_r = timed_moves(torch, cr, ctx, args.steps, flush)
    prof_r = L.hs_profile_read(ctx.handle)
    L.hs_profile_enable(ctx.handle, False)
    L.hs_profile_phases(ctx.handle, None)
    del cr


    # ---- {Z2, dense} x {FP64+syevd, TF32x3+syevd, FP64+subspace, TF32x3+subspace} ----
    table = None
    speedup = None
    if not args.no_table:
        table = {"z2": {}, "dense": {}}
        for basis, key in (("hermitian", "z2"), ("dense", "dense")):
            # the eigen-decomposition arms: every move costs the same, 5 timed moves after W
            table[key]["f64_syevd"] = arm(torch, ctx, A, chi, flush, basis, "f64", "f64", args.warmup, 5, 10, h)
            table[key]["tf32x3_syevd"] = arm(torch, ctx, A, chi, flush, basis, "tf32x3", "f64", args.warmup, 5, 10, h)
            # FP64 block GEMMs with the subspace eigensolver: the FP64 comparison without the library
            # eigensolver's poor scaling at n = chi q / 2 (W warm-up, K timed, |dE| at move 30)
            try:
                table[key]["f64_subspace"] = arm(torch, ctx, A, chi, flush, basis, "f64", "subspace",
                                                 args.warmup, args.steps, 30, h)
            except L.HsError as e:
                table[key]["f64_subspace"] = {"error": str(e)[:120]}
            # the subspace arm: the headline's own moves (W warm-up, K timed), |dE| at move 30
            if key == "z2":
                table[key]["tf32x3_subspace"] = {"moves_per_s": r3(value / world), "abs_dE": r3(dE),
                                                 "moves": f"{args.warmup + 1}-{args.warmup + args.steps}",
                                                 "dE_at": 50, "subspace_converged": conv_timed}
            else:
                table[key]["tf32x3_subspace"] = arm(torch, ctx, A, chi, flush, basis, "tf32x3", "subspace",
                                                    args.warmup, args.steps, 30, h)
        table["note"] = ("subspace columns: the same solver and settings in both bases; a move whose iteration "
                         "does not reach its tolerance falls back to the FP32 library eigensolver + an FP64 "
                         "Loewdin step (subspace_converged counts the moves that converged)")
        speedup = {k: r3(table["z2"][k]["moves_per_s"] / table["dense"][k]["moves_per_s"])
                   for k in table["z2"] if "moves_per_s" in table["z2"][k] and "moves_per_s" in table["dense"][k]}

    # ---- accuracy per dtype (same eigensolver): |dE| and max |d rho| after 50 moves ----
    per_dtype = None
    if not args.no_dtypes and rank == 0:
        g3 = golden_snapshot(50)
        if g3 is not None:
            rho_ref = np.array(g3["rho_re"]) + 1j * np.array(g3["rho_im"])
            per_dtype = {}
            for prec_ in ("tf32", "bf16x3", "tf32x3", "f64"):
                cp = CTMRG(ctx, A, chi, basis="hermitian", precision=prec_, backend="own", eig=args.eig)
                cp.run(50)
                rho_, t0_, t1_ = cp.rdm2(h)
                rho_ = rho_.cpu().numpy() / t0_
                per_dtype[prec_] = [r3(abs(t1_ / t0_ - g3["energy"])), r3(float(np.abs(rho_ - rho_ref).max()))]
                del cp

    # ---- complex tensors (Sec. II.C): graded path in the Hermitian basis against the plain
    # complex path (four real GEMMs per complex product, complex Hermitian eigensolver), D=5 chi=100
    cplx = None
    if not args.no_complex and rank == 0:
        w5 = inputs.WORKLOADS[5]
        A5 = inputs.workload_tensor(5)
        cplx = {"workload": "complex C4v iPEPS d=2 D=5 chi=100, Re/Im ~ N(0,1/2)"}
        for label, basis_, prec_, eig_, nw, nt in (("graded_f64_syevd", "hermitian", "f64", "f64", 5, 5),
                                                   ("dense_f64_zheevd", "dense", "f64", "f64", 5, 5),
                                                   ("graded_tf32x3_subspace", "hermitian", "tf32x3", "subspace",
                                                    args.warmup, args.steps)):
            try:
                cc = CTMRG(ctx, A5, w5["chi"], basis=basis_, precision=prec_, eig=eig_)
                cc.run(nw)
                msc = timed_moves(torch, cc, ctx, nt, flush)
                at = 10 if nw + nt <= 10 else w5["moves"]
                cc.run(at - nw - nt)
                ref5 = golden_energy(at, 5)
                cplx[label] = {"moves_per_s": r3(nt / (np.sum(msc) / 1e3)), "moves": f"{nw + 1}-{nw + nt}",
                               "abs_dE": r3(abs(cc.energy(h) - ref5) if ref5 is not None else None), "dE_at": at}
                del cc
            except L.HsError as e:
                cplx[label] = {"error": str(e)[:120]}
        try:
            cplx["speedup_f64"] = r3(cplx["graded_f64_syevd"]["moves_per_s"] / cplx["dense_f64_zheevd"]["moves_per_s"])
        except (KeyError, TypeError, ZeroDivisionError):
            pass

    # ---- many independent instances (32 real iPEPS, D uniform in 3..7, chi = 4 D^2) ----
    batched = None
    if not args.no_batched and rank == 0:
        from paper_2410_11596_gb300.api import BatchedCTMRG
        wl = inputs.batched_workload()
        bt = BatchedCTMRG([A_ for _, _, A_ in wl], [chi_ for _, chi_, _ in wl], device=local,
                          precision=args.precision, eig=args.eig)
        nwarm = max(args.warmup, 15)
        bt.run(nwarm)
        torch.cuda.synchronize()
        nb = 10
        t0 = time.perf_counter()
        bt.run(nb)
        torch.cuda.synchronize()
        tb = time.perf_counter() - t0
        lat = np.array(bt.latencies_ms[-nb:]).reshape(-1)
        t0 = time.perf_counter()
        for _ in range(nb):
            for m_ in bt.members:
                m_.move()
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        batched = {"instance_moves_per_s": r3(len(wl) * nb / tb), "one_by_one": r3(len(wl) * nb / ts),
                   "latency_ms_p50": r3(float(np.percentile(lat, 50))),
                   "latency_ms_p99": r3(float(np.percentile(lat, 99))),
                   "moves": f"{nwarm + 1}-{nwarm + nb}", "mode": bt.mode}
        bt.close()
        del bt

    hotrg = None
    if not args.no_hotrg and rank == 0:
        hotrg = hotrg_line(torch, ctx)
    directional = None
    if not args.no_directional and rank == 0:
        directional = directional_line(torch, ctx)

    # ---- end to end through the public API: host A -> device, double layer, move, corner -> host ----
    A_host = torch.from_numpy(np.ascontiguousarray(A)).pin_memory()
    ce = CTMRG(ctx, A, chi, basis="hermitian", precision=args.precision, backend="own", eig=args.eig)
    ce.run(args.warmup)
    C_host = torch.empty(ce.C_buf.numel(), dtype=torch.float64).pin_memory()
    s = ctx.stream
    e2e_ms = []
    n_c = 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        with torch.cuda.stream(s):
            ce.A.copy_(A_host, non_blocking=True)
        ce.a = L.hs_double_layer_hermitian(ctx.handle, ce.A, ce.d, ce.D, L.HS_F64, L.HS_BASIS_HERMITIAN,
                                           ce.a_buf)
        ce.move()
        n_c = ce.env.chi_even ** 2 + ce.env.chi_odd ** 2
        with torch.cuda.stream(s):
            C_host[:n_c].copy_(ce.C_buf[:n_c], non_blocking=True)
        e1.record(s)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_sec = float(np.sum(e2e_ms)) / 1e3
    h2d = A_host.numel() * 8
    d2h = n_c * 8
    del ce

    # ---- roofline of the dominant libhs kernel ----
    total_ms = float(np.sum(ms_r))
    if args.precision == "f64":
        k_ms, k_flops = prof_r["phase_ms"]["gemm"], prof_r["phase_flops"]["gemm"]
        src, key = "paper_2410_11596_gb300/csrc/k_gemm_f64.cu", "gemm_f64"
        peak, bound, kname = fp64_peak_tflops(torch, dev), "alu", "gemm_f64_nt_kernel (Z2 block GEMM, DFMA)"
        psrc = "FP64: cuBLAS DGEMM 4096^3 measured in this run"
    else:
        # the dominant kernel: the split-output instantiation of the tcgen05 GEMM (the enlarged corner
        # and edge products G2-G5, 35% of a steady-state move's kernel time in the ncu launch list);
        # all tensor-core launches (with the small subspace products) are reported beside it
        k_ms, k_flops = prof_r["phase_ms"]["gemm_tc_split"], prof_r["phase_flops"]["gemm_tc_split"]
        all_ms, all_flops = prof_r["phase_ms"]["gemm_tc"], prof_r["phase_flops"]["gemm_tc"]
        src, key = "paper_2410_11596_gb300/csrc/k_gemm_tc.cu", "gemm_tc_split_" + args.precision
        bf16, how = measured_bf16_tflops()
        passes = 1 if args.precision == "tf32" else 3
        ratio = 1.0 if args.precision == "bf16x3" else 1.1 / 2.25   # nominal dense tf32 / bf16
        peak = bf16 * ratio / passes
        bound = "tensor"
        kname = (f"gemm_tc_kernel<{args.precision}, split-output epilogue> (tcgen05, TMEM, TMA): the enlarged "
                 f"corner and edge products, output written as the next product's permuted split operand")
        psrc = (f"bf16 burst {bf16:.1f} TF/s (of {how}) x nominal "
                f"{'tf32/bf16 1.1/2.25' if ratio < 1 else '1'} / {passes} MMA passes per algorithmic product")
    tr = NCU_TRAFFIC.get(key)
    traffic = tr["bytes_per_launch"] if tr and tr["source_sha"] == source_sha(src) else None
    achieved = k_flops / (k_ms * 1e-3) / 1e12 if k_ms > 0 else None
    roof = {"bound": bound, "kernel": kname, "achieved": r3(achieved), "peak": r3(peak), "unit": "TFLOP/s",
            "frac": r3(achieved / peak) if achieved else None, "traffic": traffic, "peak_source": psrc,
            "share_of_timed_moves": r3(k_ms / total_ms),
            "timing": "events around every launch of the kernel, over a replica of the timed moves "
                      "(moves %d-%d of a second run; the headline moves carry no events)" % (
                          args.warmup + 1, args.warmup + args.steps)}
    if args.precision != "f64":
        a_all = all_flops / (all_ms * 1e-3) / 1e12 if all_ms > 0 else None
        tr_all = NCU_TRAFFIC.get("gemm_tc_" + args.precision)
        roof["all_tensor_core_launches"] = {
            "achieved": r3(a_all), "frac": r3(a_all / peak) if a_all else None,
            "share_of_timed_moves": r3(all_ms / total_ms),
            "traffic": tr_all["bytes_per_launch"] if tr_all and tr_all["source_sha"] == source_sha(src) else None}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "moves/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": ("f64" if args.precision == "f64" else f"{args.precision} GEMM (fp32 accumulate)") +
                         {"f64": " + f64 eig", "f32p": " + f32 eig, f64 projection",
                          "subspace": " + subspace eig (f32 Ritz), f64 projection",
                          "adaptive": " + subspace eig (f32 Ritz, adaptive tolerance), f64 projection"}[args.eig],
                "data": "synthetic",
                "config": {"workload": workload_name(WORKLOAD), "basis": "hermitian", "eig": EIG_LABEL[args.eig],
                           "l2": "flushed (512 MB write) between timed moves", "parallelism": f"replicas{world}",
                           "moves_timed": f"{args.warmup + 1}-{args.warmup + args.steps}"},
                "table": table, "hotrg": hotrg, "directional": directional, "complex": cplx, "batched": batched,
                "per_dtype_dE_drho": per_dtype, "steady_state": steady,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": args.steps / e2e_sec, "unit": "moves/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": prof["launches"], "wall_s_timed_region": r3(t_wall), "clocks": clk.summary(),
                # last, so that a reader of the line's tail sees them: the Z2/dense ratio at equal
                # arithmetic, the transient and steady-state rates, the energy error
                "transient_moves_per_s": r3(transient),
                "steady_moves_per_s": steady["moves_per_s"] if steady else None,
                "abs_dE_vs_oracle_50_moves": r3(dE), "speedup_vs_dense": speedup}
        emit(line)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    global WORKLOAD
    args = parse()
    WORKLOAD = args.workload
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_region:
        run_profile_region(args)
    elif args.profile_directional:
        run_profile_directional(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
