#!/usr/bin/env python
"""Benchmark of the nodal P2 Mueller solver hot path on one GB300.

One step = the whole hot path on the level-3 sphere workload (1280 curved P2
triangles, N = 10248 unknowns, eps_r = 2.25, k_a = 5):
  tangent frame + point geometry -> assembly (regular pairs in FP32 into a
  complex64 Z, touching pairs by Sauter-Schwab and the mass in FP64 into the
  near blocks, right-hand side) -> Morton block-Jacobi build (B = 256, FP64
  LU -> inverses) -> GMRES(50) with complex64 inner solves and FP64
  refinement to ||b - Zx|| <= 1e-8 ||b|| -> far field and cross sections.
value = element pairs (F^2) per second of the whole step, summed over ranks
(each rank solves its own copy: replicas, weak scaling).

Also reported (measured outside the timed region): per-kernel CUDA-event
times, the roofline of the dominant kernel, assembly-only throughput, the
plain FP64 GPU solve against the mixed one, the end-to-end number through
host buffers, and the oracle on the host cores.

--impl reference times the CPU oracle (the only reference this method has)
on bounded samples of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

WORKLOAD = "sphere_L3_eps2.25_ka5"
METRIC = "element-pairs/s assembled; GMRES solve s, mixed vs FP64 GPU, at rel err <=1e-6"
UNIT = "element-pairs/s"

SMS = 152
SM_MAX_HZ = 2.070e9
# peaks of the plain ALU pipes from unit counts and the maximum SM clock:
# FP64 2 DFMA/clk/SM (1.26 TFLOP/s, the nominal 1.25), FP32 128 FFMA/clk/SM
PEAK_FP64 = SMS * 2 * 2 * SM_MAX_HZ
PEAK_FP32 = SMS * 128 * 2 * SM_MAX_HZ


def measured_hbm_gbs() -> tuple:
    """(GB/s, source): the measured copy bandwidth of the GB300s from
    MEASURED_PEAKS.json, else the recipe's fallback figure."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback"


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-extras", action="store_true", help="skip the untimed extra measurements")
    # one untimed invocation of part of the path on a sphere, for profiler
    # captures (ncu -k <kernel> ... python bench.py --profile-case assemble)
    ap.add_argument("--profile-case", default=None,
                    choices=["assemble", "assemble64", "precond", "solve", "mrhs", "farfield",
                             "shapegrad"])
    ap.add_argument("--level", type=int, default=2, help="--profile-case: icosphere level")
    ap.add_argument("--rhs", type=int, default=16,
                    help="--profile-case mrhs, farfield: right-hand sides")
    ap.add_argument("--block", type=int, default=256, help="--profile-case: cluster size B")
    return ap.parse_args(argv)


# --------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (sm clock, throttle reasons)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------ flop models
# DRAM bytes (read + written) per touching pair of the touching kernel's
# launches, from its ncu capture on the level-2 sphere (4100 touching pairs);
# None while the kernel has changed since that capture.
TOUCH_DRAM_PER_PAIR = 59.044e6 / 4100


def touching_points(n_tri: int, n_touch: int, ns: int) -> float:
    """Sauter-Schwab points of all touching pairs: 6, 5 and 2 regions of ns^4
    points for the coincident, common-edge and common-vertex pairs."""
    n_vert = n_touch - 4 * n_tri
    return float(ns ** 4) * (6 * n_tri + 5 * 3 * n_tri + 2 * n_vert)


def touching_flops_algorithmic(n_tri: int, n_touch: int, ns: int, q: int) -> float:
    """The algorithmic count of the touching pairs: per Sauter-Schwab point
    about 60 flops of singular kernel and 8 real accumulators x 36 node pairs
    (576), with the point geometry precomputed; per touching pair the
    remainder kappa - kappa^s on the Q x Q rule (Q^2 540 + Q 1728 flops, the
    regular-pair count)."""
    return touching_points(n_tri, n_touch, ns) * (60.0 + 576.0) + \
        n_touch * (q * q * 540.0 + q * 1728.0)


def touching_flops(n_tri: int, n_touch: int, ns: int, q: int) -> float:
    """FP64 flops of one touching_kernel launch (all touching pairs).

    The Sauter-Schwab points are processed in groups of ns that share one
    side.  A point geometry (P2 map, derivatives and interpolated nodal frame
    from monomial coefficients, normal, one Gram-Schmidt step for t1, t2 from
    n x t1 and the sign of u2) costs 189 flops.  Per point: R and its
    direction 12, the weight product 2, the 11 frame dot products and 8
    singular kernels 85, the 6 shape weights 6 and the 48 multiply-adds 96,
    and the eta3-affine map with the weight 5 (206; 202 where the geometry
    comes from the tables and only the weight is mapped).  Per group the
    6 x 48 contraction costs 576.  Coincident and
    common-edge groups evaluate 1 + ns geometries; common-vertex pairs
    (ns <= 5) evaluate the 2 (ns^2 + ns^3) distinct ones once.  Groups whose
    shared side depends on (a, b) only are folded by sets of ns before the
    contraction.  Per pair,
    the remainder kappa - kappa^s on the Q x Q rule (~900 flops per point
    pair) and its 6 x 6 x 12 contraction (2 * 432 * Q * 2)."""
    n_coinc = n_tri
    n_edge = 3 * n_tri
    n_vert = n_touch - n_coinc - n_edge
    g_ce = (6 * n_coinc + 5 * n_edge) * ns ** 3
    g_v = 2 * n_vert * ns ** 3
    tab = ns <= 5
    geo = g_ce * (1 + ns) + (n_vert * 2 * (ns ** 2 + ns ** 3) if tab else g_v * (1 + ns))
    per_point = g_ce * ns * 206.0 + g_v * ns * (202.0 if tab else 206.0)
    per_pair = q * q * 900 + 2 * 432 * q * 2
    # contraction 576 per group; where the shared side depends on (a, b)
    # only (common-edge regions 1 and 3, both common-vertex regions) the ns
    # groups of a set are folded first (48 (ns - 1) adds) and contracted once
    sets_shared = (2 * n_edge + 2 * n_vert) * ns ** 2
    g_plain = (6 * n_coinc + 3 * n_edge) * ns ** 3
    contraction = g_plain * 576.0 + sets_shared * (576.0 + 48.0 * (ns - 1))
    return geo * 189.0 + per_point + contraction + n_touch * per_pair


def regular_flops(n_tri: int, n_touch: int, q: int) -> float:
    """FP32 flops of one regular_kernel launch: per non-touching element pair,
    Q*Q point pairs of the fused 12-component kernel (~300 flops: R, the
    complex exponentials and the four radial scalars, 17 frame dot products,
    12 complex kernel values) and the two contractions (2 * 432 * Q * 2)."""
    pairs = n_tri * n_tri - n_touch
    return pairs * (q * q * 300.0 + 2 * 432 * q * 2)


# ---------------------------------------------------------------- ranks
def job_timing(ms_local: float, units_per_rank: float, world: int, device=None):
    """Whole-job timing of N replicas (weak scaling, one process per GPU, no
    collective on the data path): the step time is the slowest rank's, the
    value the units all ranks processed in that time.  Returns
    (ms_max, units per second)."""
    ms_max = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([ms_local], dtype=torch.float64,
                         device=device if device is not None else "cpu")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_max = float(t.item())
    return ms_max, units_per_rank * world / (ms_max / 1e3)


# ---------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2604_21181_gb300 as mu

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    xyz, tri6, inc, w = workloads.workload(args.workload)
    p = mu.Params.from_workload(w)
    F = tri6.shape[0]
    pairs = float(F) * F
    block = int(w["block"])
    r = inc.shape[0]
    opts = mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=int(w["restart"]), tol=float(w["tol"]),
                         inner_tol=1e-5, use_precond=1)

    mesh = mu.Mesh(xyz, tri6)
    N = mesh.N
    info = mesh.info()
    Z = torch.empty((N, N), dtype=torch.complex64, device=dev)
    near = torch.empty(mesh.near_bytes() // 16, dtype=torch.complex128, device=dev)
    B = torch.empty((r, N), dtype=torch.complex128, device=dev)
    X = torch.zeros((r, N), dtype=torch.complex128, device=dev)
    op = mu.Operator(mesh, Z, near, mu.MUELLER_C64_NEAR64)
    Pbuf = None

    def step():
        nonlocal Pbuf
        mesh.tangent_frame(p.frame_rule, out=False)
        mu.assemble(mesh, p, mu.MUELLER_C64_NEAR64, inc=inc, Z=Z, near=near, B=B)
        Pbuf = mu.precond_build(op, block)
        _, sinfo = mu.solve(op, B, opts, X=X, work=work)
        _, xs = mu.far_field(mesh, p, X, inc)
        return sinfo, xs

    mesh.tangent_frame(p.frame_rule, out=False)
    mu.assemble(mesh, p, mu.MUELLER_C64_NEAR64, inc=inc, Z=Z, near=near, B=B)
    mu.precond_build(op, block)
    work = torch.empty(mu.solve_workspace_bytes(op, r, opts), dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = mu.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    infos = []
    for _ in range(args.steps):
        infos.append(step())
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    launches = (mu.launch_count() - l0) // max(1, args.steps)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max, value = job_timing(ms, pairs, world, dev)
    sinfo, xs = infos[-1]

    extras = {}
    roofline = None
    e2e = None
    cpu = None
    if rank == 0 and not args.no_extras:
        # ---- per-kernel CUDA-event times of one step (profiling on)
        mu.profile_reset()
        mu.profile_enable(True)
        step()
        mu.profile_enable(False)
        prof = mu.profile_report()
        kernels = sorted(((v[0], k, v[1]) for k, v in prof.items()), reverse=True)
        tot = sum(v[0] for v in kernels)
        extras["kernels_ms"] = {k: {"ms": round(ms_, 3), "launches": n, "share": round(ms_ / tot, 4)}
                                for ms_, k, n in kernels[:12]}
        top_ms, top_name, top_n = kernels[0]
        q, ns = int(w["q_regular"]), int(w["ssq_order"])
        if top_name.startswith("touching_kernel"):
            # all touching pairs, in top_n launches (coincident and common-edge
            # pairs, then common-vertex pairs): algorithmic flops of all of
            # them over their summed CUDA-event time; beside it the flops the
            # kernel executes by its own model
            fl = touching_flops_algorithmic(F, info["n_touching"], ns, q)
            ach = fl / (top_ms / 1e3) / 1e12
            fx = touching_flops(F, info["n_touching"], ns, q)
            ax = fx / (top_ms / 1e3) / 1e12
            # DRAM bytes of the step's launches, scaled per touching pair from
            # the ncu capture of this kernel on the level-2 sphere
            traffic = (int(round(TOUCH_DRAM_PER_PAIR * info["n_touching"]))
                       if TOUCH_DRAM_PER_PAIR else None)
            roofline = {"kernel": top_name, "launches": top_n, "bound": "alu", "pipe": "fp64",
                        "achieved": round(ach, 4),
                        "peak": round(PEAK_FP64 / 1e12, 4), "unit": "TFLOP/s",
                        "frac": round(ach / (PEAK_FP64 / 1e12), 4), "traffic": traffic,
                        "algorithmic_gflop": round(fl / 1e9, 3),
                        "definition": "Sauter-Schwab points x (60 + 576) flops + touching pairs "
                                      "x (Q^2 540 + Q 1728) remainder flops",
                        "executed_model": {"gflop": round(fx / 1e9, 3), "achieved": round(ax, 4),
                                           "frac": round(ax / (PEAK_FP64 / 1e12), 4)},
                        "peak_source": "152 SMs x 2 DFMA/clk x 2.07 GHz (unit counts, max clock)"}
        elif top_name.startswith("regular_kernel"):
            fl = regular_flops(F, info["n_touching"], q)
            ach = fl / (top_ms / top_n / 1e3) / 1e12
            roofline = {"kernel": top_name, "bound": "alu", "pipe": "fp32", "achieved": round(ach, 3),
                        "peak": round(PEAK_FP32 / 1e12, 3), "unit": "TFLOP/s",
                        "frac": round(ach / (PEAK_FP32 / 1e12), 4), "traffic": None,
                        "peak_source": "152 SMs x 128 FFMA/clk x 2.07 GHz"}
        else:
            roofline = {"kernel": top_name, "bound": None, "note": "no model for this kernel"}
        # ---- assembly-only throughput, mixed and FP64
        def timed(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        t_asm_mixed = timed(lambda: mu.assemble(mesh, p, mu.MUELLER_C64_NEAR64, inc=inc, Z=Z,
                                                near=near, B=B))
        extras["assembly_mixed_ms"] = round(t_asm_mixed, 3)
        extras["assembly_mixed_pairs_per_s"] = pairs / (t_asm_mixed / 1e3)
        # mixed solve alone (operator and preconditioner ready)
        mu.precond_build(op, block)
        t_solve_mixed = timed(lambda: mu.solve(op, B, opts, X=X, work=work), reps=2)
        _, sinfo = mu.solve(op, B, opts, X=X, work=work)
        Xmix = X.clone()
        # FP64 path: complex128 Z, FP64 GMRES with the same preconditioner size
        del Pbuf
        Z64 = torch.empty((N, N), dtype=torch.complex128, device=dev)
        t_asm64 = timed(lambda: mu.assemble(mesh, p, mu.MUELLER_C128, inc=inc, Z=Z64, B=B), reps=1)
        op64 = mu.Operator(mesh, Z64, dtype=mu.MUELLER_C128)
        mu.precond_build(op64, block)
        o64 = mu.SolverOpts(mode=mu.SOLVE_GMRES, restart=int(w["restart"]), tol=float(w["tol"]),
                            use_precond=1)
        X64 = torch.zeros_like(X)
        w64 = torch.empty(mu.solve_workspace_bytes(op64, r, o64), dtype=torch.uint8, device=dev)
        t_solve64 = timed(lambda: mu.solve(op64, B, o64, X=X64, work=w64), reps=2)
        _, info64 = mu.solve(op64, B, o64, X=X64, work=w64)
        rel = (torch.linalg.norm(Xmix - X64) / torch.linalg.norm(X64)).item()
        extras["assembly_fp64_ms"] = round(t_asm64, 3)
        extras["assembly_fp64_pairs_per_s"] = pairs / (t_asm64 / 1e3)
        extras["solve"] = {
            "mixed_s": round(t_solve_mixed / 1e3, 5), "fp64_s": round(t_solve64 / 1e3, 5),
            "speedup": round(t_solve64 / t_solve_mixed, 3),
            "mixed_iters": sinfo["iters"], "mixed_refinements": sinfo["refinements"],
            "mixed_relres": sinfo["relres"], "fp64_iters": info64["iters"],
            "fp64_relres": info64["relres"], "rel_err_mixed_vs_fp64": rel,
        }
        del Z64, op64, w64
        extras["cross_sections"] = {"C_ext": float(xs[0, 0]), "C_sca": float(xs[0, 1]),
                                    "C_abs": float(xs[0, 2])}
        # ---- end to end through host buffers: mesh from host arrays, result
        # (cross sections) back to the host
        def e2e_step():
            m2 = mu.Mesh(xyz, tri6)
            m2.tangent_frame(p.frame_rule, out=False)
            mu.assemble(m2, p, mu.MUELLER_C64_NEAR64, inc=inc, Z=Z, near=near, B=B)
            o2 = mu.Operator(m2, Z, near, mu.MUELLER_C64_NEAR64)
            mu.precond_build(o2, block)
            mu.solve(o2, B, opts, X=X, work=work)
            _, xs2 = mu.far_field(m2, p, X, inc)
            m2.free()
            return xs2

        e2e_step()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            e2e_step()
        b.record()
        torch.cuda.synchronize()
        ms_e2e = a.elapsed_time(b) / args.steps
        e2e = {"value": pairs / (ms_e2e / 1e3), "unit": UNIT, "ms_per_step": round(ms_e2e, 3),
               "h2d_bytes_per_step": int(xyz.nbytes + tri6.nbytes + inc.nbytes),
               "d2h_bytes_per_step": int(r * 3 * 8)}
        extras["level4_16rhs"] = level4_16rhs(mu, torch, dev)
        extras["multibody64"] = multibody64(mu, torch, dev)
        extras["lspr_sweep"] = lspr_sweep(mu, torch, dev)
        extras["gradients_L3"] = gradients_l3(mu, torch, dev)
        cpu = cpu_baseline(args.workload)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_tri": F, "n_dof": N, "element_pairs": int(pairs),
                       "eps_r": list(w["eps_r"]), "ka": w["ka"], "q_regular": w["q_regular"],
                       "ssq_order": w["ssq_order"], "block": block, "restart": w["restart"],
                       "tol": w["tol"], "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (complex64 Z = %.2f GB)" % (N * N * 8 / 1e9)},
            "clocks": clk, "gpu_launches": int(launches),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "solve_info": {"iters": sinfo["iters"], "refinements": sinfo["refinements"],
                           "relres": sinfo["relres"]},
        }
        line.update(extras)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def level4_16rhs(mu, torch, dev):
    """The level-4 plasmonic sphere (N = 40968, complex64 Z of 13.4 GB) with
    16 incidences: mixed assembly, block-Jacobi build (B = 512), the
    lockstep GMRES-IR solve of all 16 right-hand sides, and the tensor-core
    product alone (achieved HBM bandwidth of the complex64 Z read)."""
    xyz, tri6, inc, w = workloads.workload("sphere_L4_eps-10+1i_ka10")
    p = mu.Params.from_workload(w)
    F = tri6.shape[0]
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(p.frame_rule, out=False)

    def ev_time(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            out = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, out

    Z = torch.empty((m.N, m.N), dtype=torch.complex64, device=dev)
    near = torch.empty(m.near_bytes() // 16, dtype=torch.complex128, device=dev)
    B = torch.empty((inc.shape[0], m.N), dtype=torch.complex128, device=dev)
    t_asm, _ = ev_time(lambda: mu.assemble(m, p, mu.MUELLER_C64_NEAR64, inc=inc, Z=Z, near=near, B=B))
    op = mu.Operator(m, Z, near, mu.MUELLER_C64_NEAR64)
    t_pre, _ = ev_time(lambda: mu.precond_build(op, int(w["block"])))
    opts = mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=50, tol=1e-8)
    X = torch.zeros_like(B)
    t_solve, (X, info) = ev_time(lambda: mu.solve(op, B, opts, X=X))
    X32 = X.to(torch.complex64)
    t_mm, _ = ev_time(lambda: mu.matvec_mrhs(op, X32), reps=5)
    _, xs = mu.far_field(m, p, X, inc)
    # algorithmic bytes: the three-block form (Z00, Z01, Z10: Z11 = -Z00 is
    # not read again) for r <= 16, else all of Z, plus X and Y
    r = int(inc.shape[0])
    zbytes = (0.75 if r <= 16 else 1.0) * m.N * m.N * 8
    gbs = (zbytes + 2 * r * m.N * 8) / (t_mm / 1e3) / 1e9
    return {"n_dof": m.N, "rhs": int(inc.shape[0]), "assembly_ms": round(t_asm, 2),
            "assembly_pairs_per_s": F * F / (t_asm / 1e3), "precond_ms": round(t_pre, 2),
            "solve_s": round(t_solve / 1e3, 4), "iters_lockstep": info["iters"] // inc.shape[0],
            "refinements": info["refinements"], "relres": info["relres"],
            "mrhs_product_ms": round(t_mm, 3), "mrhs_product_hbm_gbs": round(gbs, 1),
            "mrhs_product_hbm_frac": round(gbs / measured_hbm_gbs()[0], 3),
            "mrhs_product_bytes": "complex64 Z read once per product (three quarters of it "
                                  "when Z11 = -Z00 and r <= 16) + X, Y",
            "C_ext_mean": float(xs[:, 0].mean())}


def multibody64(mu, torch, dev):
    """The batched uneven workload: 64 seeded prolate and oblate spheroids
    (levels 1-3, 80-1280 P2 triangles, lossy eps_r, k_a in [0.5, 5]), each lit
    by 32 Fibonacci incidences x 2 polarisations.  Mixed assembly of all
    bodies in one launch per kernel (beside a loop of single-body
    assemblies), then per body the block-Jacobi build, the lockstep GMRES-IR
    solve of its 64 right-hand sides and the cross sections."""
    import time as _t

    spec = workloads.multibody_spec()
    inc = workloads.fibonacci_plane_waves(32)
    meshes, params = [], []
    for b in spec:
        xyz, tri6 = workloads.multibody_mesh(b)
        m = mu.Mesh(xyz, tri6)
        m.tangent_frame(mu.FRAME_PAPER, out=False)
        meshes.append(m)
        params.append(mu.Params(ka=b["ka"], eps_r=b["eps_r"], mu_r=b["mu_r"], q_regular=6,
                                ssq_order=5, frame_rule=mu.FRAME_PAPER))
    pairs = float(sum(m.nt * m.nt for m in meshes))
    incs = [inc] * len(meshes)

    def ev(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            out = fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps, out

    t_batch, out = ev(lambda: mu.assemble_batch(meshes, params, mu.MUELLER_C64_NEAR64, incs=incs))
    t_loop, _ = ev(lambda: [mu.assemble(m, p, mu.MUELLER_C64_NEAR64, inc=inc, Z=Z, near=nr, B=B)
                            for m, p, (Z, nr, B) in zip(meshes, params, out)])
    opts = mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=50, tol=1e-8)
    ops = [mu.Operator(m, Z, nr, mu.MUELLER_C64_NEAR64) for m, (Z, nr, B) in zip(meshes, out)]
    blocks = [min(256, m.N // 2) for m in meshes]
    # the block-Jacobi builds of all bodies: one batched LU, and per body
    t_pre_loop, _ = ev(lambda: [mu.precond_build(op, b) for op, b in zip(ops, blocks)], reps=1)
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    mu.precond_build_batch(ops, blocks)
    torch.cuda.synchronize()
    t_pre = _t.perf_counter() - t0
    t_sol, t_far = 0.0, 0.0
    worst, iters, bal, by_level = 0.0, 0, {}, {}
    for m, p, op, (Z, nr, B) in zip(meshes, params, ops, out):
        key = "L%d" % {80: 1, 320: 2, 1280: 3}.get(m.nt, 0)
        tb = _t.perf_counter()
        X, info = mu.solve(op, B, opts)
        torch.cuda.synchronize()
        tc = _t.perf_counter()
        t_sol += tc - tb
        worst = max(worst, info["relres"])
        iters += info["iters"] // inc.shape[0]
        _, xs = mu.far_field(m, p, X, inc)
        td = _t.perf_counter()
        t_far += td - tc
        lv = by_level.setdefault(key, {"bodies": 0, "solve_s": 0.0, "far_field_s": 0.0})
        lv["bodies"] += 1
        lv["solve_s"] += tc - tb
        lv["far_field_s"] += td - tc
        # |C_ext - C_sca - C_abs| / C_ext: the discretisation error of the body's mesh
        e = float(np.max(np.abs(xs[:, 0] - xs[:, 1] - xs[:, 2]) / np.abs(xs[:, 0])))
        bal[key] = max(bal.get(key, 0.0), e)
    t_all = _t.perf_counter() - t0
    for lv in by_level.values():
        lv["solve_s"] = round(lv["solve_s"], 3)
        lv["far_field_s"] = round(lv["far_field_s"], 3)
    for m in meshes:
        m.free()
    return {"bodies": len(meshes), "rhs_per_body": int(inc.shape[0]),
            "triangles": [int(min(m.nt for m in meshes)), int(max(m.nt for m in meshes))],
            "element_pairs": pairs, "assembly_batched_ms": round(t_batch, 2),
            "assembly_batched_pairs_per_s": pairs / (t_batch / 1e3),
            "assembly_loop_ms": round(t_loop, 2),
            "assembly_loop_pairs_per_s": pairs / (t_loop / 1e3),
            "precond_batched_s": round(t_pre, 3),
            "precond_loop_s": round(t_pre_loop / 1e3, 3), "solve_total_s": round(t_sol, 3),
            "far_field_total_s": round(t_far, 3), "by_level": by_level,
            "solve_and_far_field_wall_s": round(t_all, 3), "lockstep_iters_total": iters,
            "worst_relres": worst, "worst_energy_balance_by_level": bal}


def gradients_l3(mu, torch, dev):
    """Adjoint gradients on the level-3 spheroid of axis ratio 1.5 (eps_r =
    3 + 0.2i, mu_r = 1, k_a = 3, incidence +z, x polarised, the paper's frame
    rule): the FP64 forward state (assembly, block-Jacobi, GMRES to 1e-12,
    far field); then (a) the full gradients of (C_ext, C_sca, C_abs) by one
    adjoint solve with three right-hand sides: the 3 x 4 material Jacobian
    and the 3 x 2562 x 3 node-coordinate gradient, per stage; (b) one
    reverse-mode product w^T (gradients) as an autograd backward makes it
    (one adjoint solve, one pass of each derivative kernel); (c) the
    tangent-linear material Jacobian for comparison.  Wall times with the
    device synchronised, after a warm-up of every path."""
    import time as _t

    xyz, tri6 = workloads.spheroid_p2(3, 1.0, 1.5)
    p = mu.Params(ka=3.0, eps_r=(3.0, 0.2), mu_r=(1.0, 0.0), q_regular=6, ssq_order=5, frame_rule=0)
    inc = workloads.plane_wave((0.0, 0.0, 1.0), (1.0, 0.0, 0.0))

    def fwd():
        m = mu.Mesh(xyz, tri6)
        m.tangent_frame(0, out=False)
        xs, state = mu.grad.forward_state(m, p, inc)
        return m, xs, state

    # warm-up (tuning, rules, first launches of the derivative kernels, workspace)
    m, _, state = fwd()
    mu.grad.adjoint_gradients(state)
    mu.grad.vjp(state, np.ones(3))
    mu.grad.material_jacobian(state)
    m.free()
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    m, xs, state = fwd()
    torch.cuda.synchronize()
    t1 = _t.perf_counter()
    stages = {}
    J, G = mu.grad.adjoint_gradients(state, timings=stages)
    t2 = _t.perf_counter()
    mu.grad.vjp(state, np.array([1.0, 0.5, 0.25]))
    torch.cuda.synchronize()
    t3 = _t.perf_counter()
    Jt = mu.grad.material_jacobian(state)
    torch.cuda.synchronize()
    t4 = _t.perf_counter()
    m.free()
    return {"n_dof": int(m.N), "n_nodes": int(len(xyz)), "forward_ms": round((t1 - t0) * 1e3, 1),
            "adjoint_gradients_ms": round((t2 - t1) * 1e3, 1), "adjoint_stages_ms": stages,
            "vjp_ms": round((t3 - t2) * 1e3, 1),
            "tangent_jacobian_ms": round((t4 - t3) * 1e3, 1),
            "jacobian_adjoint_vs_tangent": float(np.abs(J - Jt).max() / np.abs(Jt).max()),
            "cross_sections": [float(v) for v in xs],
            "jacobian_rows_ext_sca_abs_cols_re_eps_im_eps_re_mu_im_mu": J.round(6).tolist(),
            "coordinate_gradient_max_abs": [float(np.abs(G[o]).max()) for o in range(3)],
            "translation_residual": [float(np.abs(G[o].sum(axis=0)).max() / np.abs(G[o]).max())
                                     for o in range(3)]}


def lspr_sweep(mu, torch, dev):
    """Wavelength sweep of a silver prolate spheroid (semi-axes 15 : 15 : 45
    nm, level-3 P2 mesh standing in for the paper's 3072-element mesh), lit
    across its major axis with E along it, permittivity interpolated from the
    paper's silver table: 350-800 nm, 1 nm steps over 475-525 nm and 5 nm
    elsewhere.  Chunks of 16 wavelengths are assembled by one batched call
    each; every wavelength is then solved (mixed GMRES-IR to 1e-8)."""
    import time as _t

    lam = np.unique(np.concatenate([np.arange(350.0, 476.0, 5.0), np.arange(475.0, 526.0, 1.0),
                                    np.arange(530.0, 801.0, 5.0)]))
    unit = 15.0
    xyz, tri6 = workloads.spheroid_p2(3, 1.0, 3.0)
    inc = workloads.plane_wave((1.0, 0.0, 0.0), (0.0, 0.0, 1.0))
    m = mu.Mesh(xyz, tri6)
    m.tangent_frame(mu.FRAME_PAPER, out=False)
    ka = 2.0 * np.pi * unit / lam
    eps = workloads.eps_silver(lam)
    mu.sweep.spectrum(m, ka[:2], eps[:2], inc, chunk=2)  # warm-up
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    res = mu.sweep.spectrum(m, ka, eps, inc, chunk=16)
    torch.cuda.synchronize()
    t = _t.perf_counter() - t0
    xs = res["xs"][:, 0, :] * unit * unit  # nm^2
    k = int(np.argmax(xs[:, 0]))
    bal = np.abs(xs[:, 0] - xs[:, 1] - xs[:, 2]) / np.abs(xs[:, 0])
    m.free()
    return {"n_dof": int(4 * xyz.shape[0]), "wavelengths": int(lam.size), "total_s": round(t, 3),
            "ms_per_wavelength": round(1e3 * t / lam.size, 2),
            "peak_nm": float(lam[k]), "C_ext_peak_nm2": float(xs[k, 0]),
            "C_sca_peak_nm2": float(xs[k, 1]), "C_abs_peak_nm2": float(xs[k, 2]),
            "iters_at_peak": int(res["iters"][k]), "worst_relres": res["worst_relres"],
            "worst_energy_balance": float(bal.max())}


# ------------------------------------------------------------ CPU oracle
def oracle_sample(workload: str, n_test_elems: int):
    """Oracle assembly of the rows of the first n_test_elems Morton elements'
    nodes.  Returns (element pairs processed, seconds, threads)."""
    import oracle

    xyz, tri6, inc, w = workloads.workload(workload)
    om = oracle.Mesh(xyz, tri6)
    pw = dict(ka=w["ka"], eps_r=w["eps_r"], mu_r=w["mu_r"], q_regular=w["q_regular"],
              ssq_order=w["ssq_order"])
    nodes = np.unique(om.tri6[:n_test_elems].ravel())
    sel = np.zeros(om.nn, bool)
    sel[nodes] = True
    n_ex = int(np.any(sel[om.tri6], axis=1).sum())  # test elements the oracle visits
    t0 = time.perf_counter()
    om.assemble(pw, rows=nodes)
    dt = time.perf_counter() - t0
    return n_ex * om.nt, dt, oracle.num_threads()


def oracle_step(workload: str) -> dict:
    """The oracle's whole step on the workload, the same scope as one GPU
    step: mesh (Morton, frame), FP64 assembly, right-hand side, Morton
    block-Jacobi build + GMRES(m) to the workload's tolerance (complex128
    throughout), far field and cross sections.  Seconds per part."""
    import oracle

    xyz, tri6, inc, w = workloads.workload(workload)
    pw = dict(ka=w["ka"], eps_r=w["eps_r"], mu_r=w["mu_r"], q_regular=w["q_regular"],
              ssq_order=w["ssq_order"])
    t = [time.perf_counter()]
    om = oracle.Mesh(xyz, tri6)
    om.frame()
    t.append(time.perf_counter())
    Z = om.assemble(pw)
    t.append(time.perf_counter())
    B = om.rhs(pw, inc)
    X = np.zeros_like(B)
    for s in range(B.shape[0]):
        X[s], _ = oracle.gmres(Z, B[s], block=int(w["block"]), restart=int(w["restart"]),
                               tol=float(w["tol"]))
    t.append(time.perf_counter())
    om.far_field(pw, X, inc)
    t.append(time.perf_counter())
    return {"mesh_s": t[1] - t[0], "assembly_s": t[2] - t[1], "solve_s": t[3] - t[2],
            "far_field_s": t[4] - t[3], "total_s": t[4] - t[0], "threads": oracle.num_threads(),
            "element_pairs": float(tri6.shape[0]) ** 2}


def oracle_single_thread(workload: str, n_test_elems: int):
    """oracle_sample in a child process limited to one OpenMP thread (the
    plain-loop baseline).  Returns (pairs, seconds, threads) or None."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(%r, %d)))" % (ROOT, workload, n_test_elems))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                           timeout=300)
        return tuple(json.loads(r.stdout.strip().splitlines()[-1]))
    except Exception:
        return None


def cpu_baseline(workload: str):
    """The oracle timed on the host cores: its whole step once (value, in
    the metric's unit), its assembly alone, and an assembly sample on one
    thread."""
    st = oracle_step(workload)
    F = int(round(st["element_pairs"] ** 0.5))
    n1 = max(1, F // 64)
    one = oracle_single_thread(workload, n1)
    out = {"value": st["element_pairs"] / st["total_s"], "unit": UNIT, "cores": st["threads"],
           "kind": "oracle",
           "sample": (f"one whole oracle step of the workload (mesh + frame, FP64 assembly of all "
                      f"{F * F} element pairs, RHS, block-Jacobi + GMRES to tol, far field): "
                      f"{st['total_s']:.2f} s on {st['threads']} threads"),
           "parts_s": {k: round(v, 3) for k, v in st.items() if k.endswith("_s")},
           "assembly_only_pairs_per_s": st["element_pairs"] / st["assembly_s"]}
    if one is not None:
        out["single_thread"] = {"value": one[0] / one[1], "unit": UNIT, "cores": 1,
                                "sample": f"FP64 assembly of the Z rows of the nodes of {n1} of "
                                          f"{F} test elements ({one[0]} element pairs), "
                                          f"{one[1]:.2f} s, OMP_NUM_THREADS=1"}
    return out


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    xyz, tri6, inc, w = workloads.workload(args.workload)
    F = tri6.shape[0]
    # warm-up: page the oracle in on a small assembly sample
    for _ in range(args.warmup):
        oracle_sample(args.workload, max(1, F // 256))
    steps = [oracle_step(args.workload) for _ in range(args.steps)]
    tot_s = sum(s["total_s"] for s in steps)
    tot_pairs = sum(s["element_pairs"] for s in steps)
    th = steps[-1]["threads"]
    value = tot_pairs / tot_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * tot_s / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "n_tri": F, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": th, "kind": "oracle",
                             "sample": "per step: the oracle's whole step (mesh + frame, FP64 "
                                       "assembly of all element pairs, RHS, block-Jacobi + "
                                       "GMRES to tol, far field), the scope of one GPU step",
                             "assembly_s_per_step": round(sum(s["assembly_s"] for s in steps)
                                                          / args.steps, 3)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def profile_case(args):
    """One untimed run of part of the hot path on the level-L sphere (eps_r =
    2.25, k_a = 5, Q = 6, Ns = 5), for profiler captures, then exit:
      assemble    tangent frame + mixed assembly (regular pairs FP32)
      assemble64  tangent frame + FP64 assembly
      precond     mixed assembly + block-Jacobi build (FP64 LU, FP32 inverse)
      solve       mixed assembly + block-Jacobi + one GMRES-IR solve
      mrhs        mixed assembly + one tensor-core product of --rhs vectors
      farfield    mixed assembly + block-Jacobi + GMRES-IR solve of --rhs
                  Fibonacci incidences + their far fields (48 x 96 sphere rule)
      shapegrad   the level-L spheroid of axis ratio 1.5 (eps_r = 3 + 0.2i,
                  k_a = 3): FP64 forward state and one reverse-mode product
                  of the node-coordinate gradient (adjoint solve, VJP kernels)
    """
    import torch

    import paper_2604_21181_gb300 as mu

    if args.profile_case == "shapegrad":
        xyz, tri6 = workloads.spheroid_p2(args.level, 1.0, 1.5)
        p = mu.Params(ka=3.0, eps_r=(3.0, 0.2), q_regular=6, ssq_order=5, frame_rule=0)
        mesh = mu.Mesh(xyz, tri6)
        mesh.tangent_frame(0, out=False)
        _, state = mu.grad.forward_state(mesh, p, workloads.plane_wave())
        mu.grad.vjp(state, np.ones(3), material=False)
        torch.cuda.synchronize()
        print("ok", args.profile_case, "level", args.level, "N", mesh.N)
        return
    xyz, tri6 = workloads.icosphere_p2(args.level)
    p = mu.Params(ka=5.0, eps_r=(2.25, 0.0), q_regular=6, ssq_order=5)
    mesh = mu.Mesh(xyz, tri6)
    mesh.tangent_frame(p.frame_rule, out=False)
    inc = workloads.plane_wave()
    if args.profile_case == "farfield":
        inc = workloads.fibonacci_plane_waves((args.rhs + 1) // 2)[:args.rhs]
    dtype = mu.MUELLER_C128 if args.profile_case == "assemble64" else mu.MUELLER_C64_NEAR64
    Z, near, B = mu.assemble(mesh, p, dtype, inc=inc)
    op = mu.Operator(mesh, Z, near, dtype)
    if args.profile_case in ("precond", "solve", "farfield"):
        mu.precond_build(op, args.block)
    if args.profile_case in ("solve", "farfield"):
        X, _ = mu.solve(op, B, mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=50, tol=1e-8))
    if args.profile_case == "farfield":
        mu.far_field(mesh, p, X, inc)
    if args.profile_case == "mrhs":
        g = torch.Generator().manual_seed(1)
        X = torch.randn((args.rhs, mesh.N), dtype=torch.complex64, generator=g).cuda()
        mu.matvec_mrhs(op, X)
    torch.cuda.synchronize()
    print("ok", args.profile_case, "level", args.level, "N", mesh.N)


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
