"""One assembly (or one solve) of a sphere workload, for profiler captures.

    python -m paper_2604_21181_gb300.profile_case --level 2 --what assemble

Runs the mesh load, the tangent frame and one mixed-precision assembly of the
level-L sphere with eps_r = 2.25, k_a = 5; with --what solve also the
block-Jacobi build and one GMRES-IR solve, with --what mrhs one tensor-core
product with --rhs random right-hand sides; then exits.
"""

from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    import paper_2604_21181_gb300 as mu
    import workloads

    ap = argparse.ArgumentParser()
    ap.add_argument("--level", type=int, default=2)
    ap.add_argument("--what", default="assemble", choices=["assemble", "solve", "mrhs"])
    ap.add_argument("--rhs", type=int, default=16)
    ap.add_argument("--ka", type=float, default=5.0)
    ap.add_argument("--eps", type=float, nargs=2, default=(2.25, 0.0))
    ap.add_argument("--block", type=int, default=256)
    a = ap.parse_args()
    xyz, tri6 = workloads.icosphere_p2(a.level)
    p = mu.Params(ka=a.ka, eps_r=tuple(a.eps), q_regular=6, ssq_order=5)
    mesh = mu.Mesh(xyz, tri6)
    mesh.tangent_frame(p.frame_rule, out=False)
    inc = workloads.plane_wave()
    Z, near, B = mu.assemble(mesh, p, mu.MUELLER_C64_NEAR64, inc=inc)
    if a.what == "mrhs":
        op = mu.Operator(mesh, Z, near, mu.MUELLER_C64_NEAR64)
        g = torch.Generator().manual_seed(1)
        X = torch.randn((a.rhs, mesh.N), dtype=torch.complex64, generator=g).cuda()
        mu.matvec_mrhs(op, X)
    if a.what == "solve":
        op = mu.Operator(mesh, Z, near, mu.MUELLER_C64_NEAR64)
        mu.precond_build(op, a.block)
        mu.solve(op, B, mu.SolverOpts(mode=mu.SOLVE_GMRES_IR, restart=50, tol=1e-8))
    torch.cuda.synchronize()
    print("ok", mesh.N)


if __name__ == "__main__":
    main()
