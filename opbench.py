"""Operator and solver micro-benchmarks through the C ABI, for timing and
for profiling single kernels in isolation (e.g. under ncu).

  python opbench.py --cells 200 40 42 --op mf32f64 --reps 20
  python opbench.py --cells 200 40 42 --solve fpcg_learned --tol 1e-8

--op: repeated raw operator applications (sfem_time_operator); prints the
mean device ms per application, DOF/s and the algorithmic bytes of the FP32
matrix-free operator.
--solve: one solve of the cantilever (pcg64 on CSR, the mixed-precision
ir32_64, flexible PCG without (fpcg) or with an untrained learned correction
(fpcg_learned, patches of 8 x 8 x 8 nodes)); --precond 1 adds the two-level
preconditioner (the library's default coarse grid unless --coarse-dims) to
pcg64 and ir32_64; prints iterations and time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OPS = {"csr64": 0, "mf64": 1, "mf32": 2, "mf32f64": 3, "ns64": 4, "es64": 5}
SOLVES = ("pcg64", "ir32_64", "fpcg", "fpcg_learned")


def tiled_source_sha() -> str:
    """SHA-256 of the sources of the tiled FP32 operator kernel (a stored
    DRAM-traffic figure is valid only for the kernel it was measured on)."""
    h = hashlib.sha256()
    for f in ("tiles.cu", "tile_apply.cuh"):
        with open(os.path.join(ROOT, "paper_2001_08849_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def batch_main(a):
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_08849_gb300 import sfem as S
    from inputs.kuhn_beam import batch_beams
    probs = batch_beams(64, seed=5)
    ctxs = [S.FsFem(p, on_device=True) for p in probs]
    try:
        us = [torch.zeros((p.nrhs, c.ndof), dtype=torch.float64, device="cuda") for p, c in zip(probs, ctxs)]
        n_sys = sum(p.nrhs for p in probs)
        opts = S.batch_opts(tol=a.tol, u_on_device=True, precond=a.batch)
        S.sfem_batch_solve([c.h for c in ctxs], us, opts, n_sys, check=False)
        for u in us:
            u.zero_()
        torch.cuda.synchronize()
        infos, stats = S.sfem_batch_solve([c.h for c in ctxs], us, opts, n_sys, check=False)
        out = {"batch": a.batch, "beams": len(probs), "systems": n_sys, "solves_per_s": n_sys / (stats["ms"] / 1e3),
               "converged": sum(1 for i in infos if i["status"] == 0),
               "max_true_relres": max(i["true_relres"] for i in infos), **stats}
    finally:
        for c in ctxs:
            c.close()
    print(json.dumps(out), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, nargs=3, default=[200, 40, 42])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--nu", type=float, default=0.3, help="Poisson ratio")
    ap.add_argument("--op", choices=sorted(OPS), default="mf32")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--solve", choices=SOLVES, default=None)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--max-iter", type=int, default=0)
    ap.add_argument("--window", type=int, default=0, help="learned_window of the fpcg_learned solve")
    ap.add_argument("--precond", type=int, default=0, help="1: two-level preconditioner (pcg64, ir32_64)")
    ap.add_argument("--coarse-dims", type=int, nargs=3, default=None,
                    help="patch centres per axis (default: the library's, patches 8 mean node spacings wide)")
    ap.add_argument("--repeat", type=int, default=1, help="solves (the last one is reported)")
    ap.add_argument("--fp32-vectors", type=int, default=0, help="ir32_64 vector precision (sfem_solve_opts)")
    ap.add_argument("--inner-tol", type=float, default=0.0, help="ir32_64 reliable-update threshold (0: 0.1)")
    ap.add_argument("--recover", action="store_true",
                    help="time sfem_recover (face and nodal strain / stress) on a solved displacement")
    ap.add_argument("--batch", type=int, default=None, metavar="PRECOND",
                    help="the batched solve of 64 uneven cantilevers x 4 load cases (sfem_batch_solve) with "
                         "this precond (0 Jacobi, 1 per system, 2 two-level in the persistent launch): one "
                         "untimed call (coarse spaces, autotuner), then one timed call")
    a = ap.parse_args(argv)
    if a.batch is not None:
        return batch_main(a)
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_08849_gb300 import sfem as S
    from inputs.kuhn_beam import cantilever
    t_mesh = time.perf_counter()
    p = cantilever(*a.cells, seed=a.seed, nu=a.nu)
    t_mesh = time.perf_counter() - t_mesh
    with S.FsFem(p, on_device=True) as ctx:
        n_tets = p.mesh.n_tets
        if a.recover:
            S.sfem_coarse_setup(ctx.h)
            u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
            S.sfem_solve(ctx.h, u, S.solve_opts(kind=S.SFEM_SOLVE_IR32_64, tol=1e-8, u_on_device=True, precond=1,
                                                fp32_vectors=3, inner_tol=0.03))
            S.sfem_recover(ctx.h, u)  # warm-up
            ts = []
            for _ in range(a.reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                S.sfem_recover(ctx.h, u)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            nf = ctx.info["n_faces"]
            out = {"recover": True, "cells": a.cells, "n_tets": n_tets, "n_faces": nf, "ndof": ctx.ndof,
                   "ms_median": 1e3 * sorted(ts)[len(ts) // 2],
                   "output_bytes": 8 * (12 * nf + 13 * (ctx.ndof // 3))}
        elif a.solve is None:
            if a.op == "csr64":
                S.sfem_assemble(ctx.h)
            ms = S.sfem_time_operator(ctx.h, OPS[a.op], a.reps)
            torch.cuda.synchronize()
            out = {"op": a.op, "cells": a.cells, "n_tets": n_tets, "ndof": ctx.ndof, "ms_per_apply": ms,
                   "gdof_per_s": ctx.ndof / ms / 1e6,
                   "alg_bytes_mf32": 72 * n_tets + (16 if a.op == "mf32f64" else 8) * ctx.ndof,
                   "tiled_source_sha256": tiled_source_sha(), "tiles": S.sfem_tile_info(ctx.h)}
        else:
            model = None
            coarse = None
            if a.precond:
                dims = tuple(a.coarse_dims) if a.coarse_dims else (0, 0, 0)  # library default
                for _ in range(a.repeat):
                    coarse = S.sfem_coarse_setup(ctx.h, patch_dims=dims)
            if a.solve == "pcg64":
                S.sfem_assemble(ctx.h)
                o = S.solve_opts(kind=S.SFEM_SOLVE_PCG64, op64=S.SFEM_OP_CSR64, tol=a.tol, u_on_device=True,
                                 max_iter=a.max_iter, precond=a.precond)
            elif a.solve == "ir32_64":
                o = S.solve_opts(kind=S.SFEM_SOLVE_IR32_64, tol=a.tol, u_on_device=True, max_iter=a.max_iter,
                                 precond=a.precond, fp32_vectors=a.fp32_vectors, inner_tol=a.inner_tol)
            else:
                S.sfem_assemble(ctx.h)
                if a.solve == "fpcg_learned":
                    dims = tuple(-(-(c + 1) // 8) for c in a.cells)
                    model = S.Learned(ctx.h, patch_dims=dims, seed=1, keepalive=ctx._keep)
                o = S.solve_opts(kind=S.SFEM_SOLVE_FPCG_LEARNED, op64=S.SFEM_OP_CSR64, tol=a.tol,
                                 u_on_device=True, learned=model, max_iter=a.max_iter, learned_window=a.window)
            for _ in range(a.repeat):
                u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                info = S.sfem_solve(ctx.h, u, o, check=False)
                torch.cuda.synchronize()
            out = {"solve": a.solve, "cells": a.cells, "nu": a.nu, "n_tets": n_tets, "ndof": ctx.ndof,
                   "mesh_gen_s": t_mesh, "time_s": time.perf_counter() - t0, "mesh_setup_ms": ctx.info["setup_ms"], "coarse": coarse,
                   **info}
            if model is not None:
                model.close()
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
