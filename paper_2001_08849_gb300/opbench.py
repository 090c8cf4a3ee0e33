"""Operator micro-benchmark: repeated raw operator applications on a Kuhn
cantilever, through the C ABI (sfem_time_operator).

  python -m paper_2001_08849_gb300.opbench --cells 200 40 42 --op mf32 --reps 20

Prints one JSON line: mean device ms per application, DOF/s and the
algorithmic bytes of the FP32 matrix-free operator.  Used to time and
profile the operator kernels in isolation (e.g. under ncu).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

OPS = {"csr64": 0, "mf64": 1, "mf32": 2}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, nargs=3, default=[200, 40, 42])
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--op", choices=sorted(OPS), default="mf32")
    ap.add_argument("--reps", type=int, default=20)
    a = ap.parse_args(argv)
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2001_08849_gb300 import sfem as S
    from inputs.kuhn_beam import cantilever
    p = cantilever(*a.cells, seed=a.seed)
    with S.FsFem(p, on_device=True) as ctx:
        if a.op == "csr64":
            S.sfem_assemble(ctx.h)
        ms = S.sfem_time_operator(ctx.h, OPS[a.op], a.reps)
        torch.cuda.synchronize()
        n_tets = p.mesh.n_tets
        out = {"op": a.op, "cells": a.cells, "n_tets": n_tets, "ndof": ctx.ndof, "ms_per_apply": ms,
               "gdof_per_s": ctx.ndof / ms / 1e6,
               "alg_bytes_mf32": 72 * n_tets + 8 * ctx.ndof,
               "tiles": None}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
