"""Write tests/golden/beam_2m_reference.json with the FP64 oracle only.

Workload: the 200 x 40 x 42-cell Kuhn cantilever (2,016,000 tets) on
[0,10] x [0,1] x [0,1] m, jitter seed 2, E = 210 GPa, nu = 0.3, x = 0 clamped,
traction (0, 0, -1e6) Pa on x = 10.  The oracle assembles K (Eq. 7 / Eq. 9 /
Eq. 12 route, chunked) and runs its Jacobi-PCG; the file records

  * iterations_1e-8: the iteration at which the recursive residual first
    reached 1e-8 (the count a Jacobi-PCG at tol 1e-8 performs),
  * the final true relative residual of the tight solve and its iterations,
  * the tip deflection (mean -u_z over the x = 10 face nodes) and ||u||_2,
  * u at a seeded sample of nodes, for sampled full-size comparisons,
  * phase timings of the oracle on this machine (context only).

Run: python tests/golden/make_beam_2m_reference.py  (about half an hour).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from inputs.kuhn_beam import cantilever, face_nodes  # noqa: E402
from oracle import fsfem as F  # noqa: E402
from oracle import solve as OS  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "beam_2m_reference.json")


def main(nx=200, ny=40, nz=42, seed=2, tight=1e-10):
    t0 = time.time()
    p = cantilever(nx, ny, nz, seed=seed)
    m = p.mesh
    t1 = time.time()
    asm = F.assemble(m.xyz, m.tets, p.E, p.nu, chunk=200000)
    t2 = time.time()
    f = F.traction_load(m.n_nodes, m.xyz, p.trac_tris, p.trac)[0]
    A, b, _, _ = F.dirichlet_system(asm.matrix(), f, p.dir_dofs, p.dir_vals)
    t3 = time.time()
    res = OS.jacobi_pcg(A, b, tight, max_iter=60000, max_restarts=3)
    t4 = time.time()
    hist = np.array(res.history)
    it8 = int(np.argmax(hist <= 1e-8)) if (hist <= 1e-8).any() else -1
    u = res.x
    tip = face_nodes(m, 0, 1)
    rng = np.random.default_rng(1234)
    sample = np.unique(np.concatenate([rng.integers(0, m.n_nodes, 200), tip[::37]]))
    out = {
        "workload": f"Kuhn cantilever {nx}x{ny}x{nz} cells x 6 tets, seed {seed}",
        "n_nodes": int(m.n_nodes), "n_tets": int(m.n_tets), "ndof": int(asm.ndof),
        "n_faces": int(asm.faces.n), "n_interior": int(asm.faces.n_interior),
        "n_boundary": int(asm.faces.n_boundary), "nnz": int(asm.indices.size),
        "n_triplets": int(asm.n_triplets),
        "iterations_1e-8": it8,
        "tight_tol": tight, "tight_iterations": int(res.iterations),
        "tight_true_relres": float(res.true_relres),
        "bnorm": float(np.linalg.norm(b)),
        "tip_deflection": float(-u.reshape(-1, 3)[tip, 2].mean()),
        "u_norm2": float(np.linalg.norm(u)),
        "sample_nodes": sample.tolist(),
        "sample_u": u.reshape(-1, 3)[sample].tolist(),
        "timing_s": {"generate": t1 - t0, "assemble": t2 - t1, "bc_load": t3 - t2, "pcg": t4 - t3},
    }
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps({k: v for k, v in out.items() if not k.startswith("sample")}, indent=1))


if __name__ == "__main__":
    main()
