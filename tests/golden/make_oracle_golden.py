"""Writes tests/golden/oracle_<grid>.json: the CPU oracle's own double-precision
CG solve of a synthetic FEM system (iterations, residuals, norms and the
solution at seeded sample positions).  Calls only femgen (inputs) and oracle/.

Usage: python tests/golden/make_oracle_golden.py 128 [sym|csr] [tol]
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import femgen  # noqa: E402
import oracle  # noqa: E402

GRIDS = {"31": femgen.PAPER_SIZE, "64": femgen.DIFF, "128": femgen.LARGE, "256": femgen.LARGEST}


def main():
    key = sys.argv[1] if len(sys.argv) > 1 else "128"
    fmt = sys.argv[2] if len(sys.argv) > 2 else "sym"
    tol = float(sys.argv[3]) if len(sys.argv) > 3 else 1e-10
    g = GRIDS[key]
    s = femgen.build_system(g)
    arrs = s.upper() if fmt == "sym" else (s.ptr, s.idx, s.val)
    t0 = time.time()
    r = oracle.cg(fmt, *arrs, s.b, tol=tol)
    secs = time.time() - t0
    rng = np.random.default_rng(12345)
    sample = np.sort(rng.choice(s.n, size=min(4096, s.n), replace=False))
    out = {
        "_what": "CPU oracle (oracle/oracle.c, double precision, single thread) CG solve of a femgen system",
        "_script": "tests/golden/make_oracle_golden.py",
        "grid": [g.nx, g.ny, g.nz], "n_incl": g.n_incl, "contrast": g.contrast, "seed_mesh": g.seed_mesh,
        "seed_x": g.seed_x, "format": fmt, "tol": tol, "n": s.n, "nnz": s.nnz,
        "status": r.status, "iterations": r.iterations, "restarts": r.restarts,
        "rel_res_true": r.rel_res_true, "rel_res_recursive": r.rel_res_recursive,
        "x_norm": float(np.linalg.norm(r.x)), "err_vs_xstar": float(np.linalg.norm(r.x - s.xstar) / np.linalg.norm(s.xstar)),
        "oracle_seconds_single_thread": secs, "seconds_per_iteration": secs / max(r.iterations, 1),
        "sample_index": sample.tolist(), "sample_x": r.x[sample].tolist(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_{key}_{fmt}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, r.status, r.iterations, r.rel_res_true, secs)


if __name__ == "__main__":
    main()
