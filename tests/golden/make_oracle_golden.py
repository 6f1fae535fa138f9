"""Writes tests/golden/oracle_<grid>_<fmt>[_ru].json: the CPU oracle's own solve
of a synthetic FEM system -- iterations, updates or restarts, residuals, norms
and the solution at seeded sample positions.  Calls only femgen (inputs) and
oracle/.

  python tests/golden/make_oracle_golden.py GRID [sym|csr] [TOL] [--method cg|ru] [--threads N]

--method cg: the double-precision CG of the Section III listing (oracle.cg);
--method ru: single-precision iterations with double-precision reliable
updates (oracle.cg_ru), the mixed-precision form of Section IV's
single-precision variant.  --threads N > 1 runs the oracle's multi-threaded
build, which gives the single-threaded build's bits (pinned by
tests/test_oracle_threads.py); the file records which build ran.
"""
import argparse
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
    ap = argparse.ArgumentParser()
    ap.add_argument("grid", choices=sorted(GRIDS))
    ap.add_argument("fmt", nargs="?", default="sym", choices=["sym", "csr"])
    ap.add_argument("tol", nargs="?", type=float, default=1e-10)
    ap.add_argument("--method", default="cg", choices=["cg", "ru"])
    ap.add_argument("--threads", type=int, default=1)
    a = ap.parse_args()
    g = GRIDS[a.grid]
    s = femgen.build_system(g)
    arrs = s.upper() if a.fmt == "sym" else (s.ptr, s.idx, s.val)
    lib = oracle.load_threaded(a.threads) if a.threads > 1 else oracle.load()
    t0 = time.time()
    if a.method == "cg":
        r = oracle.cg(a.fmt, *arrs, s.b, tol=a.tol, lib=lib, scalar_history=min(s.n, 400000))
    else:
        r = oracle.cg_ru(a.fmt, *arrs, s.b, tol=a.tol, lib=lib)
    secs = time.time() - t0
    rng = np.random.default_rng(12345)
    sample = np.sort(rng.choice(s.n, size=min(4096, s.n), replace=False))
    what = {"cg": "double-precision CG", "ru": "single-precision CG with double-precision reliable updates"}
    out = {
        "_what": f"CPU oracle (oracle/oracle.c) {what[a.method]} solve of a femgen system",
        "_script": "tests/golden/make_oracle_golden.py",
        "method": a.method, "oracle_threads": oracle.threads(lib),
        "grid": [g.nx, g.ny, g.nz], "n_incl": g.n_incl, "contrast": g.contrast, "seed_mesh": g.seed_mesh,
        "seed_x": g.seed_x, "format": a.fmt, "tol": a.tol, "n": s.n, "nnz": s.nnz,
        "status": r.status, "iterations": r.iterations, "restarts": r.restarts,
        "rel_res_true": r.rel_res_true, "rel_res_recursive": r.rel_res_recursive,
        "x_norm": float(np.linalg.norm(r.x)), "err_vs_xstar": float(np.linalg.norm(r.x - s.xstar) / np.linalg.norm(s.xstar)),
        "oracle_seconds": secs, "seconds_per_iteration": secs / max(r.iterations, 1),
        "sample_index": sample.tolist(), "sample_x": r.x[sample].tolist(),
    }
    if a.method == "cg" and oracle.threads(lib) == 1:
        out["oracle_seconds_single_thread"] = secs
    if a.method == "cg":
        # extreme eigenvalue estimates (Ritz values of the CG-Lanczos
        # tridiagonal) of the run before any restart: kappa_hat bounds the
        # solution difference of two solves to relative residual tol by
        # 2 kappa tol
        m = r.alpha.shape[0] if r.restarts == 0 else int(0.9 * r.alpha.shape[0])
        lo, hi = oracle.lanczos_extremes(r.alpha[:m], r.beta[:m])
        out.update({"lanczos_steps": m, "lambda_min_ritz": lo, "lambda_max_ritz": hi, "kappa_hat": hi / lo})
    suffix = "" if a.method == "cg" else "_ru"
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_{a.grid}_{a.fmt}{suffix}.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(path, r.status, r.iterations, r.restarts, r.rel_res_true, secs)


if __name__ == "__main__":
    main()
