"""Writes gmres_poisson100.json: the oracle's s-step GMRES on the 3D Poisson workload
(7-point Dirichlet Laplacian on a 100^3 grid, n = 1e6, Jacobi, b = A 1, x0 = 0,
m = 60, s = 5, tol 1e-10) with one-stage randomized BCGS2 and with the two-stage
scheme (s_hat = 20): iteration counts, restarts, final true relative residuals and
the per-restart residual histories (Section 4, s-step GMRES; Sections 5-7 for the
orthogonalization).  Calls only the oracle and the seeded input generators; the GPU
parity test at this size and the benchmark's reference arm read the file.

Run:  python tests/golden/make_gmres_poisson100.py     (about 4 minutes on 8 cores)
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import krylov  # noqa: E402


def main():
    A = synth.poisson3d_csr(100)
    b = synth.ones_rhs(A)
    out = {"workload": "3D Poisson 7-point 100^3 (n=1e6), Jacobi, b=A*1, x0=0, m=60, s=5, tol 1e-10",
           "n": int(A.n), "nnz": int(A.nnz), "m": 60, "s": 5, "tol": 1e-10, "sketch": "sparse-sign d=244 zeta=8 seed 42"}
    for name, kw in (("one_stage", dict(scheme="one")), ("two_stage", dict(scheme="two", s_hat=20))):
        t0 = time.perf_counter()
        r = krylov.sstep_gmres(A, b, s=5, m=60, tol=1e-10, max_restarts=200, **kw)
        dt = time.perf_counter() - t0
        out[name] = {"s_hat": kw.get("s_hat", 5), "converged": bool(r.converged),
                     "iterations": int(r.iterations), "restarts": int(r.restarts),
                     "relres": float(r.relres), "max_abs_x_minus_1": float(np.abs(r.x - 1.0).max()),
                     "history": [[int(i), float(v)] for i, v in r.history], "oracle_seconds": dt}
        print(name, out[name]["iterations"], out[name]["relres"], f"{dt:.1f} s", flush=True)
    out["cores"] = os.cpu_count()
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "gmres_poisson100.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
