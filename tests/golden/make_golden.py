"""Writes the stored expected values under tests/golden/ that come from the
oracle at full workload sizes (too slow to recompute in every test run).

Calls only oracle/ and the seeded workload generators.  Run from the repo
root:  python tests/golden/make_golden.py [name ...]   (default: all)
  q1hex96      Q1 hex 96^3: FP64 PCG, single-reduction PCG, refined PCG
  poisson3d192 7-point 192^3: FP64 PCG and single-reduction PCG at rtol 1e-10
  edge1024     2D edge diffusion 1024^2: forward PCG at rtol 1e-8 and 1e-12,
               the adjoint at rtol 1e-12 (loss, gradient norms, sampled
               entries of lambda and dL/dkappa)
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2406_08646_gb300 import workloads as W  # noqa: E402


def _assemble(p):
    A = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(A, p.v)
    return A


def _timed(fn, *a, **k):
    t0 = time.perf_counter()
    out = fn(*a, **k)
    return out, time.perf_counter() - t0


def q1hex96():
    """Q1 hex 96^3 (seed 1002) to rtol 1e-8: PCG, single-reduction PCG and
    the refined solve (inner_rtol 1e-4) with its inner counts per step."""
    p = W.q1_hex(96, seed=W.SEED_C2)
    A = _assemble(p)
    (x, r), dt = _timed(oracle.pcg, A, p.b, rtol=1e-8)
    (xs, rs), dts = _timed(oracle.pcg_sr, A, p.b, rtol=1e-8)
    (xr, rr, trace), dtr = _timed(oracle.pcg_refined, A, p.b, rtol=1e-8, inner_rtol=1e-4,
                                  want_trace=True)
    return {"workload": "q1hex_96 seed 1002", "nrows": p.nrows, "nnz": A.nnz,
            "ncoo": p.ncoo, "rtol": 1e-8, "result": r, "x_norm": float(np.linalg.norm(x)),
            "result_sr": rs, "result_refined": rr, "refined_inner_per_outer": trace,
            "note": f"oracle solves took {dt:.1f} / {dts:.1f} / {dtr:.1f} s (PCG / single-"
                    f"reduction / refined) on the machine that wrote this file"}


def poisson3d192():
    """7-point 192^3 (seed 1003) to rtol 1e-10: PCG and single-reduction PCG."""
    p = W.poisson3d(192, seed=W.SEED_C3)
    A = _assemble(p)
    (x, r), dt = _timed(oracle.pcg, A, p.b, rtol=1e-10)
    (xs, rs), dts = _timed(oracle.pcg_sr, A, p.b, rtol=1e-10)
    return {"workload": "poisson3d_192 seed 1003", "nrows": p.nrows, "nnz": A.nnz,
            "rtol": 1e-10, "result": r, "result_sr": rs,
            "note": f"oracle solves took {dt:.1f} / {dts:.1f} s on the machine that wrote "
                    f"this file"}


def edge1024():
    """2D edge diffusion 1024^2 (seed 1004): forward to rtol 1e-8 (counts) and
    1e-12 (the point the adjoint is taken at), the adjoint lambda = A^-1 g,
    g = x - x_target, at rtol 1e-12; dL/dkappa_e = sum of the edge's four
    dL/dv entries times their signs (+1, +1, -1, -1); sampled entries."""
    p = W.edge_diffusion(1024, seed=W.SEED_C4)
    A = _assemble(p)
    (x8, r8), dt8 = _timed(oracle.pcg, A, p.b, rtol=1e-8)
    (x, r12), dt12 = _timed(oracle.pcg, A, p.b, rtol=1e-12)
    g = x - p.extra["x_target"]
    (lam, dlda, dldv, ra), dta = _timed(oracle.adjoint, A, x, g, rtol=1e-12)
    gk = (dldv.reshape(-1, 4) * W.EDGE_SIGNS).sum(axis=1)
    rng = np.random.default_rng(4)
    rows = sorted(set(rng.integers(0, p.nrows, 24).tolist()) | {0, p.nrows - 1})
    edges = sorted(set(rng.integers(0, gk.shape[0], 24).tolist()) | {0, gk.shape[0] - 1})
    return {"workload": "edge_diffusion_1024 seed 1004", "nrows": p.nrows, "nnz": A.nnz,
            "ncoo": p.ncoo, "forward_rtol_1e-8": r8, "forward_rtol_1e-12": r12,
            "x_norm": float(np.linalg.norm(x)), "loss": float(0.5 * np.dot(g, g)),
            "adjoint_rtol_1e-12": ra, "lambda_norm": float(np.linalg.norm(lam)),
            "dLdkappa_norm": float(np.linalg.norm(gk)),
            "lambda_sample": {str(i): float(lam[i]) for i in rows},
            "dLdkappa_sample": {str(e): float(gk[e]) for e in edges},
            "note": f"oracle solves took {dt8:.1f} / {dt12:.1f} / {dta:.1f} s on the machine "
                    f"that wrote this file"}


MAKERS = {"q1hex96": ("q1hex96_oracle_pcg.json", q1hex96),
          "poisson3d192": ("poisson3d192_oracle_pcg.json", poisson3d192),
          "edge1024": ("edge1024_oracle.json", edge1024)}

if __name__ == "__main__":
    names = sys.argv[1:] or list(MAKERS)
    for nm in names:
        fname, fn = MAKERS[nm]
        out = os.path.join(HERE, fname)
        data = fn()
        with open(out, "w") as f:
            json.dump(data, f, indent=1)
        print(open(out).read())
