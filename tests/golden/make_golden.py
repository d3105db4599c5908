"""Writes the stored expected values under tests/golden/ that come from the
oracle at full workload sizes (too slow to recompute in every test run).

Calls only oracle/ and the seeded workload generators.  Run from the repo
root:  python tests/golden/make_golden.py
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


def q1hex96_pcg():
    """Q1 hex 96^3 (seed 1002): oracle FP64 Jacobi-PCG to rtol 1e-8."""
    p = W.q1_hex(96, seed=W.SEED_C2)
    A = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    oracle.coo_numeric(A, p.v)
    t0 = time.perf_counter()
    x, r = oracle.pcg(A, p.b, rtol=1e-8)
    dt = time.perf_counter() - t0
    return {"workload": "q1hex_96 seed 1002", "nrows": p.nrows, "nnz": A.nnz,
            "ncoo": p.ncoo, "rtol": 1e-8, "result": r, "x_norm": float(np.linalg.norm(x)),
            "note": f"oracle solve took {dt:.1f} s on the machine that wrote this file"}


if __name__ == "__main__":
    out = os.path.join(HERE, "q1hex96_oracle_pcg.json")
    with open(out, "w") as f:
        json.dump(q1hex96_pcg(), f, indent=1)
    print(open(out).read())
