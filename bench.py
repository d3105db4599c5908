#!/usr/bin/env python
"""Benchmark of the sparse SPD solver path on one GB300 (or N replicas).

One step is one pass of the whole hot path over the Q1 hexahedral FE Poisson
workload (96^3 elements, 912,673 rows, 56,623,104 COO entries, 24,137,569
nonzeros), inputs (the element coefficients kappa and b) resident in HBM:
  q1_hex_element_coo / q1_hex_element_values (the COO triples generated on
  the device from kappa, the user Jacobian kernel pattern),
  mat_create_coo (symbolic COO -> CSR on the device), mat_set_values_coo
  (duplicate-summing numeric stage + Jacobi), FP64 fused PCG to rtol 1e-8,
  100 SpMVs, FP32-inner / FP64-refined PCG to rtol 1e-8, adjoint solve plus
  gradient scatter, mat_destroy.
The headline value is the FP64 CG solve time in seconds (lower is better);
SpMV GB/s, the refined and adjoint times, the per-phase device times of the
solve loop and the roofline of the sliced-ELL SpMV kernel (the row product
that also runs the solve's SpMV phase) are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--host-loop]

--host-loop runs the solves with the host-stepped loop instead of the CUDA
graph (same kernels, same grids, bit-identical results) so that a profiler's
launch list sees every kernel of the loop.

--workload selects the comparison runs of the other configurations (each
prints its own JSON line; the default is the Q1 benchmark above):
  c3  7-point Laplacian 192^3: FP64 PCG vs FP32-inner / FP64-refined PCG at
      rtol 1e-10 and 1e-8 (true residuals reported)
  c4  2D edge diffusion 1024^2: forward FP64 solve vs adjoint solve + gradient
      scatter, and dL/dkappa through the edge signs
  c5  512 independent systems (~51.6M rows): one batched launch (FP64 and
      refined) vs 512 sequential single-system solves vs the stacked ensemble
      solve, plus the batched adjoint
  vec vector COO assembly of the Q1 96^3 element load vector (7.08M entries
      into 912,673 nodes): symbolic and numeric stage times, numeric GB/s
  async  time per solve against NNZ (Sec. 6.2's comparison, 2D 5-point, 3D
      7-point and 3D 27-point problems, 5e3 to 2.7e7 nonzeros): the three-kernel
      CG loop, the two-kernel and one-kernel single-reduction CG, the one-kernel
      pipelined CG, the per-CTA CG (up to 2M nonzeros) and TFQMR, all
      device-driven
  nonsym  batched TFQMR and BiCG (Jacobi) on 16, 64, 256 and 1024 independent
      2D convection-diffusion systems (1k-50k rows each, Peclet 1-100): solves
      per second of the batched solve on the per-CTA solver and on the phase
      kernels, against the stacked ensemble solve (Sec. 7's comparison)

--impl reference times the FP64 CPU oracle (the plain C implementation in
oracle/) on a bounded sample of the same workload on the host cores.
Multi-GPU (torchrun): independent replicas, one per GPU, no collective on the
data path; max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("CG solve s and SpMV GB/s (% of HBM peak) at rtol 1e-8; "
          "FP32-refined/batched/adjoint vs FP64")
WORKLOAD = "q1hex_{ne}: 3D Q1 FE Poisson, {ne}^3 elements, log-uniform kappa, seed 1002"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_sha() -> str:
    """Hash of the source of the sliced-ELL SpMV kernel -- spmv.cu, sell.cu,
    device_util.cuh and the sell_rows product in phases.cuh -- which ties a
    stored ncu traffic figure to the code it was measured on."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2406_08646_gb300", "csrc")
    for f in ("spmv.cu", "sell.cu", "device_util.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    with open(os.path.join(csrc, "phases.cuh")) as fh:
        src = fh.read()
    a = src.index("struct Pair;")
    h.update(src[a:src.index("// The row products of block b", a)].encode())
    return h.hexdigest()[:16]


def stored_traffic(name: str):
    """Per-launch DRAM bytes recorded in profiles/<name>.md by an ncu capture
    of the current kernel source, else None."""
    try:
        kv = {}
        with open(os.path.join(ROOT, "profiles", name + ".md")) as f:
            for line in f:
                if ":" in line and line.startswith("- "):
                    k, v = line[2:].split(":", 1)
                    kv[k.strip()] = v.strip().strip("`")
        if kv.get("source_sha") != source_sha():
            return None
        return float(kv["dram_bytes_per_launch"])
    except Exception:
        return None


PATTERNS = "tuned"  # --patterns


def force_patterns(h):
    """Applies --patterns on / off after the autotuner (which otherwise picks)."""
    if PATTERNS != "tuned":
        from paper_2406_08646_gb300 import binding
        binding.mat_set_slice_patterns(h, PATTERNS == "on")


def pcg_alg_bytes(n: int, nnz: int, iterations: int) -> float:
    """Algorithmic bytes of one FP64 PCG launch: per iteration the floor
    12 nnz + 4 (n+1) + 72 n (A once; x, r, p read and written; D^-1 read; q
    written and read), plus setup (b, D^-1 read; x, r, p written: 40 n) and the
    closing true-residual product (12 nnz + 4 (n+1) + 16 n)."""
    it = 12.0 * nnz + 4.0 * (n + 1) + 72.0 * n
    return iterations * it + 40.0 * n + 12.0 * nnz + 4.0 * (n + 1) + 16.0 * n


def pcg_fp64_ops(n: int, nnz: int, iterations: int) -> float:
    """FP64 pipe instructions (FMA, multiply or add, one slot each, per lane)
    of one FP64 PCG launch on the phase kernels: per iteration one FMA per
    stored nonzero and one per row for q = A p and p.q, five per row in the
    update (r, z, x, r.z, r.r) and one in the direction (p); the setup and the
    closing residual add about nnz + 7 n.  Reductions are not counted."""
    return iterations * (nnz + 7.0 * n) + nnz + 7.0 * n


def fp64_peak_gops(clk: dict) -> float:
    """The FP64 pipe's peak in G instructions (per lane) per second: 2 per
    clock per SM at the SM clock sampled during the run."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    return 2.0 * nsm * mhz * 1e6 / 1e9


def solve_fp64_pipe(n: int, nnz: int, iterations: int, seconds: float, clk: dict):
    """The whole FP64 solve against the FP64 pipe (its co-bound with HBM on
    this part), or None if it cannot be computed."""
    try:
        peak = fp64_peak_gops(clk)
        got = pcg_fp64_ops(n, nnz, iterations) / seconds / 1e9
        return {"achieved": got, "peak": peak, "unit": "G FP64 op/s", "frac": got / peak,
                "what": "FP64 instructions of the solve (bench.pcg_fp64_ops: nnz + 7 n per "
                        "iteration) over its event time, against 2 per SM per clock"}
    except Exception:
        return None


def fp64_pipe(nnz: int, seconds: float, clk: dict) -> dict:
    """The SpMV's other bound: one FP64 FMA per stored nonzero against the FP64
    pipe's peak, 2 FMAs per clock per SM (GB300's FP64 rate, 1.25 TFLOP/s
    nominal) times the SMs and the SM clock sampled during the run."""
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz") or 2070.0
    peak = 2.0 * nsm * mhz * 1e6 / 1e9  # G FMA/s
    got = nnz / seconds / 1e9
    return {"achieved": got, "peak": peak, "unit": "G FMA/s", "frac": got / peak,
            "what": "the row product's FP64 FMAs (one per nonzero) over the FP64 pipe's "
                    "peak at the sampled SM clock"}


def s0_rows(med: dict, ne: int, hbm: float) -> dict:
    """The device-side COO generation of the step against HBM: the values
    kernel reads kappa (8 B per element) and writes 64 doubles per element;
    the index kernel writes 64 (i, j) int32 pairs per element."""
    E = float(ne) ** 3
    out = {}
    for key, alg in (("gen_values", 8.0 * E + 512.0 * E), ("gen_indices", 512.0 * E)):
        s = med[key] / 1e3
        out[key] = {"us": s * 1e6, "alg_bytes": alg, "gbs": alg / s / 1e9,
                    "frac": alg / s / 1e9 / hbm}
    return out


def spmv_alg_bytes(n: int, nnz: int) -> float:
    """Values and column indices once (12 B per nonzero), x once and y once
    (16 B per row); the sliced layout's slice offsets replace row pointers and
    are not counted."""
    return 12.0 * nnz + 16.0 * n


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle

def oracle_sample(p):
    """Times the oracle on the workload: its COO assembly, then its full FP64
    PCG solve to rtol 1e-8, once as it stands (one thread) and once in its
    all-cores build (the same loops split over the host's cores, same
    results); about 10 s in all."""
    import oracle
    t0 = time.perf_counter()
    A = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    t1 = time.perf_counter()
    oracle.coo_numeric(A, p.v)
    t2 = time.perf_counter()
    x, r = oracle.pcg(A, p.b, rtol=1e-8)
    t3 = time.perf_counter()
    oracle.coo_numeric(A, p.v, omp=True)
    t4 = time.perf_counter()
    xo, ro = oracle.pcg(A, p.b, rtol=1e-8, omp=True)
    t5 = time.perf_counter()
    return {"symbolic_s": t1 - t0, "numeric_s": t2 - t1, "solve_s": t3 - t2,
            "numeric_all_s": t4 - t3, "solve_all_s": t5 - t4, "cores": oracle.threads(),
            "iterations": r["iterations"], "status": r["status"],
            "same_bits": bool(x.tobytes() == xo.tobytes())}


def run_reference(args, rank: int, world: int):
    """The oracle as it stands, timed on the host cores: each step is its
    numeric COO stage plus its full FP64 PCG solve of the workload."""
    if rank != 0:
        return 0
    from paper_2406_08646_gb300 import workloads as W
    import oracle
    p = W.q1_hex(96, seed=W.SEED_C2)
    A = oracle.coo_symbolic(p.nrows, p.ncols, p.i, p.j)
    times, steps = [], []
    its = None
    cores = oracle.threads()
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.coo_numeric(A, p.v, omp=True)
        t1 = time.perf_counter()
        x, r = oracle.pcg(A, p.b, rtol=1e-8, omp=True)
        t2 = time.perf_counter()
        its = r["iterations"]
        if step >= args.warmup:
            times.append(t2 - t1)
            steps.append(t2 - t0)
    value = statistics.median(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(steps), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(ne=96), "nrows": p.nrows, "nnz": A.nnz,
                       "ncoo": p.ncoo,
                       "rtol": 1e-8, "iterations": its},
            "cpu_baseline": {"value": value, "unit": "s", "cores": cores, "kind": "oracle",
                             "sample": "whole workload: each step is the oracle's numeric "
                                       "COO stage and its full FP64 PCG solve, plain C "
                                       "with its SpMV and vector loops split over all "
                                       f"{cores} host cores (OpenMP; inner products "
                                       "sequential, same results as one thread)"},
            "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- GPU arm

# ----------------------------------------------------------------- other configs

def _ev_time(stream, fn, reps=3, warm=1):
    """Median CUDA-event time (s) of fn() on `stream` over `reps` after `warm`."""
    import torch
    out = []
    for k in range(warm + reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        if k >= warm:
            out.append(e0.elapsed_time(e1) / 1e3)
    return statistics.median(out), r


def _base_line(args, metric_value, config, extra):
    hbm, kind = peaks()
    line = {"metric": METRIC, "value": metric_value, "unit": "s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config, "peak_hbm_gbs": hbm, "peak_kind": kind}
    line.update(extra)
    return line


def tfqmr_alg_bytes(n: int, nnz: int, products: int) -> float:
    """Algorithmic bytes of the fused TFQMR loop per product with A D^-1: the
    matrix once (12 B per nonzero) and 17.5 FP64 vectors of n (a step of two
    products reads or writes 35: the first half step 10, the product fused
    with the second half step 10 plus its gathered vector, the y1 / x update
    8, the product with the v update 5 plus its gathered vector)."""
    return products * (12.0 * nnz + 140.0 * n)


def bicg_alg_bytes(n: int, nnz: int, iterations: int) -> float:
    """Algorithmic bytes of the fused BiCG loop per iteration: A and A^T once
    each (24 B per nonzero) and 23 FP64 vectors of n (directions 7, products 4
    plus the two gathered vectors, updates 10)."""
    return iterations * (24.0 * nnz + 184.0 * n)


def run_suite(args):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_08646_gb300 import binding as B
    from paper_2406_08646_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream(dev)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    reps = max(1, args.steps)
    hbm, _ = peaks()

    if args.workload == "c3":
        p = W.poisson3d(192, seed=W.SEED_C3)
        A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
        A.set_values(t(p.v))
        b = t(p.b)
        x = torch.empty_like(b)
        y = torch.empty_like(b)
        sp, _ = _ev_time(stream, lambda: [A.mult(b, y) for _ in range(20)], reps=reps)
        spmv_s = sp / 20
        import tempfile
        A.autotune(os.path.join(tempfile.mkdtemp(prefix="gbs_bench_c3_"), "tuning.txt"))
        force_patterns(A.h)
        rows = {}
        for rtol in (1e-10, 1e-8):
            for prec, name in ((B.FP64, "fp64"), (B.FP32_REFINED, "fp32_refined")):
                ts, (_, r) = _ev_time(stream, lambda: A.solve(b, x, rtol=rtol, precision=prec),
                                      reps=reps)
                ph = A.phase_ns()
                rows[f"{name}@{rtol:g}"] = {
                    "s": ts, "iterations": r["iterations"],
                    "outer_iterations": r["outer_iterations"], "status": r["status"],
                    "true_rel_residual": r["true_rel_residual"],
                    "us_per_iteration": {k: v / 1e3 / max(r["iterations"], 1)
                                         for k, v in ph.items()
                                         if k in ("spmv", "update_xr", "update_p")}}
        n, nnz = p.nrows, A.nnz
        line = _base_line(
            args, rows["fp64@1e-10"]["s"],
            {"workload": "poisson3d_192: 7-point Laplacian 192^3, random-normal rhs, seed 1003",
             "nrows": n, "nnz": nnz, "plan": dict(A.plan(), patterns=A.slices()["pattern_slices"] > 0)},
            {"solves": rows,
             "refined_vs_fp64": {k: rows[f"fp32_refined@{k}"]["s"] / rows[f"fp64@{k}"]["s"]
                                 for k in ("1e-10", "1e-08")},
             "spmv": {"us": spmv_s * 1e6, "gbs": spmv_alg_bytes(n, nnz) / spmv_s / 1e9,
                      "frac": spmv_alg_bytes(n, nnz) / spmv_s / 1e9 / hbm},
             "solve_gbs_fp64@1e-10": pcg_alg_bytes(n, nnz, rows["fp64@1e-10"]["iterations"])
                                     / rows["fp64@1e-10"]["s"] / 1e9,
             "solve_roofline_fp64@1e-10": {
                 "frac": pcg_alg_bytes(n, nnz, rows["fp64@1e-10"]["iterations"])
                         / rows["fp64@1e-10"]["s"] / 1e9 / hbm,
                 "what": "PCG floor bytes (bench.pcg_alg_bytes) over the solve's event time, "
                         "against the measured copy peak"},
             "tuning": A.tuning()})
        print(json.dumps(line), flush=True)
        A.close()
        return 0

    if args.workload == "c4":
        p = W.edge_diffusion(1024, seed=W.SEED_C4)
        A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
        A.set_values(t(p.v))
        b, xt = t(p.b), t(p.extra["x_target"])
        x = torch.empty_like(b)
        untuned_s, _ = _ev_time(stream, lambda: A.solve(b, x, rtol=1e-8), reps=reps)
        import tempfile
        A.autotune(os.path.join(tempfile.mkdtemp(prefix="gbs_bench_c4_"), "tuning.txt"))
        force_patterns(A.h)
        tf, (_, rf) = _ev_time(stream, lambda: A.solve(b, x, rtol=1e-8), reps=reps)
        g = (x - xt).contiguous()
        ta, (lam, _, dldv, ra) = _ev_time(
            stream, lambda: A.adjoint(x, g, dlda=False, dldv=True, rtol=1e-8), reps=reps)
        signs = t(W.EDGE_SIGNS)
        gk = (dldv.view(-1, 4) * signs).sum(dim=1)
        line = _base_line(
            args, tf,
            {"workload": "edge_diffusion_1024: 2D 5-point variable-coefficient diffusion, "
                         "kappa log-uniform [0.1, 10], seed 1004",
             "nrows": p.nrows, "nnz": A.nnz, "ncoo": p.ncoo,
             "plan": dict(A.plan(), patterns=A.slices()["pattern_slices"] > 0)},
            {"forward": {"s": tf, "iterations": rf["iterations"], "status": rf["status"],
                         "true_rel_residual": rf["true_rel_residual"],
                         "untuned_s": untuned_s, "tuning": A.tuning()},
             "adjoint": {"s": ta, "iterations": ra[0]["iterations"], "status": ra[0]["status"],
                         "true_rel_residual": ra[0]["true_rel_residual"],
                         "what": "A^T lambda = x - x_target solve plus the dL/dv scatter"},
             "adjoint_vs_forward": ta / tf,
             "loss": float(0.5 * ((x - xt) ** 2).sum()),
             "grad_norms": {"dL/db": float(lam.norm()), "dL/dkappa": float(gk.norm())}})
        print(json.dumps(line), flush=True)
        A.close()
        return 0

    if args.workload == "vec":
        n, iv, vv = W.q1_load_vector(96)
        i_d, v_d = t(iv), t(vv)
        y = torch.zeros(n, dtype=torch.float64, device=dev)
        tc, V = _ev_time(stream, lambda: B.Vec(n, i_d), reps=reps)
        ts, _ = _ev_time(stream, lambda: [V.set_values(v_d, y) for _ in range(20)], reps=reps)
        ts /= 20
        ne = V.info["nentries"]
        alg = 12.0 * iv.shape[0] + 28.0 * ne
        line = _base_line(
            args, ts,
            {"workload": "q1_load_vector_96: 8 entries per element of the Q1 96^3 mesh",
             "n": n, "ncoo": int(iv.shape[0]), "nentries": ne},
            {"symbolic_s": tc, "numeric_s": ts, "numeric_alg_bytes": alg,
             "numeric_gbs": alg / ts / 1e9, "numeric_frac": alg / ts / 1e9 / hbm,
             "what": "numeric = vec_set_values_coo (in-order sums + scatter into y), "
                     "algorithmic bytes 12 per COO entry + 28 per distinct index"})
        print(json.dumps(line), flush=True)
        V.close()
        return 0

    if args.workload == "c5":
        t0 = time.perf_counter()
        bt = W.batch(512, seed=W.SEED_C5)
        gen_s = time.perf_counter() - t0
        A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
        A.set_values(t(bt.v))
        b = t(bt.b)
        x = torch.empty_like(b)
        rows = {}
        # the batched FP64 solve on each engine: per-CTA, phase kernels, and
        # the size split with the k largest systems on the phase kernels
        order = np.sort(bt.nrows)[::-1]
        engines = {}
        # (plans: automatic blocks, or 4096-row SpMV / 8192-row update blocks;
        # the per-CTA solver at one CTA per SM, or two under a cap of two)
        for name, solver, k, plan in (
                ("cta", B.SOLVER_CTA, 0, (0, 0, 0)), ("cta_2_per_sm", B.SOLVER_CTA, 0, (0, 0, 2)),
                ("phases", B.SOLVER_PHASES, 0, (0, 0, 0)),
                ("phases_4096", B.SOLVER_PHASES, 0, (4096, 8192, 0)),
                ("split_8", B.SOLVER_SPLIT, 8, (4096, 8192, 0)),
                ("split_32", B.SOLVER_SPLIT, 32, (4096, 8192, 0)),
                ("split_128", B.SOLVER_SPLIT, 128, (4096, 8192, 0))):
            A.set_plan(plan[0], plan[1], B.SPMV_SELL, plan[2])
            A.set_solver(solver, split_rows=int(order[k - 1]) if k else None)
            te_, (_, rs_) = _ev_time(stream, lambda: A.solve_batched(b, x, rtol=1e-8), reps=reps)
            engines[name] = {"s": te_, "ok": sum(q["status"] == B.OK for q in rs_),
                             "iterations_max": max(q["iterations"] for q in rs_)}
        # the autotuner's choice (30-iteration candidate runs), then the rows below
        import tempfile
        tune_path = os.path.join(tempfile.mkdtemp(prefix="gbs_bench_c5_"), "tuning.txt")
        A.autotune(tune_path)
        force_patterns(A.h)
        tuned = A.tuning()
        rows["engines"] = engines
        rows["autotuned"] = {"solver": tuned["solver"], "split_rows": tuned["split_rows"],
                             "plan": A.plan(), "patterns": A.slices()["pattern_slices"] > 0}
        for prec, name in ((B.FP64, "batched_fp64"), (B.FP32_REFINED, "batched_fp32_refined")):
            ts, (_, rs) = _ev_time(stream, lambda: A.solve_batched(b, x, rtol=1e-8,
                                                                   precision=prec), reps=reps)
            its = [q["iterations"] for q in rs]
            rows[name] = {"s": ts, "ok": sum(q["status"] == B.OK for q in rs),
                          "iterations_max": max(its), "iterations_mean": float(np.mean(its)),
                          "true_rel_residual_max": max(q["true_rel_residual"] for q in rs)}
        te, (_, re) = _ev_time(stream, lambda: A.solve(b, x, rtol=1e-8), reps=reps)
        rows["ensemble_fp64"] = {"s": te, "iterations": re["iterations"], "status": re["status"],
                                 "what": "the stacked block-diagonal system, one global norm"}
        # roofline of the batched FP64 solve: per system its iterations times
        # the PCG floor bytes and FP64 operations, summed, over the solve time
        _, rs64 = A.solve_batched(b, x, rtol=1e-8)
        rp = A.csr()[0].cpu().numpy().astype(np.int64)
        ro_ = bt.row_off
        alg = ops = 0.0
        for q in range(bt.nsys):
            n_q = int(ro_[q + 1] - ro_[q])
            nz_q = int(rp[ro_[q + 1]] - rp[ro_[q]])
            alg += pcg_alg_bytes(n_q, nz_q, rs64[q]["iterations"])
            ops += pcg_fp64_ops(n_q, nz_q, rs64[q]["iterations"])
        hbm_, _ = peaks()
        t64 = rows["batched_fp64"]["s"]
        clk_ = {"sm_mhz": None}
        rows["roofline"] = {"bound": "hbm", "achieved": alg / t64 / 1e9, "peak": hbm_,
                            "unit": "GB/s", "frac": alg / t64 / 1e9 / hbm_, "alg_bytes": alg,
                            "fp64": {"achieved": ops / t64 / 1e9, "peak": fp64_peak_gops(clk_),
                                     "unit": "G FP64 op/s",
                                     "frac": ops / t64 / 1e9 / fp64_peak_gops(clk_)},
                            "what": "sum over systems of iterations x (12 nnz + 4 (n + 1) + 72 n) "
                                    "plus setup and closing residual (bench.pcg_alg_bytes), and "
                                    "of the FP64 operations (bench.pcg_fp64_ops), over the "
                                    "autotuned batched FP64 solve's time"}
        xb, _ = A.solve_batched(b, rtol=1e-8)
        g = (xb - t(bt.extra["x_target"])).contiguous()
        tadj, (_, _, _, ra) = _ev_time(
            stream, lambda: A.adjoint(xb, g, dlda=False, dldv=True, batched=True, rtol=1e-8),
            reps=reps)
        rows["batched_adjoint"] = {"s": tadj, "ok": sum(q["status"] == B.OK for q in ra)}
        A.close()
        # 512 separate single-system handles, solved one after another
        ro, co = bt.row_off, bt.coo_off
        mats, bs, xs = [], [], []
        for q in range(bt.nsys):
            sl = slice(int(co[q]), int(co[q + 1]))
            M = B.Mat.from_coo(int(bt.nrows[q]), int(bt.nrows[q]), t(bt.i[sl]), t(bt.j[sl]))
            M.set_values(t(bt.v[sl]))
            mats.append(M)
            bs.append(b[int(ro[q]):int(ro[q + 1])])
            xs.append(torch.empty_like(bs[-1]))

        def seq():
            for M, bq, xq in zip(mats, bs, xs):
                M.solve(bq, xq, rtol=1e-8, want_result=False)
            return None
        ts, _ = _ev_time(stream, seq, reps=max(1, reps // 2))
        res = [M.solve(bq, xq, rtol=1e-8)[1] for M, bq, xq in zip(mats, bs, xs)]
        rows["sequential_fp64"] = {"s": ts, "ok": sum(r["status"] == B.OK for r in res),
                                   "what": "512 single-system handles, ksp_solve_cg each"}
        for M in mats:
            M.close()
        line = _base_line(
            args, rows["batched_fp64"]["s"],
            {"workload": "batch_512: 2D 5-point / 3D 7-point edge-diffusion systems, rows "
                         "uniform on [1k, 200k], kappa log-uniform [0.1, 10], seed 1005",
             "nsys": bt.nsys, "nrows": int(bt.nrows.sum()), "ncoo": int(bt.ncoo.sum()),
             "generate_s": gen_s},
            {"solves": rows,
             "batched_vs_sequential": rows["batched_fp64"]["s"] / rows["sequential_fp64"]["s"],
             "batched_vs_ensemble": rows["batched_fp64"]["s"] / rows["ensemble_fp64"]["s"],
             "refined_vs_fp64": rows["batched_fp32_refined"]["s"] / rows["batched_fp64"]["s"]})
        print(json.dumps(line), flush=True)
        return 0
    if args.workload == "async":
        problems = ([("poisson2d", m, lambda m=m: W.poisson2d(m))
                     for m in (32, 64, 128, 256, 512, 1024, 2048)]
                    + [("poisson3d", m, lambda m=m: W.poisson3d(m, seed=W.SEED_C3))
                       for m in (16, 32, 64, 128)]
                    + [("q1hex", m, lambda m=m: W.q1_hex(m, seed=W.SEED_C2))
                       for m in (8, 16, 32, 64, 96)])
        if args.async_problems:
            keep = set(args.async_problems.split(","))
            problems = [q for q in problems if f"{q[0]}_{q[1]}" in keep]
        rows = []
        for kind, m, make in problems:
            p = make()
            if kind == "poisson2d":  # its own rhs is an eigenvector: use a random one
                p.b = np.random.default_rng(W.SEED_C7 + m).standard_normal(p.nrows)
            A = B.Mat.from_coo(p.nrows, p.ncols, t(p.i), t(p.j))
            A.set_values(t(p.v))
            b = t(p.b)
            x = torch.empty_like(b)
            row = {"problem": f"{kind}_{m}", "n": p.nrows, "nnz": A.nnz}
            TB, SR2, SR1 = B.CG_TEXTBOOK, B.CG_SINGLE_REDUCTION, B.CG_SINGLE_KERNEL
            runs = [("cg", B.KSP_CG, B.SOLVER_PHASES, TB), ("cgsr", B.KSP_CGSR, B.SOLVER_PHASES, SR2),
                    ("cgsr1", B.KSP_CGSR, B.SOLVER_PHASES, SR1),
                    ("pipecg", B.KSP_PIPECG, B.SOLVER_PHASES, TB),
                    ("tfqmr", B.KSP_TFQMR, B.SOLVER_PHASES, TB)]
            if A.nnz <= 2_000_000:
                runs.append(("cg_cta", B.KSP_CG, B.SOLVER_CTA, TB))
            for name, method, solver, form in runs:
                A.set_solver(solver)
                A.set_cg_form(form)
                ts, (_, r) = _ev_time(stream, lambda: A.solve(b, x, rtol=1e-8, method=method,
                                                              host_loop=args.host_loop),
                                      reps=max(1, min(reps, 3)), warm=1)
                row[name] = {"s": ts, "iterations": r["iterations"], "status": r["status"],
                             "us_per_iteration": ts * 1e6 / max(r["iterations"], 1),
                             "true_rel_residual": r["true_rel_residual"]}
                if name in ("cg", "cgsr"):
                    ph = A.phase_ns()
                    row[name]["phase_us_per_iteration"] = {
                        k: v / 1e3 / max(r["iterations"], 1) for k, v in ph.items()
                        if k in ("spmv", "update_xr", "update_p")}
            row["pipecg_vs_cg"] = row["cg"]["s"] / row["pipecg"]["s"]
            row["cgsr_vs_cg"] = row["cg"]["s"] / row["cgsr"]["s"]
            row["cgsr1_vs_cg"] = row["cg"]["s"] / row["cgsr1"]["s"]
            rows.append(row)
            A.close()
        big = rows[-1]
        line = _base_line(
            args, big["pipecg"]["s"],
            {"workload": "stencil sweep: poisson2d 32^2..2048^2 (random rhs, seed 1007 + m), "
                         "poisson3d 16^3..128^3 (seed 1003), q1_hex 8^3..96^3 (seed 1002); "
                         "value = pipelined CG on q1_hex_64",
             "rtol": 1e-8},
            {"sweep": rows,
             "what": "s = CUDA-event time of one solve (inputs resident); pipecg_vs_cg = "
                     "CG time / pipelined CG time"})
        print(json.dumps(line), flush=True)
        return 0

    if args.workload == "nonsym":
        sweep = {}
        sizes = [int(v) for v in args.nonsym_sizes.split(",")]
        for nsys in sizes:
            bt = W.convdiff_batch(nsys, seed=W.SEED_C6)
            A = B.Mat.from_coo_batched(bt.nrows, bt.ncoo, t(bt.i), t(bt.j))
            A.set_values(t(bt.v))
            b = t(bt.b)
            x = torch.empty_like(b)
            ro = bt.row_off
            nnz_s = None
            entry = {"rows": int(bt.nrows.sum()), "nnz": A.nnz}
            for mname, method in (("tfqmr", B.KSP_TFQMR), ("bicg", B.KSP_BICG)):
                res = {}
                for sname, solver in (("cta", B.SOLVER_CTA), ("phases", B.SOLVER_PHASES)):
                    A.set_solver(solver)
                    ts, (_, rs) = _ev_time(stream, lambda: A.solve_batched(
                        b, x, rtol=1e-8, method=method), reps=1, warm=1)
                    if nnz_s is None:
                        rp = A.csr()[0].cpu().numpy()
                        nnz_s = np.diff(rp[ro])
                    its = np.array([q["iterations"] for q in rs])
                    alg = (tfqmr_alg_bytes if method == B.KSP_TFQMR else bicg_alg_bytes)(
                        np.diff(ro), nnz_s, its).sum()
                    res[f"batched_{sname}"] = {
                        "s": ts, "solves_per_s": nsys / ts,
                        "ok": int(sum(q["status"] == B.OK for q in rs)),
                        "iterations_max": int(its.max()), "iterations_mean": float(its.mean()),
                        "gbs": float(alg / ts / 1e9), "frac": float(alg / ts / 1e9 / hbm)}
                A.set_solver(B.SOLVER_AUTO)
                _, rs = A.solve_batched(b, x, rtol=1e-8, method=method)
                res["auto_picks"] = "cta" if rs[0]["solver"] == B.SOLVER_CTA else "phases"
                A.set_solver(B.SOLVER_PHASES)
                te, (_, re) = _ev_time(stream, lambda: A.solve(b, x, rtol=1e-8, method=method),
                                       reps=1, warm=1)
                res["ensemble"] = {"s": te, "solves_per_s": nsys / te, "status": re["status"],
                                   "iterations": re["iterations"]}
                best = min(res["batched_cta"]["s"], res["batched_phases"]["s"])
                res["batched_vs_ensemble_speedup"] = te / best
                entry[mname] = res
            sweep[str(nsys)] = entry
            A.close()
        top = sweep[str(sizes[-1])]["tfqmr"]
        line = _base_line(
            args, min(top["batched_cta"]["s"], top["batched_phases"]["s"]),
            {"workload": "convdiff_batch: 2D upwind convection-diffusion systems, rows "
                         "uniform on [1k, 50k], Peclet log-uniform [1, 100], seed 1006; "
                         f"value = batched TFQMR on {sizes[-1]} systems",
             "batch_sizes": sizes},
            {"sweep": sweep,
             "what": "solves_per_s = systems / solve time; ensemble = the stacked system "
                     "with one global norm on the phase kernels; gbs = algorithmic bytes "
                     "(bench.tfqmr_alg_bytes / bicg_alg_bytes over each system's "
                     "iterations) / time"})
        print(json.dumps(line), flush=True)
        return 0
    raise SystemExit(f"unknown workload {args.workload}")


def max_over_ranks(vals, device):
    """Each value's maximum over the ranks of the default process group (a
    replica job takes as long as its slowest rank); unchanged on one rank or
    without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def run_gpu(args, rank: int, world: int):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2406_08646_gb300 import binding as B
    from paper_2406_08646_gb300 import workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    L = B.lib()
    p = W.q1_hex(args.ne, seed=W.SEED_C2)
    rng = np.random.default_rng(77)
    xt_h = rng.standard_normal(p.nrows)
    # the step's inputs are the element coefficients and b; the COO triples
    # are generated on the device each step (S0), then assembled
    kappa_d = torch.from_numpy(p.extra["kappa"]).to(dev)
    i_d = torch.empty(p.ncoo, dtype=torch.int32, device=dev)
    j_d = torch.empty(p.ncoo, dtype=torch.int32, device=dev)
    v_d = torch.empty(p.ncoo, dtype=torch.float64, device=dev)
    b_d = torch.from_numpy(p.b).to(dev)
    xt_d = torch.from_numpy(xt_h).to(dev)
    n, ncoo = p.nrows, p.ncoo
    x64 = torch.empty(n, dtype=torch.float64, device=dev)
    x32 = torch.empty(n, dtype=torch.float64, device=dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    g = torch.empty(n, dtype=torch.float64, device=dev)
    lam = torch.empty(n, dtype=torch.float64, device=dev)
    dldv = torch.empty(ncoo, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = B._stream(stream)
    hl = bool(args.host_loop)
    o64 = B.make_opts(rtol=1e-8, host_loop=hl)
    o32 = B.make_opts(rtol=1e-8, precision=B.FP32_REFINED, host_loop=hl)
    oadj = B.make_opts(rtol=1e-8, host_loop=hl)
    SPMV_REPS = 100
    # the autotuner's file for this run: the first warm-up step tunes the
    # matrix, later steps (new handles of the same matrix) reload its choice
    import tempfile
    tune_path = args.tune_file or os.path.join(tempfile.mkdtemp(prefix="gbs_bench_"),
                                               "tuning.txt")
    tune_hits = []

    def check(st):
        if st != B.OK:
            raise B.GbsError(st, B.last_error())

    def step(record):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        eg = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        res = {}
        eg[0].record(stream)
        check(L.q1_hex_element_coo(args.ne, B._dev(i_d, torch.int32), B._dev(j_d, torch.int32),
                                   sp))
        eg[1].record(stream)
        check(L.q1_hex_element_values(args.ne, B._dev(kappa_d, torch.float64),
                                      B._dev(v_d, torch.float64), sp))
        ev[0].record(stream)
        A = B.mat_create_coo(n, n, i_d, j_d, stream)
        ev[1].record(stream)
        check(L.mat_set_values_coo(A, B._dev(v_d, torch.float64), B.INSERT, sp))
        et = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        et[0].record(stream)
        tune_hits.append(B.mat_autotune_file(A, tune_path, stream))
        force_patterns(A)
        et[1].record(stream)
        ev[2].record(stream)
        check(L.ksp_solve_cg(A, B._dev(b_d, torch.float64), B._dev(x64, torch.float64),
                             B.ctypes.byref(o64), None, sp))
        ev[3].record(stream)
        res["fp64"] = B.ksp_get_result(A, 1, stream)[0]
        res["phases_fp64"] = B.ksp_get_phase_ns(A, stream)
        ev[4].record(stream)
        for _ in range(SPMV_REPS):
            check(L.mat_mult(A, B._dev(b_d, torch.float64), B._dev(y, torch.float64), sp))
        ev[5].record(stream)
        check(L.ksp_solve_cg(A, B._dev(b_d, torch.float64), B._dev(x32, torch.float64),
                             B.ctypes.byref(o32), None, sp))
        ev[6].record(stream)
        res["fp32_refined"] = B.ksp_get_result(A, 1, stream)[0]
        res["phases_fp32_refined"] = B.ksp_get_phase_ns(A, stream)
        torch.sub(x64, xt_d, out=g)
        ev7 = torch.cuda.Event(enable_timing=True)
        ev7.record(stream)
        check(L.ksp_adjoint(A, B._dev(x64, torch.float64), B._dev(g, torch.float64),
                            B._dev(lam, torch.float64), None, B._dev(dldv, torch.float64),
                            B.ctypes.byref(oadj), None, sp))
        ev[7].record(stream)
        res["adjoint"] = B.ksp_get_result(A, 1, stream)[0]
        nnz = B.mat_get_info(A)["nnz"]
        plan = dict(B.mat_get_plan(A), **B.mat_get_tuning(A),
                    patterns=B.mat_get_slices(A)["pattern_slices"] > 0)
        B.mat_destroy(A)
        stream.synchronize()
        t = {"gen_indices": eg[0].elapsed_time(eg[1]), "gen_values": eg[1].elapsed_time(ev[0]),
             "create": ev[0].elapsed_time(ev[1]), "set_values": ev[1].elapsed_time(et[0]),
             "tune": et[0].elapsed_time(et[1]),
             "solve_fp64": ev[2].elapsed_time(ev[3]),
             "spmv_x100": ev[4].elapsed_time(ev[5]),
             "solve_fp32_refined": ev[5].elapsed_time(ev[6]),
             "adjoint": ev7.elapsed_time(ev[7]), "step": eg[0].elapsed_time(ev[7])}
        return t, res, nnz, plan

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step(False)
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    c0 = B.launch_count()
    w0 = time.perf_counter()
    rows, results = [], []
    for _ in range(args.steps):
        t, res, nnz, plan = step(True)
        rows.append(t)
        results.append(res)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - w0
    launches = (B.launch_count() - c0) / max(args.steps, 1)
    clk = clocks.stop()

    med = {k: statistics.median(r[k] for r in rows) for k in rows[0]}
    step_ms = statistics.mean(r["step"] for r in rows)
    solve_s = med["solve_fp64"] / 1e3
    solve_s, step_ms = max_over_ranks([solve_s, step_ms], dev)

    # ---- end to end through the C-ABI from pinned host buffers (H2D + D2H in region)
    e2e = None if args.no_e2e else e2e_time(p, dev, stream, sp, L, B, o64, check, tune_path)
    if e2e is not None:
        e2e["kappa"]["value"], e2e["host_coo"]["value"] = max_over_ranks(
            [e2e["kappa"]["value"], e2e["host_coo"]["value"]], dev)

    r64 = results[-1]["fp64"]
    it = r64["iterations"]
    hbm, peak_kind = peaks()
    solve_gbs = pcg_alg_bytes(n, nnz, it) / solve_s / 1e9
    spmv_s = med["spmv_x100"] / 1e3 / SPMV_REPS
    spmv_gbs = spmv_alg_bytes(n, nnz) / spmv_s / 1e9
    traffic = stored_traffic(f"spmv_sell_q1hex{args.ne}")

    def per_iter(ph, its):
        return {k: v / 1e3 / max(its, 1) for k, v in ph.items()
                if k in ("spmv", "update_xr", "update_p")}
    last = results[-1]
    phases = {"fp64_us_per_iteration": per_iter(last["phases_fp64"], it),
              "fp32_refined_us_per_iteration":
                  per_iter(last["phases_fp32_refined"], last["fp32_refined"]["iterations"]),
              "what": "device clock of CTA 0 from each phase kernel's start to the next "
                      "one's start (launch gaps included), summed over the loop"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.ne == 96:
        s = oracle_sample(p)
        cpu = {"value": s["solve_all_s"], "unit": "s", "cores": s["cores"], "kind": "oracle",
               "sample": (f"whole workload, once: oracle COO assembly "
                          f"({s['symbolic_s']:.1f} s symbolic, {s['numeric_s']:.2f} s numeric) "
                          f"then its full FP64 PCG solve ({s['iterations']} iterations, "
                          f"status {s['status']}), on all {s['cores']} host cores (OpenMP "
                          f"row and vector loops, sequential inner products; "
                          f"bit-identical to one thread: {s['same_bits']}); value = the "
                          f"solve"),
               "one_core": {"value": s["solve_s"], "unit": "s", "cores": 1}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": solve_s, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD.format(ne=args.ne), "nrows": n, "nnz": nnz,
                       "ncoo": ncoo,
                       "rtol": 1e-8, "spmv_reps": SPMV_REPS,
                       "l2": "no flush: every input is larger than L2 (CSR 290 MB, COO 906 MB)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "plan": plan, "loop": "host-stepped" if hl else "graph",
                       "tuning": (f"mat_autotune_file: {sum(tune_hits)} of "
                                  f"{len(tune_hits)} steps reloaded the tuning from its file "
                                  f"({sum(tune_hits[-args.steps:])}/{args.steps} timed steps)"
                                  + ("" if args.tune_file else
                                     "; the first warm-up step tuned the matrix"))},
            "rows_ms": med,
            "iterations": {k: last[k]["iterations"] for k in ("fp64", "fp32_refined", "adjoint")},
            "outer_iterations_fp32_refined": last["fp32_refined"]["outer_iterations"],
            "true_rel_residual": {k: last[k]["true_rel_residual"]
                                  for k in ("fp64", "fp32_refined", "adjoint")},
            "status": {k: last[k]["status"] for k in ("fp64", "fp32_refined", "adjoint")},
            "spmv": {"gbs": spmv_gbs, "frac": spmv_gbs / hbm, "us": spmv_s * 1e6,
                     "alg_bytes": spmv_alg_bytes(n, nnz)},
            "generate": s0_rows(med, args.ne, hbm),
            "roofline": {"kernel": "k_spmv_sell (MatMult, sliced-ELL FP64 row product)",
                         "bound": "hbm", "achieved": spmv_gbs, "peak": hbm, "unit": "GB/s",
                         "frac": spmv_gbs / hbm, "peak_kind": f"{peak_kind} (copy, burst)",
                         "traffic": traffic, "alg_bytes": spmv_alg_bytes(n, nnz),
                         "timing": f"CUDA events around {SPMV_REPS} back-to-back launches "
                                   "on the launching stream, median over steps",
                         "fp64": fp64_pipe(nnz, spmv_s, clk)},
            "solve_roofline": {"what": "whole FP64 solve (one graph launch): PCG floor bytes "
                                       "12 nnz + 4(n+1) + 72 n per iteration, plus setup and "
                                       "closing residual, over the solve's event time",
                               "achieved": solve_gbs, "peak": hbm, "unit": "GB/s",
                               "frac": solve_gbs / hbm,
                               "alg_bytes": pcg_alg_bytes(n, nnz, it)},
            "solve_fp64_pipe": solve_fp64_pipe(n, nnz, it, solve_s, clk),
            "solve_phases": phases,
            "refined_vs_fp64": med["solve_fp32_refined"] / med["solve_fp64"],
            "adjoint_vs_fp64": med["adjoint"] / med["solve_fp64"],
            "e2e": None if e2e is None else {
                "value": e2e["kappa"]["value"], "unit": "s",
                "h2d_bytes_per_step": e2e["kappa"]["h2d_bytes"],
                "d2h_bytes_per_step": e2e["kappa"]["d2h_bytes"],
                "stages_ms": e2e["kappa"]["stages_ms"],
                "what": "pinned host kappa + b -> device, COO triples generated on the "
                        "device, assemble, FP64 solve, x -> host",
                "host_coo": dict(e2e["host_coo"], what="pinned host COO (i, j, v) + b -> "
                                 "device, assemble, FP64 solve, x -> host")},
            "gpu_launches": launches,
            "clocks": clk,
            "wall_s": wall,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    return 0


def e2e_time(p, dev, stream, sp, L, B, o64, check, tune_path):
    """End to end through the C-ABI from pinned host memory, two ways, each the
    median over 2 timed reps (after 1 untimed), all on one stream, CUDA events
    between the stages:
      kappa:    the element coefficients and b copied to the device, the COO
                triples generated there (q1_hex_element_coo / _values), then
                mat_create_coo, mat_set_values_coo, FP64 ksp_solve_cg, x copied
                back to the host;
      host_coo: the COO triples (i, j, v) and b copied to the device, then the
                same assembly, solve and copy back.
    After the numeric stage each applies the autotuner's stored choice for the
    matrix (mat_autotune_file, a lookup: the bench's warm-up tuned it); its
    time is in the set_values stage.
    Returns {name: {"value": s, "stages_ms": {...}, "h2d_bytes": B, "d2h_bytes": B}}."""
    import torch
    n, ne = p.nrows, p.extra["ne"]
    kap = p.extra["kappa"]
    pin = lambda a: torch.from_numpy(a).pin_memory()
    i_h, j_h, v_h, b_h, k_h = pin(p.i), pin(p.j), pin(p.v), pin(p.b), pin(kap)
    x_h = torch.empty(n, dtype=torch.float64).pin_memory()
    i2 = torch.empty(p.ncoo, dtype=torch.int32, device=dev)
    j2 = torch.empty(p.ncoo, dtype=torch.int32, device=dev)
    v2 = torch.empty(p.ncoo, dtype=torch.float64, device=dev)
    b2 = torch.empty(n, dtype=torch.float64, device=dev)
    k2 = torch.empty(kap.shape[0], dtype=torch.float64, device=dev)
    x2 = torch.empty(n, dtype=torch.float64, device=dev)
    names = ("h2d", "generate", "create", "set_values", "solve", "d2h")

    def run(from_kappa):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
        torch.cuda.synchronize()
        ev[0].record(stream)
        if from_kappa:
            k2.copy_(k_h, non_blocking=True)
        else:
            i2.copy_(i_h, non_blocking=True)
            j2.copy_(j_h, non_blocking=True)
            v2.copy_(v_h, non_blocking=True)
        b2.copy_(b_h, non_blocking=True)
        ev[1].record(stream)
        if from_kappa:
            check(L.q1_hex_element_coo(ne, B._dev(i2, torch.int32), B._dev(j2, torch.int32), sp))
            check(L.q1_hex_element_values(ne, B._dev(k2, torch.float64),
                                          B._dev(v2, torch.float64), sp))
        ev[2].record(stream)
        A = B.mat_create_coo(n, n, i2, j2, stream)
        ev[3].record(stream)
        check(L.mat_set_values_coo(A, B._dev(v2, torch.float64), B.INSERT, sp))
        B.mat_autotune_file(A, tune_path, stream)
        force_patterns(A)
        ev[4].record(stream)
        check(L.ksp_solve_cg(A, B._dev(b2, torch.float64), B._dev(x2, torch.float64),
                             B.ctypes.byref(o64), None, sp))
        ev[5].record(stream)
        x_h.copy_(x2, non_blocking=True)
        ev[6].record(stream)
        ev[6].synchronize()
        r = B.ksp_get_result(A, 1, stream)[0]
        B.mat_destroy(A)
        if r["status"] != B.OK:
            raise B.GbsError(r["status"], "end-to-end solve failed")
        st = {nm: ev[k].elapsed_time(ev[k + 1]) for k, nm in enumerate(names)}
        return ev[0].elapsed_time(ev[6]) / 1e3, st

    out = {}
    for name, from_kappa in (("kappa", True), ("host_coo", False)):
        reps = [run(from_kappa) for _ in range(3)][1:]
        tot = statistics.median(t for t, _ in reps)
        stages = {nm: statistics.median(st[nm] for _, st in reps) for nm in names}
        h2d = (kap.nbytes if from_kappa else p.i.nbytes + p.j.nbytes + p.v.nbytes) + p.b.nbytes
        out[name] = {"value": tot, "stages_ms": stages, "h2d_bytes": int(h2d),
                     "d2h_bytes": int(n * 8)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gbs", choices=["gbs", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--async-problems", default="",
                    help="--workload async: only these problems (e.g. poisson2d_32,q1hex_8)")
    ap.add_argument("--nonsym-sizes", default="16,64,256,1024",
                    help="batch sizes of --workload nonsym (comma-separated)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "vec", "nonsym", "async"],
                    help="c2 = the benchmark (default); c3/c4/c5 = comparison runs")
    ap.add_argument("--host-loop", action="store_true",
                    help="run the solves' loop from the host (for profiler launch lists)")
    ap.add_argument("--tune-file", default="",
                    help="the autotuner's file for the Q1 workload (default: a new one, so "
                         "the first warm-up step tunes; an existing file skips the tuning, "
                         "e.g. for launch lists)")
    ap.add_argument("--patterns", default="tuned", choices=["tuned", "on", "off"],
                    help="column patterns of the sliced copy: the autotuner's choice "
                         "(default), or forced on / off after it (for profiling captures)")
    ap.add_argument("--ne", type=int, default=96,
                    help="elements per side of the Q1 workload (96 = the benchmark; "
                         "smaller only for profiling captures)")
    args = ap.parse_args()
    global PATTERNS
    PATTERNS = args.patterns
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "c2":
        return run_suite(args) if rank == 0 else 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    try:
        return run_gpu(args, rank, world)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
