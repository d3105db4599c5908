"""Host-side arithmetic of bench.py on CPU: the algorithmic byte and FP64
instruction counts behind its roofline figures."""


def test_bench_roofline_helpers():
    """The bench's algorithmic counts: PCG floor bytes and FP64 instructions
    per iteration grow by exactly one iteration's worth per iteration, and the
    FP64-pipe figure degrades to None when no device can be queried."""
    import bench
    n, nnz = 1000, 5000
    assert bench.pcg_alg_bytes(n, nnz, 11) - bench.pcg_alg_bytes(n, nnz, 10) == \
        12.0 * nnz + 4.0 * (n + 1) + 72.0 * n
    assert bench.pcg_fp64_ops(n, nnz, 11) - bench.pcg_fp64_ops(n, nnz, 10) == nnz + 7.0 * n
    assert bench.spmv_alg_bytes(n, nnz) == 12.0 * nnz + 16.0 * n
    import torch
    if not torch.cuda.is_available():
        assert bench.solve_fp64_pipe(n, nnz, 10, 1e-3, {"sm_mhz": 2070.0}) is None
