"""CPU checks of the benchmark's bookkeeping: the config line states the sizes the
generator really produces (ragged block partitions included), and the algorithmic byte
counts behind the roofline figures follow their stated formulas."""
import argparse

import bench
from workloads import config_scale


def _args(side, block):
    return argparse.Namespace(side=side, block=block, nev=32, rtol=1e-8, gpus=1)


def test_config_line_matches_generated_workload():
    for side, block in ((256, 64), (100, 32)):
        P = config_scale(side=side, block=block)
        cfg = bench.solve_config(_args(side, block), 1)
        assert f"n={P.n}, m={P.m}, nnz={P.nnz}" in cfg["workload"]
        assert f"N{P.nparts}:" in cfg["workload"] and f"{P.nparts} subdomains" in cfg["workload"]


def test_both_arms_share_the_config():
    a = _args(1024, 64)
    assert bench.solve_config(a, 1) == bench.solve_config(a, 1)
    assert bench.solve_config(a, 1)["workload"].startswith(
        "grid1024-r3k8-N256: n=1048576, m=5242880, nnz=34603008, 256 subdomains 64x64")


def test_spmv_bytes_formula():
    # A p: 12 B per entry, 8 B per row pointer, p read, q written; A^T q the same over
    # the CSC copy plus the fused p . w read of p
    m, n, nnz = 5242880, 1048576, 34603008
    assert bench.spmv_bytes(m, n, nnz) == 2 * 12 * nnz + (m + 1) * 8 + (n + 1) * 8 + 2 * m * 8 + 3 * n * 8
    assert bench.spmv_bytes(m, n, nnz) == 989855760


def test_local_solve_bytes_terms():
    st = {"fac_elems": 1024 * 10, "total_local": 100, "zbar_elems": 7}
    f32 = bench.local_solve_bytes(st, "f32")
    assert f32 == 2 * 10240 * 4 + 100 * 28 + 7 * 8
    assert bench.local_solve_bytes(st, "f32", restrict=False) == f32 - 7 * 8
    # BF16: two bytes per element plus one FP32 scale per 32 x 32 tile, read by both sweeps
    assert bench.local_solve_bytes(st, "bf16") == 2 * 10240 * 2 + 2 * 10 * 4 + 100 * 28 + 7 * 8
    assert bench.local_solve_bytes(st, "f64") == 2 * 10240 * 8 + 100 * 28 + 7 * 8
