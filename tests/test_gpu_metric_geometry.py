"""Parity at the geometry of the n = 1M benchmark, on a 256 x 256 sample of it.

Same generator and sizes per subdomain as the benchmark workload: radius 3, 8 nonzeros
per random row, 4 random rows per grid point plus 1e-2 I, 64 x 64 blocks (N = 16), at
most 32 coarse vectors per subdomain, threshold automatic.  The four inner subdomains
come close to the bound n_i <= 76^2 = 5,776 columns (Omega_Gamma holds the columns the
rows actually reach, up to six grid lines deep: about 5,740, 180 block rows of 32), so
the local solve runs the same ring of stages and the same shared-memory window as at
n = 1M.  The oracle
runs in banded mode (LAPACK banded Cholesky, ARPACK on the standard form).

Tolerances: FP64 as in the other parity tests.  The FP32 and BF16 local solves are
compared with a model of their rounding computed from the oracle's own factors: each
oracle Cholesky factor rounded to the factor precision (BF16: round to nearest even on
the top 16 bits of the FP32 value) and applied in FP64.  The device rounds other
quantities of the same relative size on top (the gathered right-hand side, the inverse
diagonal tiles it stores instead of L_bb, whose rounding is amplified by up to
cond(L_bb), and FP32 sums of up to ~480 terms), so its error may exceed the model's: by
at most 100x for FP32 (unit roundoff 2^-24, where these extra terms dominate) and 10x
for BF16 (2^-9, where the factor rounding itself dominates).
"""
import numpy as np
import pytest
import scipy.linalg as sl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2107_09006_gb300 as L  # noqa: E402
import oracle as O  # noqa: E402
from workloads import config_scale  # noqa: E402

NEV = 32


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def geo():
    P = config_scale(side=256, block=64)
    A = O.schwarz.as_csr(P.m, P.n, P.row_ptr, P.col, P.val)
    M = O.build_two_level(A, P.part, P.nparts, tau=0.0, nev_max=NEV, mode="banded")
    return dict(P=P, A=A, M=M)


def _solver(g, **kw):
    P = g["P"]
    return L.Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, nev_max=NEV, **kw)


def _round(a, prec):
    if prec == "f32":
        return a.astype(np.float32).astype(np.float64)
    u = a.astype(np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def _local_model(M, r, prec):
    """sum_i R_i^T (L_i~ L_i~^T)^{-1} R_i r with each oracle factor rounded to prec."""
    z = np.zeros_like(r)
    for idx, (cb, lower) in M.local:
        y = sl.cho_solve_banded((_round(cb, prec), lower), r[idx])
        np.add.at(z, idx, y)
    return z


def test_geometry_and_index_sets(geo):
    P, M = geo["P"], geo["M"]
    S = _solver(geo, coarse=0)
    sz = S.sizes()
    inner = np.sort(sz[:, 0])[-4:]
    assert 5700 <= inner.min() and inner.max() <= 5776 and np.sort(sz[:, 0])[-5] < 5400
    assert S.storage()["total_blocks"] >= 4 * 179
    for i in range(P.nparts):
        assert np.array_equal(S.omega(i), M.S.Om[i])
        assert np.array_equal(S.xi(i), M.S.Xi[i])
    S.close()


def test_coarse_dimension_and_two_level_apply_fp64(geo):
    M = geo["M"]
    S = _solver(geo)
    assert S.sizes()[:, 3].tolist() == list(M.ks) and S.info()["n0"] == M.n0
    r = np.random.default_rng(3).standard_normal(geo["P"].n)
    assert rel(S.apply_preconditioner(r, 0).cpu().numpy(), M.apply(r)) < 1e-9
    assert rel(S.apply_preconditioner(r, 1).cpu().numpy(), M.apply_local(r)) < 1e-12
    S.close()


@pytest.mark.parametrize("config", [1, 2])
def test_pcg_fixed_iterations_fp64(geo, config):
    P, M = geo["P"], geo["M"]
    S = _solver(geo, fixed_iters=6, local_config=config)
    x, _ = S.solve(P.b, rtol=1e-8)
    xo, _ = O.pcg(geo["A"], P.b, M.apply, fixed_iters=6)
    assert rel(x.cpu().numpy(), xo) < 1e-10
    S.close()


@pytest.mark.parametrize("prec,config", [("f32", 1), ("f32", 2), ("f32", 3), ("bf16", 1), ("bf16", 2)])
def test_one_level_apply_mixed(geo, prec, config):
    M = geo["M"]
    S = _solver(geo, coarse=0, factor_prec=prec, local_config=config)
    r = np.random.default_rng(4).standard_normal(geo["P"].n)
    exact = M.apply_local(r)
    e_dev = rel(S.apply_preconditioner(r, 1).cpu().numpy(), exact)
    e_model = rel(_local_model(M, r, prec), exact)
    print(f"{prec} one-level apply: device error {e_dev:.2e}, rounded-factor model {e_model:.2e}")
    assert e_dev <= (100 if prec == "f32" else 10) * e_model
    S.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_mixed_solve_error(geo, prec):
    """Converged mixed-form solve against the FP64 oracle: error within 10x the FP64
    oracle PCG's own error at the same tolerance 1e-8 (reference: oracle PCG at 1e-13)."""
    P, M, A = geo["P"], geo["M"], geo["A"]
    if "ref" not in geo:
        geo["ref"] = O.pcg(A, P.b, M.apply, rtol=1e-13)[0]
        geo["fp64_1e8"] = O.pcg(A, P.b, M.apply, rtol=1e-8)[0]
    S = _solver(geo, factor_prec=prec)
    x, info = S.solve(P.b, rtol=1e-8)
    assert info["relres_true"] <= 1e-8
    e_dev, e_fp64 = rel(x.cpu().numpy(), geo["ref"]), rel(geo["fp64_1e8"], geo["ref"])
    print(f"{prec} solve to 1e-8: {info['iters']} iterations, error {e_dev:.2e} "
          f"(FP64 oracle at 1e-8: {e_fp64:.2e})")
    assert e_dev <= 10 * e_fp64
    S.close()
