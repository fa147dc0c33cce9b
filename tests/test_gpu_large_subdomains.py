"""Parity on subdomains too large for the shared-memory Lanczos vectors.

256 x 128 grid (n = 32,768, radius 3, 8 nonzeros per row), two 128 x 128 subdomains:
n_i = 17,148 columns each, so the device eigensolver keeps its two work vectors in
global memory and the FP64 local solve holds a 137 KB right-hand side in shared
memory.  The oracle runs in banded mode (LAPACK banded Cholesky, ARPACK on the
standard form).  Tolerances as in the other parity tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2107_09006_gb300 as L  # noqa: E402
import oracle as O  # noqa: E402
from workloads import make_grid_ls, block_partition  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def big():
    m, n, rp, c, v, b, _ = make_grid_ls(256, 128, 4, 8, 3, 0)
    part = block_partition(256, 128, 128, 128)
    A = O.schwarz.as_csr(m, n, rp, c, v)
    M = O.build_two_level(A, part, 2, tau=0.0, nev_max=16, mode="banded")
    return dict(m=m, n=n, rp=rp, c=c, v=v, b=b, part=part, A=A, M=M)


def _solver(d, **kw):
    return L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 2, nev_max=16, **kw)


def test_sizes_and_index_sets(big):
    S = _solver(big, coarse=0)
    sets = O.index_sets(big["A"], big["part"], 2)
    for i in range(2):
        assert np.array_equal(S.omega(i), sets.Om[i])
        assert np.array_equal(S.xi(i), sets.Xi[i])
    assert S.sizes()[:, 0].min() > 12_000  # beyond the shared-memory eigensolver path
    S.close()


def test_eigenvalues_and_coarse_dimension(big):
    S = _solver(big)
    M = big["M"]
    for i in range(2):
        lg = S.eigvals(i)
        lo = np.asarray(M.lams[i])[: len(lg)]
        k = min(len(lg), len(lo))
        assert np.max(np.abs(lg[:k] - lo[:k])) <= 1e-10 * max(1.0, np.abs(lo).max())
    assert S.sizes()[:, 3].tolist() == list(M.ks)
    assert S.info()["n0"] == M.n0
    S.close()


@pytest.mark.parametrize("prec,tol,config", [("f64", 1e-9, 1), ("f64", 1e-9, 2), ("f32", 1e-5, 1), ("f32", 1e-5, 2),
                                             ("f32", 1e-5, 3)])
def test_two_level_apply(big, prec, tol, config):
    S = _solver(big, factor_prec=prec, local_config=config)
    r = np.random.default_rng(3).standard_normal(big["n"])
    assert rel(S.apply_preconditioner(r, 0).cpu().numpy(), big["M"].apply(r)) < tol
    S.close()


def test_pcg_fixed_iterations(big):
    S = _solver(big, fixed_iters=6)
    x, _ = S.solve(big["b"], rtol=1e-8)
    xo, _ = O.pcg(big["A"], big["b"], big["M"].apply, fixed_iters=6)
    assert rel(x.cpu().numpy(), xo) < 1e-10
    S.close()
