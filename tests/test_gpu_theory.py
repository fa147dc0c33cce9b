"""The paper's central claim on the device at growing subdomain counts.

Zero-sum 128 x 128 grid (radius 3, 8 nonzeros per row, each random row centred to sum
to zero, plus 1e-2 I rows): C behaves like a graph Laplacian, so one-level Schwarz
degrades as N grows.  For N = 4, 16, 64 square subdomains (nev_max 16, tau automatic):

* the device's Lanczos estimate of kappa(M^{-1} C) (from the CG coefficients of a solve
  to 1e-10) stays below Theorem 2.6's bound (k_c + 1)(2 + (2 k_c + 1) k_m / tau), with
  k_c (greedy colouring) and k_m (row multiplicity, Lemma 3.1) computed by the oracle
  from the index sets and tau the threshold the device used;
* the two-level iteration counts stay within a factor 1.5 of each other, while the
  one-level counts grow by more than that.
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


@pytest.fixture(scope="module")
def grid():
    m, n, rp, c, v, b, _ = make_grid_ls(128, 128, 4, 8, 3, 0, zero_sum=True)
    return m, n, rp, c, v, b, O.schwarz.as_csr(m, n, rp, c, v)


def test_bound_and_flat_iterations(grid):
    m, n, rp, c, v, b, A = grid
    two, one = [], []
    for blk in (64, 32, 16):
        part = block_partition(128, 128, blk, blk)
        N = int(part.max()) + 1
        S = L.Solver(m, n, rp, c, v, part, N, nev_max=16)
        x, info = S.solve(b, rtol=1e-10)
        sets = O.index_sets(A, part, N)
        kc, km = O.colouring_kc(A, sets), O.multiplicity_km(A, sets)
        bound = O.theorem26_bound(kc, km, info["tau_used"])
        assert 1.0 <= info["kappa_lanczos"] <= bound, (N, info["kappa_lanczos"], bound)
        two.append(info["iters"])
        S.close()
        S1 = L.Solver(m, n, rp, c, v, part, N, coarse=0, nev_max=0, maxit=5000)
        _, i1 = S1.solve(b, rtol=1e-10)
        one.append(i1["iters"])
        S1.close()
        print(f"N={N}: kappa {info['kappa_lanczos']:.2f} <= bound {bound:.1f} (kc={kc}, km={km}, "
              f"tau={info['tau_used']:.3f}); two-level {info['iters']}, one-level {i1['iters']} iterations")
    assert max(two) <= 1.5 * min(two)
    assert one[-1] > 1.5 * one[0]
    assert min(one) > max(two)
