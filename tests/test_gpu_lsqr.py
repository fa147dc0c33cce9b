"""Parity of the preconditioned LSQR outer solver (option solver = 1; the paper's solver,
Section 4.1.3) with the oracle, FP64 factors: six fixed iterations (<= 1e-10 relative,
and equal to the device's PCG iterates: both minimise ||b - A x|| over the same Krylov
space), converged solves (iterations +-1, the bidiagonal's kappa estimate), with the
additive and the balanced second level; the mixed forms meet the tolerance."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2107_09006_gb300 as L  # noqa: E402
import oracle as O  # noqa: E402
from workloads import config_tiny, make_grid_ls, block_partition, bisection_partition  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _tiny():
    P = config_tiny()
    return P.m, P.n, P.row_ptr, P.col, P.val, P.b, P.part, P.nparts, 16


def _mid():
    m, n, rp, c, v, b, _ = make_grid_ls(96, 96, 4, 8, 3, 0)
    return m, n, rp, c, v, b, block_partition(96, 96, 32, 32), 9, 16


def _uneven():
    m, n, rp, c, v, b, _ = make_grid_ls(60, 52, 4, 6, 2, 5)
    part = bisection_partition(60, 52, 700, 9)
    return m, n, rp, c, v, b, part, int(part.max()) + 1, 8


CASES = {"tiny": _tiny, "mid": _mid, "uneven": _uneven}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    m, n, rp, c, v, b, part, N, nev = CASES[request.param]()
    A = O.schwarz.as_csr(m, n, rp, c, v)
    M = O.build_two_level(A, part, N, tau=0.0, nev_max=nev)
    return dict(m=m, n=n, rp=rp, c=c, v=v, b=b, part=part, N=N, nev=nev, A=A, M=M)


def _solver(d, **kw):
    return L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], d["N"], nev_max=d["nev"], **kw)


def test_lsqr_fixed_iterations(case):
    S = _solver(case, solver=1, fixed_iters=6)
    x, _ = S.solve(case["b"], rtol=1e-8)
    xo, _ = O.preconditioned_lsqr(case["A"], case["b"], case["M"].apply, fixed_iters=6)
    assert rel(x.cpu().numpy(), xo) < 1e-10
    P = _solver(case, fixed_iters=6)
    xp, _ = P.solve(case["b"], rtol=1e-8)
    assert rel(x.cpu().numpy(), xp.cpu().numpy()) < 1e-9
    S.close()
    P.close()


@pytest.mark.parametrize("variant", [0, 1])
def test_lsqr_converged(case, variant):
    S = _solver(case, solver=1, variant=variant)
    x, info = S.solve(case["b"], rtol=1e-10)
    M = case["M"]
    apply = M.apply if variant == 0 else (lambda r: M.apply_balanced(case["A"], r))
    xo, io = O.preconditioned_lsqr(case["A"], case["b"], apply, rtol=1e-10)
    assert info["relres_true"] <= 1e-10
    assert abs(info["iters"] - io["iters"]) <= 1
    assert rel(x.cpu().numpy(), xo) < 1e-7
    ko = O.lsqr_kappa(io["alphas"], io["betas"])
    if info["iters"] == io["iters"]:
        assert abs(info["kappa_lanczos"] - ko) <= 1e-6 * ko
    print(f"LSQR ({'balanced' if variant else 'additive'}): {info['iters']} iterations, kappa {info['kappa_lanczos']:.3f}")
    S.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_lsqr_mixed_forms(case, prec):
    S = _solver(case, solver=1, factor_prec=prec)
    x, info = S.solve(case["b"], rtol=1e-8)
    assert info["relres_true"] <= 1e-8
    S.close()


def test_lsqr_rejected_on_block_path(case):
    S = _solver(case, solver=1)
    with pytest.raises(L.LSError) as ex:
        S.solve(np.stack([case["b"], case["b"]]), rtol=1e-8)
    assert ex.value.status == L.LS_ERR_UNSUPPORTED
    S.close()
