"""Parity of RAS with the deflated second level (Section 2: Q + M_RAS (I - CQ), option
variant = 2) and of restarted GMRES (option solver = 2), the paper's pairing for the
nonsymmetric variant, with the oracle; FP64 factors: the operator (<= 1e-9 relative),
six fixed GMRES steps (<= 1e-10), converged solves (iterations +-1) with the deflated
and the additive operators; the mixed forms meet the tolerance; a symmetric-only solver
with the deflated variant is rejected."""
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


def test_deflated_apply(case):
    S = _solver(case, variant=2, solver=2)
    r = np.random.default_rng(3).standard_normal(case["n"])
    ref = case["M"].apply_deflated(case["A"], r)
    assert rel(S.apply_preconditioner(r, 0).cpu().numpy(), ref) < 1e-9
    S.close()


def test_gmres_fixed_iterations(case):
    S = _solver(case, variant=2, solver=2, fixed_iters=6)
    x, _ = S.solve(case["b"], rtol=1e-8)
    xo, _ = O.fgmres(case["A"], case["b"], lambda r: case["M"].apply_deflated(case["A"], r), fixed_iters=6)
    assert rel(x.cpu().numpy(), xo) < 1e-10
    S.close()


@pytest.mark.parametrize("variant", [2, 0])
def test_gmres_converged(case, variant):
    S = _solver(case, variant=variant, solver=2)
    x, info = S.solve(case["b"], rtol=1e-10)
    M, A = case["M"], case["A"]
    apply = (lambda r: M.apply_deflated(A, r)) if variant == 2 else M.apply
    xo, io = O.fgmres(A, case["b"], apply, rtol=1e-10)
    assert info["relres_true"] <= 1e-10
    assert abs(info["iters"] - io["iters"]) <= 1
    assert rel(x.cpu().numpy(), xo) < 1e-7
    print(f"GMRES ({'deflated RAS' if variant == 2 else 'additive'}): {info['iters']} iterations")
    S.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_gmres_mixed_forms(case, prec):
    S = _solver(case, variant=2, solver=2, factor_prec=prec)
    x, info = S.solve(case["b"], rtol=1e-8)
    assert info["relres_true"] <= 1e-8
    S.close()


def test_deflated_needs_gmres(case):
    with pytest.raises(L.LSError) as ex:
        _solver(case, variant=2, solver=0)
    assert ex.value.status == L.LS_ERR_INVALID
