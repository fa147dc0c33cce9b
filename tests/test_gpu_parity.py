"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP64 form): the library and the oracle compute the same operators in a
different summation order, so products and preconditioner applications agree to a
few ulps times the condition of the operation: 1e-12 relative for A^T A p and the
local solves, 1e-9 for the full two-level apply and 1e-10 for PCG iterates (the
eigen-subspaces enter through Lanczos on the device and dense eigh in the oracle;
their difference is bounded by eig_tol / (relative spectral gap)).  Integer work
(index sets, coarse dimensions) is compared bit-exactly.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2107_09006_gb300 as L  # noqa: E402
import oracle as O  # noqa: E402
from workloads import (config_tiny, make_grid_ls, block_partition, strip_partition,  # noqa: E402
                       paper_example, csr_from_dense, bisection_partition)


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class Case:
    def __init__(self, name, m, n, rp, c, v, b, part, N, nev=16, tau=0.0):
        self.name, self.m, self.n, self.rp, self.c, self.v, self.b, self.part, self.N = name, m, n, rp, c, v, b, part, N
        self.nev, self.tau = nev, tau
        self.A = O.schwarz.as_csr(m, n, rp, c, v)
        self._M = None

    def solver(self, **kw):
        opts = dict(nev_max=self.nev, tau=self.tau)
        opts.update(kw)
        return L.Solver(self.m, self.n, self.rp, self.c, self.v, self.part, self.N, **opts)

    def oracle(self, coarse=True):
        key = (coarse, self.N, self.tau)
        if self._M is None or self._M[0] != key:
            self._M = (key, O.build_two_level(self.A, self.part, self.N, tau=self.tau, nev_max=self.nev,
                                              coarse=coarse))
        return self._M[1]


def _tiny():
    P = config_tiny()
    return Case("tiny", P.m, P.n, P.row_ptr, P.col, P.val, P.b, P.part, P.nparts)


def _mid():
    # several 32-row tiles per subdomain and a ragged last tile (n_i not a multiple of 32)
    m, n, rp, c, v, b, _ = make_grid_ls(96, 96, 4, 8, 3, 0)
    return Case("grid96-N9", m, n, rp, c, v, b, block_partition(96, 96, 32, 32), 9)


def _uneven():
    m, n, rp, c, v, b, _ = make_grid_ls(60, 52, 4, 6, 2, 5)
    part = bisection_partition(60, 52, 700, 9)
    return Case("bisect-uneven", m, n, rp, c, v, b, part, int(part.max()) + 1, nev=8)


def _example():
    A, part = paper_example()
    rp, c, v = csr_from_dense(A)
    return Case("paper-example", 5, 4, rp, c, v, np.arange(1.0, 6.0), part, 2, nev=2, tau=0.6)


CASES = {"tiny": _tiny, "mid": _mid, "uneven": _uneven, "example": _example}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    return CASES[request.param]()


def test_index_sets_bit_exact(case):
    S = case.solver(coarse=0)
    M = O.index_sets(case.A, case.part, case.N)
    for i in range(case.N):
        assert np.array_equal(S.omega(i), M.Om[i])
        assert np.array_equal(S.xi(i), M.Xi[i])
    S.close()


def test_normal_product(case):
    S = case.solver(coarse=0)
    p = np.random.default_rng(1).standard_normal(case.n)
    w = S.apply_normal(p).cpu().numpy()
    assert rel(w, case.A.T @ (case.A @ p)) < 1e-13
    S.close()


@pytest.mark.parametrize("config", [1, 2])
def test_one_level_apply(case, config):
    """Both configurations of the local solve (option local_config: 256 threads with 16 KB
    stages, 512 threads with 32 KB stages)."""
    S = case.solver(coarse=0, local_config=config)
    assert S.info()["local_config"] == config
    M = case.oracle(coarse=False)
    r = np.random.default_rng(2).standard_normal(case.n)
    assert rel(S.apply_preconditioner(r, 1).cpu().numpy(), M.apply_local(r)) < 1e-12
    S.close()


def test_eigenvalues_and_coarse_dimension(case):
    S = case.solver()
    M = case.oracle()
    for i in range(case.N):
        lg = S.eigvals(i)
        lo = M.lams[i][: len(lg)]
        assert np.max(np.abs(lg - lo)) <= 1e-10 * max(1.0, np.abs(lo).max())
    assert S.sizes()[:, 3].tolist() == list(M.ks)
    assert S.info()["n0"] == M.n0
    S.close()


def test_two_level_apply(case):
    S = case.solver()
    M = case.oracle()
    r = np.random.default_rng(3).standard_normal(case.n)
    assert rel(S.apply_preconditioner(r, 0).cpu().numpy(), M.apply(r)) < 1e-9
    assert rel(S.apply_preconditioner(r, 2).cpu().numpy(), M.apply_coarse(r)) < 1e-8
    S.close()


def test_coarse_span_matches(case):
    """The device coarse basis spans the oracle's (compared through projectors)."""
    S = case.solver()
    M = case.oracle()
    Rg = M.R0T.toarray()
    if Rg.shape[1] == 0:
        pytest.skip("empty coarse space")
    Zd = [S.zbar(i) for i in range(case.N)]
    Rd = np.zeros_like(Rg)
    off = 0
    for i, Z in enumerate(Zd):
        k = Z.shape[0]
        Rd[M.S.OI[i], off:off + k] = Z.T
        off += k
    Qg, _ = np.linalg.qr(Rg)
    Qd, _ = np.linalg.qr(Rd)
    # largest principal angle between the two spans: sin = sqrt(1 - sigma_min(Qg^T Qd)^2)
    smin = np.linalg.svd(Qg.T @ Qd, compute_uv=False).min()
    assert np.sqrt(max(0.0, 1.0 - smin ** 2)) < 1e-7
    S.close()


def test_split_local_solve(case):
    """Local-solve configuration 3 (FP32 factors; each subdomain split over a cluster of
    two CTAs that exchange partial sums and solution blocks through distributed shared
    memory; the paper example and the tiny case have subdomains of one or two block
    rows, in which the second CTA owns no chunk): the one-level apply against the oracle
    within the FP32 tolerance of the other configurations, against configuration 1 to
    FP32 rounding, and a converged solve."""
    M = case.oracle(coarse=False)
    r = np.random.default_rng(2).standard_normal(case.n)
    S = case.solver(coarse=0, factor_prec="f32", local_config=3)
    assert S.info()["local_config"] == 3
    z3 = S.apply_preconditioner(r, 1).cpu().numpy()
    S.close()
    S = case.solver(coarse=0, factor_prec="f32", local_config=1)
    z1 = S.apply_preconditioner(r, 1).cpu().numpy()
    S.close()
    exact = M.apply_local(r)
    assert rel(z3, exact) < 1e-5 and rel(z3, z1) < 1e-5
    S = case.solver(factor_prec="f32", local_config=3)
    x, info = S.solve(case.b, rtol=1e-8)
    assert info["relres_true"] <= 1e-8
    S.close()


@pytest.mark.parametrize("config", [1, 2])
def test_pcg_fixed_iterations(case, config):
    S = case.solver(fixed_iters=6, local_config=config)
    M = case.oracle()
    x, _ = S.solve(case.b, rtol=1e-8)
    xo, _ = O.pcg(case.A, case.b, M.apply, fixed_iters=6)
    assert rel(x.cpu().numpy(), xo) < 1e-10
    S.close()


def test_pcg_converged(case):
    S = case.solver()
    M = case.oracle()
    x, info = S.solve(case.b, rtol=1e-8)
    xo, io = O.pcg(case.A, case.b, M.apply, rtol=1e-8)
    assert info["relres_true"] <= 1e-8
    assert abs(info["iters"] - io["iters"]) <= 1
    x13, i13 = S.solve(case.b, rtol=1e-13)
    xo13, _ = O.pcg(case.A, case.b, M.apply, rtol=1e-13)
    assert rel(x13.cpu().numpy(), xo13) < 1e-10
    if i13["restarts"] == 0 and case.n > 10:
        assert abs(i13["kappa_lanczos"] - O.lanczos_kappa(*_coeffs(case, M))) < 1e-6 * i13["kappa_lanczos"]
    S.close()


def _coeffs(case, M):
    _, io = O.pcg(case.A, case.b, M.apply, rtol=1e-13)
    return io["alphas"], io["betas"]


@pytest.mark.parametrize("prec,tol", [("f32", 1e-8), ("bf16", 1e-8)])
def test_mixed_forms_meet_tolerance(prec, tol):
    """The mixed forms reach the true-residual test, and their error against the FP64
    solution (oracle PCG to 1e-13) is at most 10x the error of the oracle's own FP64 PCG
    stopped at the same tolerance: the low-precision local factors cost no accuracy
    beyond what the stopping test allows."""
    c = _mid()
    S = c.solver(factor_prec=prec)
    x, info = S.solve(c.b, rtol=tol)
    assert info["relres_true"] <= tol
    M = c.oracle()
    xo, _ = O.pcg(c.A, c.b, M.apply, rtol=1e-13)
    xt, _ = O.pcg(c.A, c.b, M.apply, rtol=tol)
    e_mixed, e_fp64 = rel(x.cpu().numpy(), xo), rel(xt, xo)
    print(f"{prec}: error {e_mixed:.2e} against the FP64 oracle's {e_fp64:.2e} at rtol {tol:g}")
    assert e_mixed <= 10 * e_fp64
    S.close()


def test_one_subdomain_exact():
    c = _tiny()
    c.part = np.zeros(c.n, np.int32)
    c.N = 1
    c.tau = 0.6
    S = c.solver()
    assert S.info()["n0"] == 0
    x, info = S.solve(c.b, rtol=1e-8)
    assert info["iters"] <= 3
    S.close()


def test_backward_against_dense_gradient():
    c = _tiny()
    S = c.solver()
    x, _ = S.solve(c.b, rtol=1e-13)
    xs = np.random.default_rng(7).standard_normal(c.n)
    gx = 2 * (x.cpu().numpy() - xs)
    gb, gv, _ = S.backward(c.b, x, gx, rtol=1e-13)
    Ad = c.A.toarray()
    C = Ad.T @ Ad
    xd = np.linalg.solve(C, Ad.T @ c.b)
    gbo, gvo, _ = O.adjoint_gradient(c.A, c.b, xd, 2 * (xd - xs), lambda g: np.linalg.solve(C, g))
    assert rel(gb.cpu().numpy(), gbo) < 1e-9
    assert rel(gv.cpu().numpy(), gvo) < 1e-9
    S.close()


def test_errors_are_reported():
    c = _tiny()
    with pytest.raises(L.LSError) as e:
        L.Solver(c.m, c.n, c.rp, c.c, c.v, np.full(c.n, 99, np.int32), c.N)
    assert e.value.status == L.LS_ERR_INVALID
    bad = c.c.copy()
    bad[1], bad[2] = bad[2], bad[1]  # unsorted row
    with pytest.raises(L.LSError) as e:
        L.Solver(c.m, c.n, c.rp, bad, c.v, c.part, c.N)
    assert e.value.status == L.LS_ERR_INVALID
    v = c.v.copy()
    v[3] = np.nan
    with pytest.raises(L.LSError) as e:
        L.Solver(c.m, c.n, c.rp, c.c, v, c.part, c.N)
    assert e.value.status == L.LS_ERR_NONFINITE
    S = c.solver(maxit=2)
    x, info = S.solve(c.b, rtol=1e-12, raise_on_fail=False)
    assert info["status"] == L.LS_ERR_NOT_CONVERGED and info["iters"] == 2
    S.close()


def test_tau_argument_selects_like_oracle():
    """ls_setup's threshold argument (Algorithm 1's input tau): with 1/tau placed in a gap
    of the local spectra, every subdomain keeps exactly the oracle's vectors."""
    c = _mid()
    M0 = c.oracle()
    lam = np.sort(np.concatenate([np.asarray(l[: c.nev + 1]) for l in M0.lams]))[::-1]
    lam = lam[(lam > 1.05) & (lam < lam[0])]
    gaps = lam[:-1] / lam[1:]
    j = int(np.argmax(gaps[: max(1, len(gaps) // 2)]))  # a wide gap among the larger eigenvalues
    thr = float(np.sqrt(lam[j] * lam[j + 1]))
    tau = 1.0 / thr
    M = O.build_two_level(c.A, c.part, c.N, tau=tau, nev_max=c.nev)
    S = c.solver(tau=tau)
    assert S.sizes()[:, 3].tolist() == list(M.ks)
    assert S.info()["n0"] == M.n0 and 0 < M.n0
    assert abs(S.info()["tau_used"] - tau) <= 1e-15 * tau
    r = np.random.default_rng(8).standard_normal(c.n)
    assert rel(S.apply_preconditioner(r, 0).cpu().numpy(), M.apply(r)) < 1e-9
    S.close()
    for bad, status in ((1.0, L.LS_ERR_UNSUPPORTED), (float("nan"), L.LS_ERR_INVALID)):
        with pytest.raises(L.LSError) as e:
            c.solver(tau=bad)
        assert e.value.status == status


def test_solve_orders_against_caller_stream():
    """ls_solve(..., stream): the solve starts after the work queued on the caller's
    stream (here b is written there behind a ~20 ms device sleep, without any host
    synchronisation) and the caller's later work sees x; the same for ls_backward."""
    c = _tiny()
    S = c.solver()
    xo, _ = S.solve(c.b, rtol=1e-10)
    side = torch.cuda.Stream()
    b_src = torch.as_tensor(c.b, device="cuda")
    torch.cuda.synchronize()
    b = torch.zeros(c.m, dtype=torch.float64, device="cuda")
    x = torch.zeros(c.n, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(side):
        torch.cuda._sleep(40_000_000)
        b.copy_(b_src)
        L.ls_solve(S.h, b, 1, 1e-10, x, stream=side.cuda_stream)
        x2 = x.clone()  # queued on the caller's stream after the call
    side.synchronize()
    assert rel(x2.cpu().numpy(), xo.cpu().numpy()) < 1e-12
    g = torch.zeros(c.n, dtype=torch.float64, device="cuda")
    g_src = torch.as_tensor(np.random.default_rng(9).standard_normal(c.n), device="cuda")
    gb_ref, _, _ = S.backward(c.b, xo, g_src, rtol=1e-10)
    gb = torch.zeros(c.m, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        torch.cuda._sleep(40_000_000)
        g.copy_(g_src)
        L.ls_backward(S.h, b, x, g, 1, 1e-10, gb, None, stream=side.cuda_stream)
        gb2 = gb.clone()
    side.synchronize()
    assert rel(gb2.cpu().numpy(), gb_ref.cpu().numpy()) < 1e-12
    S.close()


def test_device_loop_matches_host_loop():
    """The PCG loop run on the device (a conditional graph node, one host wait per pass)
    gives the same iterates, bit for bit, as the host-driven loop (one wait per
    iteration): the same kernels in the same order, with deterministic reductions.  The
    sparse-product kernel is fixed (option spmv) so that the handles do not each pick
    their own by timing.  With kernel timing on, every iteration's local solve and
    products are timed."""
    c = _mid()
    res = {}
    for name, kw in (("host", dict(use_graph=0)), ("device", {}), ("device-timed", dict(time_kernels=1))):
        kw = dict(kw, spmv=2)
        for prec in ("f64", "f32"):
            S = c.solver(factor_prec=prec, **kw)
            x, info = S.solve(c.b, rtol=1e-10)
            S2 = c.solver(factor_prec=prec, fixed_iters=7, **kw)
            x7, i7 = S2.solve(c.b, rtol=1e-8)
            res[name, prec] = (x.cpu().numpy(), info, x7.cpu().numpy(), i7)
            S.close()
            S2.close()
    for prec in ("f64", "f32"):
        xh, ih, x7h, i7h = res["host", prec]
        for name in ("device", "device-timed"):
            xd, idv, x7d, i7d = res[name, prec]
            assert np.array_equal(xd, xh) and idv["iters"] == ih["iters"], (name, prec)
            assert np.array_equal(x7d, x7h) and i7d["iters"] == i7h["iters"] == 7, (name, prec)
            assert idv["relres_true"] <= 1e-10
        it = res["device-timed", prec][1]
        assert it["ms_local"] > 0 and it["ms_spmv"] > 0 and it["ms_iter"] >= it["ms_local"] + it["ms_spmv"]
        assert it["local_launches"] == it["iters"] + 1 + it["restarts"]
