"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle through a route that does not reuse the oracle's own
formula: the worked example printed in Section 3, exact rational arithmetic,
principal angles, dense least squares, dense eigenvalues, brute force on tiny
inputs and finite differences.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sl
import scipy.sparse as sp

import oracle as O
from oracle.schwarz import as_csr, restriction, partition_of_unity
from workloads import paper_example, csr_from_dense, make_grid_ls, strip_partition, block_partition

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _example():
    A, part = paper_example()
    rp, c, v = csr_from_dense(A)
    return A, as_csr(5, 4, rp, c, v), part


# --------------------------------------------------------------------------- P1
def test_worked_example_index_sets():
    """Section 3 worked example: Xi_i, Omega_Gamma_i, R_i and D_i exactly as printed."""
    g = json.load(open(os.path.join(GOLD, "paper_example.json")))
    Ad, A, part = _example()
    assert np.array_equal(Ad, np.array(g["A"], float))
    S = O.index_sets(A, part, 2)
    for i in range(2):
        assert (S.OI[i] + 1).tolist() == g["Omega_I"][i]
        assert (S.Xi[i] + 1).tolist() == g["Xi"][i]
        assert (S.OG[i] + 1).tolist() == g["Omega_Gamma"][i]
        xi_c = sorted(set(range(1, 6)) - set((S.Xi[i] + 1).tolist()))
        assert xi_c == g["Xi_c"][i]
        om_c = sorted(set(range(1, 5)) - set((S.Om[i] + 1).tolist()))
        assert om_c == g["Omega_c"][i]
        assert np.array_equal(restriction(S.Om[i], 4), np.array(g["R"][i], float))
        assert np.array_equal(partition_of_unity(len(S.OI[i]), len(S.Om[i])), np.array(g["D"][i], float))
        # the permuted matrix A([Xi, Xi_c], [Omega_I, Omega_Gamma, Omega_c]) of the example
        rows = np.concatenate([S.Xi[i], np.array(g["Xi_c"][i]) - 1])
        cols = np.concatenate([S.Om[i], np.array(g["Omega_c"][i]) - 1])
        assert np.array_equal(Ad[np.ix_(rows, cols)], np.array(g[f"permuted_A_{i + 1}"], float))


def test_worked_example_local_matrices():
    g = json.load(open(os.path.join(GOLD, "paper_example.json")))["hand_derived"]
    _, A, part = _example()
    S = O.index_sets(A, part, 2)
    for i, (kc, kt) in enumerate([("C11", "Ct11"), ("C22", "Ct22")]):
        Cii, Ct = O.local_matrices(A, S, i, 0.0)
        assert np.array_equal(Cii, np.array(g[kc], float))
        assert np.array_equal(Ct, np.array(g[kt], float))


def test_worked_example_gevp_exact():
    """The pencil D C_ii D - lambda C~_ii, solved exactly in rational arithmetic, against
    the oracle's shifted FP64 eigenvalues; at tau = 0.6 only subdomain 2 keeps a vector."""
    sympy = pytest.importorskip("sympy")
    _, A, part = _example()
    S = O.index_sets(A, part, 2)
    lam_sym = sympy.Symbol("lam")
    for i in range(2):
        Cii, Ct = O.local_matrices(A, S, i, 0.0)
        nI = len(S.OI[i])
        d = np.diag(partition_of_unity(nI, 3))
        DCD = sympy.Matrix((d @ Cii @ d).astype(int).tolist())
        Ctm = sympy.Matrix(Ct.astype(int).tolist())
        poly = sympy.Poly((DCD - lam_sym * Ctm).det(), lam_sym)
        roots = sorted(float(r) for r in sympy.roots(poly, multiple=True)) if poly.degree() > 0 else []
        exact = sorted(roots + [0.0] * (3 - len(roots)))  # zero roots dropped by degree loss
        lam, _ = O.gevp_local(Cii, Ct, nI, s_rel=1e-8)
        assert np.allclose(sorted(lam), exact, rtol=1e-6, atol=1e-7)
    lam1, _ = O.gevp_local(*O.local_matrices(A, S, 0, 0.0), 2)
    lam2, _ = O.gevp_local(*O.local_matrices(A, S, 1, 0.0), 2)
    assert abs(lam1[0] / (13 / 9) - 1) < 2e-6 and abs(lam2[0] / (213 / 100) - 1) < 2e-6
    M = O.build_two_level(A, part, 2, tau=0.6, nev_max=300, delta_rel=0.0)
    assert M.ks == [0, 1]


# --------------------------------------------------------------------------- P2
def _rand_subdomain(seed=3, m=40, n=16):
    rng = np.random.default_rng(seed)
    Ad = np.where(rng.random((m, n)) < 0.25, rng.standard_normal((m, n)), 0.0)
    Ad[np.arange(n), np.arange(n)] += 1.0  # full column rank
    part = (np.arange(n) >= n // 2).astype(np.int32)
    rp, c, v = csr_from_dense(Ad)
    return as_csr(m, n, rp, c, v), part


@pytest.mark.parametrize("case", ["random", "tiny"])
def test_gevp_principal_angles(case, tiny):
    """For s -> 0 the nonzero eigenvalues of the local pencil are 1/sin^2(theta_k) for the
    principal angles between range A(Xi, Omega_I) and range A(Xi, Omega_Gamma), padded
    with ones (the interior block of C~_ii equals that of C_ii)."""
    if case == "random":
        A, part = _rand_subdomain()
        N = 2
    else:
        A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
        part, N = tiny.part, 3  # first three strips only
    S = O.index_sets(A, part, int(part.max()) + 1)
    for i in range(N):
        Cii, Ct = O.local_matrices(A, S, i, 0.0)
        nI = len(S.OI[i])
        lam, _ = O.gevp_local(Cii, Ct, nI, s_rel=1e-13)
        AI = A[S.Xi[i], :][:, S.OI[i]].toarray()
        AG = A[S.Xi[i], :][:, S.OG[i]].toarray()
        th = sl.subspace_angles(AI, AG) if AG.shape[1] else np.zeros(0)
        ref = np.concatenate([1.0 / np.sin(th) ** 2, np.ones(nI - len(th))])
        ref = np.sort(ref)[::-1]
        assert np.allclose(lam[:nI], ref, rtol=1e-6)
        assert np.all(np.abs(lam[nI:]) < 1e-6)  # the Gamma-only directions: lambda = 0
        assert lam[nI - 1] >= 1 - 1e-6  # every nonzero eigenvalue is >= 1


# --------------------------------------------------------------------------- P3
@pytest.mark.parametrize("N,blk", [(8, 4), (4, 8)])
def test_pcg_matches_dense_lstsq(N, blk):
    m, n, rp, c, v, b, _ = make_grid_ls(32, 32, 4, 4, 2, 0)
    A = as_csr(m, n, rp, c, v)
    part = strip_partition(32, 32, blk)
    M = O.build_two_level(A, part, N, tau=0.0, nev_max=16)
    x, info = O.pcg(A, b, M.apply, rtol=1e-14)
    xl = np.linalg.lstsq(A.toarray(), b, rcond=None)[0]
    kappa = np.linalg.cond(A.toarray()) ** 2
    assert np.linalg.norm(x - xl) / np.linalg.norm(xl) <= kappa * 1e-14
    assert info["relres_true"] <= 1e-14


# --------------------------------------------------------------------------- P4, P5
def test_splitting_inequality_and_km(tiny):
    """0 <= u^T C~_i u <= u^T C u (Section 2.1, eq. (3.2)) and sum_i C~_i <= k_m C with
    k_m = max_j m_j (Lemma 3.1), checked with dense eigenvalues."""
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    S = O.index_sets(A, tiny.part, tiny.nparts)
    C = (A.T @ A).toarray()
    nC = np.linalg.norm(C, 2)
    Ssum = np.zeros_like(C)
    for i in range(S.N):
        _, Ct = O.local_matrices(A, S, i, 0.0)
        R = restriction(S.Om[i], tiny.n)
        Cti = R.T @ Ct @ R
        assert np.linalg.eigvalsh(Cti).min() >= -1e-12 * nC
        assert np.linalg.eigvalsh(C - Cti).min() >= -1e-12 * nC
        Ssum += Cti
    km = O.multiplicity_km(A, S)
    # brute-force m_j by scanning every row against every interior set
    Ad = A.toarray()
    mj = [sum(1 for i in range(S.N) if np.any(Ad[j, S.OI[i]] != 0)) for j in range(tiny.m)]
    assert km == max(mj)
    top = sl.eigh(Ssum, C, eigvals_only=True)[-1]
    assert top <= km * (1 + 1e-10)


# --------------------------------------------------------------------------- P6
def test_one_subdomain_is_exact_solve(tiny):
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    part = np.zeros(tiny.n, np.int32)
    M = O.build_two_level(A, part, 1, tau=0.6, nev_max=16)
    assert M.n0 == 0 and len(M.S.OG[0]) == 0
    C = (A.T @ A).toarray()
    r = np.random.default_rng(1).standard_normal(tiny.n)
    z = M.apply(r)
    assert np.allclose(z, np.linalg.solve(C + M.delta * np.eye(tiny.n), r), rtol=1e-9)
    x, info = O.pcg(A, tiny.b, M.apply, rtol=1e-8)
    assert info["iters"] <= 3
    M0 = O.build_two_level(A, part, 1, tau=0.6, nev_max=16, delta_rel=0.0)
    x0, info0 = O.pcg(A, tiny.b, M0.apply, rtol=1e-8)
    assert info0["iters"] == 1


# --------------------------------------------------------------------------- projector invariants
def test_coarse_and_local_terms_are_c_projectors(tiny):
    """R_0^T C_00^{-1} R_0 (C + delta I) and R_i^T C_ii^{-1} R_i (C + delta I) are the
    (C + delta I)-orthogonal projectors onto range R_0^T and range R_i^T."""
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    M = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16)
    Cd = (A.T @ A).toarray() + M.delta * np.eye(tiny.n)
    R0T = M.R0T.toarray()
    P0 = np.column_stack([M.apply_coarse(Cd[:, j]) for j in range(tiny.n)])
    assert np.allclose(P0 @ R0T, R0T, atol=1e-9 * np.abs(R0T).max())
    assert np.allclose(P0 @ P0, P0, atol=1e-8)
    i = 2
    R = restriction(M.S.Om[i], tiny.n)
    Pi = R.T @ sl.cho_solve(M.local[i][1], R @ Cd)
    assert np.allclose(Pi @ R.T, R.T, atol=1e-9)
    # M^{-1} is the sum of the two terms applied to the same vector
    r = np.random.default_rng(2).standard_normal(tiny.n)
    assert np.allclose(M.apply(r), M.apply_local(r) + M.apply_coarse(r))


# --------------------------------------------------------------------------- P7
def test_condition_bound_theorem26(tiny):
    """kappa(M_additive^{-1} C) from dense eigenvalues stays under Theorem 2.6's bound
    (and under the looser restatement of Section 3.2); the CG-Lanczos estimate agrees."""
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    M = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16)
    C = (A.T @ A).toarray()
    Minv = np.column_stack([M.apply(e) for e in np.eye(tiny.n)])
    Minv = 0.5 * (Minv + Minv.T)
    ev = sl.eigh(C, np.linalg.inv(Minv), eigvals_only=True)
    kappa = ev[-1] / ev[0]
    S = M.S
    km, kc = O.multiplicity_km(A, S), O.colouring_kc(A, S)
    assert kappa <= O.theorem26_bound(kc, km, M.tau)
    assert kappa <= O.theorem26_bound(kc, km, M.tau, "sec32")
    x, info = O.pcg(A, tiny.b, M.apply, rtol=1e-14)
    kl = O.lanczos_kappa(info["alphas"], info["betas"])
    assert abs(kl - kappa) / kappa < 0.02
    # the one-level operator has a larger condition number than the bound needs; the
    # two-level one has lambda_min bounded below by 1/(2 + (2kc+1) km / tau) (Lemma 2.5)
    assert ev[0] >= 1.0 / (2 + (2 * kc + 1) * km / M.tau)
    assert ev[-1] <= kc + 1 + 1e-9


# --------------------------------------------------------------------------- balanced variant
def test_balanced_variant(tiny):
    """The balanced two-level operator of Section 2, Q + (I - CQ)^T M_1 (I - CQ), pinned by
    what its definition implies (built with delta = 0 so that C_00 = R_0 C R_0^T exactly):
    it is symmetric, it inverts C on the coarse space (M_bal C R_0^T = R_0^T, so M_bal C
    has the eigenvalue 1 with multiplicity n_0), it conditions C better than the additive
    operator (the paper's reason to use it), and PCG with it reaches the least-squares
    solution."""
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    M = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16, delta_rel=0.0)
    C = (A.T @ A).toarray()
    R0T = M.R0T.toarray()
    for j in range(0, R0T.shape[1], 7):
        z = M.apply_balanced(A, C @ R0T[:, j])
        assert np.linalg.norm(z - R0T[:, j]) <= 1e-10 * np.linalg.norm(R0T[:, j])
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal(tiny.n), rng.standard_normal(tiny.n)
    assert abs(M.apply_balanced(A, x) @ y - x @ M.apply_balanced(A, y)) <= 1e-12 * abs(x @ M.apply_balanced(A, y))
    Mb = np.column_stack([M.apply_balanced(A, e) for e in np.eye(tiny.n)])
    Ma = np.column_stack([M.apply(e) for e in np.eye(tiny.n)])
    eb = sl.eigh(C, np.linalg.inv(0.5 * (Mb + Mb.T)), eigvals_only=True)
    ea = sl.eigh(C, np.linalg.inv(0.5 * (Ma + Ma.T)), eigvals_only=True)
    assert eb[0] > 0 and int(np.sum(np.abs(eb - 1.0) < 1e-8)) == M.n0
    assert eb[-1] / eb[0] < ea[-1] / ea[0]
    xb, ib = O.pcg(A, tiny.b, lambda r: M.apply_balanced(A, r), rtol=1e-12)
    xl = np.linalg.lstsq(A.toarray(), tiny.b, rcond=None)[0]
    assert np.linalg.norm(xb - xl) <= 1e-8 * np.linalg.norm(xl)
    _, ia = O.pcg(A, tiny.b, M.apply, rtol=1e-12)
    assert ib["iters"] < ia["iters"]


# --------------------------------------------------------------------------- preconditioned LSQR
def test_preconditioned_lsqr(tiny):
    """The LSQR outer solver: with M = I it is textbook LSQR (scipy's iterates); with the
    two-level operator its iterates are PCG's on the normal equations (both minimise
    ||b - A x|| over the same Krylov space), its bidiagonal gives PCG's Lanczos kappa,
    and it reaches the least-squares solution."""
    import scipy.sparse.linalg as sla
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    for k in (1, 3, 6):
        x, _ = O.preconditioned_lsqr(A, tiny.b, lambda v: v, fixed_iters=k)
        xs = sla.lsqr(A, tiny.b, atol=0, btol=0, conlim=0, iter_lim=k)[0]
        assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)
    M = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16)
    for k in (1, 6, 10):
        xl, _ = O.preconditioned_lsqr(A, tiny.b, M.apply, fixed_iters=k)
        xp, _ = O.pcg(A, tiny.b, M.apply, fixed_iters=k)
        assert np.linalg.norm(xl - xp) <= 1e-10 * np.linalg.norm(xp)
    xl, il = O.preconditioned_lsqr(A, tiny.b, M.apply, rtol=1e-10)
    _, ip = O.pcg(A, tiny.b, M.apply, rtol=1e-10)
    assert il["relres_true"] <= 1e-10 and abs(il["iters"] - ip["iters"]) <= 1
    xd = np.linalg.lstsq(A.toarray(), tiny.b, rcond=None)[0]
    assert np.linalg.norm(xl - xd) <= 1e-6 * np.linalg.norm(xd)
    kl, kp = O.lsqr_kappa(il["alphas"], il["betas"]), O.lanczos_kappa(ip["alphas"], ip["betas"])
    assert abs(kl - kp) <= 1e-6 * kp


# --------------------------------------------------------------------------- RAS, deflated, GMRES
def test_ras_deflated_and_fgmres(tiny):
    """RAS (Section 2): the D_i form a partition of unity (sum_i R_i^T D_i R_i = I) and
    with one subdomain RAS is the exact inverse of C + delta I; the deflated operator
    Q + M_RAS (I - CQ) inverts C on the coarse space (delta = 0); GMRES's iterates are
    the minimisers of ||A^T b - C x|| over independently built (preconditioned) Krylov
    bases, and it reaches the least-squares solution."""
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    C = (A.T @ A).toarray()
    g = A.T @ tiny.b
    M = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16)
    cover = np.zeros(tiny.n)
    for i in range(tiny.nparts):
        R = restriction(M.S.Om[i], tiny.n)
        d = np.isin(M.S.Om[i], M.S.OI[i]).astype(float)
        cover += R.T @ d
    assert np.array_equal(cover, np.ones(tiny.n))
    M1 = O.build_two_level(A, np.zeros(tiny.n, np.int32), 1, tau=0.6, nev_max=16)
    r = np.random.default_rng(5).standard_normal(tiny.n)
    assert np.allclose(M1.apply_ras(r), np.linalg.solve(C + M1.delta * np.eye(tiny.n), r), rtol=1e-9)
    M0 = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16, delta_rel=0.0)
    R0T = M0.R0T.toarray()
    for j in range(0, R0T.shape[1], 7):
        z = M0.apply_deflated(A, C @ R0T[:, j])
        assert np.linalg.norm(z - R0T[:, j]) <= 1e-10 * np.linalg.norm(R0T[:, j])
    for apply in (lambda v: v, lambda v: M.apply_deflated(A, v)):
        for k in (1, 3, 5):
            x, _ = O.fgmres(A, tiny.b, apply, fixed_iters=k)
            cols, v = [], g.copy()
            for _ in range(k):
                z = apply(v)
                cols.append(z)
                v = C @ z
            Qk, _ = np.linalg.qr(np.column_stack(cols))
            xk = Qk @ np.linalg.lstsq(C @ Qk, g, rcond=None)[0]
            assert np.linalg.norm(x - xk) <= 1e-10 * np.linalg.norm(xk)
    x, info = O.fgmres(A, tiny.b, lambda v: M.apply_deflated(A, v), rtol=1e-10)
    xl = np.linalg.lstsq(A.toarray(), tiny.b, rcond=None)[0]
    assert info["relres_true"] <= 1e-10 and np.linalg.norm(x - xl) <= 1e-6 * np.linalg.norm(xl)


# --------------------------------------------------------------------------- tau rule
def test_auto_tau_and_cap(tiny):
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    M = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16)
    assert max(M.ks) == 16 and M.n0 == sum(M.ks)
    for lam, k in zip(M.lams, M.ks):
        assert np.all(lam[:k] > M.thr) and (len(lam) <= k or lam[k] <= M.thr)
    M2 = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.6, nev_max=4)
    for lam, k in zip(M2.lams, M2.ks):
        assert k == min(4, int(np.sum(lam > 1 / 0.6)))


# --------------------------------------------------------------------------- flexible PCG
def test_flexible_pcg_equals_pcg_for_fixed_preconditioner(tiny):
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    M = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16)
    x1, _ = O.pcg(A, tiny.b, M.apply, fixed_iters=8)
    x2, _ = O.flexible_pcg(A, tiny.b, M.apply, fixed_iters=8)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-10
    # and a wrong beta (sign flipped) would not: sanity of the comparison's power
    x3, info = O.flexible_pcg(A, tiny.b, M.apply, rtol=1e-8)
    assert info["relres_true"] <= 1e-8


# --------------------------------------------------------------------------- banded mode
def test_banded_mode_matches_dense(tiny):
    A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
    Md = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16)
    Mb = O.build_two_level(A, tiny.part, tiny.nparts, tau=0.0, nev_max=16, mode="banded")
    assert Md.ks == Mb.ks and abs(Md.tau - Mb.tau) < 1e-10 * Md.tau
    r = np.random.default_rng(4).standard_normal(tiny.n)
    assert np.linalg.norm(Md.apply(r) - Mb.apply(r)) <= 1e-9 * np.linalg.norm(Md.apply(r))
    for lb, ld in zip(Mb.lams, Md.lams):
        assert np.allclose(lb[:17], ld[:17], rtol=1e-10)


# --------------------------------------------------------------------------- brute-force index sets
def test_index_sets_brute_force():
    m, n, rp, c, v, b, _ = make_grid_ls(12, 12, 2, 4, 2, 7)
    A = as_csr(m, n, rp, c, v)
    part = block_partition(12, 12, 5, 4)  # ragged blocks
    N = int(part.max()) + 1
    S = O.index_sets(A, part, N)
    Ad = A.toarray() != 0
    for i in range(N):
        OI = [j for j in range(n) if part[j] == i]
        Xi = [r for r in range(m) if any(Ad[r, j] for j in OI)]
        cols = sorted({j for r in Xi for j in range(n) if Ad[r, j]})
        OG = [j for j in cols if part[j] != i]
        assert S.OI[i].tolist() == OI and S.Xi[i].tolist() == Xi and S.OG[i].tolist() == OG
        assert S.Om[i].tolist() == OI + OG


# --------------------------------------------------------------------------- gradient
def test_adjoint_gradient_finite_differences():
    """grad_b = A lambda and grad_A = rho lambda^T - (A lambda) x^T on the pattern, checked
    by central differences of x(A, b) = argmin ||A x - b|| through numpy's lstsq."""
    m, n, rp, c, v, b, _ = make_grid_ls(6, 6, 3, 4, 2, 11)
    A = as_csr(m, n, rp, c, v)
    xs = np.random.default_rng(12).standard_normal(n)

    def loss(vals, bb):
        Ad = as_csr(m, n, rp, c, vals).toarray()
        x = np.linalg.lstsq(Ad, bb, rcond=None)[0]
        return float(np.sum((x - xs) ** 2))

    Ad = A.toarray()
    x = np.linalg.lstsq(Ad, b, rcond=None)[0]
    gbar = 2 * (x - xs)
    C = Ad.T @ Ad
    gb, gv, _ = O.adjoint_gradient(A, b, x, gbar, lambda g: np.linalg.solve(C, g))
    h = 1e-6
    rng = np.random.default_rng(13)
    for k in rng.choice(len(v), 12, replace=False):
        vp, vm = v.copy(), v.copy()
        vp[k] += h
        vm[k] -= h
        fd = (loss(vp, b) - loss(vm, b)) / (2 * h)
        assert abs(fd - gv[k]) <= 1e-6 * max(1.0, abs(fd))
    for k in rng.choice(m, 8, replace=False):
        bp, bm = b.copy(), b.copy()
        bp[k] += h
        bm[k] -= h
        fd = (loss(v, bp) - loss(v, bm)) / (2 * h)
        assert abs(fd - gb[k]) <= 1e-6 * max(1.0, abs(fd))


# --------------------------------------------------------------------------- shifts (Section 4.1.2)
def _hand():
    return json.load(open(os.path.join(GOLD, "paper_example.json")))["hand_derived"]


def test_global_shift_worked_example():
    """delta = 1e-10 ||C||_F with C = A^T A (Section 4.1.2), against ||C||_F^2 = 18592 worked
    out by hand from the printed 5x4 A; delta enters every C_ii (dense and banded modes)
    and nothing else.  ||A||_F (204), the spectral norm of C or a missing square root
    would all fail here."""
    h = _hand()
    Ad, A, part = _example()
    assert np.array_equal(Ad.T @ Ad, np.array(h["C"], float))
    assert float(np.sum(np.array(h["C"], float) ** 2)) == h["C_frob_sq"]
    want = 1e-10 * np.sqrt(h["C_frob_sq"])
    assert abs(O.global_shift(A, 1e-10) / want - 1) < 1e-15
    assert abs(O.global_shift(A, 0.25) / (0.25 * np.sqrt(h["C_frob_sq"])) - 1) < 1e-15
    M = O.build_two_level(A, part, 2, tau=0.6, nev_max=300)
    assert abs(M.delta / want - 1) < 1e-15
    S = O.index_sets(A, part, 2)
    from oracle.schwarz import _local_banded
    for i, (kc, kt) in enumerate([("C11", "Ct11"), ("C22", "Ct22")]):
        Cii, Ct = O.local_matrices(A, S, i, want)
        assert np.allclose(Cii, np.array(h[kc], float) + want * np.eye(3), rtol=0, atol=1e-14)
        assert np.array_equal(Ct, np.array(h[kt], float))  # the splitting carries no delta
        srt, Cb, Ctb, s, _, _ = _local_banded(A, S, i, want, 1e-8)
        perm = [list(S.Om[i]).index(j) for j in srt]  # banded mode: ascending global order
        assert np.allclose(Cb.toarray(), (np.array(h[kc], float) + want * np.eye(3))[np.ix_(perm, perm)],
                           rtol=0, atol=1e-14)


@pytest.mark.parametrize("s_rel", [1e-8, 1e-1])
def test_gevp_shift_worked_example(s_rel):
    """The GEVP shift s_i = s_rel ||C~_ii||_F (Section 4.1.2) with ||C~_11||_F^2 = 1948 and
    ||C~_22||_F^2 = 17044 worked out by hand: the oracle's eigenvalues of
    D C_ii D v = lambda (C~_ii + s_i I) v equal the roots of the exact characteristic
    polynomial of that pencil (sympy, 40 digits).  At s_rel = 0.1 a shift taken with
    another norm would move the eigenvalues by percent; at the paper's 1e-8 by about
    1e-9 relative, still far above the 1e-12 tolerance.  The banded mode computes the
    same s."""
    sympy = pytest.importorskip("sympy")
    h = _hand()
    _, A, part = _example()
    S = O.index_sets(A, part, 2)
    from oracle.schwarz import _local_banded
    lam_sym = sympy.Symbol("lam")
    for i, (kc, kt, kf) in enumerate([("C11", "Ct11", "Ct11_frob_sq"), ("C22", "Ct22", "Ct22_frob_sq")]):
        assert int(np.sum(np.array(h[kt]) ** 2)) == h[kf]
        s = sympy.Float(s_rel, 40) * sympy.sqrt(h[kf])
        d = sympy.diag(1, 1, 0)
        DCD = d * sympy.Matrix(h[kc]) * d
        B = sympy.Matrix(h[kt]) + s * sympy.eye(3)
        poly = sympy.Poly((DCD - lam_sym * B).det(), lam_sym)
        exact = sorted((float(sympy.re(r)) for r in poly.nroots(n=40)), reverse=True)
        exact = exact + [0.0] * (3 - len(exact))
        Cii, Ct = O.local_matrices(A, S, i, 0.0)
        lam, _ = O.gevp_local(Cii, Ct, 2, s_rel=s_rel)
        top = max(abs(x) for x in exact)
        assert np.allclose(lam, exact, rtol=1e-12, atol=1e-12 * top), (lam, exact)
        _, _, _, sb, _, _ = _local_banded(A, S, i, 0.0, s_rel)
        assert abs(sb / float(s) - 1) < 1e-14


def test_select_coarse_kappa_branch():
    """Eq. (3.6): keep lambda > 1/tau, or lambda >= 1/(kappa(C_ii) eps) when that bound is
    the smaller one, largest first and at most nev_max (hand-made spectrum)."""
    lam = np.array([10.0, 5.0, 3.0, 2.0, 0.5])
    V = np.eye(5)
    Z, kept = O.select_coarse(lam, V, 5, tau=0.1, nev_max=10)  # 1/tau = 10: strict, nothing kept
    assert kept.size == 0 and Z.shape == (5, 0)
    kappa = 1.0 / (3.0 * np.finfo(float).eps)  # 1/(kappa eps) = 3 < 10
    Z, kept = O.select_coarse(lam, V, 5, tau=0.1, nev_max=10, kappa_cii=kappa)
    assert kept.tolist() == [10.0, 5.0, 3.0] and np.array_equal(Z, V[:, :3])
    Z, kept = O.select_coarse(lam, V, 3, tau=0.1, nev_max=2, kappa_cii=kappa)
    assert kept.tolist() == [10.0, 5.0] and Z.shape == (3, 2)
    Z, kept = O.select_coarse(lam, V, 5, tau=1 / 2.5, nev_max=10, kappa_cii=1.0)  # bound 1/eps: unused
    assert kept.tolist() == [10.0, 5.0, 3.0]


# --------------------------------------------------------------------------- k_c (Lemma 2.2)
def _subdomain_graph_dense(A, S):
    """i ~ j iff the structural C = |A|^T |A| couples Omega_i and Omega_j (dense check)."""
    B = (A.toarray() != 0).astype(float)
    C = B.T @ B
    return C, [[j for j in range(S.N) if j != i and C[np.ix_(S.Om[i], S.Om[j])].any()] for i in range(S.N)]


def _chromatic_number(adj):
    """Fewest colours of a proper colouring, by backtracking (tiny graphs only)."""
    N = len(adj)
    for k in range(1, N + 1):
        col = [-1] * N

        def place(i):
            if i == N:
                return True
            for c in range(k):
                if all(col[j] != c for j in adj[i] if j < i):
                    col[i] = c
                    if place(i + 1):
                        return True
            col[i] = -1
            return False

        if place(0):
            return k
    return 0


@pytest.mark.parametrize("case", ["tiny", "blocks12_r1", "blocks12_r2"])
def test_colouring_proper_and_minimal(case, tiny):
    """k_c of Lemma 2.2: the oracle's colouring is proper (same-coloured subdomains are
    mutually C-orthogonal, checked on the dense C), so its count bounds k_c from above,
    and here it equals the brute-force chromatic number, so the Theorem 2.6 checks that
    use it are not loosened by an over-count."""
    if case == "tiny":
        A = as_csr(tiny.m, tiny.n, tiny.row_ptr, tiny.col, tiny.val)
        part, N = tiny.part, tiny.nparts
    else:
        r, k = (1, 3) if case == "blocks12_r1" else (2, 4)
        m, n, rp, c, v, _, _ = make_grid_ls(12, 12, 2, k, r, 3)
        A = as_csr(m, n, rp, c, v)
        part, N = block_partition(12, 12, 4, 4), 9
    S = O.index_sets(A, part, N)
    colour = O.subdomain_colouring(A, S)
    C, adj = _subdomain_graph_dense(A, S)
    for i in range(N):
        for j in range(i + 1, N):
            if colour[i] == colour[j]:
                assert not C[np.ix_(S.Om[i], S.Om[j])].any(), (i, j)
    kc = O.colouring_kc(A, S)
    assert kc == max(colour) + 1 == _chromatic_number(adj)


@pytest.mark.parametrize("s,kc_hand", [(2, 3), (3, 2), (4, 2)])
def test_colouring_chain_by_hand(s, kc_hand):
    """A 1-D chain (row r couples columns r and r+1, plus identity rows): C is tridiagonal
    and Omega_i is strip i widened by one column on each side.  Strips of s >= 3 columns
    then touch only their neighbours (a path: two colours); strips of 2 columns also
    touch the strip after next (three colours)."""
    n = 12
    Ad = np.zeros((2 * n - 1, n))
    for r in range(n - 1):
        Ad[r, r], Ad[r, r + 1] = 1.0, 1.0 + 0.5 * r
    Ad[n - 1 + np.arange(n), np.arange(n)] = 1e-2
    rp, c, v = csr_from_dense(Ad)
    A = as_csr(2 * n - 1, n, rp, c, v)
    part = (np.arange(n) // s).astype(np.int32)
    N = int(part.max()) + 1
    S = O.index_sets(A, part, N)
    for i in range(N):
        lo, hi = max(0, s * i - 1), min(n - 1, s * i + s)
        assert sorted(S.Om[i].tolist()) == list(range(lo, hi + 1))
    assert O.colouring_kc(A, S) == kc_hand


def test_theorem26_bound_hand_values():
    """Theorem 2.6's bound (k_c + 1)(2 + (2 k_c + 1) k_m / tau) and its Section 3.2
    restatement (k_c + 1)(2 + 2 (k_c + 1) k_m / tau), evaluated by hand at k_c = 4,
    k_m = 3, tau = 1/2: 5 (2 + 54) = 280 and 5 (2 + 60) = 310."""
    assert O.theorem26_bound(4, 3, 0.5) == 280.0
    assert O.theorem26_bound(4, 3, 0.5, "sec32") == 310.0
    assert O.theorem26_bound(0, 1, 1.0) == 3.0  # one colour: 1 (2 + 1)
