"""Plain FP64 restatement of the two-level Schwarz method for sparse normal equations.

Test infrastructure only (see the package docstring).  Every function states
the passage of arXiv 2107.09006 it follows.  Library primitives used as single
steps: scipy.sparse products, scipy.linalg Cholesky / eigh / banded solvers and
ARPACK (``eigsh``) for the banded (large) mode.  There is no blocking, fusion or
reordering beyond what the paper's definitions state, except that the banded
mode factors each local matrix in ascending global column order (a symmetric
permutation of [Omega_I, Omega_Gamma], which leaves C_ii^{-1} as an operator
unchanged) so that LAPACK's banded Cholesky can hold it.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sl
import scipy.sparse as sp
import scipy.sparse.linalg as sla
from scipy.linalg import lapack as sla_lapack

EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------------------
# Index sets (Section 3, eq. (3.1) and the 5x4 worked example; Algorithm 1 steps 3-4)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class IndexSets:
    N: int
    OI: list  # Omega_I,i: interior columns, ascending
    Xi: list  # Xi_i: rows with a stored entry in an interior column, ascending
    OG: list  # Omega_Gamma,i: other columns of A(Xi_i, :), ascending
    Om: list  # Omega_i = [Omega_I,i, Omega_Gamma,i] (concatenation; order matters)


def as_csr(m, n, row_ptr, col, val) -> sp.csr_matrix:
    return sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(row_ptr)),
                         shape=(m, n))


def index_sets(A: sp.csr_matrix, part: np.ndarray, N: int) -> IndexSets:
    """Xi_i = nonzero rows of A(:, Omega_I,i); Omega_Gamma,i = nonzero columns of
    A(Xi_i, :) not in Omega_I,i; Omega_i = [Omega_I,i, Omega_Gamma,i] (Section 3).

    "Nonzero" is structural: a stored entry counts even if its value is 0.
    """
    Acsc = A.tocsc()
    OI, Xi, OG, Om = [], [], [], []
    for i in range(N):
        oi = np.nonzero(part == i)[0].astype(np.int64)
        rows = np.unique(Acsc[:, oi].indices) if oi.size else np.zeros(0, np.int64)
        cols = np.unique(A[rows, :].indices) if rows.size else np.zeros(0, np.int64)
        og = np.setdiff1d(cols, oi)
        OI.append(oi)
        Xi.append(rows.astype(np.int64))
        OG.append(og.astype(np.int64))
        Om.append(np.concatenate([oi, og]))
    return IndexSets(N, OI, Xi, OG, Om)


def restriction(Om_i: np.ndarray, n: int) -> np.ndarray:
    """R_i = I_n(Omega_i, :) as a dense 0/1 matrix (Section 2; small cases only)."""
    R = np.zeros((len(Om_i), n))
    R[np.arange(len(Om_i)), Om_i] = 1.0
    return R


def partition_of_unity(nI: int, ni: int) -> np.ndarray:
    """D_i: ones on the n_I,i interior positions, zeros on Omega_Gamma,i (Section 3.3.1)."""
    d = np.zeros(ni)
    d[:nI] = 1.0
    return d


# ---------------------------------------------------------------------------
# Shifts and local matrices (Section 4.1.2; Section 3.1; eq. (3.2))
# ---------------------------------------------------------------------------
def global_shift(A: sp.csr_matrix, rel: float = 1e-10) -> float:
    """delta = rel * ||C||_F with C = A^T A formed explicitly (Section 4.1.2)."""
    C = (A.T @ A).tocsr()
    return rel * float(np.sqrt((C.data ** 2).sum()))


def local_matrices(A: sp.csr_matrix, S: IndexSets, i: int, delta: float):
    """Dense C_ii = A(:, Omega_i)^T A(:, Omega_i) + delta I (Section 3.1, shifted as in
    Section 4.1.2) and C~_ii = A(Xi_i, Omega_i)^T A(Xi_i, Omega_i) (eq. (3.2)),
    both in the [Omega_I, Omega_Gamma] order."""
    Ao = A[:, S.Om[i]]
    Cii = (Ao.T @ Ao).toarray() + delta * np.eye(len(S.Om[i]))
    Ax = A[S.Xi[i], :][:, S.Om[i]]
    Ct = (Ax.T @ Ax).toarray()
    return Cii, Ct


def gevp_local(Cii: np.ndarray, Ct: np.ndarray, nI: int, s_rel: float = 1e-8):
    """All eigenpairs of D C_ii D v = lambda (C~_ii + s I) v, s = s_rel ||C~_ii||_F
    (eqs. (3.3)-(3.4) with the shift of Section 4.1.2).  Returned in descending lambda."""
    ni = Cii.shape[0]
    d = partition_of_unity(nI, ni)
    s = s_rel * np.linalg.norm(Ct)
    lam, V = sl.eigh(d[:, None] * Cii * d[None, :], Ct + s * np.eye(ni))
    order = np.argsort(-lam, kind="stable")
    return lam[order], V[:, order]


def select_coarse(lam: np.ndarray, V: np.ndarray, nI: int, tau: float, nev_max: int,
                  kappa_cii: float | None = None, thr: float | None = None):
    """Z_i from eq. (3.6): eigenvectors with lambda > 1/tau (strict, Lemma 2.4), or
    lambda >= 1/(kappa(C_ii) eps) if that is smaller, largest first, at most nev_max
    (Section 4).  ``thr`` gives the threshold 1/tau directly (auto mode, where it is an
    eigenvalue and 1/(1/thr) could round past it).  Returns Zbar_i = the interior rows
    of D_i Z_i (the Gamma rows of D_i Z_i are zero because D_i vanishes there)."""
    if thr is None:
        thr = 1.0 / tau
    keep = lam > thr
    if kappa_cii is not None and 1.0 / (kappa_cii * EPS) < thr:
        keep = lam >= 1.0 / (kappa_cii * EPS)
    idx = np.nonzero(keep)[0][:nev_max]
    return V[:nI, idx].copy(), lam[idx].copy()


def auto_threshold(lams: list, nev_max: int) -> float:
    """1/tau = max_i lambda_{i, nev_max+1}: with strict selection no subdomain keeps
    more than nev_max vectors and the cap never truncates (so Theorem 2.6 applies
    with this tau).  Returns 0 when no subdomain has more than nev_max eigenvalues."""
    cut = [l[nev_max] for l in lams if len(l) > nev_max]
    return float(max(cut)) if cut else 0.0


def auto_tau(lams: list, nev_max: int) -> float:
    thr = auto_threshold(lams, nev_max)
    return 1.0 / thr if thr > 0 else np.inf


# ---------------------------------------------------------------------------
# Coarse space (Lemma 2.5, eq. (2.6); Algorithm 1 steps 9-10)
# ---------------------------------------------------------------------------
def coarse_operator(A: sp.csr_matrix, S: IndexSets, Zbars: list, delta: float):
    """R_0^T = [R_1^T D_1 Z_1, ..., R_N^T D_N Z_N] (only interior rows survive D_i) and
    C_00 = (A R_0^T)^T (A R_0^T) + delta R_0 R_0^T (Algorithm 1 with the shift of
    Section 4.1.2)."""
    n = A.shape[1]
    rows, cols, vals = [], [], []
    off = 0
    for i, Z in enumerate(Zbars):
        k = Z.shape[1]
        if k:
            rr, cc = np.meshgrid(S.OI[i], np.arange(off, off + k), indexing="ij")
            rows.append(rr.ravel())
            cols.append(cc.ravel())
            vals.append(Z.ravel())
        off += k
    n0 = off
    if n0 == 0:
        return sp.csr_matrix((n, 0)), np.zeros((0, 0))
    R0T = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(n, n0))
    AR = (A @ R0T).toarray()
    C00 = AR.T @ AR + delta * (R0T.T @ R0T).toarray()
    return R0T, C00


# ---------------------------------------------------------------------------
# The preconditioner (eq. (2.3))
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class TwoLevel:
    S: IndexSets
    n: int
    local: list  # per subdomain: (index array in factor order, factor object)
    R0T: sp.csr_matrix
    C00f: tuple | None
    lams: list
    ks: list
    tau: float
    delta: float
    thr: float
    mode: str

    @property
    def n0(self) -> int:
        return self.R0T.shape[1]

    def apply_local(self, r: np.ndarray) -> np.ndarray:
        """sum_i R_i^T C_ii^{-1} R_i r (one-level additive Schwarz, eq. (2.1))."""
        z = np.zeros(self.n)
        for idx, fac in self.local:
            if self.mode == "dense":
                y = sl.cho_solve(fac, r[idx])
            else:
                y = sl.cho_solve_banded(fac, r[idx])
            np.add.at(z, idx, y)
        return z

    def apply_coarse(self, r: np.ndarray) -> np.ndarray:
        """R_0^T C_00^{-1} R_0 r (the second-level term of eq. (2.3))."""
        if self.n0 == 0:
            return np.zeros(self.n)
        return self.R0T @ sl.cho_solve(self.C00f, self.R0T.T @ r)

    def apply(self, r: np.ndarray) -> np.ndarray:
        """M_additive^{-1} r = R_0^T C_00^{-1} R_0 r + sum_i R_i^T C_ii^{-1} R_i r (eq. (2.3))."""
        return self.apply_local(r) + self.apply_coarse(r)

    def apply_ras(self, r: np.ndarray) -> np.ndarray:
        """Restricted additive Schwarz, sum_i R_i^T D_i C_ii^{-1} R_i r (Section 2, eq. RAS):
        every subdomain's local solution contributes only on its own interior columns
        (D_i is 1 on Omega_I,i and 0 on Omega_Gamma,i)."""
        z = np.zeros(self.n)
        for i, (idx, fac) in enumerate(self.local):
            if self.mode == "dense":
                y = sl.cho_solve(fac, r[idx])
            else:
                y = sl.cho_solve_banded(fac, r[idx])
            d = np.isin(idx, self.S.OI[i])
            z[idx[d]] += y[d]
        return z

    def apply_deflated(self, A: sp.csr_matrix, r: np.ndarray) -> np.ndarray:
        """The deflated two-level preconditioner of Section 2 (eq. deflated) with the RAS
        first level: Q r + M_RAS (I - C Q) r, Q = R_0^T C_00^{-1} R_0, C = A^T (A .)."""
        qr = self.apply_coarse(r)
        return qr + self.apply_ras(r - A.T @ (A @ qr))

    def apply_balanced(self, A: sp.csr_matrix, r: np.ndarray) -> np.ndarray:
        """The balanced two-level preconditioner of Section 2 (eq. balanced) applied to r:
        Q r + (I - C Q)^T M_1 (I - C Q) r with Q = R_0^T C_00^{-1} R_0, the one-level
        additive operator M_1 = sum_i R_i^T C_ii^{-1} R_i and C = A^T A applied as
        A^T (A .).  (I - C Q)^T = I - Q C because C and Q are symmetric."""
        def C(v):
            return A.T @ (A @ v)
        qr = self.apply_coarse(r)
        u = self.apply_local(r - C(qr))
        return qr + u - self.apply_coarse(C(u))


def _band_lower(M: sp.spmatrix, bw: int) -> np.ndarray:
    """LAPACK lower banded storage: ab[d, j] = M[j + d, j] for d = 0..bw."""
    n = M.shape[0]
    ab = np.zeros((bw + 1, n))
    Md = M.tocoo()
    sel = Md.row >= Md.col
    d = Md.row[sel] - Md.col[sel]
    ab[d, Md.col[sel]] = Md.data[sel]
    return ab


def _local_banded(A, S, i, delta, s_rel):
    """Banded mode: C_ii + delta I and C~_ii + s I in ascending global order."""
    srt = np.sort(S.Om[i])
    Ao = A[:, srt]
    Cii = (Ao.T @ Ao).tocsr() + delta * sp.eye(len(srt), format="csr")
    Ax = A[S.Xi[i], :][:, srt]
    Ct = (Ax.T @ Ax).tocsr()
    s = s_rel * float(np.sqrt((Ct.data ** 2).sum()))
    coo = Cii.tocoo()
    bw = int(np.max(np.abs(coo.row - coo.col))) if coo.nnz else 0
    interior = np.isin(srt, S.OI[i])
    return srt, Cii, Ct, s, bw, interior


def _gevp_banded(Cii, Ct, s, bw, interior, kwant):
    """Top-kwant eigenpairs of D C_ii D v = lambda (C~_ii + s I) v through the standard
    form L^{-1} D C_ii D L^{-T} with C~_ii + s I = L L^T (banded Cholesky) and ARPACK."""
    ni = Cii.shape[0]
    B = Ct + s * sp.eye(ni, format="csr")
    Lb = sl.cholesky_banded(_band_lower(B, bw), lower=True)
    d = interior.astype(np.float64)
    DCD = sp.diags(d) @ Cii @ sp.diags(d)

    # L^{-1} x and L^{-T} x with the banded factor (LAPACK's triangular banded solve)
    def lsolve(x):
        y, info = sla_lapack.dtbtrs(Lb, x.reshape(-1, 1), uplo='L', trans='N')
        assert info == 0
        return y.ravel()

    def ltsolve(x):
        y, info = sla_lapack.dtbtrs(Lb, x.reshape(-1, 1), uplo='L', trans='T')
        assert info == 0
        return y.ravel()

    def mv(u):
        return lsolve(DCD @ ltsolve(u))

    kk = min(kwant, ni - 1)
    if kk <= 0:
        return np.zeros(0), np.zeros((ni, 0))
    op = sla.LinearOperator((ni, ni), matvec=mv, dtype=np.float64)
    v0 = np.ones(ni)
    lam, U = sla.eigsh(op, k=kk, which="LA", tol=1e-13, ncv=min(ni, max(2 * kk + 20, 80)), v0=v0)
    order = np.argsort(-lam)
    lam, U = lam[order], U[:, order]
    V = np.column_stack([ltsolve(U[:, j]) for j in range(U.shape[1])]) if U.size else U
    return lam, V


def build_two_level(A: sp.csr_matrix, part: np.ndarray, N: int, tau: float = 0.0,
                    nev_max: int = 16, delta_rel: float = 1e-10, s_rel: float = 1e-8,
                    mode: str = "dense", coarse: bool = True) -> TwoLevel:
    """Algorithm 1: index sets, local factors of C_ii (+delta), the shifted local GEVPs,
    Z_i under threshold tau (tau <= 0 means "auto from nev_max"), R_0 and chol(C_00)."""
    n = A.shape[1]
    S = index_sets(A, part, N)
    delta = global_shift(A, delta_rel)
    local, lams, Vs, nIs = [], [], [], []
    for i in range(N):
        nI = len(S.OI[i])
        if mode == "dense":
            Cii, Ct = local_matrices(A, S, i, delta)
            fac = sl.cho_factor(Cii, lower=True)
            local.append((S.Om[i], fac))
            if coarse:
                lam, V = gevp_local(Cii, Ct, nI, s_rel)
                # interior rows of V are the first nI rows in [Omega_I, Omega_Gamma] order
                lams.append(lam)
                Vs.append(V[:nI])
        else:
            srt, Cii, Ct, s, bw, interior = _local_banded(A, S, i, delta, s_rel)
            cb = sl.cholesky_banded(_band_lower(Cii, bw), lower=True)
            local.append((srt, (cb, True)))
            if coarse:
                lam, V = _gevp_banded(Cii, Ct, s, bw, interior, nev_max + 1)
                lams.append(lam)
                Vs.append(V[interior])
        nIs.append(nI)
    ks = [0] * N
    R0T, C00f = sp.csr_matrix((n, 0)), None
    if coarse:
        thr = auto_threshold(lams, nev_max) if tau <= 0 else 1.0 / tau
        tau_used = 1.0 / thr if thr > 0 else np.inf
        Zbars = []
        for i in range(N):
            Z, _ = select_coarse(lams[i], Vs[i], Vs[i].shape[0], tau_used, nev_max, thr=thr)
            Zbars.append(Z)
            ks[i] = Z.shape[1]
        R0T, C00 = coarse_operator(A, S, Zbars, delta)
        if R0T.shape[1]:
            C00f = sl.cho_factor(C00, lower=True)
    else:
        tau_used, thr = tau, (1.0 / tau if tau > 0 else 0.0)
    return TwoLevel(S, n, local, R0T, C00f, lams, ks, tau_used, delta, thr, mode)


# ---------------------------------------------------------------------------
# Krylov solvers on C x = A^T b, C applied as A^T (A .) (Section 4.1.3)
# ---------------------------------------------------------------------------
def pcg(A: sp.csr_matrix, b: np.ndarray, apply_M, rtol: float = 1e-8, maxit: int = 1000,
        fixed_iters: int | None = None):
    """Preconditioned CG on the normal equations, x_0 = 0 (Section 4).

    Stops when ||A^T (b - A x)|| <= rtol ||A^T b||: whenever the recursive residual
    passes the test, the true residual is recomputed; if it fails, the iteration
    restarts from the true residual (z = M r, p = z).  With ``fixed_iters`` it runs
    exactly that many iterations instead.
    Returns x and a dict with iterations, residuals and the CG coefficients.
    """
    At = A.T.tocsr()
    g = At @ b
    gn = np.linalg.norm(g)
    x = np.zeros(A.shape[1])
    r = g.copy()
    z = apply_M(r)
    p = z.copy()
    rz = r @ z
    alphas, betas, hist = [], [], []
    it = 0
    while True:
        if fixed_iters is not None and it >= fixed_iters:
            break
        if fixed_iters is None and it >= maxit:
            break
        w = At @ (A @ p)
        pw = p @ w
        alpha = rz / pw
        x += alpha * p
        r -= alpha * w
        it += 1
        alphas.append(alpha)
        rn = np.linalg.norm(r)
        hist.append(rn / gn)
        if fixed_iters is None and rn <= rtol * gn:
            rt = At @ (b - A @ x)
            if np.linalg.norm(rt) <= rtol * gn:
                break
            r = rt
            z = apply_M(r)
            rz = r @ z
            p = z.copy()
            betas.append(0.0)
            continue
        z = apply_M(r)
        rz_new = r @ z
        beta = rz_new / rz
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
    relres_true = np.linalg.norm(At @ (b - A @ x)) / gn
    return x, dict(iters=it, relres_true=relres_true, alphas=alphas, betas=betas, hist=hist)


def preconditioned_lsqr(A: sp.csr_matrix, b: np.ndarray, apply_M, rtol: float = 1e-8, maxit: int = 1000,
                        fixed_iters: int | None = None, check_factor: float = 10.0):
    """LSQR with a symmetric positive definite preconditioner applied as z = M^{-1} s, the
    outer solver the paper uses (Section 4.1.3: left-preconditioned LSQR, which needs
    only applications of M^{-1}).

    Golub-Kahan bidiagonalization of A between R^m (Euclidean) and R^n with the inner
    product <x, y> = x^T M y, in which the adjoint of A is M^{-1} A^T:
        beta_1 u_1 = b,  alpha_1 v_1 = M^{-1} A^T u_1,
        beta_{k+1} u_{k+1} = A v_k - alpha_k u_k,
        alpha_{k+1} v_{k+1} = M^{-1} A^T u_{k+1} - beta_{k+1} v_k,
    where the M-norm alpha = (s^T M^{-1} s)^{1/2} of s = A^T u - beta M v is computed
    from s and t = M^{-1} s (M v is carried along as q = s / alpha).  The least-squares
    problem min ||beta_1 e_1 - B_k y|| is solved by the usual plane rotations, so
    x_k = V_k y_k minimises ||b - A x|| over the Krylov space of M^{-1} A^T A started
    from M^{-1} A^T b: the same iterates as PCG on the normal equations in exact
    arithmetic.

    Stopping: the configs' test ||A^T (b - A x)|| <= rtol ||A^T b||, evaluated on the
    true residual from the first iteration at which LSQR's own estimate of the
    preconditioned normal residual, ||M^{-1} A^T r_k||_M = phibar_{k+1} alpha_{k+1} |c_k|,
    has fallen below check_factor * rtol times its initial value alpha_1 beta_1.
    With ``fixed_iters`` it runs exactly that many iterations.
    Returns x and a dict with iterations, the true relative residual and the
    bidiagonal entries (alphas, betas).
    """
    At = A.T.tocsr()
    gn = np.linalg.norm(At @ b)
    n = A.shape[1]
    x = np.zeros(n)
    beta = np.linalg.norm(b)
    if beta == 0.0 or gn == 0.0:
        return x, dict(iters=0, relres_true=0.0, alphas=[], betas=[])
    u = b / beta
    s = At @ u
    t = apply_M(s)
    alpha = np.sqrt(s @ t)
    v, q = t / alpha, s / alpha
    w = v.copy()
    phibar, rhobar = beta, alpha
    est0 = alpha * beta
    alphas, betas = [alpha], [beta]
    it = 0
    checking = False
    while True:
        if fixed_iters is not None and it >= fixed_iters:
            break
        if fixed_iters is None and it >= maxit:
            break
        u = A @ v - alpha * u
        beta = np.linalg.norm(u)
        u = u / beta
        s = At @ u - beta * q
        t = apply_M(s)
        alpha = np.sqrt(s @ t)
        v, q = t / alpha, s / alpha
        rho = np.hypot(rhobar, beta)
        c, sn = rhobar / rho, beta / rho
        theta = sn * alpha
        rhobar = -c * alpha
        phi = c * phibar
        phibar = sn * phibar
        x = x + (phi / rho) * w
        w = v - (theta / rho) * w
        it += 1
        alphas.append(alpha)
        betas.append(beta)
        if fixed_iters is None:
            if not checking and phibar * alpha * abs(c) <= check_factor * rtol * est0:
                checking = True
            if checking and np.linalg.norm(At @ (b - A @ x)) <= rtol * gn:
                break
    relres_true = np.linalg.norm(At @ (b - A @ x)) / gn
    return x, dict(iters=it, relres_true=relres_true, alphas=alphas, betas=betas)


def fgmres(A: sp.csr_matrix, b: np.ndarray, apply_M, rtol: float = 1e-8, restart: int = 100,
           maxit: int = 1000, fixed_iters: int | None = None):
    """Restarted GMRES on C x = A^T b (C applied as A^T (A .)), right-preconditioned in
    the flexible form (the preconditioned directions z_j = M^{-1} v_j are kept, so a
    preconditioner that is not exactly the same operator every time is allowed): the
    outer solver the paper pairs with RAS and the deflated second level.

    Arnoldi with classical Gram-Schmidt applied twice, Givens rotations on the
    Hessenberg matrix; |gamma_{j+1}| is the residual norm ||A^T b - C x_j||, the quantity
    the configs' test bounds.  When it passes rtol ||A^T b|| (or after `restart` steps)
    x is updated; a pass is confirmed on the true residual, otherwise GMRES restarts from
    it.  With ``fixed_iters`` it runs exactly that many steps (restarting as needed).
    Returns x and a dict with iterations and the true relative residual."""
    At = A.T.tocsr()
    g = At @ b
    gn = np.linalg.norm(g)
    n = A.shape[1]
    x = np.zeros(n)
    if gn == 0.0:
        return x, dict(iters=0, relres_true=0.0)
    it = 0
    while True:
        r = g - At @ (A @ x)
        beta = np.linalg.norm(r)
        if fixed_iters is None and beta <= rtol * gn:
            break
        if (fixed_iters is not None and it >= fixed_iters) or (fixed_iters is None and it >= maxit):
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        gam = np.zeros(restart + 1)
        gam[0] = beta
        j = 0
        while j < restart:
            z = apply_M(V[j])
            Z.append(z)
            w = At @ (A @ z)
            Vm = np.column_stack(V)
            h = Vm.T @ w
            w = w - Vm @ h
            h2 = Vm.T @ w
            w = w - Vm @ h2
            h = h + h2
            H[: j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j])
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j], H[j + 1, j] = den, 0.0
            gam[j + 1] = -sn[j] * gam[j]
            gam[j] = cs[j] * gam[j]
            j += 1
            it += 1
            if fixed_iters is not None and it >= fixed_iters:
                break
            if fixed_iters is None and (abs(gam[j]) <= rtol * gn or it >= maxit):
                break
        y = sl.solve_triangular(H[:j, :j], gam[:j])
        x = x + np.column_stack(Z) @ y
    relres_true = np.linalg.norm(g - At @ (A @ x)) / gn
    return x, dict(iters=it, relres_true=relres_true)


def lsqr_kappa(alphas, betas) -> float:
    """kappa of M^{-1} A^T A estimated from the bidiagonal: the Lanczos matrix of the
    normal-equations operator is B_k^T B_k, with diagonal alpha_j^2 + beta_{j+1}^2 and
    off-diagonal alpha_{j+1} beta_{j+1} (alphas[0] = alpha_1, betas[0] = beta_1)."""
    k = len(alphas) - 1
    if k < 1:
        return 0.0
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = alphas[j] ** 2 + betas[j + 1] ** 2
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = alphas[j + 1] * betas[j + 1]
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])


def flexible_pcg(A: sp.csr_matrix, b: np.ndarray, apply_M, rtol: float = 1e-8,
                 maxit: int = 1000, fixed_iters: int | None = None):
    """Flexible PCG: beta = z_{k+1}^T (r_{k+1} - r_k) / (z_k^T r_k) (Polak-Ribiere form),
    otherwise as :func:`pcg` (same stopping and restart rule)."""
    At = A.T.tocsr()
    g = At @ b
    gn = np.linalg.norm(g)
    x = np.zeros(A.shape[1])
    r = g.copy()
    z = apply_M(r)
    p = z.copy()
    rz = r @ z
    it = 0
    hist = []
    while True:
        if fixed_iters is not None and it >= fixed_iters:
            break
        if fixed_iters is None and it >= maxit:
            break
        w = At @ (A @ p)
        alpha = rz / (p @ w)
        x += alpha * p
        r_old = r.copy()
        r = r - alpha * w
        it += 1
        rn = np.linalg.norm(r)
        hist.append(rn / gn)
        if fixed_iters is None and rn <= rtol * gn:
            rt = At @ (b - A @ x)
            if np.linalg.norm(rt) <= rtol * gn:
                break
            r = rt
            z = apply_M(r)
            rz = r @ z
            p = z.copy()
            continue
        z = apply_M(r)
        beta = (z @ (r - r_old)) / rz
        rz = r @ z
        p = z + beta * p
    relres_true = np.linalg.norm(At @ (b - A @ x)) / gn
    return x, dict(iters=it, relres_true=relres_true, hist=hist)


def lanczos_kappa(alphas, betas) -> float:
    """Condition estimate of M^{-1} C from the CG coefficients through the CG-Lanczos
    relation: T_kk = 1/alpha_k + beta_{k-1}/alpha_{k-1}, T_{k,k+1} = sqrt(beta_k)/alpha_k."""
    k = len(alphas)
    if k == 0:
        return 1.0
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev[-1] / ev[0])


# ---------------------------------------------------------------------------
# Adjoint gradient of x(A, b) = C^{-1} A^T b
# ---------------------------------------------------------------------------
def adjoint_gradient(A: sp.csr_matrix, b: np.ndarray, x: np.ndarray, gbar: np.ndarray,
                     solve_C):
    """lambda = C^{-1} gbar; grad_b = A lambda; grad on the stored entries (r, c) of A:
    rho_r lambda_c - (A lambda)_r x_c with rho = b - A x (differentiating C x = A^T b)."""
    lam = solve_C(gbar)
    Al = A @ lam
    rho = b - A @ x
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    gvals = rho[rows] * lam[A.indices] - Al[rows] * x[A.indices]
    return Al, gvals, lam


# ---------------------------------------------------------------------------
# Constants of the theory (Lemma 3.1, Lemma 2.2, Theorem 2.6)
# ---------------------------------------------------------------------------
def multiplicity_km(A: sp.csr_matrix, S: IndexSets) -> int:
    """k_m = max_j m_j, m_j = #{i : row j in Xi_i} (Lemma 3.1)."""
    cnt = np.zeros(A.shape[0], dtype=np.int64)
    for xi in S.Xi:
        cnt[xi] += 1
    return int(cnt.max()) if cnt.size else 0


def subdomain_colouring(A: sp.csr_matrix, S: IndexSets) -> list:
    """Greedy colouring of the subdomain graph of Lemma 2.2: i ~ j iff C(Omega_i, Omega_j)
    has a structural nonzero, so that subdomains of one colour span mutually
    C-orthogonal spaces.  Subdomains are visited in index order and each takes the
    smallest colour none of its coloured neighbours has.  Returns one colour per
    subdomain (0-based)."""
    C = (abs(A).T @ abs(A)).tocsr()
    N = S.N
    n = A.shape[1]
    memb = [[] for _ in range(n)]
    for i in range(N):
        for j in S.Om[i]:
            memb[j].append(i)
    adj = [set() for _ in range(N)]
    for i in range(N):
        reach = np.unique(C[S.Om[i], :].indices)
        for j in reach:
            for k in memb[j]:
                if k != i:
                    adj[i].add(k)
    colour = [-1] * N
    for i in range(N):
        used = {colour[k] for k in adj[i] if colour[k] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    return colour


def colouring_kc(A: sp.csr_matrix, S: IndexSets) -> int:
    """Upper bound on k_c of Lemma 2.2 (the fewest colours such that same-coloured
    subdomains are mutually C-orthogonal): the number of colours of the greedy
    colouring above."""
    colour = subdomain_colouring(A, S)
    return max(colour) + 1 if colour else 0


def theorem26_bound(kc: int, km: int, tau: float, variant: str = "thm") -> float:
    """kappa(M_additive^{-1} C) <= (k_c + 1)(2 + (2 k_c + 1) k_m / tau) (Theorem 2.6);
    variant "sec32" gives the restatement (k_c + 1)(2 + 2 (k_c + 1) k_m / tau) of Section 3.2."""
    if variant == "thm":
        return (kc + 1) * (2 + (2 * kc + 1) * km / tau)
    return (kc + 1) * (2 + 2 * (kc + 1) * km / tau)
