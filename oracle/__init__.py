"""FP64 CPU oracle for the two-level Schwarz-preconditioned normal equations.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
legs of ``bench.py`` use it.  It shares no code with the CUDA path; both take
their inputs from the seeded generators in ``workloads``.

It follows Al Daas, Jolivet & Scott, "A robust algebraic domain decomposition
preconditioner for sparse normal equations" (arXiv 2107.09006):

* index sets Xi_i, Omega_Gamma_i, Omega_i              (Section 3, eq. (3.1))
* partition of unity D_i                                (Section 3.3.1)
* local matrices C_ii and splittings C~_ii              (Section 3.1, eq. (3.2))
* shifted generalized eigenproblems, threshold tau      (Section 3.3.2, eqs. (3.3)-(3.6))
* coarse space R_0 and C_00                             (Lemma 2.5, Algorithm 1)
* two-level additive preconditioner                     (eq. (2.3))
* PCG on C x = A^T b with C applied as A^T (A .)        (Section 4.1.3)
* flexible PCG, Lanczos condition estimate, adjoint gradient (solver-side additions)

Parity status: every function is pinned by ``tests/test_oracle_pins.py``; none is
"parity unpinned".
"""
from .schwarz import (  # noqa: F401
    IndexSets,
    index_sets,
    local_matrices,
    global_shift,
    gevp_local,
    select_coarse,
    auto_tau,
    auto_threshold,
    coarse_operator,
    TwoLevel,
    build_two_level,
    pcg,
    flexible_pcg,
    lanczos_kappa,
    preconditioned_lsqr,
    lsqr_kappa,
    fgmres,
    adjoint_gradient,
    multiplicity_km,
    subdomain_colouring,
    colouring_kc,
    theorem26_bound,
)
