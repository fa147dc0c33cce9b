"""Object wrapper around the C ABI and the autograd function whose backward is the
adjoint solve.  PyTorch only provides device memory here; all arithmetic runs in
libls_schwarz.so."""
from __future__ import annotations

import numpy as np
import torch

from . import (ls_setup, ls_setup_batched, ls_solve, ls_backward, ls_free, ls_default_options, ls_handle_info,
               ls_update_values, ls_apply_preconditioner, ls_apply_normal, ls_query, LS_Q_SIZES, LS_Q_OMEGA,
               LS_Q_XI, LS_Q_EIGVALS, LS_Q_ZBAR, LS_Q_EIGSTEPS, LS_Q_STORAGE, LS_Q_BATCH, LS_Q_NORMAL)


def _dev(a, dtype, device):
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=device)


class Solver:
    """Owns one ls_handle: ``Solver(m, n, row_ptr, col, val, part, nparts, **options)``.

    ``tau`` is ls_setup's threshold (keep lambda > 1/tau; <= 0: automatic).  The other
    options are the fields of ls_options (nev_max, delta_rel, s_rel, factor_prec
    ('f64' | 'f32' | 'bf16'), maxit, coarse, fixed_iters, eig_maxit, eig_tol,
    use_graph, time_kernels, equilibrate, variant (0 additive, 1 balanced second level,
    2 RAS with the deflated second level), solver (0 PCG, 1 preconditioned LSQR, 2
    GMRES), restart (GMRES restart length), spmv (0: the sparse-product kernels are
    chosen by timing at setup; else one kernel code for both products)).  Arrays may be
    numpy arrays or tensors; they
    are copied by setup.  ``solve`` takes b of shape [m] or [nrhs, m] (up to 32 right-hand
    sides advance together).
    """

    def __init__(self, m, n, row_ptr, col, val, part, nparts, device="cuda", stream=None, problems=None,
                 tau=0.0, **options):
        """``stream``: a torch.cuda.Stream the handle runs on (None: its own stream).
        ``problems``: None, or (m_off, n_off) row/column offsets of independent problems
        stored block-diagonally in (row_ptr, col, val) (ls_setup_batched)."""
        self.device = torch.device(device)
        self.m, self.n = int(m), int(n)
        self.row_ptr = _dev(row_ptr, torch.int64, self.device)
        self.col = _dev(col, torch.int32, self.device)
        self.val = _dev(val, torch.float64, self.device)
        self.part = _dev(part, torch.int32, self.device)
        self.nparts = int(nparts)
        self.opt = ls_default_options(**options)
        self.tau = float(tau)
        self.nprob = 1 if problems is None else len(problems[0]) - 1
        with torch.cuda.device(self.device):
            torch.cuda.synchronize(self.device)  # the inputs above were written on torch's stream
            s = stream.cuda_stream if stream is not None else None
            if problems is None:
                self.h = ls_setup(self.m, self.n, self.row_ptr, self.col, self.val, self.nparts, self.part, 1,
                                  self.tau, self.opt, s)
            else:
                self.h = ls_setup_batched(problems[0], problems[1], self.row_ptr, self.col, self.val, self.nparts,
                                          self.part, 1, self.tau, self.opt, s)
        self.stream = stream

    def close(self):
        if getattr(self, "h", None):
            ls_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        return ls_handle_info(self.h)

    def _fence(self):
        """Order torch's pending writes of the inputs before the library's stream reads them."""
        if self.stream is None:
            torch.cuda.current_stream(self.device).synchronize()

    def _torch_stream(self):
        """torch's current stream on the solver's device, which the solve and the
        adjoint order themselves against (the inputs were written there)."""
        return torch.cuda.current_stream(self.device).cuda_stream

    def solve(self, b, rtol=1e-8, raise_on_fail=True):
        """x = argmin ||A x - b|| for b of shape [m] or [nrhs, m] (one right-hand side per row)."""
        b = _dev(b, torch.float64, self.device)
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        x = torch.empty((self.n,) if b.dim() == 1 else (nrhs, self.n), dtype=torch.float64, device=self.device)
        info = ls_solve(self.h, b, nrhs, rtol, x, raise_on_fail, stream=self._torch_stream())
        return x, info

    def backward(self, b, x, grad_x, rtol=1e-10, want_b=True, want_vals=True):
        b = _dev(b, torch.float64, self.device)
        x = _dev(x, torch.float64, self.device)
        g = _dev(grad_x, torch.float64, self.device)
        nrhs = 1 if b.dim() == 1 else b.shape[0]
        gb = torch.empty_like(b) if want_b else None
        gv = torch.empty(self.val.shape[0], dtype=torch.float64, device=self.device) if want_vals else None
        info = ls_backward(self.h, b, x, g, nrhs, rtol, gb, gv, stream=self._torch_stream())
        return gb, gv, info

    def update_values(self, val):
        """Replace A's values in the operator (the preconditioner is kept)."""
        v = _dev(val, torch.float64, self.device)
        self._fence()
        ls_update_values(self.h, v)

    def apply_preconditioner(self, r, which=0):
        r = _dev(r, torch.float64, self.device)
        z = torch.empty_like(r)
        self._fence()
        ls_apply_preconditioner(self.h, r, z, which)
        return z

    def apply_normal(self, p):
        p = _dev(p, torch.float64, self.device)
        w = torch.empty_like(p)
        self._fence()
        ls_apply_normal(self.h, p, w)
        return w

    # ---- inspection -------------------------------------------------------------
    def sizes(self) -> np.ndarray:
        out = np.zeros(self.nparts * 4, np.int64)
        return ls_query(self.h, LS_Q_SIZES, 0, out).reshape(self.nparts, 4)

    def omega(self, i) -> np.ndarray:
        return ls_query(self.h, LS_Q_OMEGA, i, np.zeros(int(self.sizes()[i, 0]), np.int32))

    def xi(self, i) -> np.ndarray:
        return ls_query(self.h, LS_Q_XI, i, np.zeros(int(self.sizes()[i, 2]), np.int32))

    def eigvals(self, i) -> np.ndarray:
        ni = int(self.sizes()[i, 0])
        return ls_query(self.h, LS_Q_EIGVALS, i, np.zeros(min(self.opt.nev_max + 1, ni), np.float64))

    def zbar(self, i) -> np.ndarray:
        s = self.sizes()[i]
        k, nI = int(s[3]), int(s[1])
        out = np.zeros(max(k * nI, 1), np.float64)
        if k:
            ls_query(self.h, LS_Q_ZBAR, i, out)
        return out[: k * nI].reshape(k, nI)

    def storage(self) -> dict:
        o = ls_query(self.h, LS_Q_STORAGE, 0, np.zeros(8, np.int64))
        keys = ("fac_elems", "total_local", "total_blocks", "zbar_elems", "n0", "n0_padded", "nnz", "prec")
        return {k: int(v) for k, v in zip(keys, o)}

    def normal_tiles(self) -> dict:
        """Layout of the row tiles of the normal product (zeros for the two-product form)."""
        o = ls_query(self.h, LS_Q_NORMAL, 0, np.zeros(12, np.int64))
        keys = ("tiles", "row_entries", "col_entries", "row_slices", "col_slices", "window_sum", "kernel")
        d = {k: int(v) for k, v in zip(keys, o)}
        d["setup_ms"] = {"two_products": o[7] * 1e-6, **{f"kernel_{c}": o[7 + c] * 1e-6 for c in range(1, 5)}}
        return d

    def eig_steps(self) -> np.ndarray:
        return ls_query(self.h, LS_Q_EIGSTEPS, 0, np.zeros(self.nparts, np.int32))

    def batch_stats(self, nrhs) -> tuple:
        """(iterations, true relative residuals) of the last multi right-hand-side solve,
        each of shape [nprob, nrhs]."""
        out = ls_query(self.h, LS_Q_BATCH, 0, np.zeros(2 * self.nprob * nrhs, np.float64))
        k = self.nprob * nrhs
        return out[:k].reshape(self.nprob, nrhs).astype(np.int64), out[k:].reshape(self.nprob, nrhs)


class LSSolve(torch.autograd.Function):
    """x = LSSolve.apply(vals, b, solver, rtol): the LS solution for A with the solver's
    pattern and the values ``vals`` (caller's CSR order).  Backward is the adjoint solve
    lambda = C^{-1} grad_x with the same preconditioner: grad_b = A lambda,
    grad_vals = rho lambda^T - (A lambda) x^T on the stored entries (rho = b - A x).
    The operator takes ``vals`` (ls_update_values); the preconditioner stays the one
    the solver was set up with."""

    @staticmethod
    def forward(ctx, vals, b, solver, rtol=1e-10):
        solver.update_values(vals.detach())
        x, info = solver.solve(b.detach(), rtol)
        ctx.solver, ctx.rtol = solver, rtol
        ctx.save_for_backward(b.detach(), x)
        return x

    @staticmethod
    def backward(ctx, gx):
        b, x = ctx.saved_tensors
        gb, gv, _ = ctx.solver.backward(b, x, gx.contiguous(), ctx.rtol)
        return gv, gb, None, None
