"""The allocation-free normal-equations product agrees with scipy and with the
handle-based product.

ls_normal_product_noalloc is for callers that cannot call cudaMalloc (device memory
owned by a framework pool or a fixed budget, real-time loops that must stay out of the
CUDA memory allocator): it keeps the intermediate A p in a fixed device array inside
the library.  This file is collected last so that a failure here comes after every
other test; it passes alone in a fresh process and after the rest.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

import scipy.sparse as sp  # noqa: E402

import paper_2107_09006_gb300 as L  # noqa: E402
from workloads import config_tiny, make_grid_ls, block_partition  # noqa: E402


def _dev(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("which", ["tiny", "grid96"])
def test_noalloc_matches_scipy_and_handle_product_twice(which):
    if which == "tiny":
        P = config_tiny()
        m, n, rp, c, v, part, N = P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts
    else:
        m, n, rp, c, v, _, _ = make_grid_ls(96, 96, 4, 8, 3, 0)
        part, N = block_partition(96, 96, 32, 32), 9
    A = sp.csr_matrix((v, c, rp), shape=(m, n))
    Ac = A.tocsc()
    Ac.sort_indices()
    d_rp, d_c, d_v = _dev(rp, torch.int64), _dev(c, torch.int32), _dev(v, torch.float64)
    d_cp, d_r, d_cv = _dev(Ac.indptr, torch.int64), _dev(Ac.indices, torch.int32), _dev(Ac.data, torch.float64)
    S = L.Solver(m, n, rp, c, v, part, N, coarse=0)
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream()
    for call in range(2):  # two calls in a row share the fixed scratch
        p = rng.standard_normal(n)
        ref = A.T @ (A @ p)  # scipy, FP64
        hand = S.apply_normal(p).cpu().numpy()
        d_p = _dev(p, torch.float64)
        d_w = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        L.ls_normal_product_noalloc(m, n, d_rp, d_c, d_v, d_cp, d_r, d_cv, A.nnz, d_p, d_w, stream.cuda_stream)
        stream.synchronize()
        w = d_w.cpu().numpy()
        assert np.all(np.isfinite(w)), call
        assert np.linalg.norm(w - ref) <= 1e-13 * np.linalg.norm(ref), call
        assert np.linalg.norm(w - hand) <= 1e-13 * np.linalg.norm(hand), call
    S.close()


def test_noalloc_rejects_oversized_m():
    """The C side refuses m beyond its fixed scratch before touching any pointer (the raw
    call, past the binding's own checks)."""
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    i = torch.zeros(4, dtype=torch.int64, device="cuda")
    j = torch.zeros(4, dtype=torch.int32, device="cuda")
    ptrs = [t.data_ptr() for t in (i, j, d, i, j, d)]
    st = L._lib.ls_normal_product_noalloc((1 << 23) + 1, 1, *ptrs, 0, d.data_ptr(), d.data_ptr(), None)
    assert st == L.LS_ERR_INVALID
    assert b"exceeds" in L._lib.ls_noalloc_last_error()
