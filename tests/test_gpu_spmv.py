"""Every kernel of the products with A and A^T (option spmv), against the oracle.

Each kernel code is forced for both products and checked on:

* the 96 x 96 grid (9 subdomains): w = A^T (A p) against scipy's sparse product to 1e-12
  relative (same sums, different order), and six fixed PCG iterations against the
  oracle's PCG to 1e-10 (the A^T product carries the fused p . w of every iteration);
* a 48 x 48 grid with one dense row and one dense column appended (one subdomain): the
  dense row of A and the dense column (a row of A^T) hold more than 768 entries, so the
  warp-stream kernels take their warp-per-row path for them, and the sliced-ELL slices
  holding them are 2,000+ entries wide.

The autotuned default must pick one of the codes and give the same product.

The row-tile form of the whole product (option normal_product = 2: tiles of consecutive
rows, A p and A^T of it per tile in shared memory, partial windows summed per column in
tile order) is checked the same way, plus: a window as wide as the matrix (the dense
row), empty rows and columns, bitwise repeatability, new values through
ls_update_values, and a matrix whose single row is too wide for a block (forced: the
setup refuses; automatic: the two products run).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

import scipy.sparse as sp  # noqa: E402

import paper_2107_09006_gb300 as L  # noqa: E402
import oracle as O  # noqa: E402
from workloads import make_grid_ls, block_partition  # noqa: E402

CODES = [-3, -2, -1, 1, 2, 4, 8, 16, 32]


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def grid96():
    m, n, rp, c, v, b, _ = make_grid_ls(96, 96, 4, 8, 3, 0)
    part = block_partition(96, 96, 32, 32)
    A = O.schwarz.as_csr(m, n, rp, c, v)
    return dict(m=m, n=n, rp=rp, c=c, v=v, b=b, part=part, A=A, M=O.build_two_level(A, part, 9, tau=0.0, nev_max=8))


@pytest.fixture(scope="module")
def dense_parts():
    m, n, rp, c, v, b, _ = make_grid_ls(48, 48, 4, 8, 3, 1)
    A = O.schwarz.as_csr(m, n, rp, c, v).tolil()
    rng = np.random.default_rng(5)
    A[:, n - 1] = rng.standard_normal((m, 1))            # a dense column: m entries
    A = sp.vstack([A.tocsr(), sp.csr_matrix(rng.standard_normal((1, n)))]).tocsr()  # a dense row: n entries
    A.sort_indices()
    assert A.getnnz(axis=1).max() > 2048 and A.getnnz(axis=0).max() > 2048
    return A


@pytest.mark.parametrize("code", CODES)
def test_normal_product_every_kernel(grid96, code):
    d = grid96
    S = L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 9, nev_max=8, spmv=code)
    p = np.random.default_rng(3).standard_normal(d["n"])
    w = S.apply_normal(p).cpu().numpy()
    assert rel(w, d["A"].T @ (d["A"] @ p)) < 1e-12
    S.close()


@pytest.mark.parametrize("code", [-3, -2, -1, 1, 4, 32])
def test_pcg_fixed_iterations_every_kernel(grid96, code):
    d = grid96
    S = L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 9, nev_max=8, spmv=code, fixed_iters=6)
    x, info = S.solve(d["b"], rtol=1e-8)
    assert (info["lanes_csr"], info["lanes_csc"]) == (code, code)
    xo, _ = O.pcg(d["A"], d["b"], d["M"].apply, fixed_iters=6)
    assert rel(x.cpu().numpy(), xo) < 1e-10
    S.close()


@pytest.mark.parametrize("code", CODES)
def test_long_rows_every_kernel(dense_parts, code):
    A = dense_parts
    m, n = A.shape
    S = L.Solver(m, n, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data, np.zeros(n, np.int32), 1,
                 coarse=0, nev_max=0, spmv=code)
    p = np.random.default_rng(4).standard_normal(n)
    w = S.apply_normal(p).cpu().numpy()
    assert rel(w, A.T @ (A @ p)) < 1e-12
    S.close()


def test_autotuned_choice(grid96):
    d = grid96
    S = L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 9, nev_max=8)
    x, info = S.solve(d["b"], rtol=1e-8)
    assert info["lanes_csr"] in CODES and info["lanes_csc"] in CODES
    p = np.random.default_rng(3).standard_normal(d["n"])
    assert rel(S.apply_normal(p).cpu().numpy(), d["A"].T @ (d["A"] @ p)) < 1e-12
    S.close()


def test_bad_code_rejected(grid96):
    d = grid96
    with pytest.raises(L.LSError) as ex:
        L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 9, nev_max=8, spmv=3)
    with pytest.raises(L.LSError):
        L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 9, nev_max=8, spmv=64)
    assert ex.value.status == L.LS_ERR_INVALID


def _tiles(A, part=None, nparts=1, **kw):
    m, n = A.shape
    part = np.zeros(n, np.int32) if part is None else part
    return L.Solver(m, n, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data, part, nparts,
                    coarse=0, nev_max=0, **kw)


@pytest.fixture(scope="module")
def holes():
    """The 96 x 96 grid with every 7th row emptied and columns 100-163 removed."""
    m, n, rp, c, v, b, _ = make_grid_ls(96, 96, 4, 8, 3, 2)
    A = O.schwarz.as_csr(m, n, rp, c, v).tolil()
    A[::7, :] = 0.0
    A[:, 100:164] = 0.0
    A = A.tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    assert (A.getnnz(axis=1) == 0).sum() > 6000 and (A.getnnz(axis=0) == 0).sum() == 64
    return A


@pytest.mark.parametrize("kernel", [1, 2, 3, 4])
@pytest.mark.parametrize("case", ["grid96", "dense", "holes"])
def test_row_tiles_normal_product(grid96, dense_parts, holes, case, kernel):
    A = {"grid96": grid96["A"], "dense": dense_parts, "holes": holes}[case]
    S = _tiles(A, normal_product=2, normal_kernel=kernel)
    assert S.info()["normal_product"] == 2 and S.normal_tiles()["kernel"] == kernel
    p = np.random.default_rng(6).standard_normal(A.shape[1])
    w = S.apply_normal(p).cpu().numpy()
    assert rel(w, A.T @ (A @ p)) < 1e-12
    assert np.array_equal(S.apply_normal(p).cpu().numpy(), w)  # fixed summation order
    S.close()


def test_row_tiles_pcg_and_repeatability(grid96):
    d = grid96
    kw = dict(nev_max=8, normal_product=2, fixed_iters=6)
    S = L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 9, **kw)
    x, info = S.solve(d["b"], rtol=1e-8)
    assert info["normal_product"] == 2
    xo, _ = O.pcg(d["A"], d["b"], d["M"].apply, fixed_iters=6)
    assert rel(x.cpu().numpy(), xo) < 1e-10
    x2, _ = S.solve(d["b"], rtol=1e-8)
    assert torch.equal(x, x2)
    S.close()
    S = L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 9, nev_max=8, normal_product=2)
    x, info = S.solve(d["b"], rtol=1e-10)
    assert info["relres_true"] <= 1e-10
    _, io = O.pcg(d["A"], d["b"], d["M"].apply, rtol=1e-10)
    assert abs(info["iters"] - io["iters"]) <= 1
    S.close()


def test_row_tiles_follow_new_values(grid96):
    d = grid96
    S = L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 9, nev_max=8, normal_product=2)
    v2 = d["v"] * np.random.default_rng(8).uniform(0.5, 2.0, size=d["v"].shape)
    S.update_values(v2)
    A2 = O.schwarz.as_csr(d["m"], d["n"], d["rp"], d["c"], v2)
    p = np.random.default_rng(9).standard_normal(d["n"])
    assert rel(S.apply_normal(p).cpu().numpy(), A2.T @ (A2 @ p)) < 1e-12
    S.close()


def test_row_tiles_refused_for_a_row_wider_than_a_block():
    """A 192 x 192 grid (n = 36,864) plus one row holding columns 0 and n - 1: no block's
    shared memory holds that row's window."""
    m, n, rp, c, v, b, _ = make_grid_ls(192, 192, 4, 8, 3, 3)
    A = sp.vstack([O.schwarz.as_csr(m, n, rp, c, v), sp.csr_matrix(([1.0, 1.0], ([0, 0], [0, n - 1])), shape=(1, n))])
    A = A.tocsr()
    A.sort_indices()
    part = block_partition(192, 192, 64, 64)
    with pytest.raises(L.LSError) as ex:
        _tiles(A, part, 9, normal_product=2)
    assert ex.value.status == L.LS_ERR_UNSUPPORTED and "normal_product" in str(ex.value)
    S = _tiles(A, part, 9)
    assert S.info()["normal_product"] == 1
    p = np.random.default_rng(10).standard_normal(n)
    assert rel(S.apply_normal(p).cpu().numpy(), A.T @ (A @ p)) < 1e-12
    S.close()


def test_forced_kernel_keeps_two_products(grid96):
    d = grid96
    S = L.Solver(d["m"], d["n"], d["rp"], d["c"], d["v"], d["part"], 9, nev_max=8, spmv=2)
    assert S.info()["normal_product"] == 1
    S.close()
