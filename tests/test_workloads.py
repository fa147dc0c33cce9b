"""The seeded generators produce the documented shapes, windows and partitions."""
import numpy as np

from workloads import (make_grid_ls, config_tiny, block_partition, strip_partition,
                       bisection_partition, config_batch_sizes)


def test_tiny_shape(tiny):
    assert (tiny.m, tiny.n, tiny.nnz, tiny.nparts) == (5120, 1024, 17408, 8)
    assert np.all(np.diff(tiny.row_ptr) > 0)
    # strips of 32x4
    assert np.all(np.bincount(tiny.part) == 128)


def test_rows_lie_in_windows_and_are_sorted():
    W, H, r, k = 20, 17, 3, 8
    m, n, rp, c, v, b, _ = make_grid_ls(W, H, 4, k, r, 5)
    mr = 4 * n
    cols = c[: mr * k].reshape(mr, k).astype(np.int64)
    assert np.all(np.diff(cols, axis=1) > 0)  # distinct, ascending
    gx, gy = cols % W, cols // W
    assert np.all(gx.max(1) - gx.min(1) <= 2 * r) and np.all(gy.max(1) - gy.min(1) <= 2 * r)
    assert np.all(c[mr * k:] == np.arange(n)) and np.all(v[mr * k:] == 1e-2)
    assert b.shape == (m,)


def test_determinism_and_chunking():
    a = make_grid_ls(30, 30, 4, 8, 3, 1)
    b = make_grid_ls(30, 30, 4, 8, 3, 1)
    for x, y in zip(a[2:6], b[2:6]):
        assert np.array_equal(x, y)


def test_partitions():
    p = block_partition(1024, 1024, 64, 64)
    assert p.max() == 255 and np.all(np.bincount(p) == 4096)
    assert p[0] == 0 and p[64] == 1 and p[64 * 1024] == 16
    s = strip_partition(32, 32, 4)
    assert s[128] == 1
    q = bisection_partition(200, 180, 8192, 3)
    sizes = np.bincount(q)
    assert sizes.max() <= 8192 and sizes.min() > 1000


def test_batch_sizes():
    sides = config_batch_sizes()
    assert len(sides) == 64
    assert min(s * s for s in sides) >= 16000 and max(s * s for s in sides) <= 263000


def test_batched_block_diagonal():
    from workloads import config_batch
    B = config_batch(nprob=5, nrhs=2, lo=1024, hi=4096, max_cols=600)
    assert B.b.shape == (2, B.m) and B.m_off[-1] == B.m and B.n_off[-1] == B.n
    assert B.row_ptr[0] == 0 and B.row_ptr[-1] == len(B.col) == len(B.val)
    nid = 0
    for q in range(B.nprob):
        r0, r1 = B.m_off[q], B.m_off[q + 1]
        cols = B.col[B.row_ptr[r0]:B.row_ptr[r1]]
        assert cols.min() >= B.n_off[q] and cols.max() < B.n_off[q + 1]
        ids = np.unique(B.part[B.n_off[q]:B.n_off[q + 1]])
        assert ids[0] == nid and np.array_equal(ids, np.arange(ids[0], ids[-1] + 1))
        nid = ids[-1] + 1
        m, n, rp, c, v, part, N, b = B.problem(q)
        assert m == 5 * n and rp[0] == 0 and c.max() < n and part.max() == N - 1 and b.shape == (2, m)
    assert nid == B.nparts


def test_zero_sum_rows():
    """The zero-sum variant takes the same draws and centres each random row."""
    m, n, rp, c, v, b, _ = make_grid_ls(20, 20, 4, 6, 2, 3)
    m2, n2, rp2, c2, v2, b2, _ = make_grid_ls(20, 20, 4, 6, 2, 3, zero_sum=True)
    assert np.array_equal(c, c2) and np.array_equal(b, b2)
    k = 6
    vr, vr2 = v[: 4 * n * k].reshape(-1, k), v2[: 4 * n * k].reshape(-1, k)
    assert np.allclose(vr2.sum(axis=1), 0.0, atol=1e-12)
    assert np.allclose(vr2, vr - vr.mean(axis=1, keepdims=True))
    assert np.array_equal(v[4 * n * k:], v2[4 * n * k:])
