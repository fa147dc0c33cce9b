"""Seeded generators for sparse least-squares problems on a 2-D grid of unknowns.

Shape class: the paper studies large sparse LS problems min ||Ax - b|| with
m >= n, a few nonzeros per row and a sparse normal-equations matrix C = A^T A
(Section 1, Section 4).  The generators below draw matrices of that class on a
W x H grid of unknowns (column j <-> grid point (j % W, j // W)):

* ``rows_per_point * n`` random rows.  Each row picks a centre uniformly on the
  grid, then ``k`` distinct grid points inside the Chebyshev window of radius
  ``radius`` around it (window clipped to the grid, points drawn uniformly
  without replacement), with N(0, 1) values.
* ``n`` identity rows ``ident_scale * e_j^T`` appended after the random rows, so
  A has full column rank.
* optional column scaling by 10**u_j, u_j ~ U(-3, 3) (an ill-conditioned C).

Draw order and seeds are fixed: the matrix uses ``default_rng(seed)`` (centres,
then point choices, then values); right-hand sides ``seed + 1``; the target
``x*`` ``seed + 2``; column scales ``seed + 3``.

Nothing here computes any part of the solver.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_CHUNK = 1 << 18


@dataclasses.dataclass
class GridLS:
    """A sparse LS instance in CSR form plus its column partition."""

    m: int
    n: int
    row_ptr: np.ndarray  # int64[m+1]
    col: np.ndarray  # int32[nnz], sorted within each row
    val: np.ndarray  # float64[nnz]
    part: np.ndarray  # int32[n], subdomain id of every column
    nparts: int
    b: np.ndarray  # float64[m] or [nrhs, m]
    xstar: np.ndarray | None = None  # float64[n]
    W: int = 0
    H: int = 0
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        """Dense copy of A (small cases only)."""
        A = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        A[rows, self.col] = self.val
        return A


def _window_offsets(radius: int):
    w = 2 * radius + 1
    cells = np.arange(w * w)
    return cells % w - radius, cells // w - radius


def make_grid_ls(W: int, H: int, rows_per_point: int, k: int, radius: int, seed: int,
                 ident_scale: float = 1e-2, col_scale: bool = False, nrhs: int = 1,
                 with_xstar: bool = False, name: str = "", zero_sum: bool = False) -> tuple:
    """Draw the CSR matrix, right-hand side(s) and optional x* of one grid problem.

    Returns ``(m, n, row_ptr, col, val, b, xstar)``; ``b`` has shape ``[m]`` when
    ``nrhs == 1`` else ``[nrhs, m]`` (one right-hand side per row).

    ``zero_sum``: the values of every random row are centred to sum to zero (the same
    draws, minus their row mean).  Every random row then annihilates constant vectors,
    so C = A^T A behaves like a graph Laplacian whose near null space (smooth, slowly
    varying vectors) is lifted only by the 1e-2 I rows: a hard case for one-level
    Schwarz, which the coarse space is there to fix.
    """
    n = W * H
    m_rand = rows_per_point * n
    m = m_rand + n
    w = 2 * radius + 1
    if k > (radius + 1) ** 2:
        raise ValueError("a corner window must hold at least k points")
    rng = np.random.default_rng(seed)
    cx = rng.integers(0, W, size=m_rand)
    cy = rng.integers(0, H, size=m_rand)
    dx, dy = _window_offsets(radius)
    cols = np.empty((m_rand, k), dtype=np.int64)
    for s in range(0, m_rand, _CHUNK):
        e = min(m_rand, s + _CHUNK)
        keys = rng.random((e - s, w * w))
        gx = cx[s:e, None] + dx[None, :]
        gy = cy[s:e, None] + dy[None, :]
        valid = (gx >= 0) & (gx < W) & (gy >= 0) & (gy < H)
        keys[~valid] = 2.0
        pick = np.argpartition(keys, k - 1, axis=1)[:, :k]
        px = np.take_along_axis(gx, pick, axis=1)
        py = np.take_along_axis(gy, pick, axis=1)
        cols[s:e] = np.sort(py * W + px, axis=1)
    vals = rng.standard_normal((m_rand, k))
    if zero_sum:
        vals = vals - vals.mean(axis=1, keepdims=True)

    row_ptr = np.empty(m + 1, dtype=np.int64)
    row_ptr[: m_rand + 1] = np.arange(m_rand + 1, dtype=np.int64) * k
    row_ptr[m_rand + 1:] = m_rand * k + np.arange(1, n + 1, dtype=np.int64)
    col = np.concatenate([cols.reshape(-1), np.arange(n, dtype=np.int64)]).astype(np.int32)
    val = np.concatenate([vals.reshape(-1), np.full(n, ident_scale)])
    if col_scale:
        u = np.random.default_rng(seed + 3).uniform(-3.0, 3.0, size=n)
        val = val * np.power(10.0, u)[col]
    rb = np.random.default_rng(seed + 1)
    b = rb.standard_normal(m) if nrhs == 1 else rb.standard_normal((nrhs, m))
    xstar = np.random.default_rng(seed + 2).standard_normal(n) if with_xstar else None
    return m, n, row_ptr, col, val, b, xstar


def strip_partition(W: int, H: int, rows_per_strip: int) -> np.ndarray:
    """Strips of ``rows_per_strip`` full grid rows: strip i = grid rows [i*r, (i+1)*r)."""
    gy = np.arange(W * H) // W
    return (gy // rows_per_strip).astype(np.int32)


def block_partition(W: int, H: int, bw: int, bh: int) -> np.ndarray:
    """Rectangular bw x bh blocks; block (bx, by) has id by * ceil(W / bw) + bx."""
    j = np.arange(W * H)
    gx, gy = j % W, j // W
    nbx = -(-W // bw)
    return ((gy // bh) * nbx + gx // bw).astype(np.int32)


def bisection_partition(W: int, H: int, max_cols: int, seed: int) -> np.ndarray:
    """Seeded recursive coordinate bisection into uneven rectangles of <= max_cols points.

    The longer side of a rectangle is cut at a fraction drawn from U(0.35, 0.65),
    rounded to a grid line, until every piece holds at most ``max_cols`` grid
    points.  Pieces are numbered depth first, lower/left piece first.
    """
    rng = np.random.default_rng(seed)
    part = np.empty(W * H, dtype=np.int32)
    nxt = [0]

    def rec(x0, x1, y0, y1):
        if (x1 - x0) * (y1 - y0) <= max_cols:
            ys, xs = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
            part[(ys * W + xs).reshape(-1)] = nxt[0]
            nxt[0] += 1
            return
        f = rng.uniform(0.35, 0.65)
        if (x1 - x0) >= (y1 - y0):
            c = min(max(x0 + int(round(f * (x1 - x0))), x0 + 1), x1 - 1)
            rec(x0, c, y0, y1)
            rec(c, x1, y0, y1)
        else:
            c = min(max(y0 + int(round(f * (y1 - y0))), y0 + 1), y1 - 1)
            rec(x0, x1, y0, c)
            rec(x0, x1, c, y1)

    rec(0, W, 0, H)
    return part


def _pack(name, W, H, m, n, row_ptr, col, val, b, xstar, part) -> GridLS:
    return GridLS(m=m, n=n, row_ptr=row_ptr, col=col, val=val, part=part,
                  nparts=int(part.max()) + 1, b=b, xstar=xstar, W=W, H=H, name=name)


def config_tiny(seed: int = 0) -> GridLS:
    """n = 1024 on a 32x32 grid, 4096 rows of 4 nonzeros (radius 2) + 1e-2 I, 8 strips of 32x4."""
    W = H = 32
    m, n, rp, c, v, b, xs = make_grid_ls(W, H, 4, 4, 2, seed, with_xstar=True)
    return _pack("tiny-n1024-N8", W, H, m, n, rp, c, v, b, xs, strip_partition(W, H, 4))


def config_scale(side: int = 1024, block: int = 64, seed: int = 0, col_scale: bool = False,
                 name: str | None = None, zero_sum: bool = False) -> GridLS:
    """Grid side x side, 4n rows of 8 nonzeros (radius 3) + 1e-2 I, square block subdomains.

    side = 1024, block = 64 is the n = 1,048,576 / 256-subdomain workload; block 128
    and 32 give 64 and 1024 subdomains.
    """
    W = H = side
    m, n, rp, c, v, b, xs = make_grid_ls(W, H, 4, 8, 3, seed, col_scale=col_scale, zero_sum=zero_sum)
    nm = name or f"grid{side}-r3k8-N{(side // block) ** 2}" + ("-colscale" if col_scale else "") + \
        ("-zerosum" if zero_sum else "")
    return _pack(nm, W, H, m, n, rp, c, v, b, xs, block_partition(W, H, block, block))


def config_precision(side: int = 1024, block: int = 64, seed: int = 0) -> GridLS:
    """The scale workload with every column j scaled by 10**u_j, u_j ~ U(-3, 3)."""
    return config_scale(side, block, seed, col_scale=True)


def config_diff(side: int = 512, block: int = 64, seed: int = 0) -> GridLS:
    """n = 262,144 on 512x512, 4n rows of 8 nonzeros (radius 3) + 1e-2 I, 64 subdomains, x* drawn."""
    W = H = side
    m, n, rp, c, v, b, xs = make_grid_ls(W, H, 4, 8, 3, seed, with_xstar=True)
    return _pack(f"diff-grid{side}-N{(side // block) ** 2}", W, H, m, n, rp, c, v, b, xs,
                 block_partition(W, H, block, block))


def config_batch_sizes(nprob: int = 64, lo: int = 16384, hi: int = 262144, seed: int = 999):
    """Grid sides of the batched workload: n log-uniform in [lo, hi], side = round(sqrt(n))."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(lo), math.log(hi), size=nprob))
    return [int(round(math.sqrt(x))) for x in ns]


@dataclasses.dataclass
class BatchLS:
    """Independent problems stored as one block-diagonal CSR matrix: problem q owns the
    rows [m_off[q], m_off[q+1]) and the columns [n_off[q], n_off[q+1]); its subdomain
    ids follow those of problem q - 1.  b has shape [nrhs, m]."""
    m: int
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    part: np.ndarray
    nparts: int
    b: np.ndarray
    m_off: np.ndarray
    n_off: np.ndarray
    sides: list
    name: str

    @property
    def nprob(self) -> int:
        return len(self.sides)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def problem(self, q: int):
        """(m, n, row_ptr, col, val, part, nparts, b) of problem q alone (local indices)."""
        r0, r1 = int(self.m_off[q]), int(self.m_off[q + 1])
        c0, c1 = int(self.n_off[q]), int(self.n_off[q + 1])
        e0, e1 = int(self.row_ptr[r0]), int(self.row_ptr[r1])
        part = self.part[c0:c1]
        p0 = int(part.min())
        return (r1 - r0, c1 - c0, self.row_ptr[r0:r1 + 1] - e0, self.col[e0:e1] - c0, self.val[e0:e1],
                (part - p0).astype(np.int32), int(part.max()) - p0 + 1, self.b[:, r0:r1])


def config_batch(nprob: int = 64, nrhs: int = 32, lo: int = 16384, hi: int = 262144, max_cols: int = 8192,
                 size_seed: int = 999, name: str | None = None) -> BatchLS:
    """Batched workload: nprob square grids with n log-uniform in [lo, hi] (sizes from
    size_seed), each 4n random rows of 6 nonzeros within radius 2 (seed 1000 + q) plus
    1e-2 I rows, nrhs right-hand sides b ~ N(0, 1), and uneven subdomains from seeded
    recursive bisection (seed 2000 + q) into pieces of at most max_cols columns."""
    sides = config_batch_sizes(nprob, lo, hi, size_seed)
    rps, cols, vals, parts, bs = [], [], [], [], []
    m_off, n_off = [0], [0]
    nparts = 0
    for q, s in enumerate(sides):
        m, n, rp, c, v, b, _ = make_grid_ls(s, s, 4, 6, 2, 1000 + q, nrhs=nrhs)
        part = bisection_partition(s, s, max_cols, 2000 + q)
        nnz_before = (rps[-1][-1] if rps else 0)
        rps.append((rp[1:] if rps else rp) + nnz_before)
        cols.append(c + n_off[-1])
        vals.append(v)
        parts.append(part + nparts)
        nparts += int(part.max()) + 1
        bs.append(b.reshape(nrhs, m))
        m_off.append(m_off[-1] + m)
        n_off.append(n_off[-1] + n)
    row_ptr = np.concatenate(rps).astype(np.int64)
    return BatchLS(m=m_off[-1], n=n_off[-1], row_ptr=row_ptr, col=np.concatenate(cols).astype(np.int32),
                   val=np.concatenate(vals), part=np.concatenate(parts).astype(np.int32), nparts=nparts,
                   b=np.concatenate(bs, axis=1), m_off=np.array(m_off, np.int64), n_off=np.array(n_off, np.int64),
                   sides=sides, name=name or f"batch{nprob}x{nrhs}-n[{lo},{hi}]-r2k6-sub{max_cols}")


def paper_example():
    """The 5x4 worked example of Section 3 with Omega_I1 = {1, 3}, Omega_I2 = {2, 4} (1-based)."""
    A = np.array([[1, 0, 6, 0],
                  [2, 4, 0, 0],
                  [3, 0, 0, 0],
                  [0, 5, 0, 7],
                  [0, 0, 0, 8]], dtype=np.float64)
    part = np.array([0, 1, 0, 1], dtype=np.int32)
    return A, part


def csr_from_dense(A: np.ndarray):
    """CSR arrays (int64 row_ptr, int32 col, float64 val) of the structurally nonzero entries."""
    mask = A != 0
    row_ptr = np.concatenate([[0], np.cumsum(mask.sum(axis=1))]).astype(np.int64)
    rows, cols = np.nonzero(mask)
    return row_ptr, cols.astype(np.int32), A[rows, cols].astype(np.float64)
