"""Seeded synthetic inputs for the sparse-fusion hot path.

This module only draws inputs: CSR patterns, their values and the right-hand sides.
It holds none of the method's arithmetic (no solve, no product, no factorisation, no
level, order or partition computation), so the oracle tests, the GPU tests and the
benchmark can all share it without the oracle and the CUDA path sharing code.

The paper measures on SuiteSparse SPD matrices (Table 1, §4) that are not available
here; the workloads below are synthetic stand-ins with the shapes, sizes, row-length
distributions and dependence depths described for each one.

Random numbers come from a counter-based generator: the SplitMix64 output function
(Steele, Lea and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014)
applied to the 64-bit counter ``seed*G1 + stream*G2 + index``. Every value is a pure
function of (seed, stream, index), so results are identical on any machine and for any
chunking of the work.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_M64 = (1 << 64) - 1
_G1 = 0x9E3779B97F4A7C15
_G2 = 0xD1B54A32D192ED03

# stream ids: one per kind of draw, so that no two draws share counters
S_PATTERN, S_VALUES, S_RHS, S_XIN, S_GRAD, S_LEN, S_KEYS, S_SIZE = range(1, 9)


# --------------------------------------------------------------------------- rng
def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = x + np.uint64(_G1)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _bits(seed: int, stream: int, idx) -> np.ndarray:
    base = np.uint64((seed * _G1 + stream * _G2) & _M64)
    i = np.asarray(idx).astype(np.uint64)
    return splitmix64(i + base)


def uniform01(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (_bits(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_pm1(seed: int, stream: int, idx) -> np.ndarray:
    """Uniform doubles in [-1, 1); exact (2u - 1 is representable)."""
    return 2.0 * uniform01(seed, stream, idx) - 1.0


def uniform_below(seed: int, stream: int, idx, bound) -> np.ndarray:
    """Integers uniform in [0, bound) by multiply-shift of the top 32 bits (bound < 2**32)."""
    hi = _bits(seed, stream, idx) >> np.uint64(32)
    b = np.asarray(bound).astype(np.uint64)
    return ((hi * b) >> np.uint64(32)).astype(np.int64)


# --------------------------------------------------------------------------- csr
@dataclass
class Csr:
    """CSR matrix: int32 rowptr[n_rows+1], int32 colidx[nnz] (ascending in each row),
    float64 vals[nnz]."""
    n_rows: int
    n_cols: int
    rowptr: np.ndarray
    colidx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.rowptr.astype(np.int64))


def _rowptr_from_lengths(lengths: np.ndarray) -> np.ndarray:
    rp = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=rp[1:])
    if rp[-1] >= 2 ** 31:
        raise ValueError("nnz must stay below 2**31 for int32 CSR")
    return rp


def _row_of_entry(rowptr: np.ndarray) -> np.ndarray:
    n = len(rowptr) - 1
    return np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))


def _entries_of_rows(rowptr: np.ndarray, rows: np.ndarray) -> np.ndarray:
    starts = rowptr[rows]
    lens = rowptr[rows + 1] - starts
    tot = int(lens.sum())
    if tot == 0:
        return np.zeros(0, dtype=np.int64)
    excl = np.zeros(len(rows), dtype=np.int64)
    np.cumsum(lens[:-1], out=excl[1:])
    return np.repeat(starts - excl, lens) + np.arange(tot, dtype=np.int64)


def _sort_within_rows(rowptr: np.ndarray, cols: np.ndarray, n_cols: int) -> np.ndarray:
    rows = _row_of_entry(rowptr)
    key = rows * np.int64(n_cols + 1) + cols
    return cols[np.argsort(key, kind="stable")]


def _distinct_columns(seed: int, stream: int, rowptr: np.ndarray, draw, valid) -> np.ndarray:
    """Draw one column per entry with ``draw(entries, round)``, redrawing entries whose
    column is invalid for its row or repeats a column already in the row."""
    rows = _row_of_entry(rowptr)
    E = len(rows)
    cols = draw(np.arange(E, dtype=np.int64), 0)
    rnd = 1
    check = np.arange(E, dtype=np.int64)
    n_big = np.int64(1 << 32)
    while True:
        bad = check[~valid(rows[check], cols[check])]
        while bad.size:
            cols[bad] = draw(bad, rnd)
            rnd += 1
            bad = bad[~valid(rows[bad], cols[bad])]
        urows = np.unique(rows[check])
        ent = _entries_of_rows(rowptr, urows)
        key = rows[ent] * n_big + cols[ent]
        srt = np.argsort(key, kind="stable")
        ks = key[srt]
        dup = ent[srt[1:][ks[1:] == ks[:-1]]]
        if dup.size == 0:
            return cols
        cols[dup] = draw(dup, rnd)
        rnd += 1
        check = dup


# --------------------------------------------------------------------------- stencils
def _stencil_pattern(dims, offsets):
    """Pattern of a stencil on a grid in natural order (x fastest). ``offsets`` is a list
    of integer vectors; entries outside the grid are dropped. Columns come out ascending."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    coords = np.indices(dims[::-1]).reshape(len(dims), -1)[::-1]  # coords[a][p]
    lin = [sum(o[a] * strides[a] for a in range(len(dims))) for o in offsets]
    offs = [o for _, o in sorted(zip(lin, offsets))]
    lin = sorted(lin)
    masks = []
    for o in offs:
        m = np.ones(n, dtype=bool)
        for a in range(len(dims)):
            c = coords[a] + o[a]
            m &= (c >= 0) & (c < dims[a])
        masks.append(m)
    M = np.stack(masks, axis=1)  # n x n_off
    lengths = M.sum(axis=1)
    rowptr = _rowptr_from_lengths(lengths)
    p = np.arange(n, dtype=np.int64)[:, None] + np.asarray(lin, dtype=np.int64)[None, :]
    cols = p[M]
    return n, rowptr, cols, [tuple(o) for o in offs], M


def _finish(n_rows, n_cols, rowptr, cols, vals) -> Csr:
    return Csr(n_rows, n_cols, rowptr.astype(np.int32), cols.astype(np.int32),
               np.ascontiguousarray(vals, dtype=np.float64))


def _diag_dominant_values(seed, stream, rowptr, cols):
    """Off-diagonals uniform[-1,1]; diagonal = 1 + sum of |off-diagonals| of the same row."""
    rows = _row_of_entry(rowptr)
    v = uniform_pm1(seed, stream, np.arange(len(cols), dtype=np.int64))
    isdiag = cols == rows
    v[isdiag] = 0.0
    s = np.bincount(rows, weights=np.abs(v), minlength=len(rowptr) - 1)
    v[isdiag] = 1.0 + s[rows[isdiag]]
    return v


def grid_lower_laplacian(dims, seed: int, stream: int = S_VALUES) -> Csr:
    """Lower triangle of the 5-point (2D) or 7-point (3D) Laplacian pattern with seeded
    uniform[-1,1] off-diagonals and diagonal 1 + sum|off-diagonals| of the row."""
    nd = len(dims)
    offs = [tuple(0 for _ in range(nd))]
    for a in range(nd):
        o = [0] * nd
        o[a] = -1
        offs.append(tuple(o))
    n, rowptr, cols, _, _ = _stencil_pattern(dims, offs)
    return _finish(n, n, rowptr, cols, _diag_dominant_values(seed, stream, rowptr, cols))


def grid_full_stencil_random(dims, seed: int, stream: int = S_VALUES) -> Csr:
    """Full 5-point / 7-point pattern with every value (diagonal included) uniform[-1,1]."""
    nd = len(dims)
    offs = [tuple(0 for _ in range(nd))]
    for a in range(nd):
        for s in (-1, 1):
            o = [0] * nd
            o[a] = s
            offs.append(tuple(o))
    n, rowptr, cols, _, _ = _stencil_pattern(dims, offs)
    return _finish(n, n, rowptr, cols, uniform_pm1(seed, stream, np.arange(len(cols))))


def aniso_laplacian_3d(dims, coeffs=(1.0, 10.0, 100.0), diag=222.001) -> Csr:
    """Anisotropic 7-point Laplacian with Dirichlet boundary: -c_a on the +-a neighbours
    (x fastest), the same diagonal on every row (out-of-grid neighbours dropped)."""
    offs = [(0, 0, 0)]
    for a in range(3):
        for s in (-1, 1):
            o = [0, 0, 0]
            o[a] = s
            offs.append(tuple(o))
    n, rowptr, cols, soffs, M = _stencil_pattern(dims, offs)
    per_off = []
    for o in soffs:
        if o == (0, 0, 0):
            per_off.append(diag)
        else:
            a = [i for i in range(3) if o[i] != 0][0]
            per_off.append(-coeffs[a])
    vals = np.broadcast_to(np.asarray(per_off), M.shape)[M]
    return _finish(n, n, rowptr, cols, vals)


def lower_part(A: Csr) -> Csr:
    """tril(A) as its own CSR (structural selection, columns stay ascending)."""
    rows = _row_of_entry(A.rowptr.astype(np.int64))
    keep = A.colidx.astype(np.int64) <= rows
    lengths = np.bincount(rows[keep], minlength=A.n_rows)
    rp = _rowptr_from_lengths(lengths)
    return _finish(A.n_rows, A.n_cols, rp, A.colidx[keep].astype(np.int64), A.vals[keep])


# --------------------------------------------------------------------------- random patterns
def band_random(n: int, per_row: int, halfband: int, seed: int,
                stream_pat: int = S_PATTERN, stream_val: int = S_VALUES) -> Csr:
    """``per_row`` distinct columns per row at integer offsets uniform in
    [-halfband, halfband] (diagonal allowed); offsets landing outside [0, n) or repeating
    a column of the row are redrawn. Values uniform[-1,1]."""
    if per_row > min(n, 2 * halfband + 1):
        raise ValueError("per_row too large for the band")
    rowptr = _rowptr_from_lengths(np.full(n, per_row, dtype=np.int64))
    rows = _row_of_entry(rowptr)
    E = len(rows)
    width = 2 * halfband + 1

    def draw(ent, rnd):
        return rows[ent] - halfband + uniform_below(seed, stream_pat, ent + np.int64(rnd) * E, width)

    def valid(r, c):
        return (c >= 0) & (c < n)

    cols = _distinct_columns(seed, stream_pat, rowptr, draw, valid)
    cols = _sort_within_rows(rowptr, cols, n)
    return _finish(n, n, rowptr, cols, uniform_pm1(seed, stream_val, np.arange(E)))


def powerlaw_alpha(mean: float, lmax: int) -> float:
    """Exponent a of P(l) ~ l^-a on [1, lmax] with E[l] = mean (bisection, pure Python)."""
    def m(a):
        w = [l ** (-a) for l in range(1, lmax + 1)]
        return sum(l * wl for l, wl in zip(range(1, lmax + 1), w)) / sum(w)
    lo, hi = 0.0, 6.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if m(mid) > mean:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def powerlaw_lengths(n: int, mean: float, lmax: int, seed: int, stream: int = S_LEN) -> np.ndarray:
    """Row lengths drawn from the truncated discrete power law with the given mean."""
    a = powerlaw_alpha(mean, lmax)
    w = [l ** (-a) for l in range(1, lmax + 1)]
    tot = math.fsum(w)
    cdf, acc = [], 0.0
    for wl in w:
        acc += wl
        cdf.append(acc / tot)
    cdf[-1] = 1.0
    u = uniform01(seed, stream, np.arange(n, dtype=np.int64))
    return np.searchsorted(np.asarray(cdf), u, side="right").astype(np.int64) + 1


def powerlaw_lower(n: int, mean: float, lmax: int, seed: int) -> Csr:
    """Random lower-triangular CSR: row i has l_i (power law, diagonal included, clamped
    to i+1) entries; off-diagonal columns distinct and uniform in [0, i); off-diagonals
    uniform[-1,1]; diagonal 1 + sum|off-diagonals|."""
    ell = np.minimum(powerlaw_lengths(n, mean, lmax, seed), np.arange(n, dtype=np.int64) + 1)
    m = ell - 1                                     # off-diagonal count per row
    rp_off = _rowptr_from_lengths(m)
    rows = _row_of_entry(rp_off)
    E = len(rows)
    cols = np.zeros(E, dtype=np.int64)
    dense = (m > 0) & (2 * m >= np.arange(n))       # rows taking at least half of [0, i)
    # dense rows: the m_i smallest of i random keys, one per candidate column
    drows = np.nonzero(dense)[0]
    if drows.size:
        cand_rp = _rowptr_from_lengths(drows.astype(np.int64))
        crow = np.repeat(drows, drows)
        ccol = np.arange(int(cand_rp[-1]), dtype=np.int64) - np.repeat(cand_rp[:-1], drows)
        keys = _bits(seed, S_KEYS, crow * np.int64(1 << 20) + ccol)
        srt = np.lexsort((keys, crow))
        rank = np.arange(len(srt), dtype=np.int64) - np.repeat(cand_rp[:-1], drows)
        take = rank < np.repeat(m[drows], drows)
        picked = ccol[srt][take]
        cols[_entries_of_rows(rp_off, drows)] = picked
    sparse_rows = np.nonzero((m > 0) & ~dense)[0]
    if sparse_rows.size:
        sub_m = m[sparse_rows]
        sub_rp = _rowptr_from_lengths(sub_m)
        sub_rows = sparse_rows[_row_of_entry(sub_rp)]
        gent = _entries_of_rows(rp_off, sparse_rows)

        def draw(ent, rnd):
            return uniform_below(seed, S_PATTERN, gent[ent] + np.int64(rnd) * E, sub_rows[ent])

        def valid(r, c):
            return np.ones(len(r), dtype=bool)

        cols[gent] = _distinct_columns(seed, S_PATTERN, sub_rp, draw, valid)
    # add the diagonal and sort each row
    rowptr = _rowptr_from_lengths(ell)
    allrows = _row_of_entry(rowptr)
    full = np.empty(int(rowptr[-1]), dtype=np.int64)
    isdiag_pos = rowptr[1:] - 1                     # diagonal goes last after sorting
    offmask = np.ones(len(full), dtype=bool)
    offmask[isdiag_pos] = False
    full[offmask] = cols
    full[isdiag_pos] = np.arange(n, dtype=np.int64)
    full = _sort_within_rows(rowptr, full, n)
    del allrows
    return _finish(n, n, rowptr, full, _diag_dominant_values(seed, S_VALUES, rowptr, full))


def powerlaw_band(n: int, mean: float, lmax: int, halfband: int, seed: int) -> Csr:
    """Square CSR with power-law row lengths (diagonal included); off-diagonal columns
    distinct and uniform in [max(0,i-h), min(n,i+h+1)) minus {i}; off-diagonals
    uniform[-1,1]; diagonal 1 + sum|off-diagonals| of the row."""
    lo = np.maximum(0, np.arange(n, dtype=np.int64) - halfband)
    hi = np.minimum(n, np.arange(n, dtype=np.int64) + halfband + 1)
    win = hi - lo - 1
    ell = np.minimum(powerlaw_lengths(n, mean, lmax, seed), win + 1)
    m = ell - 1
    if np.any(2 * m > win):
        raise ValueError("band too narrow for the row lengths")
    rp_off = _rowptr_from_lengths(m)
    rows = _row_of_entry(rp_off)
    E = len(rows)

    def draw(ent, rnd):
        r = rows[ent]
        c = lo[r] + uniform_below(seed, S_PATTERN, ent + np.int64(rnd) * E, win[r])
        return c + (c >= r)

    def valid(r, c):
        return np.ones(len(r), dtype=bool)

    cols = _distinct_columns(seed, S_PATTERN, rp_off, draw, valid)
    rowptr = _rowptr_from_lengths(ell)
    full = np.empty(int(rowptr[-1]), dtype=np.int64)
    offmask = np.ones(len(full), dtype=bool)
    offmask[rowptr[1:] - 1] = False
    full[offmask] = cols
    full[rowptr[1:] - 1] = np.arange(n, dtype=np.int64)
    full = _sort_within_rows(rowptr, full, n)
    return _finish(n, n, rowptr, full, _diag_dominant_values(seed, S_VALUES, rowptr, full))


def dense_vectors(n: int, k: int, seed: int, stream: int) -> np.ndarray:
    """n x k row-major block of uniform[-1,1] values."""
    return uniform_pm1(seed, stream, np.arange(n * k, dtype=np.int64)).reshape(n, k)


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """floor(exp(U(ln lo, ln(hi+1)))) for each instance, clamped to [lo, hi]."""
    u = uniform01(seed, S_SIZE, np.arange(count, dtype=np.int64))
    a, b = math.log(lo), math.log(hi + 1)
    out = [min(hi, max(lo, int(math.floor(math.exp(a + (b - a) * float(x)))))) for x in u]
    return np.asarray(out, dtype=np.int64)


# --------------------------------------------------------------------------- workloads
@dataclass
class Workload:
    """One problem instance (or a batch). ``pair`` is 'trsv_spmv', 'spmv_trsv' or
    'ic0_trsv'. For 'ic0_trsv' L holds tril(A) (the matrix to factor); for 'spmv_trsv'
    L = tril(A) and M = A; for 'trsv_spmv' M is the SpMV operand."""
    name: str
    pair: str
    n: int
    k: int
    L: Csr
    M: Optional[Csr]
    b: np.ndarray
    x_in: Optional[np.ndarray] = None
    gy: Optional[np.ndarray] = None
    instances: List["Workload"] = field(default_factory=list)


def trsv_spmv_lap2d(nx: int = 64, seed: int = 1) -> Workload:
    """SpTRSV then SpMV on a 2D grid: L = lower 5-point pattern (diagonally dominant
    random values), M = full 5-point pattern (uniform values), 1 RHS."""
    L = grid_lower_laplacian((nx, nx), seed)
    M = grid_full_stencil_random((nx, nx), seed, stream=S_VALUES + 100)
    n = L.n_rows
    return Workload(f"trsv_spmv_lap2d_{nx}x{nx}", "trsv_spmv", n, 1, L, M,
                    dense_vectors(n, 1, seed, S_RHS), gy=dense_vectors(n, 1, seed, S_GRAD))


def trsv_spmv_lap3d_band(nx: int = 128, per_row: int = 8, halfband: int = 1000,
                         seed: int = 2, k: int = 1) -> Workload:
    """SpTRSV then SpMV: L = lower 7-point pattern on an nx^3 grid (diagonally dominant
    random values), M = random band matrix with ``per_row`` entries at offsets within
    +-halfband (uniform values)."""
    L = grid_lower_laplacian((nx, nx, nx), seed)
    n = L.n_rows
    hb = min(halfband, n)
    M = band_random(n, min(per_row, n, 2 * hb + 1), hb, seed, stream_val=S_VALUES + 100)
    return Workload(f"trsv_spmv_lap3d_{nx}^3_band{halfband}", "trsv_spmv", n, k, L, M,
                    dense_vectors(n, k, seed, S_RHS), gy=dense_vectors(n, k, seed, S_GRAD))


def ic0_trsv_aniso3d(nx: int = 100, k: int = 32, seed: int = 3) -> Workload:
    """SpIC0 then SpTRSV: A = anisotropic 7-point Laplacian on nx^3 (coefficients
    1, 10, 100 and diagonal 222.001); L holds tril(A); k uniform right-hand sides."""
    A = aniso_laplacian_3d((nx, nx, nx))
    L = lower_part(A)
    n = A.n_rows
    return Workload(f"ic0_trsv_aniso3d_{nx}^3_k{k}", "ic0_trsv", n, k, L, None,
                    dense_vectors(n, k, seed, S_RHS))


def spmv_trsv_powerlaw(n: int = 1 << 22, k: int = 16, mean: float = 16.0, lmax: int = 2000,
                       halfband: int = 5000, seed: int = 5) -> Workload:
    """SpMV then SpTRSV (one Gauss-Seidel half-sweep z = tril(A)^-1 (b - A x_in)) on a
    square matrix with power-law rows and columns in a +-halfband band."""
    A = powerlaw_band(n, mean, lmax, halfband, seed)
    L = lower_part(A)
    return Workload(f"spmv_trsv_powerlaw_n{n}_k{k}", "spmv_trsv", n, k, L, A,
                    dense_vectors(n, k, seed, S_RHS), x_in=dense_vectors(n, k, seed, S_XIN),
                    gy=dense_vectors(n, k, seed, S_GRAD))


def batched_trsv_spmv(count: int = 512, nmin: int = 1024, nmax: int = 65536,
                      mean: float = 8.0, lmax: int = 256, seed: int = 4, k: int = 1) -> Workload:
    """``count`` independent SpTRSV-then-SpMV instances with log-uniform sizes; L and M
    are independently seeded power-law lower-triangular matrices."""
    sizes = log_uniform_sizes(count, nmin, nmax, seed)
    inst = []
    for t, nt in enumerate(sizes):
        s = seed * 100003 + t
        L = powerlaw_lower(int(nt), mean, lmax, s)
        M = powerlaw_lower(int(nt), mean, lmax, s + 7919 * 1000003)
        inst.append(Workload(f"inst{t}", "trsv_spmv", int(nt), k, L, M,
                             dense_vectors(int(nt), k, s, S_RHS),
                             gy=dense_vectors(int(nt), k, s, S_GRAD)))
    n = int(sizes.sum())
    b = np.concatenate([w.b for w in inst], axis=0)
    gy = np.concatenate([w.gy for w in inst], axis=0)
    return Workload(f"batched_trsv_spmv_{count}x[{nmin},{nmax}]", "trsv_spmv", n, k,
                    inst[0].L, inst[0].M, b, gy=gy, instances=inst)
