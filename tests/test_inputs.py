"""Pins of the seeded input generators (CPU): the counter-based random numbers against the
published SplitMix64 sequence, the power-law exponents against the defining mean, and the
stencil, band and power-law patterns and values against the recipes they implement."""
import math

import numpy as np
import pytest

from paper_2111_12238_gb300 import inputs as I

M64 = (1 << 64) - 1


def test_splitmix64_matches_the_published_sequence():
    # SplitMix64 started at state 0 (Steele, Lea and Flood, OOPSLA 2014): the state advances by
    # the golden gamma before each output
    g = 0x9E3779B97F4A7C15
    states = np.array([0, g, (2 * g) & M64], dtype=np.uint64)
    assert [int(v) for v in I.splitmix64(states)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_draws_are_in_range_and_reproducible():
    idx = np.arange(200000)
    u = I.uniform01(7, I.S_VALUES, idx)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert np.all(u * 2.0 ** 53 == np.floor(u * 2.0 ** 53))            # 53-bit grid
    assert abs(u.mean() - 0.5) < 0.005
    assert np.array_equal(u, I.uniform01(7, I.S_VALUES, idx))          # a pure function of the counter
    assert not np.array_equal(u[:100], I.uniform01(7, I.S_RHS, idx[:100]))
    p = I.uniform_pm1(7, I.S_VALUES, idx)
    assert np.array_equal(p, 2.0 * u - 1.0)
    k = I.uniform_below(7, I.S_PATTERN, idx, 10)
    assert k.min() == 0 and k.max() == 9
    assert np.all(np.abs(np.bincount(k, minlength=10) / len(k) - 0.1) < 0.005)


@pytest.mark.parametrize("mean,lmax,alpha", [(8.0, 256, 1.6648), (16.0, 2000, 1.6773)])
def test_powerlaw_exponent_gives_the_mean(mean, lmax, alpha):
    a = I.powerlaw_alpha(mean, lmax)
    assert a == pytest.approx(alpha, abs=5e-5)
    ell = np.arange(1, lmax + 1, dtype=np.float64)
    w = ell ** (-a)
    assert float((ell * w).sum() / w.sum()) == pytest.approx(mean, rel=1e-9)
    lens = I.powerlaw_lengths(400000, mean, lmax, 11)
    assert lens.min() >= 1 and lens.max() <= lmax
    assert lens.mean() == pytest.approx(mean, rel=0.03)


def test_grid_lower_laplacian_pattern_and_values():
    nx, ny = 7, 5
    L = I.grid_lower_laplacian((nx, ny), seed=1)
    n = nx * ny
    assert L.n_rows == n and L.nnz == n + (nx - 1) * ny + nx * (ny - 1)
    for i in range(n):
        cols = L.colidx[L.rowptr[i]:L.rowptr[i + 1]].tolist()
        vals = L.vals[L.rowptr[i]:L.rowptr[i + 1]]
        x, y = i % nx, i // nx
        want = ([i - nx] if y > 0 else []) + ([i - 1] if x > 0 else []) + [i]
        assert cols == want
        assert vals[-1] == pytest.approx(1.0 + np.abs(vals[:-1]).sum(), rel=1e-14)
        assert np.all(np.abs(vals[:-1]) <= 1.0)


def test_aniso_laplacian_values():
    A = I.aniso_laplacian_3d((4, 3, 2))
    nx, ny = 4, 3
    D = np.zeros((A.n_rows, A.n_cols))
    for i in range(A.n_rows):
        D[i, A.colidx[A.rowptr[i]:A.rowptr[i + 1]]] = A.vals[A.rowptr[i]:A.rowptr[i + 1]]
    assert np.all(np.diag(D) == 222.001)
    assert np.array_equal(D, D.T)
    i = 1 + nx * 1 + nx * ny * 0          # (1, 1, 0)
    assert (D[i, i - 1], D[i, i + 1], D[i, i - nx], D[i, i + nx], D[i, i + nx * ny]) == (-1, -1, -10, -10, -100)
    assert set(np.unique(D[D != 0])) <= {-1.0, -10.0, -100.0, 222.001}


def test_band_random_rows():
    n, per_row, h = 3000, 8, 40
    M = I.band_random(n, per_row, h, seed=2)
    assert np.all(np.diff(M.rowptr) == per_row)
    rows = np.repeat(np.arange(n), per_row)
    off = M.colidx.astype(np.int64) - rows
    assert np.all(np.abs(off) <= h) and M.colidx.min() >= 0 and M.colidx.max() < n
    for i in range(0, n, 97):
        c = M.colidx[M.rowptr[i]:M.rowptr[i + 1]]
        assert np.all(np.diff(c) > 0)                                      # distinct, ascending


def test_powerlaw_lower_rows():
    n = 4000
    L = I.powerlaw_lower(n, 8, 256, 4)
    lens = np.diff(L.rowptr)
    assert lens.min() >= 1 and lens.max() <= 256 and np.all(lens <= np.arange(n) + 1)
    for i in range(0, n, 61):
        c = L.colidx[L.rowptr[i]:L.rowptr[i + 1]]
        v = L.vals[L.rowptr[i]:L.rowptr[i + 1]]
        assert c[-1] == i and np.all(np.diff(c) > 0)
        assert v[-1] == pytest.approx(1.0 + np.abs(v[:-1]).sum(), rel=1e-14)


def test_log_uniform_sizes():
    s = I.log_uniform_sizes(20000, 1024, 65536, 4)
    assert s.min() >= 1024 and s.max() <= 65536
    mid = 0.5 * (math.log(1024) + math.log(65537))
    assert float(np.log(s).mean()) == pytest.approx(mid, abs=0.03)
