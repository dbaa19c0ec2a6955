"""Pins of the oracle's kernels against what mathematics fixes independently of it:
dense triangular solves and Cholesky (library routines on tiny dense inputs), exact
integer arithmetic, closed forms and the defining invariant of zero fill-in IC.
CPU only."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2111_12238_gb300 import inputs as I
from tests._mats import (csr_to_dense, dense_to_csr, pattern_dense, random_lower, random_square,
                         rel_err)


@pytest.mark.parametrize("n,density,k,seed", [(1, 0.5, 1, 1), (7, 0.4, 1, 2), (33, 0.2, 3, 3),
                                               (64, 0.1, 2, 4), (64, 0.9, 1, 5)])
def test_trsv_matches_dense_triangular_solve(n, density, k, seed):
    D = random_lower(n, density, seed)
    L = dense_to_csr(D)
    b = I.dense_vectors(n, k, seed, I.S_RHS)
    x = oracle.trsv_lower(L, b)
    ref = sla.solve_triangular(D, b, lower=True)
    assert rel_err(x, ref) < 1e-13


def test_trsv_recovers_known_solution():
    # b = L x* with x* exact in binary; forward substitution must give x* back to ~cond*u
    w = I.trsv_spmv_lap3d_band(8, per_row=4, halfband=20, seed=9)
    L = w.L
    xs = I.dense_vectors(L.n_rows, 2, 9, I.S_XIN)
    b = csr_to_dense(L) @ xs
    x = oracle.trsv_lower(L, b)
    assert rel_err(x, xs) < 1e-13


def test_trsv_integer_exact():
    # unit diagonal, entries in {-1,0,1}, integer b: every intermediate is an exact integer
    n = 48
    D = random_lower(n, 0.08, 17, unit_int=True)
    L = dense_to_csr(D)
    b = (np.arange(n) % 7 - 3).astype(np.float64).reshape(n, 1)
    x = oracle.trsv_lower(L, b)
    xi = [0] * n
    for i in range(n):
        s = int(b[i, 0])
        for j in range(i):
            if D[i, j] != 0:
                s -= int(D[i, j]) * xi[j]
        xi[i] = s
    assert max(abs(v) for v in xi) < 2 ** 53
    assert np.array_equal(x[:, 0], np.asarray(xi, dtype=np.float64))


def test_trsv_diagonal_closed_form():
    n = 20
    d = 1.0 + np.arange(n) * 0.37
    L = dense_to_csr(np.diag(d))
    b = I.dense_vectors(n, 3, 4, I.S_RHS)
    x = oracle.trsv_lower(L, b)
    assert np.array_equal(x, b / d[:, None])


def test_trsv_missing_diagonal_is_an_error():
    D = random_lower(6, 0.5, 3)
    P = D != 0
    P[4, 4] = False
    L = dense_to_csr(D, P)
    with pytest.raises(oracle.OracleError) as e:
        oracle.trsv_lower(L, np.ones(6))
    assert e.value.code == -(4 + 1)


def test_spmv_integer_exact_and_identity():
    n = 40
    D = np.round(random_square(n, 0.2, 7) * 10)
    M = dense_to_csr(D)
    x = (np.arange(n * 2) % 11 - 5).astype(np.float64).reshape(n, 2)
    assert np.array_equal(oracle.spmv(M, x), D @ x)
    Id = dense_to_csr(np.eye(n))
    xr = I.dense_vectors(n, 2, 1, I.S_XIN)
    assert np.array_equal(oracle.spmv(Id, xr), xr)
    b = (np.arange(n * 2) % 5).astype(np.float64).reshape(n, 2)
    assert np.array_equal(oracle.residual(M, x, b), b - D @ x)


def test_spmv_rectangular_and_empty_rows():
    D = np.zeros((5, 3))
    D[0, 2] = 2.0
    D[3, 0] = -1.0
    M = dense_to_csr(D)
    x = np.array([1.0, 2.0, 4.0])
    assert np.array_equal(oracle.spmv(M, x)[:, 0], D @ x)


def test_transposed_kernels_match_dense():
    n = 30
    D = random_lower(n, 0.2, 31)
    L = dense_to_csr(D)
    u = I.dense_vectors(n, 2, 31, I.S_GRAD)
    lam = oracle.trsv_lower_T(L, u)
    assert rel_err(lam, sla.solve_triangular(D.T, u, lower=False)) < 1e-13
    S = random_square(n, 0.15, 32)
    M = dense_to_csr(S)
    assert rel_err(oracle.spmv_T(M, u), S.T @ u) < 1e-14


def _ic0_invariant(L, lf):
    P = pattern_dense(L)
    LL = csr_to_dense(L, lf)
    prod = LL @ LL.T
    A = csr_to_dense(L)
    A = A + np.tril(A, -1).T
    Psym = P | P.T
    return np.max(np.abs(prod - A)[Psym]) / np.max(np.abs(A))


@pytest.mark.parametrize("dims", [(6, 5, 4), (9, 9, 9)])
def test_ic0_zero_fill_invariant_aniso(dims):
    A = I.aniso_laplacian_3d(dims)
    L = I.lower_part(A)
    lf = oracle.ic0(L)
    assert _ic0_invariant(L, lf) < 1e-12


def test_ic0_zero_fill_invariant_with_intersections():
    # 9-point 2D pattern: rows i and j = i-nx share column i-nx-1, so the intersection sum
    # in the up-looking update is exercised
    nx = 12
    offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    n, rowptr, cols, soffs, Msk = I._stencil_pattern((nx, nx), offs)
    vals = np.where(np.asarray([o == (0, 0) for o in soffs])[None, :], 9.0, -1.0)
    vals = np.broadcast_to(vals, Msk.shape)[Msk]
    A = I._finish(n, n, rowptr, cols, vals)
    L = I.lower_part(A)
    lf = oracle.ic0(L)
    assert _ic0_invariant(L, lf) < 1e-12
    # the pattern really exercises the intersection term: some k < j < i with k in both
    # row i and row j of the lower pattern
    P = pattern_dense(L)
    i, j = nx + 1, 1                                 # (x=1,y=1) and (x=1,y=0)
    assert P[i, j] and P[i, 0] and P[j, 0]


@pytest.mark.parametrize("shape", ["tridiag", "arrow"])
def test_ic0_equals_cholesky_without_fill(shape):
    n = 24
    D = np.zeros((n, n))
    if shape == "tridiag":
        for i in range(1, n):
            D[i, i - 1] = D[i - 1, i] = -1.0 + 0.01 * i
    else:  # arrow pointing at the last row: tree pattern, no fill in Cholesky
        for i in range(n - 1):
            D[n - 1, i] = D[i, n - 1] = 0.3 - 0.02 * i
    np.fill_diagonal(D, 4.0 + np.abs(D).sum(axis=1))
    L = dense_to_csr(np.tril(D))
    lf = oracle.ic0(L)
    ch = np.linalg.cholesky(D)
    assert rel_err(csr_to_dense(L, lf), ch) < 1e-14


def test_ic0_breakdown_reports_row():
    D = np.array([[1.0, 0, 0], [2.0, 1.0, 0], [0, 0, 1.0]])
    L = dense_to_csr(D)
    with pytest.raises(oracle.OracleError) as e:
        oracle.ic0(L)
    assert e.value.code == 2   # row 1 (1-based 2): 1 - 2^2 < 0


def test_pairs_match_dense_compositions():
    n = 40
    DL = random_lower(n, 0.15, 41)
    DM = random_square(n, 0.2, 42)
    L, M = dense_to_csr(DL), dense_to_csr(DM)
    b = I.dense_vectors(n, 3, 4, I.S_RHS)
    x, y = oracle.trsv_spmv(L, M, b)
    xr = sla.solve_triangular(DL, b, lower=True)
    assert rel_err(x, xr) < 1e-13 and rel_err(y, DM @ xr) < 1e-13
    xin = I.dense_vectors(n, 3, 4, I.S_XIN)
    z = oracle.spmv_trsv(M, L, xin, b)
    assert rel_err(z, sla.solve_triangular(DL, b - DM @ xin, lower=True)) < 1e-13
    A = I.aniso_laplacian_3d((5, 4, 3))
    LA = I.lower_part(A)
    bb = I.dense_vectors(A.n_rows, 2, 5, I.S_RHS)
    lf, yy = oracle.ic0_trsv(LA, bb)
    assert rel_err(yy, sla.solve_triangular(csr_to_dense(LA, lf), bb, lower=True)) < 1e-13
