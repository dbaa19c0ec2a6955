"""Pins of the oracle routines for two further kernel pairs of Table 2: combination 1
(SpTRSV -> SpTRSV with the same L) and combination 6 (zero fill-in SpILU0 -> SpTRSV with the
unit lower factor). Checked against dense solves, exact integer arithmetic, closed forms,
the defining zero-fill property of ILU(0), the no-fill cases where ILU(0) is the exact LU
factorisation, and the relation to the (separately pinned) IC0 factor on symmetric input."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2111_12238_gb300 import inputs as I
from tests._mats import csr_to_dense, dense_to_csr, pattern_dense, random_lower, random_square, rel_err


# ------------------------------------------------------------------ combination 1
@pytest.mark.parametrize("n,k", [(1, 1), (17, 1), (40, 3)])
def test_trsv_trsv_matches_two_dense_solves(n, k):
    D = random_lower(n, 0.3, 51 + n)
    L = dense_to_csr(D)
    b = I.dense_vectors(n, k, 52, 1)
    x, z = oracle.trsv_trsv(L, b)
    x_ref = sla.solve_triangular(D, b, lower=True)
    assert rel_err(x, x_ref) < 1e-13
    assert rel_err(z, sla.solve_triangular(D, x_ref, lower=True)) < 1e-13


def test_trsv_trsv_integer_exact():
    # unit diagonal, off-diagonals in {-1, 0, 1}, integer b: every intermediate is an integer
    # below 2^53, so the result is exact; the reference is integer forward substitution
    n = 24
    D = random_lower(n, 0.15, 53, unit_int=True)
    L = dense_to_csr(D)
    b = np.arange(1, n + 1, dtype=np.int64).reshape(n, 1) % 5 - 2
    Di = D.astype(np.int64)

    def fwd(rhs):
        out = [0] * n
        for i in range(n):
            out[i] = int(rhs[i]) - sum(int(Di[i, j]) * out[j] for j in range(i))
        return out

    xi = fwd(b[:, 0])
    zi = fwd(xi)
    assert max(abs(v) for v in zi) < 2 ** 53
    x, z = oracle.trsv_trsv(L, b.astype(np.float64))
    assert np.array_equal(x[:, 0], np.asarray(xi, dtype=np.float64))
    assert np.array_equal(z[:, 0], np.asarray(zi, dtype=np.float64))


def test_trsv_trsv_diagonal_closed_form():
    d = np.array([2.0, 4.0, 0.5, 8.0])
    L = dense_to_csr(np.diag(d))
    b = np.array([[1.0], [2.0], [3.0], [4.0]])
    x, z = oracle.trsv_trsv(L, b)
    assert np.array_equal(x[:, 0], b[:, 0] / d)
    assert np.array_equal(z[:, 0], b[:, 0] / d / d)


# ------------------------------------------------------------------ combination 6
def _diag_dominant(S):
    """S with its diagonal replaced by 1 + the absolute row sum of its off-diagonals."""
    A = S.copy()
    np.fill_diagonal(A, 0.0)
    np.fill_diagonal(A, 1.0 + np.abs(A).sum(axis=1))
    return A


def _factors(A_csr, lu):
    LU = csr_to_dense(A_csr, lu)
    n = A_csr.n_rows
    Lf = np.tril(LU, -1) + np.eye(n)
    Uf = np.triu(LU)
    return Lf, Uf


def _stencil9(nx):
    offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    n, rowptr, cols, soffs, Msk = I._stencil_pattern((nx, nx), offs)
    vals = np.where(np.asarray([o == (0, 0) for o in soffs])[None, :], 9.0, -1.0)
    return I._finish(n, n, rowptr, cols, np.broadcast_to(vals, Msk.shape)[Msk])


@pytest.mark.parametrize("case", ["random", "stencil9"])
def test_ilu0_zero_fill_property(case):
    # ILU(0): (L U)_ij = A_ij at every position of A's pattern (the fill outside it is dropped)
    if case == "random":
        A = dense_to_csr(_diag_dominant(random_square(60, 0.12, 54)))
    else:
        A = _stencil9(9)
    lu = oracle.ilu0(A)
    Lf, Uf = _factors(A, lu)
    P = pattern_dense(A)
    Ad = csr_to_dense(A)
    prod = Lf @ Uf
    assert np.max(np.abs(prod - Ad)[P]) / np.max(np.abs(Ad)) < 1e-13
    # the dropped fill is really there for these patterns, so the test is not vacuous
    assert np.max(np.abs(prod - Ad)[~P]) > 1e-6


@pytest.mark.parametrize("shape", ["dense", "tridiagonal", "arrow_down"])
def test_ilu0_without_fill_is_the_exact_lu(shape):
    # patterns closed under elimination: ILU(0) is the LU factorisation, L U = A everywhere
    n = 12
    S = random_square(n, 1.0, 55)
    if shape == "tridiagonal":
        S = np.triu(np.tril(S, 1), -1)
    elif shape == "arrow_down":
        keep = np.zeros((n, n), bool)
        keep[-1, :] = keep[:, -1] = True
        S = np.where(keep, S, 0.0)
    A_d = _diag_dominant(S)
    A = dense_to_csr(A_d, pattern=(A_d != 0) | np.eye(n, dtype=bool))
    Lf, Uf = _factors(A, oracle.ilu0(A))
    assert rel_err(Lf @ Uf, A_d) < 1e-14


@pytest.mark.parametrize("case", ["aniso", "stencil9"])
def test_ilu0_on_symmetric_input_relates_to_ic0(case):
    # A symmetric positive definite: U = diag(U) L^T, and the IC0 factor of tril(A) is
    # L diag(U)^(1/2) (the 9-point pattern exercises the intersection terms of both)
    A = I.aniso_laplacian_3d((5, 4, 3)) if case == "aniso" else _stencil9(8)
    lu = oracle.ilu0(A)
    Lf, Uf = _factors(A, lu)
    d = np.diag(Uf)
    assert np.all(d > 0)
    assert rel_err(Uf, np.diag(d) @ Lf.T) < 1e-13
    Lt = I.lower_part(A)
    lc = csr_to_dense(Lt, oracle.ic0(Lt))
    assert rel_err(lc, Lf @ np.diag(np.sqrt(d))) < 1e-13


def test_ilu0_zero_pivot_is_reported():
    A_d = np.array([[0.0, 1.0, 0.0], [1.0, 2.0, 0.0], [0.0, 0.0, 1.0]])
    A = dense_to_csr(A_d, pattern=(A_d != 0) | np.eye(3, dtype=bool))
    with pytest.raises(oracle.OracleError) as e:
        oracle.ilu0(A)
    assert e.value.code == 1               # pivot u_00 = 0, met by row 1


def test_ilu0_trsv_matches_a_unit_lower_dense_solve():
    A = dense_to_csr(_diag_dominant(random_square(50, 0.15, 56)))
    b = I.dense_vectors(50, 4, 57, 1)
    lu, y = oracle.ilu0_trsv(A, b)
    assert np.array_equal(lu, oracle.ilu0(A))
    Lf, _ = _factors(A, lu)
    assert rel_err(y, sla.solve_triangular(Lf, b, lower=True, unit_diagonal=True)) < 1e-13
