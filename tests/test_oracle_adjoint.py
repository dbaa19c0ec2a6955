"""Pins of the oracle's adjoints (not in the paper; needed by the differentiable form of
the fused pairs): the dot-product identity, dense closed forms on tiny inputs, and central
finite differences along random directions. CPU only."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2111_12238_gb300 import inputs as I
from tests._mats import csr_to_dense, dense_to_csr, random_lower, random_square, rel_err


def _mats(n, seed):
    DL = random_lower(n, 0.2, seed)
    DM = random_square(n, 0.25, seed + 1)
    return DL, DM, dense_to_csr(DL), dense_to_csr(DM)


@pytest.mark.parametrize("k", [1, 3])
def test_adj_trsv_spmv_dense_closed_form(k):
    n = 24
    DL, DM, L, M = _mats(n, 5)
    b = I.dense_vectors(n, k, 5, I.S_RHS)
    gy = I.dense_vectors(n, k, 5, I.S_GRAD)
    x, y = oracle.trsv_spmv(L, M, b)
    gb, gL, gM = oracle.adj_trsv_spmv(L, M, x, gy)
    lam = sla.solve_triangular(DL.T, DM.T @ gy, lower=False)
    assert rel_err(gb, lam) < 1e-13
    GL = -(lam @ x.T)
    GM = gy @ x.T
    assert rel_err(gL, GL[DL != 0]) < 1e-13
    assert rel_err(gM, GM[DM != 0]) < 1e-13


def test_adj_trsv_spmv_dot_product_identity():
    w = I.trsv_spmv_lap3d_band(10, per_row=6, halfband=40, seed=3)
    x, y = oracle.trsv_spmv(w.L, w.M, w.b)
    gb, _, _ = oracle.adj_trsv_spmv(w.L, w.M, x, w.gy)
    db = I.dense_vectors(w.n, 1, 77, I.S_XIN)
    _, dy = oracle.trsv_spmv(w.L, w.M, db)        # y is linear in b
    lhs = float(np.sum(w.gy * dy))
    rhs = float(np.sum(gb * db))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)


def _fd_dir(f, theta, d, h):
    return (f(theta + h * d) - f(theta - h * d)) / (2 * h)


def test_adj_trsv_spmv_finite_differences():
    w = I.trsv_spmv_lap3d_band(6, per_row=5, halfband=30, seed=11)
    L, M = w.L, w.M
    x, y = oracle.trsv_spmv(L, M, w.b)
    gb, gL, gM = oracle.adj_trsv_spmv(L, M, x, w.gy)

    def loss(lv=None, mv=None, b=None):
        LL = I.Csr(L.n_rows, L.n_cols, L.rowptr, L.colidx, L.vals if lv is None else lv)
        MM = I.Csr(M.n_rows, M.n_cols, M.rowptr, M.colidx, M.vals if mv is None else mv)
        return float(np.sum(w.gy * oracle.trsv_spmv(LL, MM, w.b if b is None else b)[1]))

    for t in range(8):
        dL = I.uniform_pm1(100 + t, 1, np.arange(L.nnz))
        dM = I.uniform_pm1(200 + t, 1, np.arange(M.nnz))
        db = I.uniform_pm1(300 + t, 1, np.arange(w.n)).reshape(w.n, 1)
        h = 1e-6
        assert abs(_fd_dir(lambda v: loss(lv=v), L.vals, dL, h) - gL @ dL) <= 1e-6 * max(1, abs(gL @ dL))
        assert abs(_fd_dir(lambda v: loss(mv=v), M.vals, dM, h) - gM @ dM) <= 1e-6 * max(1, abs(gM @ dM))
        assert abs(_fd_dir(lambda v: loss(b=v), w.b, db, h) - np.sum(gb * db)) <= 1e-6 * max(1, abs(np.sum(gb * db)))


@pytest.mark.parametrize("k", [1, 2])
def test_adj_spmv_trsv_dense_closed_form(k):
    n = 20
    DL, DA, L, A = _mats(n, 9)
    xin = I.dense_vectors(n, k, 9, I.S_XIN)
    b = I.dense_vectors(n, k, 9, I.S_RHS)
    gz = I.dense_vectors(n, k, 9, I.S_GRAD)
    z = oracle.spmv_trsv(A, L, xin, b)
    gb, gx, gL, gA = oracle.adj_spmv_trsv(A, L, xin, z, gz)
    lam = sla.solve_triangular(DL.T, gz, lower=False)
    assert rel_err(gb, lam) < 1e-13
    assert rel_err(gx, -(DA.T @ lam)) < 1e-13
    assert rel_err(gL, (-(lam @ z.T))[DL != 0]) < 1e-13
    assert rel_err(gA, (-(lam @ xin.T))[DA != 0]) < 1e-13


def test_adj_spmv_trsv_finite_differences():
    w = I.spmv_trsv_powerlaw(n=300, k=2, mean=6, lmax=20, halfband=50, seed=13)
    A, L = w.M, w.L
    z = oracle.spmv_trsv(A, L, w.x_in, w.b)
    gb, gx, gL, gA = oracle.adj_spmv_trsv(A, L, w.x_in, z, w.gy)

    def loss(av=None, lv=None, xin=None):
        AA = I.Csr(A.n_rows, A.n_cols, A.rowptr, A.colidx, A.vals if av is None else av)
        LL = I.Csr(L.n_rows, L.n_cols, L.rowptr, L.colidx, L.vals if lv is None else lv)
        return float(np.sum(w.gy * oracle.spmv_trsv(AA, LL, w.x_in if xin is None else xin, w.b)))

    for t in range(4):
        dA = I.uniform_pm1(400 + t, 1, np.arange(A.nnz))
        dL = I.uniform_pm1(500 + t, 1, np.arange(L.nnz))
        dx = I.uniform_pm1(600 + t, 1, np.arange(w.n * 2)).reshape(w.n, 2)
        h = 1e-6
        for fd, an in ((_fd_dir(lambda v: loss(av=v), A.vals, dA, h), gA @ dA),
                       (_fd_dir(lambda v: loss(lv=v), L.vals, dL, h), gL @ dL),
                       (_fd_dir(lambda v: loss(xin=v), w.x_in, dx, h), np.sum(gx * dx))):
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
