"""Parity of Table 2 combinations 1 (SpTRSV -> SpTRSV) and 6 (SpILU0 -> SpTRSV), and of the
shared-storage SpMV -> SpTRSV row (L = tril(A) read from A's rows), with the FP64 oracle:
element-wise results, exact integer cases compared bit for bit, bit-exact inspector output,
bounded-wait timeouts and the errors each entry point reports."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t, vec_rel_err
from tests._mats import dense_to_csr, random_square

pytestmark = pytest.mark.gpu


def _rhs(n, k, seed=3):
    return I.dense_vectors(n, k, seed, I.S_RHS)


def _nonsym_stencil(nx, seed):
    """2D 9-point pattern with U[-1,1] off-diagonals and diagonal 1 + sum |off| of the row
    (rows diagonally dominant, so ILU0 has nonzero pivots)."""
    offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    n, rowptr, cols, _, _ = I._stencil_pattern((nx, nx), offs)
    return I._finish(n, n, rowptr, cols, I._diag_dominant_values(seed, 5, rowptr, cols))


def _random_sparse(n, density, seed):
    D = random_square(n, density, seed)
    np.fill_diagonal(D, 0.0)
    np.fill_diagonal(D, 1.0 + np.abs(D).sum(axis=1))
    return dense_to_csr(D)


def _ilu_inputs():
    return {
        "aniso10": lambda: I.aniso_laplacian_3d((10, 10, 10)),
        "stencil9_nonsym": lambda: _nonsym_stencil(24, 7),
        "random400": lambda: _random_sparse(400, 0.03, 11),
    }


# ------------------------------------------------------------------ SpTRSV -> SpTRSV
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,ef", [(1, False), (1, True), (3, False), (16, False), (16, True)])
@pytest.mark.parametrize("lpr", [0, 1, 8, 32])
def test_trsv_trsv(dtype, k, ef, lpr):
    need_cuda()
    w = I.trsv_spmv_lap3d_band(11, per_row=6, halfband=200, seed=21, k=k)
    x_ref, z_ref = oracle.trsv_trsv(w.L, w.b)
    if lpr and lpr < min(k, 32) and k > 1:
        pytest.skip("lanes per row below the RHS tile is raised to the tile")
    sch = sf.inspect("trsv_trsv", dev_csr(w.L), lanes_per_row=lpr, epoch_flags=ef)
    sch.validate()
    xs = torch.empty((w.n, k), device="cuda", dtype=dtype)
    z = sch.execute(t(w.L.vals, dtype), b=t(w.b, dtype), x_save=xs)
    sch.check()
    assert col_rel_err(host(xs), x_ref) < TOL[dtype]
    assert col_rel_err(host(z), z_ref) < TOL[dtype]


def test_trsv_trsv_long_rows_and_scratch_x():
    # power-law rows up to 256 entries, several of them wide (whole-warp partitions); x_save
    # omitted (library-owned intermediate)
    need_cuda()
    n = 20000
    L = I.powerlaw_lower(n, 8, 256, 4)
    b = _rhs(n, 2)
    x_ref, z_ref = oracle.trsv_trsv(L, b)
    for lpr in (1, 4):
        sch = sf.inspect("trsv_trsv", dev_csr(L), lanes_per_row=lpr)
        z = sch.execute(t(L.vals), b=t(b))
        sch.check()
        assert col_rel_err(host(z), z_ref) < 1e-12


def test_trsv_trsv_integer_exact_bitwise():
    # unit lower {-1,0,1} L with b = L (L x_int): x = L x_int and z = x_int exactly
    need_cuda()
    n = 3000
    pat = I.powerlaw_lower(n, 3, 12, 77)
    Lv = np.where(pat.colidx == np.repeat(np.arange(n), np.diff(pat.rowptr)), 1.0, np.sign(pat.vals))
    L = I.Csr(n, n, pat.rowptr, pat.colidx, Lv.astype(np.float64))
    x_int = (np.arange(n) % 5 - 2).astype(np.float64).reshape(n, 1)
    b = oracle.spmv(L, oracle.spmv(L, x_int))
    x_ref, z_ref = oracle.trsv_trsv(L, b)
    assert np.array_equal(z_ref, x_int)
    for lpr, ef in ((1, False), (4, False), (32, False), (4, True)):
        sch = sf.inspect("trsv_trsv", dev_csr(L), lanes_per_row=lpr, epoch_flags=ef)
        xs = torch.empty((n, 1), device="cuda", dtype=torch.float64)
        z = sch.execute(t(L.vals), b=t(b), x_save=xs)
        sch.check()
        assert np.array_equal(host(xs), x_ref)
        assert np.array_equal(host(z), z_ref)


@pytest.mark.parametrize("ef", [False, True])
def test_trsv_trsv_timeout_is_reported(ef):
    # a chain in one partition with its first two items swapped: row 1 waits for row 0,
    # which the same team would run only later; the bounded wait ends with SF_ERR_TIMEOUT
    need_cuda()
    n = 64
    L = dense_to_csr(np.eye(n) * 2 + np.eye(n, k=-1))
    b = np.ones((n, 1))
    sch = sf.inspect("trsv_trsv", dev_csr(L), lanes_per_row=32, part_cost_target=10 ** 9, epoch_flags=ef)
    assert sch.info()["n_parts"] == 1
    sch.set_timeout(2_000_000)
    sch.debug_swap(0, 1)
    Lv, bb = t(L.vals), t(b)
    sch.execute(Lv, b=bb)
    assert sch.check_status() == (5, 1)
    sch.debug_swap(0, 1)
    z = sch.execute(Lv, b=bb)
    sch.check()
    assert col_rel_err(host(z), oracle.trsv_trsv(L, b)[1]) < 1e-14


# ------------------------------------------------------------------ SpILU0 -> SpTRSV
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k", [1, 5, 32])
@pytest.mark.parametrize("name", list(_ilu_inputs()))
def test_ilu0_trsv(dtype, k, name):
    need_cuda()
    A = _ilu_inputs()[name]()
    L = I.lower_part(A)
    b = _rhs(A.n_rows, k)
    lu_ref, y_ref = oracle.ilu0_trsv(A, b)
    sch = sf.inspect("ilu0_trsv", dev_csr(L), dev_csr(A), rhs_tile=min(32, 1 << (k - 1).bit_length()))
    sch.validate()
    lu = torch.empty(A.nnz, device="cuda", dtype=dtype)
    y = sch.execute(None, t(A.vals, dtype), b=t(b, dtype), x_save=lu)
    sch.check()
    assert vec_rel_err(host(lu), lu_ref) < TOL[dtype]
    assert col_rel_err(host(y), y_ref) < TOL[dtype]


def test_ilu0_trsv_repeated_and_scratch_factor():
    need_cuda()
    A = _nonsym_stencil(30, 9)
    L = I.lower_part(A)
    b = _rhs(A.n_rows, 4)
    _, y_ref = oracle.ilu0_trsv(A, b)
    sch = sf.inspect("ilu0_trsv", dev_csr(L), dev_csr(A))
    Av, bb = t(A.vals), t(b)
    y = torch.empty_like(bb)
    for _ in range(5):
        sch.execute(None, Av, b=bb, y=y)
    sch.check()
    assert col_rel_err(host(y), y_ref) < 1e-12


def test_ilu0_trsv_integer_exact_bitwise():
    # A = L0 U0 with L0 unit lower bidiagonal ({-1, 1} below the diagonal) and U0 upper
    # bidiagonal (diagonal in {1, 2, 4}, {-1, 1} above): A is tridiagonal, ILU0 has no fill to
    # drop and every division is by a power of two, so the factor is exactly (L0, U0) and
    # y = L0^-1 (L0 y_int) = y_int, bit for bit
    need_cuda()
    n = 300
    idx = np.arange(n)
    c = np.where(I.uniform_below(3, 1, idx, 2) == 0, -1.0, 1.0)
    d = 2.0 ** I.uniform_below(3, 2, idx, 3)
    e = np.where(I.uniform_below(3, 3, idx, 2) == 0, -1.0, 1.0)
    L0 = np.eye(n) + np.diag(c[1:], -1)
    U0 = np.diag(d) + np.diag(e[:-1], 1)
    A = dense_to_csr(L0 @ U0, pattern=(np.abs(idx[:, None] - idx[None, :]) <= 1))
    y_int = (idx % 7 - 3).astype(np.float64).reshape(n, 1)
    b = L0 @ y_int
    lu_ref, y_ref = oracle.ilu0_trsv(A, b)
    assert np.array_equal(y_ref, y_int)
    sch = sf.inspect("ilu0_trsv", dev_csr(I.lower_part(A)), dev_csr(A))
    lu = torch.empty(A.nnz, device="cuda", dtype=torch.float64)
    y = sch.execute(None, t(A.vals), b=t(b), x_save=lu)
    sch.check()
    assert np.array_equal(host(lu), lu_ref)
    assert np.array_equal(host(y), y_ref)


def test_ilu0_zero_pivot_and_timeout_reported():
    need_cuda()
    # u_00 = 0: row 1 divides by it
    A = dense_to_csr(np.array([[0.0, 1.0], [1.0, 1.0]]), pattern=np.ones((2, 2), dtype=bool))
    sch = sf.inspect("ilu0_trsv", dev_csr(I.lower_part(A)), dev_csr(A))
    sch.execute(None, t(A.vals), b=t(np.ones((2, 1))))
    assert sch.check_status() == (6, 0)       # SF_ERR_BREAKDOWN at row 0
    # a chain in one partition with its first two items swapped: the bounded polls end it
    n = 48
    D = np.eye(n) * 4 - np.eye(n, k=-1) - np.eye(n, k=1)
    A = dense_to_csr(D)
    b = _rhs(n, 3)
    sch = sf.inspect("ilu0_trsv", dev_csr(I.lower_part(A)), dev_csr(A), part_cost_target=10 ** 9)
    assert sch.info()["n_parts"] == 1
    sch.set_timeout(2_000_000)
    sch.debug_swap(0, 1)
    Av, bb = t(A.vals), t(b)
    sch.execute(None, Av, b=bb)
    assert sch.check_status() == (5, 1)
    sch.debug_swap(0, 1)
    y = sch.execute(None, Av, b=bb)
    sch.check()
    assert col_rel_err(host(y), oracle.ilu0_trsv(A, b)[1]) < 1e-13


def test_ilu0_rejects_bad_inputs():
    need_cuda()
    A = _random_sparse(60, 0.1, 3)
    L = I.lower_part(A)
    # L is not tril(A)'s pattern
    Lbad = dense_to_csr(np.eye(60))
    with pytest.raises(sf.SparseFusionError) as ei:
        sf.inspect("ilu0_trsv", dev_csr(Lbad), dev_csr(A))
    assert ei.value.status == 2
    # a row of A without its diagonal
    D = np.eye(4) + np.eye(4, k=1)
    P = D != 0
    P[2, 2] = False
    Anod = dense_to_csr(D, pattern=P)
    with pytest.raises(sf.SparseFusionError) as ei:
        sf.inspect("ilu0_trsv", dev_csr(dense_to_csr(np.eye(4))), dev_csr(Anod))
    assert ei.value.status == 2
    # rows longer than an ILU0 row keeps on chip
    Dl = np.eye(300)
    Dl[299, :] = 1.0
    Dl[299, 299] = 400.0
    Al = dense_to_csr(Dl)
    with pytest.raises(sf.SparseFusionError) as ei:
        sf.inspect("ilu0_trsv", dev_csr(I.lower_part(Al)), dev_csr(Al))
    assert ei.value.status == 8
    # value arrays: L_vals must be NULL, M_vals (A) present
    sch = sf.inspect("ilu0_trsv", dev_csr(L), dev_csr(A))
    with pytest.raises(sf.SparseFusionError):
        sch.execute(t(L.vals), t(A.vals), b=t(_rhs(60, 1)))


# ------------------------------------------------------------------ shared-storage SpMV -> SpTRSV
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,lpr", [(1, 0), (1, 1), (1, 8), (1, 32), (2, 16), (2, 32), (16, 0), (16, 32)])
def test_spmv_trsv_shared_storage(dtype, k, lpr):
    # L = tril(A) read from A's rows (L_vals NULL) gives the oracle's z = L^-1 (b - A x_in)
    need_cuda()
    w = I.spmv_trsv_powerlaw(n=20000, k=k, mean=16, lmax=400, halfband=900, seed=31)
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), lanes_per_row=lpr)
    z = sch.execute(None, t(w.M.vals, dtype), b=t(w.b, dtype), x_in=t(w.x_in, dtype))
    sch.check()
    assert col_rel_err(host(z), z_ref) < TOL[dtype]


def test_spmv_trsv_shared_storage_rules():
    need_cuda()
    w = I.spmv_trsv_powerlaw(n=3000, k=1, mean=8, lmax=60, halfband=200, seed=33)
    Lp = I.lower_part(w.M)
    assert np.array_equal(Lp.rowptr, w.L.rowptr) and np.array_equal(Lp.colidx, w.L.colidx)
    # L's pattern differs from tril(A): L_vals is required
    Ld = dense_to_csr(np.eye(w.n))
    sch = sf.inspect("spmv_trsv", dev_csr(Ld), dev_csr(w.M))
    with pytest.raises(sf.SparseFusionError):
        sch.execute(None, t(w.M.vals), b=t(w.b), x_in=t(w.x_in))
    # epoch flags: shared storage is a value-flag path
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), epoch_flags=True)
    with pytest.raises(sf.SparseFusionError):
        sch.execute(None, t(w.M.vals), b=t(w.b), x_in=t(w.x_in))
    # several right-hand sides publish through values only with 16 or more lanes per row
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), lanes_per_row=8)
    b2, x2 = t(np.repeat(w.b, 2, axis=1)), t(np.repeat(w.x_in, 2, axis=1))
    with pytest.raises(sf.SparseFusionError) as ei:
        sch.execute(None, t(w.M.vals), b=b2, x_in=x2)
    assert ei.value.status == 8
    # the two storage forms agree on the same schedule
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M))
    z1 = sch.execute(t(w.L.vals), t(w.M.vals), b=t(w.b), x_in=t(w.x_in))
    z2 = sch.execute(None, t(w.M.vals), b=t(w.b), x_in=t(w.x_in))
    sch.check()
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    assert col_rel_err(host(z1), z_ref) < 1e-12 and col_rel_err(host(z2), z_ref) < 1e-12


# ------------------------------------------------------------------ inspector parity
@pytest.mark.parametrize("target", [0, 1, 57, 10 ** 12])
@pytest.mark.parametrize("case", ["trsv_trsv_lap3d", "trsv_trsv_plower", "ilu0_stencil9", "ilu0_random"])
def test_next_schedules_match_oracle(case, target):
    need_cuda()
    if case.startswith("trsv_trsv"):
        L = (I.trsv_spmv_lap3d_band(13, per_row=5, halfband=300, seed=7).L if case.endswith("lap3d")
             else I.powerlaw_lower(5000, 8, 256, 4))
        A, pair, what = None, "trsv_trsv", oracle.COST_TRSV_TRSV
    else:
        A = _nonsym_stencil(20, 4) if case.endswith("stencil9") else _random_sparse(500, 0.02, 6)
        L, pair, what = I.lower_part(A), "ilu0_trsv", oracle.COST_ILU0_TRSV
    sch = sf.inspect(pair, dev_csr(L), dev_csr(A) if A is not None else None, part_cost_target=target)
    sch.validate()
    info = sch.info()
    C, W = info["part_cost_target"], info["wide_cost"]
    if target:
        assert C == target
    ref = oracle.schedule(oracle.PAIRED, what, L, A, C, wide=W)
    got = sch.export(0)
    assert np.array_equal(got["level"], ref["level"])
    assert got["depth"] == ref["depth"]
    assert np.array_equal(got["order"], ref["order"])
    assert np.array_equal(got["part_ptr"], ref["part_ptr"])
    assert oracle.validate(oracle.PAIRED, L, None, got["order"], got["part_ptr"]) == 0
    assert info["reuse_ratio"] == pytest.approx(
        oracle.reuse_ratio(sf.PAIRS[pair], L.n_rows, L.nnz, A.nnz if A is not None else 0), rel=1e-15)
