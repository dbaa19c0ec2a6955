"""Batched many-instance launches (one persistent launch over a block-diagonal queue,
CUDA-graph replay, FP64 and FP32, forward and adjoint) and device-side failure reporting
without any GPU fault: a dependence wait that runs out, an IC0 breakdown, a zero pivot."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t, vec_rel_err
from tests._mats import dense_to_csr

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_forward_adjoint_and_graph(dtype):
    need_cuda()
    w = I.batched_trsv_spmv(count=12, nmin=100, nmax=6000, seed=4)
    sch = sf.inspect_batched("trsv_spmv", [dev_csr(x.L) for x in w.instances], [dev_csr(x.M) for x in w.instances],
                             want_adjoint=True)
    Lv = t(np.concatenate([x.L.vals for x in w.instances]), dtype)
    Mv = t(np.concatenate([x.M.vals for x in w.instances]), dtype)
    b, gy = t(w.b, dtype), t(w.gy, dtype)
    xs = torch.empty_like(b)
    y = torch.empty_like(b)
    g = sf.GraphedExecute(sch, L_vals=Lv, M_vals=Mv, b=b, y=y, x_save=xs)
    for _ in range(3):
        g.replay()
    gL, gM = torch.empty_like(Lv), torch.empty_like(Mv)
    gb = sch.adjoint(Lv, Mv, gy, saved=xs, gL=gL, gM=gM)
    sch.check()
    off, offL, offM = 0, 0, 0
    tol = TOL[dtype]
    for x in w.instances:
        xr, yr = oracle.trsv_spmv(x.L, x.M, x.b)
        gbr, gLr, gMr = oracle.adj_trsv_spmv(x.L, x.M, xr, x.gy)
        sl = slice(off, off + x.n)
        assert col_rel_err(host(y)[sl], yr) < TOL[dtype]
        assert col_rel_err(host(gb)[sl], gbr) < tol
        assert vec_rel_err(host(gL)[offL:offL + x.L.nnz], gLr) < tol
        assert vec_rel_err(host(gM)[offM:offM + x.M.nnz], gMr) < tol
        off += x.n
        offL += x.L.nnz
        offM += x.M.nnz


def test_batched_matches_single_instance_bitwise():
    # same rows, same per-row summation order: batched and single launches agree exactly
    need_cuda()
    w = I.batched_trsv_spmv(count=5, nmin=500, nmax=4000, seed=8)
    sch = sf.inspect_batched("trsv_spmv", [dev_csr(x.L) for x in w.instances], [dev_csr(x.M) for x in w.instances],
                             lanes_per_row=4)
    y = sch.execute(t(np.concatenate([x.L.vals for x in w.instances])),
                    t(np.concatenate([x.M.vals for x in w.instances])), b=t(w.b))
    sch.check()
    off = 0
    for x in w.instances:
        s1 = sf.inspect("trsv_spmv", dev_csr(x.L), dev_csr(x.M), lanes_per_row=4)
        y1 = s1.execute(t(x.L.vals), t(x.M.vals), b=t(x.b))
        s1.check()
        assert np.array_equal(host(y)[off:off + x.n], host(y1))
        off += x.n


@pytest.mark.parametrize("ef", [False, True])
def test_timeout_is_reported_not_hung(ef):
    # a chain (bidiagonal L) in one partition run by one warp; swapping its first two items
    # makes that warp wait for a row only it would compute later: a flag nothing sets.
    # The bounded wait (2 ms here) must end the launch with SF_ERR_TIMEOUT.
    need_cuda()
    n = 64
    D = np.eye(n) * 2 + np.eye(n, k=-1)
    L = dense_to_csr(D)
    b = np.ones((n, 1))
    sch = sf.inspect("trsv", dev_csr(L), lanes_per_row=32, part_cost_target=10 ** 9, epoch_flags=ef,
                     exec_mode=1)
    assert sch.info()["n_parts"] == 1
    sch.set_timeout(2_000_000)
    sch.debug_swap(0, 1)
    Lv, bb = t(L.vals), t(b)
    x = sch.execute(Lv, b=bb)
    st, row = sch.check_status()
    assert st == 5                      # SF_ERR_TIMEOUT
    assert row == 1                     # row 1 waited for row 0
    # the schedule state recovers: restore the order and run again
    sch.debug_swap(0, 1)
    x = sch.execute(Lv, b=bb)
    sch.check()
    assert col_rel_err(host(x), oracle.trsv_lower(L, b)) < 1e-14


@pytest.mark.parametrize("pair,k", [("ic0_trsv", 4), ("ic0", 1)])
def test_ic0_value_flag_timeout_is_reported(pair, k):
    # IC0 rows poll 1 / L_jj and their columns of y (value flags). A chain in one partition
    # with its first two items swapped makes row 1 poll values that only row 0, later in the
    # same team's list, would write; the bounded poll must end with SF_ERR_TIMEOUT.
    need_cuda()
    n = 48
    D = np.eye(n) * 4 - np.eye(n, k=-1)
    L = dense_to_csr(D)
    b = I.dense_vectors(n, k, 9, 1)
    sch = sf.inspect(pair, dev_csr(L), lanes_per_row=32, part_cost_target=10 ** 9)
    assert sch.info()["n_parts"] == 1 and sch.info()["ic0_use_pairs"] == 1
    sch.set_timeout(2_000_000)
    sch.debug_swap(0, 1)
    lf = torch.empty(L.nnz, device="cuda", dtype=torch.float64)
    Lv, bb = t(L.vals), t(b)
    run = (lambda: sch.execute(Lv, b=bb, x_save=lf)) if pair == "ic0_trsv" else (lambda: sch.execute(Lv, x_save=lf))
    run()
    st, row = sch.check_status()
    assert (st, row) == (5, 1)          # SF_ERR_TIMEOUT at row 1
    sch.debug_swap(0, 1)
    y = run()
    sch.check()
    assert vec_rel_err(host(lf), oracle.ic0(L)) < 1e-14
    if pair == "ic0_trsv":
        assert col_rel_err(host(y), oracle.ic0_trsv(L, b)[1]) < 1e-13


def test_ic0_breakdown_and_zero_pivot_reported():
    need_cuda()
    D = np.array([[1.0, 0, 0], [2.0, 1.0, 0], [0, 0, 1.0]])
    L = dense_to_csr(D)
    sch = sf.inspect("ic0", dev_csr(L))
    lf = torch.empty(L.nnz, device="cuda", dtype=torch.float64)
    sch.execute(t(L.vals), x_save=lf)
    st, row = sch.check_status()
    assert (st, row) == (6, 1)          # SF_ERR_BREAKDOWN at row 1
    Z = dense_to_csr(np.array([[1.0, 0], [1.0, 0.0]]), np.array([[True, False], [True, True]]))
    s2 = sf.inspect("trsv", dev_csr(Z))
    s2.execute(t(Z.vals), b=t(np.ones((2, 1))))
    st, row = s2.check_status()
    assert (st, row) == (7, 1)          # SF_ERR_NONFINITE: zero diagonal at row 1
    st, _ = s2.check_status()
    assert st == 0                      # the report is cleared once read


def test_ic0_alone_rejects_solve_operands():
    need_cuda()
    L = dense_to_csr(np.eye(4) * 4 - np.eye(4, k=-1))
    sch = sf.inspect("ic0", dev_csr(L))
    lf = torch.empty(L.nnz, device="cuda", dtype=torch.float64)
    with pytest.raises(sf.SparseFusionError) as e:
        sch.execute(t(L.vals), y=torch.empty((4, 1), device="cuda", dtype=torch.float64), x_save=lf)
    assert e.value.status == 1
    sch.execute(t(L.vals), x_save=lf)
    sch.check()
    assert vec_rel_err(host(lf), oracle.ic0(L)) < 1e-14


def test_invalid_execute_arguments():
    need_cuda()
    w = I.trsv_spmv_lap2d(8, seed=1)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M))
    with pytest.raises(sf.SparseFusionError) as e:
        sch.execute(t(w.L.vals), None, b=t(w.b))
    assert e.value.status == 1
    with pytest.raises(ValueError):
        sch.execute(torch.from_numpy(w.L.vals), t(w.M.vals), b=t(w.b))
