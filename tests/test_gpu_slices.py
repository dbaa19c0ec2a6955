"""Long rows split at execution time (sf_schedule_set_slices): each costly row runs as several
slices on several teams whose partial sums the owner slice adds in order. Results must match
the FP64 oracle for every kind the executor splits (SpTRSV rows, SpMV -> SpTRSV rows in both
storage forms, the transposed solve rows of both adjoints), for one and many right-hand sides,
after re-cuts, and with the dynamic ticket queue."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t, vec_rel_err

pytestmark = pytest.mark.gpu


def _powerlaw(k, seed=31):
    return I.spmv_trsv_powerlaw(n=20000, k=k, mean=16, lmax=800, halfband=1500, seed=seed)


def _split_happened(sch, which=0):
    info = sch.info()
    units = info["slice_units"] if which == 0 else info["adj_slice_units"]
    parts = info["n_parts"] if which == 0 else info["adj_n_parts"]
    return units > parts


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,lpr", [(1, 0), (1, 4), (16, 16), (16, 32)])
@pytest.mark.parametrize("cost", [24, 160])
def test_spmv_trsv_slices(dtype, k, lpr, cost):
    need_cuda()
    w = _powerlaw(k)
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    gb_ref, gx_ref, gL_ref, gA_ref = oracle.adj_spmv_trsv(w.M, w.L, w.x_in, z_ref, w.gy)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, lanes_per_row=lpr)
    sch.set_slices(-1, cost)
    # the rows of L^T (columns of L) are short in this band: only the forward splits rows
    assert _split_happened(sch, 0)
    Lv, Av, xin, b = t(w.L.vals, dtype), t(w.M.vals, dtype), t(w.x_in, dtype), t(w.b, dtype)
    z = sch.execute(Lv, Av, b=b, x_in=xin)
    zs = sch.execute(None, Av, b=b, x_in=xin)                  # L read from A's rows
    gx, gL, gA = torch.empty_like(xin), torch.empty_like(Lv), torch.empty_like(Av)
    gb = sch.adjoint(Lv, Av, t(w.gy, dtype), saved=z, x_in=xin, gx=gx, gL=gL, gM=gA)
    sch.check()
    assert col_rel_err(host(z), z_ref) < TOL[dtype]
    assert col_rel_err(host(zs), z_ref) < TOL[dtype]
    assert col_rel_err(host(gb), gb_ref) < TOL[dtype]
    assert col_rel_err(host(gx), gx_ref) < TOL[dtype]
    assert vec_rel_err(host(gL), gL_ref) < TOL[dtype]
    assert vec_rel_err(host(gA), gA_ref) < TOL[dtype]


@pytest.mark.parametrize("k,lpr", [(1, 0), (1, 2), (16, 16), (32, 32)])
def test_trsv_and_trsv_spmv_slices(k, lpr):
    need_cuda()
    n = 20000
    L = I.powerlaw_lower(n, 8, 600, 4)
    Mp = I.band_random(n, 8, 500, 5)
    b = I.dense_vectors(n, k, 3, I.S_RHS)
    gy = I.dense_vectors(n, k, 4, I.S_RHS)
    x_ref, y_ref = oracle.trsv_spmv(L, Mp, b)
    gb_ref, gL_ref, gM_ref = oracle.adj_trsv_spmv(L, Mp, x_ref, gy)
    st = sf.inspect("trsv", dev_csr(L), lanes_per_row=lpr)
    st.set_slices(0, 20)
    assert _split_happened(st)
    x = st.execute(t(L.vals), b=t(b))
    st.check()
    assert col_rel_err(host(x), x_ref) < 1e-12
    sch = sf.inspect("trsv_spmv", dev_csr(L), dev_csr(Mp), want_adjoint=True, lanes_per_row=lpr)
    sch.set_slices(-1, 20)
    assert _split_happened(sch, 0)
    xs = torch.empty((n, k), device="cuda", dtype=torch.float64)
    y = sch.execute(t(L.vals), t(Mp.vals), b=t(b), x_save=xs)
    gL, gM = torch.empty(L.nnz, device="cuda", dtype=torch.float64), torch.empty(Mp.nnz, device="cuda",
                                                                               dtype=torch.float64)
    gb = sch.adjoint(t(L.vals), t(Mp.vals), t(gy), saved=xs, gL=gL, gM=gM)
    sch.check()
    assert col_rel_err(host(xs), x_ref) < 1e-12
    assert col_rel_err(host(y), y_ref) < 1e-12
    assert col_rel_err(host(gb), gb_ref) < 1e-12
    assert vec_rel_err(host(gL), gL_ref) < 1e-12
    assert vec_rel_err(host(gM), gM_ref) < 1e-12


def test_slices_follow_recut_and_dynamic_queue_and_turn_off():
    need_cuda()
    w = _powerlaw(1, seed=35)
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    args = (t(w.L.vals), t(w.M.vals))
    kw = dict(b=t(w.b), x_in=t(w.x_in))
    for dyn in (False, True):
        sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), dynamic_queue=dyn)
        sch.set_slices(0, 40)
        assert _split_happened(sch)
        sch.recut(0, 90, 1, 32)
        assert _split_happened(sch) and sch.info()["part_cost_target"] == 90
        z = sch.execute(*args, **kw)
        sch.check()
        assert col_rel_err(host(z), z_ref) < 1e-12
        sch.set_slices(0, 0)
        assert sch.info()["slice_units"] == 0
        z = sch.execute(*args, **kw)
        sch.check()
        assert col_rel_err(host(z), z_ref) < 1e-12


def test_slices_integer_exact_bitwise():
    # unit lower {-1, 0, 1} L with long rows and b = L x_int: the split sums are exact integers
    need_cuda()
    n = 4000
    pat = I.powerlaw_lower(n, 6, 400, 78)
    Lv = np.where(pat.colidx == np.repeat(np.arange(n), np.diff(pat.rowptr)), 1.0, np.sign(pat.vals))
    L = I.Csr(n, n, pat.rowptr, pat.colidx, Lv.astype(np.float64))
    x_int = (np.arange(n) % 3 - 1).astype(np.float64).reshape(n, 1)
    b = oracle.spmv(L, x_int)
    sch = sf.inspect("trsv", dev_csr(L))
    sch.set_slices(0, 8)
    assert _split_happened(sch)
    x = sch.execute(t(L.vals), b=t(b))
    sch.check()
    assert np.array_equal(host(x), x_int)


def test_rhs_tile_per_direction():
    # the forward and adjoint passes of one schedule keep their own right-hand-side tiles
    need_cuda()
    w = _powerlaw(16, seed=37)
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    gb_ref, gx_ref, _, _ = oracle.adj_spmv_trsv(w.M, w.L, w.x_in, z_ref, w.gy)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, lanes_per_row=16)
    Lv, Av, xin = t(w.L.vals), t(w.M.vals), t(w.x_in)
    for fwd_rt, adj_rt in ((4, 16), (16, 2), (0, 8)):
        sch.set_rhs_tile(0, fwd_rt)
        sch.set_rhs_tile(1, adj_rt)
        info = sch.info()
        assert (info["fwd_rhs_tile"], info["adj_rhs_tile"]) == (fwd_rt, adj_rt)
        z = sch.execute(Lv, Av, b=t(w.b), x_in=xin)
        gx = torch.empty_like(xin)
        gb = sch.adjoint(Lv, Av, t(w.gy), saved=z, x_in=xin, gx=gx)
        sch.check()
        assert col_rel_err(host(z), z_ref) < 1e-12
        assert col_rel_err(host(gb), gb_ref) < 1e-12
        assert col_rel_err(host(gx), gx_ref) < 1e-12
