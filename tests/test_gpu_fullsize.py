"""Parity at full workload sizes: every output of the fused forward and adjoint passes
compared element by element with the FP64 oracle (which runs the whole workload in C),
in the default launch shape and, for the default benchmark workload, in an autotuned one.
Generation of the two largest workloads takes about a minute each."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t, vec_rel_err

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _trsv_spmv_full(w, dtype=torch.float64, tune=False):
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True)
    Lv, Mv, b, gy = t(w.L.vals, dtype), t(w.M.vals, dtype), t(w.b, dtype), t(w.gy, dtype)
    xs = torch.empty_like(b)
    if tune:
        from paper_2111_12238_gb300 import autotune
        autotune.tune(sch, lambda: sch.execute(Lv, Mv, b=b, x_save=xs), which=0, dtype=dtype, budget_s=3,
                      use_cache=False)
        autotune.tune(sch, lambda: sch.adjoint(Lv, Mv, gy, saved=xs), which=1, dtype=dtype, budget_s=3,
                      use_cache=False)
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    gL, gM = torch.empty_like(Lv), torch.empty_like(Mv)
    gb = sch.adjoint(Lv, Mv, gy, saved=xs, gL=gL, gM=gM)
    sch.check()
    return host(xs), host(y), host(gb), host(gL), host(gM)


@pytest.mark.parametrize("tune", [False, True])
def test_lap3d128_forward_and_adjoint_full(tune):
    need_cuda()
    w = I.trsv_spmv_lap3d_band(128, seed=2)
    x, y, gb, gL, gM = _trsv_spmv_full(w, tune=tune)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    gb_ref, gL_ref, gM_ref = oracle.adj_trsv_spmv(w.L, w.M, x_ref, w.gy)
    assert col_rel_err(x, x_ref) < 1e-12
    assert col_rel_err(y, y_ref) < 1e-12
    assert col_rel_err(gb, gb_ref) < 1e-12
    assert vec_rel_err(gL, gL_ref) < 1e-12
    assert vec_rel_err(gM, gM_ref) < 1e-12


def test_lap2d64_forward_full():
    need_cuda()
    w = I.trsv_spmv_lap2d(64, seed=1)
    x, y, gb, _, _ = _trsv_spmv_full(w)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    assert col_rel_err(y, y_ref) < 1e-12 and col_rel_err(x, x_ref) < 1e-12


def test_aniso100_ic0_trsv_k32_full():
    need_cuda()
    w = I.ic0_trsv_aniso3d(100, k=32, seed=3)
    sch = sf.inspect("ic0_trsv", dev_csr(w.L), rhs_tile=32)
    lf = torch.empty(w.L.nnz, device="cuda", dtype=torch.float64)
    y = sch.execute(t(w.L.vals), b=t(w.b), x_save=lf)
    sch.check()
    lf_ref, y_ref = oracle.ic0_trsv(w.L, w.b)
    assert vec_rel_err(host(lf), lf_ref) < 1e-12
    assert col_rel_err(host(y), y_ref) < 1e-12


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched512_forward_adjoint_full(dtype):
    need_cuda()
    w = I.batched_trsv_spmv(512, seed=4)
    sch = sf.inspect_batched("trsv_spmv", [dev_csr(x.L) for x in w.instances], [dev_csr(x.M) for x in w.instances],
                             want_adjoint=True)
    Lv = t(np.concatenate([x.L.vals for x in w.instances]), dtype)
    Mv = t(np.concatenate([x.M.vals for x in w.instances]), dtype)
    b, gy = t(w.b, dtype), t(w.gy, dtype)
    xs = torch.empty_like(b)
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    gL, gM = torch.empty_like(Lv), torch.empty_like(Mv)
    gb = sch.adjoint(Lv, Mv, gy, saved=xs, gL=gL, gM=gM)
    sch.check()
    y, gb, gL, gM = host(y), host(gb), host(gL), host(gM)
    tol = TOL[dtype]
    off = offL = offM = 0
    worst = 0.0
    for x in w.instances:
        xr, yr = oracle.trsv_spmv(x.L, x.M, x.b)
        gbr, gLr, gMr = oracle.adj_trsv_spmv(x.L, x.M, xr, x.gy)
        worst = max(worst, col_rel_err(y[off:off + x.n], yr), col_rel_err(gb[off:off + x.n], gbr),
                    vec_rel_err(gL[offL:offL + x.L.nnz], gLr), vec_rel_err(gM[offM:offM + x.M.nnz], gMr))
        off += x.n
        offL += x.L.nnz
        offM += x.M.nnz
    assert worst < tol


def test_powerlaw4m_spmv_trsv_k16_full():
    need_cuda()
    w = I.spmv_trsv_powerlaw(seed=5)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, rhs_tile=16)
    Lv, Av, xin, b, gz = t(w.L.vals), t(w.M.vals), t(w.x_in), t(w.b), t(w.gy)
    z = sch.execute(Lv, Av, b=b, x_in=xin)
    gx, gL, gA = torch.empty_like(xin), torch.empty_like(Lv), torch.empty_like(Av)
    gb = sch.adjoint(Lv, Av, gz, saved=z, x_in=xin, gx=gx, gL=gL, gM=gA)
    sch.check()
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    assert col_rel_err(host(z), z_ref) < 1e-12
    gb_ref, gx_ref, gL_ref, gA_ref = oracle.adj_spmv_trsv(w.M, w.L, w.x_in, z_ref, w.gy)
    assert col_rel_err(host(gb), gb_ref) < 1e-12
    assert col_rel_err(host(gx), gx_ref) < 1e-12
    assert vec_rel_err(host(gL), gL_ref) < 1e-12
    assert vec_rel_err(host(gA), gA_ref) < 1e-12
