"""Fused adjoint passes: parity with the oracle's closed-form gradients, and the
autograd wrappers checked by central finite differences on the GPU's own forward pass
(a 16^3 copy of the 128^3 workload) and by torch.autograd.gradcheck on tiny inputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t, vec_rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,ef", [(1, False), (1, True), (4, False), (32, False)])
@pytest.mark.parametrize("lpr", [0, 1, 32])
def test_adjoint_trsv_spmv(dtype, k, ef, lpr):
    need_cuda()
    w = I.trsv_spmv_lap3d_band(11, per_row=6, halfband=150, seed=41, k=k)
    x_ref, _ = oracle.trsv_spmv(w.L, w.M, w.b)
    gb_ref, gL_ref, gM_ref = oracle.adj_trsv_spmv(w.L, w.M, x_ref, w.gy)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, lanes_per_row=lpr,
                     epoch_flags=ef)
    Lv, Mv = t(w.L.vals, dtype), t(w.M.vals, dtype)
    xs = torch.empty((w.n, k), device="cuda", dtype=dtype)
    sch.execute(Lv, Mv, b=t(w.b, dtype), x_save=xs)
    gL, gM = torch.empty_like(Lv), torch.empty_like(Mv)
    gb = sch.adjoint(Lv, Mv, t(w.gy, dtype), saved=xs, gL=gL, gM=gM)
    sch.check()
    tol = TOL[dtype]
    assert col_rel_err(host(gb), gb_ref) < tol
    assert vec_rel_err(host(gL), gL_ref) < tol
    assert vec_rel_err(host(gM), gM_ref) < tol


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,ef", [(1, False), (1, True), (16, False)])
@pytest.mark.parametrize("lpr", [0, 1, 16, 32])
def test_adjoint_spmv_trsv(dtype, k, ef, lpr):
    need_cuda()
    w = I.spmv_trsv_powerlaw(n=12000, k=k, mean=16, lmax=300, halfband=700, seed=43)
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    gb_ref, gx_ref, gL_ref, gA_ref = oracle.adj_spmv_trsv(w.M, w.L, w.x_in, z_ref, w.gy)
    if lpr and lpr < k:
        pytest.skip("lanes per row below the RHS tile is raised to the tile")
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, lanes_per_row=lpr,
                     epoch_flags=ef)
    Lv, Av, xin = t(w.L.vals, dtype), t(w.M.vals, dtype), t(w.x_in, dtype)
    z = sch.execute(Lv, Av, b=t(w.b, dtype), x_in=xin)
    gx, gL, gA = torch.empty_like(xin), torch.empty_like(Lv), torch.empty_like(Av)
    gb = sch.adjoint(Lv, Av, t(w.gy, dtype), saved=z, x_in=xin, gx=gx, gL=gL, gM=gA)
    sch.check()
    tol = TOL[dtype]
    assert col_rel_err(host(gb), gb_ref) < tol
    assert col_rel_err(host(gx), gx_ref) < tol
    assert vec_rel_err(host(gL), gL_ref) < tol
    assert vec_rel_err(host(gA), gA_ref) < tol


def test_adjoint_optional_outputs():
    need_cuda()
    w = I.spmv_trsv_powerlaw(n=3000, k=1, mean=8, lmax=50, halfband=200, seed=45)
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    gb_ref, _, _, _ = oracle.adj_spmv_trsv(w.M, w.L, w.x_in, z_ref, w.gy)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True)
    gb = sch.adjoint(t(w.L.vals), t(w.M.vals), t(w.gy))      # only gb requested
    sch.check()
    assert col_rel_err(host(gb), gb_ref) < 1e-12
    plain = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M))
    with pytest.raises(sf.SparseFusionError) as e:
        plain.adjoint(t(w.L.vals), t(w.M.vals), t(w.gy))
    assert e.value.status == 8


def _fd(f, p, d, h):
    with torch.no_grad():
        return (f(p + h * d) - f(p - h * d)) / (2 * h)


def test_autograd_trsv_spmv_finite_differences_16cubed():
    need_cuda()
    w = I.trsv_spmv_lap3d_band(16, seed=2)          # the 16^3 copy of the 128^3 workload
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True)
    Lv = t(w.L.vals).requires_grad_()
    Mv = t(w.M.vals).requires_grad_()
    b = t(w.b).requires_grad_()
    gy = t(w.gy)
    y = sf.fused(sch, Lv, Mv, b)
    (y * gy).sum().backward()
    for r in range(8):
        dL = t(I.uniform_pm1(900 + r, 1, np.arange(w.L.nnz)))
        dM = t(I.uniform_pm1(910 + r, 1, np.arange(w.M.nnz)))
        db = t(I.uniform_pm1(920 + r, 1, np.arange(w.n)).reshape(w.n, 1))
        h = 1e-6
        fL = _fd(lambda v: (sch.execute(v, Mv.detach(), b=b.detach()) * gy).sum(), Lv.detach(), dL, h)
        fM = _fd(lambda v: (sch.execute(Lv.detach(), v, b=b.detach()) * gy).sum(), Mv.detach(), dM, h)
        fb = _fd(lambda v: (sch.execute(Lv.detach(), Mv.detach(), b=v) * gy).sum(), b.detach(), db, h)
        for fd, an in ((fL, (Lv.grad * dL).sum()), (fM, (Mv.grad * dM).sum()), (fb, (b.grad * db).sum())):
            assert abs(float(fd) - float(an)) <= 1e-6 * max(1.0, abs(float(an)))
    sch.check()


def test_autograd_spmv_trsv_gradcheck_tiny():
    need_cuda()
    w = I.spmv_trsv_powerlaw(n=40, k=2, mean=4, lmax=8, halfband=12, seed=47)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True)
    Lv = t(w.L.vals).requires_grad_()
    Av = t(w.M.vals).requires_grad_()
    xin = t(w.x_in).requires_grad_()
    b = t(w.b).requires_grad_()
    assert torch.autograd.gradcheck(lambda a, c, d, e: sf.fused(sch, a, c, d, e), (Lv, Av, xin, b),
                                    eps=1e-6, atol=1e-7, rtol=1e-5)
    sch.check()


def test_autograd_trsv_spmv_gradcheck_tiny():
    need_cuda()
    w = I.trsv_spmv_lap2d(6, seed=5)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True)
    Lv = t(w.L.vals).requires_grad_()
    Mv = t(w.M.vals).requires_grad_()
    b = t(w.b).requires_grad_()
    assert torch.autograd.gradcheck(lambda a, c, d: sf.fused(sch, a, c, d), (Lv, Mv, b), eps=1e-6, atol=1e-7,
                                    rtol=1e-5)
    sch.check()
