"""Separated packing of SpMV -> SpTRSV (sf_schedule_set_packing(0), §3.2.3): every group of the
partition executor computes r = b - A x_in for its rows before it takes partitions and
publishes it by value; the solve rows then wait for their r_i and walk L's strict part only.
Results must match the FP64 oracle for both storage forms of L, one and many right-hand
sides, both element types, with rows split over teams and with the ticket queue; an exact
integer system must match bit for bit; what separated packing does not serve is refused."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t

pytestmark = pytest.mark.gpu

UNSUPPORTED = 8


def _powerlaw(k, seed=51):
    return I.spmv_trsv_powerlaw(n=20000, k=k, mean=16, lmax=800, halfband=1500, seed=seed)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,lpr", [(1, 0), (1, 4), (16, 16)])
@pytest.mark.parametrize("shared", [False, True])
@pytest.mark.parametrize("slices", [0, 40])
def test_separated_matches_oracle(dtype, k, lpr, shared, slices):
    need_cuda()
    w = _powerlaw(k)
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), lanes_per_row=lpr)
    assert sch.info()["packing"] == 1
    sch.set_packing(0)
    assert sch.info()["packing"] == 0
    sch.set_slices(0, slices)
    Lv, Av, xin, b = t(w.L.vals, dtype), t(w.M.vals, dtype), t(w.x_in, dtype), t(w.b, dtype)
    z = sch.execute(None if shared else Lv, Av, b=b, x_in=xin)
    z2 = sch.execute(None if shared else Lv, Av, b=b, x_in=xin)   # the r buffer is reset per call
    sch.check()
    assert col_rel_err(host(z), z_ref) < TOL[dtype]
    assert col_rel_err(host(z2), z_ref) < TOL[dtype]
    if lpr < 16:
        # narrow groups add a row's products in entry order; wide ones (16 or more lanes) add
        # the operands that were not yet published when first read at the end of the lane's
        # walk, so their rounding order (not their tolerance) varies from call to call
        assert torch.equal(z, z2)
    sch.set_packing(1)
    zi = sch.execute(None if shared else Lv, Av, b=b, x_in=xin)
    sch.check()
    assert col_rel_err(host(zi), z_ref) < TOL[dtype]


def test_separated_with_ticket_queue():
    need_cuda()
    w = _powerlaw(1, seed=53)
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), dynamic_queue=True)
    sch.set_packing(0)
    sch.set_slices(0, 30)
    z = sch.execute(None, t(w.M.vals), b=t(w.b), x_in=t(w.x_in))
    sch.check()
    assert col_rel_err(host(z), z_ref) < 1e-12


def test_separated_integer_exact_bitwise():
    # A = L (unit lower, entries in {-1, 0, 1}) plus an upper band of small integers; b is chosen
    # so that r = b - A x_in = L z_int: every value on the way is an exact integer
    need_cuda()
    n = 5000
    pat = I.powerlaw_lower(n, 6, 300, 61)
    diag = pat.colidx == np.repeat(np.arange(n), np.diff(pat.rowptr))
    L = I.Csr(n, n, pat.rowptr, pat.colidx, np.where(diag, 1.0, np.sign(pat.vals)))
    up = I.band_random(n, 4, 50, 62)
    rows = []
    for i in range(n):
        lc = L.colidx[L.rowptr[i]:L.rowptr[i + 1]]
        lv = L.vals[L.rowptr[i]:L.rowptr[i + 1]]
        uc = up.colidx[up.rowptr[i]:up.rowptr[i + 1]]
        uv = np.round(up.vals[up.rowptr[i]:up.rowptr[i + 1]] * 3)
        keep = uc > i
        cols = np.concatenate([lc, uc[keep]])
        vals = np.concatenate([lv, uv[keep]])
        o = np.argsort(cols, kind="stable")
        rows.append((cols[o], vals[o]))
    rp = np.concatenate([[0], np.cumsum([len(c) for c, _ in rows])]).astype(np.int32)
    A = I.Csr(n, n, rp, np.concatenate([c for c, _ in rows]).astype(np.int32),
              np.concatenate([v for _, v in rows]).astype(np.float64))
    x_in = (np.arange(n) % 5 - 2).astype(np.float64).reshape(n, 1)
    z_int = (np.arange(n) % 7 - 3).astype(np.float64).reshape(n, 1)
    b = oracle.spmv(A, x_in) + oracle.spmv(L, z_int)
    sch = sf.inspect("spmv_trsv", dev_csr(L), dev_csr(A))
    sch.set_packing(0)
    for Lv in (t(L.vals), None):
        z = sch.execute(Lv, t(A.vals), b=t(b), x_in=t(x_in))
        sch.check()
        assert np.array_equal(host(z), z_int)


def test_separated_refusals():
    need_cuda()
    w = _powerlaw(4, seed=55)
    # epoch flags (no value flags) cannot wait for r by value
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), epoch_flags=True, lanes_per_row=4)
    sch.set_packing(0)
    with pytest.raises(sf.SparseFusionError) as ei:
        sch.execute(t(w.L.vals), t(w.M.vals), b=t(w.b), x_in=t(w.x_in))
    assert ei.value.status == UNSUPPORTED
    # other pairs have one packing
    s2 = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M))
    with pytest.raises(sf.SparseFusionError) as ei:
        s2.set_packing(1)
    assert ei.value.status == UNSUPPORTED
    with pytest.raises(sf.SparseFusionError):
        sch.set_packing(2)
