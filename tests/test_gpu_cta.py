"""Single-CTA executor (exec_mode 5, k = 1): the whole joint DAG of a small SpTRSV -> SpMV (or
SpTRSV alone) runs in one CTA with x in shared memory and one CTA barrier per level segment.
Results match the FP64 oracle for both element types, with L staged in shared memory and
read from global memory when it does not fit; exact integer systems match bit for bit; what
it does not serve is refused with SF_ERR_UNSUPPORTED before anything runs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t

pytestmark = pytest.mark.gpu

UNSUPPORTED = 8


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nx", [64, 150])
def test_trsv_spmv_lap2d_matches_oracle(dtype, nx):
    # 64 x 64: L and x in shared memory; 150 x 150 (n = 22500): x alone, L from global memory
    need_cuda()
    w = I.trsv_spmv_lap2d(nx, seed=3)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M))
    sch.reblock(0, 0, 5, 0)
    inf = sch.info()
    assert inf["exec_mode"] == 5 and inf["n_blocks"] == 1
    assert sch.launches(0, 1) == 1
    Lv, Mv, b = t(w.L.vals, dtype), t(w.M.vals, dtype), t(w.b, dtype)
    xs = torch.empty_like(b)
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    sch.check()
    assert col_rel_err(host(xs), x_ref) < TOL[dtype]
    assert col_rel_err(host(y), y_ref) < TOL[dtype]
    # without x_save, and again after the partition executor ran in between
    y2 = sch.execute(Lv, Mv, b=b)
    sch.check()
    assert torch.equal(y2, y)
    sch.reblock(0, 0, 1, 0)
    y3 = sch.execute(Lv, Mv, b=b)
    sch.reblock(0, 0, 5, 0)
    y4 = sch.execute(Lv, Mv, b=b)
    sch.check()
    assert col_rel_err(host(y3), y_ref) < TOL[dtype]
    assert torch.equal(y4, y)


@pytest.mark.parametrize("n", [3000, 6000])
def test_trsv_alone_integer_exact_bitwise(n):
    # unit lower {-1, 0, 1} L with power-law rows and b = L x_int: every sum is an exact integer
    # (3000 rows: L staged in shared memory; 6000 rows: L read from global memory)
    need_cuda()
    pat = I.powerlaw_lower(n, 4, 60, 81)
    Lv = np.where(pat.colidx == np.repeat(np.arange(n), np.diff(pat.rowptr)), 1.0, np.sign(pat.vals))
    L = I.Csr(n, n, pat.rowptr, pat.colidx, Lv.astype(np.float64))
    x_int = (np.arange(n) % 7 - 3).astype(np.float64).reshape(n, 1)
    b = oracle.spmv(L, x_int)
    sch = sf.inspect("trsv", dev_csr(L))
    sch.reblock(0, 0, 5, 0)
    x = sch.execute(t(L.vals), b=t(b))
    sch.check()
    assert np.array_equal(host(x), x_int)


def test_wide_levels_and_ragged_segments():
    # a band of random lower rows: level segments wider than the CTA's 1024 threads next to
    # segments of a few rows
    need_cuda()
    n = 9000
    L = I.powerlaw_lower(n, 3, 40, 83)
    Mp = I.band_random(n, 5, 200, 84)
    b = I.dense_vectors(n, 1, 85, I.S_RHS)
    x_ref, y_ref = oracle.trsv_spmv(L, Mp, b)
    sch = sf.inspect("trsv_spmv", dev_csr(L), dev_csr(Mp))
    sch.reblock(0, 0, 5, 0)
    xs = torch.empty((n, 1), device="cuda", dtype=torch.float64)
    y = sch.execute(t(L.vals), t(Mp.vals), b=t(b), x_save=xs)
    sch.check()
    assert col_rel_err(host(xs), x_ref) < 1e-12
    assert col_rel_err(host(y), y_ref) < 1e-12


def test_refusals():
    need_cuda()
    w = I.trsv_spmv_lap2d(32, seed=4)
    Lv, Mv = t(w.L.vals), t(w.M.vals)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True)
    sch.reblock(-1, 0, 5, 0)
    # several right-hand sides
    with pytest.raises(sf.SparseFusionError) as ei:
        sch.execute(Lv, Mv, b=t(np.ones((w.n, 4))))
    assert ei.value.status == UNSUPPORTED
    # the adjoint pass
    xs = torch.empty((w.n, 1), device="cuda", dtype=torch.float64)
    sch.execute(Lv, Mv, b=t(w.b), x_save=xs)
    with pytest.raises(sf.SparseFusionError) as ei:
        sch.adjoint(Lv, Mv, t(w.gy), saved=xs)
    assert ei.value.status == UNSUPPORTED
    # x larger than one CTA's shared memory (40000 doubles); the same system in FP32 fits
    n = 40000
    L = I.powerlaw_lower(n, 3, 20, 86)
    b = I.dense_vectors(n, 1, 87, I.S_RHS)
    s2 = sf.inspect("trsv", dev_csr(L))
    s2.reblock(0, 0, 5, 0)
    with pytest.raises(sf.SparseFusionError) as ei:
        s2.execute(t(L.vals), b=t(b))
    assert ei.value.status == UNSUPPORTED
    x = s2.execute(t(L.vals, torch.float32), b=t(b, torch.float32))
    s2.check()
    assert col_rel_err(host(x), oracle.trsv_lower(L, b)) < TOL[torch.float32]
