"""Single-CTA executor (exec_mode 5, k = 1): the joint DAG of a SpTRSV -> SpMV (or SpTRSV alone)
runs on one CTA per instance (the whole system, or each instance of a batch) with one CTA
barrier per level segment and x, the order and L in shared memory as far as they fit. Results
match the FP64 oracle for both element types whatever is staged (everything, x and the order,
x alone, nothing); exact integer systems match bit for bit; the per-instance block order equals
the oracle's; what the executor does not serve is refused before anything runs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t

UNSUPPORTED = 8
INVALID_ARG = 1

pytestmark = pytest.mark.gpu


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
    # whole instances only: no block size, and 1, 2 or 4 CTAs per SM
    with pytest.raises(sf.SparseFusionError) as ei:
        sch.reblock(0, 512, 5, 0)
    assert ei.value.status == INVALID_ARG
    with pytest.raises(sf.SparseFusionError) as ei:
        sch.reblock(0, 0, 5, 32)
    assert ei.value.status == INVALID_ARG


def test_x_larger_than_shared_memory():
    # 40000 doubles do not fit in one CTA's shared memory: x lives in the output buffer; the
    # same system in FP32 keeps x on chip
    need_cuda()
    n = 40000
    L = I.powerlaw_lower(n, 3, 20, 86)
    b = I.dense_vectors(n, 1, 87, I.S_RHS)
    x_ref = oracle.trsv_lower(L, b)
    sch = sf.inspect("trsv", dev_csr(L))
    sch.reblock(0, 0, 5, 0)
    for dtype in (torch.float64, torch.float32):
        x = sch.execute(t(L.vals, dtype), b=t(b, dtype))
        sch.check()
        assert col_rel_err(host(x), x_ref) < TOL[dtype]


def _blockdiag(mats):
    n = sum(m.n_rows for m in mats)
    rp, ci, vals, off, eoff = [np.zeros(1, np.int32)], [], [], 0, 0
    for m in mats:
        rp.append((m.rowptr[1:] + eoff).astype(np.int32))
        ci.append((m.colidx + off).astype(np.int32))
        vals.append(m.vals)
        off += m.n_rows
        eoff += int(m.rowptr[-1])
    return I.Csr(n, n, np.concatenate(rp), np.concatenate(ci), np.concatenate(vals))


@pytest.mark.parametrize("cps", [1, 2, 4])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_one_cta_per_instance(cps, dtype):
    # instance sizes 300 .. 40000: at 4 CTAs per SM (56 KB each) the large ones keep nothing on
    # chip, at 1 CTA per SM the small ones stage everything
    need_cuda()
    w = I.batched_trsv_spmv(count=24, nmin=300, nmax=40000, seed=12)
    sch = sf.inspect_batched("trsv_spmv", [dev_csr(x.L) for x in w.instances], [dev_csr(x.M) for x in w.instances])
    sch.reblock(0, 0, 5, cps)
    inf = sch.info()
    assert inf["exec_mode"] == 5 and inf["n_blocks"] == 24
    assert sch.launches(0, 1) == 1
    Lv = t(np.concatenate([x.L.vals for x in w.instances]), dtype)
    Mv = t(np.concatenate([x.M.vals for x in w.instances]), dtype)
    b = t(w.b, dtype)
    xs = torch.empty_like(b)
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    sch.check()
    off = 0
    for x in w.instances:
        xr, yr = oracle.trsv_spmv(x.L, x.M, x.b)
        assert col_rel_err(host(xs)[off:off + x.n], xr) < TOL[dtype]
        assert col_rel_err(host(y)[off:off + x.n], yr) < TOL[dtype]
        off += x.n
    # back to the row-block executor at its automatic size, then to the partitions
    sch.reblock(0, 0, 3, 0)
    B = min(8192, -(-w.n // 32) * 32)
    assert sch.info()["n_blocks"] == -(-w.n // B)
    y3 = sch.execute(Lv, Mv, b=b)
    sch.reblock(0, 0, 1, 0)
    y1 = sch.execute(Lv, Mv, b=b)
    sch.check()
    assert col_rel_err(host(y3), host(y)) < TOL[dtype] and col_rel_err(host(y1), host(y)) < TOL[dtype]


def test_per_instance_block_order_matches_oracle():
    need_cuda()
    w = I.batched_trsv_spmv(count=9, nmin=50, nmax=3000, seed=7)
    Lb = _blockdiag([x.L for x in w.instances])
    Mb = _blockdiag([x.M for x in w.instances])
    sch = sf.inspect_batched("trsv_spmv", [dev_csr(x.L) for x in w.instances], [dev_csr(x.M) for x in w.instances])
    sch.reblock(0, 0, 5, 0)
    got = sch.export_blocks(0)
    n = w.n
    lev = oracle.levels(oracle.SEP, Lb, Mb)
    inst_ptr = np.concatenate([[0], np.cumsum([x.n for x in w.instances])]).astype(np.int32)
    ref_o, ref_bp = oracle.block_order_instances(oracle.SEP, n, lev, inst_ptr)
    assert np.array_equal(got["order"], ref_o)
    assert np.array_equal(got["block_ptr"], ref_bp)
    ref_sp, ref_bs = oracle.block_segments(oracle.SEP, n, got["order"], got["block_ptr"], lev)
    assert np.array_equal(got["seg_ptr"], ref_sp) and np.array_equal(got["block_seg"], ref_bs)
    assert oracle.validate(oracle.SEP, Lb, Mb, got["order"], got["block_ptr"]) == 0
