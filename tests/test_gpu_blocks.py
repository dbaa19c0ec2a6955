"""Row-block executor (k = 1): its block order and level segments equal the oracle's bit for bit, and every
mode it serves matches the FP64 oracle for several block sizes (ragged last blocks, one
block, many tiny blocks), lane counts and both element types; its waits are bounded."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t, vec_rel_err
from tests._mats import dense_to_csr

pytestmark = pytest.mark.gpu

KINDS = {"trsv_spmv": (oracle.SEP, oracle.PAIRED_T), "spmv_trsv": (oracle.PAIRED, oracle.SEP_T),
         "trsv": (oracle.PAIRED, None)}


def _work(pair):
    if pair == "trsv_spmv":
        return I.trsv_spmv_lap3d_band(13, per_row=6, halfband=300, seed=21)
    if pair == "spmv_trsv":
        return I.spmv_trsv_powerlaw(n=9000, k=1, mean=10, lmax=120, halfband=500, seed=31)
    return I.trsv_spmv_lap3d_band(12, seed=5)


@pytest.mark.parametrize("pair", ["trsv_spmv", "spmv_trsv", "trsv"])
@pytest.mark.parametrize("B", [32, 1000, 4096, 10 ** 5])
def test_block_order_matches_oracle(pair, B):
    need_cuda()
    w = _work(pair)
    M = w.M if pair != "trsv" else None
    sch = sf.inspect(pair, dev_csr(w.L), dev_csr(M) if M is not None else None, want_adjoint=pair != "trsv",
                     block_rows=B)
    for which, kind in enumerate(KINDS[pair]):
        if kind is None:
            continue
        useM = M if kind in (oracle.SEP, oracle.SEP_T) else None
        lev = oracle.levels(kind, w.L, useM)
        ref_o, ref_bp = oracle.block_order(kind, w.L, useM, lev, B)
        got = sch.export_blocks(which)
        assert got["block_rows"] == B
        assert np.array_equal(got["order"], ref_o)
        assert np.array_equal(got["block_ptr"], ref_bp)
        ref_sp, ref_bs = oracle.block_segments(kind, w.n, ref_o, ref_bp, lev)
        assert np.array_equal(got["seg_ptr"], ref_sp)
        assert np.array_equal(got["block_seg"], ref_bs)
        assert oracle.validate(kind, w.L, useM, got["order"], got["block_ptr"]) == 0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lanes", [1, 2, 4, 32])
@pytest.mark.parametrize("B", [64, 1000, 8192])
def test_trsv_spmv_blocks_forward_adjoint(dtype, lanes, B):
    need_cuda()
    w = _work("trsv_spmv")
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    gb_ref, gL_ref, gM_ref = oracle.adj_trsv_spmv(w.L, w.M, x_ref, w.gy)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, block_rows=B, exec_mode=2)
    sch.reblock(-1, 0, 2, lanes)
    inf = sch.info()
    assert inf["exec_mode"] == 2 and inf["block_lanes"] == lanes and inf["n_blocks"] == -(-w.n // B)
    Lv, Mv, b, gy = t(w.L.vals, dtype), t(w.M.vals, dtype), t(w.b, dtype), t(w.gy, dtype)
    xs = torch.empty_like(b)
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    gL, gM = torch.empty_like(Lv), torch.empty_like(Mv)
    gb = sch.adjoint(Lv, Mv, gy, saved=xs, gL=gL, gM=gM)
    sch.check()
    tol = TOL[dtype]
    assert col_rel_err(host(xs), x_ref) < TOL[dtype]
    assert col_rel_err(host(y), y_ref) < TOL[dtype]
    assert col_rel_err(host(gb), gb_ref) < tol
    assert vec_rel_err(host(gL), gL_ref) < tol and vec_rel_err(host(gM), gM_ref) < tol


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("lanes,B", [(1, 512), (2, 2048), (4, 3000), (32, 9000)])
def test_spmv_trsv_blocks_forward_adjoint(dtype, lanes, B):
    need_cuda()
    w = _work("spmv_trsv")
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    gb_ref, gx_ref, gL_ref, gA_ref = oracle.adj_spmv_trsv(w.M, w.L, w.x_in, z_ref, w.gy)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, block_rows=B, exec_mode=2)
    sch.reblock(-1, 0, 2, lanes)
    Lv, Av, xin = t(w.L.vals, dtype), t(w.M.vals, dtype), t(w.x_in, dtype)
    z = sch.execute(Lv, Av, b=t(w.b, dtype), x_in=xin)
    gx, gL, gA = torch.empty_like(xin), torch.empty_like(Lv), torch.empty_like(Av)
    gb = sch.adjoint(Lv, Av, t(w.gy, dtype), saved=z, x_in=xin, gx=gx, gL=gL, gM=gA)
    sch.check()
    tol = TOL[dtype]
    assert col_rel_err(host(z), z_ref) < TOL[dtype]
    assert col_rel_err(host(gb), gb_ref) < tol and col_rel_err(host(gx), gx_ref) < tol
    assert vec_rel_err(host(gL), gL_ref) < tol and vec_rel_err(host(gA), gA_ref) < tol


def test_trsv_alone_blocks_and_integer_exact():
    need_cuda()
    n = 5000
    pat = I.powerlaw_lower(n, 3, 12, 77)
    Lv = np.where(pat.colidx == np.repeat(np.arange(n), np.diff(pat.rowptr)), 1.0, np.sign(pat.vals))
    L = I.Csr(n, n, pat.rowptr, pat.colidx, Lv)
    x_int = (np.arange(n) % 5 - 2).astype(np.float64).reshape(n, 1)
    b = oracle.spmv(L, x_int)
    for B in (128, 2048, 8192):
        sch = sf.inspect("trsv", dev_csr(L), block_rows=B, exec_mode=2)
        x = sch.execute(t(L.vals), b=t(b))
        sch.check()
        assert np.array_equal(host(x), x_int)


def test_batched_blocks_match_oracle():
    need_cuda()
    w = I.batched_trsv_spmv(count=10, nmin=300, nmax=9000, seed=12)
    sch = sf.inspect_batched("trsv_spmv", [dev_csr(x.L) for x in w.instances], [dev_csr(x.M) for x in w.instances],
                             want_adjoint=True, block_rows=4096, exec_mode=2)
    Lv = t(np.concatenate([x.L.vals for x in w.instances]))
    Mv = t(np.concatenate([x.M.vals for x in w.instances]))
    b, gy = t(w.b), t(w.gy)
    xs = torch.empty_like(b)
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    gb = sch.adjoint(Lv, Mv, gy, saved=xs)
    sch.check()
    off = 0
    for x in w.instances:
        xr, yr = oracle.trsv_spmv(x.L, x.M, x.b)
        gbr, _, _ = oracle.adj_trsv_spmv(x.L, x.M, xr, x.gy)
        assert col_rel_err(host(y)[off:off + x.n], yr) < 1e-12
        assert col_rel_err(host(gb)[off:off + x.n], gbr) < 1e-12
        off += x.n


def test_block_executor_timeout_is_reported():
    # one block of a bidiagonal system: every level segment holds one row. Swapping the
    # positions of rows 0 and 32 makes the first segment wait for row 31, which only a later
    # segment computes; the bounded wait must end the launch with SF_ERR_TIMEOUT.
    need_cuda()
    n = 64
    L = dense_to_csr(np.eye(n) * 2 + np.eye(n, k=-1))
    sch = sf.inspect("trsv", dev_csr(L), block_rows=64, exec_mode=2)
    sch.reblock(0, 0, 2, 32)
    sch.set_timeout(2_000_000)
    sch.debug_swap(0, 32)
    Lv, bb = t(L.vals), t(np.ones((n, 1)))
    sch.execute(Lv, b=bb)
    st, _ = sch.check_status()
    assert st == 5
    sch.debug_swap(0, 32)
    x = sch.execute(Lv, b=bb)
    sch.check()
    assert col_rel_err(host(x), oracle.trsv_lower(L, np.ones((n, 1)))) < 1e-14


# ---- warp-specialised row-block executor (exec_mode 3): producer warps stage each level's
# records in shared memory, consumer warps only compute

@pytest.mark.parametrize("mode", [3, 4])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("B", [64, 1000, 8192])
@pytest.mark.parametrize("g2", [0, -1])
def test_ws_trsv_spmv_forward_adjoint(mode, dtype, B, g2):
    need_cuda()
    w = _work("trsv_spmv")
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    gb_ref, gL_ref, gM_ref = oracle.adj_trsv_spmv(w.L, w.M, x_ref, w.gy)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, block_rows=B, exec_mode=mode,
                     g2_placement=g2)
    assert sch.info()["exec_mode"] == mode
    Lv, Mv, b, gy = t(w.L.vals, dtype), t(w.M.vals, dtype), t(w.b, dtype), t(w.gy, dtype)
    xs = torch.empty_like(b)
    for _ in range(2):
        y = sch.execute(Lv, Mv, b=b, x_save=xs)
        gL, gM = torch.empty_like(Lv), torch.empty_like(Mv)
        gb = sch.adjoint(Lv, Mv, gy, saved=xs, gL=gL, gM=gM)
        sch.check()
    tol = TOL[dtype]
    assert col_rel_err(host(xs), x_ref) < TOL[dtype]
    assert col_rel_err(host(y), y_ref) < TOL[dtype]
    assert col_rel_err(host(gb), gb_ref) < tol
    assert vec_rel_err(host(gL), gL_ref) < tol and vec_rel_err(host(gM), gM_ref) < tol


@pytest.mark.parametrize("mode", [3, 4])
@pytest.mark.parametrize("B", [512, 9000])
def test_ws_spmv_trsv_forward_adjoint(mode, B):
    # long A rows (power-law lengths up to 120) exercise the entries beyond the staged eight
    need_cuda()
    w = _work("spmv_trsv")
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    gb_ref, gx_ref, gL_ref, gA_ref = oracle.adj_spmv_trsv(w.M, w.L, w.x_in, z_ref, w.gy)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, block_rows=B, exec_mode=mode)
    Lv, Av, xin = t(w.L.vals), t(w.M.vals), t(w.x_in)
    z = sch.execute(Lv, Av, b=t(w.b), x_in=xin)
    gx, gL, gA = torch.empty_like(xin), torch.empty_like(Lv), torch.empty_like(Av)
    gb = sch.adjoint(Lv, Av, t(w.gy), saved=z, x_in=xin, gx=gx, gL=gL, gM=gA)
    sch.check()
    assert col_rel_err(host(z), z_ref) < 1e-12
    assert col_rel_err(host(gb), gb_ref) < 1e-12 and col_rel_err(host(gx), gx_ref) < 1e-12
    assert vec_rel_err(host(gL), gL_ref) < 1e-12 and vec_rel_err(host(gA), gA_ref) < 1e-12


@pytest.mark.parametrize("mode", [3, 4])
def test_ws_trsv_integer_exact_and_batched(mode):
    need_cuda()
    n = 5000
    pat = I.powerlaw_lower(n, 3, 12, 77)
    Lv = np.where(pat.colidx == np.repeat(np.arange(n), np.diff(pat.rowptr)), 1.0, np.sign(pat.vals))
    L = I.Csr(n, n, pat.rowptr, pat.colidx, Lv)
    x_int = (np.arange(n) % 5 - 2).astype(np.float64).reshape(n, 1)
    b = oracle.spmv(L, x_int)
    for B in (128, 8192):
        sch = sf.inspect("trsv", dev_csr(L), block_rows=B, exec_mode=mode)
        x = sch.execute(t(L.vals), b=t(b))
        sch.check()
        assert np.array_equal(host(x), x_int)
    wb = I.batched_trsv_spmv(count=10, nmin=300, nmax=9000, seed=12)
    sb = sf.inspect_batched("trsv_spmv", [dev_csr(x.L) for x in wb.instances], [dev_csr(x.M) for x in wb.instances],
                            want_adjoint=True, block_rows=4096, exec_mode=mode)
    Lb = t(np.concatenate([x.L.vals for x in wb.instances]))
    Mb = t(np.concatenate([x.M.vals for x in wb.instances]))
    xs = torch.empty_like(t(wb.b))
    y = sb.execute(Lb, Mb, b=t(wb.b), x_save=xs)
    gb = sb.adjoint(Lb, Mb, t(wb.gy), saved=xs)
    sb.check()
    off = 0
    for x in wb.instances:
        xr, yr = oracle.trsv_spmv(x.L, x.M, x.b)
        gbr, _, _ = oracle.adj_trsv_spmv(x.L, x.M, xr, x.gy)
        assert col_rel_err(host(y)[off:off + x.n], yr) < 1e-12
        assert col_rel_err(host(gb)[off:off + x.n], gbr) < 1e-12
        off += x.n


@pytest.mark.parametrize("mode", [3, 4])
def test_ws_timeout_is_reported(mode):
    # a row placed in a level segment before its input: the bounded wait ends the launch
    need_cuda()
    n = 64
    L = dense_to_csr(np.eye(n) * 2 + np.eye(n, k=-1))
    sch = sf.inspect("trsv", dev_csr(L), block_rows=64, exec_mode=mode)
    sch.set_timeout(2_000_000)
    sch.debug_swap(0, 32)
    Lv, bb = t(L.vals), t(np.ones((n, 1)))
    sch.execute(Lv, b=bb)
    st, _ = sch.check_status()
    assert st == 5
    sch.debug_swap(0, 32)
    x = sch.execute(Lv, b=bb)
    sch.check()
    assert col_rel_err(host(x), oracle.trsv_lower(L, np.ones((n, 1)))) < 1e-14


def test_tma_reblock_and_replace_repack():
    # the packed records follow the block order through re-blocking and re-placement
    need_cuda()
    w = _work("trsv_spmv")
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), block_rows=1000)
    Lv, Mv, b = t(w.L.vals), t(w.M.vals), t(w.b)
    for B, g2 in ((1000, 0), (4096, 0), (4096, -1), (512, 3)):
        sch.reblock(0, B, 4, 0)
        sch.replace(0, g2)
        y = sch.execute(Lv, Mv, b=b)
        sch.check()
        assert col_rel_err(host(y), y_ref) < 1e-12
