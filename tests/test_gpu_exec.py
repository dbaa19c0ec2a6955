"""Fused executor parity with the FP64 oracle on small and ragged inputs: every pair,
both element types, several right-hand-side counts and launch shapes, exact integer
cases, and the unfused two-launch path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import TOL, col_rel_err, dev_csr, host, need_cuda, t, vec_rel_err
from tests._mats import dense_to_csr, random_lower

pytestmark = pytest.mark.gpu


def _lap3d(nx=14, k=1):
    return I.trsv_spmv_lap3d_band(nx, per_row=6, halfband=200, seed=21, k=k)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,ef", [(1, False), (1, True), (3, False), (16, False), (32, False), (40, False)])
@pytest.mark.parametrize("lpr", [0, 1, 4, 32])
def test_trsv_spmv(dtype, k, ef, lpr):
    need_cuda()
    w = _lap3d(11, k)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), lanes_per_row=lpr, epoch_flags=ef)
    xs = torch.empty((w.n, k), device="cuda", dtype=dtype)
    y = sch.execute(t(w.L.vals, dtype), t(w.M.vals, dtype), b=t(w.b, dtype), x_save=xs)
    sch.check()
    assert col_rel_err(host(xs), x_ref) < TOL[dtype]
    assert col_rel_err(host(y), y_ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,ef", [(1, False), (1, True), (2, False), (16, False)])
@pytest.mark.parametrize("lpr", [0, 1, 8, 32])
def test_spmv_trsv(dtype, k, ef, lpr):
    need_cuda()
    w = I.spmv_trsv_powerlaw(n=20000, k=k, mean=16, lmax=400, halfband=900, seed=31)
    z_ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    sch = sf.inspect("spmv_trsv", dev_csr(w.L), dev_csr(w.M), lanes_per_row=lpr, epoch_flags=ef)
    z = sch.execute(t(w.L.vals, dtype), t(w.M.vals, dtype), b=t(w.b, dtype), x_in=t(w.x_in, dtype))
    sch.check()
    assert col_rel_err(host(z), z_ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("k", [1, 32])
@pytest.mark.parametrize("lpr", [0, 4, 32])
def test_ic0_trsv(dtype, k, lpr):
    need_cuda()
    w = I.ic0_trsv_aniso3d(12, k=k)
    lf_ref, y_ref = oracle.ic0_trsv(w.L, w.b)
    sch = sf.inspect("ic0_trsv", dev_csr(w.L), lanes_per_row=lpr)
    lf = torch.empty(w.L.nnz, device="cuda", dtype=dtype)
    y = sch.execute(t(w.L.vals, dtype), b=t(w.b, dtype), x_save=lf)
    sch.check()
    assert vec_rel_err(host(lf), lf_ref) < TOL[dtype]
    assert col_rel_err(host(y), y_ref) < TOL[dtype]


def test_ic0_with_intersections_and_alone():
    need_cuda()
    nx = 30
    offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    n, rowptr, cols, soffs, Msk = I._stencil_pattern((nx, nx), offs)
    vals = np.where(np.asarray([o == (0, 0) for o in soffs])[None, :], 9.0, -1.0)
    A = I._finish(n, n, rowptr, cols, np.broadcast_to(vals, Msk.shape)[Msk])
    L = I.lower_part(A)
    lf_ref = oracle.ic0(L)
    for lpr in (1, 4, 32):
        sch = sf.inspect("ic0", dev_csr(L), lanes_per_row=lpr)
        lf = torch.empty(L.nnz, device="cuda", dtype=torch.float64)
        sch.execute(t(L.vals), x_save=lf)
        sch.check()
        assert vec_rel_err(host(lf), lf_ref) < 1e-12


def _ic0_pair_count(L):
    """Brute force over the pattern: sum over entries (i, j), j < i, of the columns k < j in
    both row i and row j."""
    rp, ci = np.asarray(L.rowptr), np.asarray(L.colidx)
    rows = [set(ci[rp[i]:rp[i + 1]].tolist()) for i in range(L.n_rows)]
    total = 0
    for i in range(L.n_rows):
        for j in ci[rp[i]:rp[i + 1] - 1].tolist():
            total += sum(1 for c in rows[i] & rows[j] if c < j)
    return total


def _ic0_dense_rows(n, density, seed):
    """Lower part of a symmetric M-matrix with rows longer than a warp: off-diagonals
    -|U[-1,1]|, diagonal 1 + the absolute row sum of the symmetric matrix."""
    D = random_lower(n, density, seed)
    off = -np.abs(np.tril(D, -1))
    diag = 1.0 + np.abs(off + off.T).sum(axis=1)
    return dense_to_csr(off + np.diag(diag))


@pytest.mark.parametrize("case", ["stencil9", "long_rows"])
@pytest.mark.parametrize("path", ["value_flags", "epoch_flags", "search"])
def test_ic0_pairs_and_search_paths(case, path):
    # value_flags: pair lists, every value its own ready flag (the default); epoch_flags: pair
    # lists with per-row flags; search: common columns searched per call (per-row flags)
    need_cuda()
    if case == "stencil9":
        nx = 30
        offs = [(dx, dy) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
        n, rowptr, cols, soffs, Msk = I._stencil_pattern((nx, nx), offs)
        vals = np.where(np.asarray([o == (0, 0) for o in soffs])[None, :], 9.0, -1.0)
        L = I.lower_part(I._finish(n, n, rowptr, cols, np.broadcast_to(vals, Msk.shape)[Msk]))
    else:
        L = _ic0_dense_rows(300, 0.25, 41)
    n = L.n_rows
    lf_ref = oracle.ic0(L)
    b = I.dense_vectors(n, 8, 5, 1)
    lf_ref2, y_ref = oracle.ic0_trsv(L, b)
    for lpr, kt in ((1, 0), (4, 0), (32, 0), (32, 4)):
        use_pairs = path != "search"
        ef = path == "epoch_flags"
        sch = sf.inspect("ic0", dev_csr(L), lanes_per_row=lpr, epoch_flags=ef)
        assert sch.info()["ic0_pairs"] == _ic0_pair_count(L)
        sch.set_ic0_pairs(use_pairs)
        assert sch.info()["ic0_use_pairs"] == int(use_pairs)
        lf = torch.empty(L.nnz, device="cuda", dtype=torch.float64)
        sch.execute(t(L.vals), x_save=lf)
        sch.check()
        assert vec_rel_err(host(lf), lf_ref) < 1e-12
        st = sf.inspect("ic0_trsv", dev_csr(L), lanes_per_row=lpr, rhs_tile=kt, epoch_flags=ef)
        st.set_ic0_pairs(use_pairs)
        lf2 = torch.empty(L.nnz, device="cuda", dtype=torch.float64)
        y = st.execute(t(L.vals), b=t(b), x_save=lf2)
        st.check()
        assert vec_rel_err(host(lf2), lf_ref2) < 1e-12
        assert col_rel_err(host(y), y_ref) < 1e-12


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_ic0_occupancy_variant(dtype):
    need_cuda()
    w = I.ic0_trsv_aniso3d(14, k=32)
    lf_ref, y_ref = oracle.ic0_trsv(w.L, w.b)
    sch = sf.inspect("ic0_trsv", dev_csr(w.L), lanes_per_row=32, rhs_tile=32)
    sch.set_occupancy(0, 3)
    assert sch.info()["min_blocks"] == 3
    lf = torch.empty(w.L.nnz, device="cuda", dtype=dtype)
    y = sch.execute(t(w.L.vals, dtype), b=t(w.b, dtype), x_save=lf)
    sch.check()
    assert vec_rel_err(host(lf), lf_ref) < TOL[dtype]
    assert col_rel_err(host(y), y_ref) < TOL[dtype]


def test_ic0_pairs_setter_rejects_other_pairs():
    need_cuda()
    w = _lap3d(6, 1)
    sch = sf.inspect("trsv", dev_csr(w.L))
    assert sch.info()["ic0_pairs"] == 0
    with pytest.raises(sf.SparseFusionError):
        sch.set_ic0_pairs(True)


@pytest.mark.parametrize("k,ef", [(1, False), (1, True), (5, False)])
def test_trsv_alone_and_unfused_path(k, ef):
    need_cuda()
    w = _lap3d(10, k)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    st = sf.inspect("trsv", dev_csr(w.L), epoch_flags=ef)
    x = st.execute(t(w.L.vals), b=t(w.b))
    y = sf.spmv(dev_csr(w.M), t(w.M.vals), x)
    st.check()
    assert col_rel_err(host(x), x_ref) < 1e-12
    assert col_rel_err(host(y), y_ref) < 1e-12
    r = sf.spmv(dev_csr(w.M), t(w.M.vals), t(w.b), b=t(w.b))
    torch.cuda.synchronize()
    assert col_rel_err(host(r), oracle.residual(w.M, w.b, w.b)) < 1e-12


def test_integer_exact_bitwise():
    # unit lower-triangular {-1,0,1} L, integer M and b: every partial sum is an exact
    # integer, so the fused result must equal the oracle bit for bit in any summation order
    need_cuda()
    n = 3000
    rng_pat = I.powerlaw_lower(n, 3, 12, 77)
    Lv = np.where(rng_pat.colidx == np.repeat(np.arange(n), np.diff(rng_pat.rowptr)), 1.0,
                  np.sign(rng_pat.vals)).astype(np.float64)
    L = I.Csr(n, n, rng_pat.rowptr, rng_pat.colidx, Lv)
    # keep the solution bounded: b = L * x_int with small integer x_int
    x_int = (np.arange(n) % 5 - 2).astype(np.float64).reshape(n, 1)
    b = oracle.spmv(L, x_int)
    Mp = I.band_random(n, 4, 20, 5)
    M = I.Csr(n, n, Mp.rowptr, Mp.colidx, np.round(Mp.vals * 4))
    x_ref, y_ref = oracle.trsv_spmv(L, M, b)
    assert np.array_equal(x_ref, x_int)
    for lpr, ef in ((1, False), (4, False), (32, False), (4, True)):
        sch = sf.inspect("trsv_spmv", dev_csr(L), dev_csr(M), lanes_per_row=lpr, epoch_flags=ef)
        xs = torch.empty((n, 1), device="cuda", dtype=torch.float64)
        y = sch.execute(t(L.vals), t(M.vals), b=t(b), x_save=xs)
        sch.check()
        assert np.array_equal(host(xs), x_ref)
        assert np.array_equal(host(y), y_ref)


def test_edge_cases_tiny_and_diagonal():
    need_cuda()
    # n = 1
    L1 = dense_to_csr(np.array([[4.0]]))
    M1 = dense_to_csr(np.array([[-2.0]]))
    b1 = np.array([[3.0]])
    sch = sf.inspect("trsv_spmv", dev_csr(L1), dev_csr(M1))
    y = sch.execute(t(L1.vals), t(M1.vals), b=t(b1))
    sch.check()
    assert host(y)[0, 0] == -2.0 * (3.0 / 4.0)
    # diagonal L (depth 1) and an M with empty rows
    n = 1000
    d = 1.0 + np.arange(n) % 7
    L = dense_to_csr(np.diag(d))
    D = np.zeros((n, n))
    D[::3, 5] = 1.5
    M = dense_to_csr(D)
    b = I.dense_vectors(n, 2, 3, I.S_RHS)
    x_ref, y_ref = oracle.trsv_spmv(L, M, b)
    sch = sf.inspect("trsv_spmv", dev_csr(L), dev_csr(M))
    assert sch.info()["depth"] == 2
    y = sch.execute(t(L.vals), t(M.vals), b=t(b))
    sch.check()
    assert col_rel_err(host(y), y_ref) < 1e-15
    # dense lower triangle (long rows, depth n)
    Dd = random_lower(200, 1.0, 5)
    Ld = dense_to_csr(Dd)
    bd = I.dense_vectors(200, 1, 2, I.S_RHS)
    for lpr in (1, 32):
        sch = sf.inspect("trsv", dev_csr(Ld), lanes_per_row=lpr)
        x = sch.execute(t(Ld.vals), b=t(bd))
        sch.check()
        assert col_rel_err(host(x), oracle.trsv_lower(Ld, bd)) < 1e-12


@pytest.mark.parametrize("ef", [False, True])
def test_repeated_launches_and_epochs(ef):
    # many launches of one schedule: flags are never cleared, the epoch advances; value
    # flags are reset by the launch itself
    need_cuda()
    w = _lap3d(9, 1)
    _, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), epoch_flags=ef)
    Lv, Mv, b = t(w.L.vals), t(w.M.vals), t(w.b)
    y = torch.empty_like(b)
    for _ in range(50):
        sch.execute(Lv, Mv, b=b, y=y)
    sch.check()
    assert col_rel_err(host(y), y_ref) < 1e-12
    # changing k between launches reuses the same schedule
    b3 = t(np.repeat(w.b, 3, axis=1))
    y3 = sch.execute(Lv, Mv, b=b3)
    sch.check()
    assert col_rel_err(host(y3), np.repeat(y_ref, 3, axis=1)) < 1e-12


@pytest.mark.parametrize("ef", [False, True])
def test_cuda_graph_replay(ef):
    need_cuda()
    w = _lap3d(10, 1)
    _, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), epoch_flags=ef)
    g = sf.GraphedExecute(sch, L_vals=t(w.L.vals), M_vals=t(w.M.vals), b=t(w.b), y=torch.empty((w.n, 1), device="cuda",
                                                                                             dtype=torch.float64))
    for _ in range(5):
        out = g.replay()
    sch.check()
    assert col_rel_err(host(out), y_ref) < 1e-12


@pytest.mark.parametrize("bps", [1, 2])
def test_grid_limits_and_set_launch(bps):
    # fewer resident blocks and launch-shape changes after inspection keep results exact
    need_cuda()
    w = _lap3d(12, 1)
    _, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), blocks_per_sm=bps)
    Lv, Mv, b = t(w.L.vals), t(w.M.vals), t(w.b)
    for lpr, ef in ((1, 0), (8, 1), (32, 0)):
        sch.set_launch(lanes_per_row=lpr, epoch_flags=ef)
        y = sch.execute(Lv, Mv, b=b)
        sch.check()
        assert col_rel_err(host(y), y_ref) < 1e-12
    assert sch.info()["blocks_per_sm"] == bps


@pytest.mark.parametrize("pair", ["trsv_spmv", "spmv_trsv"])
@pytest.mark.parametrize("lpr", [1, 4])
def test_dynamic_ticket_queue(pair, lpr):
    need_cuda()
    if pair == "trsv_spmv":
        w = _lap3d(12, 1)
        ref = oracle.trsv_spmv(w.L, w.M, w.b)[1]
    else:
        w = I.spmv_trsv_powerlaw(n=20000, k=1, mean=16, lmax=400, halfband=900, seed=31)
        ref = oracle.spmv_trsv(w.M, w.L, w.x_in, w.b)
    sch = sf.inspect(pair, dev_csr(w.L), dev_csr(w.M), lanes_per_row=lpr, dynamic_queue=True)
    assert sch.info()["dynamic_queue"] == 1
    y = sch.execute(t(w.L.vals), t(w.M.vals), b=t(w.b), x_in=t(w.x_in) if w.x_in is not None else None)
    sch.check()
    assert col_rel_err(host(y), ref) < 1e-12


def test_recut_and_autotune_keep_results_exact():
    need_cuda()
    from paper_2111_12238_gb300 import autotune
    w = _lap3d(12, 1)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    gb_ref, _, _ = oracle.adj_trsv_spmv(w.L, w.M, x_ref, w.gy)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True)
    Lv, Mv, b, gy = t(w.L.vals), t(w.M.vals), t(w.b), t(w.gy)
    xs = torch.empty_like(b)
    p0 = sch.info()["n_parts"]
    sch.recut(0, 10 ** 9, 32)
    assert sch.info()["n_parts"] == 1 and sch.info()["lanes_per_row"] == 32
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    sch.check()
    assert col_rel_err(host(y), y_ref) < 1e-12
    res = autotune.tune(sch, lambda: sch.execute(Lv, Mv, b=b, x_save=xs), which=0, budget_s=2.0, use_cache=False)
    resa = autotune.tune(sch, lambda: sch.adjoint(Lv, Mv, gy, saved=xs), which=1, budget_s=2.0, use_cache=False)
    inf = sch.info()
    # the schedule is left in the winning launch shape of each direction
    for r, pre in ((res, ""), (resa, "adj_")):
        assert r["ms"] > 0
        if r["exec"] == "blocks":
            assert inf[pre + "exec_mode"] == 2 and inf[pre + "block_lanes"] == r["block_lanes"]
            assert inf[pre + "block_rows"] == r["block_rows"]
        elif r["exec"] in ("ws", "tma"):
            assert inf[pre + "exec_mode"] == (3 if r["exec"] == "ws" else 4)
            assert inf[pre + "block_rows"] == r["block_rows"]
        elif r["exec"] == "cta":
            assert pre == "" and inf["exec_mode"] == 5 and inf["n_blocks"] == 1
        else:
            assert inf[pre + "exec_mode"] == 1 and r["lanes"] in autotune.DEFAULT_LANES
            assert inf[pre + "lanes_per_row"] == r["lanes"]
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    gb = sch.adjoint(Lv, Mv, gy, saved=xs)
    sch.check()
    sch.validate()
    assert col_rel_err(host(y), y_ref) < 1e-12
    assert col_rel_err(host(gb), gb_ref) < 1e-12
    # the re-cut schedule equals the oracle's cut for the same target, wide threshold and
    # placement of the second kernel's rows
    got = sch.export(0)
    ref = oracle.schedule(oracle.SEP, oracle.COST_SEP, w.L, w.M, inf["part_cost_target"], wide=inf["wide_cost"],
                          g2=inf["g2_placement"])
    assert np.array_equal(got["part_ptr"], ref["part_ptr"])
    assert p0 > 0


@pytest.mark.parametrize("team,lpr", [(8, 1), (8, 4), (8, 8), (32, 1), (32, 8)])
def test_team_widths(team, lpr):
    need_cuda()
    w = _lap3d(12, 1)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    gb_ref, gL_ref, gM_ref = oracle.adj_trsv_spmv(w.L, w.M, x_ref, w.gy)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, lanes_per_row=lpr,
                     team_lanes=team)
    inf = sch.info()
    assert inf["team_lanes"] == team and inf["adj_team_lanes"] == team
    Lv, Mv, b = t(w.L.vals), t(w.M.vals), t(w.b)
    xs = torch.empty_like(b)
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    gL, gM = torch.empty_like(Lv), torch.empty_like(Mv)
    gb = sch.adjoint(Lv, Mv, t(w.gy), saved=xs, gL=gL, gM=gM)
    sch.check()
    assert col_rel_err(host(y), y_ref) < 1e-12
    assert col_rel_err(host(gb), gb_ref) < 1e-12
    assert vec_rel_err(host(gL), gL_ref) < 1e-12 and vec_rel_err(host(gM), gM_ref) < 1e-12


@pytest.mark.parametrize("pct", [0, 10, 50, 90, 99])
def test_partition_class_split_is_exact(pct):
    # separated schedules with the teams split between the partitions that open with a
    # first-kernel row and the others: forward SpTRSV -> SpMV and the SpMV -> SpTRSV adjoint
    need_cuda()
    w = _lap3d(12, 1)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), part_cost_target=9)
    sch.set_split(0, pct)
    inf = sch.info()
    assert inf["split_pct"] == pct and 0 < inf["parts_class0"] < inf["n_parts"]
    Lv, Mv, b = t(w.L.vals), t(w.M.vals), t(w.b)
    xs = torch.empty_like(b)
    for _ in range(2):
        y = sch.execute(Lv, Mv, b=b, x_save=xs)
        sch.check()
        assert col_rel_err(host(xs), x_ref) < 1e-12 and col_rel_err(host(y), y_ref) < 1e-12
    p = I.spmv_trsv_powerlaw(n=6000, k=1, mean=10, lmax=80, halfband=400, seed=41)
    z_ref = oracle.spmv_trsv(p.M, p.L, p.x_in, p.b)
    gb_ref, gx_ref, _, _ = oracle.adj_spmv_trsv(p.M, p.L, p.x_in, z_ref, p.gy)
    s2 = sf.inspect("spmv_trsv", dev_csr(p.L), dev_csr(p.M), want_adjoint=True, part_cost_target=12)
    s2.set_split(1, pct)
    assert s2.info()["adj_split_pct"] == pct
    Lv2, Av, xin = t(p.L.vals), t(p.M.vals), t(p.x_in)
    z = s2.execute(Lv2, Av, b=t(p.b), x_in=xin)
    gx = torch.empty_like(xin)
    gb = s2.adjoint(Lv2, Av, t(p.gy), saved=z, x_in=xin, gx=gx)
    s2.check()
    assert col_rel_err(host(gb), gb_ref) < 1e-12 and col_rel_err(host(gx), gx_ref) < 1e-12


@pytest.mark.parametrize("g2", [-1, 2, 40])
def test_g2_placement_is_exact(g2):
    # forward SpTRSV -> SpMV and the SpMV -> SpTRSV adjoint with second-kernel rows placed late
    need_cuda()
    w = _lap3d(12, 1)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), g2_placement=g2)
    Lv, Mv, b = t(w.L.vals), t(w.M.vals), t(w.b)
    xs = torch.empty_like(b)
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    sch.check()
    assert col_rel_err(host(xs), x_ref) < 1e-12 and col_rel_err(host(y), y_ref) < 1e-12
    for mode in (1, 2):
        sch.reblock(0, 2048, mode, 0)
        y = sch.execute(Lv, Mv, b=b, x_save=xs)
        sch.check()
        assert col_rel_err(host(y), y_ref) < 1e-12
    p = I.spmv_trsv_powerlaw(n=6000, k=1, mean=10, lmax=80, halfband=400, seed=41)
    z_ref = oracle.spmv_trsv(p.M, p.L, p.x_in, p.b)
    gb_ref, gx_ref, _, _ = oracle.adj_spmv_trsv(p.M, p.L, p.x_in, z_ref, p.gy)
    s2 = sf.inspect("spmv_trsv", dev_csr(p.L), dev_csr(p.M), want_adjoint=True)
    s2.replace(1, g2)
    Lv2, Av, xin = t(p.L.vals), t(p.M.vals), t(p.x_in)
    z = s2.execute(Lv2, Av, b=t(p.b), x_in=xin)
    gx = torch.empty_like(xin)
    gb = s2.adjoint(Lv2, Av, t(p.gy), saved=z, x_in=xin, gx=gx)
    s2.check()
    assert col_rel_err(host(gb), gb_ref) < 1e-12 and col_rel_err(host(gx), gx_ref) < 1e-12


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_occupancy_variants_are_exact(lanes):
    # kernels budgeted for three resident blocks per SM (lanes above 4 fall back to the
    # default kernels): forward, adjoint and the SpTRSV-alone path
    need_cuda()
    w = _lap3d(12, 1)
    x_ref, y_ref = oracle.trsv_spmv(w.L, w.M, w.b)
    gb_ref, gL_ref, gM_ref = oracle.adj_trsv_spmv(w.L, w.M, x_ref, w.gy)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True, lanes_per_row=lanes)
    sch.set_occupancy(-1, 3)
    inf = sch.info()
    assert inf["min_blocks"] == 3 and inf["adj_min_blocks"] == 3
    Lv, Mv, b, gy = t(w.L.vals), t(w.M.vals), t(w.b), t(w.gy)
    xs = torch.empty_like(b)
    y = sch.execute(Lv, Mv, b=b, x_save=xs)
    gL, gM = torch.empty_like(Lv), torch.empty_like(Mv)
    gb = sch.adjoint(Lv, Mv, gy, saved=xs, gL=gL, gM=gM)
    sch.check()
    assert col_rel_err(host(y), y_ref) < 1e-12 and col_rel_err(host(gb), gb_ref) < 1e-12
    assert vec_rel_err(host(gL), gL_ref) < 1e-12 and vec_rel_err(host(gM), gM_ref) < 1e-12
    s2 = sf.inspect("trsv", dev_csr(w.L), lanes_per_row=lanes)
    s2.set_occupancy(0, 3)
    x = s2.execute(Lv, b=b)
    s2.check()
    assert col_rel_err(host(x), x_ref) < 1e-12


def test_launch_counts():
    need_cuda()
    w = _lap3d(10, 1)
    sch = sf.inspect("trsv_spmv", dev_csr(w.L), dev_csr(w.M), want_adjoint=True)
    assert sch.launches(0, 1) == 2 and sch.launches(1, 1) == 6       # reset + executor; gathers, reset, executor, grads
    assert sch.launches(0, 4) == 1 and sch.launches(1, 4) == 5       # epoch flags for k > 1
    sch.reblock(-1, 512, 3, 0)
    assert sch.launches(0, 1) == 2 and sch.launches(1, 1) == 5       # pre-pass + executor; one gather
    sch.reblock(-1, 512, 4, 0)
    assert sch.launches(0, 1) == 3 and sch.launches(1, 1) == 6       # pre-pass + packing + executor
