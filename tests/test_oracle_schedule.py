"""Pins of the oracle's schedule objects: closed-form wavefront numbers on grids and
simple chains, order and partition invariants, validator verdicts on planted mistakes, and
the reuse ratios of Table 2 (golden fixture). CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2111_12238_gb300 import inputs as I
from tests._mats import dense_to_csr, random_lower, random_square

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_levels_grid2d_closed_form():
    nx, ny = 7, 5
    L = I.grid_lower_laplacian((nx, ny), 1)
    M = I.grid_full_stencil_random((nx, ny), 1)
    lev = oracle.levels(oracle.SEP, L, M)
    x, y = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    x, y = x.ravel(), y.ravel()
    assert np.array_equal(lev[: nx * ny], x + y)
    # SpMV row (x,y) reads x at its forward neighbours (x+1,y), (x,y+1) when they exist
    fwd = (x < nx - 1) | (y < ny - 1)
    assert np.array_equal(lev[nx * ny:], np.where(fwd, x + y + 2, x + y + 1))
    levT = oracle.levels(oracle.PAIRED_T, L)
    assert np.array_equal(levT, (nx - 1 - x) + (ny - 1 - y))


def test_levels_grid3d_closed_form():
    d = (6, 4, 3)
    L = I.grid_lower_laplacian(d, 2)
    lev = oracle.levels(oracle.PAIRED, L)
    z, y, x = np.indices(d[::-1]).reshape(3, -1)
    assert np.array_equal(lev, x + y + z)
    _, depth = oracle.order(lev, L.n_rows)
    assert depth == sum(d) - 3 + 1


def test_levels_chain_and_diagonal():
    n = 9
    bid = np.eye(n) * 2 + np.eye(n, k=-1)
    assert np.array_equal(oracle.levels(oracle.PAIRED, dense_to_csr(bid)), np.arange(n))
    assert np.array_equal(oracle.levels(oracle.PAIRED_T, dense_to_csr(bid)), n - 1 - np.arange(n))
    dg = dense_to_csr(np.eye(n) * 3)
    assert np.array_equal(oracle.levels(oracle.PAIRED, dg), np.zeros(n))
    # SEP_T: A^T row j waits for every lambda_i with A_ij != 0; empty column -> level 0
    A = np.zeros((n, n))
    A[2, 5] = 1.0
    A[7, 5] = 1.0
    lev = oracle.levels(oracle.SEP_T, dense_to_csr(bid), dense_to_csr(A))
    lam = n - 1 - np.arange(n)
    want = np.zeros(n, dtype=np.int32)
    want[5] = max(lam[2], lam[7]) + 1
    assert np.array_equal(lev[n:], want)


def _brute_levels(edges, nv):
    """Longest path from sources by repeated relaxation (Bellman-Ford style), tiny inputs."""
    lev = np.zeros(nv, dtype=np.int64)
    for _ in range(nv + 1):
        changed = False
        for u, v in edges:
            if lev[u] + 1 > lev[v]:
                lev[v] = lev[u] + 1
                changed = True
        if not changed:
            break
    return lev


@pytest.mark.parametrize("kind", [oracle.SEP, oracle.PAIRED, oracle.PAIRED_T, oracle.SEP_T])
def test_levels_match_brute_force_relaxation(kind):
    n = 30
    DL = random_lower(n, 0.15, 61)
    DM = random_square(n, 0.1, 62)
    L, M = dense_to_csr(DL), dense_to_csr(DM)
    edges = []
    for i in range(n):
        for j in range(i):
            if DL[i, j] != 0:
                edges.append((j, i) if kind in (oracle.SEP, oracle.PAIRED) else (i, j))
    if kind == oracle.SEP:
        edges += [(j, n + i) for i in range(n) for j in range(n) if DM[i, j] != 0]
    if kind == oracle.SEP_T:
        edges += [(i, n + j) for i in range(n) for j in range(n) if DM[i, j] != 0]
    nv = oracle.n_vertices(kind, n)
    assert np.array_equal(oracle.levels(kind, L, M if kind in (oracle.SEP, oracle.SEP_T) else None),
                          _brute_levels(edges, nv))


def test_order_sorted_by_level_tag_row_and_valid():
    w = I.trsv_spmv_lap2d(12, seed=3)
    lev = oracle.levels(oracle.SEP, w.L, w.M)
    o, depth = oracle.order(lev, w.n)
    tag = (o.view(np.uint32) >> 31).astype(np.int64)
    row = (o.view(np.uint32) & 0x7FFFFFFF).astype(np.int64)
    v = tag * w.n + row
    assert np.array_equal(np.sort(v), np.arange(2 * w.n))
    ref = np.lexsort((row, tag, lev[v]))
    assert np.array_equal(ref, np.arange(2 * w.n))   # already in (level, tag, row) order
    assert depth == lev.max() + 1
    pp = oracle.partition(o, w.n, oracle.costs(oracle.COST_SEP, w.L, w.M), 40)
    assert oracle.validate(oracle.SEP, w.L, w.M, o, pp) == 0


@pytest.mark.parametrize("target", [1, 7, 64, 10 ** 9])
def test_partition_cut_invariants(target):
    w = I.trsv_spmv_lap2d(9, seed=4)
    s = oracle.schedule(oracle.SEP, oracle.COST_SEP, w.L, w.M, target)
    o, pp, c = s["order"], s["part_ptr"], s["cost"]
    v = (o.view(np.uint32) >> 31).astype(np.int64) * w.n + (o.view(np.uint32) & 0x7FFFFFFF)
    S = np.concatenate([[0], np.cumsum(c[v])])[:-1]
    q = S // target
    assert pp[0] == 0 and pp[-1] == len(o) and np.all(np.diff(pp) > 0)
    for p in range(len(pp) - 1):
        seg = q[pp[p]:pp[p + 1]]
        assert np.all(seg == seg[0])                 # one quotient per partition
        if p + 1 < len(pp) - 1:
            assert q[pp[p + 1]] > seg[0]             # maximal runs
    if target == 1:
        assert len(pp) - 1 == len(o)
    if target == 10 ** 9:
        assert len(pp) - 1 == 1


def test_costs_hand_computed():
    # L = [[1,0,0],[1,1,0],[1,1,1]], M = [[1,0,1],[0,1,0],[0,0,1]]
    L = dense_to_csr(np.tril(np.ones((3, 3))))
    M = dense_to_csr(np.array([[1.0, 0, 1], [0, 1, 0], [0, 0, 1]]))
    assert oracle.costs(oracle.COST_SEP, L, M).tolist() == [2, 3, 4, 3, 2, 2]
    assert oracle.costs(oracle.COST_TRSV, L).tolist() == [2, 3, 4]
    # IC0 row i touches its row and each earlier row j of the pattern: 1+0, 2+1, 3+(1+2)
    assert oracle.costs(oracle.COST_IC0, L).tolist() == [2, 4, 7]
    assert oracle.costs(oracle.COST_IC0_TRSV, L).tolist() == [3, 6, 10]
    assert oracle.costs(oracle.COST_SPMV_TRSV, L, M).tolist() == [4, 4, 5]
    # column counts: L^T rows 3,2,1; M^T rows 1,1,2
    assert oracle.costs(oracle.COST_PAIRED_T, L, M).tolist() == [1 + 3 + 1, 1 + 2 + 1, 2 + 1 + 1]
    assert oracle.costs(oracle.COST_SEP_T, L, M).tolist() == [3 + 1, 2 + 1, 1 + 1, 2, 2, 3]
    # SpTRSV -> SpTRSV reads the row of L twice
    assert oracle.costs(oracle.COST_TRSV_TRSV, L).tolist() == [3, 5, 7]
    # SpILU0 -> SpTRSV on A = [[1,0,1],[1,1,0],[1,1,1]], L = tril(A): row i of A, the rows of A
    # it eliminates with (none; row 0; rows 0 and 1), the solve row: 2+0+1+1, 2+2+2+1, 3+4+3+1
    Ad = np.array([[1.0, 0, 1], [1, 1, 0], [1, 1, 1]])
    assert oracle.costs(oracle.COST_ILU0_TRSV, dense_to_csr(np.tril(Ad)), dense_to_csr(Ad)).tolist() == [4, 7, 11]


def test_partition_isolates_wide_items():
    # items costing more than the wide threshold form partitions of their own
    w = I.spmv_trsv_powerlaw(n=3000, k=1, mean=8, lmax=200, halfband=400, seed=6)
    s = oracle.schedule(oracle.PAIRED, oracle.COST_SPMV_TRSV, w.L, w.M, 60, wide=40)
    o, pp, c = s["order"], s["part_ptr"], s["cost"]
    v = (o.view(np.uint32) & 0x7FFFFFFF).astype(np.int64)
    wide = c[v] > 40
    assert wide.any() and not wide.all()
    for p in range(len(pp) - 1):
        seg = wide[pp[p]:pp[p + 1]]
        if seg.any():
            assert len(seg) == 1
    plain = oracle.schedule(oracle.PAIRED, oracle.COST_SPMV_TRSV, w.L, w.M, 60)
    assert len(plain["part_ptr"]) < len(pp)
    assert oracle.validate(oracle.PAIRED, w.L, None, o, pp) == 0


def test_validator_catches_planted_mistakes():
    w = I.trsv_spmv_lap2d(8, seed=5)
    s = oracle.schedule(oracle.SEP, oracle.COST_SEP, w.L, w.M, 30)
    o, pp = s["order"].copy(), s["part_ptr"]
    assert oracle.validate(oracle.SEP, w.L, w.M, o, pp) == 0
    bad = o.copy()
    bad[[0, -1]] = bad[[-1, 0]]                       # a sink before a source
    assert oracle.validate(oracle.SEP, w.L, w.M, bad, pp) == 2
    dup = o.copy()
    dup[3] = dup[4]
    assert oracle.validate(oracle.SEP, w.L, w.M, dup, pp) == 1
    badp = pp.copy()
    badp[1] = badp[2]
    assert oracle.validate(oracle.SEP, w.L, w.M, o, badp) == 3
    # the transposed schedule must be reversed: the forward order is invalid for PAIRED_T
    sT = oracle.schedule(oracle.PAIRED_T, oracle.COST_PAIRED_T, w.L, w.M, 30)
    assert oracle.validate(oracle.PAIRED_T, w.L, None, sT["order"], sT["part_ptr"]) == 0
    sF = oracle.schedule(oracle.PAIRED, oracle.COST_TRSV, w.L, None, 30)
    assert oracle.validate(oracle.PAIRED_T, w.L, None, sF["order"], sF["part_ptr"]) == 2


def test_reuse_ratio_table2_golden():
    with open(os.path.join(GOLDEN, "reuse_ratio_table2.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        num, den = case["expected"].split("/")
        got = oracle.reuse_ratio(case["pair"], case["n"], case["size_L"], case["size_M"])
        assert got == pytest.approx(float(num) / float(den), rel=1e-15)
        assert (got >= 1.0) == case["interleaved"]


@pytest.mark.parametrize("kind", [oracle.SEP, oracle.PAIRED, oracle.PAIRED_T, oracle.SEP_T])
@pytest.mark.parametrize("B", [1, 7, 64, 10 ** 6])
def test_block_order_is_a_valid_blocked_linearisation(kind, B):
    w = I.spmv_trsv_powerlaw(n=500, k=1, mean=6, lmax=30, halfband=60, seed=8)
    L, M = w.L, w.M
    useM = M if kind in (oracle.SEP, oracle.SEP_T) else None
    lev = oracle.levels(kind, L, useM)
    o, bp = oracle.block_order(kind, L, useM, lev, B)
    n = L.n_rows
    nb = -(-n // B)
    assert len(bp) == nb + 1 and bp[0] == 0 and bp[-1] == len(o)
    # every DAG and F edge points forward (blocks are contiguous, levels sorted inside)
    assert oracle.validate(kind, L, useM, o, bp) == 0
    # first-kernel rows sit in their own row block (reversed for the transposed kinds)
    rev = kind in (oracle.PAIRED_T, oracle.SEP_T)
    ov = o.view(np.uint32)
    for b in range(nb):
        seg = ov[bp[b]:bp[b + 1]]
        rows = (seg & 0x7FFFFFFF)[(seg >> 31) == 0].astype(np.int64)
        want = (nb - 1 - b) if rev else b
        assert np.all(rows // B == want)
        v = (seg >> 31).astype(np.int64) * n + (seg & 0x7FFFFFFF)
        key = lev[v].astype(np.int64) * (2 * n) + v
        assert np.all(np.diff(key) > 0)           # (level, tag, row) inside a block
    if B >= n:
        ref, _ = oracle.order(lev, n)
        assert np.array_equal(o, ref)             # one block: the plain level order


@pytest.mark.parametrize("kind", [oracle.SEP, oracle.PAIRED, oracle.PAIRED_T, oracle.SEP_T])
@pytest.mark.parametrize("B", [1, 7, 64, 10 ** 6])
def test_block_segments_are_independent_level_runs(kind, B):
    w = I.spmv_trsv_powerlaw(n=400, k=1, mean=6, lmax=30, halfband=50, seed=9)
    L, M = w.L, w.M
    useM = M if kind in (oracle.SEP, oracle.SEP_T) else None
    lev = oracle.levels(kind, L, useM)
    o, bp = oracle.block_order(kind, L, useM, lev, B)
    n = L.n_rows
    sp, bs = oracle.block_segments(kind, n, o, bp, lev)
    ov = o.view(np.uint32)
    v = (ov >> 31).astype(np.int64) * n + (ov & 0x7FFFFFFF)
    nb = len(bp) - 1
    # brute force: the distinct levels of every block, in increasing order, one segment each
    want_ptr = []
    want_bs = []
    for b in range(nb):
        want_bs.append(len(want_ptr))
        seen = None
        for q in range(bp[b], bp[b + 1]):
            if seen is None or lev[v[q]] != seen:
                want_ptr.append(q)
                seen = lev[v[q]]
    want_bs.append(len(want_ptr))
    want_ptr.append(len(o))
    assert sp.tolist() == want_ptr and bs.tolist() == want_bs
    assert len(sp) - 1 == sum(len(set(lev[v[bp[b]:bp[b + 1]]].tolist())) for b in range(nb))
    # no vertex of a segment reads another vertex of the same segment: the DAG edges j -> i
    # (strict lower L, or its transpose) and the F edges never join two positions of a run
    seg_of = np.zeros(len(o), dtype=np.int64)
    for s in range(len(sp) - 1):
        seg_of[sp[s]:sp[s + 1]] = s
    pos = np.empty(len(o), dtype=np.int64)
    pos[v] = np.arange(len(o))
    Lrp, Lci = L.rowptr, L.colidx
    for i in range(n):
        for e in range(Lrp[i], Lrp[i + 1] - 1):
            j = int(Lci[e])
            a, b_ = (j, i) if kind in (oracle.SEP, oracle.PAIRED) else (i, j)
            assert seg_of[pos[a]] < seg_of[pos[b_]]
    if kind == oracle.SEP:
        for i in range(n):
            for e in range(M.rowptr[i], M.rowptr[i + 1]):
                assert seg_of[pos[int(M.colidx[e])]] < seg_of[pos[n + i]]
    if kind == oracle.SEP_T:
        for i in range(n):
            for e in range(M.rowptr[i], M.rowptr[i + 1]):
                assert seg_of[pos[i]] < seg_of[pos[n + int(M.colidx[e])]]


@pytest.mark.parametrize("kind", [oracle.SEP, oracle.SEP_T])
def test_g2_placement_keeps_every_edge_forward(kind):
    # second-kernel vertices are sinks: placing them anywhere from their earliest wavefront to
    # the last keeps the schedule valid (checked edge by edge by the validator), leaves the
    # first kernel's levels and the depth alone, and moves later as the delay grows
    w = I.spmv_trsv_powerlaw(n=700, k=1, mean=6, lmax=40, halfband=80, seed=23)
    L, M = w.L, w.M
    n = L.n_rows
    what = oracle.COST_SEP if kind == oracle.SEP else oracle.COST_SEP_T
    asap = oracle.levels(kind, L, M)
    depth = int(asap.max()) + 1
    prev = asap
    for g2 in (1, 3, 17, 10 ** 6):
        lev = oracle.levels(kind, L, M, g2)
        assert np.array_equal(lev[:n], asap[:n])
        assert np.all(lev[n:] >= prev[n:]) and np.all(lev[n:] <= depth - 1) and int(lev.max()) + 1 == depth
        sch = oracle.schedule(kind, what, L, M, 30, g2=g2)
        assert np.array_equal(sch["level"], lev)
        assert oracle.validate(kind, L, M, sch["order"], sch["part_ptr"]) == 0
        prev = lev
    alap = oracle.levels(kind, L, M, -1)
    assert np.all(alap[n:] == depth - 1) and np.array_equal(alap[:n], asap[:n])
    assert np.array_equal(oracle.levels(kind, L, M, 10 ** 6), alap)
    sch = oracle.schedule(kind, what, L, M, 30, g2=-1)
    assert oracle.validate(kind, L, M, sch["order"], sch["part_ptr"]) == 0
    # paired kinds ignore the placement
    assert np.array_equal(oracle.levels(oracle.PAIRED, L, None, -1), oracle.levels(oracle.PAIRED, L, None))


def _blockdiag(mats):
    """Block-diagonal CSR of the given square CSRs (columns shifted by the row offsets)."""
    n = sum(m.n_rows for m in mats)
    rp, ci, vals, off, eoff = [np.zeros(1, np.int32)], [], [], 0, 0
    for m in mats:
        rp.append((np.asarray(m.rowptr[1:]) + eoff).astype(np.int32))
        ci.append((np.asarray(m.colidx) + off).astype(np.int32))
        vals.append(np.asarray(m.vals))
        off += m.n_rows
        eoff += int(m.rowptr[-1])
    return I.Csr(n, n, np.concatenate(rp), np.concatenate(ci), np.concatenate(vals))


@pytest.mark.parametrize("kind", [oracle.SEP, oracle.PAIRED, oracle.PAIRED_T, oracle.SEP_T])
def test_block_order_instances_is_the_instance_level_sort(kind):
    # one block per instance of a block-diagonal system: the (instance, level, tag, row) sort,
    # written out here with numpy, a valid linearisation, and block pointers at the instances'
    # vertex counts
    sizes = [37, 1, 120, 64, 9]
    Ls = [I.powerlaw_lower(m, 4, 20, 70 + t) for t, m in enumerate(sizes)]
    Ms = [I.band_random(m, min(3, m), 10, 80 + t) for t, m in enumerate(sizes)]
    L, M = _blockdiag(Ls), _blockdiag(Ms)
    n = L.n_rows
    useM = M if kind in (oracle.SEP, oracle.SEP_T) else None
    lev = oracle.levels(kind, L, useM)
    inst_ptr = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    o, bp = oracle.block_order_instances(kind, n, lev, inst_ptr)
    nv = len(lev)
    v = np.arange(nv)
    inst = np.searchsorted(inst_ptr, v % n, side="right") - 1
    perm = np.lexsort((v, lev, inst))
    ref = np.where(perm < n, perm, (perm - n) | (1 << 31)).astype(np.int64).astype(np.uint32).view(np.int32)
    assert np.array_equal(o, ref)
    per = np.array(sizes) * (2 if nv == 2 * n else 1)
    assert np.array_equal(bp, np.concatenate([[0], np.cumsum(per)]))
    assert oracle.validate(kind, L, useM, o, bp) == 0


@pytest.mark.parametrize("kind", [oracle.SEP, oracle.PAIRED, oracle.PAIRED_T, oracle.SEP_T])
def test_block_order_instances_single_instance_is_the_one_block_order(kind):
    w = I.spmv_trsv_powerlaw(n=300, k=1, mean=6, lmax=30, halfband=40, seed=12)
    useM = w.M if kind in (oracle.SEP, oracle.SEP_T) else None
    lev = oracle.levels(kind, w.L, useM)
    o, bp = oracle.block_order_instances(kind, w.n, lev, np.array([0, w.n], np.int32))
    ref_o, ref_bp = oracle.block_order(kind, w.L, useM, lev, 10 ** 6)
    assert np.array_equal(o, ref_o) and np.array_equal(bp, ref_bp)


def test_block_order_instances_rejects_bad_boundaries():
    lev = np.zeros(10, np.int32)
    for bad in ([0, 4], [1, 10], [0, 7, 5, 10]):
        with pytest.raises(oracle.OracleError):
            oracle.block_order_instances(oracle.PAIRED, 10, lev, np.array(bad, np.int32))
