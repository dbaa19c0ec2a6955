"""GPU inspector parity: wavefront levels, the (level, kernel, row) order and the
partition cut must equal the oracle's bit for bit, and every schedule must validate."""
import numpy as np
import pytest

import oracle
from paper_2111_12238_gb300 import inputs as I
from paper_2111_12238_gb300 import sparsefusion as sf
from tests._gpu import dev_csr, need_cuda

pytestmark = pytest.mark.gpu

KIND_OF = {"trsv_spmv": (oracle.SEP, oracle.COST_SEP), "spmv_trsv": (oracle.PAIRED, oracle.COST_SPMV_TRSV),
           "ic0_trsv": (oracle.PAIRED, oracle.COST_IC0_TRSV), "trsv": (oracle.PAIRED, oracle.COST_TRSV),
           "ic0": (oracle.PAIRED, oracle.COST_IC0)}
ADJ_OF = {"trsv_spmv": (oracle.PAIRED_T, oracle.COST_PAIRED_T), "spmv_trsv": (oracle.SEP_T, oracle.COST_SEP_T)}


def _workloads():
    return {
        "lap2d64": lambda: I.trsv_spmv_lap2d(64, seed=1),
        "lap3d16": lambda: I.trsv_spmv_lap3d_band(16, seed=2),
        "lap3d13_ragged": lambda: I.trsv_spmv_lap3d_band(13, per_row=5, halfband=300, seed=7),
        "aniso12": lambda: I.ic0_trsv_aniso3d(12, k=1),
        "powerlaw": lambda: I.spmv_trsv_powerlaw(n=30000, k=1, mean=16, lmax=300, halfband=700, seed=5),
        "plower": lambda: I.Workload("plower", "trsv", 5000, 1, I.powerlaw_lower(5000, 8, 256, 4), None,
                                     np.zeros((5000, 1))),
    }


CASES = [("lap2d64", "trsv_spmv"), ("lap3d16", "trsv_spmv"), ("lap3d13_ragged", "trsv_spmv"),
         ("aniso12", "ic0_trsv"), ("aniso12", "ic0"), ("aniso12", "trsv"), ("powerlaw", "spmv_trsv"),
         ("plower", "trsv"), ("lap3d16", "spmv_trsv")]


@pytest.mark.parametrize("wname,pair", CASES)
@pytest.mark.parametrize("target", [0, 1, 57, 10 ** 12])
def test_schedule_matches_oracle(wname, pair, target):
    need_cuda()
    w = _workloads()[wname]()
    L = w.L
    M = w.M if pair in ("trsv_spmv", "spmv_trsv") else None
    want_adj = pair in ADJ_OF
    sch = sf.inspect(pair, dev_csr(L), dev_csr(M) if M is not None else None, want_adjoint=want_adj,
                     part_cost_target=target)
    sch.validate()
    info = sch.info()
    for which, (kind, what) in enumerate([KIND_OF[pair]] + ([ADJ_OF[pair]] if want_adj else [])):
        C = info["part_cost_target"] if which == 0 else info["adj_part_cost_target"]
        W = info["wide_cost"] if which == 0 else info["adj_wide_cost"]
        if target:
            assert C == target
        ref = oracle.schedule(kind, what, L, M, C, wide=W)
        got = sch.export(which)
        assert np.array_equal(got["level"], ref["level"]), f"levels differ ({wname}, {pair}, dir {which})"
        assert got["depth"] == ref["depth"]
        assert np.array_equal(got["order"], ref["order"])
        assert np.array_equal(got["part_ptr"], ref["part_ptr"])
        assert oracle.validate(kind, L, M if kind in (oracle.SEP, oracle.SEP_T) else None,
                               got["order"], got["part_ptr"]) == 0
        # partition classes of separated schedules: partitions that open with a first-kernel row
        first = ref["order"].view(np.uint32)[ref["part_ptr"][:-1]] >> 31
        n0 = int((first == 0).sum()) if kind in (oracle.SEP, oracle.SEP_T) else 0
        assert info["parts_class0" if which == 0 else "adj_parts_class0"] == n0


def test_grid_levels_closed_form_on_gpu():
    need_cuda()
    d = (20, 11, 7)
    L = I.grid_lower_laplacian(d, 3)
    sch = sf.inspect("trsv", dev_csr(L))
    got = sch.export(0)
    z, y, x = np.indices(d[::-1]).reshape(3, -1)
    assert np.array_equal(got["level"], x + y + z)
    assert got["depth"] == sum(d) - 2


def test_batched_schedule_is_blockdiagonal_union():
    need_cuda()
    w = I.batched_trsv_spmv(count=6, nmin=64, nmax=3000, seed=9)
    Ls = [dev_csr(x.L) for x in w.instances]
    Ms = [dev_csr(x.M) for x in w.instances]
    sch = sf.inspect_batched("trsv_spmv", Ls, Ms, want_adjoint=True, part_cost_target=100)
    sch.validate()
    # levels: each instance's own levels, concatenated per kernel
    got = sch.export(0)
    n = w.n
    lev1, lev2 = [], []
    for x in w.instances:
        lv = oracle.levels(oracle.SEP, x.L, x.M)
        lev1.append(lv[: x.n])
        lev2.append(lv[x.n:])
    assert np.array_equal(got["level"], np.concatenate(lev1 + lev2))
    # order is (level, kernel, global row) with rows offset per instance
    o = got["order"].view(np.uint32).astype(np.int64)
    key = np.stack([got["level"][(o >> 31) * n + (o & 0x7FFFFFFF)], o >> 31, o & 0x7FFFFFFF])
    assert np.all(np.diff(key[0]) >= 0)
    same = np.diff(key[0]) == 0
    k2 = key[1] * n + key[2]
    assert np.all(np.diff(k2)[same] > 0)
    assert sch.info()["instances"] == 6


def test_invalid_patterns_rejected():
    need_cuda()
    from tests._mats import dense_to_csr
    D = np.tril(np.ones((5, 5)))
    P = D != 0
    P[3, 3] = False                               # missing diagonal
    bad = dense_to_csr(D, P)
    with pytest.raises(sf.SparseFusionError) as e:
        sf.inspect("trsv", dev_csr(bad))
    assert e.value.status == 2 and "diagonal" in e.value.detail
    U = dense_to_csr(np.triu(np.ones((4, 4))))    # upper entries in L
    with pytest.raises(sf.SparseFusionError) as e:
        sf.inspect("trsv", dev_csr(U))
    assert e.value.status == 2
    L = dense_to_csr(np.tril(np.ones((4, 4))))
    with pytest.raises(sf.SparseFusionError) as e:
        sf.inspect("trsv_spmv", dev_csr(L), None)
    assert e.value.status == 1
    with pytest.raises(sf.SparseFusionError) as e:
        sf.inspect("ic0_trsv", dev_csr(L), want_adjoint=True)
    assert e.value.status == 8


@pytest.mark.parametrize("g2", [-1, 1, 6])
def test_g2_placement_matches_oracle(g2):
    # second-kernel vertices placed by slack, at inspection and by re-placement afterwards
    need_cuda()
    w = _workloads()["lap3d13_ragged"]()
    p = _workloads()["powerlaw"]()
    for pair, ww, kinds in (("trsv_spmv", w, [KIND_OF["trsv_spmv"]]),
                            ("spmv_trsv", p, [KIND_OF["spmv_trsv"], ADJ_OF["spmv_trsv"]])):
        for via_replace in (False, True):
            sch = sf.inspect(pair, dev_csr(ww.L), dev_csr(ww.M), want_adjoint=pair == "spmv_trsv",
                             part_cost_target=57, g2_placement=0 if via_replace else g2)
            if via_replace:
                sch.replace(-1, g2)
            sch.validate()
            info = sch.info()
            for which, (kind, what) in enumerate(kinds):
                sep = kind in (oracle.SEP, oracle.SEP_T)
                ref = oracle.schedule(kind, what, ww.L, ww.M, 57, wide=info["wide_cost" if which == 0 else "adj_wide_cost"],
                                      g2=g2 if sep else 0)
                got = sch.export(which)
                assert np.array_equal(got["level"], ref["level"])
                assert np.array_equal(got["order"], ref["order"])
                assert np.array_equal(got["part_ptr"], ref["part_ptr"])
                assert info["g2_placement" if which == 0 else "adj_g2_placement"] == (g2 if sep else 0)


def _hub_lower(n, hubs, seed):
    """Lower-triangular pattern whose first `hubs` rows are sources and every later row reads
    all of them (plus its predecessor row): the hubs' successor lists hold n - hubs entries, the
    later rows' own lists hubs + 1, long lists in both the forward and the reversed DAG."""
    rows = []
    for i in range(n):
        if i < hubs:
            cols = [i]
        else:
            cols = list(range(hubs)) + ([i - 1] if i - 1 >= hubs else []) + [i]
        rows.append(cols)
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    ci = np.concatenate([np.asarray(r, np.int32) for r in rows])
    vals = I.uniform_pm1(seed, I.S_VALUES, np.arange(len(ci), dtype=np.int64)) + (ci == np.repeat(np.arange(n), np.diff(rp))) * 4
    return I.Csr(n, n, rp, ci, vals)


@pytest.mark.parametrize("hubs", [3, 300, 700])
def test_levels_with_long_successor_lists(hubs):
    # successor lists far beyond what one warp expands in a batch: the hubs in the forward DAG,
    # the later rows in the reversed one, hundreds of them in one round
    need_cuda()
    n = 6000
    L = _hub_lower(n, hubs, 91)
    M = I.band_random(n, 6, 400, 92)
    sch = sf.inspect("trsv_spmv", dev_csr(L), dev_csr(M), want_adjoint=True)
    info = sch.info()
    for which, (kind, what) in enumerate([KIND_OF["trsv_spmv"], ADJ_OF["trsv_spmv"]]):
        C = info["part_cost_target"] if which == 0 else info["adj_part_cost_target"]
        W = info["wide_cost"] if which == 0 else info["adj_wide_cost"]
        ref = oracle.schedule(kind, what, L, M, C, wide=W)
        got = sch.export(which)
        assert np.array_equal(got["level"], ref["level"])
        assert got["depth"] == ref["depth"]
        assert np.array_equal(got["order"], ref["order"])
