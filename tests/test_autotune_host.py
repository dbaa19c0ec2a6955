"""The autotuner's search logic on the CPU: a fake schedule records the launch shape the
tuner applies, and a deterministic model of its time stands in for the GPU timing. Checks
the candidate order, the slack-placement, occupancy, class-split, right-hand-side-tile and
row-slice phases, skipping of row-block sizes that do not fit, and that the schedule is left
set to the best shape."""
import pytest

from paper_2111_12238_gb300 import autotune
from paper_2111_12238_gb300 import sparsefusion as sf


class FakeSched:
    def __init__(self, pair="trsv_spmv", separated=True, n=5000, tma_fails=False, instances=1):
        self.pair, self.separated, self.n, self.tma_fails = pair, separated, n, tma_fails
        self.instances = instances
        self.state = dict(exec="partitions", C=0, lanes=0, team=0, g2=0, occ=1, split=0, B=0, blanes=0, rt=0,
                          slices=0)

    def info(self):
        nv = 2 * self.n if self.separated else self.n
        # rows costlier than 100 exist (rows are split at slice costs below that)
        units = nv + 50 if 0 < self.state["slices"] < 100 else 0
        return dict(n_items=nv, adj_n_items=0, cost_total=4 * nv, adj_cost_total=0, n=self.n,
                    parts_class0=7 if self.separated else 0, adj_parts_class0=0, depth=50, adj_depth=0,
                    instances=self.instances, slice_units=units, adj_slice_units=0)

    def replace(self, which, g2):
        self.state["g2"] = g2

    def set_occupancy(self, which, occ):
        self.state["occ"] = occ

    def reblock(self, which, B, mode, lanes):
        if mode == 4 and self.tma_fails:
            raise sf.SparseFusionError(8, "sf_schedule_reblock", "does not fit")
        if mode == 5:
            assert B == 0
            self.state.update(exec="cta", B=0, cps=lanes)
        elif mode in (2, 3, 4):
            self.state.update(exec={2: "blocks", 3: "ws", 4: "tma"}[mode], B=B, blanes=lanes)
        else:
            self.state["exec"] = "partitions"

    def recut(self, which, C, lanes, team):
        self.state.update(C=C, lanes=lanes, team=team)

    def set_split(self, which, pct):
        self.state["split"] = pct

    def set_rhs_tile(self, which, rt):
        self.state["rt"] = rt

    def set_slices(self, which, cost):
        self.state["slices"] = cost

    def set_packing(self, packing):
        self.state["packing"] = packing

    def check(self):
        pass


def _model(st):
    """Milliseconds of a launch shape: partitions are best at 4 lanes, 16 items of cost 4
    (C = 64) and 32-lane teams; the last-wavefront placement, the occupancy variant and an 80 %
    class split each help a little; the row blocks are slower."""
    if st["exec"] != "partitions":
        return 3.0 + st["B"] / 1e5 - (0.5 if st["g2"] == -1 else 0.0)
    ms = 1.0 + 0.1 * abs(st["lanes"] - 4) + abs(st["C"] - 64) / 800 - (0.05 if st["team"] == 32 else 0.0)
    ms -= 0.2 if st["g2"] == -1 else 0.0
    ms -= 0.03 if st["occ"] == 3 else 0.0
    ms -= 0.01 if st["split"] == 80 else 0.0
    ms -= 0.02 if st["slices"] == 64 else 0.0
    ms -= 2.0 if st["rt"] == 8 and st["lanes"] == 32 else 0.0
    return ms


@pytest.fixture
def fake_timing(monkeypatch):
    holder = {}
    monkeypatch.setattr(autotune, "_time", lambda run, reps: _model(holder["sched"].state))
    monkeypatch.setattr(autotune, "signature", lambda *a, **k: "fake")
    return holder


def test_tuner_finds_and_applies_the_best_shape(fake_timing):
    s = FakeSched()
    fake_timing["sched"] = s
    best = autotune.tune(s, lambda: None, k=1, budget_s=60, use_cache=False)
    assert (best["exec"], best["lanes"], best["items"], best["team"]) == ("partitions", 4, 16, 32)
    assert (best["g2"], best["occ"], best["split"], best["slices"]) == (-1, 3, 80, 64)
    assert best["ms"] == pytest.approx(min(t["ms"] for t in best["trials"]))
    # the schedule is left in the winning shape
    shape = {key: s.state[key] for key in ("exec", "C", "lanes", "team", "g2", "occ", "split", "slices")}
    assert shape == dict(exec="partitions", C=64, lanes=4, team=32, g2=-1, occ=3, split=80, slices=64)
    # slice costs at which nothing splits are not timed; no right-hand-side tiles for k = 1
    assert not any(t.get("slices", 0) >= 100 for t in best["trials"])
    assert not any("rt" in t for t in best["trials"])
    # every row-block executor was tried, and placements were tried on the best row-block shape too
    kinds = {t["exec"] for t in best["trials"]}
    assert kinds == {"partitions", "ws", "tma", "blocks", "cta"}
    assert any(t["exec"] != "partitions" and t.get("g2") == -1 for t in best["trials"])


def test_candidate_order_starts_at_the_tile_width_and_stops_at_the_budget(fake_timing):
    s = FakeSched()
    fake_timing["sched"] = s
    r = autotune.tune(s, lambda: None, k=1, budget_s=0, placements=(), splits=(), occupancy=False, slices=(),
                      use_cache=False)
    # one candidate within a zero budget: one lane per row, whole-warp teams, eight items
    assert len(r["trials"]) == 1
    assert (r["lanes"], r["team"], r["items"]) == (1, 32, 8)


def test_wide_right_hand_sides_use_whole_warps_and_skip_row_blocks(fake_timing):
    s = FakeSched(pair="ic0_trsv", separated=False)
    fake_timing["sched"] = s
    r = autotune.tune(s, lambda: None, k=32, budget_s=60, use_cache=False)
    assert {t["exec"] for t in r["trials"]} == {"partitions"}
    assert all(t["lanes"] == 32 for t in r["trials"])
    assert not any("g2" in t or "split" in t for t in r["trials"])      # paired: no slack, no classes
    assert any(t.get("occ") == 3 for t in r["trials"])                   # IC0 occupancy variant tried


def test_rhs_tile_phase_for_several_right_hand_sides(fake_timing):
    # k = 16: the default tile is 16; the tuner also tries the other tiles with lanes at least
    # the tile, and keeps the (32 lanes, tile 8) shape the model favours
    s = FakeSched(pair="spmv_trsv", separated=False)
    fake_timing["sched"] = s
    r = autotune.tune(s, lambda: None, k=16, budget_s=60, use_cache=False)
    tiles = {t.get("rt") for t in r["trials"] if "rt" in t}
    assert {1, 2, 4, 8, 32} <= tiles
    assert all(t["lanes"] >= t["rt"] for t in r["trials"] if "rt" in t)
    assert (r["rt"], r["lanes"]) == (8, 32) and s.state["rt"] == 8 and s.state["lanes"] == 32


def test_row_block_sizes_that_do_not_fit_are_skipped(fake_timing):
    s = FakeSched(tma_fails=True)
    fake_timing["sched"] = s
    r = autotune.tune(s, lambda: None, k=1, budget_s=60, use_cache=False)
    assert "tma" not in {t["exec"] for t in r["trials"]}
    assert r["exec"] == "partitions"


def test_batches_try_the_single_cta_executor_at_each_sm_share(fake_timing):
    # a batch of large instances: one CTA per instance at 2, 1 and 4 CTAs per SM, right after
    # the first partition shape; a single large system does not try it
    s = FakeSched(n=2_000_000, instances=512)
    fake_timing["sched"] = s
    r = autotune.tune(s, lambda: None, k=1, budget_s=60, use_cache=False)
    cta = [t for t in r["trials"] if t["exec"] == "cta"]
    assert [t["cps"] for t in cta[:3]] == [2, 1, 4]
    assert r["trials"][0]["exec"] == "partitions" and r["trials"][1]["exec"] == "cta"
    s1 = FakeSched(n=2_000_000)
    fake_timing["sched"] = s1
    r1 = autotune.tune(s1, lambda: None, k=1, budget_s=60, use_cache=False)
    assert not any(t["exec"] == "cta" for t in r1["trials"])


def test_spmv_trsv_tries_separated_packing(fake_timing):
    # SpMV -> SpTRSV forward: the best partition shape is also timed with separated packing,
    # and every other candidate runs interleaved
    s = FakeSched(pair="spmv_trsv", separated=False)
    fake_timing["sched"] = s
    r = autotune.tune(s, lambda: None, k=1, budget_s=60, use_cache=False)
    sep = [t for t in r["trials"] if t.get("packing") == 0]
    assert len(sep) == 1 and sep[0]["exec"] == "partitions"
    assert s.state["packing"] == r.get("packing", 1)
