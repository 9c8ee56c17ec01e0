"""Schedule strategies (one pair at a time, pair blocks, load/free list in
connection order, graph partitions) and cm_schedule_from_rows: every strategy
places every pair exactly once, keeps the resident set within the budget,
and passes the library's residency replay; malformed rows are rejected."""
import numpy as np
import pytest

import paper_2505_22089_b300 as cm
import synth
from paper_2505_22089_b300 import strategies as st


def _case():
    wl = synth.scaled("grid500", gx=8, gy=6, nmin=2000, nmax=6000)
    p = cm.Params.make()
    ib = np.array([cm.image_bytes(p, int(n)) for n in wl.n_desc], dtype=np.int64)
    return wl, p, ib


def _check(rows, wl, ib, budget):
    placed = sorted(k for r in rows for k in r["pairs"])
    assert placed == list(range(len(wl.pairs)))
    assert st.residency(rows, ib)["peak_resident_bytes"] <= budget
    s = cm.schedule_from_rows(rows, wl.pairs, wl.n_images)   # the library replays residency
    assert len(s.rows) == len(rows)
    s.close()


def test_every_strategy_is_a_valid_schedule_within_the_budget():
    wl, p, ib = _case()
    budget = int(ib.sum() // 4)
    order = st.connection_order(wl.pairs, wl.n_images, cm.gps_order)
    assert sorted(order) == list(range(wl.n_images))
    _check(st.per_pair(wl.pairs), wl, ib, budget)
    _check(st.pair_blocks(wl.pairs, ib, budget), wl, ib, budget)
    _check(st.load_free_list(wl.pairs, ib, budget, order), wl, ib, budget)
    part = int(budget // 2 // ib.max())
    _check(st.graph_partition(wl.pairs, ib, budget, order, part), wl, ib, budget)


def test_strategies_move_different_amounts_of_data():
    wl, p, ib = _case()
    budget = int(ib.sum() // 4)
    order = st.connection_order(wl.pairs, wl.n_images, cm.gps_order)
    loads = {name: st.residency(rows, ib)["loads"] for name, rows in (
        ("per_pair", st.per_pair(wl.pairs)),
        ("blocks", st.pair_blocks(wl.pairs, ib, budget)),
        ("lru", st.load_free_list(wl.pairs, ib, budget, order)),
        ("part", st.graph_partition(wl.pairs, ib, budget, order, int(budget // 2 // ib.max()))))}
    assert loads["per_pair"] == 2 * len(wl.pairs)
    assert min(loads.values()) >= wl.n_images
    assert loads["lru"] < loads["per_pair"] and loads["blocks"] < loads["per_pair"]


def test_schedule_from_rows_rejects_bad_rows():
    pairs = np.array([[0, 1], [1, 2]], dtype=np.int32)
    good = [{"load": [0, 1], "free": [0], "pairs": [0]}, {"load": [2], "free": [1, 2], "pairs": [1]}]
    cm.schedule_from_rows(good, pairs, 3).close()
    bad = [
        [{"load": [0, 1], "free": [], "pairs": [0]}, {"load": [1, 2], "free": [], "pairs": [1]}],   # reload
        [{"load": [0], "free": [], "pairs": [0]}, {"load": [1, 2], "free": [], "pairs": [1]}],      # 1 absent
        [{"load": [0, 1, 2], "free": [], "pairs": [0, 1, 1]}],                                     # repeated
        [{"load": [0, 1, 2], "free": [], "pairs": [0]}],                                           # pair 1 missing
        [{"load": [0, 1, 2], "free": [3], "pairs": [0, 1]}],                                       # free of a stranger
        [{"load": [0, 1, 5], "free": [], "pairs": [0, 1]}],                                        # id out of range
    ]
    for rows in bad:
        with pytest.raises(cm.CMError) as e:
            cm.schedule_from_rows(rows, pairs, 3)
        assert e.value.status == cm.CM_ERR_INVALID
