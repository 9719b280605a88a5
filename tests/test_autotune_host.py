"""Host logic of the batch autotuner's persisted table (no GPU)."""
import json
import os

import pytest

from paper_2009_06657_gb300.autotune import DEFAULT_TABLE, TABLE_ENV, BatchTable, table_path


def _table():
    t = BatchTable(device="test")
    t.add(8, 8, 1, {"1": 0.5, "2": 0.7})
    t.add(12, 8, 4)
    t.add(16, 8, 16)
    t.add(12, 64, 8)
    return t


def test_exact_lookup():
    t = _table()
    assert t.lookup(8, 8) == 1 and t.lookup(12, 8) == 4 and t.lookup(16, 8) == 16 and t.lookup(12, 64) == 8


def test_nearest_n_of_the_same_rank_smaller_on_ties():
    t = _table()
    assert t.lookup(9, 8) == 1      # 8 is nearest
    assert t.lookup(10, 8) == 1     # tie between 8 and 12: the smaller n
    assert t.lookup(11, 8) == 4
    assert t.lookup(14, 8) == 4     # tie between 12 and 16
    assert t.lookup(18, 8) == 16
    assert t.lookup(18, 64) == 8    # only entry of r = 64


def test_untuned_rank_takes_the_library_rule():
    assert _table().lookup(12, 16) == 0
    assert BatchTable().lookup(10, 8) == 0


def test_splits_for_a_batch_and_round_trip(tmp_path):
    t = _table()
    circs = [{"n": 8, "r": 8}, {"n": 13, "r": 8}, {"n": 12, "r": 32}, {"n": 17, "r": 64}]
    assert t.splits_for(circs) == [1, 4, 0, 8]
    p = tmp_path / "sub" / "table.json"
    t.save(str(p))
    u = BatchTable.load(str(p))
    assert u.entries == t.entries and u.device == "test"
    assert u.times[(8, 8)] == {"1": 0.5, "2": 0.7}
    assert u.splits_for(circs) == t.splits_for(circs)


def test_rejects_nonpositive_counts():
    with pytest.raises(ValueError):
        BatchTable().add(8, 8, 0)


def test_committed_table_covers_the_batch_workload():
    if not os.path.exists(DEFAULT_TABLE):
        pytest.skip("no tuned table committed")
    d = json.load(open(DEFAULT_TABLE))
    t = BatchTable.load(DEFAULT_TABLE)
    assert d["device"] and t.entries
    for n in range(8, 19):
        for r in (8, 16, 32, 64):
            sp = t.lookup(n, r)
            assert (n, r) in t.entries and 1 <= sp <= min(64, 1 << (n - 1))
            ms = t.times[(n, r)]
            assert min(ms, key=lambda k: (ms[k], int(k))) == str(sp)  # the fastest candidate was kept


def test_environment_variable_names_the_table(tmp_path, monkeypatch):
    p = tmp_path / "mine.json"
    _table().save(str(p))
    monkeypatch.setenv(TABLE_ENV, str(p))
    assert table_path() == str(p)
    t = BatchTable.load_or_empty()
    assert t.device == "test" and t.lookup(12, 64) == 8
    monkeypatch.setenv(TABLE_ENV, str(tmp_path / "missing.json"))
    assert BatchTable.load_or_empty().entries == {}  # a named file that does not exist: no table
    monkeypatch.delenv(TABLE_ENV)
    assert table_path() == DEFAULT_TABLE
