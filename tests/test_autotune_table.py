"""The autotuner's table format: first-match lookup finds each problem's own cell."""
import itertools
import json

from paper_1602_08477_gb300 import autotune


def test_first_match_is_the_problems_own_cell():
    T = autotune.THRESHOLDS
    entries = [(m, n, k, "64x64") for m in T for n in T for k in T]
    for m, n, k in itertools.product([1, 17, 32, 33, 64, 100, 128, 129, 300, 512], repeat=3):
        first = next(e for e in entries if m <= e[0] and n <= e[1] and k <= e[2])
        assert first[:3] == (autotune.cell_of(m), autotune.cell_of(n), autotune.cell_of(k))


def test_shipped_table_covers_every_cell(tmp_path):
    entries = autotune.load(apply=False)
    native = [e for e in entries if autotune.kind_of(e[3]) == "native"]
    T = autotune.THRESHOLDS
    assert {e[:3] for e in native} == {(m, n, k) for m in T for n in T for k in T}
    assert all(e[3] in autotune.CANDIDATES for e in native)
    # slice counts: one entry per K cell, for every m and n, each a candidate
    slices = [e for e in entries if autotune.kind_of(e[3]) == "slices"]
    if slices:
        assert [e[:3] for e in slices] == [(autotune.ANY, autotune.ANY, k) for k in T]
        assert all(int(e[3][len("emu_s"):]) in autotune.SLICE_CANDIDATES + (autotune.REF_SLICES,)
                   for e in slices)
    # save/load round trip
    p = tmp_path / "t.json"
    autotune.save(entries, str(p))
    assert autotune.load(str(p), apply=False) == entries
    assert json.load(open(p))["thresholds"] == list(T)


def test_table_path_prefers_argument_then_environment(tmp_path, monkeypatch):
    monkeypatch.delenv("GB_TUNE_TABLE", raising=False)
    assert autotune.table_path() == autotune.DEFAULT_TABLE
    own = tmp_path / "own.json"
    autotune.save([(32, 32, 32, "32x32")], str(own))
    monkeypatch.setenv("GB_TUNE_TABLE", str(own))
    assert autotune.table_path() == str(own)
    assert autotune.load(apply=False) == [(32, 32, 32, "32x32")]
    assert autotune.table_path("x.json") == "x.json"


def test_entry_kinds():
    assert autotune.kind_of("32x64") == "native"
    assert autotune.kind_of("emu_cols") == "emulated"
    assert autotune.kind_of("emu_s10") == "slices"
    assert autotune.kind_of(111) == "slices"
    assert autotune.kind_of(5) == "emulated"


def test_slice_choice_keeps_the_default_unless_clearly_faster():
    E = autotune.EMU_SLICES
    assert autotune.choose_slices({}) == autotune.REF_SLICES       # nothing met the target
    assert autotune.choose_slices({E: 1.0, E + 1: 1.2}) == E
    assert autotune.choose_slices({E - 1: 0.99, E: 1.0}) == E      # 1 % is not enough
    assert autotune.choose_slices({E - 1: 0.90, E: 1.0}) == E - 1
    assert autotune.choose_slices({E + 1: 0.5}) == E + 1           # default over the target
