"""Host-side tuning table of the grouped kernel (no device work)."""
import pytest

from paper_1602_08477_gb300 import build


@pytest.fixture(scope="module")
def gb():
    build()
    import paper_1602_08477_gb300 as gb
    return gb


def test_default_size_rule(gb):
    gb.tune_set([])
    assert gb.tune_get() == []
    assert gb.tune_lookup(500, 500, 500) == "64x64"
    assert gb.tune_lookup(500, 20, 500) == "64x32"
    assert gb.tune_lookup(20, 500, 500) == "32x64"
    assert gb.tune_lookup(20, 20, 500) == "32x32"


def test_first_matching_entry_wins(gb):
    gb.tune_set([(64, 64, 1 << 30, "32x32"), (1 << 30, 1 << 30, 128, "64x32")])
    try:
        assert gb.tune_get() == [(64, 64, 1 << 30, "32x32"), (1 << 30, 1 << 30, 128, "64x32")]
        assert gb.tune_lookup(60, 60, 4000) == "32x32"
        assert gb.tune_lookup(300, 300, 100) == "64x32"
        assert gb.tune_lookup(300, 300, 300) == "64x64"   # no entry: size rule
    finally:
        gb.tune_set([])


def test_invalid_entries_rejected(gb):
    with pytest.raises(gb.GbError, match="INVALID_ARG"):
        gb.tune_set([(1, 1, 1, 0)])
    with pytest.raises(gb.GbError, match="INVALID_ARG"):
        gb.tune_set([(1, 1, 1, 7)])


def test_emulated_orientation_padding_rule(gb):
    # no emulated entry: the orientation with fewer padded output slots (128 x bn
    # tiles, bn = 32 at s = 11): wide problems put B's columns on the 128-line side
    gb.tune_set([])
    assert gb.tune_lookup_emulated(500, 20, 64) == "emu_rows"
    assert gb.tune_lookup_emulated(20, 500, 64) == "emu_cols"
    assert gb.tune_lookup_emulated(128, 128, 64) == "emu_rows"   # equal padding: rows
    with pytest.raises(gb.GbError, match="INVALID_ARG"):
        gb.tune_lookup_emulated(10, 10, 10, slices=17)


def test_entries_of_each_kind_apply_to_their_own_problems(gb):
    # an emulated entry does not change native lookups and a native entry does not
    # change emulated ones; first match per kind
    gb.tune_set([(64, 64, 1 << 30, "emu_cols"), (64, 64, 1 << 30, "32x64"),
                 (1 << 30, 1 << 30, 1 << 30, "emu_rows")])
    try:
        assert gb.tune_lookup(60, 60, 100) == "32x64"
        assert gb.tune_lookup(300, 300, 100) == "64x64"          # size rule
        assert gb.tune_lookup_emulated(60, 60, 100) == "emu_cols"
        assert gb.tune_lookup_emulated(20, 500, 100) == "emu_rows"  # second emulated entry
    finally:
        gb.tune_set([])


def test_slice_count_entries(gb):
    # slice-count entries (GB_TUNE_SLICES + s) give emulated problems with
    # slices = 0 their count; no matching entry: 11; native tiles and emulated
    # orientations are unaffected
    big = (1 << 31) - 1
    gb.tune_set([])
    assert gb.tune_lookup_slices(100, 100, 100) == 11
    gb.tune_set([(big, big, 64, "emu_s12"), (big, big, 512, "emu_s10"),
                 (64, 64, 1 << 30, "32x32")])
    try:
        assert gb.tune_get()[0] == (big, big, 64, "emu_s12")
        assert gb.tune_lookup_slices(300, 300, 40) == 12
        assert gb.tune_lookup_slices(300, 300, 64) == 12
        assert gb.tune_lookup_slices(300, 300, 65) == 10
        assert gb.tune_lookup_slices(300, 300, 512) == 10
        assert gb.tune_lookup_slices(300, 300, 513) == 11     # no entry
        assert gb.tune_lookup(60, 60, 100) == "32x32"
        assert gb.tune_lookup(300, 300, 100) == "64x64"       # size rule
        # orientation of a problem given slices = 0 follows the table's count: at
        # s = 10 the product tiles are 128 x 48, at s = 12 128 x 32
        assert gb.tune_lookup_emulated(40, 100, 200, slices=0) == \
            gb.tune_lookup_emulated(40, 100, 200, slices=10)
        assert gb.tune_lookup_emulated(40, 100, 20, slices=0) == \
            gb.tune_lookup_emulated(40, 100, 20, slices=12)
    finally:
        gb.tune_set([])


def test_slice_count_entries_outside_range_rejected(gb):
    for t in (100, 117, 99, 200):
        with pytest.raises(gb.GbError, match="INVALID_ARG"):
            gb.tune_set([(1, 1, 1, t)])
    gb.tune_set([(1, 1, 1, 101), (1, 1, 1, 116)])
    try:
        assert [e[3] for e in gb.tune_get()] == ["emu_s1", "emu_s16"]
    finally:
        gb.tune_set([])
