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
