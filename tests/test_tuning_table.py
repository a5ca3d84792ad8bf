"""Host side of the tuning table: the entry of the largest size class not
above a filter's size applies, per kind; unknown knobs are refused."""
import pytest

import paper_2212_09005_gb300 as gf
from paper_2212_09005_gb300 import tuning


def test_lookup_takes_largest_class_not_above(monkeypatch):
    monkeypatch.setattr(tuning, "_table", {
        "tcf": {"20": {"tcf_path": 1}, "26": {"tcf_path": 2, "tcf_tile_target": 512}},
        "gqf": {"18": {"gqf_region_groups": 16}},
    })
    assert tuning.lookup(gf.FILTER_TCF, 19) == {}
    assert tuning.lookup(gf.FILTER_TCF, 20) == {"tcf_path": 1}
    assert tuning.lookup(gf.FILTER_TCF, 25) == {"tcf_path": 1}
    assert tuning.lookup(gf.FILTER_TCF, 30) == {"tcf_path": 2, "tcf_tile_target": 512}
    assert tuning.lookup(gf.FILTER_GQF, 28) == {"gqf_region_groups": 16}
    assert tuning.lookup(gf.FILTER_GQF, 17) == {}


def test_struct_packs_knobs():
    t = tuning.struct({"tcf_path": 2, "tcf_tile_target": 256, "gqf_region_groups": 4, "tcf_tiled_min_blocks": 1 << 20})
    assert (t.tcf_path, t.tcf_tile_target, t.gqf_region_groups, t.tcf_tiled_min_blocks) == (2, 256, 4, 1 << 20)
    with pytest.raises(gf.FilterError):
        tuning.struct({"bogus": 1})


def test_missing_table_means_defaults(monkeypatch, tmp_path):
    monkeypatch.setattr(tuning, "_table", None)
    monkeypatch.setattr(tuning, "TABLE_PATH", str(tmp_path / "none.json"))
    assert tuning.table() == {}
    assert tuning.lookup(gf.FILTER_TCF, 28) == {}


def test_group_rows_cover_groups_from_their_class(monkeypatch):
    monkeypatch.setattr(tuning, "_table", {
        "tcf": {"20": {"tcf_path": 1}, "28": {"tcf_path": 2}},
        "tcf_group": {"27": {"tcf_path": 1}},
    })
    assert tuning.lookup(gf.FILTER_TCF, 28) == {"tcf_path": 2}               # one filter
    assert tuning.lookup(gf.FILTER_TCF, 28, group=True) == {"tcf_path": 1}   # a group of as many slots
    assert tuning.lookup(gf.FILTER_TCF, 22, group=True) == {"tcf_path": 1}   # below the group class: filter rows
    assert tuning.lookup(gf.FILTER_TCF, 12, group=True) == {}
