"""Host logic of the launch-shape autotuner: bucket selection from a table."""
from paper_2401_05301_gb300.autotune import tuned_options

TABLE = {"buckets": [
    {"form": "dense", "chi": 64, "d": 4, "max_slots": 24, "panel_blocks": 1},
    {"form": "dense", "chi": 256, "d": 4, "max_slots": 8, "panel_blocks": 3},
    {"form": "dense", "chi": 256, "d": 5, "max_slots": 16, "panel_blocks": 2},
    {"form": "u1", "chi": 1024, "d": 5, "max_slots": 4, "panel_blocks": 2},
]}


def test_nearest_chi_same_form_and_d():
    assert tuned_options(TABLE, "dense", 100, 4) == {"max_slots": 24, "panel_blocks": 1}
    assert tuned_options(TABLE, "dense", 200, 4) == {"max_slots": 8, "panel_blocks": 3}
    assert tuned_options(TABLE, "dense", 512, 5) == {"max_slots": 16, "panel_blocks": 2}


def test_other_d_falls_back_to_the_form():
    assert tuned_options(TABLE, "dense", 256, 8) == {"max_slots": 8, "panel_blocks": 3}
    assert tuned_options(TABLE, "u1", 300, 4) == {"max_slots": 4, "panel_blocks": 2}


def test_unknown_form_gives_no_options():
    assert tuned_options(TABLE, "supersite", 64, 25) == {}
    assert tuned_options({}, "dense", 64, 4) == {}
