"""The batched executor's autotuner table (host side, CPU only): export,
import, replacement, validation and the JSON file of the binding.  The
table lives in host memory, so none of this needs a GPU."""
import json

import pytest

from paper_2112_15071_gb300 import ews


@pytest.fixture
def table():
    ews.load()
    ews.ews_batch_tuning_clear()
    yield
    ews.ews_batch_tuning_clear()


ENTRIES = [
    {"nx": 96, "ny": 96, "nz": 96, "boundary": "sponge", "free_surface": False, "zchunk": 8},
    {"nx": 64, "ny": 48, "nz": 40, "boundary": "cpml", "free_surface": True, "zchunk": 40},
    {"nx": 64, "ny": 48, "nz": 40, "boundary": "cpml", "free_surface": False, "zchunk": 12},
]


def key(e):
    return (e["nx"], e["ny"], e["nz"], ews.BOUNDARY[e["boundary"]], e["free_surface"])


def test_empty_after_clear(table):
    assert ews.ews_batch_tuning_export() == []
    assert ews.ews_batch_tuned_zchunk(ews.ews_grid(96, 96, 96, 10.0, 10.0, 10.0), 1, False) == 0


def test_import_export_and_lookup(table):
    ews.ews_batch_tuning_import(ENTRIES)
    got = ews.ews_batch_tuning_export()
    assert got == sorted(ENTRIES, key=key)
    g = ews.ews_grid(64, 48, 40, 10.0, 10.0, 10.0)
    # the surface form keeps its own entry
    assert ews.ews_batch_tuned_zchunk(g, ews.EWS_BOUNDARY_CPML, True) == 40
    assert ews.ews_batch_tuned_zchunk(g, ews.EWS_BOUNDARY_CPML, False) == 12
    assert ews.ews_batch_tuned_zchunk(g, ews.EWS_BOUNDARY_SPONGE, False) == 0


def test_same_key_is_replaced(table):
    ews.ews_batch_tuning_import(ENTRIES[:1])
    ews.ews_batch_tuning_import([dict(ENTRIES[0], zchunk=24)])
    got = ews.ews_batch_tuning_export()
    assert len(got) == 1 and got[0]["zchunk"] == 24


@pytest.mark.parametrize("bad", [
    {"nx": 0}, {"nz": -3}, {"boundary": 7}, {"free_surface": 2}, {"zchunk": 0}, {"zchunk": 97}])
def test_invalid_entry_imports_nothing(table, bad):
    e = dict(ENTRIES[0])
    e.update(bad)
    if bad.get("free_surface") == 2:              # the binding maps truth values to 0 / 1
        arr = (ews.ews_tuned_zchunk * 1)(ews.ews_tuned_zchunk(96, 96, 96, 1, 2, 8))
        assert ews.load().ews_batch_tuning_import(arr, 1) == ews.EWS_EINVAL
    else:
        with pytest.raises(ews.EwsError) as err:
            ews.ews_batch_tuning_import([ENTRIES[2], e])
        assert err.value.status == ews.EWS_EINVAL
        assert "nothing imported" in str(err.value)
    assert ews.ews_batch_tuning_export() == []


def test_export_with_small_capacity(table):
    ews.ews_batch_tuning_import(ENTRIES)
    lib = ews.load()
    assert lib.ews_batch_tuning_export(None, 0) == 3
    arr = (ews.ews_tuned_zchunk * 1)()
    assert lib.ews_batch_tuning_export(arr, 1) == 3
    assert (arr[0].nx, arr[0].ny, arr[0].nz) == (64, 48, 40)


def test_json_roundtrip_and_device_tag(table, tmp_path):
    ews.ews_batch_tuning_import(ENTRIES)
    path = str(tmp_path / "tuning.json")
    assert ews.save_batch_tuning(path, device="GPU A") == 3
    doc = json.load(open(path))
    assert doc["format"] == ews.TUNING_FORMAT and doc["device"] == "GPU A"
    ews.ews_batch_tuning_clear()
    # entries timed on another GPU are not taken
    assert ews.load_batch_tuning(path, device="GPU B") == 0
    assert ews.ews_batch_tuning_export() == []
    assert ews.load_batch_tuning(path, device="GPU A") == 3
    assert ews.ews_batch_tuning_export() == sorted(ENTRIES, key=key)


def test_json_of_another_format_is_refused(table, tmp_path):
    path = tmp_path / "other.json"
    path.write_text(json.dumps({"format": "something-else", "entries": []}))
    with pytest.raises(ValueError):
        ews.load_batch_tuning(str(path), device="GPU A")
