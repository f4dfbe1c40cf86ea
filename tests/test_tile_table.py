"""The tile-shape table of the forward passes (host side, CPU only):
export, import, replacement, validation, lookup, and the JSON file of the
binding, which carries it beside the batch z-chunk table.  The table lives
in host memory, so none of this needs a GPU."""
import json

import pytest

from paper_2112_15071_gb300 import ews


@pytest.fixture
def table():
    ews.load()
    ews.ews_tile_tuning_clear()
    ews.ews_batch_tuning_clear()
    yield
    ews.ews_tile_tuning_clear()
    ews.ews_batch_tuning_clear()


ENTRIES = [
    {"nx": 256, "ny": 256, "nz": 256, "boundary": "cpml", "storage": "f32", "shape": "32x8"},
    {"nx": 256, "ny": 256, "nz": 256, "boundary": "sponge", "storage": "f32", "shape": "32x4"},
    {"nx": 256, "ny": 256, "nz": 256, "boundary": "sponge", "storage": "bf16", "shape": "32x16"},
]


def key(e):
    return (e["nx"], e["ny"], e["nz"], ews.BOUNDARY[e["boundary"]], ews.STORAGE[e["storage"]])


def test_empty_after_clear(table):
    assert ews.ews_tile_tuning_export() == []
    assert ews.ews_tile_tuned(ews.ews_grid(256, 256, 256, 20.0, 20.0, 20.0), "cpml", "f32") == 0


def test_import_export_and_lookup(table):
    ews.ews_tile_tuning_import(ENTRIES)
    assert ews.ews_tile_tuning_export() == sorted(ENTRIES, key=key)
    g = ews.ews_grid(256, 256, 256, 20.0, 20.0, 20.0)
    # one entry per boundary and storage type of a grid size
    assert ews.ews_tile_tuned(g, "cpml", "f32") == ews.EWS_TILE_32X8
    assert ews.ews_tile_tuned(g, "sponge", "f32") == ews.EWS_TILE_32X4
    assert ews.ews_tile_tuned(g, "sponge", "bf16") == ews.EWS_TILE_32X16
    assert ews.ews_tile_tuned(g, "none", "f32") == 0
    # an import replaces the entry with the same key
    ews.ews_tile_tuning_import([dict(ENTRIES[1], shape="32x16")])
    assert ews.ews_tile_tuned(g, "sponge", "f32") == ews.EWS_TILE_32X16
    assert len(ews.ews_tile_tuning_export()) == 3


def test_fused_entries(table):
    """The fused step is a valid entry for FP32 storage without C-PML only."""
    ok = {"nx": 96, "ny": 96, "nz": 64, "boundary": "sponge", "storage": "f32", "shape": "fused"}
    ews.ews_tile_tuning_import([ok])
    g = ews.ews_grid(96, 96, 64, 20.0, 20.0, 20.0)
    assert ews.ews_tile_tuned(g, "sponge", "f32") == ews.EWS_TILE_FUSED
    assert ews.ews_tile_tuning_export() == [ok]
    for bad in (dict(ok, boundary="cpml"), dict(ok, storage="bf16"), dict(ok, storage="f16")):
        with pytest.raises(ews.EwsError):
            ews.ews_tile_tuning_import([bad])
    assert ews.ews_tile_tuning_export() == [ok]


@pytest.mark.parametrize("bad", [dict(ENTRIES[0], shape=0), dict(ENTRIES[0], shape=4),
                                 dict(ENTRIES[0], shape=5),
                                 dict(ENTRIES[0], nx=3), dict(ENTRIES[0], boundary=3),
                                 dict(ENTRIES[0], storage=5)])
def test_an_invalid_entry_imports_nothing(table, bad):
    with pytest.raises(ews.EwsError) as e:
        ews.ews_tile_tuning_import([ENTRIES[1], bad])
    assert e.value.status == ews.EWS_EINVAL
    assert ews.ews_tile_tuning_export() == []


def test_json_file_carries_both_tables(table, tmp_path):
    ews.ews_tile_tuning_import(ENTRIES)
    ews.ews_batch_tuning_import([{"nx": 96, "ny": 96, "nz": 96, "boundary": "sponge",
                                  "free_surface": False, "zchunk": 8}])
    path = str(tmp_path / "tuning.json")
    ews.save_batch_tuning(path, device="GB300-test")
    doc = json.load(open(path))
    assert doc["tiles"] == sorted(ENTRIES, key=key)
    ews.ews_tile_tuning_clear()
    ews.ews_batch_tuning_clear()
    assert ews.load_batch_tuning(path, device="GB300-test") == 1
    assert ews.ews_tile_tuning_export() == sorted(ENTRIES, key=key)
    # another GPU's tables are not loaded
    ews.ews_tile_tuning_clear()
    ews.ews_batch_tuning_clear()
    assert ews.load_batch_tuning(path, device="another GPU") == 0
    assert ews.ews_tile_tuning_export() == []


def test_shape_calls_validate_without_a_device():
    with pytest.raises(ews.EwsError) as e:
        ews.ews_set_tile_shape(None, "32x4")
    assert e.value.status == ews.EWS_EINVAL
    assert ews.ews_get_tile_shape(None) == 0
