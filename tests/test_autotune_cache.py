"""The autotuner's cache file (host only, no GPU): round trip, rejection of
malformed or invalid files without partial updates."""
from __future__ import annotations

import json

import pytest

from paper_2501_14030_gb300 import nrr


@pytest.fixture(autouse=True, scope="module")
def _built_library():
    from paper_2501_14030_gb300 import build
    build.build()
    nrr.lib()


ENTRIES = [
    {"coord": 0, "n": [128, 128, 16], "ng": 4, "fp32": 0, "variant": 0, "zc": 1,
     "block": 64, "pdl": 1},
    {"coord": 2, "n": [256, 256, 256], "ng": 4, "fp32": 1, "variant": 1, "zc": 16,
     "block": 128, "pdl": 1},
    {"coord": 3, "n": [128, 64, 16], "ng": 4, "fp32": 1, "variant": 3, "zc": 8,
     "block": 128, "pdl": 0},
]


def _write(path, entries):
    path.write_text(json.dumps({"nrr_autotune": 1, "entries": entries}))


def _saved(path):
    nrr.autotune_save(str(path))
    return json.loads(path.read_text())["entries"]


def _key(e):
    return (e["coord"], tuple(e["n"]), e["ng"], e["fp32"])


def test_cache_round_trip(tmp_path):
    nrr.autotune_clear()
    _write(tmp_path / "in.json", ENTRIES)
    nrr.autotune_load(str(tmp_path / "in.json"))
    out = _saved(tmp_path / "out.json")
    assert sorted(out, key=_key) == sorted(ENTRIES, key=_key)
    nrr.autotune_clear()
    assert _saved(tmp_path / "empty.json") == []


@pytest.mark.parametrize("bad", [
    dict(variant=9), dict(zc=3), dict(block=96), dict(pdl=2), dict(coord=7),
    dict(fp32=2),
])
def test_invalid_entry_rejected_without_partial_update(tmp_path, bad):
    nrr.autotune_clear()
    entries = [dict(ENTRIES[0]), dict(ENTRIES[1], **bad)]
    _write(tmp_path / "bad.json", entries)
    with pytest.raises(nrr.NrrError):
        nrr.autotune_load(str(tmp_path / "bad.json"))
    assert _saved(tmp_path / "after.json") == []


def test_malformed_files_rejected(tmp_path):
    nrr.autotune_clear()
    (tmp_path / "a.json").write_text('{"something": 1}')
    (tmp_path / "b.json").write_text('{"nrr_autotune": 1, "entries": [{"coord": 0')
    (tmp_path / "c.json").write_text('{"nrr_autotune": 1, "entries": [{"coord": 0}]}')
    for name in ("a.json", "b.json", "c.json", "missing.json"):
        with pytest.raises(nrr.NrrError):
            nrr.autotune_load(str(tmp_path / name))
    assert _saved(tmp_path / "after.json") == []
