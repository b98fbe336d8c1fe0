"""The autotuner's schedule cache on the host (no GPU): entries written in
the library's file format load back into its table, which saves them again
unchanged; malformed files merge nothing."""

import json
import os

import pytest

from paper_1404_0424_gb300 import cabi


def cache_text(entries):
    """The library's file format: a JSON array, one object per line."""
    return "[\n" + ",\n".join(json.dumps(e) for e in entries) + "\n]\n"


@pytest.fixture(scope="module")
def lib():
    try:
        from paper_1404_0424_gb300 import build
        return cabi.library(build.build())
    except (OSError, RuntimeError) as e:
        pytest.skip(f"libcgmimo not available: {e}")


ENTRIES = [
    {"key": "NVIDIA GB300|0,32,1,256,14,0,11|0,16,1,128,14,0,10", "precision": 4, "order": 1,
     "concurrent": 0, "grid_pct": 100, "ms": 0.0831},
    {"key": "NVIDIA GB300|1,8,1,64,4,0,3", "precision": 3, "order": 0, "concurrent": 1,
     "grid_pct": 50, "ms": 0.0123},
]


def test_cache_round_trip(lib, tmp_path):
    src = tmp_path / "tune.json"
    src.write_text(cache_text(ENTRIES))
    before = cabi.cg_tune_cache_size()
    assert cabi.cg_tune_cache_load(str(src)) == 2
    assert cabi.cg_tune_cache_size() == before + 2
    out = tmp_path / "saved.json"
    assert cabi.cg_tune_cache_save(str(out)) == cabi.cg_tune_cache_size()
    saved = {e["key"]: e for e in json.loads(out.read_text())}
    for e in ENTRIES:
        got = saved[e["key"]]
        for f in ("precision", "order", "concurrent", "grid_pct"):
            assert got[f] == e[f]
        assert abs(got["ms"] - e["ms"]) < 1e-6
    # loading the saved file again changes nothing
    assert cabi.cg_tune_cache_load(str(out)) == len(saved)
    assert cabi.cg_tune_cache_size() == before + 2


@pytest.mark.parametrize("bad", [
    {"key": "x", "precision": 9, "order": 1, "concurrent": 1, "grid_pct": 100},   # precision
    {"key": "x", "precision": 4, "order": 2, "concurrent": 1, "grid_pct": 100},   # order
    {"key": "x", "precision": 4, "order": 1, "concurrent": 1, "grid_pct": 0},     # grid share
    {"precision": 4, "order": 1, "concurrent": 1, "grid_pct": 100},               # no key
])
def test_malformed_files_merge_nothing(lib, tmp_path, bad):
    f = tmp_path / "bad.json"
    good = {"key": "y", "precision": 4, "order": 1, "concurrent": 1, "grid_pct": 100}
    f.write_text(cache_text([good, bad]))
    before = cabi.cg_tune_cache_size()
    assert cabi.cg_tune_cache_load(str(f)) == cabi.CG_EINVAL
    assert cabi.cg_tune_cache_size() == before


def test_missing_file(lib, tmp_path):
    assert cabi.cg_tune_cache_load(str(tmp_path / "none.json")) == cabi.CG_EINVAL
    assert not os.path.exists(tmp_path / "none.json")
