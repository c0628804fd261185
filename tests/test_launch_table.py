"""The autotuned launch table (paper_2608_04283_b300/tuning.json) and the way
bench.py reads it: every entry is a shape vklb_set_tiling accepts (tile_x a
multiple of 32 in 32..256, tile_y in 1..256 or -1 for the wave-fit height), a
variant entry belongs to a tuned entry, and the nearest tuned side is used."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

TABLE = json.load(open(os.path.join(ROOT, "paper_2608_04283_b300", "tuning.json")))


def test_entries_are_valid_shapes():
    for key, ent in TABLE.items():
        if key.startswith("_"):
            continue
        system, prec = key.split("/")
        assert system in ("swe", "euler", "mhd_glm", "advection") and prec in ("fp32", "fp64", "bf16")
        for side, (tx, ty) in ent.items():
            assert int(side) > 0
            assert tx % 32 == 0 and 32 <= tx <= 256
            assert ty == -1 or 1 <= ty <= 256


def test_variant_entries_belong_to_tuned_entries():
    for key, var in TABLE.get("_variants", {}).items():
        system, prec, side = key.split("/")
        assert side in TABLE[f"{system}/{prec}"]
        assert var[0] in (0, 1) and (var[0] == 0 or 2 <= var[1] <= 8)


def test_launch_shape_uses_nearest_side():
    for key, ent in TABLE.items():
        if key.startswith("_"):
            continue
        system, prec = key.split("/")
        for side, tile in ent.items():
            n = int(side)
            tile_got, var = bench.launch_shape(system, prec, (n, n))
            assert tuple(tile_got) == tuple(tile)
            assert var == tuple(TABLE.get("_variants", {}).get(f"{system}/{prec}/{side}", (0, 0)))
    assert bench.launch_shape("nonexistent", "fp32", (64, 64)) is None
