"""bench.py's work model on the host: the algorithmic bytes per stage that the roofline
fractions divide by follow the per-unit figures of the kernels (entries of a 16-bit tile id and
a 32-bit value when the tile bits fit 16, else a 32-bit key and a value; exact mode 64-bit keys)."""
from __future__ import annotations

import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stats(passes, b_d=17, tiles_x=240, tiles_y=135):
    return {"n_gaussians": 3_000_000, "n_front": 2_500_000, "n_visible": 2_000_000, "n_entries": 60_000_000,
            "tiles_x": tiles_x, "tiles_y": tiles_y, "sort_passes": passes, "b_d": b_d,
            "n_pairs": 600_000_000, "n_blends": 400_000_000}


def test_roofgs_16_bit_entries():
    st = _stats(2)
    w = bench.stage_work("roofgs", st, 3840, 2160)
    N, nf, nv, nd = 3_000_000, 2_500_000, 2_000_000, 60_000_000
    assert w["sort_pass"] == 12 * nd  # 2 B tile id + 4 B value, read and written
    assert w["front"] == 20 * N + 16 * nf + 80 * nv + 6 * nd
    # the front end counted the digits: the histogram kernel clears 1 KB of look-back status per
    # 6144-entry tile and sums 16 copies of [2][256] counts
    assert w["hist"] == 1024 * ((nd + 6143) // 6144) + 17 * 512 * 4
    assert w["depth"] == 24 * N + 16 * 3 * N  # b_d = 17: three 8-bit passes of 16 B per pair
    assert w["ranges"] == 0
    assert w["raster_ops"] == 5 * 600_000_000 + 11 * 400_000_000


def test_roofgs_more_than_16_tile_bits_and_exact_mode():
    nd = 60_000_000
    w = bench.stage_work("roofgs", _stats(3, b_d=15, tiles_x=480, tiles_y=270), 7680, 4320)
    assert w["sort_pass"] == 16 * nd and w["hist"] == 4 * nd  # 32-bit keys, keys read for the digits
    assert w["front"] == 20 * 3_000_000 + 16 * 2_500_000 + 80 * 2_000_000 + 8 * nd
    w = bench.stage_work("exact", _stats(6), 3840, 2160)
    assert w["sort_pass"] == 24 * nd and w["depth"] == 0
    # the duplicate kernel counts the digits of all 6 passes (4 depth + 2 tile digits)
    assert w["hist"] == 1024 * ((nd + 4095) // 4096) + 17 * 6 * 256 * 4
    assert w["front"] == 32 * 3_000_000 + 28 * 2_500_000 + 280 * 2_000_000 + 12 * nd
    assert w["ranges"] == 8 * nd + 8 * 240 * 135
    w = bench.stage_work("exact", _stats(7, tiles_x=480, tiles_y=270), 7680, 4320)
    assert w["hist"] == 8 * nd  # 3 tile digits: the keys are read for the digits


def test_roofgs_row_bucketed_front_end():
    """The row-bucketed front end (the default where the tile grid fits 256 x 256 and the tile bits
    16): the fused kernel's bytes plus the row data it stores and reads back, and one column pass."""
    st = dict(_stats(1), b_t=15)
    assert bench.row_buckets(st, ordered=False)
    assert not bench.row_buckets(st, ordered=True)
    assert not bench.row_buckets(dict(st, tiles_x=480, tiles_y=270, b_t=17), ordered=False)
    assert not bench.row_buckets(dict(st, tiles_x=120, tiles_y=270), ordered=False)  # 32 x 8 tiles at 4K
    w = bench.stage_work("roofgs", st, 3840, 2160, rows=True)
    N, nf, nv, nd = 3_000_000, 2_500_000, 2_000_000, 60_000_000
    nb = (N + 255) // 256
    # + 4 B of tile rows per slot written and read, 48 B row test + 4 B order per visible Gaussian
    # (written / read back), 4 B per (tile row, block) counted, scanned both ways and read
    assert w["front"] == 20 * N + 16 * nf + 80 * nv + 6 * nd + 8 * N + 100 * nv + 16 * 135 * nb
    assert w["sort_pass"] == 12 * nd and w["passes"] == 1
    # one pass's digit counts summed from the front end's 16 copies
    assert w["hist"] == 1024 * ((nd + 6143) // 6144) + 17 * 256 * 4
