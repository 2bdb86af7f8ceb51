"""Host logic of the Python binding (no GPU): tile grids, the sort's bit
range and the configuration flags."""
import pytest

from paper_2602_03207_gb300 import capi, render


def test_tile_grid_and_key_bits():
    assert render.tile_grid(1920, 1080, 16) == (120, 68)
    assert render.tile_grid(3840, 2160, 16) == (240, 135)
    assert render.tile_grid(1, 1, 16) == (1, 1)
    # keys are (tile << 31) | depth bits: 13 tile bits at 1080p, 15 at 2160p
    assert render.key_end_bit(1920, 1080, 16) == 31 + 13
    assert render.key_end_bit(3840, 2160, 16) == 31 + 15
    assert render.key_end_bit(16, 16, 16) == 31  # one tile: the depth bits alone
    assert render.key_end_bit(32, 16, 16) == 32
    # every tile id fits below the end bit
    for w, h, t in ((1920, 1080, 8), (1280, 720, 32), (257, 255, 16)):
        tx, ty = render.tile_grid(w, h, t)
        assert tx * ty - 1 < 1 << (render.key_end_bit(w, h, t) - 31)


def test_config_flags():
    assert render.config_flags(0, "segmented") == capi.WS_CFG_SORT_SEGMENTED
    assert render.config_flags(0, "lsd") == 0
    assert render.config_flags(0, "lookback") == capi.WS_CFG_SORT_LOOKBACK
    assert render.config_flags(capi.WS_CFG_FIXED_RADIUS, "lsd") == capi.WS_CFG_FIXED_RADIUS
    with pytest.raises(ValueError):
        render.config_flags(0, "bitonic")
