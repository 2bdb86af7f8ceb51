"""Pair counts past the 32-bit range and past the key capacity (ws_cull).

A frame can cover more (tile, splat) pairs than 2^32 when screen-filling
splats are kept (for instance with the culling switched off at 4K). The
compaction must then raise WS_FLAG_CAPACITY, clamp the key count to the
capacity and write nothing past it, instead of letting the 32-bit slot
arithmetic wrap onto valid slots. The inputs are crafted tile counts and
rectangles handed straight to ws_cull through the C ABI."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SAT = 0xFFFFFFFF


def _cull(touched, rect, cap, width=8192, height=8192, tile=8, guard=4096):
    import torch
    from paper_2602_03207_gb300 import capi
    n = touched.size
    cam = capi.camera({"viewmat": np.eye(3, 4), "fx": 100.0, "fy": 100.0, "cx": width / 2, "cy": height / 2,
                       "width": width, "height": height, "znear": 0.2, "bg": (0, 0, 0)})
    cfg = capi.config(tile=tile, digit_bits=8)
    t = torch.from_numpy(touched.astype(np.uint32).view(np.int32)).cuda()
    r = torch.from_numpy(rect.astype(np.uint16).view(np.int16)).cuda()
    depth = torch.full((n,), 2.5, dtype=torch.float32, device="cuda")
    offsets = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    keys = torch.full((cap + guard,), -3, dtype=torch.int64, device="cuda")
    vals = torch.full((cap + guard,), -9, dtype=torch.int32, device="cuda")
    num = torch.zeros(4, dtype=torch.int32, device="cuda")
    ws = torch.zeros(capi.ws_workspace_bytes(n, cap, cam, cfg), dtype=torch.uint8, device="cuda")
    capi.ws_cull(n, t, r, depth, cam, cfg, offsets, keys, vals, cap, num, ws)
    flags = capi.ws_read_status(ws)
    return (flags, int(num[0].item()) & SAT, offsets.cpu().numpy().view(np.uint32),
            keys.cpu().numpy().view(np.uint64), vals.cpu().numpy().view(np.uint32))


def _first_keys(count, tiles_x, x1, depth_bits):
    j = np.arange(count, dtype=np.uint64)
    w = np.uint64(x1 + 1)
    tile = (j // w) * np.uint64(tiles_x) + (j % w)
    return (tile << np.uint64(31)) | np.uint64(depth_bits)


def test_total_pairs_past_two_to_the_32_are_flagged_and_dropped():
    """5,000 screen-filling splats on a 1024 x 1024 tile grid: 5,000 * 2^20
    pairs (> 2^32). Offsets saturate at 2^32 - 1, the count is the capacity,
    the first capacity pairs are Gaussian 0's tiles in row-major order, and
    the buffers past the capacity are untouched."""
    from paper_2602_03207_gb300 import capi
    n, per, cap = 5000, 1 << 20, 10_000
    touched = np.full(n, per, np.uint64)
    rect = np.tile(np.array([0, 0, 1023, 1023], np.uint16), (n, 1))
    flags, num, offsets, keys, vals = _cull(touched, rect, cap)
    assert flags & capi.WS_FLAG_CAPACITY
    assert num == cap
    expect_off = np.minimum(np.arange(n + 1, dtype=np.uint64) * np.uint64(per), np.uint64(SAT))
    np.testing.assert_array_equal(offsets.astype(np.uint64), expect_off)
    dbits = int(np.float32(2.5).view(np.uint32))
    np.testing.assert_array_equal(keys[:cap], _first_keys(cap, 1024, 1023, dbits))
    np.testing.assert_array_equal(vals[:cap], np.zeros(cap, np.uint32))
    assert (keys[cap:] == np.uint64(2 ** 64 - 3)).all() and (vals[cap:] == np.uint32(2 ** 32 - 9)).all()


def test_one_chunk_summing_past_two_to_the_32():
    """Three Gaussians of one compaction chunk whose tile counts alone sum
    past 2^32 (crafted counts, larger than their rectangles): the chunk's sum
    saturates, the frame is flagged, and only slots below the capacity are
    written."""
    from paper_2602_03207_gb300 import capi
    cap = 3000
    touched = np.array([3_000_000_000, 3_000_000_000, 5], np.uint64)
    rect = np.tile(np.array([0, 0, 1023, 1023], np.uint16), (3, 1))
    flags, num, offsets, keys, vals = _cull(touched, rect, cap)
    assert flags & capi.WS_FLAG_CAPACITY
    assert num == cap
    assert offsets[0] == 0 and offsets[1] == 3_000_000_000 and offsets[3] == SAT
    dbits = int(np.float32(2.5).view(np.uint32))
    np.testing.assert_array_equal(keys[:cap], _first_keys(cap, 1024, 1023, dbits))
    assert (keys[cap:] == np.uint64(2 ** 64 - 3)).all()


def test_exact_capacity_is_not_flagged():
    """Total pairs equal to the capacity: no flag, every slot written."""
    n, cap = 3, 3 * 16
    touched = np.full(n, 16, np.uint64)
    rect = np.tile(np.array([2, 5, 5, 8], np.uint16), (n, 1))
    flags, num, offsets, keys, vals = _cull(touched, rect, cap, width=64, height=96)
    assert flags == 0 and num == cap
    np.testing.assert_array_equal(offsets, [0, 16, 32, 48])
    np.testing.assert_array_equal(vals[:cap], np.repeat(np.arange(3, dtype=np.uint32), 16))
