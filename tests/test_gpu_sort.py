"""GPU parity of ws_sort (the wait-free radix sort of §3.3.2) on its own:
the sorted keys and values must equal a stable sort of the same input,
bit for bit, for every input shape, size and digit width."""
import numpy as np
import pytest

import oracle
from paper_2602_03207_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def gpu_sort(keys, vals, digit_bits=8, begin_bit=0, end_bit=64, capacity=None, flags=0):
    import torch
    from paper_2602_03207_gb300 import capi
    n = keys.size
    cap = max(capacity or n, 1)
    kt = torch.zeros(cap, dtype=torch.int64, device="cuda")
    vt = torch.zeros(cap, dtype=torch.int32, device="cuda")
    if n:
        kt[:n] = torch.from_numpy(keys.view(np.int64))
        vt[:n] = torch.from_numpy(vals.view(np.int32))
    ka = torch.empty_like(kt)
    va = torch.empty_like(vt)
    num = torch.tensor([n, 0, 0, 0], dtype=torch.int32, device="cuda")
    cfg = capi.config(digit_bits=digit_bits, flags=flags)
    cam = capi.camera(S.small_forward()[1])
    ws = torch.zeros(capi.ws_workspace_bytes(0, cap, cam, cfg), dtype=torch.uint8, device="cuda")
    in_alt = capi.ws_sort(num, cap, begin_bit, end_bit, kt, vt, ka, va, cfg, ws)
    torch.cuda.synchronize()
    k, v = (ka, va) if in_alt else (kt, vt)
    return k[:n].cpu().numpy().view(np.uint64), v[:n].cpu().numpy().view(np.uint32)


def _keys(kind, n, rng):
    if kind == "random":
        return rng.integers(0, 2 ** 45, n, dtype=np.uint64)
    if kind == "equal":
        return np.full(n, 77, np.uint64)
    if kind == "sorted":
        return np.sort(rng.integers(0, 2 ** 45, n, dtype=np.uint64))
    if kind == "reversed":
        return np.sort(rng.integers(0, 2 ** 45, n, dtype=np.uint64))[::-1].copy()
    return rng.integers(0, 4, n).astype(np.uint64) << np.uint64(40)  # few distinct


@pytest.mark.parametrize("n", [0, 1, 31, 4097, 8192 * 3 + 17])
@pytest.mark.parametrize("kind", ["random", "equal", "sorted", "reversed", "few"])
def test_sort_matches_stable_sort(n, kind):
    rng = np.random.default_rng(n * 7 + len(kind))
    keys = _keys(kind, n, rng)
    vals = rng.permutation(n).astype(np.uint32)
    k, v = gpu_sort(keys, vals, digit_bits=8, end_bit=45)
    ek, ev = oracle.sort_pairs(keys, vals)
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)


@pytest.mark.parametrize("bits", [4, 5, 6, 7, 8, 9, 10, 11])
def test_digit_widths_and_partial_bit_ranges(bits):
    """Digit widths that do not divide the bit range (a short last pass)
    and a begin bit above 0 (low bits then keep their input order)."""
    rng = np.random.default_rng(bits)
    keys = rng.integers(0, 2 ** 50, 50_000, dtype=np.uint64)
    vals = np.arange(keys.size, dtype=np.uint32)
    k, v = gpu_sort(keys, vals, digit_bits=bits, begin_bit=3, end_bit=50)
    perm = np.argsort(keys >> np.uint64(3), kind="stable")
    np.testing.assert_array_equal(k, keys[perm])
    np.testing.assert_array_equal(v, vals[perm])


def test_capacity_larger_than_count():
    """Grids sized by the capacity; blocks past the device-side count idle."""
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 2 ** 44, 10_000, dtype=np.uint64)
    vals = np.arange(10_000, dtype=np.uint32)
    k, v = gpu_sort(keys, vals, end_bit=44, capacity=1 << 20)
    ek, ev = oracle.sort_pairs(keys, vals)
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)


def test_standalone_4m_tile_depth_keys():
    """The sort-only workload: 4,194,304 (tile, depth) keys over 8,160 tiles."""
    keys, vals = S.sort_keys()
    k, v = gpu_sort(keys, vals, digit_bits=8, end_bit=44)
    ek, ev = oracle.sort_pairs(keys, vals)
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)


# ---------------------------------------------- single-sweep look-back variant

def gpu_sort_lookback(keys, vals, digit_bits=8, begin_bit=0, end_bit=64):
    import torch
    from paper_2602_03207_gb300 import capi
    n = keys.size
    cap = max(n, 1)
    kt = torch.zeros(cap, dtype=torch.int64, device="cuda")
    vt = torch.zeros(cap, dtype=torch.int32, device="cuda")
    if n:
        kt[:n] = torch.from_numpy(keys.view(np.int64))
        vt[:n] = torch.from_numpy(vals.view(np.int32))
    ka, va = torch.empty_like(kt), torch.empty_like(vt)
    num = torch.tensor([n, 0, 0, 0], dtype=torch.int32, device="cuda")
    cfg = capi.config(digit_bits=digit_bits, flags=capi.WS_CFG_SORT_LOOKBACK)
    ws = torch.zeros(capi.ws_workspace_bytes(0, cap, capi.camera(S.small_forward()[1]), cfg),
                     dtype=torch.uint8, device="cuda")
    in_alt = capi.ws_sort(num, cap, begin_bit, end_bit, kt, vt, ka, va, cfg, ws)
    assert capi.ws_read_status(ws) == 0
    k, v = (ka, va) if in_alt else (kt, vt)
    return k[:n].cpu().numpy().view(np.uint64), v[:n].cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("n", [0, 1, 31, 4097, 24_593, 1_000_000])
@pytest.mark.parametrize("kind", ["random", "equal", "sorted", "few"])
def test_lookback_matches_stable_sort(n, kind):
    rng = np.random.default_rng(n * 3 + len(kind))
    keys = _keys(kind, n, rng)
    vals = rng.permutation(n).astype(np.uint32)
    k, v = gpu_sort_lookback(keys, vals, digit_bits=8, end_bit=45)
    ek, ev = oracle.sort_pairs(keys, vals)
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)


@pytest.mark.parametrize("bits", [4, 5, 6, 7, 8, 9])
def test_lookback_digit_widths(bits):
    rng = np.random.default_rng(100 + bits)
    keys = rng.integers(0, 2 ** 50, 200_000, dtype=np.uint64)
    vals = np.arange(keys.size, dtype=np.uint32)
    k, v = gpu_sort_lookback(keys, vals, digit_bits=bits, begin_bit=3, end_bit=50)
    perm = np.argsort(keys >> np.uint64(3), kind="stable")
    np.testing.assert_array_equal(k, keys[perm])
    np.testing.assert_array_equal(v, vals[perm])


def test_lookback_stalled_tile_times_out_instead_of_hanging():
    """A predecessor that never publishes makes every later tile's bounded
    wait run out: the call returns, WS_FLAG_TIMEOUT is raised, and the
    context stays usable (a normal sort right after is correct)."""
    import time
    import torch
    from paper_2602_03207_gb300 import capi
    rng = np.random.default_rng(7)
    n = 50_000  # 25 tiles of 2048 keys
    keys = rng.integers(0, 2 ** 40, n, dtype=np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    kt = torch.from_numpy(keys.view(np.int64)).cuda()
    vt = torch.from_numpy(vals.view(np.int32)).cuda()
    ka, va = torch.empty_like(kt), torch.empty_like(vt)
    num = torch.tensor([n, 0, 0, 0], dtype=torch.int32, device="cuda")
    cfg = capi.config(digit_bits=8, flags=capi.WS_CFG_SORT_LOOKBACK)
    ws = torch.zeros(capi.ws_workspace_bytes(0, n, capi.camera(S.small_forward()[1]), cfg),
                     dtype=torch.uint8, device="cuda")
    t0 = time.time()
    capi.ws_sort_test_stalled_tile(num, n, 0, 40, kt, vt, ka, va, cfg, ws, 3)
    flags = capi.ws_read_status(ws)
    assert flags & capi.WS_FLAG_TIMEOUT
    assert time.time() - t0 < 30
    k, v = gpu_sort_lookback(keys, vals, digit_bits=8, end_bit=40)
    ek, ev = oracle.sort_pairs(keys, vals)
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)


# ---------------------------------------------------------------- segmented
SEG = 16  # WS_CFG_SORT_SEGMENTED


def _tile_depth_keys(sizes, rng, depth_levels=None):
    """(tile << 31) | float32 depth bits, tile t holding sizes[t] keys, in a
    shuffled (emission-like) order; depth_levels forces ties."""
    tiles = np.repeat(np.arange(len(sizes), dtype=np.uint64), sizes)
    if depth_levels:
        depth = rng.integers(1, depth_levels + 1, tiles.size).astype(np.float32)
    else:
        depth = rng.uniform(0.2, 80.0, tiles.size).astype(np.float32)
    keys = (tiles << np.uint64(31)) | depth.view(np.uint32).astype(np.uint64)
    perm = rng.permutation(keys.size)
    return keys[perm], perm.astype(np.uint32)


@pytest.mark.parametrize("ties", [None, 3])
def test_segmented_sort_all_segment_paths(ties):
    """Segment sizes around every path boundary of the segmented sort: one
    warp (<= 256 keys), the block in shared memory (<= 2048) and the block
    through global memory (> 2048), plus empty and one-key segments."""
    sizes = [0, 1, 2, 31, 32, 33, 255, 256, 257, 0, 0, 1000, 2047, 2048, 2049, 5000, 1, 70_000, 3, 0, 300]
    sizes += [int(x) for x in np.random.default_rng(11).integers(0, 400, 1500)]
    rng = np.random.default_rng(12 if ties else 13)
    keys, vals = _tile_depth_keys(sizes, rng, ties)
    end = 31 + int(np.ceil(np.log2(len(sizes))))
    k, v = gpu_sort(keys, vals, digit_bits=9, end_bit=end, flags=SEG)
    ek, ev = oracle.sort_pairs(keys, vals)
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)


@pytest.mark.parametrize("n", [0, 1, 31, 4097, 8192 * 3 + 17])
@pytest.mark.parametrize("kind", ["random", "equal", "sorted", "reversed", "few"])
def test_segmented_matches_stable_sort(n, kind):
    """Generic 45-bit keys through the segmented path (capacity large enough
    for its 2^14 segment starts): 'equal' and 'few' put all keys in one or
    four segments (the global-memory path)."""
    rng = np.random.default_rng(n * 5 + len(kind))
    keys = _keys(kind, n, rng)
    vals = rng.permutation(n).astype(np.uint32)
    k, v = gpu_sort(keys, vals, digit_bits=8, end_bit=45, capacity=1 << 16, flags=SEG)
    ek, ev = oracle.sort_pairs(keys, vals)
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)


def test_segmented_begin_bit_and_small_capacity_fallback():
    """begin_bit > 0 (low bits keep input order), and a capacity too small
    for the segment starts (ws_sort then runs the full-key passes): both
    equal the stable sort of the selected bits."""
    rng = np.random.default_rng(21)
    keys = rng.integers(0, 2 ** 44, 60_000, dtype=np.uint64)
    vals = np.arange(keys.size, dtype=np.uint32)
    perm = np.argsort(keys >> np.uint64(5), kind="stable")
    k, v = gpu_sort(keys, vals, begin_bit=5, end_bit=44, flags=SEG)
    np.testing.assert_array_equal(k, keys[perm])
    np.testing.assert_array_equal(v, vals[perm])
    small = keys[:300] & np.uint64((1 << 44) - 1)
    k, v = gpu_sort(small, vals[:300], end_bit=44, flags=SEG)
    ek, ev = oracle.sort_pairs(small, vals[:300])
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)


def test_segmented_sort_of_standard_keys():
    """The 4,194,304 (tile, depth) keys of the sort benchmark."""
    keys, vals = S.sort_keys()
    k, v = gpu_sort(keys, vals, digit_bits=9, end_bit=44, flags=SEG)
    ek, ev = oracle.sort_pairs(keys, vals)
    np.testing.assert_array_equal(k, ek)
    np.testing.assert_array_equal(v, ev)


@pytest.mark.parametrize("flags", [0, SEG, 4], ids=["lsd", "segmented", "lookback"])
def test_count_above_capacity_is_clamped(flags):
    """A device-side count larger than key_capacity is clamped to it: the
    first key_capacity pairs come out sorted, and nothing past key_capacity
    in the four key/value buffers, nor past the workspace, is written."""
    import torch
    from paper_2602_03207_gb300 import capi
    assert flags != 4 or capi.WS_CFG_SORT_LOOKBACK == 4
    rng = np.random.default_rng(31 + flags)
    cap, guard = 20_000, 4096
    keys, vals = _tile_depth_keys([int(x) for x in rng.integers(24, 40, 1024)], rng)
    keys, vals = keys[:cap + guard], vals[:cap + guard]
    assert keys.size == cap + guard
    kt = torch.from_numpy(keys.view(np.int64)).cuda()
    vt = torch.from_numpy(vals.view(np.int32)).cuda()
    ka = torch.full_like(kt, -5)
    va = torch.full_like(vt, -7)
    before = [t.clone() for t in (kt, vt, ka, va)]
    num = torch.tensor([cap + 3000, 0, 0, 0], dtype=torch.int32, device="cuda")
    cfg = capi.config(digit_bits=8, flags=flags)
    wsb = capi.ws_workspace_bytes(0, cap, capi.camera(S.small_forward()[1]), cfg)
    ws = torch.full((wsb + 4096,), 0xAB, dtype=torch.uint8, device="cuda")
    in_alt = capi.ws_sort(num, cap, 0, 41, kt, vt, ka, va, cfg, ws)
    torch.cuda.synchronize()
    k, v = (ka, va) if in_alt else (kt, vt)
    ek, ev = oracle.sort_pairs(keys[:cap], vals[:cap])
    np.testing.assert_array_equal(k[:cap].cpu().numpy().view(np.uint64), ek)
    np.testing.assert_array_equal(v[:cap].cpu().numpy().view(np.uint32), ev)
    for t, b in zip((kt, vt, ka, va), before):
        assert torch.equal(t[cap:], b[cap:])
    assert bool((ws[wsb:] == 0xAB).all())


@pytest.mark.parametrize("sizes_seed", [0, 1, 2])
def test_sort_tiles_writes_the_tile_ranges(sizes_seed):
    """ws_sort_tiles: the segmented sort's output (bit-identical to ws_sort)
    plus, for every tile t < ntiles, [start, end) of its keys in the sorted
    list (empty tiles included), equal to a search of the sorted keys."""
    import torch
    from paper_2602_03207_gb300 import capi
    rng = np.random.default_rng(50 + sizes_seed)
    ntiles = [1000, 8160, 3][sizes_seed]
    sizes = [int(x) for x in rng.integers(0, 300, ntiles)]
    if sizes_seed == 2:
        sizes = [0, 0, 0]
    keys, vals = _tile_depth_keys(sizes, rng)
    n = keys.size
    end = 31 + max(1, int(np.ceil(np.log2(ntiles))))
    cap = max(n, 1 << (end - 31) + 1, 4096)
    kt = torch.zeros(cap, dtype=torch.int64, device="cuda")
    vt = torch.zeros(cap, dtype=torch.int32, device="cuda")
    if n:
        kt[:n] = torch.from_numpy(keys.view(np.int64))
        vt[:n] = torch.from_numpy(vals.view(np.int32))
    ka, va = torch.empty_like(kt), torch.empty_like(vt)
    num = torch.tensor([n, 0, 0, 0], dtype=torch.int32, device="cuda")
    cfg = capi.config(digit_bits=9, flags=SEG)
    ws = torch.zeros(capi.ws_workspace_bytes(0, cap, capi.camera(S.small_forward()[1]), cfg), dtype=torch.uint8,
                     device="cuda")
    ranges = torch.full((ntiles, 2), -1, dtype=torch.int32, device="cuda")
    alt = capi.ws_sort_tiles(num, cap, end, kt, vt, ka, va, cfg, ws, ranges, ntiles)
    torch.cuda.synchronize()
    k, v = (ka, va) if alt else (kt, vt)
    ek, ev = oracle.sort_pairs(keys, vals)
    np.testing.assert_array_equal(k[:n].cpu().numpy().view(np.uint64), ek)
    np.testing.assert_array_equal(v[:n].cpu().numpy().view(np.uint32), ev)
    tiles = (ek >> np.uint64(31)).astype(np.int64)
    t = np.arange(ntiles)
    expect = np.stack([np.searchsorted(tiles, t, side="left"), np.searchsorted(tiles, t, side="right")], axis=1)
    np.testing.assert_array_equal(ranges.cpu().numpy(), expect)


def test_sort_tiles_rejects_what_the_segmented_sort_cannot_take():
    """A single-tile key range (end_bit 31) is not segmented: WS_ERR_UNSUPPORTED."""
    import torch
    from paper_2602_03207_gb300 import capi
    num = torch.zeros(4, dtype=torch.int32, device="cuda")
    k = torch.zeros(16, dtype=torch.int64, device="cuda")
    v = torch.zeros(16, dtype=torch.int32, device="cuda")
    ranges = torch.zeros((1, 2), dtype=torch.int32, device="cuda")
    cfg = capi.config(digit_bits=8, flags=SEG)
    ws = torch.zeros(capi.ws_workspace_bytes(0, 16, capi.camera(S.small_forward()[1]), cfg), dtype=torch.uint8,
                     device="cuda")
    with pytest.raises(capi.WsError) as e:
        capi.ws_sort_tiles(num, 16, 31, k, v, k, v, cfg, ws, ranges, 1)
    assert e.value.status == capi.WS_ERR_UNSUPPORTED
