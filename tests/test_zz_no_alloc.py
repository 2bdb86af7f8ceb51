"""ws_sort_noalloc: the sort for callers that cannot allocate device
memory (an engine that owns every device allocation and hands over only
its buffers, or a frame loop that must not call cudaMalloc). It keeps its
histogram scratch in a static device array inside the library. Checked
through the C ABI against ws_sort (the workspace version) on two calls in a
row with different data, so stale scratch from the first call would show.
Integer work: the results must be identical."""
import numpy as np
import pytest

from paper_2602_03207_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def _buffers(keys, vals, cap):
    import torch
    n = keys.size
    kt = torch.zeros(cap, dtype=torch.int64, device="cuda")
    vt = torch.zeros(cap, dtype=torch.int32, device="cuda")
    kt[:n] = torch.from_numpy(keys.view(np.int64))
    vt[:n] = torch.from_numpy(vals.view(np.int32))
    num = torch.tensor([n, 0, 0, 0], dtype=torch.int32, device="cuda")
    return kt, vt, torch.empty_like(kt), torch.empty_like(vt), num


def _with_workspace(keys, vals, end_bit, bits):
    import torch
    from paper_2602_03207_gb300 import capi
    cap = keys.size
    kt, vt, ka, va, num = _buffers(keys, vals, cap)
    cfg = capi.config(digit_bits=bits)
    ws = torch.zeros(capi.ws_workspace_bytes(0, cap, capi.camera(S.small_forward()[1]), cfg),
                     dtype=torch.uint8, device="cuda")
    alt = capi.ws_sort(num, cap, 0, end_bit, kt, vt, ka, va, cfg, ws)
    torch.cuda.synchronize()
    k, v = (ka, va) if alt else (kt, vt)
    return k.cpu().numpy(), v.cpu().numpy()


def _no_alloc(keys, vals, end_bit, bits):
    import torch
    from paper_2602_03207_gb300 import capi
    cap = keys.size
    kt, vt, ka, va, num = _buffers(keys, vals, cap)
    alt = capi.ws_sort_noalloc(num, cap, 0, end_bit, kt, vt, ka, va, digit_bits=bits)
    torch.cuda.synchronize()
    k, v = (ka, va) if alt else (kt, vt)
    return k.cpu().numpy(), v.cpu().numpy()


def test_no_alloc_sort_matches_workspace_sort_twice():
    rng = np.random.default_rng(2024)
    cases = [(rng.integers(0, 2 ** 44, 1_000_003, dtype=np.uint64), 44, 8),
             (rng.integers(0, 2 ** 40, 300_001, dtype=np.uint64), 40, 6)]
    for keys, end_bit, bits in cases:  # two calls in a row, different sizes and digits
        vals = rng.permutation(keys.size).astype(np.uint32)
        ek, ev = _with_workspace(keys, vals, end_bit, bits)
        gk, gv = _no_alloc(keys, vals, end_bit, bits)
        np.testing.assert_array_equal(gk, ek)
        np.testing.assert_array_equal(gv, ev)


def test_no_alloc_rejects_oversize_capacity():
    import torch
    from paper_2602_03207_gb300 import capi
    cap = capi.ws_sort_noalloc_max_keys()
    assert cap == 8_388_608
    num = torch.zeros(4, dtype=torch.int32, device="cuda")
    k = torch.zeros(4, dtype=torch.int64, device="cuda")
    v = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(capi.WsError) as e:
        capi.ws_sort_noalloc(num, cap + 1, 0, 40, k, v, k, v)
    assert e.value.status == capi.WS_ERR_INVALID_ARG


def test_no_alloc_at_the_maximum_capacity():
    """key_capacity equal to ws_sort_noalloc_max_keys() with 8-bit digits:
    the histogram matrix and the digit totals then fill the whole static
    array. A count just below the capacity sorts like ws_sort."""
    import torch
    from paper_2602_03207_gb300 import capi
    cap = capi.ws_sort_noalloc_max_keys()
    n = cap - 1234
    rng = np.random.default_rng(77)
    keys = rng.integers(0, 2 ** 44, n, dtype=np.uint64)
    vals = rng.permutation(n).astype(np.uint32)
    ek, ev = _with_workspace(keys, vals, 44, 8)
    kt, vt, ka, va, num = _buffers(keys, vals, cap)
    alt = capi.ws_sort_noalloc(num, cap, 0, 44, kt, vt, ka, va, digit_bits=8)
    torch.cuda.synchronize()
    k, v = (ka, va) if alt else (kt, vt)
    np.testing.assert_array_equal(k[:n].cpu().numpy(), ek)
    np.testing.assert_array_equal(v[:n].cpu().numpy(), ev)


def test_no_alloc_count_above_capacity_is_clamped():
    """A device-side count above key_capacity sorts the first key_capacity
    pairs and writes nothing past them."""
    import torch
    from paper_2602_03207_gb300 import capi
    rng = np.random.default_rng(78)
    cap, extra = 50_000, 4096
    keys = rng.integers(0, 2 ** 40, cap + extra, dtype=np.uint64)
    vals = np.arange(cap + extra, dtype=np.uint32)
    kt = torch.from_numpy(keys.view(np.int64)).cuda()
    vt = torch.from_numpy(vals.view(np.int32)).cuda()
    ka, va = torch.full_like(kt, -1), torch.full_like(vt, -1)
    before = [t.clone() for t in (kt, vt, ka, va)]
    num = torch.tensor([cap + extra, 0, 0, 0], dtype=torch.int32, device="cuda")
    alt = capi.ws_sort_noalloc(num, cap, 0, 40, kt, vt, ka, va, digit_bits=8)
    torch.cuda.synchronize()
    k, v = (ka, va) if alt else (kt, vt)
    perm = np.argsort(keys[:cap], kind="stable")
    np.testing.assert_array_equal(k[:cap].cpu().numpy().view(np.uint64), keys[:cap][perm])
    np.testing.assert_array_equal(v[:cap].cpu().numpy().view(np.uint32), vals[:cap][perm])
    for t, b in zip((kt, vt, ka, va), before):
        assert torch.equal(t[cap:], b[cap:])


def test_no_alloc_rejects_unsupported_digit_width():
    """Digit widths outside 4..8 return WS_ERR_UNSUPPORTED before any launch."""
    import torch
    from paper_2602_03207_gb300 import capi
    num = torch.zeros(4, dtype=torch.int32, device="cuda")
    k = torch.zeros(4, dtype=torch.int64, device="cuda")
    v = torch.zeros(4, dtype=torch.int32, device="cuda")
    for bits in (3, 9, 11):
        with pytest.raises(capi.WsError) as e:
            capi.ws_sort_noalloc(num, 4, 0, 40, k, v, k, v, digit_bits=bits)
        assert e.value.status == capi.WS_ERR_UNSUPPORTED
