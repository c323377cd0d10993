"""The allocation-free entry point agrees with the regular matcher.

cashash_match_pair_noalloc serves callers that cannot allocate device memory
when they match (its scratch is a fixed array inside the library).  Its
match lists must be identical to those of cashash_match_pairs for the same
pair; two calls in a row check that the shared scratch is cleared between
calls.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1805_08995_gb300 as m
    torch.cuda.set_device(0)
    return m


def _regular(ch, ctx, ds, a, b, cap):
    moff = torch.zeros(2, dtype=torch.int64, device="cuda")
    mt = torch.zeros((max(cap, 1), 2), dtype=torch.int32, device="cuda")
    ch.cashash_match_pairs(ctx, ds, np.array([[a, b]], np.uint32), moff, mt, cap)
    assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK
    n = int(moff[1].item())
    return n, mt[:n].cpu().numpy()


def test_noalloc_matches_regular_entry_point_twice_in_a_row(ch):
    sizes = [3000, 5200, 0, 9000, 700]
    s = synth.random_set(909, sizes)
    p = ch.cashash_default_params()
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    torch.cuda.synchronize()
    cap = max(sizes)
    for (a, b) in [(0, 1), (0, 1), (3, 1), (1, 3), (4, 0), (2, 1), (1, 2)]:
        n_ref, ref = _regular(ch, ctx, ds, a, b, cap)
        moff = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        mt = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
        for _ in range(2):
            ch.cashash_match_pair_noalloc(p, ds, a, b, moff, mt, cap)
            torch.cuda.synchronize()
            off = moff.cpu().numpy()
            assert off[0] == 0 and off[1] == n_ref
            assert np.array_equal(mt[:n_ref].cpu().numpy(), ref)
    ctx.close()


def test_noalloc_truncates_and_rejects_oversized_queries(ch):
    s = synth.random_set(910, [2000, 2500])
    p = ch.cashash_default_params()
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    n_ref, ref = _regular(ch, ctx, ds, 0, 1, 2000)
    assert n_ref > 20
    moff = torch.zeros(2, dtype=torch.int64, device="cuda")
    mt = torch.full((20, 2), -3, dtype=torch.int32, device="cuda")
    ch.cashash_match_pair_noalloc(p, ds, 0, 1, moff, mt, 10)
    torch.cuda.synchronize()
    assert int(moff[1].item()) == n_ref
    got = mt.cpu().numpy()
    assert np.array_equal(got[:10], ref[:10]) and (got[10:] == -3).all()
    with pytest.raises(ch.CashashError) as e:
        ch.cashash_match_pair_noalloc(p, ds, 0, 2, moff, mt, 10)
    assert e.value.status == ch.CASHASH_EINVAL
    big = ch.CASHASH_NOALLOC_MAX_QUERIES if hasattr(ch, "CASHASH_NOALLOC_MAX_QUERIES") else 65536
    s2 = synth.random_set(911, [big + 1, 10])
    ds2 = ch.DeviceSet(p, s2.img_off, s2.desc)
    ch.cashash_build_codes(ctx, ds2)
    with pytest.raises(ch.CashashError) as e:
        ch.cashash_match_pair_noalloc(p, ds2, 0, 1, moff, mt, 10)
    assert e.value.status == ch.CASHASH_EINVAL
    ctx.close()
