"""The allocation-free entry point against the oracle and the regular matcher.

cashash_match_pair_noalloc serves callers that cannot allocate device memory
when they match: a real-time loop that must not allocate (or implicitly
synchronise) after start-up, or a host whose device memory belongs to its own
pool.  Its scratch is a fixed array inside the library.  Its match lists must
be the oracle's for the same pair, and identical to cashash_match_pairs;
two calls in a row check that the shared scratch is cleared between calls,
and cashash_noalloc_status reports the device errors of the calls.  This
file is collected last on purpose.
"""
import math

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


def _regular(ch, ctx, ds, a, b, cap, F=None):
    moff = torch.zeros(2, dtype=torch.int64, device="cuda")
    mt = torch.zeros((max(cap, 1), 2), dtype=torch.int32, device="cuda")
    ch.cashash_match_pairs(ctx, ds, np.array([[a, b]], np.uint32), moff, mt, cap, F=F)
    assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK
    n = int(moff[1].item())
    return n, mt[:n].cpu().numpy().view(np.uint32)


def _oracle(orc, s, po, codes, buckets, a, b, F=None):
    A = slice(int(s.img_off[a]), int(s.img_off[a + 1]))
    B = slice(int(s.img_off[b]), int(s.img_off[b + 1]))
    kw = {}
    if F is not None:
        kw = dict(F=F, kptsA=s.kpts[A], kptsB=s.kpts[B])
    m = orc.match_pair(s.desc[A], codes[A], buckets[A], s.desc[B], codes[B], buckets[B], po, **kw)
    q = np.nonzero(m >= 0)[0]
    return np.stack([q, m[q]], axis=1).astype(np.uint32) if q.size else np.zeros((0, 2), np.uint32)


def _noalloc_twice(ch, p, ds, a, b, cap, F=None):
    """Two calls in a row into outputs poisoned before each; both lists are returned."""
    outs = []
    for _ in range(2):
        moff = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        mt = torch.full((max(cap, 1), 2), -1, dtype=torch.int32, device="cuda")
        ch.cashash_match_pair_noalloc(p, ds, a, b, moff, mt, cap, F=F)
        torch.cuda.synchronize()
        off = moff.cpu().numpy()
        assert off[0] == 0
        n = int(off[1])
        outs.append(mt[:n].cpu().numpy().view(np.uint32))
    return outs


@pytest.mark.parametrize("flags", [0, 2])
def test_noalloc_matches_oracle_and_regular_entry_point_twice_in_a_row(ch, orc, flags):
    sizes = [3000, 5200, 0, 9000, 700]
    s = synth.random_set(909, sizes)
    p = ch.cashash_default_params(flags=flags)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    torch.cuda.synchronize()
    po = orc.params(flags=flags)
    codes, buckets = ds.codes_np(), ds.buckets_np(6)
    ec, eb = orc.hash_codes(s.desc, orc.mean(s.desc), s.R, po)
    assert np.array_equal(codes, ec) and np.array_equal(buckets, eb)
    cap = max(sizes)
    assert ch.cashash_noalloc_status() == ch.CASHASH_OK  # clears what earlier tests left
    for (a, b) in [(0, 1), (0, 1), (3, 1), (1, 3), (4, 0), (2, 1), (1, 2)]:
        exp = _oracle(orc, s, po, codes, buckets, a, b)
        n_ref, ref = _regular(ch, ctx, ds, a, b, cap)
        assert np.array_equal(ref, exp)
        for got in _noalloc_twice(ch, p, ds, a, b, cap):
            assert np.array_equal(got, exp), "pair (%d, %d)" % (a, b)
    assert ch.cashash_noalloc_status() == ch.CASHASH_OK
    ctx.close()


@pytest.mark.parametrize("flags", [0, 2])
def test_noalloc_epipolar_band(ch, orc, flags):
    """Sec. 7.2 band (4 px) with a device F per call, compared with the
    oracle and with cashash_match_pairs on the same pairs, both directions."""
    s = synth.epipolar_set(41, n_views=7, n_points=24000, arc=2 * math.pi * 7 / 250, z_max=0.355)
    p = ch.cashash_default_params(epi_px=4.0, flags=flags)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc, s.kpts)
    ch.cashash_build_codes(ctx, ds)
    torch.cuda.synchronize()
    po = orc.params(epi_px=4.0, flags=flags)
    codes, buckets = ds.codes_np(), ds.buckets_np(6)
    cap = int(s.sizes().max())
    total = 0
    for i in range(min(4, len(s.pairs))):
        a, b = (int(x) for x in s.pairs[i])
        for (qa, qb, Fi) in [(a, b, s.F[i]), (b, a, s.F[i].reshape(3, 3).T.ravel())]:
            F_dev = torch.from_numpy(np.ascontiguousarray(Fi)).cuda()
            exp = _oracle(orc, s, po, codes, buckets, qa, qb, F=Fi)
            total += len(exp)
            n_ref, ref = _regular(ch, ctx, ds, qa, qb, cap, F=F_dev)
            assert np.array_equal(ref, exp)
            for got in _noalloc_twice(ch, p, ds, qa, qb, cap, F=F_dev):
                assert np.array_equal(got, exp), "pair (%d, %d)" % (qa, qb)
    assert total > 0
    assert ch.cashash_noalloc_status() == ch.CASHASH_OK
    ctx.close()


def test_noalloc_truncates_reports_and_rejects(ch, orc):
    s = synth.random_set(910, [2000, 2500])
    p = ch.cashash_default_params()
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    n_ref, ref = _regular(ch, ctx, ds, 0, 1, 2000)
    assert n_ref > 20
    assert ch.cashash_noalloc_status() == ch.CASHASH_OK
    moff = torch.zeros(2, dtype=torch.int64, device="cuda")
    mt = torch.full((20, 2), -3, dtype=torch.int32, device="cuda")
    ch.cashash_match_pair_noalloc(p, ds, 0, 1, moff, mt, 10)
    torch.cuda.synchronize()
    assert int(moff[1].item()) == n_ref
    got = mt.cpu().numpy()
    assert np.array_equal(got[:10].view(np.uint32), ref[:10]) and (got[10:] == -3).all()
    assert ch.cashash_noalloc_status() == ch.CASHASH_EOVERFLOW
    assert ch.cashash_noalloc_status() == ch.CASHASH_OK  # read and cleared
    with pytest.raises(ch.CashashError) as e:
        ch.cashash_match_pair_noalloc(p, ds, 0, 2, moff, mt, 10)
    assert e.value.status == ch.CASHASH_EINVAL
    pm = ch.cashash_default_params(flags=1)
    with pytest.raises(ch.CashashError) as e:
        ch.cashash_match_pair_noalloc(pm, ds, 0, 1, moff, mt, 10)
    assert e.value.status == ch.CASHASH_ENOTSUP
    pb = ch.cashash_default_params(epi_px=4.0)
    with pytest.raises(ch.CashashError) as e:  # the band needs F and key-points
        ch.cashash_match_pair_noalloc(pb, ds, 0, 1, moff, mt, 10)
    assert e.value.status == ch.CASHASH_EINVAL
    big = ch.CASHASH_NOALLOC_MAX_QUERIES
    s2 = synth.random_set(911, [big + 1, 10])
    ds2 = ch.DeviceSet(p, s2.img_off, s2.desc)
    ch.cashash_build_codes(ctx, ds2)
    with pytest.raises(ch.CashashError) as e:
        ch.cashash_match_pair_noalloc(p, ds2, 0, 1, moff, mt, 10)
    assert e.value.status == ch.CASHASH_EINVAL
    # the oversized query image is still accepted as the candidate side
    ch.cashash_match_pair_noalloc(p, ds2, 1, 0, moff, mt, 10)
    torch.cuda.synchronize()
    assert ch.cashash_noalloc_status() in (ch.CASHASH_OK, ch.CASHASH_EOVERFLOW)
    ctx.close()
