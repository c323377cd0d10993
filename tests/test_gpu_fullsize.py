"""Full-size workloads in the launch configuration bench.py times.

The oracle cannot re-match every pair at these sizes in seconds, so:
  * hash codes and bucket ids are compared for every feature (config 1) or
    for every feature of the sampled images (config 3);
  * the match lists of a random sample of pairs are compared entry for entry;
  * every pair's list is checked for properties that hold at any size.
"""
import threading

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


def _oracle_codes(orc, desc, R, po, mu, threads=16):
    n = desc.shape[0]
    codes = np.zeros((n, 4), np.uint32)
    buckets = np.zeros((n, po.n_tables), np.uint8)
    step = max(1, (n + threads - 1) // threads)

    def work(s):
        codes[s:s + step], buckets[s:s + step] = orc.hash_codes(desc[s:s + step], mu, R, po)

    ts = [threading.Thread(target=work, args=(s,)) for s in range(0, n, step)]
    [t.start() for t in ts]
    [t.join() for t in ts]
    return codes, buckets


def _run_gpu(ch, s, precision=0, repeats=2, **pk):
    p = ch.cashash_default_params(precision=precision, schedule=ch.CASHASH_SCHED_PERSISTENT, **pk)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc, s.kpts if "epi_px" in pk else None)
    plan = ch.cashash_plan_create(ctx, ds, s.pairs)
    F = torch.from_numpy(np.ascontiguousarray(s.F)).cuda() if "epi_px" in pk else None
    P = len(s.pairs)
    cap = int(s.sizes()[s.pairs[:, 0]].sum())
    moff = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
    mt = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
    outs = []
    for _ in range(repeats):  # the second pass replays the captured graph with learned thresholds
        ch.cashash_build_codes(ctx, ds)
        ch.cashash_match_plan(ctx, plan, moff, mt, cap, F=F)
        assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK
        off = moff.cpu().numpy().astype(np.uint64)
        outs.append((off, mt[:int(off[-1])].cpu().numpy().view(np.uint32).copy()))
    stats = ch.cashash_get_stats(ctx)
    mu = ch.cashash_get_mean(ctx)
    return ctx, ds, plan, outs, stats, mu


def _properties(s, off, mt):
    sizes = s.sizes()
    assert off[0] == 0 and np.all(np.diff(off.astype(np.int64)) >= 0)
    for i, (a, b) in enumerate(s.pairs):
        seg = mt[int(off[i]):int(off[i + 1])]
        if len(seg):
            assert seg[:, 0].max() < sizes[a] and seg[:, 1].max() < sizes[b]
            assert np.all(np.diff(seg[:, 0].astype(np.int64)) > 0)   # strictly ascending queries


def _sample_check(orc, s, off, mt, codes_of, mu, n_sample, seed, po=None):
    po = po or orc.params()
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(len(s.pairs), size=min(n_sample, len(s.pairs)), replace=False))
    for i in pick:
        a, b = (int(x) for x in s.pairs[i])
        A = slice(int(s.img_off[a]), int(s.img_off[a + 1]))
        B = slice(int(s.img_off[b]), int(s.img_off[b + 1]))
        cA, bA = codes_of(a)
        cB, bB = codes_of(b)
        kw = {}
        if s.F is not None:
            kw = dict(F=s.F[i], kptsA=s.kpts[A], kptsB=s.kpts[B])
        m = orc.match_pair(s.desc[A], cA, bA, s.desc[B], cB, bB, po, **kw)
        q = np.nonzero(m >= 0)[0]
        exp = np.stack([q, m[q]], axis=1).astype(np.uint32) if q.size else np.zeros((0, 2), np.uint32)
        assert np.array_equal(mt[int(off[i]):int(off[i + 1])], exp), "pair %d (%d, %d)" % (i, a, b)


@pytest.mark.parametrize("precision", [0, 1])
def test_config1_full_size(ch, orc, precision):
    """precision 0: config 1 (plain FP32 form); 1: config 2 (BF16 tensor-core
    projection with exact re-evaluation under its rounding bound)."""
    s = synth.config1()
    ctx, ds, plan, outs, stats, mu = _run_gpu(ch, s, precision=precision)
    po = orc.params()
    assert np.array_equal(mu, orc.mean(s.desc))
    codes, buckets = _oracle_codes(orc, s.desc, s.R, po, mu)
    assert np.array_equal(ds.codes_np(), codes)
    assert np.array_equal(ds.buckets_np(6), buckets)
    (off1, mt1), (off2, mt2) = outs
    assert np.array_equal(off1, off2) and np.array_equal(mt1, mt2)
    _properties(s, off2, mt2)

    def codes_of(i):
        a, b = int(s.img_off[i]), int(s.img_off[i + 1])
        return codes[a:b], buckets[a:b]

    _sample_check(orc, s, off2, mt2, codes_of, mu, 40, 5)
    plan.close()
    ctx.close()


def test_config3_full_size(ch, orc):
    s = synth.config3()
    ctx, ds, plan, outs, stats, mu = _run_gpu(ch, s, precision=1)
    po = orc.params()
    assert np.array_equal(mu, orc.mean(s.desc))
    (off1, mt1), (off2, mt2) = outs
    assert np.array_equal(off1, off2) and np.array_equal(mt1, mt2)
    _properties(s, off2, mt2)
    gcodes, gbuckets = ds.codes_np(), ds.buckets_np(6)
    cache = {}

    def codes_of(i):
        if i not in cache:
            a, b = int(s.img_off[i]), int(s.img_off[i + 1])
            c, bk = orc.hash_codes(s.desc[a:b], mu, s.R, po)
            assert np.array_equal(gcodes[a:b], c) and np.array_equal(gbuckets[a:b], bk)
            cache[i] = (c, bk)
        return cache[i]

    _sample_check(orc, s, off2, mt2, codes_of, mu, 24, 6)
    plan.close()
    ctx.close()


def test_config4_full_size(ch, orc):
    """Config 4 (Sec. 6.2 band, 4 px): 500 views, 14,613 pairs, the batched
    join with its band test as bench.py runs it; sampled images' codes and 24
    sampled pairs entry for entry, every pair's list checked for properties."""
    s = synth.config4()
    ctx, ds, plan, outs, stats, mu = _run_gpu(ch, s, precision=1, epi_px=4.0)
    assert ch.cashash_plan_get_tuning(plan)["kernel"] == ch.CASHASH_KERNEL_JOIN
    po = orc.params(epi_px=4.0)
    assert np.array_equal(mu, orc.mean(s.desc))
    (off1, mt1), (off2, mt2) = outs
    assert np.array_equal(off1, off2) and np.array_equal(mt1, mt2)
    _properties(s, off2, mt2)
    gcodes, gbuckets = ds.codes_np(), ds.buckets_np(6)
    cache = {}

    def codes_of(i):
        if i not in cache:
            a, b = int(s.img_off[i]), int(s.img_off[i + 1])
            c, bk = orc.hash_codes(s.desc[a:b], mu, s.R, po)
            assert np.array_equal(gcodes[a:b], c) and np.array_equal(gbuckets[a:b], bk)
            cache[i] = (c, bk)
        return cache[i]

    _sample_check(orc, s, off2, mt2, codes_of, mu, 24, 7, po=po)
    plan.close()
    ctx.close()


def test_config4_ga_stage1_full_size(ch):
    """Ga-CasHash first stage on config 4 as bench.py --ga runs it (all 14,613
    pairs, BF16 codes, per-query subset matching); 24 sampled pairs are redone
    by the oracle on the images they touch (selection, subset codes with the
    full set's centre, CasHash, RANSAC with the same words): selection, counts,
    the winning hypothesis and acceptance identical, F within 1e-8."""
    import oracle as orc
    from oracle import ga as oga
    orc.build()
    s = synth.config4()
    bf = dict(precision=ch.CASHASH_BF16, schedule=ch.CASHASH_SCHED_PERSISTENT)
    p1, p2 = ch.cashash_default_params(**bf), ch.cashash_default_params(epi_px=4.0, **bf)
    ctx1, ctx2 = ch.cashash_create(p1, s.R), ch.cashash_create(p2, s.R)
    ds = ch.DeviceSet(p2, s.img_off, s.desc, s.kpts)
    ch.cashash_build_codes(ctx2, ds)
    mu = ch.cashash_get_mean(ctx2)
    assert np.array_equal(mu, orc.mean(s.desc))
    gp = ch.cashash_ga_default_params()
    words = synth.ransac_words(4, len(s.pairs), gp.n_hyp)
    F, info = ch.cashash_ga_stage1(ctx1, ds, torch.from_numpy(s.scale).cuda(), mu, s.pairs,
                                   torch.from_numpy(words.view(np.int32)).cuda(), gp)
    torch.cuda.synchronize()
    F = F.cpu().numpy()
    info = info.cpu().numpy().view(np.uint32)
    assert info[:, 3].sum() > 0.9 * len(s.pairs)
    sel, sub = ch.cashash_ga_select(torch.from_numpy(s.scale).cuda(), s.img_off, gp.top_pct)
    esel, esub = oga.top_scale(s.scale, s.img_off, gp.top_pct)
    assert np.array_equal(sub, esub) and np.array_equal(sel.cpu().numpy().view(np.uint32).astype(np.uint64), esel)
    pick = np.sort(np.random.default_rng(11).choice(len(s.pairs), 24, replace=False))
    imgs = np.unique(s.pairs[pick])
    remap = {int(i): k for k, i in enumerate(imgs)}
    rows = np.concatenate([np.arange(int(s.img_off[i]), int(s.img_off[i + 1])) for i in imgs])
    off = np.zeros(len(imgs) + 1, np.uint64)
    off[1:] = np.cumsum(s.sizes()[imgs])
    pr = np.array([[remap[int(a)], remap[int(b)]] for a, b in s.pairs[pick]], np.uint32)
    ogp = oga.GaParams(top_pct=gp.top_pct, min_matches=gp.min_matches, n_hyp=gp.n_hyp,
                       inlier_num=gp.inlier_num, inlier_den=gp.inlier_den, thresh_px=gp.thresh_px,
                       confidence=gp.confidence)
    eF, einfo, *_ = oga.stage1(s.desc[rows], off, s.kpts[rows], s.scale[rows], mu, s.R, pr, orc.params(), ogp,
                               words[pick])
    assert np.array_equal(info[pick], einfo)
    assert np.abs(F[pick] - eF).max() <= 1e-8
    ctx1.close()
    ctx2.close()
