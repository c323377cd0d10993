"""Full-size workloads in the launch configuration bench.py times.

Every list is compared with the oracle entry for entry:
  * configs 1 and 2 (the same 100-image set, FP32 and BF16 projection): all
    4,950 pairs, and every feature's code and bucket ids;
  * config 4 (epipolar band, 500 views): all 14,613 pairs and every code;
  * config 3 (2,000 images, 59,556 pairs): every code and one pair in ten,
    taken evenly along the N_A * N_B cost order (so small, median and large
    pairs, and the persistent kernel's tail, are all represented);
every pair's list is also checked for properties that hold at any size.
The oracle runs on all host cores; its results for one workload are cached
across the tests that share it.
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


_CACHE = {}


def _oracle_all(orc, key, s, po, pairs=None):
    """Oracle centre, codes of every feature, and the lists of `pairs` (all
    of the workload's pairs by default), cached under `key`."""
    if key not in _CACHE:
        mu = orc.mean(s.desc)
        codes, buckets = _oracle_codes(orc, s.desc, s.R, po, mu)
        pr = s.pairs if pairs is None else pairs
        kw = dict(F=s.F, kpts=s.kpts) if s.F is not None else {}
        if s.F is not None and pairs is not None:
            raise ValueError("a pair subset of a band workload needs its F rows")
        cap = int(s.sizes()[pr[:, 0]].sum())
        eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pr, po, n_threads=0, cap=cap, **kw)
        _CACHE[key] = (mu, codes, buckets, eoff, emt)
    return _CACHE[key]


def _lists_of(off, mt, idx):
    """The lists of pairs idx (ascending) of a full result, re-based."""
    segs = [mt[int(off[i]):int(off[i + 1])] for i in idx]
    sub_off = np.zeros(len(idx) + 1, np.uint64)
    sub_off[1:] = np.cumsum([len(x) for x in segs])
    cat = np.concatenate(segs) if segs else np.zeros((0, 2), np.uint32)
    return sub_off, cat.reshape(-1, 2)


def _first_mismatch(off, mt, eoff, emt):
    for i in range(len(off) - 1):
        a = mt[int(off[i]):int(off[i + 1])]
        b = emt[int(eoff[i]):int(eoff[i + 1])]
        if not np.array_equal(a, b):
            return i
    return None


def _run_gpu(ch, s, precision=0, repeats=2, tuning=None, **pk):
    p = ch.cashash_default_params(precision=precision, schedule=ch.CASHASH_SCHED_PERSISTENT, **pk)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc, s.kpts if "epi_px" in pk else None)
    plan = ch.cashash_plan_create(ctx, ds, s.pairs)
    if tuning is not None:
        ch.cashash_plan_set_tuning(plan, *tuning)
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


@pytest.mark.parametrize("precision", [0, 1])
def test_config1_full_size(ch, orc, precision):
    """precision 0: config 1 (plain FP32 form); 1: config 2 (BF16 tensor-core
    projection with exact re-evaluation under its rounding bound).  All 4,950
    pairs entry for entry."""
    s = synth.config1()
    ctx, ds, plan, outs, stats, mu = _run_gpu(ch, s, precision=precision)
    po = orc.params()
    emu, codes, buckets, eoff, emt = _oracle_all(orc, "config1", s, po)
    assert np.array_equal(mu, emu)
    assert np.array_equal(ds.codes_np(), codes)
    assert np.array_equal(ds.buckets_np(6), buckets)
    (off1, mt1), (off2, mt2) = outs
    assert np.array_equal(off1, off2) and np.array_equal(mt1, mt2)
    _properties(s, off2, mt2)
    assert np.array_equal(off2, eoff), "pair %s" % _first_mismatch(off2, mt2, eoff, emt)
    assert np.array_equal(mt2, emt), "pair %s" % _first_mismatch(off2, mt2, eoff, emt)
    assert len(emt) > 100_000
    plan.close()
    ctx.close()


@pytest.mark.parametrize("kernel", ["query", "join"])
def test_config3_full_size(ch, orc, kernel):
    """Config 3 (BF16, batched): every code, and one pair in ten along the
    N_A * N_B cost order entry for entry, with the per-query kernel of 512
    queries per CTA (the autotuner's choice on this workload, as bench.py
    runs it) and with the bucket join."""
    s = synth.config3()
    tuning = (ch.CASHASH_KERNEL_QUERY, 512, 0) if kernel == "query" else (ch.CASHASH_KERNEL_JOIN, 4, 0)
    ctx, ds, plan, outs, stats, mu = _run_gpu(ch, s, precision=1, tuning=tuning)
    assert ch.cashash_plan_get_tuning(plan)["kernel"] == tuning[0]
    po = orc.params()
    sizes = s.sizes()
    cost = sizes[s.pairs[:, 0]].astype(np.int64) * sizes[s.pairs[:, 1]]
    order = np.argsort(cost, kind="stable")
    pick = np.sort(order[::10])
    emu, codes, buckets, eoff, emt = _oracle_all(orc, "config3", s, po, pairs=s.pairs[pick])
    assert np.array_equal(mu, emu)
    assert np.array_equal(ds.codes_np(), codes)
    assert np.array_equal(ds.buckets_np(6), buckets)
    (off1, mt1), (off2, mt2) = outs
    assert np.array_equal(off1, off2) and np.array_equal(mt1, mt2)
    _properties(s, off2, mt2)
    goff, gmt = _lists_of(off2, mt2, pick)
    assert len(pick) >= len(s.pairs) // 10
    assert np.array_equal(goff, eoff), "sampled pair %s" % _first_mismatch(goff, gmt, eoff, emt)
    assert np.array_equal(gmt, emt), "sampled pair %s" % _first_mismatch(goff, gmt, eoff, emt)
    plan.close()
    ctx.close()


def test_config4_full_size(ch, orc):
    """Config 4 (Sec. 7.2 band, 4 px): 500 views, 14,613 pairs, the batched
    join with its band test as bench.py runs it; every code and every pair's
    list entry for entry."""
    s = synth.config4()
    ctx, ds, plan, outs, stats, mu = _run_gpu(ch, s, precision=1, epi_px=4.0)
    assert ch.cashash_plan_get_tuning(plan)["kernel"] == ch.CASHASH_KERNEL_JOIN
    po = orc.params(epi_px=4.0)
    emu, codes, buckets, eoff, emt = _oracle_all(orc, "config4", s, po)
    assert np.array_equal(mu, emu)
    assert np.array_equal(ds.codes_np(), codes)
    assert np.array_equal(ds.buckets_np(6), buckets)
    (off1, mt1), (off2, mt2) = outs
    assert np.array_equal(off1, off2) and np.array_equal(mt1, mt2)
    _properties(s, off2, mt2)
    assert np.array_equal(off2, eoff), "pair %s" % _first_mismatch(off2, mt2, eoff, emt)
    assert np.array_equal(mt2, emt), "pair %s" % _first_mismatch(off2, mt2, eoff, emt)
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


def _bound_margins(ch, orc, s, ctx, ds, mu, rows, feats, chunk=100_000):
    """Over the features `feats` (ascending ranges): the largest |v~ - v| / E
    over all projections and over the unflagged ones (|v~| > E, which take the
    sign of v~), and the number flagged; asserts the bound holds everywhere."""
    worst_all, worst_unflagged, flagged = 0.0, 0.0, 0
    for lo, hi in feats:
        for f0 in range(lo, hi, chunk):
            n = min(chunk, hi - f0)
            approx, bound = ch.cashash_projection_bounds(ctx, ds, f0, n)
            a = approx.cpu().numpy().astype(np.float64)
            e = bound.cpu().numpy().astype(np.float64)
            v = orc.projections(s.desc[f0:f0 + n], mu, s.R, rows, threads=16)
            err = np.abs(a - v)
            assert (err <= e).all(), "bound violated at %s" % (np.argwhere(err > e)[:4] + [f0, 0]).tolist()
            r = err / e
            fl = np.abs(a) <= e
            flagged += int(fl.sum())
            worst_all = max(worst_all, float(r.max()))
            if (~fl).any():
                worst_unflagged = max(worst_unflagged, float(r[~fl].max()))
    return worst_all, worst_unflagged, flagged


@pytest.mark.parametrize("precision", [0, 1])
def test_projection_bound_margins_config1(ch, orc, precision):
    """The rounding bound E of the projection (FP32 form: 2^-16 ||R_b|| ||x||
    + beta_b; BF16 form: 2^-15 ||R_b|| ||x|| + beta_b, which assumes a
    pessimistic adder model for the tensor cores' FP32 accumulation) against
    the oracle's exact ordered-double values on every feature of config 1:
    |v~ - v| <= E everywhere, the flagged count is the library's re-evaluation
    count, and the largest |v~ - v| / E over the unflagged projections is
    below 0.5 (the bound holds with a factor of two to spare)."""
    s = synth.config1()
    p = ch.cashash_default_params(precision=precision)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    mu = ch.cashash_get_mean(ctx)
    n_reeval = ch.cashash_get_stats(ctx)["n_reevaluated"]
    rows = 128 + 6 * 8
    worst_all, worst_unflagged, flagged = _bound_margins(ch, orc, s, ctx, ds, mu, rows, [(0, s.desc.shape[0])])
    print("config1 precision %d: max |v~-v|/E all %.4g, unflagged %.4g, flagged %d"
          % (precision, worst_all, worst_unflagged, flagged))
    assert flagged == n_reeval
    assert worst_unflagged < 0.5
    ctx.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_projection_bound_margins_config3_sample(ch, orc, precision):
    """The same on 30 sampled config-3 images (1,000 to 20,000 features)."""
    s = synth.config3()
    p = ch.cashash_default_params(precision=precision)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    mu = ch.cashash_get_mean(ctx)
    rows = 128 + 6 * 8
    pick = np.sort(np.random.default_rng(33).choice(s.n_images, 30, replace=False))
    feats = [(int(s.img_off[i]), int(s.img_off[i + 1])) for i in pick]
    worst_all, worst_unflagged, flagged = _bound_margins(ch, orc, s, ctx, ds, mu, rows, feats)
    print("config3 sample precision %d: max |v~-v|/E all %.4g, unflagged %.4g, flagged %d over %d features"
          % (precision, worst_all, worst_unflagged, flagged, sum(b - a for a, b in feats)))
    assert worst_unflagged < 0.5
    ctx.close()
