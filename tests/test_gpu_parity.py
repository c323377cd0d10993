"""CUDA path vs the CPU oracle, element by element, through the C-ABI.

Codes and bucket ids are compared bit for bit, lookup tables as sets per
bucket, match lists entry for entry (the output order is defined: pairs in
input order, ascending query index).
"""
import threading

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

JC = 3968          # features per lookup-table chunk (library layout)
OFF_STRIDE = 264   # uint16 offsets per (chunk, table)


@pytest.fixture(scope="module")
def ch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1805_08995_gb300 as m
    torch.cuda.set_device(0)
    return m


def oracle_codes(orc, desc, R, po, mu=None, threads=8):
    """Oracle codes, computed in parallel row blocks (ctypes releases the GIL)."""
    if mu is None:
        mu = orc.mean(desc)
    n = desc.shape[0]
    codes = np.zeros((n, 4), np.uint32)
    buckets = np.zeros((n, po.n_tables), np.uint8)
    step = max(1, (n + threads - 1) // threads)

    def work(s):
        c, b = orc.hash_codes(desc[s:s + step], mu, R, po)
        codes[s:s + step] = c
        buckets[s:s + step] = b

    ts = [threading.Thread(target=work, args=(s,)) for s in range(0, n, step)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return mu, codes, buckets


def gpu_run(ch, s, pairs, tuning=None, **pk):
    """tuning: (kernel, tile, ctas_per_sm) forced on a batched plan, or None
    for cashash_match_pairs with the default choice."""
    p = ch.cashash_default_params(**pk)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc, s.kpts)
    ch.cashash_build_codes(ctx, ds)
    pairs = np.asarray(pairs, np.uint32).reshape(-1, 2)
    P = pairs.shape[0]
    cap = int(s.sizes()[pairs[:, 0]].sum()) if P else 0
    moff = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
    mt = torch.zeros((max(cap, 1), 2), dtype=torch.int32, device="cuda")
    F = None if s.F is None else torch.from_numpy(np.ascontiguousarray(s.F)).cuda()
    if tuning is None:
        ch.cashash_match_pairs(ctx, ds, pairs, moff, mt, cap, F=F)
    else:
        plan = ch.cashash_plan_create(ctx, ds, pairs)
        ch.cashash_plan_set_tuning(plan, *tuning)
        assert ch.cashash_plan_get_tuning(plan)["kernel"] == tuning[0]
        for _ in range(2):  # the second run starts from the thresholds the first learned
            ch.cashash_match_plan(ctx, plan, moff, mt, cap, F=F)
        torch.cuda.synchronize()
        plan.close()
    assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK
    off = moff.cpu().numpy().astype(np.uint64)
    got = mt[:int(off[-1])].cpu().numpy().view(np.uint32)
    stats = ch.cashash_get_stats(ctx)
    return ctx, ds, off, got, stats


def oparams(orc, pk):
    return orc.params(code_bits=pk.get("code_bits", 128), n_tables=pk.get("n_tables", 6),
                      bits_per_table=pk.get("bits_per_table", 8), top_k=pk.get("top_k", 10),
                      ratio=(pk.get("ratio_num", 4), pk.get("ratio_den", 5)), tau=pk.get("tau", None),
                      epi_px=pk.get("epi_px", -1.0), flags=pk.get("flags", 0))


def check_case(ch, orc, s, pairs, tuning=None, **pk):
    ctx, ds, off, got, stats = gpu_run(ch, s, pairs, tuning=tuning, **pk)
    po = oparams(orc, pk)
    mu, codes, buckets = oracle_codes(orc, s.desc, s.R, po)
    assert np.array_equal(ch.cashash_get_mean(ctx), mu)
    assert np.array_equal(ds.codes_np(), codes)
    assert np.array_equal(ds.buckets_np(po.n_tables), buckets)
    assert not ds.buckets[:ds.n, po.n_tables:].any().item()
    sq = (s.desc.astype(np.int64) ** 2).sum(axis=1)
    assert np.array_equal(ds.sqnorm[:ds.n].cpu().numpy().astype(np.int64), sq)
    eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pairs, po, F=s.F, kpts=s.kpts)
    assert np.array_equal(off, eoff)
    assert np.array_equal(got, emt)
    ctx.close()
    return ds, codes, buckets, stats


SIZES = [300, 1, 0, 2500, 5000, 3969, 3968, 33, 8000]


def _pairs(sizes, extra=()):
    n = len(sizes)
    pr = [(i, k) for i in range(n) for k in range(n) if i != k and (i + k) % 3 != 1]
    pr += [(i, i) for i in (3, 4) if i < n] + list(extra)
    return np.array(pr, np.uint32)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("sched", [0, 1])
def test_default_parameters_ragged_images(ch, orc, sched, prec):
    s = synth.random_set(101, SIZES)
    check_case(ch, orc, s, _pairs(SIZES), schedule=sched, precision=prec)


@pytest.mark.parametrize("pk", [
    dict(code_bits=64), dict(code_bits=32, n_tables=2), dict(code_bits=96, n_tables=4, bits_per_table=6),
    dict(n_tables=8, bits_per_table=8), dict(n_tables=1, bits_per_table=0, top_k=8), dict(n_tables=3, bits_per_table=5),
])
def test_bf16_projection_row_counts(ch, orc, pk):
    """Tensor-core projection with every padded row count it supports."""
    sizes = [700, 1300, 0, 129, 4500]
    s = synth.random_set(212, sizes)
    check_case(ch, orc, s, _pairs(sizes), precision=1, **pk)


@pytest.mark.parametrize("pk", [
    dict(top_k=4), dict(top_k=16), dict(top_k=32), dict(top_k=1), dict(top_k=2),
    dict(bits_per_table=4, n_tables=3), dict(bits_per_table=0, n_tables=1, top_k=8),
    dict(n_tables=8, bits_per_table=8), dict(n_tables=1, bits_per_table=5),
    dict(code_bits=64), dict(code_bits=32, n_tables=2), dict(code_bits=96, n_tables=4, bits_per_table=6),
    dict(tau=40), dict(tau=0), dict(ratio_num=9, ratio_den=10),
    dict(flags=1), dict(flags=2), dict(flags=3), dict(flags=3, tau=50, top_k=4),
])
@pytest.mark.parametrize("sched", [0, 1])
def test_parameter_variants(ch, orc, pk, sched):
    sizes = [700, 1300, 0, 260, 4500]
    s = synth.random_set(202, sizes)
    check_case(ch, orc, s, _pairs(sizes), schedule=sched, **pk)


@pytest.mark.parametrize("kernel", ["join", "join_tc"])
@pytest.mark.parametrize("hint,fixed", [(0, True), (30, True), (50, True), (53, True), (56, False), (0, False),
                                        (64, True), (100, True)])
def test_speculative_threshold_never_changes_results(ch, orc, hint, fixed, kernel):
    """The batched kernel's Hamming threshold is a guess; queries it starves
    are re-matched exactly.  Forcing bad guesses (0: every query falls back;
    near the median k-th distance: about half do; 64 and above: padding rows
    of the tensor-core tiles pass the compare and must be masked, and most
    survivor lists overflow) must not change a match."""
    sizes = [2600, 4100, 0, 900, 5200]
    s = synth.random_set(707, sizes)
    pairs = _pairs(sizes)
    p = ch.cashash_default_params(schedule=1)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    plan = ch.cashash_plan_create(ctx, ds, pairs)
    if kernel == "join_tc":
        ch.cashash_plan_set_tuning(plan, ch.CASHASH_KERNEL_JOIN_TC)
        assert ch.cashash_plan_get_tuning(plan)["kernel"] == ch.CASHASH_KERNEL_JOIN_TC
    ch.cashash_plan_set_threshold_hint(plan, hint, fixed)
    P = len(pairs)
    cap = int(s.sizes()[pairs[:, 0]].sum())
    moff = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
    mt = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
    po = orc.params()
    mu, codes, buckets = oracle_codes(orc, s.desc, s.R, po)
    eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pairs, po)
    for _ in range(2):
        ch.cashash_match_plan(ctx, plan, moff, mt, cap)
        assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK
        off = moff.cpu().numpy().astype(np.uint64)
        assert np.array_equal(off, eoff)
        assert np.array_equal(mt[:int(off[-1])].cpu().numpy().view(np.uint32), emt)
    plan.close()
    ctx.close()


@pytest.mark.parametrize("case", ["join", "large_image", "huge_candidate", "band"])
def test_batched_kernel_choice(ch, orc, case):
    """The batched schedule runs the tensor-core bucket join by default
    (calibration + join + fallback + scan + compaction = 5 launches; with the
    band no calibration, 4) unless a query image exceeds the join's
    shared-memory counters; then the speculative per-query kernel (also
    calibrated: 5 launches).  Both match the oracle.  A candidate image of more than 65,535
    features takes the join tables' global-scatter builder."""
    import math
    pk = dict(schedule=1)
    if case == "band":
        s = synth.epipolar_set(43, n_views=4, n_points=9000, arc=2 * math.pi * 4 / 250, z_max=0.355)
        pairs = np.concatenate([s.pairs, s.pairs[:, ::-1]])
        s.F = np.concatenate([s.F, s.F.reshape(-1, 3, 3).transpose(0, 2, 1).reshape(-1, 9)])
        pk["epi_px"] = 4.0
    else:
        sizes = {"join": [3000, 2500, 700], "large_image": [56000, 1500], "huge_candidate": [70000, 1500]}[case]
        s = synth.random_set(808, sizes)
        pairs = {"join": _pairs(sizes), "large_image": np.array([[0, 1], [1, 0]], np.uint32),
                 "huge_candidate": np.array([[1, 0]], np.uint32)}[case]
    p = ch.cashash_default_params(**pk)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc, s.kpts)
    ch.cashash_build_codes(ctx, ds)
    plan = ch.cashash_plan_create(ctx, ds, pairs)
    P = len(pairs)
    cap = int(s.sizes()[pairs[:, 0]].sum())
    moff = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
    mt = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
    F = None if s.F is None else torch.from_numpy(np.ascontiguousarray(s.F)).cuda()
    n0 = ch.cashash_get_stats(ctx)["n_launches"]
    ch.cashash_match_plan(ctx, plan, moff, mt, cap, F=F)
    assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK
    assert ch.cashash_get_stats(ctx)["n_launches"] - n0 == (4 if case == "band" else 5)
    kern = ch.cashash_plan_get_tuning(plan)["kernel"]
    assert kern == (ch.CASHASH_KERNEL_QUERY if case == "large_image" else ch.CASHASH_KERNEL_JOIN)
    po = oparams(orc, pk)
    mu, codes, buckets = oracle_codes(orc, s.desc, s.R, po)
    eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pairs, po, F=s.F, kpts=s.kpts)
    off = moff.cpu().numpy().astype(np.uint64)
    assert np.array_equal(off, eoff)
    assert np.array_equal(mt[:int(off[-1])].cpu().numpy().view(np.uint32), emt)
    plan.close()
    ctx.close()


def test_every_tuning_and_the_autotuner(ch, orc):
    """Every kernel configuration of a batched plan reproduces the oracle's
    lists (twice: direct launch, then graph replay); the autotuner keeps one
    of them and reports its sample time."""
    sizes = [3000, 4100, 900, 5200, 0]
    s = synth.random_set(909, sizes)
    pairs = _pairs(sizes)
    p = ch.cashash_default_params(schedule=1)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    po = orc.params()
    mu, codes, buckets = oracle_codes(orc, s.desc, s.R, po)
    eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pairs, po)
    plan = ch.cashash_plan_create(ctx, ds, pairs)
    t0 = ch.cashash_plan_get_tuning(plan)
    assert (t0["kernel"], t0["tile"], t0["ctas_per_sm"]) == (ch.CASHASH_KERNEL_JOIN, 4, 0)
    P = len(pairs)
    cap = int(s.sizes()[pairs[:, 0]].sum())
    moff = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
    mt = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")

    def check():
        for _ in range(2):
            ch.cashash_match_plan(ctx, plan, moff, mt, cap)
            assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK
            off = moff.cpu().numpy().astype(np.uint64)
            assert np.array_equal(off, eoff)
            assert np.array_equal(mt[:int(off[-1])].cpu().numpy().view(np.uint32), emt)

    J, Q, W = ch.CASHASH_KERNEL_JOIN, ch.CASHASH_KERNEL_QUERY, ch.CASHASH_KERNEL_WARP
    for kern, tile, ctas in [(J, 4, 0), (J, 2, 0), (J, 4, 1), (J, 2, 1), (Q, 512, 0), (Q, 256, 0), (W, 0, 0)]:
        ch.cashash_plan_set_tuning(plan, kern, tile, ctas)
        t = ch.cashash_plan_get_tuning(plan)
        assert (t["kernel"], t["tile"], t["ctas_per_sm"]) == (kern, tile, ctas)
        check()
    for mp in (5, 0):  # a sample, then the plan itself
        t = ch.cashash_plan_autotune(ctx, plan, max_pairs=mp)
        assert t["kernel"] in (J, Q, ch.CASHASH_KERNEL_JOIN_TC, W) and t["ms_sample"] > 0
        check()
    plan.close()
    ctx.close()


def test_band_kernels_and_the_autotuner(ch, orc):
    """With the band every kernel configuration (the join with its band test,
    the per-query kernel with either tile) gives the oracle's lists; a 2-tile
    join request is normalised to 4 tiles; the autotuner keeps one."""
    import math
    s = synth.epipolar_set(44, n_views=4, n_points=9000, arc=2 * math.pi * 4 / 250, z_max=0.355)
    pairs = np.concatenate([s.pairs, s.pairs[:, ::-1]])
    s.F = np.concatenate([s.F, s.F.reshape(-1, 3, 3).transpose(0, 2, 1).reshape(-1, 9)])
    pk = dict(schedule=1, epi_px=4.0)
    p = ch.cashash_default_params(**pk)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc, s.kpts)
    ch.cashash_build_codes(ctx, ds)
    plan = ch.cashash_plan_create(ctx, ds, pairs)
    J, Q = ch.CASHASH_KERNEL_JOIN, ch.CASHASH_KERNEL_QUERY
    t0 = ch.cashash_plan_get_tuning(plan)
    assert (t0["kernel"], t0["tile"]) == (J, 4)
    F = torch.from_numpy(np.ascontiguousarray(s.F)).cuda()
    P = len(pairs)
    cap = int(s.sizes()[pairs[:, 0]].sum())
    moff = torch.zeros(P + 1, dtype=torch.int64, device="cuda")
    mt = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
    po = oparams(orc, pk)
    mu, codes, buckets = oracle_codes(orc, s.desc, s.R, po)
    eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pairs, po, F=s.F, kpts=s.kpts)

    def check():
        for _ in range(2):
            ch.cashash_match_plan(ctx, plan, moff, mt, cap, F=F)
            assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK
            off = moff.cpu().numpy().astype(np.uint64)
            assert np.array_equal(off, eoff)
            assert np.array_equal(mt[:int(off[-1])].cpu().numpy().view(np.uint32), emt)

    W = ch.CASHASH_KERNEL_WARP
    for kern, tile, want in [(J, 2, 4), (J, 4, 4), (Q, 512, 512), (Q, 256, 256), (W, 0, 0)]:
        ch.cashash_plan_set_tuning(plan, kern, tile, 0)
        t = ch.cashash_plan_get_tuning(plan)
        assert (t["kernel"], t["tile"]) == (kern, want)
        check()
    t = ch.cashash_plan_autotune(ctx, plan, F=F, max_pairs=0)
    assert t["kernel"] in (J, Q, ch.CASHASH_KERNEL_JOIN_TC, W) and t["ms_sample"] > 0
    check()
    plan.close()
    ctx.close()


@pytest.mark.parametrize("case", ["plain_persistent", "plain_per_pair", "band", "tuned_query", "tuned_warp"])
def test_chunked_matching_resumes(ch, orc, case):
    """A long pair list matched in chunks: the callback stops the run after two
    chunks, a second call resumes at the returned cursor, and the chunks
    joined equal the oracle's lists for the whole list.  tuned_query /
    tuned_warp: the chunks' plans take the per-query kernel or the
    warp-per-query configuration set by cashash_set_host_tuning."""
    import math
    pk = dict(schedule=0 if case == "plain_per_pair" else 1)
    if case == "band":
        s = synth.epipolar_set(46, n_views=6, n_points=9000, arc=2 * math.pi * 6 / 250, z_max=0.355)
        pairs = np.concatenate([s.pairs, s.pairs[:, ::-1]])
        s.F = np.concatenate([s.F, s.F.reshape(-1, 3, 3).transpose(0, 2, 1).reshape(-1, 9)])
        pk["epi_px"] = 4.0
    else:
        sizes = [900, 1400, 0, 300, 2100, 700, 1200]
        s = synth.random_set(606, sizes)
        pairs = np.array([(i, k) for i in range(len(sizes)) for k in range(len(sizes)) if i != k], np.uint32)
    p = ch.cashash_default_params(**pk)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc, s.kpts)
    ch.cashash_build_codes(ctx, ds)
    assert ch.cashash_get_host_tuning(ctx)["kernel"] == 0
    if case == "tuned_query":
        ch.cashash_set_host_tuning(ctx, ch.CASHASH_KERNEL_QUERY, 256)
        assert ch.cashash_get_host_tuning(ctx) == {"kernel": ch.CASHASH_KERNEL_QUERY, "tile": 256, "ctas_per_sm": 0}
    if case == "tuned_warp":
        ch.cashash_set_host_tuning(ctx, ch.CASHASH_KERNEL_WARP)
        assert ch.cashash_get_host_tuning(ctx)["kernel"] == ch.CASHASH_KERNEL_WARP
    F = torch.from_numpy(np.ascontiguousarray(s.F)).cuda() if s.F is not None else None
    got = {}
    seen = []

    def stop_after_two(first, off, m):
        got[first] = (off, m)
        seen.append(first)
        return len(seen) == 2

    chunk = 5
    cur = ch.cashash_match_chunked(ctx, ds, pairs, chunk, stop_after_two, F=F)
    assert cur == min(2 * chunk, len(pairs)) and len(seen) == min(2, -(-len(pairs) // chunk))
    cur = ch.cashash_match_chunked(ctx, ds, pairs, chunk, lambda first, off, m: got.__setitem__(first, (off, m)),
                                   cursor=cur, F=F)
    assert cur == len(pairs)
    po = oparams(orc, pk)
    mu, codes, buckets = oracle_codes(orc, s.desc, s.R, po)
    eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pairs, po, F=s.F, kpts=s.kpts)
    assert sorted(got) == list(range(0, len(pairs), chunk))
    for first, (off, m) in got.items():
        n = off.shape[0] - 1
        e0, e1 = int(eoff[first]), int(eoff[first + n])
        assert np.array_equal(off.astype(np.uint64), eoff[first:first + n + 1] - eoff[first])
        assert np.array_equal(m, emt[e0:e1])
    ctx.close()


def test_lookup_tables_are_the_bucket_sets(ch, orc):
    sizes = [5000, 10, 0, 3968, 7937]
    s = synth.random_set(303, sizes)
    p = ch.cashash_default_params()
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    torch.cuda.synchronize()
    tb = ds.tables.cpu().numpy().view(np.uint16)
    buckets = ds.buckets_np(6)
    chunk_u16 = 6 * (OFF_STRIDE + JC)
    k = 0
    for i in range(len(sizes)):
        a0 = int(s.img_off[i])
        n = sizes[i]
        for c in range(0, n, JC):
            blk = tb[k * chunk_u16:(k + 1) * chunk_u16]
            ln = min(JC, n - c)
            for t in range(6):
                off = blk[t * OFF_STRIDE:t * OFF_STRIDE + 257].astype(np.int64)
                idx = blk[6 * OFF_STRIDE + t * JC:6 * OFF_STRIDE + t * JC + ln].astype(np.int64)
                assert off[0] == 0 and off[256] == ln and np.all(np.diff(off) >= 0)
                bb = buckets[a0 + c:a0 + c + ln, t]
                exp_off = np.concatenate([[0], np.cumsum(np.bincount(bb, minlength=256))])
                assert np.array_equal(off, exp_off)
                for v in range(0, 256, 17):
                    got = idx[off[v]:off[v + 1]]
                    assert np.array_equal(got, np.nonzero(bb == v)[0])
            k += 1
    ctx.close()


def test_bucket_sorted_tables(ch, orc):
    """The bucket-sorted tables (after the chunked ones): per image and table,
    offsets of the 256 buckets, the features of each bucket in index order,
    and each feature's 128-bit code inline."""
    sizes = [5000, 10, 0, 3968, 7937]
    s = synth.random_set(304, sizes)
    p = ch.cashash_default_params()
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    torch.cuda.synchronize()
    raw = ds.tables.cpu().numpy()
    codes, buckets = ds.codes_np(), ds.buckets_np(6)
    n_chunks = sum((n + JC - 1) // JC for n in sizes)
    o = max(n_chunks, 1) * 6 * (OFF_STRIDE + JC) * 2
    for i, n in enumerate(sizes):
        a0 = int(s.img_off[i])
        blk = 1040 + 4 * ((n + 3) // 4 * 4) + 16 * n
        for t in range(6):
            b = raw[o + t * blk:o + (t + 1) * blk]
            off = b[:1040].view(np.uint32)[:257].astype(np.int64)
            idx = b[1040:1040 + 4 * n].view(np.uint32)
            rec = b[1040 + 4 * ((n + 3) // 4 * 4):].view(np.uint32).reshape(-1, 4)
            exp_off = np.concatenate([[0], np.cumsum(np.bincount(buckets[a0:a0 + n, t], minlength=256))])
            assert np.array_equal(off, exp_off)
            order = np.argsort(buckets[a0:a0 + n, t], kind="stable")
            assert np.array_equal(idx, order)
            assert np.array_equal(rec, codes[a0 + order])
        o += 6 * blk
    ctx.close()


def test_one_pair_workload_config0(ch, orc):
    s = synth.config0()
    for sched in (0, 1):
        check_case(ch, orc, s, s.pairs, schedule=sched)


def test_identical_and_degenerate_descriptors(ch, orc):
    """Single-feature images, empty images, and a set whose descriptors are
    all identical: the centre equals every descriptor, every projection is
    exactly 0, every row goes through the double re-evaluation and every bit
    is 0 (sign at exactly zero)."""
    rng = np.random.default_rng(5)
    one = synth.sift_like(rng, 1)
    desc = np.concatenate([np.repeat(one, 40, axis=0), synth.sift_like(rng, 1), synth.sift_like(rng, 30)])
    s = synth.ImageSet(desc, np.array([0, 40, 41, 41, 71], np.uint64),
                       np.array([[0, 0], [0, 1], [1, 0], [2, 0], [0, 2], [3, 0], [0, 3], [3, 3]], np.uint32),
                       synth.projection_matrix(5))
    for prec in (0, 1):
        check_case(ch, orc, s, s.pairs, precision=prec)
        same = synth.ImageSet(np.repeat(one, 50, axis=0), np.array([0, 20, 50], np.uint64),
                              np.array([[0, 1], [1, 0], [0, 0]], np.uint32), synth.projection_matrix(6))
        ds, codes, buckets, stats = check_case(ch, orc, same, same.pairs, precision=prec)
        assert not codes.any() and not buckets.any()
        assert stats["n_reevaluated"] == 50 * 176


@pytest.mark.parametrize("flags", [0, 1, 3])
@pytest.mark.parametrize("sched", [0, 1, "join_tc"])
def test_epipolar_band(ch, orc, sched, flags):
    """Sec. 7.2: candidates outside the 4 px band around the query's
    epipolar line are removed before ranking (small config-4 style set)."""
    import math
    s = synth.epipolar_set(41, n_views=7, n_points=24000, arc=2 * math.pi * 7 / 250, z_max=0.355)
    assert len(s.pairs) >= 10 and s.kpts is not None
    both = np.concatenate([s.pairs, s.pairs[:, ::-1]])
    s.F = np.concatenate([s.F, s.F.reshape(-1, 3, 3).transpose(0, 2, 1).reshape(-1, 9)])
    tuning = (ch.CASHASH_KERNEL_JOIN_TC, 0, 0) if sched == "join_tc" else None
    check_case(ch, orc, s, both, tuning=tuning, schedule=1 if tuning else sched, epi_px=4.0, flags=flags)


@pytest.mark.parametrize("sched", [0, 1, "join_tc"])
def test_band_edge_decisions(ch, orc, sched):
    """Sec. 7.2 at the edge of the band: candidate j is a copy of query j (so it
    shares every bucket) placed on one of the two lines at 4 px from the
    query's epipolar line, moved by a few ulps or not at all.  The kernels'
    FP32 pre-test must defer these to the FP64 predicate and agree with the
    oracle on every one."""
    import math
    rng = np.random.default_rng(515)
    nA = 1200
    A = synth.sift_like(rng, nA)
    desc = np.concatenate([A, A])
    img_off = np.array([0, nA, 2 * nA], np.uint64)
    M = rng.standard_normal((3, 3))
    U, S, Vt = np.linalg.svd(M)
    S[2] = 0.0
    F = (U * S) @ Vt
    F /= np.linalg.norm(F)
    kA = (rng.random((nA, 2)) * [1920.0, 1080.0]).astype(np.float32)
    kB = np.empty((nA, 2), np.float32)
    d = 4.0
    for j in range(nA):
        x, y = float(kA[j, 0]), float(kA[j, 1])
        a = (F[0, 0] * x + F[0, 1] * y) + F[0, 2]
        b = (F[1, 0] * x + F[1, 1] * y) + F[1, 2]
        c = (F[2, 0] * x + F[2, 1] * y) + F[2, 2]
        nrm = math.hypot(a, b)
        t = rng.uniform(-60.0, 60.0) if j % 2 else rng.uniform(-900.0, 900.0)
        p0 = np.array([-c * a, -c * b]) / nrm ** 2 + t * np.array([-b, a]) / nrm
        off = rng.choice([-1.0, 1.0]) * d * (1.0 + rng.choice([-3e-7, -1e-7, 0.0, 1e-7, 3e-7]))
        kB[j] = (p0 + off * np.array([a, b]) / nrm).astype(np.float32)
    kpts = np.concatenate([kA, kB])
    pairs = np.array([[0, 1]], np.uint32)
    s = synth.ImageSet(desc, img_off, pairs, synth.projection_matrix(515), "band edge", F=F.reshape(1, 9),
                       kpts=kpts)
    tuning = (ch.CASHASH_KERNEL_JOIN_TC, 0, 0) if sched == "join_tc" else None
    check_case(ch, orc, s, pairs, tuning=tuning, schedule=1 if tuning else sched, epi_px=d)


def test_reevaluation_ordered_path(ch, orc):
    """Sec. 5.1 signs whose ordered FP64 sum is rounding noise: rows of R made orthogonal, in FP64,
    to one feature's centred descriptor each (112 rows, 112 features).  The re-evaluation's
    warp-parallel sign test cannot decide these and evaluates the ordered sequence itself; codes,
    buckets and matches must equal the oracle's, and the constructed projections must indeed lie
    inside the parallel test's undecided zone."""
    s = synth.random_set(717, [300, 260, 280])
    R = np.array(s.R[:176], np.float64)
    mu = orc.mean(s.desc)
    rows = list(range(0, 128, 2)) + list(range(128, 176))
    for f, b in enumerate(rows):
        t = s.desc[f].astype(np.float64) - mu
        R[b] = R[b] - (R[b] @ t) / (t @ t) * t
    s2 = synth.ImageSet(s.desc, s.img_off, s.pairs, R, "orthogonal rows")
    v = orc.projections(s.desc[:len(rows)], mu, R, 176)
    undecided = 0
    for f, b in enumerate(rows):
        t = s.desc[f].astype(np.float64) - mu
        if abs(v[f, b]) <= 1.6e-14 * np.abs(R[b] * t).sum():
            undecided += 1
    assert undecided >= len(rows) // 2
    for prec in (0, 1):
        ds, codes, buckets, stats = check_case(ch, orc, s2, s2.pairs, precision=prec)
        assert stats["n_reevaluated"] >= len(rows)


def _band_copy_set(rng, nA, F, kA, kB, name):
    A = synth.sift_like(rng, nA)
    return synth.ImageSet(np.concatenate([A, A]), np.array([0, nA, 2 * nA], np.uint64),
                          np.array([[0, 1]], np.uint32), synth.projection_matrix(616), name,
                          F=np.ascontiguousarray(F.reshape(1, 9)), kpts=np.concatenate([kA, kB]).astype(np.float32))


@pytest.mark.parametrize("case", ["huge_coordinates", "large_F", "infinite_point", "nan_point", "huge_F"])
def test_band_threshold_fallbacks(ch, orc, case):
    """Sec. 7.2 with inputs that defeat the join's FP32 thresholds on |a x' + b y' + c|: key-points
    so far out that the FP32 numerator could overflow (no candidate stays in the band), an F scaled
    by 1e28 (the same decisions as unscaled, every one in FP64), an infinite or NaN candidate point
    (the image's extent becomes infinite, or the point's own test is NaN), and an F so large that
    the FP32 line overflows (the FP64 right-hand side is infinite: every candidate is kept).  Every such decision goes to the FP64 expression, which must agree with the
    oracle's; each candidate is a copy of its query, so it shares every bucket."""
    rng = np.random.default_rng(616)
    nA = 600
    M = rng.standard_normal((3, 3))
    U, S, Vt = np.linalg.svd(M)
    S[2] = 0.0
    F = (U * S) @ Vt
    F /= np.linalg.norm(F)
    kA = (rng.random((nA, 2)) * [1920.0, 1080.0]).astype(np.float32)
    kB = (rng.random((nA, 2)) * [1920.0, 1080.0]).astype(np.float32)
    # half of the candidates on the query's line (inside the band), the rest where they fall
    for j in range(0, nA, 2):
        x, y = float(kA[j, 0]), float(kA[j, 1])
        a = (F[0, 0] * x + F[0, 1] * y) + F[0, 2]
        b = (F[1, 0] * x + F[1, 1] * y) + F[1, 2]
        c = (F[2, 0] * x + F[2, 1] * y) + F[2, 2]
        nrm = np.hypot(a, b)
        kB[j] = (np.array([-c * a, -c * b]) / nrm ** 2 + rng.uniform(-300, 300) * np.array([-b, a]) / nrm)
    if case == "huge_coordinates":
        kA = kA * np.float32(1e33)
        kB = kB * np.float32(1e33)
    elif case == "large_F":
        F = F * 1e28
    elif case == "infinite_point":
        kB[1] = [np.inf, 5.0]
    elif case == "nan_point":
        kB[3] = [np.nan, 5.0]
    else:
        F = F * 1e300
    s = _band_copy_set(rng, nA, F, kA, kB, "band fallbacks: " + case)
    check_case(ch, orc, s, s.pairs, schedule=1, epi_px=4.0)


def test_many_pairs_medium(ch, orc):
    s = synth.config1(seed=11, n_images=12, lo=1500, hi=4500)
    check_case(ch, orc, s, s.pairs, schedule=1)


@pytest.mark.parametrize("kernel", ["join", "query", "join_tc"])
@pytest.mark.parametrize("tau", [20, 30, 40, 50, 60, 128])
def test_tau_sweep_values(ch, orc, tau, kernel):
    """Sec. 6 threshold at every value of the tau sweep (bench.py --tau-sweep),
    on a 12-image exhaustive set in the BF16 form, with the bucket join and
    with the per-query kernel."""
    s = synth.config1(seed=12, n_images=12, lo=3000, hi=9000)
    tuning = {"join": (ch.CASHASH_KERNEL_JOIN, 4, 0), "query": (ch.CASHASH_KERNEL_QUERY, 512, 0),
              "join_tc": (ch.CASHASH_KERNEL_JOIN_TC, 0, 0)}[kernel]
    check_case(ch, orc, s, s.pairs, tuning=tuning, schedule=1, precision=1, tau=tau)


PARAM_VARIANTS = [
    dict(top_k=4), dict(top_k=16), dict(top_k=32), dict(top_k=1), dict(top_k=2),
    dict(bits_per_table=4, n_tables=3), dict(bits_per_table=0, n_tables=1, top_k=8),
    dict(n_tables=8, bits_per_table=8), dict(n_tables=1, bits_per_table=5),
    dict(code_bits=64), dict(code_bits=32, n_tables=2), dict(code_bits=96, n_tables=4, bits_per_table=6),
    dict(tau=40), dict(tau=0), dict(ratio_num=9, ratio_den=10),
    dict(flags=1), dict(flags=2), dict(flags=3), dict(flags=3, tau=50, top_k=4),
]


@pytest.mark.parametrize("pk", [dict(), dict(precision=1), dict(epi_px=4.0)] + PARAM_VARIANTS)
def test_warp_kernel_parameter_variants(ch, orc, pk):
    """The exact warp-per-query configuration (CASHASH_KERNEL_WARP: every query by the fallback
    kernel, no threshold guess) with every parameter variant, the band included, on ragged image
    sizes with an empty image."""
    sizes = [700, 1300, 0, 260, 4500]
    s = synth.random_set(203, sizes)
    pairs = _pairs(sizes)
    if pk.get("epi_px", -1.0) >= 0:
        import math
        s = synth.epipolar_set(45, n_views=5, n_points=9000, arc=2 * math.pi * 5 / 250, z_max=0.355)
        pairs = s.pairs
    check_case(ch, orc, s, pairs, tuning=(ch.CASHASH_KERNEL_WARP, 0, 0), schedule=1, **pk)


@pytest.mark.parametrize("pk", [dict(), dict(precision=1)] + PARAM_VARIANTS)
def test_join_tc_parameter_variants(ch, orc, pk):
    """The tcgen05 bucket join (FP8 +-1 rows in shared memory, 128-row tiles,
    TMEM accumulators) with every parameter variant: k from 1 to 32, one
    bucket per table (the whole candidate image in 256-column chunks), 32-,
    64- and 96-bit codes, tau, the ratio, the mutual check and single
    candidates; ragged image sizes including empty ones."""
    sizes = [700, 1300, 0, 260, 4500]
    s = synth.random_set(202, sizes)
    check_case(ch, orc, s, _pairs(sizes), tuning=(ch.CASHASH_KERNEL_JOIN_TC, 0, 0), schedule=1, **pk)


@pytest.mark.parametrize("case", ["ragged", "one_cta_per_sm", "huge_candidate", "medium"])
def test_join_tc_workloads(ch, orc, case):
    """The tcgen05 join on ragged image sizes (several tiles, ragged tails,
    the chunk and table boundaries of the other kernels), with one CTA per
    SM, with a candidate image of 70,000 features (tables by the global
    scatter builder, long candidate runs), and on a 12-image exhaustive set."""
    T = ch.CASHASH_KERNEL_JOIN_TC
    if case == "ragged":
        check_case(ch, orc, synth.random_set(101, SIZES), _pairs(SIZES), tuning=(T, 0, 0), schedule=1)
    elif case == "one_cta_per_sm":
        check_case(ch, orc, synth.random_set(101, SIZES), _pairs(SIZES), tuning=(T, 0, 1), schedule=1, precision=1)
    elif case == "huge_candidate":
        s = synth.random_set(808, [70000, 1500])
        check_case(ch, orc, s, np.array([[1, 0]], np.uint32), tuning=(T, 0, 0), schedule=1)
    else:
        s = synth.config1(seed=11, n_images=12, lo=1500, hi=4500)
        check_case(ch, orc, s, s.pairs, tuning=(T, 0, 0), schedule=1, precision=1)


def test_capacity_overflow_reports_and_truncates(ch, orc):
    sizes = [800, 900, 700]
    s = synth.random_set(404, sizes)
    pairs = np.array([[0, 1], [1, 2], [2, 0]], np.uint32)
    p = ch.cashash_default_params()
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    moff = torch.zeros(4, dtype=torch.int64, device="cuda")
    mt = torch.full((50, 2), -7, dtype=torch.int32, device="cuda")
    ch.cashash_match_pairs(ctx, ds, pairs, moff, mt, 40)
    assert ch.cashash_sync_status(ctx) == ch.CASHASH_EOVERFLOW
    assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK  # cleared
    po = orc.params()
    mu, codes, buckets = oracle_codes(orc, s.desc, s.R, po)
    eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pairs, po)
    assert np.array_equal(moff.cpu().numpy().astype(np.uint64), eoff)
    got = mt.cpu().numpy()
    assert np.array_equal(got[:40].view(np.uint32), emt[:40])
    assert (got[40:] == -7).all()
    ctx.close()


def test_host_end_to_end_matches_device_path(ch, orc):
    sizes = [3000, 4100, 0, 2000]
    s = synth.random_set(505, sizes)
    pairs = _pairs(sizes)
    p = ch.cashash_default_params()
    ctx = ch.cashash_create(p, s.R)
    cap = int(s.sizes()[pairs[:, 0]].sum())
    po = orc.params()
    mu, codes, buckets = oracle_codes(orc, s.desc, s.R, po)
    eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pairs, po)
    pinned = torch.from_numpy(s.desc).pin_memory()
    ch.cashash_set_profiling(ctx, True)
    # 1 MiB stages: the 9,100 descriptors land in two blocks, each block's column sums taken as it lands
    for desc, stage in ((s.desc, 0), (pinned, 0), (s.desc, 1 << 20), (pinned, 1 << 20)):
        st, off, mt = ch.cashash_run_host(ctx, desc, s.img_off, pairs, cap, stage_bytes=stage)
        assert st == ch.CASHASH_OK
        assert np.array_equal(off, eoff) and np.array_equal(mt, emt)
        ms = ch.cashash_get_stats(ctx)["ms_stage"]
        assert ms["h2d"] > 0 and ms["d2h"] > 0 and ms["centre"] > 0 and ms["match"] > 0
    assert np.array_equal(ch.cashash_get_mean(ctx), mu)
    st, off, mt = ch.cashash_run_host(ctx, s.desc, s.img_off, pairs, 10)
    assert st == ch.CASHASH_EOVERFLOW and np.array_equal(off, eoff) and np.array_equal(mt, emt[:10])
    ctx.close()
    # a batched context with every host-path kernel configuration
    ctx = ch.cashash_create(ch.cashash_default_params(schedule=ch.CASHASH_SCHED_PERSISTENT), s.R)
    for kernel, tile in ((ch.CASHASH_KERNEL_QUERY, 512), (ch.CASHASH_KERNEL_JOIN, 2), (ch.CASHASH_KERNEL_QUERY, 256),
                         (ch.CASHASH_KERNEL_JOIN_TC, 0), (ch.CASHASH_KERNEL_WARP, 0), (0, 0)):
        ch.cashash_set_host_tuning(ctx, kernel, tile)
        st, off, mt = ch.cashash_run_host(ctx, pinned, s.img_off, pairs, cap)
        assert st == ch.CASHASH_OK
        assert np.array_equal(off, eoff) and np.array_equal(mt, emt)
    with pytest.raises(ch.CashashError):
        ch.cashash_set_host_tuning(ctx, 7)
    ctx.close()


def test_invalid_arguments_are_rejected(ch):
    s = synth.random_set(606, [100, 50])
    p = ch.cashash_default_params()
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctx, ds)
    moff = torch.zeros(2, dtype=torch.int64, device="cuda")
    mt = torch.zeros((100, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(ch.CashashError) as e:
        ch.cashash_match_pairs(ctx, ds, np.array([[0, 2]], np.uint32), moff, mt, 100)
    assert e.value.status == ch.CASHASH_EINVAL
    bad = ch.cashash_default_params(top_k=0)
    with pytest.raises(ch.CashashError):
        ch.cashash_create(bad, s.R)
    with pytest.raises(ch.CashashError):
        ch.cashash_create(ch.cashash_default_params(code_bits=100), s.R)
    ctx.close()


def test_stage_profiling_and_graph_replay(ch):
    """Per-stage CUDA-event times are reported for direct launches and for
    replays of the captured persistent graph (external event nodes)."""
    s = synth.random_set(808, [3000, 3500, 1200])
    pairs = _pairs([3000, 3500, 1200])
    for sched in (0, 1):
        p = ch.cashash_default_params(schedule=sched)
        ctx = ch.cashash_create(p, s.R)
        ch.cashash_set_profiling(ctx, True)
        ds = ch.DeviceSet(p, s.img_off, s.desc)
        plan = ch.cashash_plan_create(ctx, ds, pairs)
        cap = int(s.sizes()[pairs[:, 0]].sum())
        moff = torch.zeros(len(pairs) + 1, dtype=torch.int64, device="cuda")
        mt = torch.zeros((cap, 2), dtype=torch.int32, device="cuda")
        n0 = ch.cashash_get_stats(ctx)["n_launches"]
        for _ in range(3):
            ch.cashash_build_codes(ctx, ds)
            ch.cashash_match_plan(ctx, plan, moff, mt, cap)
            st = ch.cashash_get_stats(ctx)
            # the per-pair schedule has no calibration or fallback stage; the copy stages
            # belong to cashash_run_host
            used = {k: v for k, v in st["ms_stage"].items()
                    if (sched or k not in ("calibrate", "fallback")) and k not in ("h2d", "d2h")}
            assert all(v > 0 for v in used.values()), st["ms_stage"]
            assert st["ms_stage"]["h2d"] == -1.0 and st["ms_stage"]["d2h"] == -1.0
            if not sched:
                assert st["ms_stage"]["calibrate"] == -1.0 and st["ms_stage"]["fallback"] == -1.0
        assert st["n_launches"] > n0
        assert ch.cashash_sync_status(ctx) == ch.CASHASH_OK
        plan.close()
        ctx.close()


def test_shards_on_concurrent_streams(ch, orc):
    """One GPU, two shards of a pair list (the LPT split of shard.py) matched
    by two contexts on two streams, both queued before either is waited for;
    the merged lists equal the oracle's for the whole list."""
    from paper_1805_08995_gb300 import shard
    sizes = [3000, 2500, 700, 4100, 1800]
    s = synth.random_set(909, sizes)
    pairs = _pairs(sizes)
    p = ch.cashash_default_params(schedule=ch.CASHASH_SCHED_PERSISTENT)
    ctxs = [ch.cashash_create(p, s.R) for _ in range(2)]
    ds = ch.DeviceSet(p, s.img_off, s.desc)
    ch.cashash_build_codes(ctxs[0], ds)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(2)]
    runs = []
    for r in range(2):
        idx = shard.shard_pairs(pairs, s.img_off, 2, r)
        plan = ch.cashash_plan_create(ctxs[r], ds, pairs[idx])
        cap = int(s.sizes()[pairs[idx, 0]].sum())
        moff = torch.zeros(len(idx) + 1, dtype=torch.int64, device="cuda")
        mt = torch.zeros((max(cap, 1), 2), dtype=torch.int32, device="cuda")
        runs.append((idx, plan, moff, mt, cap))
    for _ in range(2):  # the second round replays both captured graphs concurrently
        for r, (idx, plan, moff, mt, cap) in enumerate(runs):
            ch.cashash_match_plan(ctxs[r], plan, moff, mt, cap, stream=streams[r])
        torch.cuda.synchronize()
    parts = []
    for r, (idx, plan, moff, mt, cap) in enumerate(runs):
        assert ch.cashash_sync_status(ctxs[r], streams[r]) == ch.CASHASH_OK
        off = moff.cpu().numpy()
        parts.append((idx, off, mt[:int(off[-1])].cpu().numpy().view(np.uint32)))
        plan.close()
    po = orc.params()
    mu, codes, buckets = oracle_codes(orc, s.desc, s.R, po)
    eoff, emt = orc.match_pairs(s.desc, s.img_off, codes, buckets, pairs, po)
    moff, mt = shard.merge_shards(len(pairs), parts)
    assert np.array_equal(moff, eoff) and np.array_equal(mt, emt)
    for c in ctxs:
        c.close()
