"""Host-side logic of bench.py and synth on CPU: the parity comparison of the
timed step, the roofline's touched-bytes accounting, and the planted
correspondences behind the tau sweep's recall."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

torch = pytest.importorskip("torch")


def _bench():
    import bench
    return bench


def test_parity_check_counts_mismatching_pairs():
    bench = _bench()
    # GPU lists of 4 pairs: counts 2, 0, 3, 1
    off = torch.tensor([0, 2, 2, 5, 6], dtype=torch.int64)
    mt = torch.tensor([[0, 5], [3, 1], [1, 1], [2, 7], [9, 9], [4, 0]], dtype=torch.int32)
    # the oracle's lists of sampled pairs 1 and 2 (re-based): equal
    smp = {"pick": np.array([1, 2]), "off": np.array([0, 0, 3], np.uint64),
           "mt": np.array([[1, 1], [2, 7], [9, 9]], np.uint32)}
    r = bench.parity_check(smp, off, mt)
    assert r["pairs_checked"] == 2 and r["matches_checked"] == 3 and r["mismatches"] == 0
    # pair 0 sampled with one entry changed, pair 3 equal
    smp = {"pick": np.array([0, 3]), "off": np.array([0, 2, 3], np.uint64),
           "mt": np.array([[0, 5], [3, 2], [4, 0]], np.uint32)}
    r = bench.parity_check(smp, off, mt)
    assert r["pairs_checked"] == 2 and r["mismatches"] == 1
    # a missing match counts as a mismatch too
    smp = {"pick": np.array([3]), "off": np.array([0, 0], np.uint64), "mt": np.zeros((0, 2), np.uint32)}
    assert bench.parity_check(smp, off, mt)["mismatches"] == 1


def test_lookup_entries_is_the_bucket_product():
    bench = _bench()
    rng = np.random.default_rng(3)
    sizes = [50, 0, 70, 30]
    off = np.zeros(5, np.uint64)
    off[1:] = np.cumsum(sizes)
    T, m = 3, 4
    buckets = rng.integers(0, 1 << m, size=(int(off[-1]), T)).astype(np.uint8)
    pairs = np.array([[0, 2], [2, 0], [3, 1], [0, 3]], np.uint32)
    brute = 0
    for a, b in pairs:
        A = buckets[off[a]:off[a + 1]]
        B = buckets[off[b]:off[b + 1]]
        for t in range(T):
            brute += int((A[:, t][:, None] == B[:, t][None, :]).sum())
    assert bench.lookup_entries(buckets, off, pairs, T, m) == brute


def test_planted_pairs_are_the_noisy_copies():
    s = synth.config1(seed=7, n_images=8, lo=300, hi=500)
    truth = s.truth["copies"]
    assert len(truth) == 8
    # every recorded copy is within the noise of its source row
    for i, t in enumerate(truth):
        for pos, k, spos in t[:20]:
            a = s.image(i)[int(pos)].astype(np.int64)
            b = s.image(int(k))[int(spos)].astype(np.int64)
            assert np.abs(a - b).mean() < 16 and abs(i - int(k)) <= 5 and i != int(k)
    planted = synth.planted_pairs(truth, s.pairs)
    for (a, b), st in zip(s.pairs, planted):
        if abs(int(a) - int(b)) > 5:
            assert not st  # copies come from index-neighbours only
    assert sum(len(x) for x in planted) == sum(len(t) for t in truth)
    # recording the truth draws no random numbers: the images are those of a plain call
    s2 = synth.config1(seed=7, n_images=8, lo=300, hi=500)
    assert np.array_equal(s.desc, s2.desc)


class _FakeCh:
    CASHASH_KERNEL_JOIN, CASHASH_KERNEL_QUERY, CASHASH_KERNEL_JOIN_TC, CASHASH_KERNEL_WARP = 1, 2, 3, 4


class _FakeDs:
    def __init__(self, buckets):
        self._b = buckets

    def buckets_np(self, T):
        return self._b[:, :T]


def test_roofline_figures_follow_the_touched_bytes_definition(monkeypatch):
    """The line's roofline, recomputed by hand: touched bytes = 20 B per lookup entry + 1,480 B per
    query (k = 10), over the kernel's event time, against the measured copy bandwidth; the DRAM
    traffic is the profiled bytes per entry times the entries, only for the join without the band."""
    bench = _bench()
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 1000.0, "bf16_tflops": 2000.0, "source": "test",
                                                 "sm_max_mhz": 2000.0})
    rng = np.random.default_rng(5)
    sizes = [40, 25, 60]
    img_off = np.zeros(4, np.uint64)
    img_off[1:] = np.cumsum(sizes)
    T, m = 6, 8
    buckets = rng.integers(0, 4, size=(int(img_off[-1]), 8)).astype(np.uint8)  # few buckets: many entries
    s = synth.ImageSet(np.zeros((int(img_off[-1]), 128), np.uint8), img_off,
                       np.array([[0, 1], [2, 0], [1, 2]], np.uint32), np.zeros((176, 128)))

    class P:
        n_tables, bits_per_table, top_k, flags, epi_px = T, m, 10, 0, -1.0
    entries = bench.lookup_entries(buckets[:, :T], img_off, s.pairs, T, m)
    queries = 40 + 60 + 25
    r = bench.roofline_of(_FakeCh, P, s, _FakeDs(buckets), {"match": [2.0, 4.0]}, {"kernel": 1}, 100)
    t = 3.0e-3
    touched = 20.0 * entries + 1480.0 * queries
    assert r["units_per_launch"] == entries and r["queries_per_launch"] == queries
    assert abs(r["achieved"] - touched / t / 1e9) < 1e-9 * r["achieved"]
    assert abs(r["frac"] - r["achieved"] / 1000.0) < 1e-12
    assert r["kernel"] == "k_join"
    prof = bench.PROFILED_TRAFFIC["k_join"]
    assert abs(r["traffic"] - prof["bytes_per_entry"] * entries) < 1e-6 * r["traffic"]
    assert abs(r["dram_frac"] - r["traffic"] / t / 1e9 / 1000.0) < 1e-12
    assert abs(r["alu_view"]["peak_gentries_s"] - 16 / 4 * 100 * 2000e6 / 1e9) < 1e-9
    # the band form and the other kernels carry no traffic figure; the warp form is timed by its fallback
    P.epi_px = 4.0
    assert bench.roofline_of(_FakeCh, P, s, _FakeDs(buckets), {"match": [3.0]}, {"kernel": 1}, 100)["traffic"] is None
    P.epi_px = -1.0
    w = bench.roofline_of(_FakeCh, P, s, _FakeDs(buckets), {"match": [], "fallback": [3.0]}, {"kernel": 4}, 100)
    assert w["kernel"] == "k_match_fallback" and w["traffic"] is None
    # the mutual check counts both directions
    P.flags = 1
    mu = bench.roofline_of(_FakeCh, P, s, _FakeDs(buckets), {"match": [3.0]}, {"kernel": 2}, 100)
    assert mu["units_per_launch"] == entries + bench.lookup_entries(buckets[:, :T], img_off, s.pairs[:, ::-1], T, m)
    assert mu["queries_per_launch"] == 2 * queries


def test_profiled_traffic_is_for_the_current_join_sources():
    """The DRAM bytes per entry that the bench scales belong to the sources they were captured on:
    the recorded SHA-256 of join.cu + join_common.cuh is that of the tree."""
    bench = _bench()
    prof = bench.PROFILED_TRAFFIC["k_join"]
    assert bench.source_sha256(prof["sources"]) == prof["sha256"]
    assert 1.0 < prof["bytes_per_entry"] < 20.0
