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
