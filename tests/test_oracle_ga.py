"""Pins of the Ga-CasHash first-stage oracle (Sec. 7.1) against facts fixed
outside it: brute-force ranks, the bijection of the sampling map, the
normalisation's defining properties, exact recovery of a known F from
noise-free views, the closest rank-2 matrix (Eckart-Young), the Sampson
distance of a rectified pair in closed form, and RANSAC on planted outliers.

CASHASH_ORACLE_GA may name a (mutated) copy of oracle/ga.py to test instead.
"""
import importlib.util
import itertools
import os
import sys

import numpy as np
import pytest


def _load_ga():
    import oracle
    path = os.environ.get("CASHASH_ORACLE_GA")
    if not path:
        from oracle import ga
        return ga
    spec = importlib.util.spec_from_file_location("oracle.ga_mutant", path)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = oracle.__name__
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


ga = _load_ga()


# --- two calibrated views of random points (built here, independently of synth) ---

def _cross(t):
    return np.array([[0, -t[2], t[1]], [t[2], 0, -t[0]], [-t[1], t[0], 0]])


def _rodrigues(w):
    th = np.linalg.norm(w)
    k = w / th
    Kx = _cross(k)
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * Kx @ Kx


def _views(n, seed=0, noise=0.0):
    rng = np.random.default_rng(seed)
    K = np.array([[800.0, 0, 320], [0, 800.0, 240], [0, 0, 1]])
    R = _rodrigues(np.array([0.05, -0.2, 0.03]))
    t = np.array([1.0, 0.15, 0.1])
    X = np.stack([rng.uniform(-2, 2, n), rng.uniform(-1.5, 1.5, n), rng.uniform(5, 9, n)], axis=1)
    xa = (X @ K.T)
    xa = xa[:, :2] / xa[:, 2:]
    Y = X @ R.T + t
    xb = Y @ K.T
    xb = xb[:, :2] / xb[:, 2:]
    Kinv = np.linalg.inv(K)
    F = Kinv.T @ _cross(t) @ R @ Kinv  # x_b^T F x_a = 0
    if noise:
        xa = xa + rng.normal(0, noise, xa.shape)
        xb = xb + rng.normal(0, noise, xb.shape)
    return xa, xb, F


def _line_dist(F, xa, xb):
    """Distance of x_b to the epipolar line F x_a and of x_a to F^T x_b."""
    ha = np.concatenate([xa, np.ones((len(xa), 1))], 1)
    hb = np.concatenate([xb, np.ones((len(xb), 1))], 1)
    la, lb = ha @ F.T, hb @ F
    r = np.abs(np.sum(hb * la, 1))
    return r / np.hypot(la[:, 0], la[:, 1]), r / np.hypot(lb[:, 0], lb[:, 1])


def _outliers(F, n, rng, min_px=50.0):
    xa, xb = [], []
    while len(xa) < n:
        a = rng.uniform([0, 0], [640, 480])
        b = rng.uniform([0, 0], [640, 480])
        db, da = _line_dist(F, a[None], b[None])
        if min(da[0], db[0]) > min_px:
            xa.append(a)
            xb.append(b)
    return np.array(xa), np.array(xb)


def _same_F(F1, F2, tol):
    a, b = F1 / np.linalg.norm(F1), F2 / np.linalg.norm(F2)
    return min(np.abs(a - b).max(), np.abs(a + b).max()) <= tol


# --- selection by scale ---

@pytest.mark.parametrize("pct", [1, 20, 37, 100])
def test_top_scale_brute_force(pct):
    rng = np.random.default_rng(pct)
    sizes = [0, 1, 2, 7, 50, 333]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    scale = np.round(rng.uniform(0, 4, off[-1]) * 2) / 2  # many ties
    scale = scale.astype(np.float32)
    sel, sub = ga.top_scale(scale, off, pct)
    want = []
    for i, n in enumerate(sizes):
        a = int(off[i])
        k = -(-n * pct // 100)
        assert int(sub[i + 1] - sub[i]) == k
        for u in range(n):
            rank = sum(1 for v in range(n) if scale[a + v] > scale[a + u] or
                       (scale[a + v] == scale[a + u] and v < u))
            if rank < k:
                want.append(a + u)
    assert sel.tolist() == want


# --- the sampling map ---

def _word(r, mk):
    """A uint32 word u with floor(u * mk / 2^32) = r."""
    u = -(-(r << 32) // mk)
    assert (u * mk) >> 32 == r and u < 2 ** 32
    return u


def test_sample_map_is_a_bijection_on_eight():
    seen = set()
    for rs in itertools.product(*[range(8 - k) for k in range(8)]):
        words = [_word(r, 8 - k) for k, r in enumerate(rs)]
        s = tuple(ga.sample_indices(words, 8))
        assert sorted(s) == list(range(8))
        seen.add(s)
    assert len(seen) == 40320


def test_sample_map_distinct_in_range():
    rng = np.random.default_rng(3)
    for m in (8, 9, 12, 100, 5000):
        for _ in range(200):
            s = ga.sample_indices(rng.integers(0, 2 ** 32, 8, dtype=np.uint64), m)
            assert len(set(s)) == 8 and all(0 <= v < m for v in s)
    assert ga.sample_indices([0] * 8, 20) == list(range(8))
    assert ga.sample_indices([2 ** 32 - 1] * 8, 20) == list(range(19, 11, -1))


# --- normalisation, 8-point, rank 2, Sampson ---

def test_hartley_normalisation():
    rng = np.random.default_rng(1)
    p = rng.uniform([0, 0], [1920, 1080], (57, 2))
    T = ga.hartley(p)
    q = (np.concatenate([p, np.ones((57, 1))], 1) @ T.T)[:, :2]
    assert np.abs(q.mean(0)).max() < 1e-12
    assert abs(np.sqrt((q ** 2).sum(1)).mean() - np.sqrt(2.0)) < 1e-12


def test_eight_point_recovers_known_F():
    xa, xb, F = _views(8, seed=2)
    Ta, Tb = ga.hartley(xa), ga.hartley(xb)
    h = lambda T, x: np.concatenate([x, np.ones((len(x), 1))], 1) @ T.T
    Fn = ga.null_f(ga.design_rows(h(Ta, xa), h(Tb, xb)))
    Fe = Tb.T @ ga.rank2(Fn) @ Ta
    assert _same_F(Fe, F, 1e-8)
    # and the estimate explains the views: residuals vanish
    da, db = _line_dist(Fe, xa, xb)
    assert max(da.max(), db.max()) < 1e-6


def test_rank2_is_the_closest_rank_two_matrix():
    rng = np.random.default_rng(5)
    for _ in range(20):
        M = rng.normal(size=(3, 3))
        R2 = ga.rank2(M)
        assert abs(np.linalg.det(R2)) < 1e-12
        smin = np.sqrt(np.linalg.eigvalsh(M.T @ M).min())
        assert abs(np.linalg.norm(M - R2) - smin) < 1e-12


def test_sampson_rectified_closed_form():
    # pure horizontal translation: epipolar lines are the rows y = const, F x_a = (0, -1, y_a)
    F = np.array([[0.0, 0, 0], [0, 0, -1], [0, 1, 0]])
    rng = np.random.default_rng(6)
    xa = np.concatenate([rng.uniform(0, 500, (30, 2)), np.ones((30, 1))], 1)
    xb = np.concatenate([rng.uniform(0, 500, (30, 2)), np.ones((30, 1))], 1)
    # the optimal correction moves both points half the vertical gap
    assert np.allclose(ga.sampson2(F, xa, xb), (xa[:, 1] - xb[:, 1]) ** 2 / 2, rtol=1e-12, atol=0)


# --- RANSAC ---

def _words(n_hyp, seed):
    return np.random.default_rng(seed).integers(0, 2 ** 32, (n_hyp, 8), dtype=np.uint64).astype(np.uint32)


def test_ransac_planted_outliers_accepted():
    xa, xb, F = _views(70, seed=7)
    oa, ob = _outliers(F, 20, np.random.default_rng(8))
    pa, pb = np.concatenate([xa, oa]), np.concatenate([xb, ob])
    perm = np.random.default_rng(9).permutation(90)
    Fe, info = ga.estimate_F(pa[perm], pb[perm], _words(256, 10), ga.GaParams())
    m, n_in, best, acc, done = info
    assert (m, n_in, acc) == (90, 70, 1) and best != ga.NONE and done % 32 == 0 and done <= 256
    assert _same_F(Fe, F, 1e-8)
    assert abs(np.linalg.norm(Fe) - 1) < 1e-12 and Fe.ravel()[np.argmax(np.abs(Fe))] > 0


def test_ransac_two_thirds_boundary_and_ties():
    xa, xb, F = _views(60, seed=11)
    oa, ob = _outliers(F, 30, np.random.default_rng(12))
    pa, pb = np.concatenate([xa, oa]), np.concatenate([xb, ob])
    # hypotheses 0 and 1 both draw only inliers (indices < 60): equal counts, the lower wins
    w = _words(64, 13)
    for h in (0, 1):
        w[h] = [_word(k + 3 * h, 90 - k) for k in range(8)]
    Fe, info = ga.estimate_F(pa, pb, w, ga.GaParams(n_hyp=64))
    # 3 * 60 >= 2 * 90 exactly; w = 2/3 never stops early: (1 - w^8)^64 = 0.078 > 0.01
    assert tuple(info) == (90, 60, 0, 1, 64)
    assert _same_F(Fe, F, 1e-8)


def test_ransac_rejects_and_skips():
    xa, xb, F = _views(40, seed=14)
    oa, ob = _outliers(F, 50, np.random.default_rng(15))
    Fe, info = ga.estimate_F(np.concatenate([xa, oa]), np.concatenate([xb, ob]), _words(256, 16), ga.GaParams())
    assert info[0] == 90 and info[3] == 0 and info[1] < 60
    Fz, info = ga.estimate_F(xa[:15], xb[:15], _words(8, 17), ga.GaParams())
    assert tuple(info) == (15, 0, ga.NONE, 0, 0) and not Fz.any()


def test_refit_does_not_depend_on_the_winning_sample():
    xa, xb, F = _views(120, seed=18, noise=0.4)
    gp = ga.GaParams(thresh_px=4.0, n_hyp=32)
    w1, w2 = _words(32, 19), _words(32, 20)
    F1, i1 = ga.estimate_F(xa, xb, w1, gp)
    F2, i2 = ga.estimate_F(xa, xb, w2, gp)
    Ta, Tb = ga.hartley(xa), ga.hartley(xb)
    h = lambda T, x: np.concatenate([x, np.ones((len(x), 1))], 1) @ T.T
    ha, hb = h(np.eye(3), xa), h(np.eye(3), xb)
    rows = ga.design_rows(h(Ta, xa), h(Tb, xb))
    H = [ga.normalise_F(Tb.T @ ga.rank2(ga.null_f(rows[ga.sample_indices(w[i[2]], 120)])) @ Ta)
         for w, i in ((w1, i1), (w2, i2))]
    # both winners take every match as an inlier, so both refits solve the same least-squares problem
    assert all(np.all(ga.sampson2(Hk, ha, hb) <= 16.0) for Hk in H)
    assert np.abs(F1 - F2).max() < 1e-10 and _same_F(F1, F, 1e-2)
    # while the winning 8-point hypotheses themselves differ on noisy data
    assert np.abs(H[0] - H[1]).max() > 1e-6


def test_ransac_stop_rule_closed_form():
    """(1 - w^8)^N <= 1 - p against the closed form, at points far from equality."""
    for best, m, done, conf, want in ((100, 100, 32, 0.99, True), (75, 100, 32, 0.99, False),
                                      (75, 100, 64, 0.99, True), (50, 100, 256, 0.99, False),
                                      (50, 100, 1280, 0.99, True), (100, 100, 4096, 1.0, False),
                                      (9, 10, 8, 0.9999, False), (9, 10, 64, 0.9999, True)):
        q = (1.0 - (best / m) ** 8) ** done
        assert (q <= 1.0 - conf if conf < 1.0 else False) == want
        assert ga.ransac_stop(best, m, done, conf) == want


def test_ransac_adaptive_batches():
    """Hypotheses run in batches of 32 until the stop rule holds."""
    xa, xb, F = _views(50, seed=21)
    _, info = ga.estimate_F(xa, xb, _words(256, 22), ga.GaParams())
    assert info[1] == 50 and info[4] == 32                      # w = 1 after the first batch
    _, info = ga.estimate_F(xa, xb, _words(256, 22), ga.GaParams(confidence=1.0))
    assert info[4] == 256                                        # no early stop
    xa, xb, F = _views(75, seed=23)
    oa, ob = _outliers(F, 25, np.random.default_rng(24))
    w = _words(256, 25)
    w[0] = [_word(k, 100 - k) for k in range(8)]                 # hypothesis 0 draws inliers only
    _, info = ga.estimate_F(np.concatenate([xa, oa]), np.concatenate([xb, ob]), w, ga.GaParams())
    assert info[1] == 75 and info[4] == 64                       # 0.0341 after 32, 0.00116 after 64
    xa, xb, F = _views(50, seed=26)
    oa, ob = _outliers(F, 50, np.random.default_rng(27))
    _, info = ga.estimate_F(np.concatenate([xa, oa]), np.concatenate([xb, ob]), _words(256, 28), ga.GaParams())
    assert info[4] == 256                                        # w <= 1/2 never stops within 256
