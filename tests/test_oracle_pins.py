"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against exact arithmetic, a closed form, a
hand-derived worked example (tests/golden/), a brute force on tiny inputs or
a structural invariant, chosen so that a dropped term, a wrong sign, a wrong
index or a transposed operand anywhere in the oracle fails at least one.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hash(orc, desc, R, p):
    mu = orc.mean(desc)
    return orc.hash_codes(desc, mu, R, p)


def _popcount_rows(codes_q, codes_c):
    x = np.bitwise_xor(codes_q[:, None, :], codes_c[None, :, :]).view(np.uint8)
    return np.unpackbits(x, axis=-1).sum(axis=-1)


# --------------------------------------------------------------------------
# centring and projection (Sec. 5.1 hash functions)
# --------------------------------------------------------------------------

def test_mean_is_correctly_rounded_rational_mean(orc):
    rng = np.random.default_rng(11)
    for n in (1, 7, 1000, 4099):
        d = rng.integers(0, 256, size=(n, 128), dtype=np.uint8)
        mu = orc.mean(d)
        for j in range(0, 128, 9):
            exact = Fraction(int(d[:, j].astype(np.int64).sum()), n)
            assert mu[j] == float(exact)  # Fraction -> float is correctly rounded


def _exact_projection(x, mu, r):
    return sum(Fraction(float(r[j])) * (Fraction(int(x[j])) - Fraction(float(mu[j]))) for j in range(128))


def test_projection_sign_matches_exact_rational_sign(orc):
    """Ordered-double projection vs exact rational value: the sign agrees
    whenever |v| exceeds the double-precision error bound, and the error is
    within that bound (Higham's gamma_n for a recursive sum of rounded
    products of rounded differences)."""
    rng = np.random.default_rng(12)
    desc = synth.sift_like(rng, 64)
    mu = orc.mean(desc)
    R = rng.standard_normal((8, 128))
    u = 2.0 ** -53
    gamma = 131 * u / (1 - 131 * u)
    checked = 0
    for f in range(desc.shape[0]):
        for b in range(R.shape[0]):
            x, r = desc[f], R[b]
            v = orc.projection(x, mu, r)
            ex = _exact_projection(x, mu, r)
            bound = gamma * float(sum(abs(Fraction(float(r[j])) * (int(x[j]) - Fraction(float(mu[j]))))
                                      for j in range(128)))
            assert abs(Fraction(v) - ex) <= Fraction(bound)
            if abs(ex) > Fraction(bound):
                assert (v > 0) == (ex > 0)
            checked += 1
    assert checked == 512


def test_block_projections_are_the_pinned_projection_and_give_the_codes(orc):
    """oracle.projections (the values the GPU's rounding bounds are measured
    against) equals the pinned per-element projection bit for bit, and its
    signs reproduce oracle_hash's code bits and bucket ids."""
    rng = np.random.default_rng(21)
    desc = synth.sift_like(rng, 300)
    mu = orc.mean(desc)
    R = synth.projection_matrix(21)
    po = orc.params()
    rows = 128 + 6 * 8
    v = orc.projections(desc, mu, R, rows, threads=3)
    for f in (0, 7, 150, 299):
        for b in (0, 31, 127, 128, 175):
            assert v[f, b] == orc.projection(desc[f], mu, R[b])
    codes, buckets = orc.hash_codes(desc, mu, R, po)
    bits = (v > 0.0)
    words = np.zeros((300, 4), np.uint32)
    for b in range(128):
        words[:, b // 32] |= bits[:, b].astype(np.uint32) << np.uint32(b % 32)
    assert np.array_equal(words, codes)
    ids = np.zeros((300, 6), np.uint8)
    for t in range(6):
        for i in range(8):
            ids[:, t] |= (bits[:, 128 + 8 * t + i].astype(np.uint8) << np.uint8(i))
    assert np.array_equal(ids, buckets)


def test_projection_near_zero_cases(orc):
    """Rows built so that the projection nearly cancels: the double result
    stays within the bound of the exact rational value and keeps its sign
    whenever the exact value is outside the bound."""
    rng = np.random.default_rng(13)
    desc = synth.sift_like(rng, 32)
    mu = orc.mean(desc)
    u = 2.0 ** -53
    gamma = 131 * u / (1 - 131 * u)
    for f in range(32):
        x = desc[f]
        t = x.astype(np.float64) - mu
        r = rng.standard_normal(128)
        k = int(np.argmax(np.abs(t)))
        r[k] = 0.0
        r[k] = -np.dot(r, t) / t[k]
        r[k] *= 1.0 + rng.uniform(-1e-15, 1e-15)
        v = orc.projection(x, mu, r)
        ex = _exact_projection(x, mu, r)
        bound = gamma * float(sum(abs(Fraction(float(r[j])) * (int(x[j]) - Fraction(float(mu[j]))))
                                  for j in range(128)))
        assert abs(Fraction(v) - ex) <= Fraction(bound)
        if abs(ex) > Fraction(bound):
            assert (v > 0) == (ex > 0)


def test_axis_aligned_projection_closed_form(orc):
    """With r_b = s_b * e_{pi(b)} the projection is s_b (x_pi(b) - mu_pi(b)),
    so bit b = [x_pi(b) > mu_pi(b)] for s_b > 0 and [x < mu] for s_b < 0.
    Pins the row-to-bit order, the word layout of the code, the bucket bit
    order and the mean."""
    rng = np.random.default_rng(14)
    desc = synth.sift_like(rng, 300)
    nb, T, m = 128, 6, 8
    rows = nb + T * m
    perm = rng.permutation(np.concatenate([np.arange(128), rng.integers(0, 128, size=rows - 128)]))
    sgn = np.where(rng.random(rows) < 0.5, -1.0, 1.0)
    scale = rng.uniform(0.5, 3.0, size=rows)
    R = np.zeros((rows, 128))
    R[np.arange(rows), perm] = sgn * scale
    p = orc.params(code_bits=nb, n_tables=T, bits_per_table=m)
    codes, buckets = _hash(orc, desc, R, p)
    S = desc.astype(np.int64).sum(axis=0)
    n = desc.shape[0]
    # x > mu  <=>  n x > S, exactly in integers
    gt = desc.astype(np.int64) * n > S[None, :]
    lt = desc.astype(np.int64) * n < S[None, :]
    bits = np.where(sgn[None, :] > 0, gt[:, perm], lt[:, perm])
    exp_codes = np.zeros((n, 4), np.uint32)
    for b in range(nb):
        exp_codes[:, b >> 5] |= (bits[:, b].astype(np.uint32) << np.uint32(b & 31))
    assert np.array_equal(codes, exp_codes)
    exp_b = np.zeros((n, T), np.uint8)
    for t in range(T):
        for i in range(m):
            exp_b[:, t] |= (bits[:, nb + t * m + i].astype(np.uint8) << np.uint8(i))
    assert np.array_equal(buckets, exp_b)


def test_single_descriptor_gives_all_zero_codes(orc):
    """N = 1: the mean is the descriptor, every centred component is exactly
    zero, every projection is exactly 0 and the strict sign test gives 0."""
    rng = np.random.default_rng(15)
    d = synth.sift_like(rng, 1)
    R = synth.projection_matrix(15)
    codes, buckets = _hash(orc, d, R, orc.params())
    assert not codes.any() and not buckets.any()


def test_identical_descriptors_give_identical_zero_codes(orc):
    rng = np.random.default_rng(16)
    d = np.repeat(synth.sift_like(rng, 1), 50, axis=0)
    codes, buckets = _hash(orc, d, synth.projection_matrix(16), orc.params())
    assert not codes.any() and not buckets.any()


def test_codes_deterministic_and_order_independent(orc):
    """Codes depend only on the descriptor, the mean and R (same seed, same
    codes; permuting the set permutes the codes)."""
    s = synth.random_set(17, [200, 150])
    p = orc.params()
    c1, b1 = _hash(orc, s.desc, s.R, p)
    c2, b2 = _hash(orc, s.desc, s.R, p)
    assert np.array_equal(c1, c2) and np.array_equal(b1, b2)
    perm = np.random.default_rng(0).permutation(s.desc.shape[0])
    mu = orc.mean(s.desc)
    c3, b3 = orc.hash_codes(s.desc[perm], mu, s.R, p)
    assert np.array_equal(c3, c1[perm]) and np.array_equal(b3, b1[perm])


# --------------------------------------------------------------------------
# worked examples derived by hand (tests/golden)
# --------------------------------------------------------------------------

def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _pad(rows):
    out = np.zeros((len(rows), 128), np.uint8)
    for i, r in enumerate(rows):
        out[i, :len(r)] = r
    return out


def test_golden_axis_worked_example(orc):
    g = _golden("axis_worked_example.json")
    gp = g["params"]
    p = orc.params(code_bits=gp["code_bits"], n_tables=gp["n_tables"], bits_per_table=gp["bits_per_table"],
                   top_k=gp["top_k"], ratio=tuple(gp["ratio"]))
    A, B = _pad(g["A"]), _pad(g["B"])
    R = np.zeros((5, 128))
    R[np.arange(5), np.arange(5)] = 1.0
    mu = orc.mean(np.concatenate([A, B]))
    assert np.allclose(mu[:5], g["mean_first5"], rtol=0, atol=1e-15)
    cA, bA = orc.hash_codes(A, mu, R, p)
    cB, bB = orc.hash_codes(B, mu, R, p)
    assert cA[:, 0].tolist() == g["codes_A"] and cB[:, 0].tolist() == g["codes_B"]
    assert not cA[:, 1:].any() and not cB[:, 1:].any()
    assert bA[:, 0].tolist() == g["buckets_A"] and bB[:, 0].tolist() == g["buckets_B"]
    m, det = orc.match_pair(A, cA, bA, B, cB, bB, p, detail=True)
    assert m.tolist() == g["match_A"]
    assert list(det[0].top_h[:det[0].n_top]) == g["top_h_A0"]
    assert list(det[0].top_d[:det[0].n_top]) == g["top_d_A0"]
    p1 = orc.params(code_bits=4, n_tables=1, bits_per_table=1, top_k=1, ratio=(4, 5))
    assert orc.match_pair(A, cA, bA, B, cB, bB, p1).tolist() == g["match_A_k1"]


def test_golden_ratio_boundary(orc):
    g = _golden("ratio_boundary_example.json")
    gp = g["params"]
    p = orc.params(code_bits=gp["code_bits"], n_tables=gp["n_tables"], bits_per_table=gp["bits_per_table"],
                   top_k=gp["top_k"], ratio=tuple(gp["ratio"]))
    R = synth.projection_matrix(1, rows=128)
    for case in g["cases"]:
        A = np.full((1, 128), g["x_value"], np.uint8)
        B = np.repeat(A, len(case["B_offsets"]), axis=0)
        for i, offs in enumerate(case["B_offsets"]):
            for dim, delta in offs:
                B[i, dim] += delta
        mu = orc.mean(np.concatenate([A, B]))
        cA, bA = orc.hash_codes(A, mu, R, p)
        cB, bB = orc.hash_codes(B, mu, R, p)
        m, det = orc.match_pair(A, cA, bA, B, cB, bB, p, detail=True)
        assert m.tolist() == [case["match"]]
        assert sorted(det[0].top_d[:det[0].n_top]) == case["d"]


# --------------------------------------------------------------------------
# Steps 1-4 against brute force on tiny inputs
# --------------------------------------------------------------------------

def _pair(orc, seed, nA, nB, p):
    s = synth.random_set(seed, [nA, nB])
    codes, buckets = _hash(orc, s.desc, s.R[:p.code_bits + p.n_tables * p.bits_per_table], p)
    A, B = slice(0, nA), slice(nA, nA + nB)
    return s.desc[A], codes[A], buckets[A], s.desc[B], codes[B], buckets[B]


@pytest.mark.parametrize("m,T", [(2, 3), (3, 6), (1, 1), (4, 2)])
def test_candidate_sets_and_ranking_match_brute_force(orc, m, T):
    """Step 1 (any-table bucket equality, as a set) and Step 3 (k smallest
    (Hamming, index) keys) re-derived by brute force over every point of B
    with numpy bit unpacking and a lexicographic sort."""
    p = orc.params(n_tables=T, bits_per_table=m, top_k=7)
    dA, cA, bA, dB, cB, bB = _pair(orc, 20 + m * 10 + T, 60, 90, p)
    _, det = orc.match_pair(dA, cA, bA, dB, cB, bB, p, detail=True)
    H = _popcount_rows(cA, cB)
    same = (bA[:, None, :] == bB[None, :, :]).any(axis=2)
    for q in range(dA.shape[0]):
        cand = np.nonzero(same[q])[0]
        assert det[q].n_cand == cand.size
        order = np.lexsort((cand, H[q, cand]))
        exp = cand[order][:7]
        got = np.array(det[q].top_j[:det[q].n_top])
        assert np.array_equal(got, exp)
        assert np.array_equal(np.array(det[q].top_h[:det[q].n_top]), H[q, exp])


@pytest.mark.parametrize("seed", [30, 31, 32])
def test_one_bucket_and_large_k_is_brute_force_nearest_neighbour(orc, seed):
    """m = 0 puts every point of B in one bucket and k >= |B| keeps all of
    them, so Steps 1-4 reduce to exact nearest neighbour with Lowe's ratio
    test, computed here from the full integer distance matrix."""
    nA, nB = 40, 50
    p = orc.params(n_tables=1, bits_per_table=0, top_k=64)
    dA, cA, bA, dB, cB, bB = _pair(orc, seed, nA, nB, p)
    m = orc.match_pair(dA, cA, bA, dB, cB, bB, p)
    D = ((dA[:, None, :].astype(np.int64) - dB[None, :, :].astype(np.int64)) ** 2).sum(axis=2)
    exp = np.full(nA, -1)
    for q in range(nA):
        order = np.lexsort((np.arange(nB), D[q]))
        d1, d2 = D[q, order[0]], D[q, order[1]]
        if np.sqrt(d1) < 0.8 * np.sqrt(d2) and 25 * d1 < 16 * d2:
            exp[q] = order[0]
    assert np.array_equal(m, exp)
    assert (m >= 0).sum() > 5


def test_structural_invariants(orc):
    p = orc.params(n_tables=6, bits_per_table=4, top_k=10)
    dA, cA, bA, dB, cB, bB = _pair(orc, 40, 120, 130, p)
    m, det = orc.match_pair(dA, cA, bA, dB, cB, bB, p, detail=True)
    H = _popcount_rows(cA, cB)
    assert np.array_equal(H, _popcount_rows(cB, cA).T)      # Hamming symmetric
    same = (bA[:, None, :] == bB[None, :, :]).any(axis=2)
    D = ((dA[:, None, :].astype(np.int64) - dB[None, :, :].astype(np.int64)) ** 2).sum(axis=2)
    for q, d in enumerate(det):
        assert d.n_top == min(10, d.n_cand)
        top = list(d.top_j[:d.n_top])
        assert len(set(top)) == len(top)
        assert all(same[q, j] for j in top)                  # top-K subset of candidates
        keys = [(d.top_h[i], top[i]) for i in range(d.n_top)]
        assert keys == sorted(keys)
        rest = [(H[q, j], j) for j in np.nonzero(same[q])[0] if j not in top]
        if rest and keys:
            assert min(rest) > keys[-1]                     # every other key is larger
        assert [d.top_d[i] for i in range(d.n_top)] == [D[q, j] for j in top]
        if d.n_top >= 2:
            assert d.d1 <= d.d2
        if m[q] >= 0:
            assert d.n_top >= 2 and 25 * d.d1 < 16 * d.d2 and D[q, m[q]] == d.d1
    # matching an image against itself: each query finds itself at Hamming 0
    m2, det2 = orc.match_pair(dA, cA, bA, dA, cA, bA, p, detail=True)
    for q, d in enumerate(det2):
        assert d.top_h[0] == 0 and d.d1 == 0


def test_degenerate_images(orc):
    p = orc.params()
    dA, cA, bA, dB, cB, bB = _pair(orc, 50, 30, 1, p)
    assert (orc.match_pair(dA, cA, bA, dB, cB, bB, p) == -1).all()              # |B| = 1
    e = np.zeros((0, 128), np.uint8)
    assert (orc.match_pair(dA, cA, bA, e, np.zeros((0, 4), np.uint32), np.zeros((0, 6), np.uint8), p) == -1).all()
    assert orc.match_pair(e, np.zeros((0, 4), np.uint32), np.zeros((0, 6), np.uint8), dA, cA, bA, p).size == 0
    # identical descriptors: every distance 0, ratio test always fails
    same = np.repeat(dA[:1], 20, axis=0)
    c, b = _hash(orc, same, synth.projection_matrix(50), p)
    assert (orc.match_pair(same, c, b, same, c, b, p) == -1).all()


def test_tau_threshold_drops_far_candidates(orc):
    """Sec. 6: candidates with Hamming distance above tau are not ranked."""
    p0 = orc.params(top_k=10)
    dA, cA, bA, dB, cB, bB = _pair(orc, 60, 200, 220, p0)
    _, d0 = orc.match_pair(dA, cA, bA, dB, cB, bB, p0, detail=True)
    p1 = orc.params(top_k=10, tau=40)
    _, d1 = orc.match_pair(dA, cA, bA, dB, cB, bB, p1, detail=True)
    for a, b in zip(d0, d1):
        assert all(h <= 40 for h in b.top_h[:b.n_top])
        exp = [(a.top_h[i], a.top_j[i]) for i in range(a.n_top) if a.top_h[i] <= 40]
        got = [(b.top_h[i], b.top_j[i]) for i in range(b.n_top)]
        assert got[:len(exp)] == exp


def test_multi_pair_driver_equals_single_pairs(orc):
    s = synth.random_set(70, [50, 0, 80, 1, 65])
    p = orc.params(bits_per_table=5)
    mu = orc.mean(s.desc)
    codes, buckets = orc.hash_codes(s.desc, mu, s.R, p)
    for nt in (1, 3):
        off, mt = orc.match_pairs(s.desc, s.img_off, codes, buckets, s.pairs, p, n_threads=nt)
        for i, (a, b) in enumerate(s.pairs):
            A = slice(int(s.img_off[a]), int(s.img_off[a + 1]))
            B = slice(int(s.img_off[b]), int(s.img_off[b + 1]))
            m = orc.match_pair(s.desc[A], codes[A], buckets[A], s.desc[B], codes[B], buckets[B], p)
            q = np.nonzero(m >= 0)[0]
            exp = np.stack([q, m[q]], axis=1) if q.size else np.zeros((0, 2))
            got = mt[int(off[i]):int(off[i + 1])]
            assert np.array_equal(got, exp)


# --------------------------------------------------------------------------
# Sec. 7.2 epipolar band
# --------------------------------------------------------------------------

def _two_views(rng):
    def rot(a, b, c):
        ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
        Rx = np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]])
        Ry = np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
        Rz = np.array([[cc, -sc, 0], [sc, cc, 0], [0, 0, 1]])
        return Rz @ Ry @ Rx
    K = np.array([[1000.0, 0, 960], [0, 1000.0, 540], [0, 0, 1]])
    R1, t1 = np.eye(3), np.zeros(3)
    R2 = rot(0.05, -0.2, 0.03)
    t2 = np.array([-0.8, 0.1, 0.05])
    X = rng.uniform(-1, 1, size=(400, 3)) + np.array([0, 0, 5.0])
    def proj(R, t):
        Y = (R @ X.T).T + t
        y = (K @ Y.T).T
        return y[:, :2] / y[:, 2:3]
    # F maps a point of view 1 to its line in view 2: x2^T F x1 = 0
    Rr = R2 @ R1.T
    tr = t2 - Rr @ t1
    tx = np.array([[0, -tr[2], tr[1]], [tr[2], 0, -tr[0]], [-tr[1], tr[0], 0]])
    F = np.linalg.inv(K).T @ tx @ Rr @ np.linalg.inv(K)
    return proj(R1, t1), proj(R2, t2), F


def test_epipolar_predicate_against_geometry(orc):
    """Noise-free correspondences lie on their epipolar lines (kept at 4 px);
    the kept/dropped decision agrees with the point-to-line distance computed
    independently from the line's direction vector, away from the boundary."""
    rng = np.random.default_rng(80)
    x1, x2, F = _two_views(rng)
    x1 = x1.astype(np.float32)
    x2 = x2.astype(np.float32)
    for i in range(x1.shape[0]):
        assert orc.epipolar_keep(F, x1[i, 0], x1[i, 1], x2[i, 0], x2[i, 1], 4.0)
    for i in range(200):
        q = rng.integers(0, x1.shape[0])
        pc = x2[rng.integers(0, x2.shape[0])] + rng.normal(0, 10, size=2).astype(np.float32)
        pc = pc.astype(np.float32)
        l = F @ np.array([x1[q, 0], x1[q, 1], 1.0], dtype=np.float64)
        # two points on the line, then the perpendicular distance by the cross product
        if abs(l[1]) > abs(l[0]):
            p0 = np.array([0.0, -l[2] / l[1]]); dvec = np.array([1.0, -l[0] / l[1]])
        else:
            p0 = np.array([-l[2] / l[0], 0.0]); dvec = np.array([-l[1] / l[0], 1.0])
        w = pc.astype(np.float64) - p0
        dist = abs(w[0] * dvec[1] - w[1] * dvec[0]) / np.hypot(dvec[0], dvec[1])
        keep = orc.epipolar_keep(F, x1[q, 0], x1[q, 1], pc[0], pc[1], 4.0)
        if abs(dist - 4.0) > 1e-6:
            assert keep == (dist <= 4.0)
    # with N(0,1) pixel jitter in both views, nearly all true pairs stay in a 4 px band
    j1 = x1 + rng.normal(0, 1, size=x1.shape).astype(np.float32)
    j2 = x2 + rng.normal(0, 1, size=x2.shape).astype(np.float32)
    kept = sum(orc.epipolar_keep(F, j1[i, 0], j1[i, 1], j2[i, 0], j2[i, 1], 4.0) for i in range(x1.shape[0]))
    assert kept >= 0.99 * x1.shape[0]


def test_epipolar_band_filters_before_ranking(orc):
    """Sec. 7.2 step order: the band is applied to the lookup candidates
    before the ranking, so every ranked candidate is inside the band, and
    with an infinite band the result equals the unguided one."""
    rng = np.random.default_rng(81)
    x1, x2, F = _two_views(rng)
    n = x1.shape[0]
    p = orc.params(bits_per_table=3)
    dA, cA, bA, dB, cB, bB = _pair(orc, 82, n, n, p)
    kA, kB = x1.astype(np.float32), x2.astype(np.float32)
    pe = orc.params(bits_per_table=3, epi_px=4.0)
    m, det = orc.match_pair(dA, cA, bA, dB, cB, bB, pe, F=F.ravel(), kptsA=kA, kptsB=kB, detail=True)
    for q, d in enumerate(det):
        for j in d.top_j[:d.n_top]:
            assert orc.epipolar_keep(F, kA[q, 0], kA[q, 1], kB[j, 0], kB[j, 1], 4.0)
    pinf = orc.params(bits_per_table=3, epi_px=1e30)
    assert np.array_equal(orc.match_pair(dA, cA, bA, dB, cB, bB, pinf, F=F.ravel(), kptsA=kA, kptsB=kB),
                          orc.match_pair(dA, cA, bA, dB, cB, bB, p))


# --------------------------------------------------------------------------
# statistics on the planted one-pair workload (sanity, not parity)
# --------------------------------------------------------------------------

def test_planted_copies_are_recovered(orc):
    s = synth.config0()
    mu = orc.mean(s.desc)
    codes, buckets = orc.hash_codes(s.desc, mu, s.R)
    A, B = slice(0, 2000), slice(2000, 4000)
    m = orc.match_pair(s.desc[A], codes[A], buckets[A], s.desc[B], codes[B], buckets[B])
    truth = {int(a): r for r, a in enumerate(s.truth["b_from_a"]) if a >= 0}
    good = sum(1 for q, r in truth.items() if m[q] == r)
    assert good / len(truth) > 0.95
    assert good / max(1, int((m >= 0).sum())) > 0.99


# --------------------------------------------------------------------------
# flags of the next scope row: single-candidate acceptance, mutual check
# --------------------------------------------------------------------------

def test_single_candidate_acceptance_against_bucket_counts(orc):
    """ACCEPT_SINGLE changes exactly the queries with one candidate: each then
    matches that candidate (counted by brute-force bucket equality); queries
    with two or more candidates are unchanged, with none stay unmatched."""
    p0 = orc.params(n_tables=1, bits_per_table=8, top_k=10)
    p1 = orc.params(n_tables=1, bits_per_table=8, top_k=10, flags=orc.ACCEPT_SINGLE)
    dA, cA, bA, dB, cB, bB = _pair(orc, 91, 300, 260, p0)
    m0 = orc.match_pair(dA, cA, bA, dB, cB, bB, p0)
    m1 = orc.match_pair(dA, cA, bA, dB, cB, bB, p1)
    same = bA[:, 0][:, None] == bB[:, 0][None, :]
    ncand = same.sum(axis=1)
    one = ncand == 1
    assert one.sum() > 20 and (ncand >= 2).sum() > 20
    assert np.array_equal(m1[one], np.argmax(same[one], axis=1))
    assert np.all(m0[one] == -1)
    assert np.array_equal(m1[~one], m0[~one])


@pytest.mark.parametrize("seed", [40, 41])
def test_mutual_check_is_brute_force_cross_check(orc, seed):
    """With one bucket (m = 0) and k >= both image sizes, matching is exact
    nearest neighbour + ratio test in each direction; MUTUAL keeps (q, j)
    exactly when the forward match of q is j and the backward match of j is
    q, both computed here from the integer distance matrix."""
    nA, nB = 45, 55
    p = orc.params(n_tables=1, bits_per_table=0, top_k=64, flags=orc.MUTUAL)
    s = synth.random_set(seed, [nA, nB])
    s.desc[nA:nA + 30] = synth.noisy_copy(np.random.default_rng(seed), s.desc[:30], 4.0)  # some true pairs
    codes, buckets = _hash(orc, s.desc, s.R[:p.code_bits + p.n_tables * p.bits_per_table], p)
    off, mt = orc.match_pairs(s.desc, s.img_off, codes, buckets, np.array([[0, 1]], np.uint32), p)

    def nn_ratio(X, Y):
        D = ((X[:, None, :].astype(np.int64) - Y[None, :, :].astype(np.int64)) ** 2).sum(axis=2)
        out = np.full(X.shape[0], -1)
        for q in range(X.shape[0]):
            order = np.lexsort((np.arange(Y.shape[0]), D[q]))
            if 25 * D[q, order[0]] < 16 * D[q, order[1]]:
                out[q] = order[0]
        return out

    A, B = s.desc[:nA], s.desc[nA:]
    fw, bw = nn_ratio(A, B), nn_ratio(B, A)
    exp = [(q, fw[q]) for q in range(nA) if fw[q] >= 0 and bw[fw[q]] == q]
    assert [tuple(r) for r in mt.tolist()] == exp
    assert len(exp) >= 10 and len(exp) < (fw >= 0).sum() + 1


def test_mutual_check_with_the_band_is_symmetric(orc):
    """Mutual lists of (A, B) under F are the transposed lists of (B, A) under
    F^T: the reverse match must use the transposed fundamental matrix (and the
    swapped key-points), or the two disagree."""
    rng = np.random.default_rng(95)
    x1, x2, F = _two_views(rng)
    n = x1.shape[0]
    base = synth.sift_like(rng, n)
    desc = np.concatenate([synth.noisy_copy(rng, base, 6.0), synth.noisy_copy(rng, base, 6.0)])
    kp = np.concatenate([x1, x2]).astype(np.float32) + rng.normal(0, 1, size=(2 * n, 2)).astype(np.float32)
    img_off = np.array([0, n, 2 * n], np.uint64)
    R = synth.projection_matrix(95)
    p = orc.params(n_tables=6, bits_per_table=5, top_k=10, epi_px=4.0, flags=orc.MUTUAL)
    codes, buckets = _hash(orc, desc, R[:p.code_bits + p.n_tables * p.bits_per_table], p)
    Fs = np.stack([F.ravel(), F.T.ravel()])
    off, mt = orc.match_pairs(desc, img_off, codes, buckets, np.array([[0, 1], [1, 0]], np.uint32), p,
                              F=Fs, kpts=kp)
    fw = mt[int(off[0]):int(off[1])]
    bw = mt[int(off[1]):int(off[2])]
    assert len(fw) > 50
    assert sorted(map(tuple, fw.tolist())) == sorted((int(j), int(q)) for q, j in bw.tolist())
    # a plain forward run keeps at least these, mostly more
    p_plain = orc.params(n_tables=6, bits_per_table=5, top_k=10, epi_px=4.0)
    off2, mt2 = orc.match_pairs(desc, img_off, codes, buckets, np.array([[0, 1]], np.uint32), p_plain,
                                F=Fs[:1], kpts=kp)
    assert set(map(tuple, fw.tolist())) <= set(map(tuple, mt2.tolist()))
