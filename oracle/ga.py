"""CPU oracle of the Ga-CasHash first stage -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product library never does.

Sec. 7.1 (first stage of Ga-CasHash): the top 20 % of each image's features
by SIFT scale are matched exhaustively with CasHash; for a pair with at least
16 matches the fundamental matrix is estimated, and the pair goes on to the
guided matching of Sec. 7.2 when at least 2/3 of its matches are inliers.
The paper names no estimator; this follows the published normalised 8-point
algorithm (Hartley, "In defense of the eight-point algorithm", 1997) inside
RANSAC (Fischler and Bolles, 1981), with the Sampson distance (Hartley and
Zisserman, Multiple View Geometry, 2nd ed., Sec. 11.4.3) as the inlier test.
Plain numpy in float64; the random draws of RANSAC are inputs (uint32 words).

Readings where the paper is silent (each is also a parameter):
  * "top 20 % scale": per image the ceil(n * pct / 100) features of largest
    scale, ties to the lower feature index, kept in feature order;
  * stage-1 codes are the full set's codes of those features (the same centre
    and projection), so stage-1 matching is CasHash restricted to the subsets;
  * RANSAC: at most n_hyp hypotheses per pair, each from 8 distinct matches
    drawn by the word-to-index map below, in batches of 32 with the adaptive
    stop of Hartley and Zisserman (Algorithm 4.5): after a batch, stop when
    (1 - w^8)^N <= 1 - confidence, N the hypotheses done and w the best inlier
    fraction so far (w^8 by three squarings, the power by binary
    exponentiation, every step one correctly rounded double operation); a
    match is an inlier when its squared Sampson distance is at most
    thresh_px^2; the hypothesis with the most inliers wins (ties to the lower
    index) and F is refitted on its inliers (least squares, same
    normalisation) when it has at least 8;
  * the accepted pair's F is the refit, scaled to unit Frobenius norm with its
    largest-magnitude entry (first on ties) positive.
Convention: x_B^T F x_A = 0 for a query point x_A of image A and its match
x_B in image B (pair (A, B)).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import hash_codes, match_pairs

NONE = 0xFFFFFFFF


@dataclasses.dataclass
class GaParams:
    top_pct: int = 20         # percent of each image's features kept by scale
    min_matches: int = 16     # fewer stage-1 matches: no F
    n_hyp: int = 256          # RANSAC hypotheses per pair
    inlier_num: int = 2       # accepted when den * inliers >= num * matches
    inlier_den: int = 3
    thresh_px: float = 3.0    # Sampson distance threshold, pixels
    confidence: float = 0.99  # adaptive stop; >= 1 runs all n_hyp hypotheses


BATCH = 32  # hypotheses between two checks of the adaptive stop


def top_scale(scale: np.ndarray, img_off: np.ndarray, pct: int):
    """Selected global feature indices (ascending within each image) and the
    subset's image offsets: image i keeps ceil(n_i * pct / 100) features of
    largest scale, ties to the lower index."""
    sel, off = [], [0]
    for i in range(len(img_off) - 1):
        a, b = int(img_off[i]), int(img_off[i + 1])
        n = b - a
        k = (n * pct + 99) // 100
        s = scale[a:b].astype(np.float32)
        order = np.lexsort((np.arange(n), -s.astype(np.float64)))  # scale descending, index ascending
        sel.append(np.sort(order[:k]) + a)
        off.append(off[-1] + k)
    sel = np.concatenate(sel).astype(np.uint64) if sel else np.zeros(0, np.uint64)
    return sel, np.array(off, np.uint64)


def sample_indices(words, m: int):
    """8 distinct match indices from 8 uint32 words: r_k = floor(u_k (m - k) /
    2^32) picks the r_k-th smallest index not drawn before."""
    picked = []
    for k in range(8):
        r = (int(words[k]) * (m - k)) >> 32
        v = r
        for p in sorted(picked):
            if p <= v:
                v += 1
        picked.append(v)
    return picked


def hartley(pts: np.ndarray) -> np.ndarray:
    """Similarity T moving the centroid of pts to the origin and scaling the
    mean distance from it to sqrt(2)."""
    c = pts.mean(axis=0)
    md = np.sqrt(((pts - c) ** 2).sum(axis=1)).mean()
    s = np.sqrt(2.0) / md
    return np.array([[s, 0.0, -s * c[0]], [0.0, s, -s * c[1]], [0.0, 0.0, 1.0]])


def _homog(T: np.ndarray, pts: np.ndarray) -> np.ndarray:
    h = np.concatenate([pts, np.ones((len(pts), 1))], axis=1)
    return h @ T.T


def design_rows(xa: np.ndarray, xb: np.ndarray) -> np.ndarray:
    """Rows of x_B^T F x_A = 0 in f = F row-major: entry (i, j) of F multiplies
    x_B[i] * x_A[j]."""
    return np.einsum("ni,nj->nij", xb, xa).reshape(len(xa), 9)


def null_f(A: np.ndarray) -> np.ndarray:
    """Least-squares f (unit norm) minimising |A f|: the last right singular
    vector (for 8 rows, the null vector)."""
    return np.linalg.svd(A)[2][-1].reshape(3, 3)


def rank2(F: np.ndarray) -> np.ndarray:
    """Closest rank-2 matrix in the Frobenius norm (smallest singular value set to 0)."""
    U, S, Vt = np.linalg.svd(F)
    S = S.copy()
    S[2] = 0.0
    return (U * S) @ Vt


def normalise_F(F: np.ndarray) -> np.ndarray:
    F = F / np.linalg.norm(F)
    f = F.ravel()
    i = int(np.argmax(np.abs(f)))  # first index of the largest magnitude
    return F if f[i] > 0 else -F


def sampson2(F: np.ndarray, xa: np.ndarray, xb: np.ndarray) -> np.ndarray:
    """Squared Sampson distance of each correspondence (homogeneous rows)."""
    Fx = xa @ F.T           # F x_A
    Ftx = xb @ F            # F^T x_B
    num = np.einsum("ni,ni->n", xb, Fx) ** 2
    den = Fx[:, 0] ** 2 + Fx[:, 1] ** 2 + Ftx[:, 0] ** 2 + Ftx[:, 1] ** 2
    return num / den


def ransac_stop(best: int, m: int, done: int, confidence: float) -> bool:
    """Adaptive stop: (1 - w^8)^done <= 1 - confidence with w = best / m."""
    if not confidence < 1.0:
        return False
    w = best / m
    w2 = w * w
    w4 = w2 * w2
    base = 1.0 - w4 * w4
    r = 1.0
    e = done
    while e:
        if e & 1:
            r = r * base
        base = base * base
        e >>= 1
    return r <= 1.0 - confidence


def estimate_F(pa: np.ndarray, pb: np.ndarray, words: np.ndarray, gp: GaParams):
    """RANSAC + normalised 8-point on the matched key-points pa (image A) and
    pb (image B), [m][2] float.  Returns (F [3][3] or zeros, info) with info =
    (n_matches, n_inliers, best_hyp, accepted, hypotheses evaluated)."""
    m = len(pa)
    if m < gp.min_matches:
        return np.zeros((3, 3)), (m, 0, NONE, 0, 0)
    pa = pa.astype(np.float64)
    pb = pb.astype(np.float64)
    Ta, Tb = hartley(pa), hartley(pb)
    na, nb = _homog(Ta, pa), _homog(Tb, pb)
    xa, xb = _homog(np.eye(3), pa), _homog(np.eye(3), pb)
    rows = design_rows(na, nb)
    t2 = gp.thresh_px * gp.thresh_px
    best, best_h, best_F = -1, NONE, None
    done = 0
    while done < gp.n_hyp:
        end = min(done + BATCH, gp.n_hyp)
        for h in range(done, end):
            idx = sample_indices(words[h], m)
            Fn = rank2(null_f(rows[idx]))
            F = Tb.T @ Fn @ Ta
            if not np.all(np.isfinite(F)):
                continue
            cnt = int(np.count_nonzero(sampson2(F, xa, xb) <= t2))
            if cnt > best:
                best, best_h, best_F = cnt, h, F
        done = end
        if best_F is not None and ransac_stop(best, m, done, gp.confidence):
            break
    if best_F is None:
        return np.zeros((3, 3)), (m, 0, NONE, 0, done)
    F = best_F
    inl = sampson2(F, xa, xb) <= t2
    if np.count_nonzero(inl) >= 8:
        F = Tb.T @ rank2(null_f(rows[inl])) @ Ta
    F = normalise_F(F)
    n_in = int(np.count_nonzero(sampson2(F, xa, xb) <= t2))
    acc = int(gp.inlier_den * n_in >= gp.inlier_num * m)
    return F, (m, n_in, best_h, acc, done)


def stage1(desc, img_off, kpts, scale, mu, R, pairs, po, gp: GaParams, words):
    """The whole first stage: subset selection, CasHash matching of the
    subsets (codes with the full set's centre mu), F per pair.  Returns
    (F [P][9], info [P][5] uint32, sel, sub_off, (match offsets, matches))."""
    sel, sub_off = top_scale(scale, img_off, gp.top_pct)
    sel_i = sel.astype(np.int64)
    d_sub = np.ascontiguousarray(desc[sel_i])
    k_sub = np.ascontiguousarray(kpts[sel_i])
    codes, buckets = hash_codes(d_sub, mu, R, po)
    moff, mt = match_pairs(d_sub, sub_off, codes, buckets, pairs, po)
    P = len(pairs)
    F = np.zeros((P, 9))
    info = np.zeros((P, 5), np.uint32)
    for p in range(P):
        a, b = int(pairs[p][0]), int(pairs[p][1])
        lo, hi = int(moff[p]), int(moff[p + 1])
        q = mt[lo:hi, 0].astype(np.int64) + int(sub_off[a])
        j = mt[lo:hi, 1].astype(np.int64) + int(sub_off[b])
        Fp, inf = estimate_F(k_sub[q], k_sub[j], words[p], gp)
        F[p] = Fp.ravel()
        info[p] = inf
    return F, info, sel, sub_off, (moff, mt)
