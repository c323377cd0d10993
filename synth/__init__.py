"""Seeded synthetic inputs for Cascade Hashing image matching.

This module draws inputs only -- descriptors, the random projection matrix,
image pair lists, key-points and fundamental matrices.  It holds none of the
matching method's arithmetic (no hashing, ranking or distances), so both the
CPU oracle and the CUDA path can consume it.

Descriptor recipe (stands in for real SIFT, which the paper matches on
Oxford/Cornell data sets not available here): each of the 128 components is
|N(0,1)|; the vector is L2-normalised, clipped at 0.2, renormalised (the SIFT
normalisation), scaled by 512, rounded half-to-even and clipped to 0..255.
A "noisy copy" adds N(0, sigma^2) per component and requantises the same way.

Workloads (sizes as in the benchmark configurations):
  config0  one pair, A = 2,000 descriptors, B = 1,000 noisy copies of A plus
           1,000 fresh ones, permuted
  config1  100 images, 4,000..12,000 descriptors each, 30 % noisy copies of
           descriptors of the 5 index-neighbours on each side; all 4,950 pairs
  config3  2,000 images, log-uniform 1,000..20,000 descriptors, 30 random
           neighbours each (pairs deduplicated, about 59,000)
  config4  500 pinhole views of 200,000 points in the unit cube with key-points,
           30 % clutter and ground-truth fundamental matrices (epipolar form)
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

DIM = 128


def sift_like(rng: np.random.Generator, n: int) -> np.ndarray:
    """n SIFT-like uint8 descriptors (recipe in the module docstring)."""
    out = np.empty((n, DIM), np.uint8)
    step = 65536
    for s in range(0, n, step):
        e = min(n, s + step)
        g = np.abs(rng.standard_normal((e - s, DIM)))
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        np.minimum(g, 0.2, out=g)
        g /= np.linalg.norm(g, axis=1, keepdims=True)
        out[s:e] = np.clip(np.rint(g * 512.0), 0, 255).astype(np.uint8)
    return out


def noisy_copy(rng: np.random.Generator, desc: np.ndarray, sigma: float = 8.0) -> np.ndarray:
    """Per-component N(0, sigma^2) noise, rounded half-to-even, clipped to 0..255."""
    noise = rng.normal(0.0, sigma, size=desc.shape)
    return np.clip(np.rint(desc.astype(np.float64) + noise), 0, 255).astype(np.uint8)


def projection_matrix(seed: int, rows: int = 192) -> np.ndarray:
    """The random vectors r_k as a [rows][128] float64 N(0,1) matrix (192 rows
    cover every parameter set: 128 code rows + up to 8 tables x 8 bits; the
    leading rows do not depend on `rows`)."""
    return np.random.default_rng(np.random.SeedSequence([seed, 0x5EED])).standard_normal((rows, DIM))


@dataclasses.dataclass
class ImageSet:
    desc: np.ndarray          # [N_total][128] uint8, images back to back
    img_off: np.ndarray       # [n_images + 1] uint64 feature offsets
    pairs: np.ndarray         # [P][2] uint32 (query image, candidate image)
    R: np.ndarray             # [192][128] float64 projection matrix (leading rows used)
    name: str = ""
    F: np.ndarray | None = None      # [P][9] float64, x_B^T F x_A = 0
    kpts: np.ndarray | None = None   # [N_total][2] float32
    truth: dict | None = None        # planted correspondences, for statistics only
    scale: np.ndarray | None = None  # [N_total] float32 key-point scale (SIFT sigma), pixels

    @property
    def n_images(self) -> int:
        return len(self.img_off) - 1

    def sizes(self) -> np.ndarray:
        return np.diff(self.img_off).astype(np.int64)

    def image(self, i: int) -> np.ndarray:
        return self.desc[self.img_off[i]:self.img_off[i + 1]]


def _offsets(sizes) -> np.ndarray:
    off = np.zeros(len(sizes) + 1, np.uint64)
    off[1:] = np.cumsum(np.asarray(sizes, np.uint64))
    return off


def config0(seed: int = 0) -> ImageSet:
    """One image pair: A has 2,000 descriptors; B has 1,000 noisy copies of
    distinct descriptors of A (sigma 8) and 1,000 fresh ones, permuted."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0]))
    A = sift_like(rng, 2000)
    src = rng.choice(2000, size=1000, replace=False)
    B = np.concatenate([noisy_copy(rng, A[src]), sift_like(rng, 1000)])
    perm = rng.permutation(2000)
    B = B[perm]
    # truth: B row r came from A row src[perm[r]] when perm[r] < 1000
    inv = np.full(2000, -1, np.int64)
    for r, s in enumerate(perm):
        if s < 1000:
            inv[r] = src[s]
    truth = {"b_from_a": inv}
    return ImageSet(np.concatenate([A, B]), _offsets([2000, 2000]), np.array([[0, 1]], np.uint32),
                    projection_matrix(seed), "config0", truth=truth)


def _copy_mix(rng, sizes, neighbours, copy_frac=0.3, truth=None):
    """Fresh descriptors for each image, then copy_frac of each image's rows
    replaced by noisy copies of fresh rows of its neighbour images.  When
    `truth` is a list, it receives one int64 array [n_copy][3] per image:
    (row of the copy in this image, source image, row of the source there);
    recording it draws no random numbers, so the images are the same."""
    n_img = len(sizes)
    n_copy = [int(round(copy_frac * s)) for s in sizes]
    fresh = [sift_like(rng, s - c) for s, c in zip(sizes, n_copy)]
    imgs, perms, srcs = [], [], []
    for i in range(n_img):
        nb = neighbours[i]
        src_img = nb[rng.integers(0, len(nb), size=n_copy[i])]
        src_row = np.zeros(n_copy[i], np.int64)
        parts = [fresh[i]]
        if n_copy[i]:
            rows = np.empty((n_copy[i], DIM), np.uint8)
            for k in np.unique(src_img):
                sel = np.nonzero(src_img == k)[0]
                pick = rng.integers(0, fresh[k].shape[0], size=sel.size)
                rows[sel] = fresh[k][pick]
                src_row[sel] = pick
            parts.append(noisy_copy(rng, rows))
        img = np.concatenate(parts)
        perm = rng.permutation(img.shape[0])
        imgs.append(img[perm])
        perms.append(perm)
        srcs.append((src_img.astype(np.int64), src_row))
    if truth is not None:
        where = []  # where[i][r]: position in image i of its r-th pre-permutation row
        for perm in perms:
            inv = np.empty(perm.size, np.int64)
            inv[perm] = np.arange(perm.size)
            where.append(inv)
        for i in range(n_img):
            nf = sizes[i] - n_copy[i]
            src_img, src_row = srcs[i]
            pos = where[i][nf + np.arange(n_copy[i])]
            spos = np.array([where[k][r] for k, r in zip(src_img, src_row)], np.int64)
            truth.append(np.stack([pos, src_img, spos], axis=1) if n_copy[i] else np.zeros((0, 3), np.int64))
    return imgs


def planted_pairs(truth, pairs):
    """Planted correspondences of each pair (A, B): the set of (q, j) with q a
    copy of B's row j or j a copy of A's row q.  Returns one set per pair."""
    by = {}
    for i, t in enumerate(truth):
        for pos, k, spos in t:
            by.setdefault((i, int(k)), []).append((int(pos), int(spos)))
    out = []
    for a, b in pairs:
        a, b = int(a), int(b)
        s = {(q, j) for q, j in by.get((a, b), [])}
        s |= {(q, j) for j, q in by.get((b, a), [])}
        out.append(s)
    return out


def config1(seed: int = 1, n_images: int = 100, lo: int = 4000, hi: int = 12000) -> ImageSet:
    """Exhaustive matching set: feature counts uniform in lo..hi; 30 % of each
    image are noisy copies of fresh descriptors of images at index distance
    1..5 (clamped to the set); every pair (i, k), i < k, i is the query image."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 1]))
    sizes = rng.integers(lo, hi + 1, size=n_images)
    neighbours = []
    for i in range(n_images):
        nb = [k for k in range(i - 5, i + 6) if k != i and 0 <= k < n_images]
        neighbours.append(np.array(nb if nb else [i], np.int64))
    truth = []
    imgs = _copy_mix(rng, sizes, neighbours, truth=truth)
    iu = np.triu_indices(n_images, 1)
    pairs = np.stack([iu[0], iu[1]], axis=1).astype(np.uint32)
    return ImageSet(np.concatenate(imgs), _offsets(sizes), pairs, projection_matrix(seed),
                    "config1:%d imgs %d..%d" % (n_images, lo, hi), truth={"copies": truth})


def config3(seed: int = 3, n_images: int = 2000, lo: int = 1000, hi: int = 20000, n_nbr: int = 30) -> ImageSet:
    """Batched uneven workload: log-uniform feature counts in lo..hi; each image
    draws n_nbr distinct random neighbours; the pair list is the deduplicated
    set of (min, max) image pairs; 30 % of each image are noisy copies of
    fresh descriptors of its neighbours."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 3]))
    sizes = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_images))).astype(np.int64)
    sizes = np.clip(sizes, lo, hi)
    nbr_sets = [set() for _ in range(n_images)]
    pairs = set()
    for i in range(n_images):
        cand = rng.choice(n_images - 1, size=n_nbr, replace=False)
        cand = cand + (cand >= i)
        for k in cand:
            k = int(k)
            nbr_sets[i].add(k)
            nbr_sets[k].add(i)
            pairs.add((min(i, k), max(i, k)))
    neighbours = [np.array(sorted(s), np.int64) for s in nbr_sets]
    imgs = _copy_mix(rng, sizes, neighbours)
    pairs = np.array(sorted(pairs), np.uint32)
    return ImageSet(np.concatenate(imgs), _offsets(sizes), pairs, projection_matrix(seed),
                    "config3:%d imgs log-uniform %d..%d, %d nbrs" % (n_images, lo, hi, n_nbr))


def random_set(seed: int, sizes, pairs=None, copy_frac: float = 0.3) -> ImageSet:
    """Small test set with the given image sizes (0 allowed).  About copy_frac
    of each image are noisy copies of fresh rows of the previous or next
    image (fresh rows when neither has any); all pairs i < k unless given."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 7]))
    sizes = [int(s) for s in sizes]
    n = len(sizes)
    n_copy = [int(round(copy_frac * s)) for s in sizes]
    fresh = [sift_like(rng, s - c) for s, c in zip(sizes, n_copy)]
    imgs = []
    for i in range(n):
        parts = [fresh[i]]
        if n_copy[i]:
            srcs = [k for k in (i - 1, i + 1) if 0 <= k < n and fresh[k].shape[0] > 0]
            if srcs:
                k = srcs[int(rng.integers(0, len(srcs)))]
                rows = fresh[k][rng.integers(0, fresh[k].shape[0], size=n_copy[i])]
                parts.append(noisy_copy(rng, rows))
            else:
                parts.append(sift_like(rng, n_copy[i]))
        img = np.concatenate(parts)
        imgs.append(img[rng.permutation(img.shape[0])])
    if pairs is None:
        iu = np.triu_indices(n, 1)
        pairs = np.stack([iu[0], iu[1]], axis=1)
    desc = np.concatenate(imgs) if imgs else np.zeros((0, DIM), np.uint8)
    return ImageSet(desc, _offsets(sizes), np.asarray(pairs, np.uint32).reshape(-1, 2), projection_matrix(seed),
                    "random:%s" % (sizes,))


# ---------------------------------------------------------------------------
# Epipolar-guided workload (config 4): views of random 3-D points
# ---------------------------------------------------------------------------

def _rot(axis_angle: np.ndarray) -> np.ndarray:
    """Rotation matrix of an axis-angle vector (Rodrigues)."""
    th = float(np.linalg.norm(axis_angle))
    if th < 1e-15:
        return np.eye(3)
    k = axis_angle / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(th) * Kx + (1 - np.cos(th)) * (Kx @ Kx)


def epipolar_set(seed: int = 4, n_views: int = 500, n_points: int = 200_000, radius: float = 0.25,
                 arc: float = 2 * math.pi, z_max: float = 0.34, focal: float = 1000.0, width: int = 1920,
                 height: int = 1080, jitter_px: float = 1.0, clutter: float = 0.3, min_overlap: float = 0.2,
                 sigma: float = 8.0, view_noise: float = 0.05, rise: float = 0.0) -> ImageSet:
    """Pinhole views of n_points uniform points in the unit cube.

    Cameras sit on a helix of the given radius around the cube centre (over
    the angle `arc`, rising by `rise` in total), each looking along the path with a small random
    rotation (view_noise radians per axis); a point is seen when it projects inside the image at depth
    0.02..z_max.  Each point carries a SIFT-like template descriptor; a view's
    key-point of it gets the template plus N(0, sigma^2) noise and its
    projection plus N(0, jitter^2) pixels.  A fraction `clutter` of each
    view's key-points are fresh descriptors at uniform image positions.
    Views are paired when they share at least min_overlap of the smaller
    visible set; F (x_cand^T F x_query = 0) is the ground truth of each pair.
    """
    rng = np.random.default_rng(np.random.SeedSequence([seed, 4]))
    srng = np.random.default_rng(np.random.SeedSequence([seed, 4, 1]))  # key-point scales only
    X = rng.random((n_points, 3))
    # a point's scale at unit depth: 1.6 px x 2^E, E ~ Exp(1) capped at 5 octaves
    s_unit = 1.6 * 2.0 ** np.minimum(srng.exponential(1.0, n_points), 5.0) * 0.2
    templates = sift_like(rng, n_points)
    Kc = np.array([[focal, 0, width / 2.0], [0, focal, height / 2.0], [0, 0, 1.0]])
    centre = np.array([0.5, 0.5, 0.5])
    cams = []
    for i in range(n_views):
        th = arc * i / n_views
        lift = rise * (i / max(1, n_views - 1) - 0.5)          # helix height
        pos = centre + np.array([radius * np.cos(th), radius * np.sin(th), lift]) + rng.normal(0, 0.01, 3)
        fwd = np.array([-np.sin(th), np.cos(th), 0.0])          # along the path
        up = np.array([0.0, 0.0, 1.0])
        right = np.cross(fwd, up)
        # camera axes: x right, y down, z forward
        Rw = np.stack([right, -up, fwd])
        Rw = _rot(rng.normal(0, view_noise, 3)) @ Rw
        t = -Rw @ pos
        cams.append((Rw, t))
    vis = []
    proj = []
    depth = []
    for Rw, t in cams:
        Y = X @ Rw.T + t
        z = Y[:, 2]
        ok = (z > 0.02) & (z < z_max)
        uv = np.full((n_points, 2), -1.0)
        uv[ok] = (Y[ok, :2] / z[ok, None]) * focal + np.array([width / 2.0, height / 2.0])
        ok &= (uv[:, 0] >= 0) & (uv[:, 0] < width) & (uv[:, 1] >= 0) & (uv[:, 1] < height)
        vis.append(np.nonzero(ok)[0])
        proj.append(uv)
        depth.append(z)
    # pairs by overlap of visible sets
    import scipy.sparse as sp
    rows = np.concatenate([np.full(len(v), i) for i, v in enumerate(vis)])
    cols = np.concatenate(vis)
    M = sp.csr_matrix((np.ones(len(rows), np.int32), (rows, cols)), shape=(n_views, n_points))
    inter = (M @ M.T).tocoo()
    nvis = np.array([len(v) for v in vis])
    pairs = []
    for a, b, c in zip(inter.row, inter.col, inter.data):
        if a < b and c >= min_overlap * max(1, min(nvis[a], nvis[b])):
            pairs.append((a, b))
    pairs = np.array(sorted(pairs), np.uint32).reshape(-1, 2)
    descs, kps, sizes, scales = [], [], [], []
    for i in range(n_views):
        v = vis[i]
        n_real = len(v)
        n_cl = int(round(n_real * clutter / (1.0 - clutter)))
        d_real = noisy_copy(rng, templates[v], sigma)
        k_real = proj[i][v] + rng.normal(0, jitter_px, (n_real, 2))
        d_cl = sift_like(rng, n_cl)
        k_cl = np.stack([rng.uniform(0, width, n_cl), rng.uniform(0, height, n_cl)], axis=1)
        d = np.concatenate([d_real, d_cl])
        k = np.concatenate([k_real, k_cl])
        perm = rng.permutation(d.shape[0])
        descs.append(d[perm])
        kps.append(k[perm].astype(np.float32))
        sizes.append(d.shape[0])
        # scale: the point's unit-depth scale over its depth, times log-normal noise; clutter
        # draws its own
        sc_real = s_unit[v] / depth[i][v] * np.exp(srng.normal(0, 0.1, n_real))
        sc_cl = 1.6 * 2.0 ** np.minimum(srng.exponential(1.0, n_cl), 5.0)
        scales.append(np.concatenate([sc_real, sc_cl])[perm].astype(np.float32))
    Kinv = np.linalg.inv(Kc)
    F = np.zeros((len(pairs), 9))
    for n, (a, b) in enumerate(pairs):
        Ra, ta = cams[a]
        Rb, tb = cams[b]
        Rr = Rb @ Ra.T
        tr = tb - Rr @ ta
        tx = np.array([[0, -tr[2], tr[1]], [tr[2], 0, -tr[0]], [-tr[1], tr[0], 0]])
        Fm = Kinv.T @ tx @ Rr @ Kinv
        F[n] = (Fm / np.linalg.norm(Fm)).ravel()
    return ImageSet(np.concatenate(descs), _offsets(sizes), pairs, projection_matrix(seed),
                    "epipolar:%d views, %d points" % (n_views, n_points), F=F,
                    kpts=np.concatenate(kps).astype(np.float32), scale=np.concatenate(scales))


def ransac_words(seed: int, n_pairs: int, n_hyp: int) -> np.ndarray:
    """Random uint32 words for RANSAC sampling: [n_pairs][n_hyp][8]."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 5]))
    return rng.integers(0, 2 ** 32, size=(n_pairs, n_hyp, 8), dtype=np.uint64).astype(np.uint32)


def config4(seed: int = 4) -> ImageSet:
    """Epipolar-guided workload: 500 views of 200,000 points on a two-turn
    helix (about 8k key-points per view with 30 % clutter); views with >= 20 %
    overlap are paired (about 14,600 pairs)."""
    return epipolar_set(seed, arc=4 * math.pi, rise=0.5, z_max=0.355)
