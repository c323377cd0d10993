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


def _copy_mix(rng, sizes, neighbours, copy_frac=0.3):
    """Fresh descriptors for each image, then copy_frac of each image's rows
    replaced by noisy copies of fresh rows of its neighbour images."""
    n_img = len(sizes)
    n_copy = [int(round(copy_frac * s)) for s in sizes]
    fresh = [sift_like(rng, s - c) for s, c in zip(sizes, n_copy)]
    imgs = []
    for i in range(n_img):
        nb = neighbours[i]
        src_img = nb[rng.integers(0, len(nb), size=n_copy[i])]
        parts = [fresh[i]]
        if n_copy[i]:
            rows = np.empty((n_copy[i], DIM), np.uint8)
            for k in np.unique(src_img):
                sel = np.nonzero(src_img == k)[0]
                pick = rng.integers(0, fresh[k].shape[0], size=sel.size)
                rows[sel] = fresh[k][pick]
            parts.append(noisy_copy(rng, rows))
        img = np.concatenate(parts)
        imgs.append(img[rng.permutation(img.shape[0])])
    return imgs


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
    imgs = _copy_mix(rng, sizes, neighbours)
    iu = np.triu_indices(n_images, 1)
    pairs = np.stack([iu[0], iu[1]], axis=1).astype(np.uint32)
    return ImageSet(np.concatenate(imgs), _offsets(sizes), pairs, projection_matrix(seed),
                    "config1:%d imgs %d..%d" % (n_images, lo, hi))


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
