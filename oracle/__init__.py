"""CPU oracle for Cascade Hashing image matching -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

Thin ctypes marshalling over ``liboracle.so`` (plain C, built from
``cashash_oracle.c`` with ``-ffp-contract=off``).  Every arithmetic step lives
in the C source; see its header for the passages of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "cashash_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
DIM = 128
MAX_K = 64

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, IEEE double without contraction)."""
    hdr = os.path.join(HERE, "cashash_oracle.h")
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


class Params(C.Structure):
    _fields_ = [("code_bits", C.c_uint32), ("n_tables", C.c_uint32), ("bits_per_table", C.c_uint32),
                ("top_k", C.c_uint32), ("ratio_num", C.c_uint32), ("ratio_den", C.c_uint32),
                ("tau", C.c_uint32), ("flags", C.c_uint32), ("epi_px", C.c_double)]


MUTUAL, ACCEPT_SINGLE = 1, 2


class QueryDetail(C.Structure):
    _fields_ = [("n_cand", C.c_uint32), ("n_top", C.c_uint32), ("top_j", C.c_uint32 * MAX_K),
                ("top_h", C.c_uint32 * MAX_K), ("top_d", C.c_int32 * MAX_K), ("match_j", C.c_int32),
                ("d1", C.c_int32), ("d2", C.c_int32)]


def params(code_bits=128, n_tables=6, bits_per_table=8, top_k=10, ratio=(4, 5), tau=None, epi_px=-1.0, flags=0):
    """flags: MUTUAL (match_pairs keeps (q, j) only when the reverse match of j
    is q) | ACCEPT_SINGLE (a query with exactly one ranked candidate matches it)."""
    return Params(code_bits, n_tables, bits_per_table, top_k, ratio[0], ratio[1],
                  code_bits if tau is None else tau, int(flags), float(epi_px))


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # a test may point at a deliberately mutated copy of the oracle
            path = os.environ.get("CASHASH_ORACLE_LIB") or build()
            lib = C.CDLL(path)
            P = C.POINTER
            lib.oracle_mean.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p]
            lib.oracle_projection.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            lib.oracle_projection.restype = C.c_double
            lib.oracle_projections.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_uint32,
                                               C.c_void_p]
            lib.oracle_hash.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, P(Params), C.c_void_p,
                                        C.c_void_p]
            lib.oracle_match_pair.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_uint32, P(Params), C.c_void_p,
                                              C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            lib.oracle_match_pair.restype = C.c_int64
            lib.oracle_match_pairs.argtypes = [C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p,
                                               C.c_void_p, C.c_uint32, P(Params), C.c_void_p, C.c_void_p,
                                               C.c_void_p, C.c_void_p, C.c_uint64, C.c_int]
            lib.oracle_match_pairs.restype = C.c_int64
            lib.oracle_epipolar_keep.argtypes = [C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_float,
                                                 C.c_double]
            lib.oracle_epipolar_keep.restype = C.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def mean(desc):
    desc = _c(desc, np.uint8).reshape(-1, DIM)
    mu = np.zeros(DIM, np.float64)
    _load().oracle_mean(_ptr(desc), desc.shape[0], _ptr(mu))
    return mu


def projection(x, mu, rrow):
    x = _c(x, np.uint8)
    mu = _c(mu, np.float64)
    rrow = _c(rrow, np.float64)
    return _load().oracle_projection(_ptr(x), _ptr(mu), _ptr(rrow))


def projections(desc, mu, R, rows, threads=1):
    """All ordered-double projections [n][rows] (row b of R against each
    feature), in `threads` row blocks of features (ctypes releases the GIL)."""
    desc = _c(desc, np.uint8).reshape(-1, DIM)
    R = np.ascontiguousarray(_c(R, np.float64)[:rows])
    mu = _c(mu, np.float64)
    n = desc.shape[0]
    v = np.zeros((n, rows), np.float64)
    lib = _load()
    step = max(1, (n + threads - 1) // threads)

    def work(s0):
        blk = np.ascontiguousarray(desc[s0:s0 + step])
        out = np.zeros((blk.shape[0], rows), np.float64)
        lib.oracle_projections(_ptr(blk), blk.shape[0], _ptr(mu), _ptr(R), rows, _ptr(out))
        v[s0:s0 + step] = out

    ts = [threading.Thread(target=work, args=(s0,)) for s0 in range(0, n, step)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return v


def hash_codes(desc, mu, R, p=None):
    """Returns (codes [n][4] uint32, buckets [n][n_tables] uint8)."""
    p = p or params()
    desc = _c(desc, np.uint8).reshape(-1, DIM)
    R = _c(R, np.float64)
    need = p.code_bits + p.n_tables * p.bits_per_table
    if R.ndim != 2 or R.shape[1] != DIM or R.shape[0] < need:
        raise ValueError("R must have at least %d rows of 128" % need)
    R = np.ascontiguousarray(R[:need])
    n = desc.shape[0]
    mu = _c(mu, np.float64)
    codes = np.zeros((n, 4), np.uint32)
    buckets = np.zeros((n, p.n_tables), np.uint8)
    _load().oracle_hash(_ptr(desc), n, _ptr(mu), _ptr(R), C.byref(p), _ptr(codes), _ptr(buckets))
    return codes, buckets


def match_pair(descA, codesA, bucketsA, descB, codesB, bucketsB, p=None, F=None, kptsA=None, kptsB=None,
               detail=False):
    """Returns match[nA] (int32, -1 = none) and, if detail, a list of QueryDetail."""
    p = p or params()
    descA = _c(descA, np.uint8).reshape(-1, DIM)
    descB = _c(descB, np.uint8).reshape(-1, DIM)
    codesA, codesB = _c(codesA, np.uint32), _c(codesB, np.uint32)
    bucketsA, bucketsB = _c(bucketsA, np.uint8), _c(bucketsB, np.uint8)
    F, kptsA, kptsB = _c(F, np.float64), _c(kptsA, np.float32), _c(kptsB, np.float32)
    nA, nB = descA.shape[0], descB.shape[0]
    m = np.full(nA, -1, np.int32)
    det = (QueryDetail * max(nA, 1))() if detail else None
    r = _load().oracle_match_pair(_ptr(descA), _ptr(codesA), _ptr(bucketsA), nA, _ptr(descB), _ptr(codesB),
                                  _ptr(bucketsB), nB, C.byref(p), _ptr(F), _ptr(kptsA), _ptr(kptsB), _ptr(m),
                                  None if det is None else C.cast(det, C.c_void_p))
    if r < 0:
        raise ValueError("oracle_match_pair rejected its arguments")
    if detail:
        return m, [det[i] for i in range(nA)]
    return m


def match_pairs(desc, img_off, codes, buckets, pairs, p=None, F=None, kpts=None, n_threads=0, cap=None):
    """All pairs; returns (match_off[P+1] uint64, matches[M][2] uint32).
    cap: capacity hint for the match list; when it suffices the oracle runs
    once, else (or without a hint) it counts first and then fills."""
    p = p or params()
    desc = _c(desc, np.uint8).reshape(-1, DIM)
    img_off = _c(img_off, np.uint64)
    pairs = _c(pairs, np.uint32).reshape(-1, 2)
    codes, buckets = _c(codes, np.uint32), _c(buckets, np.uint8)
    F, kpts = _c(F, np.float64), _c(kpts, np.float32)
    P = pairs.shape[0]
    off = np.zeros(P + 1, np.uint64)
    lib = _load()
    args = (_ptr(desc), _ptr(img_off), len(img_off) - 1, _ptr(codes), _ptr(buckets),
            _ptr(pairs), P, C.byref(p), _ptr(F), _ptr(kpts))
    if cap is not None and cap > 0:
        out = np.zeros((int(cap), 2), np.uint32)
        total = lib.oracle_match_pairs(*args, _ptr(off), _ptr(out), out.shape[0], int(n_threads))
        if total >= 0:
            return off, out[:total]
    total = lib.oracle_match_pairs(*args, _ptr(off), None, 0, int(n_threads))
    if total < 0:
        raise ValueError("oracle_match_pairs rejected its arguments")
    out = np.zeros((max(int(total), 1), 2), np.uint32)
    total2 = lib.oracle_match_pairs(*args, _ptr(off), _ptr(out), out.shape[0], int(n_threads))
    if total2 != total:
        raise RuntimeError("oracle_match_pairs is not deterministic")
    return off, out[:total]


def epipolar_keep(F, xq, yq, xc, yc, d):
    F = _c(F, np.float64).reshape(9)
    return bool(_load().oracle_epipolar_keep(_ptr(F), xq, yq, xc, yc, d))
