"""The C-ABI library builds, loads and exports every declared symbol (CPU).

No compute call is made: the library is loaded with ctypes and only its
host-side entry points that need no device are exercised.
"""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cashash.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1805_08995_gb300 import build
    path = build.build()
    return C.CDLL(path), path


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(cashash_\w+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_function_is_exported(lib):
    _, path = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(cashash_\w+)", out))
    declared = declared_functions()
    assert len(declared) >= 14
    missing = [n for n in declared if n not in exported]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_1805_08995_gb300 as ch
    assert sorted(ch.exported_symbols()) == sorted(n for n in declared_functions())


def test_binding_constants_match_header_enums():
    """Every CASHASH_ enum value the header defines that the binding also names has the same value
    there (kernel configurations, schedules, precisions, flags, stages, status codes)."""
    import paper_1805_08995_gb300 as ch
    txt = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    found = {}
    for body in re.findall(r"enum\s*\w*\s*\{([^}]*)\}", txt):
        for name, val in re.findall(r"(CASHASH_\w+)\s*=\s*(-?\w+)", body):
            found[name] = int(val, 0)
    for name, val in re.findall(r"#define\s+(CASHASH_\w+)\s+\(?(-?\d+)u?\)?", txt):
        found.setdefault(name, int(val))
    assert found.get("CASHASH_KERNEL_WARP") == 4 and found.get("CASHASH_KERNEL_JOIN_TC") == 3
    shared = [n for n in found if hasattr(ch, n)]
    assert len(shared) >= 10
    for n in shared:
        assert getattr(ch, n) == found[n], n


def test_strerror_and_defaults_without_device(lib):
    import paper_1805_08995_gb300 as ch
    assert ch.cashash_strerror(0) == "ok"
    assert ch.cashash_strerror(4) == "match capacity exceeded"
    assert ch.cashash_strerror(99) == "unknown status"
    p = ch.cashash_default_params()
    assert (p.code_bits, p.n_tables, p.bits_per_table, p.top_k, p.ratio_num, p.ratio_den) == (128, 6, 8, 10, 4, 5)
    assert p.epi_px < 0


def test_tables_bytes_host_arithmetic(lib):
    import paper_1805_08995_gb300 as ch
    p = ch.cashash_default_params()
    off = np.array([0, 3968, 3969, 3969, 20000], np.uint64)
    # chunks of 3968 features: 1 + 1 + 0 + 5 = 7; each holds 6 tables x (264 + 3968) uint16
    chunked = 7 * 6 * (264 + 3968) * 2
    # bucket-sorted tables: per image and table 257(+3) uint32 offsets, uint32 indices, 16-byte codes

    def block(n):
        return 1040 + 4 * ((n + 3) // 4 * 4) + 16 * n

    joined = 6 * sum(block(n) for n in (3968, 1, 0, 16031))
    assert ch.cashash_tables_bytes(p, off) == chunked + joined
    bad = ch.cashash_default_params(n_tables=0)
    assert ch.cashash_tables_bytes(bad, off) == 0
    assert ch.cashash_tables_bytes(p, np.array([0, 5, 3], np.uint64)) == 0


def test_create_rejects_bad_arguments_before_touching_a_device(lib):
    import paper_1805_08995_gb300 as ch
    R = np.zeros((256, 128))  # enough rows for any parameter set tried below
    for kw in (dict(top_k=0), dict(code_bits=100), dict(n_tables=9), dict(bits_per_table=9),
               dict(ratio_den=0), dict(precision=7), dict(schedule=5)):
        with pytest.raises(ch.CashashError) as e:
            ch.cashash_create(ch.cashash_default_params(**kw), R)
        assert e.value.status == ch.CASHASH_EINVAL
    Rn = R.copy()
    Rn[3, 4] = np.nan
    with pytest.raises(ch.CashashError) as e:
        ch.cashash_create(ch.cashash_default_params(), Rn)
    assert e.value.status == ch.CASHASH_EINVAL


def test_tuning_calls_reject_null_arguments(lib):
    """The plan tuning entry points check their arguments before any CUDA call."""
    import ctypes as C
    import paper_1805_08995_gb300 as ch
    L = ch._load()
    t = ch.cashash_tuning()
    assert L.cashash_plan_get_tuning(None, C.byref(t)) == ch.CASHASH_EINVAL
    assert L.cashash_plan_set_tuning(None, C.byref(t)) == ch.CASHASH_EINVAL
    assert L.cashash_plan_autotune(None, None, None, 0, None) == ch.CASHASH_EINVAL
    assert C.sizeof(ch.cashash_tuning) == 24


def test_flags_are_checked_before_touching_a_device(lib):
    """Unknown flag bits are EINVAL for every entry point; the allocation-free
    single-pair call has no scratch for a reverse pair, so MUTUAL is ENOTSUP."""
    import ctypes as C
    import paper_1805_08995_gb300 as ch
    R = np.zeros((256, 128))
    with pytest.raises(ch.CashashError) as e:
        ch.cashash_create(ch.cashash_default_params(flags=4), R)
    assert e.value.status == ch.CASHASH_EINVAL
    L = ch._load()
    st = ch.cashash_set()
    off = np.zeros(2, np.uint64)
    for flags, want in ((ch.CASHASH_FLAG_MUTUAL, ch.CASHASH_ENOTSUP), (8, ch.CASHASH_EINVAL)):
        p = ch.cashash_default_params(flags=flags)
        r = L.cashash_match_pair_noalloc(C.byref(p), C.byref(st), 0, 0, None, off.ctypes.data_as(C.c_void_p),
                                         None, 0, None)
        assert r == want


def test_chunked_matching_rejects_bad_arguments_on_the_host(lib):
    """cashash_match_chunked checks its cursor, chunk size, callback and pairs
    before any CUDA call."""
    import ctypes as C
    import paper_1805_08995_gb300 as ch
    L = ch._load()
    st = ch.cashash_set()
    st.n_images = 2
    off = np.array([0, 3, 5], np.uint64)
    st.img_off = off.ctypes.data_as(C.c_void_p)
    pairs = np.array([[0, 1], [1, 0]], np.uint32)
    fn = ch.CHUNK_FN(lambda *a: 0)
    ctx = C.c_void_p(1)  # never dereferenced: every case fails its argument checks first

    def call(cursor, chunk, f, pr=pairs):
        cur = C.c_uint64(cursor)
        return L.cashash_match_chunked(ctx, C.byref(st), pr.ctypes.data_as(C.c_void_p), pr.shape[0], None, chunk,
                                       C.byref(cur), f, None, None)

    assert call(3, 1, fn) == ch.CASHASH_EINVAL            # cursor beyond the list
    assert call(0, 0, fn) == ch.CASHASH_EINVAL            # empty chunks
    assert call(0, 1, ch.CHUNK_FN()) == ch.CASHASH_EINVAL  # no callback
    assert call(0, 1, fn, np.array([[0, 2]], np.uint32)) == ch.CASHASH_EINVAL  # image out of range


def test_ga_calls_check_arguments_on_the_host(lib):
    """The Ga-CasHash first-stage calls: defaults, subset sizes (pure host
    arithmetic) and argument checks that precede any CUDA call."""
    import ctypes as C
    import paper_1805_08995_gb300 as ch
    L = ch._load()
    g = ch.cashash_ga_default_params()
    assert (g.top_pct, g.min_matches, g.n_hyp, g.inlier_num, g.inlier_den, g.thresh_px, g.confidence) == \
        (20, 16, 256, 2, 3, 3.0, 0.99)
    assert ch.cashash_ga_subset_offsets(np.array([0, 0, 1, 5, 105, 1105], np.uint64), 20).tolist() == \
        [0, 0, 1, 2, 22, 222]
    assert ch.cashash_ga_subset_offsets(np.array([0, 7], np.uint64), 100).tolist() == [0, 7]
    off = np.array([0, 3, 5], np.uint64)
    sub = np.zeros(3, np.uint64)
    hp = lambda a: a.ctypes.data_as(C.c_void_p)
    assert L.cashash_ga_subset_offsets(hp(off), 2, 0, hp(sub)) == ch.CASHASH_EINVAL
    assert L.cashash_ga_subset_offsets(hp(off), 2, 101, hp(sub)) == ch.CASHASH_EINVAL
    assert L.cashash_ga_subset_offsets(hp(np.array([0, 3, 2], np.uint64)), 2, 20, hp(sub)) == ch.CASHASH_EINVAL
    assert L.cashash_ga_select(None, hp(off), 2, 0, None, None) == ch.CASHASH_EINVAL
    assert L.cashash_ga_select(None, hp(off), 2, 20, None, None) == ch.CASHASH_EINVAL  # no scale / output
    assert L.cashash_ga_select(None, None, 0, 20, None, None) == ch.CASHASH_OK      # nothing to do
    pairs = np.array([[0, 1]], np.uint32)
    dummy = C.c_void_p(16)  # never dereferenced: every case fails its checks first
    for bad in (dict(n_hyp=0), dict(min_matches=3), dict(inlier_num=5, inlier_den=4), dict(thresh_px=-1.0),
                dict(confidence=-0.5), dict(confidence=float("nan"))):
        gp = ch.cashash_ga_default_params(**bad)
        assert L.cashash_estimate_F(dummy, hp(off), 2, hp(pairs), 1, dummy, dummy, C.byref(gp), dummy, dummy,
                                    dummy, None) == ch.CASHASH_EINVAL
    gp = ch.cashash_ga_default_params()
    assert L.cashash_estimate_F(dummy, hp(off), 2, hp(np.array([[0, 2]], np.uint32)), 1, dummy, dummy,
                                C.byref(gp), dummy, dummy, dummy, None) == ch.CASHASH_EINVAL
    assert L.cashash_estimate_F(None, None, 0, None, 0, None, None, C.byref(gp), None, None, None, None) == \
        ch.CASHASH_OK
    p = ch.cashash_params()
    assert L.cashash_get_params(None, C.byref(p)) == ch.CASHASH_EINVAL
    assert L.cashash_set_host_tuning(None, None) == ch.CASHASH_EINVAL
    assert L.cashash_get_host_tuning(None, None) == ch.CASHASH_EINVAL
    assert L.cashash_ga_stage1(None, None, None, None, None, 0, C.byref(gp), None, None, None, None) == \
        ch.CASHASH_EINVAL


def test_package_fails_loudly_without_library(tmp_path):
    """The product path has no CPU fallback: without libcashash.so it raises."""
    import sys
    code = ("import sys; sys.path.insert(0, %r); import paper_1805_08995_gb300 as ch; "
            "ch.LIB_PATH = %r; ch._lib = None\n"
            "try:\n    ch.cashash_default_params()\nexcept ImportError as e:\n    print('raised', e)\n" %
            (ROOT, str(tmp_path / "missing.so")))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True)
    assert "raised" in r.stdout
