"""Python binding of the GB300 Cascade Hashing library (libcashash.so).

Argument marshalling only: every step of the matching path runs in the CUDA
kernels of ``csrc/`` behind the C-ABI declared in ``include/cashash.h``.  The
functions carry the C names.  PyTorch supplies device memory and streams.

There is no CPU fallback: importing this package without a built library,
or calling it without a CUDA device, raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcashash.so")
DIM = 128

CASHASH_OK, CASHASH_EINVAL, CASHASH_ENOMEM, CASHASH_ECUDA = 0, 1, 2, 3
CASHASH_EOVERFLOW, CASHASH_EDEVICE, CASHASH_ETIMEOUT, CASHASH_ENOTSUP = 4, 5, 6, 7
CASHASH_FP32, CASHASH_BF16 = 0, 1
CASHASH_SCHED_PER_PAIR, CASHASH_SCHED_PERSISTENT = 0, 1
CASHASH_NOALLOC_MAX_QUERIES = 65536
CASHASH_KERNEL_JOIN, CASHASH_KERNEL_QUERY, CASHASH_KERNEL_JOIN_TC, CASHASH_KERNEL_WARP = 1, 2, 3, 4
CASHASH_FLAG_MUTUAL, CASHASH_FLAG_ACCEPT_SINGLE = 1, 2


class CashashError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__("%s: %s (status %d)" % (what, cashash_strerror(status), status))


class cashash_params(C.Structure):
    _fields_ = [("code_bits", C.c_uint32), ("n_tables", C.c_uint32), ("bits_per_table", C.c_uint32),
                ("top_k", C.c_uint32), ("ratio_num", C.c_uint32), ("ratio_den", C.c_uint32),
                ("tau", C.c_uint32), ("precision", C.c_uint32), ("schedule", C.c_uint32),
                ("flags", C.c_uint32), ("epi_px", C.c_double)]


class cashash_set(C.Structure):
    _fields_ = [("n_images", C.c_uint32), ("reserved", C.c_uint32), ("n_features", C.c_uint64),
                ("img_off", C.c_void_p), ("desc", C.c_void_p), ("codes", C.c_void_p), ("buckets", C.c_void_p),
                ("sqnorm", C.c_void_p), ("tables", C.c_void_p), ("kpts", C.c_void_p)]


N_STAGES = 10
STAGES = ("centre", "project", "reeval", "tables", "match", "compact", "calibrate", "fallback", "h2d", "d2h")


class cashash_stats(C.Structure):
    _fields_ = [("n_features", C.c_uint64), ("n_reevaluated", C.c_uint64), ("n_pairs", C.c_uint64),
                ("n_matches", C.c_uint64), ("n_work_items", C.c_uint64), ("n_launches", C.c_uint64),
                ("ms_stage", C.c_double * N_STAGES)]


class cashash_tuning(C.Structure):
    _fields_ = [("kernel", C.c_uint32), ("tile", C.c_uint32), ("ctas_per_sm", C.c_uint32), ("reserved", C.c_uint32),
                ("ms_sample", C.c_double)]


class cashash_ga_params(C.Structure):
    _fields_ = [("top_pct", C.c_uint32), ("min_matches", C.c_uint32), ("n_hyp", C.c_uint32),
                ("inlier_num", C.c_uint32), ("inlier_den", C.c_uint32), ("kernel", C.c_uint32),
                ("thresh_px", C.c_double), ("confidence", C.c_double)]


GA_MAX_HYP = 4096
GA_NONE = 0xFFFFFFFF

CHUNK_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_uint64, C.c_uint32, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32))

_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libcashash.so is not built (run __graft_entry__.build() or "
                              "python paper_1805_08995_gb300/build.py)")
        lib = C.CDLL(LIB_PATH)
        vp, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
        P = C.POINTER
        sig = {
            "cashash_strerror": ([C.c_int], C.c_char_p),
            "cashash_default_params": ([P(cashash_params)], None),
            "cashash_tables_bytes": ([P(cashash_params), vp, u32], u64),
            "cashash_create": ([P(vp), P(cashash_params), vp], C.c_int),
            "cashash_destroy": ([vp], None),
            "cashash_build_codes": ([vp, P(cashash_set), vp, vp], C.c_int),
            "cashash_get_mean": ([vp, vp], C.c_int),
            "cashash_plan_create": ([vp, P(cashash_set), vp, u32, P(vp)], C.c_int),
            "cashash_plan_destroy": ([vp], None),
            "cashash_match_plan": ([vp, vp, vp, vp, vp, u64, vp], C.c_int),
            "cashash_match_pairs": ([vp, P(cashash_set), vp, u32, vp, vp, vp, u64, vp], C.c_int),
            "cashash_sync_status": ([vp, vp], C.c_int),
            "cashash_run_host": ([vp, vp, vp, u32, vp, vp, u32, vp, vp, vp, u64, u64], C.c_int),
            "cashash_get_stats": ([vp, P(cashash_stats)], C.c_int),
            "cashash_set_profiling": ([vp, C.c_int], C.c_int),
            "cashash_plan_set_threshold_hint": ([vp, u32, C.c_int], C.c_int),
            "cashash_match_pair_noalloc": ([P(cashash_params), P(cashash_set), u32, u32, vp, vp, vp, u64, vp],
                                           C.c_int),
            "cashash_noalloc_status": ([vp], C.c_int),
            "cashash_projection_bounds": ([vp, P(cashash_set), u64, u64, vp, vp, vp], C.c_int),
            "cashash_plan_get_tuning": ([vp, P(cashash_tuning)], C.c_int),
            "cashash_plan_set_tuning": ([vp, P(cashash_tuning)], C.c_int),
            "cashash_plan_autotune": ([vp, vp, vp, u32, vp], C.c_int),
            "cashash_match_chunked": ([vp, P(cashash_set), vp, u64, vp, u32, P(u64), CHUNK_FN, vp, vp], C.c_int),
            "cashash_get_params": ([vp, P(cashash_params)], C.c_int),
            "cashash_set_host_tuning": ([vp, P(cashash_tuning)], C.c_int),
            "cashash_get_host_tuning": ([vp, P(cashash_tuning)], C.c_int),
            "cashash_ga_default_params": ([P(cashash_ga_params)], None),
            "cashash_ga_subset_offsets": ([vp, u32, u32, vp], C.c_int),
            "cashash_ga_select": ([vp, vp, u32, u32, vp, vp], C.c_int),
            "cashash_estimate_F": ([vp, vp, u32, vp, u32, vp, vp, P(cashash_ga_params), vp, vp, vp, vp], C.c_int),
            "cashash_ga_stage1": ([vp, P(cashash_set), vp, vp, vp, u32, P(cashash_ga_params), vp, vp, vp, vp],
                                  C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def exported_symbols():
    """Names of the C-ABI entry points this binding expects."""
    return ["cashash_strerror", "cashash_default_params", "cashash_tables_bytes", "cashash_create",
            "cashash_destroy", "cashash_build_codes", "cashash_get_mean", "cashash_plan_create",
            "cashash_plan_destroy", "cashash_match_plan", "cashash_match_pairs", "cashash_sync_status",
            "cashash_run_host", "cashash_get_stats", "cashash_set_profiling", "cashash_match_pair_noalloc",
            "cashash_plan_set_threshold_hint", "cashash_plan_get_tuning", "cashash_plan_set_tuning",
            "cashash_plan_autotune", "cashash_match_chunked", "cashash_get_params", "cashash_ga_default_params",
            "cashash_ga_subset_offsets", "cashash_ga_select", "cashash_estimate_F", "cashash_ga_stage1",
            "cashash_set_host_tuning", "cashash_get_host_tuning", "cashash_noalloc_status",
            "cashash_projection_bounds"]


def _check(st, what):
    if st != CASHASH_OK:
        raise CashashError(st, what)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _hptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------------------
# C-ABI wrappers (same names)
# ---------------------------------------------------------------------------

def cashash_strerror(status: int) -> str:
    return _load().cashash_strerror(int(status)).decode()


def cashash_default_params(**over) -> cashash_params:
    p = cashash_params()
    _load().cashash_default_params(C.byref(p))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def cashash_tables_bytes(params: cashash_params, img_off: np.ndarray) -> int:
    img_off = np.ascontiguousarray(img_off, np.uint64)
    return int(_load().cashash_tables_bytes(C.byref(params), _hptr(img_off), len(img_off) - 1))


class Context:
    """Owns a cashash_ctx (projection matrix, centre, workspace)."""

    def __init__(self, params: cashash_params, R: np.ndarray):
        self.params = params
        R = np.ascontiguousarray(R, np.float64)
        rows = params.code_bits + params.n_tables * params.bits_per_table
        if R.ndim != 2 or R.shape[1] != DIM or R.shape[0] < rows:
            raise ValueError("R must have at least %d rows of 128" % rows)
        R = np.ascontiguousarray(R[:rows])
        h = C.c_void_p()
        _check(_load().cashash_create(C.byref(h), C.byref(params), _hptr(R)), "cashash_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            _load().cashash_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cashash_create(params: cashash_params, R: np.ndarray) -> Context:
    return Context(params, R)


def cashash_destroy(ctx: Context):
    ctx.close()


class DeviceSet:
    """A cashash_set whose device arrays are torch tensors on the current device."""

    def __init__(self, params: cashash_params, img_off: np.ndarray, desc, kpts=None):
        import torch
        self.img_off = np.ascontiguousarray(img_off, np.uint64)
        n = int(self.img_off[-1]) if len(self.img_off) else 0
        dev = torch.device("cuda", torch.cuda.current_device())
        if not isinstance(desc, torch.Tensor):
            desc = torch.from_numpy(np.ascontiguousarray(desc, np.uint8).reshape(-1, DIM)).to(dev)
        assert desc.dtype == torch.uint8 and desc.is_cuda and desc.is_contiguous() and desc.shape == (n, DIM)
        self.desc = desc
        self.codes = torch.empty((max(n, 1), 4), dtype=torch.int32, device=dev)
        self.buckets = torch.empty((max(n, 1), 8), dtype=torch.uint8, device=dev)
        self.sqnorm = torch.empty((max(n, 1),), dtype=torch.int32, device=dev)
        tb = cashash_tables_bytes(params, self.img_off)
        self.tables = torch.empty((max(tb, 16),), dtype=torch.uint8, device=dev)
        if kpts is not None and not isinstance(kpts, torch.Tensor):
            kpts = torch.from_numpy(np.ascontiguousarray(kpts, np.float32).reshape(-1, 2)).to(dev)
        self.kpts = kpts
        self.n = n
        self.c = cashash_set(len(self.img_off) - 1, 0, n, self.img_off.ctypes.data, desc.data_ptr(),
                             self.codes.data_ptr(), self.buckets.data_ptr(), self.sqnorm.data_ptr(),
                             self.tables.data_ptr(), kpts.data_ptr() if kpts is not None else None)

    def codes_np(self):
        return self.codes[:self.n].cpu().numpy().view(np.uint32)

    def buckets_np(self, n_tables):
        return self.buckets[:self.n, :n_tables].cpu().numpy()


def cashash_build_codes(ctx: Context, dset: DeviceSet, mean=None, stream=None):
    m = None if mean is None else np.ascontiguousarray(mean, np.float64)
    _check(_load().cashash_build_codes(ctx.handle, C.byref(dset.c), _hptr(m), _stream(stream)),
           "cashash_build_codes")


def cashash_get_mean(ctx: Context) -> np.ndarray:
    out = np.zeros(DIM, np.float64)
    _check(_load().cashash_get_mean(ctx.handle, _hptr(out)), "cashash_get_mean")
    return out


class Plan:
    def __init__(self, ctx: Context, dset: DeviceSet, pairs: np.ndarray):
        self.ctx = ctx
        self.pairs = np.ascontiguousarray(pairs, np.uint32).reshape(-1, 2)
        self.P = self.pairs.shape[0]
        h = C.c_void_p()
        _check(_load().cashash_plan_create(ctx.handle, C.byref(dset.c), _hptr(self.pairs), self.P, C.byref(h)),
               "cashash_plan_create")
        self.handle = h
        self.dset = dset

    def close(self):
        if getattr(self, "handle", None):
            _load().cashash_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cashash_plan_create(ctx: Context, dset: DeviceSet, pairs) -> Plan:
    return Plan(ctx, dset, pairs)


def cashash_plan_set_threshold_hint(plan: Plan, hamming: int, fixed: bool = False):
    _check(_load().cashash_plan_set_threshold_hint(plan.handle, int(hamming), 1 if fixed else 0),
           "cashash_plan_set_threshold_hint")


def cashash_plan_get_tuning(plan: Plan) -> dict:
    t = cashash_tuning()
    _check(_load().cashash_plan_get_tuning(plan.handle, C.byref(t)), "cashash_plan_get_tuning")
    return {k: getattr(t, k) for k, _ in cashash_tuning._fields_ if k != "reserved"}


def cashash_plan_set_tuning(plan: Plan, kernel: int, tile: int = 0, ctas_per_sm: int = 0):
    t = cashash_tuning(kernel=kernel, tile=tile, ctas_per_sm=ctas_per_sm, reserved=0, ms_sample=-1.0)
    _check(_load().cashash_plan_set_tuning(plan.handle, C.byref(t)), "cashash_plan_set_tuning")


def cashash_plan_autotune(ctx: Context, plan: Plan, F=None, max_pairs: int = 0, stream=None) -> dict:
    """Times every applicable kernel configuration on a sample of the plan's
    pairs, keeps the fastest and returns it (see include/cashash.h)."""
    _check(_load().cashash_plan_autotune(ctx.handle, plan.handle, _dptr(F), int(max_pairs), _stream(stream)),
           "cashash_plan_autotune")
    return cashash_plan_get_tuning(plan)


def cashash_set_host_tuning(ctx: Context, kernel: int = 0, tile: int = 0, ctas_per_sm: int = 0):
    """Kernel configuration of cashash_run_host's plans; kernel 0 restores the default."""
    if kernel == 0:
        _check(_load().cashash_set_host_tuning(ctx.handle, None), "cashash_set_host_tuning")
        return
    t = cashash_tuning(kernel, tile, ctas_per_sm, 0, -1.0)
    _check(_load().cashash_set_host_tuning(ctx.handle, C.byref(t)), "cashash_set_host_tuning")


def cashash_get_host_tuning(ctx: Context) -> dict:
    t = cashash_tuning()
    _check(_load().cashash_get_host_tuning(ctx.handle, C.byref(t)), "cashash_get_host_tuning")
    return {"kernel": t.kernel, "tile": t.tile, "ctas_per_sm": t.ctas_per_sm}


def cashash_plan_destroy(plan: Plan):
    plan.close()


def cashash_match_plan(ctx: Context, plan: Plan, match_off, matches, cap: int, F=None, stream=None):
    _check(_load().cashash_match_plan(ctx.handle, plan.handle, _dptr(F), _dptr(match_off), _dptr(matches), int(cap),
                                      _stream(stream)), "cashash_match_plan")


def cashash_match_pairs(ctx: Context, dset: DeviceSet, pairs, match_off, matches, cap: int, F=None, stream=None):
    pairs = np.ascontiguousarray(pairs, np.uint32).reshape(-1, 2)
    _check(_load().cashash_match_pairs(ctx.handle, C.byref(dset.c), _hptr(pairs), pairs.shape[0], _dptr(F),
                                       _dptr(match_off), _dptr(matches), int(cap), _stream(stream)),
           "cashash_match_pairs")


def cashash_sync_status(ctx: Context, stream=None) -> int:
    return int(_load().cashash_sync_status(ctx.handle, _stream(stream)))


def cashash_get_stats(ctx: Context) -> dict:
    s = cashash_stats()
    _check(_load().cashash_get_stats(ctx.handle, C.byref(s)), "cashash_get_stats")
    out = {k: int(getattr(s, k)) for k, _ in cashash_stats._fields_ if k != "ms_stage"}
    out["ms_stage"] = {name: float(s.ms_stage[i]) for i, name in enumerate(STAGES)}
    return out


def cashash_set_profiling(ctx: Context, on: bool = True):
    _check(_load().cashash_set_profiling(ctx.handle, 1 if on else 0), "cashash_set_profiling")


def cashash_match_pair_noalloc(params: cashash_params, dset: DeviceSet, image_a: int, image_b: int, match_off,
                               matches, cap: int, F=None, stream=None):
    """Allocation-free matching of one pair (see include/cashash.h): the
    library allocates nothing; scratch comes from its fixed device array."""
    _check(_load().cashash_match_pair_noalloc(C.byref(params), C.byref(dset.c), int(image_a), int(image_b),
                                              _dptr(F), _dptr(match_off), _dptr(matches), int(cap),
                                              _stream(stream)), "cashash_match_pair_noalloc")


def cashash_projection_bounds(ctx: Context, dset: DeviceSet, first: int, count: int, stream=None):
    """Diagnostic of the projection's rounding bound (see include/cashash.h):
    returns device tensors (approx, bound), each [count][rows] float32."""
    import torch
    rows = ctx.params.code_bits + ctx.params.n_tables * ctx.params.bits_per_table
    approx = torch.empty((max(count, 1), rows), dtype=torch.float32, device="cuda")
    bound = torch.empty_like(approx)
    _check(_load().cashash_projection_bounds(ctx.handle, C.byref(dset.c), int(first), int(count), _dptr(approx),
                                             _dptr(bound), _stream(stream)), "cashash_projection_bounds")
    return approx[:count], bound[:count]


def cashash_noalloc_status(stream=None) -> int:
    """Reads and clears the device status of the allocation-free calls on the
    current device (synchronises the stream): CASHASH_OK, CASHASH_EDEVICE or
    CASHASH_EOVERFLOW, returned rather than raised."""
    st = _load().cashash_noalloc_status(_stream(stream))
    if st == CASHASH_ECUDA:
        _check(st, "cashash_noalloc_status")
    return st


def cashash_match_chunked(ctx: Context, dset: DeviceSet, pairs, chunk_pairs: int, on_chunk, cursor: int = 0,
                          F=None, stream=None) -> int:
    """Resumable chunked matching (see include/cashash.h).  on_chunk(first,
    match_off, matches) receives numpy copies of one chunk's lists (match_off
    relative to the chunk) and returns True to stop.  Returns the cursor: the
    index of the first pair not yet flushed (len(pairs) when done)."""
    pairs = np.ascontiguousarray(pairs, np.uint32).reshape(-1, 2)
    cur = C.c_uint64(int(cursor))
    errors = []

    def cb(user, first, count, moff, mt):
        try:
            off = np.ctypeslib.as_array(moff, shape=(count + 1,)).copy()
            n = int(off[-1])
            m = np.ctypeslib.as_array(mt, shape=(max(n, 1), 2))[:n].copy() if n else np.zeros((0, 2), np.uint32)
            return 1 if on_chunk(int(first), off, m) else 0
        except Exception as e:  # an exception stops the run; it is raised after the C call returns
            errors.append(e)
            return 1

    fn = CHUNK_FN(cb)
    st = _load().cashash_match_chunked(ctx.handle, C.byref(dset.c), _hptr(pairs), pairs.shape[0], _dptr(F),
                                       int(chunk_pairs), C.byref(cur), fn, None, _stream(stream))
    if errors:
        raise errors[0]
    _check(st, "cashash_match_chunked")
    return int(cur.value)


def cashash_run_host(ctx: Context, desc: np.ndarray, img_off: np.ndarray, pairs: np.ndarray, cap: int,
                     kpts=None, F=None, stage_bytes: int = 0, match_off=None, matches=None):
    """End-to-end from host arrays.  desc may be a pinned torch CPU tensor or a
    numpy array.  Returns (status, match_off[P+1], matches[M][2])."""
    img_off = np.ascontiguousarray(img_off, np.uint64)
    pairs = np.ascontiguousarray(pairs, np.uint32).reshape(-1, 2)
    P = pairs.shape[0]
    if hasattr(desc, "data_ptr"):
        dptr = C.c_void_p(desc.data_ptr())
    else:
        desc = np.ascontiguousarray(desc, np.uint8)
        dptr = _hptr(desc)
    kp = None if kpts is None else np.ascontiguousarray(kpts, np.float32)
    Fh = None if F is None else np.ascontiguousarray(F, np.float64)
    if match_off is None:
        match_off = np.zeros(P + 1, np.uint64)
    if matches is None:
        matches = np.zeros((max(int(cap), 1), 2), np.uint32)
    st = _load().cashash_run_host(ctx.handle, dptr, _hptr(img_off), len(img_off) - 1, _hptr(kp), _hptr(pairs), P,
                                  _hptr(Fh), _hptr(match_off), _hptr(matches), int(cap), int(stage_bytes))
    if st not in (CASHASH_OK, CASHASH_EOVERFLOW):
        raise CashashError(st, "cashash_run_host")
    total = int(match_off[P])
    return st, match_off, matches[:min(total, int(cap))]


# ---------------------------------------------------------------------------
# Ga-CasHash first stage (Sec. 7.1)
# ---------------------------------------------------------------------------

def cashash_get_params(ctx: Context) -> cashash_params:
    p = cashash_params()
    _check(_load().cashash_get_params(ctx.handle, C.byref(p)), "cashash_get_params")
    return p


def cashash_ga_default_params(**over) -> cashash_ga_params:
    g = cashash_ga_params()
    _load().cashash_ga_default_params(C.byref(g))
    for k, v in over.items():
        setattr(g, k, v)
    return g


def cashash_ga_subset_offsets(img_off: np.ndarray, top_pct: int) -> np.ndarray:
    off = np.ascontiguousarray(img_off, np.uint64)
    sub = np.zeros(len(off), np.uint64)
    _check(_load().cashash_ga_subset_offsets(_hptr(off), len(off) - 1, top_pct, _hptr(sub)),
           "cashash_ga_subset_offsets")
    return sub


def cashash_ga_select(scale, img_off: np.ndarray, top_pct: int, stream=None):
    """Selected global feature indices (torch int32 on the device, uint32 values)
    and the subset offsets (numpy)."""
    import torch
    off = np.ascontiguousarray(img_off, np.uint64)
    sub = cashash_ga_subset_offsets(off, top_pct)
    sel = torch.empty((max(int(sub[-1]), 1),), dtype=torch.int32, device=scale.device)
    _check(_load().cashash_ga_select(_dptr(scale), _hptr(off), len(off) - 1, top_pct, _dptr(sel), _stream(stream)),
           "cashash_ga_select")
    return sel[:int(sub[-1])], sub


def _ga_out(P: int, device):
    import torch
    F = torch.empty((max(P, 1), 9), dtype=torch.float64, device=device)
    info = torch.empty((max(P, 1), 8), dtype=torch.int32, device=device)  # cashash_ga_info
    return F, info


def cashash_estimate_F(kpts, img_off: np.ndarray, pairs, match_off, matches, words, gp: cashash_ga_params = None,
                       stream=None):
    """F [P][9] (float64) and info [P][5] (int32: n_matches, n_inliers, best_hyp,
    accepted, hypotheses run) on the device, from the match lists of cashash_match_plan."""
    gp = gp or cashash_ga_default_params()
    off = np.ascontiguousarray(img_off, np.uint64)
    pr = np.ascontiguousarray(pairs, np.uint32).reshape(-1, 2)
    P = len(pr)
    F, info = _ga_out(P, kpts.device)
    _check(_load().cashash_estimate_F(_dptr(kpts), _hptr(off), len(off) - 1, _hptr(pr), P, _dptr(match_off),
                                      _dptr(matches), C.byref(gp), _dptr(words), _dptr(F), _dptr(info),
                                      _stream(stream)), "cashash_estimate_F")
    return F[:P], info[:P, :5]


def cashash_ga_stage1(ctx: Context, dset: DeviceSet, scale, mean: np.ndarray, pairs, words,
                      gp: cashash_ga_params = None, stream=None):
    """Selection, stage-1 CasHash matching of the subsets and F estimation;
    returns (F [P][9], info [P][5]) on the device."""
    gp = gp or cashash_ga_default_params()
    pr = np.ascontiguousarray(pairs, np.uint32).reshape(-1, 2)
    P = len(pr)
    m = np.ascontiguousarray(mean, np.float64)
    F, info = _ga_out(P, dset.desc.device)
    _check(_load().cashash_ga_stage1(ctx.handle, C.byref(dset.c), _dptr(scale), _hptr(m), _hptr(pr), P,
                                     C.byref(gp), _dptr(words), _dptr(F), _dptr(info), _stream(stream)),
           "cashash_ga_stage1")
    return F[:P], info[:P, :5]
