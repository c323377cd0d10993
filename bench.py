#!/usr/bin/env python
"""Benchmark: image pairs matched per second by Cascade Hashing on GB300.

One step = the whole matching path over one synthetic image set already
resident in HBM: centre, projection + signs (+ exact double re-evaluation),
lookup tables, and matching of every pair (lookup, Hamming ranking, exact
distances, ratio test, compaction of the match lists).  Default workload:
100 images of 4,000..12,000 SIFT-like uint8 descriptors (mean 8k) with all
4,950 pairs matched exhaustively.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank matches its own independent image set (weak
scaling, no data-path collective); rank 0 prints one JSON line.
--impl reference times the CPU oracle on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "image pairs matched/sec (8k x 8k SIFT) on 1 GB300 at bit-exact matches; % HBM roofline"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
POPC_PER_CLK_SM = 16          # 32-bit population counts per clock per SM (measured 15.96)
L2_FLUSH_BYTES = 256 << 20
# DRAM traffic per lookup entry of the matching kernel, from the ncu capture
# summarised in profiles/ (valid only for the kernel source it was taken on).
PROFILED_TRAFFIC = {
    "k_join": {"sources": ["paper_1805_08995_gb300/csrc/join.cu", "paper_1805_08995_gb300/csrc/join_common.cuh"],
               "sha256": "b132f2ff18a778804841d7f77457bf1c05b3e01fd14669d3cb2cab460a0f0d21",
               "bytes_per_entry": (2.608422e9 + 1.092449e9) / 861951265},
}


def source_sha256(rels):
    """SHA-256 of the concatenated kernel sources (None if one is missing)."""
    import hashlib
    h = hashlib.sha256()
    try:
        for rel in rels:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
    except OSError:
        return None
    return h.hexdigest()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    except Exception:
        d = dict(FALLBACK_PEAKS)
        d["source"] = "fallback"
        return d


def workload(name: str, rank: int, precision: str = "bf16"):
    """The synthetic image set of a named workload and its description.  On
    the 100-image exhaustive set the plain FP32 projection is config 1 and the
    BF16 tensor-core projection (with exact re-evaluation) is config 2."""
    import synth
    if name == "config1":
        s = synth.config1(seed=1 + 1000 * rank)
        tag = ("config2: BF16 tensor-core projection (exact FP64 re-evaluation under its bound) on the config-1 set"
               if precision == "bf16" else "config1: plain FP32 projection")
        desc = tag + ": 100 images x U{4000..12000} SIFT-like uint8 descriptors (30%% noisy copies of " \
               "index-neighbours), all 4950 pairs, seed %d" % (1 + 1000 * rank)
    elif name == "config0":
        s = synth.config0(seed=1000 * rank)
        desc = "config0: one pair, 2000 x 2000 descriptors, seed %d" % (1000 * rank)
    elif name == "config3":
        s = synth.config3(seed=3 + 1000 * rank)
        desc = "config3: 2000 images log-uniform 1000..20000, 30 neighbours each, %d pairs" % len(s.pairs)
    elif name == "config4":
        s = synth.config4(seed=4 + 1000 * rank)
        desc = ("config4: 500 pinhole views of 200000 points (helix cameras, 30%% clutter), views with >= 20%% "
                "overlap paired: %d pairs, epipolar band 4 px, ground-truth F" % len(s.pairs))
    else:
        raise SystemExit("unknown workload " + name)
    return s, desc


def lookup_entries(buckets: np.ndarray, img_off: np.ndarray, pairs: np.ndarray, T: int, m: int) -> int:
    """Sum over pairs and tables of |A_v| * |B_v| over buckets v: the lookup-table
    entries Step 1 visits (each needs one 128-bit Hamming distance)."""
    nb = 1 << m
    n_img = len(img_off) - 1
    hist = np.zeros((n_img, T, nb), np.int64)
    for i in range(n_img):
        b = buckets[img_off[i]:img_off[i + 1]]
        for t in range(T):
            hist[i, t] = np.bincount(b[:, t], minlength=nb)
    A = hist[pairs[:, 0].astype(np.int64)]
    B = hist[pairs[:, 1].astype(np.int64)]
    return int((A * B).sum())


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------

def oracle_codes_parallel(orc, desc, R, po, mu, threads):
    n = desc.shape[0]
    codes = np.zeros((n, 4), np.uint32)
    buckets = np.zeros((n, po.n_tables), np.uint8)
    step = max(1, (n + threads - 1) // threads)

    def work(s):
        c, b = orc.hash_codes(desc[s:s + step], mu, R, po)
        codes[s:s + step] = c
        buckets[s:s + step] = b

    ts = [threading.Thread(target=work, args=(s,)) for s in range(0, n, step)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return codes, buckets


def oracle_sample(s, n_pairs: int, seed: int = 0, flags: int = 0, threads: int = 0, tau=None):
    """Times the oracle on a bounded sample: the centre over the whole set,
    codes for the features of the images the sampled pairs touch, and the
    matching of n_pairs random pairs, on `threads` host threads (0 = all
    cores).  The whole job's time is scaled from the sample (codes by feature
    count, matching by N_A * N_B).  Returns a dict: pairs/s of the whole job,
    cores used, a description, the seconds spent, the sampled pair indices
    and the oracle's lists for them (for the parity check)."""
    import oracle as orc
    cores = threads if threads > 0 else (os.cpu_count() or 1)
    band = s.F is not None
    po = orc.params(epi_px=4.0 if band else -1.0, flags=flags, tau=tau)
    rng = np.random.default_rng(seed)
    P = len(s.pairs)
    pick = np.sort(rng.choice(P, size=min(n_pairs, P), replace=False))
    sp = s.pairs[pick]
    imgs = np.unique(sp)
    sizes = s.sizes()
    t0 = time.perf_counter()
    mu = orc.mean(s.desc)
    t_mean = time.perf_counter() - t0
    # sub-set of touched images, renumbered
    sub_off = np.zeros(len(imgs) + 1, np.uint64)
    sub_off[1:] = np.cumsum(sizes[imgs])
    sub_desc = np.concatenate([s.image(int(i)) for i in imgs])
    t0 = time.perf_counter()
    codes, buckets = oracle_codes_parallel(orc, sub_desc, s.R, po, mu, cores)
    t_hash = time.perf_counter() - t0
    remap = {int(i): k for k, i in enumerate(imgs)}
    sp2 = np.array([[remap[int(a)], remap[int(b)]] for a, b in sp], np.uint32)
    kw = {}
    if band:
        kw = dict(F=s.F[pick], kpts=np.concatenate([s.kpts[int(s.img_off[i]):int(s.img_off[i + 1])] for i in imgs]))
    t0 = time.perf_counter()
    eoff, emt = orc.match_pairs(sub_desc, sub_off, codes, buckets, sp2, po, n_threads=cores, **kw)
    t_match = time.perf_counter() - t0
    work_full = float((sizes[s.pairs[:, 0]] * sizes[s.pairs[:, 1]]).sum())
    work_smp = float((sizes[sp[:, 0]] * sizes[sp[:, 1]]).sum())
    job = t_mean + t_hash * (sizes.sum() / max(1, sub_desc.shape[0])) + t_match * (work_full / max(1.0, work_smp))
    text = ("oracle (C, %d thread%s): centre over %d features, codes of %d features (%d images), %d of %d pairs "
            "matched; the whole job's time scaled from it (codes by feature count, matching by N_A*N_B)"
            % (cores, "" if cores == 1 else "s", s.desc.shape[0], sub_desc.shape[0], len(imgs), len(sp), P))
    return {"pairs_per_s": P / job, "cores": cores, "sample": text, "seconds": t_mean + t_hash + t_match,
            "job_s": job, "pick": pick, "off": eoff, "mt": emt}


def parity_check(smp, moff_dev, mt_dev):
    """Compares the oracle's lists of the sampled pairs with the GPU lists of
    the last timed step, entry for entry."""
    off = moff_dev.cpu().numpy().view(np.uint64)
    mt = mt_dev[:int(off[-1])].cpu().numpy().view(np.uint32)
    bad, n_match = 0, 0
    for k, i in enumerate(smp["pick"]):
        g = mt[int(off[i]):int(off[i + 1])]
        e = smp["mt"][int(smp["off"][k]):int(smp["off"][k + 1])]
        n_match += len(e)
        if not np.array_equal(g, e):
            bad += 1
    return {"pairs_checked": int(len(smp["pick"])), "matches_checked": int(n_match), "mismatches": int(bad),
            "against": "oracle lists of the cpu_baseline sample vs the GPU lists of the last timed step"}


def run_flags(args) -> int:
    """The flags word of a run (1 = mutual check, 2 = single candidates accepted), same bits in the library."""
    return (1 if args.mutual else 0) | (2 if args.accept_single else 0)


def run_reference(args):
    """The oracle on the machine's host cores.  One step = a bounded sample of
    the workload (random pairs with the codes of the images they touch);
    ms_per_step is the oracle's time for that many pairs of the job, i.e. the
    sample's measured time scaled to average pairs (codes by feature count,
    matching by N_A * N_B), and value = pairs per step / that time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    s, wdesc = workload(args.workload, 0, args.precision)
    # the --ref-pairs budget is split over all steps so that the run stays within a few minutes
    sp = max(16, args.ref_pairs // max(1, args.steps + args.warmup))
    times = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(s, sp, seed=i, flags=run_flags(args), tau=args.tau)
        if i >= args.warmup:
            times.append(r["job_s"] * len(r["pick"]) / len(s.pairs))
    step_s = statistics.mean(times)
    value = sp / step_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8/f64", "data": "synthetic",
            "config": {"workload": wdesc, "pairs_per_step": sp},
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": r["cores"], "kind": "oracle",
                             "sample": "per step: " + r["sample"]},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def roofline_of(ch, p, s, ds, stage_ms, tuning, n_sm):
    """Roofline of the matching kernel (stage "match", timed alone by its own
    CUDA events on its launch stream over the timed steps).

    Unit: the lookup-table entries (q, j) that Step 1 visits, counted exactly
    (sum over pairs and tables of |A_v| * |B_v| over buckets v).  Headline
    fraction: the bytes the method touches -- per entry the candidate's index
    and 128-bit code (20 B), per query its k ranked rows, its own row, code,
    bucket ids and the 6 bucket offsets (1,480 B) -- over the kernel time,
    against the measured HBM copy bandwidth.  Most of these bytes are served
    from shared memory and L2, so the fraction can exceed 1; dram_frac is the
    same kernel's DRAM traffic (ncu) against that bandwidth, and alu_view /
    tensor_view give the integer and tensor ceilings of the Hamming step."""
    pk = peaks()
    T, m = p.n_tables, p.bits_per_table
    pairs = s.pairs
    if p.flags & 1:  # the mutual check matches every pair in both directions
        pairs = np.concatenate([s.pairs, s.pairs[:, ::-1]])
    entries = lookup_entries(ds.buckets_np(T), s.img_off, pairs, T, m)
    queries = float(s.sizes()[pairs[:, 0]].sum())
    warp_only = tuning.get("kernel") == ch.CASHASH_KERNEL_WARP  # the exact warp-per-query kernel alone
    t_match = statistics.mean(stage_ms["fallback" if warp_only else "match"]) / 1e3
    kernel = {ch.CASHASH_KERNEL_JOIN: "k_join", ch.CASHASH_KERNEL_JOIN_TC: "k_join_tc",
              ch.CASHASH_KERNEL_WARP: "k_match_fallback"}.get(tuning.get("kernel"), "k_match")
    touched = 20.0 * entries + queries * (p.top_k * 128 + 128 + 16 + 8 + 48)
    achieved = touched / t_match / 1e9
    traffic = None
    prof = PROFILED_TRAFFIC.get(kernel)
    if p.epi_px >= 0:  # the capture was taken on the join without the band
        prof = None
    if prof and prof["sha256"] == source_sha256(prof["sources"]):
        traffic = prof["bytes_per_entry"] * entries
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    ent_peak = POPC_PER_CLK_SM / 4.0 * n_sm * sm_mhz * 1e6
    ent_rate = entries / t_match
    fp8_peak = 2.0 * pk["bf16_tflops"] * 1e12  # nominal FP8 / BF16 dense ratio 4.5 / 2.25
    return {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"], "traffic": traffic, "kernel": kernel,
            "units_per_launch": entries, "unit_def": "lookup-table entries (one 128-bit Hamming each)",
            "queries_per_launch": queries, "kernel_ms": t_match * 1e3,
            "bytes_def": "touched bytes: 20 B per entry (index + code) + %d B per query (k rows, query row, "
                         "code, bucket ids, offsets)" % (p.top_k * 128 + 128 + 16 + 8 + 48),
            "peak_def": "HBM copy bandwidth (%s)" % pk["source"],
            "traffic_def": "dram bytes read + written per launch, per-entry figure of an ncu capture "
                           "scaled by the entries; null when the kernel source differs from the profiled one",
            "dram_frac": (traffic / t_match / 1e9 / pk["hbm_gbs"]) if traffic else None,
            "alu_view": {"achieved_gentries_s": ent_rate / 1e9, "peak_gentries_s": ent_peak / 1e9,
                         "frac": ent_rate / ent_peak,
                         "note": "CUDA-core Hamming ceiling: 16 POPC/clk/SM / 4 POPC per entry x %d SMs "
                                 "(queried) x %.0f MHz" % (n_sm, sm_mhz)},
            "tensor_view": {"achieved_tflops": 256.0 * entries / t_match / 1e12, "peak_tflops": fp8_peak / 1e12,
                            "frac": 256.0 * entries / t_match / fp8_peak,
                            "note": "+-1 FP8 contraction, 2 x 128 flop per entry; peak = 2 x measured BF16"}}


def run_ours(args):
    import torch
    import paper_1805_08995_gb300 as ch
    from paper_1805_08995_gb300 import build as chbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.gpus != world:
        raise SystemExit("--gpus %d but WORLD_SIZE %d" % (args.gpus, world))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        chbuild.build()
    if dist:
        dist.barrier()
    ch._load()

    split_pairs = args.split == "pairs" and world > 1
    # weak scaling: each rank its own image set; pair split: every rank the same set, its share of the pairs
    s, wdesc = workload(args.workload, 0 if args.split == "pairs" else rank, args.precision)
    if args.max_pairs and args.max_pairs < len(s.pairs):
        # profiling case: the whole image set stays resident, fewer pairs are matched
        s.pairs = s.pairs[:args.max_pairs]
        if s.F is not None:
            s.F = s.F[:args.max_pairs]
        wdesc += " (first %d pairs only)" % args.max_pairs
    P_job = len(s.pairs)
    if split_pairs:
        from paper_1805_08995_gb300 import shard as shd
        mine = shd.shard_pairs(s.pairs, s.img_off, world, rank)
        s.pairs = s.pairs[mine]
        if s.F is not None:
            s.F = s.F[mine]
        wdesc += " (pairs split over %d ranks by N_A*N_B, LPT)" % world
    if args.tau is not None:
        wdesc += ", Hamming threshold tau = %d" % args.tau
    prec = ch.CASHASH_BF16 if args.precision == "bf16" else ch.CASHASH_FP32
    sched = ch.CASHASH_SCHED_PERSISTENT if args.schedule == "persistent" else ch.CASHASH_SCHED_PER_PAIR
    band = s.F is not None
    flags = run_flags(args)
    pk = dict(epi_px=4.0) if band else {}
    if args.tau is not None:
        pk["tau"] = args.tau
    p = ch.cashash_default_params(precision=prec, schedule=sched, flags=flags, **pk)
    ctx = ch.cashash_create(p, s.R)
    ds = ch.DeviceSet(p, s.img_off, s.desc, s.kpts if band else None)
    plan = ch.cashash_plan_create(ctx, ds, s.pairs)
    P = len(s.pairs)
    cap = int(s.sizes()[s.pairs[:, 0]].sum())
    dev = torch.device("cuda", local)
    moff = torch.zeros(P + 1, dtype=torch.int64, device=dev)
    mt = torch.zeros((cap, 2), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    chunk_matches = [0]

    def count_chunk(first, off, m):
        chunk_matches[0] += int(off[-1])
        return False

    def step():
        ch.cashash_build_codes(ctx, ds, stream=stream)
        if args.chunk_pairs:  # resumable chunked path: a plan per chunk, lists flushed to host per chunk
            chunk_matches[0] = 0
            ch.cashash_match_chunked(ctx, ds, s.pairs, args.chunk_pairs, count_chunk, F=F_dev, stream=stream)
        else:
            ch.cashash_match_plan(ctx, plan, moff, mt, cap, F=F_dev, stream=stream)

    F_dev = torch.from_numpy(np.ascontiguousarray(s.F)).to(dev) if band else None
    if args.kernel != "auto" and sched == ch.CASHASH_SCHED_PERSISTENT:
        kid = {"join": ch.CASHASH_KERNEL_JOIN, "join_tc": ch.CASHASH_KERNEL_JOIN_TC, "query": ch.CASHASH_KERNEL_QUERY,
               "warp": ch.CASHASH_KERNEL_WARP}
        ch.cashash_plan_set_tuning(plan, kid[args.kernel], 4 if args.kernel == "join" else 512, 0)
    tuning = ch.cashash_plan_get_tuning(plan)
    if sched == ch.CASHASH_SCHED_PERSISTENT and not args.no_autotune and args.kernel == "auto":
        ch.cashash_build_codes(ctx, ds, stream=stream)  # the tuner matches the set's current codes
        tuning = ch.cashash_plan_autotune(ctx, plan, F=F_dev, max_pairs=0, stream=stream)
        if args.chunk_pairs:  # the chunks' plans take the tuned configuration
            ch.cashash_set_host_tuning(ctx, tuning["kernel"], tuning["tile"], tuning["ctas_per_sm"])
    # The timed steps run without the library's stage events; the stage times come from a short
    # pass with them after the timed region (the events add a few microseconds per stage).
    ch.cashash_set_profiling(ctx, False)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    if ch.cashash_sync_status(ctx) != ch.CASHASH_OK:
        raise SystemExit("device status not OK after warm-up")
    launches0 = ch.cashash_get_stats(ctx)["n_launches"]

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    step_ms, stage_ms = [], {k: [] for k in ch.STAGES}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        if args.thresholds == "fresh":
            # forget the per-pair Hamming thresholds learned by earlier steps
            ch.cashash_plan_set_threshold_hint(plan, p.code_bits, False)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    stats = ch.cashash_get_stats(ctx)
    launches = stats["n_launches"] - launches0
    if ch.cashash_sync_status(ctx) != ch.CASHASH_OK:
        raise SystemExit("device status not OK after timed steps")

    t_steps = sum(step_ms) / 1e3
    t_max = t_steps
    if dist:
        tt = torch.tensor([t_steps], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    value = (P_job if split_pairs else P * world) * args.steps / t_max
    # parity: the GPU lists of the last timed step, before anything else writes them
    smp = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        smp = oracle_sample(s, args.ref_pairs, flags=run_flags(args), tau=args.tau)
    parity = None
    if smp is not None and not args.chunk_pairs:
        parity = parity_check(smp, moff, mt)
    # stage times (CUDA events inside the library's launch sequence), outside the timed region
    ch.cashash_set_profiling(ctx, True)
    for i in range(1 + min(args.steps, 5)):
        flush.zero_()
        if args.thresholds == "fresh":
            ch.cashash_plan_set_threshold_hint(plan, p.code_bits, False)
        step()
        torch.cuda.synchronize()
        if i == 0:
            continue  # captures the graphs that record the events
        st = ch.cashash_get_stats(ctx)
        for k, v in st["ms_stage"].items():
            if v >= 0:
                stage_ms[k].append(v)
    rf = roofline_of(ch, p, s, ds, stage_ms, tuning, torch.cuda.get_device_properties(dev).multi_processor_count)
    # stage timers and counters of the chunked path cover the last chunk only: no kernel roofline
    roofline = None if args.chunk_pairs else rf

    # end-to-end through the C-ABI with host buffers (pinned descriptors)
    e2e = None
    if not args.no_e2e:
        pinned = torch.from_numpy(s.desc).pin_memory()
        kp_pin = torch.from_numpy(s.kpts).pin_memory().numpy() if band else None
        # pinned host buffers for the inputs and the results (numpy views of pinned torch tensors)
        mo_h = torch.zeros(P + 1, dtype=torch.int64).pin_memory().numpy().view(np.uint64)
        mt_h = torch.zeros((cap, 2), dtype=torch.int32).pin_memory().numpy().view(np.uint32)
        ctx2 = ch.cashash_create(p, s.R)
        ch.cashash_set_profiling(ctx2, False)  # the timed calls run without the stage events
        if tuning.get("kernel"):  # the host path matches with the same configuration as the timed plan
            ch.cashash_set_host_tuning(ctx2, tuning["kernel"], tuning["tile"], tuning["ctas_per_sm"])
        for _ in range(max(1, args.warmup)):
            ch.cashash_run_host(ctx2, pinned, s.img_off, s.pairs, cap, match_off=mo_h, matches=mt_h,
                                kpts=kp_pin, F=s.F if band else None)
        ts, parts = [], []
        dev_stages = ("centre", "project", "reeval", "tables", "calibrate", "match", "fallback", "compact")
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, off, mth = ch.cashash_run_host(ctx2, pinned, s.img_off, s.pairs, cap, match_off=mo_h,
                                               matches=mt_h, kpts=kp_pin, F=s.F if band else None)
            ts.append(time.perf_counter() - t0)
            assert st == ch.CASHASH_OK
        # per-call copy and device stage times from a few more calls with the stage events on
        ch.cashash_set_profiling(ctx2, True)
        for i in range(1 + min(args.steps, 5)):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, off, mth = ch.cashash_run_host(ctx2, pinned, s.img_off, s.pairs, cap, match_off=mo_h,
                                               matches=mt_h, kpts=kp_pin, F=s.F if band else None)
            tb = time.perf_counter() - t0
            assert st == ch.CASHASH_OK
            if i == 0:
                continue
            ms = ch.cashash_get_stats(ctx2)["ms_stage"]
            dev_ms = sum(max(ms[k], 0.0) for k in dev_stages)
            parts.append((ms["h2d"], dev_ms, ms["d2h"], tb * 1e3 - ms["h2d"] - dev_ms - ms["d2h"]))
        t_e2e = statistics.mean(ts)
        if dist:
            tt = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t_e2e = float(tt.item())
        n_m = int(mo_h[P])
        e2e = {"value": (P_job if split_pairs else P * world) / t_e2e, "unit": "pairs/s",
               "ms_each": [round(t * 1e3, 2) for t in ts],
               "h2d_bytes_per_step": int(s.desc.nbytes + 8 * (len(s.img_off)) +
                                         (s.kpts.nbytes + s.F.nbytes if band else 0)),
               "d2h_bytes_per_step": int(8 * (P + 1) + 8 * n_m),
               "breakdown_ms_each": {"h2d": [round(x[0], 3) for x in parts], "device": [round(x[1], 3) for x in parts],
                                     "d2h": [round(x[2], 3) for x in parts],
                                     "host_other": [round(x[3], 3) for x in parts]},
               "breakdown_note": "from separate calls with the library's stage events on: device = the stages "
                                 "on the compute stream after the last copy (the column sums overlap the copy); "
                                 "host_other = wall - h2d - device - d2h"}
        if parity is not None:  # the host path's lists of the sampled pairs too
            e2e["parity_mismatches"] = parity_check(smp, torch.from_numpy(mo_h.view(np.int64)),
                                                    torch.from_numpy(mt_h.view(np.int32)))["mismatches"]
        ctx2.close()

    cpu = None
    if smp is not None:
        # the same oracle on one host thread, on a sample sized for a few seconds
        one = oracle_sample(s, max(8, args.ref_pairs // 16), seed=1, flags=run_flags(args), threads=1,
                            tau=args.tau)
        cpu = {"value": smp["pairs_per_s"], "unit": "pairs/s", "cores": smp["cores"], "kind": "oracle",
               "sample": smp["sample"], "seconds": smp["seconds"],
               "single_thread": {"value": one["pairs_per_s"], "unit": "pairs/s", "cores": 1,
                                 "sample": one["sample"], "seconds": one["seconds"]}}

    extra = None
    if rank == 0 and world == 1 and args.extra_c3 and args.workload == "config1" and not args.chunk_pairs:
        extra = {"config3": config3_forms(ch, torch, dev)}

    if rank == 0:
        stages = {k: (statistics.mean(v) if v else None) for k, v in stage_ms.items()}
        line = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
                "scaling": "strong" if split_pairs else "weak", "vs_baseline": None,
                "dtype": "u8/" + ("bf16" if prec == ch.CASHASH_BF16 else "fp32") + "+f64fix",
                "data": "synthetic",
                "config": {"workload": wdesc, "images": int(s.n_images), "features": int(s.desc.shape[0]),
                           "pairs": P_job if split_pairs else P, "precision": args.precision,
                           "schedule": args.schedule,
                           "thresholds": ("fresh: every timed step calibrates the per-pair Hamming guesses anew"
                                          if args.thresholds == "fresh" else
                                          "learned: guesses carried over from earlier steps"),
                           "split": "pairs (LPT by N_A*N_B, no collective)" if split_pairs else
                                    ("independent image set per rank" if world > 1 else None),
                           "chunked": ("%d pairs per chunk, lists flushed to pinned host memory per chunk"
                                       % args.chunk_pairs) if args.chunk_pairs else None,
                           "l2": "flushed: 256 MiB write between timed steps (outside the events)",
                           "params": "n=128, 6 tables x 8 bits, k=10, ratio 0.8" + (", band 4 px" if band else "") +
                                     (", tau %d" % args.tau if args.tau is not None else "") +
                                     (", mutual check" if args.mutual else "") +
                                     (", single candidates accepted" if args.accept_single else ""),
                           "kernel_tuning": {"kernel": {1: "join", 2: "query", 3: "join_tc", 4: "warp"}.get(tuning["kernel"], "per_pair"),
                                             "tile": tuning["tile"], "ctas_per_sm": tuning["ctas_per_sm"],
                                             "autotuned": tuning["ms_sample"] > 0},
                           "matches_per_step": int(chunk_matches[0] if args.chunk_pairs else stats["n_matches"]),
                           "reevaluated_projections": int(stats["n_reevaluated"])},
                "features_per_s": s.desc.shape[0] * world * args.steps / t_max,
                "stages_ms": stages, "roofline": roofline, "parity": parity, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clocks, "wall_s_timed_region": t_wall}
        if extra:
            line["extra"] = extra
        print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()
    if parity is not None and (parity["mismatches"] or (e2e or {}).get("parity_mismatches")):
        sys.stderr.write("parity check failed: GPU lists differ from the oracle's\n")
        return 1
    return 0


def config3_forms(ch, torch, dev):
    """Config 3 (2,000 images, 59,556 pairs) in the two forms its target
    compares: the batched BF16 form (one persistent launch per step over the
    device pair list, CUDA-graph captured, autotuned on a sample of pairs) and
    the plain FP32 form with one launch per pair.  Device time per step with
    CUDA events, L2 flushed before each step."""
    import synth
    s = synth.config3()
    P = len(s.pairs)
    cap = int(s.sizes()[s.pairs[:, 0]].sum())
    moff = torch.zeros(P + 1, dtype=torch.int64, device=dev)
    mt = torch.zeros((cap, 2), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    out = {"workload": "config3: 2000 images log-uniform 1000..20000 (%d features), 30 neighbours each, "
                       "%d pairs" % (s.desc.shape[0], P)}
    forms = (("batched_bf16", ch.CASHASH_BF16, ch.CASHASH_SCHED_PERSISTENT, 3, 5),
             ("per_pair_fp32", ch.CASHASH_FP32, ch.CASHASH_SCHED_PER_PAIR, 1, 2))
    for name, prec, sched, warm, steps in forms:
        p = ch.cashash_default_params(precision=prec, schedule=sched)
        ctx = ch.cashash_create(p, s.R)
        ds = ch.DeviceSet(p, s.img_off, s.desc)
        plan = ch.cashash_plan_create(ctx, ds, s.pairs)
        tuning = None
        if sched == ch.CASHASH_SCHED_PERSISTENT:
            ch.cashash_build_codes(ctx, ds, stream=stream)
            tuning = ch.cashash_plan_autotune(ctx, plan, max_pairs=8000, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms = []
        for it in range(warm + steps):
            flush.zero_()
            e0.record(stream)
            ch.cashash_build_codes(ctx, ds, stream=stream)
            ch.cashash_match_plan(ctx, plan, moff, mt, cap, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if it >= warm:
                ms.append(e0.elapsed_time(e1))
        if ch.cashash_sync_status(ctx) != ch.CASHASH_OK:
            raise SystemExit("device status not OK in the config-3 forms")
        out[name] = {"pairs_per_s": P / (statistics.mean(ms) / 1e3), "ms_per_step": statistics.mean(ms),
                     "steps": steps, "warmup": warm, "matches": int(moff[P].item())}
        if tuning:
            out[name]["kernel_tuning"] = {"kernel": {1: "join", 2: "query", 3: "join_tc", 4: "warp"}.get(tuning["kernel"]),
                                          "tile": tuning["tile"], "ctas_per_sm": tuning["ctas_per_sm"]}
        plan.close()
        ctx.close()
    out["ratio_batched_over_per_pair"] = out["batched_bf16"]["pairs_per_s"] / out["per_pair_fp32"]["pairs_per_s"]
    out["same_matches"] = out["batched_bf16"]["matches"] == out["per_pair_fp32"]["matches"]
    return out


def run_tau_sweep(args):
    """The Hamming threshold tau of the ranking (Sec. 6) swept on the config-1
    set (BF16 form, batched, autotuned per tau): per tau the device time per
    step, the matches, the recall of the planted noisy copies (a planted
    correspondence (q, j) of pair (A, B): q is a copy of B's row j or j a copy
    of A's row q) and an oracle parity check on sampled pairs.  Prints one
    JSON line."""
    import torch
    import paper_1805_08995_gb300 as ch
    from paper_1805_08995_gb300 import build as chbuild
    import synth
    if int(os.environ.get("WORLD_SIZE", "1")) != 1 or args.gpus != 1:
        raise SystemExit("--tau-sweep runs on one GPU")
    torch.cuda.set_device(0)
    chbuild.build()
    ch._load()
    taus = [int(x) for x in args.tau_sweep.split(",") if x.strip()]
    s, wdesc = workload("config1", 0, "bf16")
    P = len(s.pairs)
    cap = int(s.sizes()[s.pairs[:, 0]].sum())
    dev = torch.device("cuda", 0)
    moff = torch.zeros(P + 1, dtype=torch.int64, device=dev)
    mt = torch.zeros((cap, 2), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    planted = synth.planted_pairs(s.truth["copies"], s.pairs)
    pk_keys = np.array(sorted((i << 48) | (q << 24) | j for i, st in enumerate(planted) for q, j in st), np.int64)
    rows = []
    sampler = ClockSampler(0)
    sampler.start()
    for tau in taus:
        p = ch.cashash_default_params(precision=ch.CASHASH_BF16, schedule=ch.CASHASH_SCHED_PERSISTENT, tau=tau)
        ctx = ch.cashash_create(p, s.R)
        ds = ch.DeviceSet(p, s.img_off, s.desc)
        plan = ch.cashash_plan_create(ctx, ds, s.pairs)
        ch.cashash_build_codes(ctx, ds, stream=stream)
        tuning = ch.cashash_plan_autotune(ctx, plan, max_pairs=0, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms = []
        for it in range(args.warmup + args.steps):
            flush.zero_()
            e0.record(stream)
            ch.cashash_build_codes(ctx, ds, stream=stream)
            ch.cashash_match_plan(ctx, plan, moff, mt, cap, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if it >= args.warmup:
                ms.append(e0.elapsed_time(e1))
        if ch.cashash_sync_status(ctx) != ch.CASHASH_OK:
            raise SystemExit("device status not OK at tau %d" % tau)
        off = moff.cpu().numpy().view(np.uint64)
        n = int(off[-1])
        m = mt[:n].cpu().numpy().view(np.uint32).astype(np.int64)
        pi = np.repeat(np.arange(P, dtype=np.int64), np.diff(off.astype(np.int64)))
        keys = (pi << 48) | (m[:, 0] << 24) | m[:, 1]
        hit = int(np.isin(keys, pk_keys, assume_unique=True).sum())
        smp = oracle_sample(s, 48, seed=tau, tau=tau)
        par = parity_check(smp, moff, mt)
        rows.append({"tau": tau, "pairs_per_s": P / (statistics.mean(ms) / 1e3), "ms_per_step": statistics.mean(ms),
                     "matches": n, "planted_found": hit, "planted": int(len(pk_keys)),
                     "recall": hit / max(1, len(pk_keys)), "precision_vs_planted": hit / max(1, n),
                     "kernel_tuning": {"kernel": {1: "join", 2: "query", 3: "join_tc", 4: "warp"}.get(tuning["kernel"]),
                                       "tile": tuning["tile"], "ctas_per_sm": tuning["ctas_per_sm"]},
                     "parity": {"pairs_checked": par["pairs_checked"], "mismatches": par["mismatches"]}})
        plan.close()
        ctx.close()
    clocks = sampler.stop()
    base = next((r for r in rows if r["tau"] >= 128), None)
    for r in rows:
        r["recall_vs_tau128"] = r["recall"] / base["recall"] if base else None
        r["speed_vs_tau128"] = r["pairs_per_s"] / base["pairs_per_s"] if base else None
    line = {"metric": METRIC, "unit": "pairs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "data": "synthetic", "dtype": "u8/bf16+f64fix",
            "config": {"workload": wdesc, "l2": "flushed: 256 MiB write before every timed step",
                       "recall_def": "planted noisy-copy correspondences found among the matches"},
            "tau_sweep": rows, "clocks": clocks}
    print(json.dumps(line))
    return 1 if any(r["parity"]["mismatches"] for r in rows) else 0


# ---------------------------------------------------------------------------
# Ga-CasHash: first stage (top-scale subsets, CasHash, RANSAC F) + guided matching
# ---------------------------------------------------------------------------

def oracle_ga_sample(s, n_pairs: int, gp, words, seed: int = 0):
    """Times the oracle's two stages on a bounded sample of pairs (all host
    cores for codes and matching; the RANSAC loop is numpy) and extrapolates:
    codes by feature count, matching by N_A * N_B, RANSAC by pairs.  Returns
    (pairs/s, cores, sample text, seconds)."""
    import oracle as orc
    from oracle import ga as oga
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    P = len(s.pairs)
    pick = np.sort(rng.choice(P, size=min(n_pairs, P), replace=False))
    sp = s.pairs[pick]
    imgs = np.unique(sp)
    sizes = s.sizes()
    remap = {int(i): k for k, i in enumerate(imgs)}
    sp2 = np.array([[remap[int(a)], remap[int(b)]] for a, b in sp], np.uint32)
    t0 = time.perf_counter()
    mu = orc.mean(s.desc)
    t_mean = time.perf_counter() - t0
    rows = np.concatenate([np.arange(int(s.img_off[i]), int(s.img_off[i + 1])) for i in imgs])
    off = np.zeros(len(imgs) + 1, np.uint64)
    off[1:] = np.cumsum(sizes[imgs])
    desc, kpts, scale = s.desc[rows], s.kpts[rows], s.scale[rows]
    po1, po2 = orc.params(), orc.params(epi_px=4.0)
    t0 = time.perf_counter()
    sel, sub = oga.top_scale(scale, off, gp.top_pct)
    d1 = np.ascontiguousarray(desc[sel.astype(np.int64)])
    c1, b1 = oracle_codes_parallel(orc, d1, s.R, po1, mu, cores)
    t_codes1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    moff, mt = orc.match_pairs(d1, sub, c1, b1, sp2, po1, n_threads=cores)
    t_match1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    k1 = kpts[sel.astype(np.int64)]
    F = np.zeros((len(sp2), 9))
    acc = np.zeros(len(sp2), bool)
    for i, (a, b) in enumerate(sp2):
        lo, hi = int(moff[i]), int(moff[i + 1])
        q = mt[lo:hi, 0].astype(np.int64) + int(sub[a])
        j = mt[lo:hi, 1].astype(np.int64) + int(sub[b])
        Fi, info = oga.estimate_F(k1[q], k1[j], words[pick[i]], gp)
        F[i], acc[i] = Fi.ravel(), bool(info[3])
    t_ransac = time.perf_counter() - t0
    t0 = time.perf_counter()
    c2, b2 = oracle_codes_parallel(orc, desc, s.R, po2, mu, cores)
    t_codes2 = time.perf_counter() - t0
    t0 = time.perf_counter()
    if acc.any():
        orc.match_pairs(desc, off, c2, b2, sp2[acc], po2, n_threads=cores, F=F[acc], kpts=kpts)
    t_match2 = time.perf_counter() - t0
    n_all, n_smp = float(sizes.sum()), float(len(rows))
    w_all = float((sizes[s.pairs[:, 0]] * sizes[s.pairs[:, 1]]).sum())
    w_smp = float((sizes[sp[:, 0]] * sizes[sp[:, 1]]).sum())
    job = (t_mean + (t_codes1 + t_codes2) * n_all / n_smp + (t_match1 + t_match2) * w_all / w_smp +
           t_ransac * P / len(sp))
    text = ("oracle (C codes and matching on %d threads, numpy RANSAC): %d of %d pairs through both stages "
            "(%d accepted); extrapolated by features, N_A*N_B and pair count" % (cores, len(sp), P, int(acc.sum())))
    return P / job, cores, text, t_mean + t_codes1 + t_match1 + t_ransac + t_codes2 + t_match2


def run_ga(args):
    """One step = full-set codes (stage-2 context), the first stage on the
    top-20 % subsets (selection, codes with the full set's centre, CasHash,
    RANSAC F per pair), then guided matching (band 4 px with the estimated F)
    of the accepted pairs; host work between the stages (reading which pairs
    were accepted, the stage-2 plan) is inside the timed step."""
    import torch
    import paper_1805_08995_gb300 as ch
    from paper_1805_08995_gb300 import build as chbuild
    import synth
    if int(os.environ.get("WORLD_SIZE", "1")) != 1 or args.gpus != 1:
        raise SystemExit("--ga runs on one GPU")
    torch.cuda.set_device(0)
    chbuild.build()
    ch._load()
    s, wdesc = workload("config4", 0)
    P = len(s.pairs)
    bf = dict(precision=ch.CASHASH_BF16, schedule=ch.CASHASH_SCHED_PERSISTENT)
    p1 = ch.cashash_default_params(**bf)
    p2 = ch.cashash_default_params(epi_px=4.0, **bf)
    ctx1, ctx2 = ch.cashash_create(p1, s.R), ch.cashash_create(p2, s.R)
    ds = ch.DeviceSet(p2, s.img_off, s.desc, s.kpts)
    dev = torch.device("cuda", 0)
    scale = torch.from_numpy(s.scale).to(dev)
    gp = ch.cashash_ga_default_params(kernel={"auto": 0, "join": 1, "query": 2}[args.ga_kernel])
    words_h = synth.ransac_words(4, P, gp.n_hyp)
    words = torch.from_numpy(words_h.view(np.int32)).to(dev)
    cap = int(s.sizes()[s.pairs[:, 0]].sum())
    moff = torch.zeros(P + 1, dtype=torch.int64, device=dev)
    mt = torch.zeros((max(cap, 1), 2), dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = {}

    def step(profile=False):
        t0 = time.perf_counter()
        ch.cashash_build_codes(ctx2, ds)
        mu = ch.cashash_get_mean(ctx2)
        F, info = ch.cashash_ga_stage1(ctx1, ds, scale, mu, s.pairs, words, gp)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        acc = torch.nonzero(info[:, 3]).squeeze(1)
        acc_h = acc.cpu().numpy()
        pairs2 = s.pairs[acc_h]
        F2 = F.index_select(0, acc).contiguous()
        cap2 = int(s.sizes()[pairs2[:, 0]].sum()) if len(pairs2) else 0
        plan = ch.cashash_plan_create(ctx2, ds, pairs2)
        ch.cashash_match_plan(ctx2, plan, moff, mt, max(cap2, 1), F=F2)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        out.update(F=F, info=info, acc=acc_h, pairs2=pairs2, matches=int(moff[len(pairs2)].item()))
        if profile:
            out["stats"] = ch.cashash_get_stats(ctx2)
        plan.close()
        return t1 - t0, t2 - t1

    for _ in range(args.warmup):
        flush.zero_()
        step()
    if ch.cashash_sync_status(ctx2) != ch.CASHASH_OK or ch.cashash_sync_status(ctx1) != ch.CASHASH_OK:
        raise SystemExit("device status not OK after warm-up")
    ch.cashash_set_profiling(ctx2, True)
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    ts1, ts2 = [], []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        a, b = step(profile=True)
        ts1.append(a)
        ts2.append(b)
    clocks = sampler.stop()
    t_step = statistics.mean(ts1) + statistics.mean(ts2)
    info = out["info"].cpu().numpy().view(np.uint32)
    Fe = out["F"].cpu().numpy()
    acc = out["acc"]
    # quality: |<F_est, F_gt>| of unit-norm matrices over the accepted pairs, and the guided matches
    # with the estimated F against those with the ground-truth F (same pairs, outside the timed steps)
    cosang = np.abs(np.sum(Fe[acc] * s.F[acc], axis=1)) if len(acc) else np.zeros(0)
    plan = ch.cashash_plan_create(ctx2, ds, out["pairs2"])
    mo2 = torch.zeros(len(acc) + 1, dtype=torch.int64, device=dev)
    mt2 = torch.zeros_like(mt)
    ch.cashash_match_plan(ctx2, plan, mo2, mt2, mt.shape[0], F=torch.from_numpy(np.ascontiguousarray(s.F[acc])).to(dev))
    torch.cuda.synchronize()
    n_gt = int(mo2[-1].item())
    same = 0
    if out["matches"] and n_gt:
        def keys(m_dev, off_dev, n):  # (pair, q, j) as one int64, q and j < 2^24
            mm = m_dev[:n].cpu().numpy().view(np.uint32).astype(np.int64)
            pi = np.repeat(np.arange(len(acc), dtype=np.int64), np.diff(off_dev[:len(acc) + 1].cpu().numpy()))
            return (pi << 48) | (mm[:, 0] << 24) | mm[:, 1]
        same = int(len(np.intersect1d(keys(mt, moff, out["matches"]), keys(mt2, mo2, n_gt))))
    plan.close()
    st = out["stats"]["ms_stage"]
    # dominant kernel: the guided stage's band join over the accepted pairs
    import types
    s2 = types.SimpleNamespace(img_off=s.img_off, pairs=out["pairs2"], sizes=s.sizes)
    roofline = roofline_of(ch, p2, s2, ds, {"match": [st["match"]]}, {"kernel": ch.CASHASH_KERNEL_JOIN},
                           torch.cuda.get_device_properties(0).multi_processor_count)
    roofline["kernel"] = "k_join (band, guided stage)"
    cpu = None
    if not args.no_cpu_baseline:
        v, cores, text, secs = oracle_ga_sample(s, max(16, args.ref_pairs // 8), oga_params(gp), words_h)
        cpu = {"value": v, "unit": "pairs/s", "cores": cores, "kind": "oracle", "sample": text, "seconds": secs}
    line = {"metric": METRIC, "value": P / t_step, "unit": "pairs/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/bf16+f64fix, f64 geometry", "data": "synthetic",
            "config": {"workload": wdesc.replace("ground-truth F", "F estimated by the first stage (Ga-CasHash)"),
                       "pairs": P, "features": int(s.desc.shape[0]),
                       "ga": {"stage1_kernel": args.ga_kernel, "confidence": gp.confidence, "top_pct": gp.top_pct, "min_matches": gp.min_matches, "n_hyp": gp.n_hyp,
                              "accept": "%d/%d inliers" % (gp.inlier_num, gp.inlier_den),
                              "thresh_px": gp.thresh_px},
                       "l2": "flushed: 256 MiB write before every step"},
            "stages_ms": {"stage1": statistics.mean(ts1) * 1e3, "stage2": statistics.mean(ts2) * 1e3,
                          "stage2_match_kernel": st["match"], "stage2_fallback": st["fallback"]},
            "ga": {"pairs_with_F": int((info[:, 2] != 0xFFFFFFFF).sum()), "accepted": int(len(acc)),
                   "stage1_matches_median": float(np.median(info[:, 0])),
                   "hypotheses_run_mean": float(np.mean(info[:, 4])),
                   "inlier_ratio_median": float(np.median(info[acc, 1] / np.maximum(info[acc, 0], 1)))
                   if len(acc) else None,
                   "cos_F_est_gt_median": float(np.median(cosang)) if len(cosang) else None,
                   "cos_F_est_gt_min": float(cosang.min()) if len(cosang) else None,
                   "guided_matches": out["matches"], "guided_matches_with_gt_F": n_gt,
                   "common_with_gt_F": same},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": None, "clocks": clocks}
    print(json.dumps(line))
    ctx1.close()
    ctx2.close()
    return 0


def oga_params(gp):
    from oracle import ga as oga
    return oga.GaParams(top_pct=gp.top_pct, min_matches=gp.min_matches, n_hyp=gp.n_hyp, inlier_num=gp.inlier_num,
                        inlier_den=gp.inlier_den, thresh_px=gp.thresh_px, confidence=gp.confidence)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config1", choices=["config0", "config1", "config3", "config4"])
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16"])
    ap.add_argument("--schedule", default="persistent", choices=["persistent", "per_pair"])
    ap.add_argument("--ref-pairs", type=int, default=1200)
    ap.add_argument("--max-pairs", type=int, default=0, help="match only the first N pairs (profiling case)")
    ap.add_argument("--thresholds", default="learned", choices=["learned", "fresh"],
                    help="fresh: clear the learned per-pair Hamming thresholds before every timed step")
    ap.add_argument("--no-autotune", action="store_true", help="keep the plan's default kernel configuration")
    ap.add_argument("--kernel", default="auto", choices=["auto", "join", "join_tc", "query", "warp"],
                    help="batched matching kernel: autotuned (auto) or forced")
    ap.add_argument("--mutual", action="store_true", help="mutual check (every pair matched in both directions)")
    ap.add_argument("--chunk-pairs", type=int, default=0,
                    help="time the resumable chunked path (cashash_match_chunked) with this many pairs per chunk")
    ap.add_argument("--accept-single", action="store_true", help="a single ranked candidate matches")
    ap.add_argument("--tau", type=int, default=None,
                    help="Hamming threshold of the ranking (Sec. 6): candidates above it are dropped; default off")
    ap.add_argument("--tau-sweep", default="",
                    help="comma-separated tau values: one line with pairs/s, matches and planted-copy recall per "
                         "tau on the config-1 set (e.g. 20,30,40,50,60,128)")
    ap.add_argument("--split", default="images", choices=["images", "pairs"],
                    help="under torchrun: each rank its own image set (weak scaling) or a share of one "
                         "workload's pairs (LPT split, strong scaling)")
    ap.add_argument("--no-extra-c3", dest="extra_c3", action="store_false",
                    help="skip the config-3 comparison of the batched BF16 form and the one-pair FP32 form")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ga", action="store_true",
                    help="Ga-CasHash on config 4: F estimated by the first stage, then guided matching")
    ap.add_argument("--ga-kernel", default="auto", choices=["auto", "join", "query"],
                    help="matching kernel of the first stage's subsets")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.ga:
        return run_ga(args)
    if args.tau_sweep:
        return run_tau_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
