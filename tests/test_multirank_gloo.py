"""Multi-rank pair sharding on CPU: world size 2 over gloo.

Each rank takes its share of the pair list (no data-path collective: pairs
are independent), matches it with the oracle, and the shards are gathered
once at the end; the reassembled lists must equal the single-rank result.
"""
import os
import socket

import numpy as np
import pytest

import synth
from paper_1805_08995_gb300 import shard

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = synth.random_set(1717, [400, 0, 350, 900, 120, 610])
    p = oracle.params(bits_per_table=6)
    mu = oracle.mean(s.desc)
    idx = shard.shard_pairs(s.pairs, s.img_off, world, rank)
    imgs = shard.images_of(s.pairs, idx)
    codes = np.zeros((s.desc.shape[0], 4), np.uint32)
    buckets = np.zeros((s.desc.shape[0], 6), np.uint8)
    for i in imgs:  # a rank hashes only the images its pairs touch
        a, b = int(s.img_off[i]), int(s.img_off[i + 1])
        codes[a:b], buckets[a:b] = oracle.hash_codes(s.desc[a:b], mu, s.R, p)
    off, mt = oracle.match_pairs(s.desc, s.img_off, codes, buckets, s.pairs[idx], p, n_threads=1)
    got = [None] * world
    dist.all_gather_object(got, (idx.tolist(), off.tolist(), mt.tolist()))
    if rank == 0:
        moff, mts = shard.merge_shards(len(s.pairs), [(np.array(i), np.array(o), np.array(m).reshape(-1, 2))
                                                      for i, o, m in got])
        c_all, b_all = oracle.hash_codes(s.desc, mu, s.R, p)
        eoff, emt = oracle.match_pairs(s.desc, s.img_off, c_all, b_all, s.pairs, p)
        ok = np.array_equal(moff, eoff) and np.array_equal(mts, emt)
        with open(os.path.join(out_dir, "result"), "w") as f:
            f.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_matching_equals_single_rank(tmp_path, orc):
    import torch.multiprocessing as mp
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    assert (tmp_path / "result").read_text() == "ok"


def test_shard_split_is_a_balanced_partition():
    s = synth.config1(seed=3, n_images=30, lo=1000, hi=3000)
    cost = shard.pair_costs(s.pairs, s.img_off)
    for world in (1, 2, 3, 4, 7):
        parts = [shard.shard_pairs(s.pairs, s.img_off, world, r) for r in range(world)]
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(s.pairs)))        # a partition
        loads = np.array([cost[p].sum() for p in parts])
        assert loads.max() <= loads.mean() + cost.max()                  # LPT bound
        assert all(np.array_equal(shard.shard_pairs(s.pairs, s.img_off, world, r), parts[r]) for r in range(world))


def test_shard_rejects_bad_rank():
    with pytest.raises(ValueError):
        shard.shard_pairs(np.zeros((1, 2), np.uint32), np.array([0, 1], np.uint64), 2, 2)
