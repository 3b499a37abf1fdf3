"""Host logic of the multi-GPU path, run as world-size-2 gloo ranks on CPU.

Sets are independent, so a batch shards by set; one huge set shards by element range and is
recombined by the component-wise lexicographic minimum of the partial signatures (Eq.
signature_def over a disjoint union).  The partial signatures here come from the oracle; the
GPU merge kernel itself is checked against whole-set sketches in test_estimate_gpu.py.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_1911_00675_gb300 import shard
from paper_1911_00675_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _lexmin(Q, Z):
    """Component-wise lexicographic (q, id) minimum over rows (test-side checker)."""
    Q = np.asarray(Q)
    Z = np.asarray(Z).view(np.uint64)
    order = np.lexsort((Z, Q), axis=0)[0]
    cols = np.arange(Q.shape[1])
    return Q[order, cols], Z[order, cols]


def _pair_sigs():
    """130 signatures of m = 24 with many equal components (rows drawn from a few base rows)."""
    rng = np.random.default_rng(31)
    base = rng.integers(0, 2**62, size=(5, 24), dtype=np.uint64)
    sig = base[rng.integers(0, 5, size=130)].copy()
    noise = rng.random(sig.shape) < 0.5
    sig[noise] = rng.integers(0, 2**62, size=int(noise.sum()), dtype=np.uint64)
    return sig


def _count_block(a, b):
    """Test-side counting: equal components of every row pair (the estimator's numerator)."""
    a = a.numpy().view(np.uint64)
    b = b.numpy().view(np.uint64)
    return (a[:, None, :] == b[None, :, :]).sum(axis=2)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # (1) a batch sharded by set: every rank sketches its contiguous range
        b = W.random_batch(7, [0, 1, 3, 40, 200, 1000, 5, 2500, 17, 60], 64, "pareto")
        bounds = shard.partition_sets(b.offsets, b.m, world)
        s0, s1, e0, e1, off = shard.rank_slice(b.offsets, bounds, rank)
        mine = np.zeros((b.num_sets, b.m), dtype=np.int64)
        for s in range(s0, s1):
            ids, w = b.set(s)
            _, z, _ = oracle.sketch("3a", ids, w, b.m, seed=2)
            mine[s] = z.view(np.int64)
        got = torch.from_numpy(mine)
        dist.all_reduce(got, op=dist.ReduceOp.SUM)      # disjoint rows: the sum is the union
        # (2) one set sharded by element range: partial signatures, gathered, then merged
        ids, w = W.random_batch(8, [3000], 128, "lognormal").set(0)
        eb = shard.partition_elements(len(ids), world)
        q, z, _ = oracle.sketch("2", ids[eb[rank]:eb[rank + 1]], w[eb[rank]:eb[rank + 1]], 128, seed=5)
        Q, Z = shard.gather_partials(torch.from_numpy(q), torch.from_numpy(z.view(np.int64)))
        # (3) all-pairs counts: rows split unevenly over the ranks, gathered, 2-D tiles per rank
        sig_all = _pair_sigs()
        cut = [0, 57, len(sig_all)]
        local = torch.from_numpy(sig_all[cut[rank]:cut[rank + 1]].view(np.int64).copy())
        n, tiles = shard.estimate_jp_sharded(local, count_block=_count_block)
        flat = [np.array([r0, r1, c0, c1] + list(cnt.reshape(-1)), dtype=np.int64) for r0, r1, c0, c1, cnt in tiles]
        np.save(os.path.join(out_dir, f"tiles{rank}.npy"), np.array(flat, dtype=object), allow_pickle=True)
        if rank == 0:
            np.save(os.path.join(out_dir, "batch.npy"), got.numpy())
            np.save(os.path.join(out_dir, "Q.npy"), Q.numpy())
            np.save(os.path.join(out_dir, "Z.npy"), Z.numpy())
            np.save(os.path.join(out_dir, "bounds.npy"), bounds)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def gloo_run(tmp_path_factory):
    import oracle
    oracle.build()
    out = tmp_path_factory.mktemp("gloo")
    mp.start_processes(_rank_main, args=(2, _free_port(), str(out)), nprocs=2, join=True, start_method="spawn")
    return out


def test_batch_shards_cover_and_match_whole(gloo_run):
    import oracle
    b = W.random_batch(7, [0, 1, 3, 40, 200, 1000, 5, 2500, 17, 60], 64, "pareto")
    got = np.load(gloo_run / "batch.npy").view(np.uint64)
    bounds = np.load(gloo_run / "bounds.npy")
    assert bounds[0] == 0 and bounds[-1] == b.num_sets and np.all(np.diff(bounds) >= 0)
    assert 0 < bounds[1] < b.num_sets                   # both ranks get work
    for s in range(b.num_sets):
        ids, w = b.set(s)
        _, z, _ = oracle.sketch("3a", ids, w, b.m, seed=2)
        assert np.array_equal(got[s], z), s


def test_element_shards_merge_to_whole_set(gloo_run):
    import oracle
    ids, w = W.random_batch(8, [3000], 128, "lognormal").set(0)
    Q = np.load(gloo_run / "Q.npy")
    Z = np.load(gloo_run / "Z.npy")
    assert Q.shape == (2, 128) and Z.shape == (2, 128)
    qm, zm = _lexmin(Q, Z)
    q, z, _ = oracle.sketch("2", ids, w, 128, seed=5)
    assert np.array_equal(zm, z) and np.array_equal(qm, q)
    # each rank's partial differs from the whole in some components (the merge does real work)
    assert not np.array_equal(Z[0].view(np.uint64), z) and not np.array_equal(Z[1].view(np.uint64), z)


def test_partition_sets_properties():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        sizes = np.floor(10 ** (5 * rng.random(500))).astype(np.int64)
        off = np.concatenate([[0], np.cumsum(sizes)])
        b = shard.partition_sets(off, 1024, world)
        assert len(b) == world + 1 and b[0] == 0 and b[-1] == 500 and np.all(np.diff(b) >= 0)
        cost = shard.set_costs(sizes, 1024)
        per_rank = [cost[b[r]:b[r + 1]].sum() for r in range(world)]
        # contiguous ranges: imbalance bounded by one set's cost
        assert max(per_rank) - cost.sum() / world <= cost.max() + 1e-6
    assert list(shard.partition_sets(np.array([0]), 8, 3)) == [0, 0, 0, 0]


def test_partition_elements_and_slices():
    e = shard.partition_elements(10, 3)
    assert list(e) == [0, 3, 6, 10]
    assert list(shard.partition_elements(0, 2)) == [0, 0, 0]
    off = np.array([0, 2, 2, 7, 10])
    s0, s1, e0, e1, sub = shard.rank_slice(off, np.array([0, 2, 4]), 1)
    assert (s0, s1, e0, e1) == (2, 4, 2, 10) and list(sub) == [0, 5, 8]
    with pytest.raises(ValueError):
        shard.partition_elements(5, 0)


def test_pair_tiles_cover_the_upper_triangle_once():
    for n, world in ((130, 2), (1000, 3), (7, 8), (64, 1), (0, 2)):
        tiles = shard.pair_tiles(n, world)
        assert len(tiles) == world
        cover = np.zeros((n, n), dtype=int)
        loads = []
        for lst in tiles:
            loads.append(sum(shard.tile_pairs(t) for t in lst))
            for r0, r1, c0, c1 in lst:
                assert r0 <= c0
                blk = np.ones((r1 - r0, c1 - c0), dtype=int)
                if (r0, r1) == (c0, c1):
                    blk = np.triu(blk)
                cover[r0:r1, c0:c1] += blk
        assert np.array_equal(cover, np.triu(np.ones((n, n), dtype=int)))
        if n >= 100 and world > 1:
            assert max(loads) <= 1.6 * (n * (n + 1) // 2) / world     # balanced within one tile


def test_allpairs_tiles_assemble_to_whole_matrix(gloo_run):
    sig = _pair_sigs()
    n = len(sig)
    full = np.full((n, n), -1, dtype=np.int64)
    for r in range(2):
        for row in np.load(gloo_run / f"tiles{r}.npy", allow_pickle=True):
            r0, r1, c0, c1 = (int(x) for x in row[:4])
            cnt = np.asarray(row[4:], dtype=np.int64).reshape(r1 - r0, c1 - c0)
            full[r0:r1, c0:c1] = np.where(full[r0:r1, c0:c1] < 0, cnt, full[r0:r1, c0:c1])
    import oracle
    ref = oracle.count_allpairs(sig).astype(np.int64)
    iu = np.triu_indices(n)
    assert np.array_equal(full[iu], ref[iu])
