"""Multi-GPU sharding of the sketch path: host logic only, the arithmetic stays in libpmh.

Sets are independent (Eq. signature_def is per set), so a batch shards by set with no data
exchange: `partition_sets` cuts the CSR batch into contiguous set ranges of about equal cost,
one per rank, and every rank sketches its range on its own GPU (weak or strong scaling with
no collective on the data path).

One huge set shards by element range.  Its signature is the lexicographic (value, id) minimum,
component by component, of the partial signatures of disjoint parts (Eq. signature_def over a
disjoint union), so each rank sketches its range with exact values (out_q), the partials are
gathered with one all_gather, and `pmh_merge` combines them.

The all-pairs estimator counts (Eq. jaccard_estimator) shard as a 2-D partition of the pair
matrix: `pair_tiles` cuts its upper triangle into square tiles dealt to the ranks by pair count;
`estimate_jp_sharded` all-gathers the signature rows (each rank holds those of its own sets: the
one exchange step) and counts the pairs of this rank's tiles with pmh_estimate_jp_block.
"""
from __future__ import annotations


import numpy as np


def harmonic(m: int) -> float:
    return float(np.sum(1.0 / np.arange(1, m + 1)))


def set_costs(sizes, m: int) -> np.ndarray:
    """Work model of one item: every element is hashed (n) plus about m*H_m*ln(n+1) points
    (the early-stop work of Sec. ProbMinHash1, the paper's m*H_m*H_n, with H_n ~ ln n)."""
    sizes = np.asarray(sizes, dtype=np.float64)
    return sizes + m * harmonic(m) * np.log1p(sizes)


def partition_sets(offsets, m: int, world: int) -> np.ndarray:
    """Set boundaries b[0..world] (b[0] = 0, b[world] = S): rank r takes sets [b[r], b[r+1]),
    contiguous, with about equal total cost."""
    offsets = np.asarray(offsets, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    S = len(offsets) - 1
    cum = np.concatenate([[0.0], np.cumsum(set_costs(np.diff(offsets), m))])
    targets = cum[-1] * np.arange(1, world) / world
    hi = np.clip(np.searchsorted(cum, targets, side="left"), 1, S)     # cum[hi-1] < t <= cum[hi]
    inner = np.where(targets - cum[hi - 1] < cum[hi] - targets, hi - 1, hi)   # the nearer set boundary
    b = np.concatenate([[0], inner, [S]]).astype(np.int64)
    return np.maximum.accumulate(b)


def partition_elements(n: int, world: int) -> np.ndarray:
    """Element boundaries e[0..world] of one set split into `world` near-equal contiguous ranges."""
    if world < 1:
        raise ValueError("world must be >= 1")
    return (np.arange(world + 1, dtype=np.int64) * int(n)) // world


def rank_slice(offsets, bounds, rank: int):
    """(set_lo, set_hi, elem_lo, elem_hi, rebased offsets) of rank `rank`'s part of a CSR batch."""
    offsets = np.asarray(offsets, dtype=np.int64)
    s0, s1 = int(bounds[rank]), int(bounds[rank + 1])
    e0, e1 = int(offsets[s0]), int(offsets[s1])
    return s0, s1, e0, e1, offsets[s0:s1 + 1] - e0


def gather_partials(q, z, group=None):
    """All-gathers one partial signature per rank: q f64[m], z i64[m] -> Q [world, m], Z [world, m]
    (rank order).  Works on any backend whose tensors q and z live on (gloo: CPU, nccl: CUDA)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    qs = [torch.empty_like(q) for _ in range(world)]
    zs = [torch.empty_like(z) for _ in range(world)]
    dist.all_gather(qs, q.contiguous(), group=group)
    dist.all_gather(zs, z.contiguous(), group=group)
    return torch.stack(qs), torch.stack(zs)


def sketch_set_sharded(handle, ids, weights, m: int, variant: str, precision: int, seed: int = 0,
                       group=None, gather=gather_partials):
    """Signature of one set whose elements are spread over the ranks of `group`: `ids`/`weights`
    are this rank's elements (device tensors).  Returns (q [m], z [m]) on every rank, identical to
    the signature of the whole set (Eq. signature_def)."""
    import torch
    dev = handle.device
    off = torch.tensor([0, ids.numel()], dtype=torch.int64, device=dev)
    z, q, st = handle.sketch_batch(ids, weights, off, m, [variant], precision, seed, with_q=True)
    code = int(st.max().item())
    if code != 0:
        from .pmh import PmhError
        raise PmhError(code, "partial sketch of this rank's elements failed")
    Q, Z = gather(q[0, 0], z[0, 0], group)
    return handle.merge(Q.contiguous(), Z.contiguous())


def pair_tiles(n: int, world: int, tile: int | None = None):
    """2-D partition of the upper triangle (diagonal included) of the n x n pair matrix.

    The rows are cut into blocks of `tile` rows (default: enough blocks for about four tiles per
    rank); tile (I, J), I <= J, covers rows of block I against rows of block J, and a diagonal tile
    holds the pairs a <= b.  Tiles go to ranks longest first, each to the rank with the fewest pairs
    so far.  Returns per rank a list of (r0, r1, c0, c1)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    n = int(n)
    if n == 0:
        return [[] for _ in range(world)]
    if tile is None:
        blocks = max(1, int(np.ceil(np.sqrt(8.0 * world))))
        tile = max(1, -(-n // blocks))
    edges = list(range(0, n, tile)) + [n]
    tiles = []
    for i in range(len(edges) - 1):
        for j in range(i, len(edges) - 1):
            r0, r1, c0, c1 = edges[i], edges[i + 1], edges[j], edges[j + 1]
            k = r1 - r0
            pairs = k * (k + 1) // 2 if i == j else k * (c1 - c0)
            tiles.append((pairs, r0, r1, c0, c1))
    tiles.sort(key=lambda t: (-t[0], t[1], t[3]))
    load = [0] * world
    out = [[] for _ in range(world)]
    for pairs, r0, r1, c0, c1 in tiles:
        r = min(range(world), key=lambda x: (load[x], x))
        load[r] += pairs
        out[r].append((r0, r1, c0, c1))
    return out


def tile_pairs(t) -> int:
    """Number of pairs a tile (r0, r1, c0, c1) holds (a <= b on the diagonal)."""
    r0, r1, c0, c1 = t
    return (r1 - r0) * (r1 - r0 + 1) // 2 if (r0, r1) == (c0, c1) else (r1 - r0) * (c1 - c0)


def gather_rows(local, group=None):
    """All-gathers row blocks of unequal length (rank order): local [k_r, m] -> [sum k_r, m]."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    k = torch.tensor([local.shape[0]], dtype=torch.int64, device=local.device)
    ks = [torch.empty_like(k) for _ in range(world)]
    dist.all_gather(ks, k, group=group)
    sizes = [int(x.item()) for x in ks]
    kmax = max(sizes) if sizes else 0
    pad = torch.zeros((kmax, local.shape[1]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:sz] for p, sz in zip(parts, sizes)])


def estimate_jp_sharded(local_sigs, group=None, count_block=None, gather=gather_rows, handle=None):
    """Equal-component counts of all signature pairs over the ranks of `group`.

    local_sigs: this rank's signature rows [k_r, m] (int64 view of uint64); the full table is the
    ranks' rows in rank order.  Every rank all-gathers the table, then counts the pairs of its own
    tiles (pair_tiles) with count_block(A, B) -> [len A, len B] counts (default: the handle's
    pmh_estimate_jp_block).  Returns (n, [(r0, r1, c0, c1, counts)]); diagonal tiles hold the full
    square block (its lower triangle repeats the upper)."""
    import torch.distributed as dist
    full = gather(local_sigs, group)
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if count_block is None:
        count_block = handle.estimate_jp_block
    out = []
    for r0, r1, c0, c1 in pair_tiles(full.shape[0], world)[rank]:
        out.append((r0, r1, c0, c1, count_block(full[r0:r1].contiguous(), full[c0:c1].contiguous())))
    return full.shape[0], out


def balance(costs_per_rank) -> float:
    """max / mean of the ranks' costs (1.0 = perfect balance)."""
    c = np.asarray(costs_per_rank, dtype=np.float64)
    return float(c.max() / c.mean()) if c.mean() > 0 else 1.0


__all__ = ["harmonic", "set_costs", "partition_sets", "partition_elements", "rank_slice", "gather_partials",
           "sketch_set_sharded", "pair_tiles", "tile_pairs", "gather_rows", "estimate_jp_sharded", "balance"]
