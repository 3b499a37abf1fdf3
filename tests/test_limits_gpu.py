"""Resource caps and the paths that keep a call correct or fail it cleanly.

The paper's loops are finite only through iteration limits (Sec. Experiments).
Here: the cap on one element's points in warp-cooperative expansion fails only
the items that need more (PMH_ERR_ITER_LIMIT, zero rows) and leaves the others
correct; an FP32 item whose contender log overflows is sketched again by the
FP64 kernel of its family in the same call, so its result is the FP64 path's.
Contenders are planted: two elements whose points for one label differ by
1e-7 relative (within the FP32 error bound of 2^-18) and are the two smallest
of that component, found with the oracle on the host.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1911_00675_gb300 import workloads as W
from parity_util import check_sets, run, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    h = pmh.Handle(0)
    yield h
    h.set_limits()
    h.close()


def _planted_pair(variant, m, seed, salt, wa=1e5, rel=1e-7):
    """(ids[2], weights[2], k): element A with weight wa and element B whose point with label k (the
    label of A's first point) lies `rel` relative above A's; both far below any ordinary element's."""
    pool = W.distinct_ids(salt << 20, 12 * m, salt)
    a = pool[:1]
    ha = oracle.sketch(variant, a, np.array([wa]), m, seed=seed)[0]
    k = int(np.argmin(ha))
    for b in pool[1:]:
        bb = np.array([b], dtype=np.uint64)
        hb1 = oracle.sketch(variant, bb, np.array([1.0]), m, seed=seed)[0]
        if int(np.argmin(hb1)) != k:
            continue
        wb = hb1[k] / (ha[k] * (1.0 + rel))
        hb = oracle.sketch(variant, bb, np.array([wb]), m, seed=seed)[0]
        gap = (hb[k] - ha[k]) / ha[k]
        if 0.3 * rel < gap < 3.0 * rel:
            return np.array([a[0], b], dtype=np.uint64), np.array([wa, wb]), k
    raise AssertionError("no partner element found")


def _batch_with_pairs(variant, m, sizes, seed, salt0):
    """Sets of uniform(0,1] weights, each with one planted contender pair."""
    rng = np.random.default_rng(salt0)
    ids_l, w_l, lens = [], [], []
    for j, n in enumerate(sizes):
        pid, pw, _ = _planted_pair(variant, m, seed, salt0 + j)
        ids = W.distinct_ids(int(rng.integers(1, 2**40)), n, int(rng.integers(0, 2**32)))
        w = 1.0 - rng.random(n)
        ids_l += [ids, pid]
        w_l += [w, pw]
        lens.append(n + 2)
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    return W.Batch(np.concatenate(ids_l), np.concatenate(w_l), off, m, (variant,))


@pytest.mark.parametrize("variant", ["1", "2", "3a", "4"])
def test_planted_contenders_resolved_exactly(H, variant):
    # default limits: the contender pair is logged and re-evaluated in FP64 at the end of the item
    from paper_1911_00675_gb300 import pmh
    b = _batch_with_pairs(variant, 256, [0, 40, 3000], seed=4, salt0=11)
    cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
    z, q, st = run(H, b, [variant], 1, seed=4, counters=cnt)
    c = dict(zip(pmh.COUNTERS, cnt.cpu().tolist()))
    assert (st == 0).all()
    assert c["contenders"] >= b.num_sets and c["resolved"] >= 2 * b.num_sets and c["redo"] == 0
    check_sets(b, variant, z[0], q[0], range(b.num_sets), seed=4)


@pytest.mark.parametrize("variant", ["1", "2", "3a", "4"])
def test_contender_overflow_redone_in_fp64(H, variant):
    # no contender records at all: every item with a near-margin event is sketched again by the
    # family's FP64 kernel in the same call, with the FP64 path's result
    from paper_1911_00675_gb300 import pmh
    b = _batch_with_pairs(variant, 256, [1, 40, 3000, 700], seed=4, salt0=21)
    z64, q64, st64 = run(H, b, [variant], 0, seed=4)
    H.set_limits(0, 0)
    try:
        cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
        z32, q32, st32 = run(H, b, [variant], 1, seed=4, counters=cnt)
    finally:
        H.set_limits()
    c = dict(zip(pmh.COUNTERS, cnt.cpu().tolist()))
    assert (st32 == 0).all() and (st64 == 0).all()
    assert c["redo"] == b.num_sets           # every set holds a planted pair
    assert np.array_equal(z32, z64) and np.array_equal(q32, q64)
    check_sets(b, variant, z32[0], q32[0], range(b.num_sets), seed=4)


def test_contender_overflow_in_grid_mode_redone_in_fp64(H):
    # a set above the grid-mode size with a planted pair: the grid item overflows its (empty)
    # contender log and is redone by one FP64 team
    from paper_1911_00675_gb300 import pmh
    b = _batch_with_pairs("3a", 512, [(1 << 20) + 5], seed=2, salt0=31)
    H.set_thresholds()          # grid mode from 2^20 elements
    z64, _, st64 = run(H, b, ["3a"], 0, with_q=False, seed=2)
    H.set_limits(0, 0)
    try:
        cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
        z32, _, st32 = run(H, b, ["3a"], 1, with_q=False, seed=2, counters=cnt)
    finally:
        H.set_limits()
    c = dict(zip(pmh.COUNTERS, cnt.cpu().tolist()))
    assert (st32 == 0).all() and (st64 == 0).all()
    assert c["redo"] == 1
    assert np.array_equal(z32, z64)


@pytest.mark.parametrize("precision", [1, 0], ids=["fp32", "fp64"])
def test_iteration_cap_fails_only_the_items_that_exceed_it(H, precision):
    # ProbMinHash1 and 3 at m = 1024: an element of a tiny set must cover all 1024 labels by itself
    # (about m H_m points), while in sets of thousands of uniform weights no element comes near 64
    # points.  A cap of 40 points (warp-cooperative groups of 32: at most 64 points) fails the
    # tiny sets' items (status, zero rows) and leaves every other item unchanged; the next call
    # with the default cap is whole again.
    b = W.random_batch(61, [1, 5, 300, 20000, 4000, 50000, 2, 9000], 1024, "uniform")
    z0, _, st0 = run(H, b, ["1", "3"], precision, with_q=False, seed=8)
    assert (st0 == 0).all()
    H.set_limits(40, -1)
    try:
        z1, _, st1 = run(H, b, ["1", "3"], precision, with_q=False, seed=8)
    finally:
        H.set_limits()
    bad = st1 != 0
    assert bad.any() and not bad.all()
    assert (st1[bad] == 3).all()                       # PMH_ERR_ITER_LIMIT
    assert (z1[bad] == 0).all()
    assert np.array_equal(z1[~bad], z0[~bad])
    sizes = np.diff(b.offsets)
    assert bad[:, sizes <= 5].all() and not bad[:, sizes >= 4000].any()
    z2, _, st2 = run(H, b, ["1", "3"], precision, with_q=False, seed=8)
    assert (st2 == 0).all() and np.array_equal(z2, z0)


def test_sync_status_reduces_item_statuses(H):
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(62, [10, 20, 30, 40], 64, "uniform")
    w = b.weights.copy()
    w[int(b.offsets[2]) + 3] = -1.0                    # set 2 has a bad weight
    bb = W.Batch(b.ids, w, b.offsets, 64)
    ids, wt, off = to_dev(bb)
    z, _, st = H.sketch_batch(ids, wt, off, 64, ["1", "4"], pmh.FP32_RECHECK, 0)
    rc, counts, first = H.sync_status(st)
    assert rc == pmh.ERR_BAD_WEIGHT and first == 2
    assert counts[0] == 6 and counts[pmh.ERR_BAD_WEIGHT] == 2 and sum(counts) == 8
    z, _, st = H.sketch_batch(ids, wt, off[:3].contiguous(), 64, ["1"], pmh.FP32_RECHECK, 0)
    rc, counts, first = H.sync_status(st)
    assert rc == pmh.OK and first == -1 and counts[0] == 2


def test_estimate_jp_equals_the_earlier_name(H):
    g = torch.Generator().manual_seed(3)
    sigs = torch.randint(0, 6, (130, 77), generator=g, dtype=torch.int64).cuda()
    a = H.estimate_jp(sigs)
    c = H.estimate_allpairs(sigs)
    torch.cuda.synchronize()
    ref = oracle.count_allpairs(sigs.cpu().numpy().view(np.uint64))
    assert np.array_equal(a.cpu().numpy().astype(np.uint16), ref.astype(np.uint16))
    assert torch.equal(a, c)
