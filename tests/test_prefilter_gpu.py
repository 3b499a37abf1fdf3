"""The prefilter lists (pmh_set_prefilter) change the work, never the result.

With the lists forced onto every set large enough to profit at all, the
signatures, q values and statuses must be bit-identical to those of a handle
with the prefilter off, in both precisions, for all six variants, the
binary-weight variants and the rejection sampler; they must match the oracle;
and the work counters must show that the lists were used (elements visited are
counted the same either way).  Sets whose survivors overflow their list
(n/2 entries) fall back to the full filter, which the small sets here do.
"""
import numpy as np
import pytest
import torch

from paper_1911_00675_gb300 import workloads as W
from parity_util import VARS, check_sets, to_dev

pytestmark = pytest.mark.gpu

SIZES = [1, 7, 60, 500, 3000, 20000, 70000]


@pytest.fixture(scope="module")
def handles():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    on, off = pmh.Handle(0), pmh.Handle(0)
    on.set_prefilter(0.05)     # every set of more than a few hundred elements is listed (if its list fits)
    off.set_prefilter(0.0)
    return on, off


def _call(H, b, variants, prec, seed=5, offsets=None):
    from paper_1911_00675_gb300 import pmh
    ids, w, off = to_dev(b)
    if offsets is not None:
        off = offsets
    cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
    z, q, st = H.sketch_batch(ids, w, off, b.m, variants, prec, seed, with_q=True, counters=cnt)
    torch.cuda.synchronize()
    return pmh.to_u64(z), q.cpu().numpy(), st.cpu().numpy(), dict(zip(pmh.COUNTERS, cnt.cpu().tolist()))


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("m", [2, 64, 1024])
def test_lists_leave_results_unchanged(handles, precision, m):
    on, off = handles
    for weight in ("uniform", "pareto"):
        b = W.random_batch(300 + m, SIZES, m, weight)
        z1, q1, s1, c1 = _call(on, b, VARS, precision)
        z0, q0, s0, c0 = _call(off, b, VARS, precision)
        assert (s1 == 0).all() and np.array_equal(s1, s0)
        assert np.array_equal(z1, z0)
        assert np.array_equal(q1, q0)
        assert c1["listed"] > 0 and c0["listed"] == 0
        assert c1["list_hashed"] > 0 and c0["list_hashed"] == 0 and c0["list_skipped"] == 0
        assert c1["elements"] == c0["elements"]
        assert c1["items"] == c0["items"]
        # the elements the prefilter rejected for a variant are counted as visited and prefiltered
        assert c1["prefiltered"] >= c1["list_skipped"] > 0


def test_lists_match_oracle(handles):
    on, _ = handles
    b = W.random_batch(17, [900, 2500, 6000], 128, "lognormal")
    for prec in (0, 1):
        z, q, st, c = _call(on, b, VARS, prec, seed=3)
        assert (st == 0).all() and c["listed"] > 0
        for vi, v in enumerate(VARS):
            check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=3)


def test_lists_with_binary_weights_and_rejection_sampler(handles):
    from paper_1911_00675_gb300 import pmh
    on, off = handles
    b = W.random_batch(23, [40, 5000, 30000], 256, "pareto")
    variants = ["1", "3u", "3au", "4u", "4", "3a"]
    for sampler in (pmh.TE_REJECTION, pmh.TE_INVERSION):
        on.set_te_sampler(sampler)
        off.set_te_sampler(sampler)
        for prec in (0, 1):
            z1, q1, s1, _ = _call(on, b, variants, prec)
            z0, q0, s0, _ = _call(off, b, variants, prec)
            assert (s1 == 0).all() and np.array_equal(z1, z0) and np.array_equal(q1, q0)


def test_offsets_not_starting_at_zero(handles):
    """A batch whose offsets start inside the element arrays (list positions count from offsets[0])."""
    on, off = handles
    b = W.random_batch(31, [5, 3001, 20000, 9, 44000], 512, "uniform")
    ids, w, offs = to_dev(b)
    shift = 7
    pad_ids = torch.cat([torch.arange(shift, dtype=torch.int64, device="cuda"), ids])
    pad_w = torch.cat([torch.full((shift,), 0.5, dtype=torch.float64, device="cuda"), w])
    offs7 = offs + shift
    from paper_1911_00675_gb300 import pmh
    outs = []
    for H in (on, off):
        cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
        z, q, st = H.sketch_batch(pad_ids, pad_w, offs7, b.m, VARS, 1, 9, with_q=True, counters=cnt)
        torch.cuda.synchronize()
        outs.append((pmh.to_u64(z), q.cpu().numpy(), st.cpu().numpy(), int(cnt[pmh.COUNTERS.index("listed")])))
    assert outs[0][3] > 0
    assert (outs[0][2] == 0).all()
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    # and the same signatures as the unshifted batch
    z, q, _, _ = _call(off, b, VARS, 1, seed=9)
    assert np.array_equal(outs[0][0], z)


def test_arrays_rewritten_in_place(handles):
    """The element count is read once per (ids, weights, offsets) arrays; a later, larger batch
    written into the same tensors only loses the lists that no longer fit."""
    from paper_1911_00675_gb300 import pmh
    on, off = handles
    small = W.random_batch(41, [100, 12000, 300], 256, "uniform")
    big = W.random_batch(42, [30000, 60000, 200], 256, "uniform")
    ids_b, w_b, off_b = to_dev(big)
    ids_s, w_s, off_s = to_dev(small)
    ids = torch.zeros_like(ids_b)
    w = torch.zeros_like(w_b)
    offs = off_s.clone()
    ids[:ids_s.numel()] = ids_s
    w[:w_s.numel()] = w_s
    cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
    on.sketch_batch(ids, w, offs, 256, VARS, 1, 0, counters=cnt)
    torch.cuda.synchronize()
    assert int(cnt[pmh.COUNTERS.index("listed")]) > 0
    ids.copy_(ids_b)             # same tensors, same number of sets, ~7x the elements
    w.copy_(w_b)
    offs.copy_(off_b)
    z1, q1, s1 = on.sketch_batch(ids, w, offs, 256, VARS, 1, 0, with_q=True)
    z0, q0, s0 = off.sketch_batch(ids_b, w_b, off_b, 256, VARS, 1, 0, with_q=True)
    torch.cuda.synchronize()
    assert (s1 == 0).all()
    assert np.array_equal(pmh.to_u64(z1), pmh.to_u64(z0))
    assert torch.equal(q1, q0)


def test_decreasing_offsets_turn_lists_off(handles):
    """Offsets that decrease make sets' element ranges overlap, and with them their share of the
    lists: no set is listed then, and every valid set gets its own signature."""
    from paper_1911_00675_gb300 import pmh
    on, off = handles
    b = W.random_batch(61, [100_000], 256, "uniform")
    ids, w, _ = to_dev(b)
    offs = torch.tensor([0, 60_000, 20_000, 30_000, 100_000], dtype=torch.int64, device="cuda")
    cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
    z1, q1, s1 = on.sketch_batch(ids, w, offs, 256, VARS, 1, 3, with_q=True, counters=cnt)
    z0, q0, s0 = off.sketch_batch(ids, w, offs, 256, VARS, 1, 3, with_q=True)
    torch.cuda.synchronize()
    s1 = s1.cpu().numpy()
    assert (s1[:, 1] == 1).all() and (s1[:, [0, 2, 3]] == 0).all()   # set 1: PMH_ERR_INVALID_ARG
    assert np.array_equal(s1, s0.cpu().numpy())
    assert int(cnt[pmh.COUNTERS.index("listed")]) == 0
    assert np.array_equal(pmh.to_u64(z1), pmh.to_u64(z0))
    assert torch.equal(q1, q0)


def test_host_pipeline_with_lists(handles):
    from paper_1911_00675_gb300 import pmh
    on, off = handles
    b = W.random_batch(51, [20000, 3, 45000, 800, 30000, 12000], 1024, "uniform")
    ids = torch.from_numpy(b.ids.view(np.int64).copy())
    w = torch.from_numpy(b.weights.copy())
    offs = torch.from_numpy(b.offsets.copy())
    zh, _, sh = on.sketch_batch_host(ids, w, offs, b.m, VARS, 1, 2, chunks=3)
    z0, _, s0, _ = _call(off, b, VARS, 1, seed=2)
    assert (sh.numpy() == 0).all()
    assert np.array_equal(pmh.to_u64(zh), z0)
