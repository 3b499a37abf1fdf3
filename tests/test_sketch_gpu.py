"""Parity of the CUDA sketch path (through the C ABI) with the CPU oracle.

Rule (winning ids): bit-exact with the oracle, except components where the
oracle's two best candidates differ by less than 1e-12 relative (near ties,
counted; at most 1e-6 of all components).  CUDA's and the host's FP64 log1p
may differ in the last ulp, which is what the exemption covers.

Rule (q values): |q_gpu - q_oracle| <= 1e-10 * q_oracle.  A point value is a
sum of at most i <= ~1e5 terms, each within 2 ulp (two log1p evaluations of at
most 1 ulp error each) plus one rounding, so the two FP64 evaluations differ
by at most ~4i * 2^-53 ~ 5e-11 relative.

Rule (precisions): the FP32-candidate path and the FP64 path return identical
ids and identical q.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1911_00675_gb300 import workloads as W
from parity_util import NEAR_REL, Q_RTOL, VARS, assert_near_tie_rate, check_sets, run, to_dev  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    return pmh.Handle(0)


SIZES = [0, 1, 2, 3, 5, 31, 32, 33, 64, 100, 257, 1000, 3001]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("m", [2, 7, 64, 300, 1024])
def test_small_batches_all_variants(H, precision, m):
    for weight in ("uniform", "pareto", "lognormal", "unit"):
        b = W.random_batch(1000 + m, SIZES, m, weight)
        z, q, st = run(H, b, VARS, precision, with_q=True, seed=3)
        assert (st == 0).all(), st
        for vi, v in enumerate(VARS):
            check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=3)


@pytest.mark.parametrize("m", [2, 33, 256, 4096])
def test_fp32_equals_fp64_bit_exact(H, m):
    b = W.random_batch(77 + m, [1, 4, 17, 200, 1500, 9000], m, "pareto")
    z64, q64, _ = run(H, b, VARS, 0, with_q=True, seed=11)
    z32, q32, _ = run(H, b, VARS, 1, with_q=True, seed=11)
    assert np.array_equal(z64, z32)
    assert np.array_equal(q64, q32)


def test_m_one_and_single_element_sets(H):
    b = W.random_batch(5, [1, 1, 2, 50], 1, "uniform")
    for prec in (0, 1):
        z, q, st = run(H, b, ["1", "1a", "2"], prec, seed=9)
        assert (st == 0).all()
        for vi, v in enumerate(["1", "1a", "2"]):
            check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=9)
    b = W.random_batch(6, [1, 1, 1], 4096, "lognormal")
    for prec in (0, 1):
        z, q, st = run(H, b, VARS, prec)
        for vi in range(6):
            for s in range(3):
                assert (z[vi, s] == b.ids[s]).all()


def test_zero_bad_and_empty_sets(H):
    ids = W.distinct_ids(0, 9, 1)
    w = np.array([0.0, 1.0, -0.0,          # set 0: one positive weight
                  0.0, 0.0,                # set 1: all zero -> empty
                  1.0, -1.0,               # set 2: negative -> bad weight
                  np.nan,                  # set 3: NaN -> bad
                  np.inf])                 # set 4: inf -> bad
    off = np.array([0, 3, 5, 7, 8, 9, 9], dtype=np.int64)   # set 5 empty
    b = W.Batch(ids, w, off, 16)
    for prec in (0, 1):
        z, q, st = run(H, b, ["1", "4"], prec)
        assert st.tolist() == [[0, 0, 2, 2, 2, 0]] * 2
        for vi in range(2):
            assert (z[vi, 0] == ids[1]).all()
            for s in (1, 2, 3, 4, 5):
                assert (z[vi, s] == 0).all() and np.isinf(q[vi, s]).all()


def test_decreasing_offsets_flagged(H):
    ids = W.distinct_ids(0, 10, 2)
    b = W.Batch(ids, np.ones(10), np.array([0, 6, 4, 10], dtype=np.int64), 8)
    _, _, st = run(H, b, ["1"], 1)
    assert st[0].tolist() == [0, 1, 0]


def test_seed_changes_signature(H):
    b = W.random_batch(8, [500], 64)
    z0, _, _ = run(H, b, ["3a"], 1, seed=0)
    z1, _, _ = run(H, b, ["3a"], 1, seed=1)
    assert (z0 != z1).any()
    check_sets(b, "3a", z1[0], None, [0], seed=1)


def test_counters_and_repeat_calls(H):
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(12, [100, 2000, 5], 256, "uniform")
    ids, w, off = to_dev(b)
    cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
    outs = []
    for _ in range(3):   # the second and third calls replay the cached graph
        z, _, st = H.sketch_batch(ids, w, off, 256, VARS, 1, 0, counters=cnt)
        torch.cuda.synchronize()
        outs.append(pmh.to_u64(z).copy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    c = dict(zip(pmh.COUNTERS, cnt.cpu().tolist()))
    assert c["elements"] >= 3 * 6 * 2105      # every positive element is visited at least once per call
    assert c["points32"] > 0
    assert c["items"] == 3 * 6 * b.num_sets   # each call counts its own items once


def test_counters_exclude_autotuning_trials(H):
    # the first call of a new batch shape runs every team shape twice before its own launch; the
    # counters report the call's work only, so it equals that of the next (tuned) call
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(13, [300, 40, 7000, 9], 128, "pareto")
    ids, w, off = to_dev(b)
    H.set_autotune(-1)
    try:
        got = []
        for _ in range(2):
            cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
            H.sketch_batch(ids, w, off, 128, ["1", "2", "3", "4"], 1, 0, counters=cnt)
            torch.cuda.synchronize()
            got.append(dict(zip(pmh.COUNTERS, cnt.cpu().tolist())))
        assert got[0]["items"] == got[1]["items"] == 4 * b.num_sets
        assert got[0]["elements"] == got[1]["elements"]
    finally:
        H.set_autotune(1)


# --------------------------------------------------------------- full sizes
def test_c1_full(H):
    b = W.batch_c1()
    for prec in (0, 1):
        z, q, st = run(H, b, ["1", "3"], prec, with_q=(prec == 0))
        assert (st == 0).all()
        for vi, v in enumerate(["1", "3"]):
            check_sets(b, v, z[vi], q[vi] if q is not None else None, range(b.num_sets))


def _sampled_parity(H, b, variants, n_sample, seed=0, label=None):
    z64, _, st64 = run(H, b, variants, 0, with_q=False)
    z32, _, st32 = run(H, b, variants, 1, with_q=False)
    assert (st64 == 0).all() and (st32 == 0).all()
    assert np.array_equal(z64, z32)              # identical output, every set, every variant
    rng = np.random.default_rng(seed)
    sizes = np.diff(b.offsets)
    # sample small and large sets alike (stratified by log size)
    order = np.argsort(sizes)
    pick = np.unique(np.concatenate([order[np.linspace(0, len(order) - 1, n_sample).astype(int)],
                                     rng.choice(len(order), n_sample // 2, replace=False)]))
    stats = {"near": 0, "components": 0}
    for vi, v in enumerate(variants):
        check_sets(b, v, z32[vi], None, pick, stats=stats, scan=True)
    assert_near_tie_rate(stats, label)


@pytest.mark.slow
def test_c2_full_sampled(H):
    _sampled_parity(H, W.batch_c2(), VARS, 24, label="c2 (20,000 sets, m=1024, six variants; sampled sets)")


@pytest.mark.slow
def test_c3_full_sampled(H):
    _sampled_parity(H, W.batch_c3(), ["2", "4"], 10, label="c3 (10,000 x 10,000, Pareto(1.5), m=4096; sampled sets)")


@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5], ids=["warp", "cta8", "quad", "pair", "quad8", "quad8l"])
def test_every_team_shape_matches_oracle(H, shape):
    # how warps share an item changes nothing in the result (Eq. signature_def is per item)
    b = W.random_batch(500 + shape, [0, 1, 2, 33, 64, 65, 130, 700, 2500], 256, "lognormal")
    H.set_team_shape(0, shape)
    try:
        for precision in (0, 1):
            z, q, st = run(H, b, VARS, precision, with_q=True, seed=6)
            assert (st == 0).all()
            assert H.last_team_shapes() == [shape] * 4
            for vi, v in enumerate(VARS):
                check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=6)
    finally:
        H.set_team_shape(0, -1)


def test_autotune_picks_a_shape_and_keeps_results(H):
    b = W.random_batch(510, [5, 50, 500, 5000], 128, "uniform")
    H.set_autotune(-1)
    z1, q1, _ = run(H, b, ["1", "2", "3a", "4"], 1, seed=1)      # tunes: one run per shape, then the call
    shapes = H.last_team_shapes()
    assert all(0 <= s <= 5 for s in shapes)
    z2, q2, _ = run(H, b, ["1", "2", "3a", "4"], 1, seed=1)      # cached choice
    assert H.last_team_shapes() == shapes
    assert np.array_equal(z1, z2) and np.array_equal(q1, q2)
    H.set_autotune(0)
    z3, q3, _ = run(H, b, ["1", "2", "3a", "4"], 1, seed=1)      # default rule
    assert np.array_equal(z1, z3) and np.array_equal(q1, q3)
    H.set_autotune(1)


@pytest.mark.parametrize("shape", [0, 3, 4], ids=["warp", "pair", "quad8"])
def test_carried_lanes_heavy_tailed_weights(H, shape):
    # Large sets with Pareto weights: most survivors end after a point or two while a few heavy
    # elements run long, so ProbMinHash1/2 warps hand busy lanes over to the next survivor batch
    # (and ProbMinHash2 defers its deep queue until no lane holds a write list).  Nothing of that
    # may change a signature.
    b = W.random_batch(920 + shape, [20000, 3, 45000, 700, 12000], 512, "pareto")
    H.set_team_shape(0, shape)
    try:
        for precision in (0, 1):
            z, q, st = run(H, b, ["1", "2", "1a"], precision, with_q=True, seed=17)
            assert (st == 0).all()
            for vi, v in enumerate(["1", "2", "1a"]):
                check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=17)
    finally:
        H.set_team_shape(0, -1)


@pytest.mark.parametrize("autotune", [1, 0], ids=["tuned", "default-rule"])
def test_largest_m(H, autotune):
    # m = PMH_MAX_M = 8192: one FP64 signature is 128 KiB of shared memory, so only the shapes
    # with one team per block fit; every variant must still run and match the oracle
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(8192, [1, 40, 900, 3000], 8192, "lognormal")
    H.set_autotune(autotune)
    try:
        z64, q64, st64 = run(H, b, VARS, 0, with_q=True, seed=21)
        z32, q32, st32 = run(H, b, VARS, 1, with_q=True, seed=21)
    finally:
        H.set_autotune(1)
    assert (st64 == 0).all() and (st32 == 0).all()
    assert np.array_equal(z64, z32) and np.array_equal(q64, q32)
    for vi, v in enumerate(VARS):
        check_sets(b, v, z64[vi], q64[vi], range(b.num_sets), seed=21)


def test_inputs_off_the_16_byte_grid(H):
    # ids and weights one element into a larger allocation: 8-byte but not 16-byte aligned (the
    # statistics read weights two at a time on the 16-byte grid and must handle both edges)
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(4242, [1, 2, 3, 600, 70001, 0, 5], 128, "exp")
    ids, w, off = to_dev(b)
    ids_u = torch.empty(ids.numel() + 1, dtype=ids.dtype, device=ids.device)[1:]
    w_u = torch.empty(w.numel() + 1, dtype=w.dtype, device=w.device)[1:]
    ids_u.copy_(ids)
    w_u.copy_(w)
    assert w_u.data_ptr() % 16 == 8
    for prec in (0, 1):
        za, qa, sa = H.sketch_batch(ids, w, off, b.m, VARS, prec, 4, with_q=True)
        zb, qb, sb = H.sketch_batch(ids_u, w_u, off, b.m, VARS, prec, 4, with_q=True)
        torch.cuda.synchronize()
        assert torch.equal(za, zb) and torch.equal(qa, qb) and torch.equal(sa, sb)
        assert int(sa.abs().sum()) == 0
    z, q, st = run(H, b, VARS, 1, with_q=True, seed=4)
    for vi, v in enumerate(VARS):
        check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=4)
