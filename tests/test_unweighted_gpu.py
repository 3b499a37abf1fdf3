"""Binary-weight specialisations (Sec. Conventional Jaccard Similarity: uniform variates, gamma_i
= i, every positive weight counts 1) on the GPU against the oracle, under the batch parity rules:
winning ids bit-exact except oracle near ties, q within 1e-10, FP32 candidates == FP64."""
import numpy as np
import pytest

from paper_1911_00675_gb300 import workloads as W
from parity_util import check_sets, run

pytestmark = pytest.mark.gpu
UVARS = ["3u", "3au", "4u"]
SIZES = [0, 1, 2, 3, 5, 31, 32, 33, 64, 100, 257, 1000, 3001]


@pytest.fixture(scope="module")
def H():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    return pmh.Handle(0)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("m", [1, 2, 7, 64, 1024])
def test_unweighted_small_batches(H, precision, m):
    for weight in ("unit", "pareto"):        # pareto: the weight values must not matter
        b = W.random_batch(700 + m, SIZES, m, weight)
        z, q, st = run(H, b, UVARS, precision, with_q=True, seed=4)
        assert (st == 0).all(), st
        for vi, v in enumerate(UVARS):
            check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=4)


@pytest.mark.parametrize("m", [2, 256, 4096])
def test_unweighted_fp32_equals_fp64_and_mixes_with_weighted(H, m):
    b = W.random_batch(720 + m, [1, 4, 17, 200, 1500, 9000], m, "unit")
    vs = ["3", "3u", "4", "4u", "1", "3au"]
    z64, q64, _ = run(H, b, vs, 0, with_q=True, seed=13)
    z32, q32, _ = run(H, b, vs, 1, with_q=True, seed=13)
    assert np.array_equal(z64, z32) and np.array_equal(q64, q32)
    assert np.array_equal(z32[1], z32[5])            # 3u == 3au
    for vi, v in enumerate(vs):
        check_sets(b, v, z32[vi], q32[vi], range(b.num_sets), seed=13)


def test_unweighted_grid_mode(H):
    H.set_thresholds(grid_min=30_000)
    try:
        b = W.random_batch(740, [40_000, 7], 512, "lognormal")
        z, q, st = run(H, b, ["3au", "4u"], 1, with_q=True, seed=6)
        assert (st == 0).all()
        for vi, v in enumerate(["3au", "4u"]):
            check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=6)
    finally:
        H.set_thresholds()


def test_all_nine_variants_and_repeats_in_one_call(H):
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(750, [3, 90, 1200], 128, "unit")
    allv = ["1", "1a", "2", "3", "3a", "4", "3u", "3au", "4u"]
    vs = allv + ["4u", "1", "3", "2", "3au", "4", "1a"]          # 16: the most one call takes
    z, q, st = run(H, b, vs, 1, with_q=True, seed=21)
    assert (st == 0).all()
    for vi, v in enumerate(vs):
        zi, qi, _ = run(H, b, [v], 1, with_q=True, seed=21)
        assert np.array_equal(z[vi], zi[0]) and np.array_equal(q[vi], qi[0]), v
    with pytest.raises(pmh.PmhError) as ei:
        run(H, b, vs + ["1"], 1)
    assert ei.value.code == pmh.ERR_INVALID_ARG
