"""ProbMinHash3/3a/4 with the paper's rejection sampler for Exp(lambda;0,1) (Sec. Truncated
Exponential Sampling) on the GPU, against the oracle run with the same sampler.

Same rules as the other parity tests: winning ids bit-exact except the oracle's near ties
(< 1e-12 relative), q within 1e-10 relative, and the FP32-candidate path identical to the
FP64 path.  The loop's draws are exact in FP64 on both sides, so the samplers agree.
"""
import numpy as np
import pytest

from paper_1911_00675_gb300 import workloads as W
from parity_util import VARS, check_sets, run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    h = pmh.Handle(0)
    h.set_te_sampler(pmh.TE_REJECTION)
    yield h
    h.set_te_sampler(pmh.TE_INVERSION)
    h.close()


SIZES = [0, 1, 2, 3, 5, 33, 64, 257, 1000, 3001]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
@pytest.mark.parametrize("m", [2, 3, 7, 64, 300, 1024])
def test_rejection_sampler_matches_oracle(H, precision, m):
    for weight in ("uniform", "pareto", "lognormal"):
        b = W.random_batch(2000 + m, SIZES, m, weight)
        z, q, st = run(H, b, VARS + ["3u", "4u"], precision, with_q=True, seed=5)
        assert (st == 0).all(), st
        for vi, v in enumerate(VARS + ["3u", "4u"]):
            # the sampler only concerns the weighted correlated variants; the oracle ignores it elsewhere
            check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=5, te_rejection=True)


@pytest.mark.parametrize("m", [2, 33, 4096])
def test_rejection_sampler_fp32_equals_fp64(H, m):
    b = W.random_batch(3000 + m, [1, 4, 17, 200, 1500, 9000], m, "pareto")
    z64, q64, _ = run(H, b, ["3", "3a", "4"], 0, with_q=True, seed=12)
    z32, q32, _ = run(H, b, ["3", "3a", "4"], 1, with_q=True, seed=12)
    assert np.array_equal(z64, z32) and np.array_equal(q64, q32)


def test_sampler_changes_only_the_truncated_exponential_variants(H):
    # the samplers draw different variates from the same words: the minima (q) of ProbMinHash3/4
    # change (the winners often do not: both variates increase with U, and for small lambda nearly
    # proportionally), while the other variants do not use Exp(lambda;0,1) at all
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(3100, [50, 700, 4000], 256, "lognormal")
    vs = ["1", "2", "3", "4", "3u", "4u"]
    z_rej, q_rej, _ = run(H, b, vs, 1, with_q=True, seed=2)
    H.set_te_sampler(pmh.TE_INVERSION)
    try:
        z_inv, q_inv, _ = run(H, b, vs, 1, with_q=True, seed=2)
    finally:
        H.set_te_sampler(pmh.TE_REJECTION)
    for vi, v in enumerate(vs):
        same = np.array_equal(q_rej[vi], q_inv[vi]) and np.array_equal(z_rej[vi], z_inv[vi])
        assert same == (v not in ("3", "4")), v


def test_rejection_sampler_grid_mode_and_largest_m(H):
    # one set above the grid-mode size, and m = 8192 (the largest tables)
    H.set_thresholds()
    b = W.random_batch(3200, [(1 << 20) + 77], 1024, "lognormal")
    z, q, st = run(H, b, ["3a", "4"], 1, with_q=False, seed=3)
    assert (st == 0).all()
    for vi, v in enumerate(["3a", "4"]):
        check_sets(b, v, z[vi], None, [0], seed=3, te_rejection=True)
    b = W.random_batch(3300, [3, 500, 20000], 8192, "pareto")
    z, q, st = run(H, b, ["3", "4"], 1, with_q=True, seed=4)
    assert (st == 0).all()
    for vi, v in enumerate(["3", "4"]):
        check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=4, te_rejection=True)
