"""Algorithm P-MinHash on the GPU against the oracle (the method the paper compares ProbMinHash with).

Rules as for the ProbMinHash kernels: winning ids bit-exact except where the oracle's two best
candidates of a component differ by less than 1e-12 relative (CUDA's and the host's FP64 log1p may
differ in the last ulp; the runner-up comes from the one-element signatures), q within 1e-10.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1911_00675_gb300 import workloads as W
from parity_util import NEAR_REL, Q_RTOL, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    h = pmh.Handle(0)
    yield h
    h.close()


def _runner_up(ids, w, m, seed):
    h = np.array([oracle.pminhash(ids[j:j + 1], w[j:j + 1], m, seed=seed)[0] for j in range(len(ids))])
    return np.sort(h, axis=0)[1] if len(ids) > 1 else np.full(m, np.inf)


def _check(b, z, q, seed, scan_limit=400):
    m = b.m
    for s in range(b.num_sets):
        ids, w = b.set(s)
        qo, zo = oracle.pminhash(ids, w, m, seed=seed)
        diff = np.nonzero(z[s] != zo)[0]
        if len(diff):
            assert len(ids) <= scan_limit, f"set {s}: {len(diff)} id mismatches"
            ru = _runner_up(ids, w, m, seed)
            assert (ru[diff] - qo[diff] < NEAR_REL * qo[diff]).all(), f"set {s}: unflagged mismatches {diff[:5]}"
        fin = np.isfinite(qo)
        assert np.array_equal(np.isfinite(q[s]), fin)
        np.testing.assert_allclose(q[s][fin], qo[fin], rtol=Q_RTOL, atol=0)


@pytest.mark.parametrize("m", [1, 2, 7, 64, 300, 1024])
def test_pminhash_matches_oracle(H, m):
    from paper_1911_00675_gb300 import pmh
    for weight in ("uniform", "pareto", "lognormal", "unit"):
        b = W.random_batch(4000 + m, [0, 1, 2, 5, 33, 257, 1000, 2500], m, weight)
        ids, w, off = to_dev(b)
        z, q, st = H.pminhash_batch(ids, w, off, m, seed=6, with_q=True)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        _check(b, pmh.to_u64(z), q.cpu().numpy(), 6)


def test_pminhash_large_m_and_large_set(H):
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(4100, [3, 90, 40000], 8192, "pareto")
    ids, w, off = to_dev(b)
    z, q, st = H.pminhash_batch(ids, w, off, 8192, seed=2, with_q=True)
    torch.cuda.synchronize()
    assert (st.cpu().numpy() == 0).all()
    _check(b, pmh.to_u64(z), q.cpu().numpy(), 2, scan_limit=100)


def test_pminhash_extreme_weight_ratios_and_bad_weights(H):
    # weights 2^-150 apart from the heaviest are below the FP32 range after scaling and are
    # compared in FP64 only; a negative weight fails its set
    from paper_1911_00675_gb300 import pmh
    ids = W.distinct_ids(10, 6, 3)
    w = np.array([1.0, 2.0 ** -150, 3.0 ** -200, 0.5, 0.0, 7.0])
    for sets, weights in (([0, 6], w), ([0, 3], np.array([2.0 ** -150, 2.0 ** -160, 2.0 ** -149]))):
        bb = W.Batch(ids[:sets[1]], weights, np.array(sets, dtype=np.int64), 16)
        d_ids, d_w, d_off = to_dev(bb)
        z, q, st = H.pminhash_batch(d_ids, d_w, d_off, 16, seed=1, with_q=True)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == 0).all()
        _check(bb, pmh.to_u64(z), q.cpu().numpy(), 1)
    wb = w.copy()
    wb[3] = -1.0
    bb = W.Batch(ids, wb, np.array([0, 2, 6], dtype=np.int64), 16)
    d_ids, d_w, d_off = to_dev(bb)
    z, q, st = H.pminhash_batch(d_ids, d_w, d_off, 16, seed=1, with_q=True)
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [pmh.OK, pmh.ERR_BAD_WEIGHT]
    assert (z[1] == 0).all() and torch.isinf(q[1]).all()
