"""Shared helpers of the GPU parity tests: device upload, one sketch call
through the C ABI, and the comparison with the CPU oracle.

Rule (winning ids): bit-exact with the oracle, except components where the
oracle's two best candidates differ by less than 1e-12 relative (near ties,
counted; at most 1e-6 of all components).  CUDA's and the host's FP64 log1p
may differ in the last ulp, which is what the exemption covers.

Rule (q values): |q_gpu - q_oracle| <= 1e-10 * q_oracle.  A point value is a
sum of at most i <= ~1e5 terms, each within 2 ulp (two log1p evaluations of at
most 1 ulp error each) plus one rounding, so the two FP64 evaluations differ
by at most ~4i * 2^-53 ~ 5e-11 relative.
"""
import numpy as np
import torch

import oracle

VARS = ["1", "1a", "2", "3", "3a", "4"]
NEAR_REL = 1e-12
NEAR_MAX_FRACTION = 1e-6
Q_RTOL = 1e-10
# (label, near ties, components scanned) of the tests that scanned every sampled set; printed at
# the end of the run by the terminal summary in conftest.py
NEAR_TIE_LOG = []


def to_dev(batch):
    dev = torch.device("cuda", 0)
    ids = torch.from_numpy(batch.ids.view(np.int64).copy()).to(dev)
    w = torch.from_numpy(np.ascontiguousarray(batch.weights)).to(dev)
    off = torch.from_numpy(np.ascontiguousarray(batch.offsets)).to(dev)
    return ids, w, off


def run(H, batch, variants, precision, with_q=True, seed=0, counters=None):
    from paper_1911_00675_gb300 import pmh
    ids, w, off = to_dev(batch)
    z, q, st = H.sketch_batch(ids, w, off, batch.m, variants, precision, seed, with_q=with_q, counters=counters)
    torch.cuda.synchronize()
    return (pmh.to_u64(z), q.cpu().numpy() if q is not None else None, st.cpu().numpy())


def check_sets(batch, variant, z, q, sets, seed=0, stats=None, scan=False, te_rejection=False):
    """Compares GPU rows z[s], q[s] with the oracle for the listed sets.

    stats (optional dict): "near" counts the oracle's near ties, "components" the components
    compared, "mismatch" the exempted id mismatches.  Without `scan` near ties are counted only
    in sets with a mismatch; with `scan` every set is scanned, so "near" / "components" is the
    near-tie rate of the sample.  te_rejection: the GPU drew Exp(lambda;0,1) with the rejection
    sampler, and so does the oracle."""
    m = batch.m
    for s in sets:
        ids, w = batch.set(s)
        qo, zo, _ = oracle.sketch(variant, ids, w, m, seed=seed, te_rejection=te_rejection)
        diff = np.nonzero(z[s] != zo)[0]
        if len(diff) or (scan and stats is not None):
            flags, _ = oracle.near_ties(variant, ids, w, m, seed, qo, zo, NEAR_REL, te_rejection=te_rejection)
            assert flags[diff].all(), f"set {s} variant {variant}: {len(diff)} unflagged id mismatches, e.g. k={diff[:5]}"
            if stats is not None:
                stats["near"] += int(flags.sum())
                stats["mismatch"] = stats.get("mismatch", 0) + len(diff)
        if stats is not None:
            stats["components"] += m
        if q is not None:
            fin = np.isfinite(qo)
            assert np.array_equal(np.isfinite(q[s]), fin)
            np.testing.assert_allclose(q[s][fin], qo[fin], rtol=Q_RTOL, atol=0)




def assert_near_tie_rate(stats, label=None):
    """The exemption's limit: near ties at most 1e-6 of the components compared."""
    if label is not None:
        NEAR_TIE_LOG.append((label, stats["near"], stats["components"], stats.get("mismatch", 0)))
    assert stats["near"] <= NEAR_MAX_FRACTION * stats["components"], stats
