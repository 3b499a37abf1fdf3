"""b-bit signatures (Algorithm "Reduction to a b-bit signature") on the GPU against the oracle:
packed codes and all-pairs equal-field counts are integers, so bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_1911_00675_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    return pmh.Handle(0)


def _unpack(packed, m, b):
    p = packed.cpu().numpy().view(np.uint64)
    n, words = p.shape
    per = 64 // b
    mask = np.uint64((1 << b) - 1) if b < 64 else np.uint64(2**64 - 1)
    out = np.zeros((n, m), dtype=np.uint64)
    for k in range(m):
        w, j = divmod(k, per)
        out[:, k] = (p[:, w] >> np.uint64(j * b)) & mask
    if m % per:
        assert np.all(p[:, -1] >> np.uint64((m % per) * b) == 0)    # unused high bits are zero
    return out


def _family_sigs(H, m):
    # signatures of perturbed families of sets, so that counts span 0..m
    b = W.batch_c4_sets(seed=41 + m, num_base=5, n=400, variants_per_base=27, m=m)   # 135 rows: ragged tiles
    dev = torch.device("cuda", 0)
    z, _, st = H.sketch_batch(torch.from_numpy(b.ids.view(np.int64).copy()).to(dev),
                              torch.from_numpy(b.weights.copy()).to(dev), torch.from_numpy(b.offsets.copy()).to(dev),
                              m, ["3a"], 1, 0)
    torch.cuda.synchronize()
    assert int(st.abs().max()) == 0
    return z[0].contiguous()


@pytest.mark.parametrize("b", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("m", [64, 100, 1000])
def test_bbit_codes_and_counts_match_oracle(H, b, m):
    from paper_1911_00675_gb300 import pmh
    z = _family_sigs(H, m)
    packed = H.bbit_reduce(z, b, seed=7)
    counts = H.bbit_allpairs(packed, m, b)
    torch.cuda.synchronize()
    ref_codes = oracle.bbit_reduce(pmh.to_u64(z), b, seed=7)
    assert np.array_equal(_unpack(packed, m, b), ref_codes)
    ref_counts = oracle.count_allpairs(ref_codes).astype(np.uint16)
    assert np.array_equal(counts.cpu().numpy().view(np.uint16), ref_counts)
    if b == 64:   # b = 64 keeps equality exactly
        assert np.array_equal(ref_counts, oracle.count_allpairs(pmh.to_u64(z)).astype(np.uint16))


def test_bbit_upper_only_and_estimates(H):
    from paper_1911_00675_gb300 import pmh
    m, b = 512, 8
    z = _family_sigs(H, m)
    n = z.shape[0]
    packed = H.bbit_reduce(z, b, seed=1)
    counts = torch.full((n, n), -1, dtype=torch.int16, device="cuda")
    H.bbit_allpairs(packed, m, b, upper_only=True, counts=counts)
    full = oracle.count_allpairs(pmh.to_u64(z))                  # exact equal-component counts
    got = counts.cpu().numpy().view(np.uint16)
    iu = np.triu_indices(n)
    assert (got[np.tril_indices(n, -1)] == 0xFFFF).all()
    est = np.array([oracle.bbit_estimate(int(c), m, b) for c in got[iu]])
    jhat = full[iu] / m
    # the corrected b-bit estimate tracks the full-signature estimate within its collision noise
    p = 2.0 ** -b
    sd = np.sqrt(np.maximum(1 - jhat, 1e-9) * p * (1 - p) / m) / (1 - p)
    assert np.all(np.abs(est - jhat) <= 6 * sd + 1e-9)
