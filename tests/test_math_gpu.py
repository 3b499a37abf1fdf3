"""The FP32 Exp(1) variate of the candidate path against FP64 -log1p(-U) (Sec. "ProbMinHash1":
exponential spacings by inversion).  The precision scheme relies on every FP32 point value being
within eta = 2^-18 of its FP64 value, with 6 ulp (2^-24) allotted to this variate; the measured
worst case must stay within that allotment."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
ULP = 2.0 ** -24


def _ref(words):
    k = (words >> np.uint64(11)).astype(np.float64)
    u = k * 2.0 ** -53
    return -np.log1p(-u)


def test_exp1_fp32_error_bound():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    rng = np.random.default_rng(0)
    w = rng.integers(0, 2**64, size=4_000_000, dtype=np.uint64)
    # edges: U = 0, the smallest U, around the 1 - sqrt(1/2) switch, U -> 1, powers of two
    k_edges = [0, 1, 2, 3, 2638147582215219 - 2, 2638147582215219 - 1, 2638147582215219, 2638147582215220,
               2**52 - 1, 2**52, 2**52 + 1, 2**53 - 3, 2**53 - 2, 2**53 - 1]
    k_edges += [2**j for j in range(53)] + [2**53 - 2**j for j in range(1, 53)]
    k_edges += list(rng.integers(2638147582215219 - 10**6, 2638147582215219 + 10**6, size=1000))
    edges = (np.array(k_edges, dtype=np.uint64) << np.uint64(11)) | np.uint64(0x5A5)
    w = np.concatenate([w, edges])
    got = pmh.check_exp1(torch.from_numpy(w.view(np.int64)).cuda()).cpu().numpy().astype(np.float64)
    ref = _ref(w)
    zero = ref == 0
    assert np.all(got[zero] == 0)
    rel = np.abs(got[~zero] - ref[~zero]) / ref[~zero]
    assert rel.max() <= 6 * ULP, rel.max() / ULP
    # and it is a real approximation of the inversion, not a looser one
    assert np.mean(rel) < 1.5 * ULP


@pytest.mark.parametrize("lam_from", ["m=2", "m=3", "m=4", "m=64", "m=1024", "m=4096", "pmh4 i=m-2", "pmh4 i=m-3"])
def test_texp_fp32_error_bound(lam_from):
    # TE_lambda = -log1p(U expm1(-lambda)) / lambda with the FP32 constants the kernels hold; the
    # precision scheme allots 12 ulp to this variate against the canonical FP64 value
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    if lam_from.startswith("m="):
        m = int(lam_from[2:])
        lam = np.log1p(1.0 / (m - 1))
    else:
        j = int(lam_from.split("-")[-1])      # lambda_i = log1p(1/(m-i)) with m - i = j
        lam = np.log1p(1.0 / j)
    c64, inv64 = np.expm1(-lam), 1.0 / lam
    rng = np.random.default_rng(int(lam * 1e6))
    w = rng.integers(0, 2**64, size=2_000_000, dtype=np.uint64)
    k_edges = [0, 1, 2**52, 2**53 - 1] + [2**j for j in range(53)] + [2**53 - 2**j for j in range(1, 53)]
    w = np.concatenate([w, (np.array(k_edges, dtype=np.uint64) << np.uint64(11))])
    got = pmh.check_texp(torch.from_numpy(w.view(np.int64)).cuda(), np.float32(c64), np.float32(inv64))
    got = got.cpu().numpy().astype(np.float64)
    u = (w >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    ref = -np.log1p(u * c64) * inv64
    zero = ref == 0
    assert np.all(got[zero] == 0)
    rel = np.abs(got[~zero] - ref[~zero]) / ref[~zero]
    assert rel.max() <= 12 * ULP, rel.max() / ULP
