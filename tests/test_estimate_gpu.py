"""Equal-component counting (Eq. jaccard_estimator) and signature merging on the GPU,
through the C ABI, against the CPU oracle.  Counts are integers: bit-exact."""
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


def _dev(b):
    dev = torch.device("cuda", 0)
    return (torch.from_numpy(b.ids.view(np.int64).copy()).to(dev), torch.from_numpy(b.weights.copy()).to(dev),
            torch.from_numpy(b.offsets.copy()).to(dev))


def _sigs(H, b, variant="3a", prec=1, seed=0, with_q=False):
    ids, w, off = _dev(b)
    z, q, st = H.sketch_batch(ids, w, off, b.m, [variant], prec, seed, with_q=with_q)
    torch.cuda.synchronize()
    assert int(st.abs().sum()) == 0
    return z[0].contiguous(), (q[0].contiguous() if q is not None else None)


@pytest.mark.parametrize("m", [1, 7, 64, 1000])
def test_allpairs_counts_bit_exact(H, m):
    from paper_1911_00675_gb300 import pmh
    # perturbed families, so that counts span 0..m (like the c4 workload, scaled down)
    b = W.batch_c4_sets(seed=11 + m, num_base=6, n=300, variants_per_base=23, m=m)
    z, _ = _sigs(H, b, "1" if m == 1 else "3a")
    cnt = H.estimate_allpairs(z)
    torch.cuda.synchronize()
    ref = oracle.count_allpairs(pmh.to_u64(z))
    got = cnt.cpu().numpy().view(np.uint16)
    assert np.array_equal(got, ref.astype(np.uint16))
    assert ref.max() == m and (ref < m).any()


def test_allpairs_upper_only_leaves_lower_triangle(H):
    from paper_1911_00675_gb300 import pmh
    b = W.batch_c4_sets(seed=5, num_base=4, n=200, variants_per_base=33, m=128)   # 132 rows: a ragged tile
    z, _ = _sigs(H, b)
    n = z.shape[0]
    counts = torch.full((n, n), -1, dtype=torch.int16, device="cuda")
    H.estimate_allpairs(z, upper_only=True, counts=counts)
    torch.cuda.synchronize()
    got = counts.cpu().numpy().view(np.uint16)
    ref = oracle.count_allpairs(pmh.to_u64(z)).astype(np.uint16)
    iu = np.triu_indices(n)
    il = np.tril_indices(n, -1)
    assert np.array_equal(got[iu], ref[iu])
    assert (got[il] == 0xFFFF).all()


def test_pairs_counts(H):
    from paper_1911_00675_gb300 import pmh
    b = W.batch_c4_sets(seed=9, num_base=3, n=400, variants_per_base=20, m=256)
    z, _ = _sigs(H, b, "2")
    rng = np.random.default_rng(0)
    pa = rng.integers(0, z.shape[0], 5000)
    pb = rng.integers(0, z.shape[0], 5000)
    cnt = H.estimate_pairs(z, z, torch.from_numpy(pa).cuda(), torch.from_numpy(pb).cuda())
    torch.cuda.synchronize()
    zn = pmh.to_u64(z)
    ref = (zn[pa] == zn[pb]).sum(1)
    assert np.array_equal(cnt.cpu().numpy(), ref)


@pytest.mark.parametrize("variant", ["1", "2", "3a", "4"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_merge_of_parts_equals_sketch_of_union(H, variant, prec):
    # Eq. signature_def: the minimum over a union of disjoint parts is the minimum of the parts' minima.
    from paper_1911_00675_gb300 import pmh
    rng = np.random.default_rng(3)
    m = 512
    whole = W.random_batch(21, [4000], m, "lognormal")
    cuts = np.sort(rng.choice(np.arange(1, 4000), 4, replace=False))
    bounds = np.concatenate([[0], cuts, [4000]])
    parts = W.Batch(whole.ids, whole.weights, bounds.astype(np.int64), m)   # five disjoint parts as sets
    zw, qw = _sigs(H, whole, variant, prec, seed=4, with_q=True)
    zp, qp = _sigs(H, parts, variant, prec, seed=4, with_q=True)
    qm, zm = H.merge(qp, zp)
    torch.cuda.synchronize()
    assert torch.equal(zm, zw[0]) and torch.equal(qm, qw[0])


def test_c1_constructed_pairs_estimate_jp(H):
    # c1's 100 constructed pairs with known J_P: the estimate count/m has variance J(1-J)/m for
    # ProbMinHash1 (Eq. jaccard_variance) and less for ProbMinHash3 (Sec. Verification).
    from paper_1911_00675_gb300 import pmh
    rng = np.random.default_rng(0xC0FFEE01)
    m = 256
    ids_l, w_l, sizes, jps = [], [], [], []
    for j in range(100):
        a, wa, b_, wb, p = W.constructed_pair(rng, j / 99.0, n_total=1000)
        jps.append(p["w_s"] / (p["w_s"] + p["a"] + p["b"] / p["c"]) if p["w_s"] > 0 else 0.0)
        ids_l += [a, b_]
        w_l += [wa, wb]
        sizes += [len(a), len(b_)]
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    batch = W.Batch(np.concatenate(ids_l), np.concatenate(w_l), off, m)
    jps = np.array(jps)
    for variant in ("1", "3"):
        z, _ = _sigs(H, batch, variant, 1, seed=1)
        za = z[0::2].contiguous()
        zb = z[1::2].contiguous()
        idx = torch.arange(100, device="cuda")
        cnt = H.estimate_pairs(za, zb, idx, idx).cpu().numpy()
        zn = pmh.to_u64(z)
        assert np.array_equal(cnt, (zn[0::2] == zn[1::2]).sum(1))      # exact counts
        est = cnt / m
        var = jps * (1 - jps) / m
        z_scores = (est - jps) / np.sqrt(np.maximum(var, 1e-12))
        assert np.all(np.abs(z_scores[(jps > 0) & (jps < 1)]) < 5.5), variant
        assert np.all(est[jps == 0] == 0) and np.all(est[jps == 1] == 1)
        assert np.mean(z_scores ** 2) < 1.5


@pytest.mark.slow
def test_c4_full_allpairs_sampled_rows(H):
    from paper_1911_00675_gb300 import pmh
    b = W.batch_c4_sets()
    z, _ = _sigs(H, b)                                  # 16,384 x 1024 ProbMinHash3a signatures
    cnt = H.estimate_allpairs(z)
    torch.cuda.synchronize()
    zn = pmh.to_u64(z)
    rng = np.random.default_rng(1)
    rows = np.concatenate([[0, zn.shape[0] - 1], rng.choice(zn.shape[0], 14, replace=False)])
    got = cnt[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint16)
    for r_i, r in enumerate(rows):
        ref = (zn == zn[r]).sum(1)
        assert np.array_equal(got[r_i], ref)
    # the family structure spans the range: within-family counts are high, across families ~0
    assert got[:, :].max() == 1024


def test_block_counts_match_oracle_and_tile_the_matrix(H):
    # one block of the pair matrix between two tables (strided output), and the 2-D tiles of the
    # multi-GPU split computed on one GPU and put together: the full all-pairs matrix
    import oracle
    from paper_1911_00675_gb300 import shard
    rng = np.random.default_rng(40)
    base = rng.integers(0, 2**62, size=(6, 300), dtype=np.uint64)
    sig = base[rng.integers(0, 6, size=333)].copy()
    noise = rng.random(sig.shape) < 0.3
    sig[noise] = rng.integers(0, 2**62, size=int(noise.sum()), dtype=np.uint64)
    ref = oracle.count_allpairs(sig).astype(np.int64)
    d = torch.from_numpy(sig.view(np.int64).copy()).cuda()
    out = torch.full((70, 141), -1, dtype=torch.int16, device="cuda")
    H.estimate_jp_block(d[5:75].contiguous(), d[190:330].contiguous(), counts=out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.int64)
    assert np.array_equal(got[:, :140], ref[5:75, 190:330]) and (got[:, 140] == -1).all()
    full = np.full((333, 333), -1, dtype=np.int64)
    for rank_tiles in shard.pair_tiles(333, 3):
        for r0, r1, c0, c1 in rank_tiles:
            c = H.estimate_jp_block(d[r0:r1].contiguous(), d[c0:c1].contiguous())
            torch.cuda.synchronize()
            full[r0:r1, c0:c1] = c.cpu().numpy().astype(np.int64)
    iu = np.triu_indices(333)
    assert np.array_equal(full[iu], ref[iu])
