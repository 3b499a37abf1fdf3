"""Pins for the CPU oracle (no GPU).

The oracle is pinned to things other than itself: published test vectors,
closed forms of the paper's distributions and tables, the brute-force
definition of the signature (Eq. def_new_exp + Eq. signature_def), the paper's
own equivalence claims (ProbMinHash1 = 1a, 3 = 3a), invariants (element order,
weight scale), the exponential-race marginals, the estimator's variance
(Eq. jaccard_variance and the MSE variance in Sec. Verification) and the
SuperMinHash improvement factor (Eq. improvement_factor).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1911_00675_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
VARS = ["1", "1a", "2", "3", "3a", "4"]


def _mix_py(z):
    m = (1 << 64) - 1
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


# ---------------------------------------------------------------- stream --
def test_splitmix64_reference_values():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [ln.split(";") for ln in f if ln.strip() and not ln.startswith("#")]
    for j, hx in rows:
        assert oracle.word(0, int(j)) == int(hx, 16)


def test_uniform_range_and_resolution():
    assert oracle.unif(0) == 0.0
    assert oracle.unif((1 << 64) - 1) == 1.0 - 2.0**-53
    assert oracle.unif(1 << 11) == 2.0**-53
    assert oracle.exp1(0) == 0.0
    assert math.isfinite(oracle.exp1((1 << 64) - 1))


def _words(n, seed=1):
    k = oracle.key(12345, seed)
    return [oracle.word(k, j) for j in range(n)]


def test_exp1_distribution():
    e = np.array([oracle.exp1(w) for w in _words(20000)])
    assert stats.kstest(e, "expon").pvalue > 1e-4
    assert abs(e.mean() - 1.0) < 0.05


@pytest.mark.parametrize("m", [2, 3, 64, 1024])
def test_truncated_exp_distribution(m):
    lam = math.log1p(1.0 / (m - 1))
    c, inv = math.expm1(-lam), 1.0 / lam
    x = np.array([oracle.texp(w, c, inv) for w in _words(20000, seed=m)])
    assert x.min() >= 0.0 and x.max() < 1.0
    cdf = lambda t: (1.0 - np.exp(-lam * t)) / (1.0 - math.exp(-lam))   # Exp(lambda;0,1)
    assert stats.kstest(x, cdf).pvalue > 1e-4


def test_uniform_int_range_and_balance():
    for r in (1, 2, 3, 7, 1000, 4096):
        ks = np.array([oracle.uint(w, r) for w in _words(6000, seed=r)])
        assert ks.min() >= 0 and ks.max() < r
        if 1 < r <= 8:
            cnt = np.bincount(ks, minlength=r)
            assert stats.chisquare(cnt).pvalue > 1e-4
    assert oracle.uint((1 << 64) - 1, 4096) == 4095
    assert oracle.uint(0, 4096) == 0


def test_key_depends_on_id_and_seed():
    assert oracle.key(1, 0) != oracle.key(2, 0)
    assert oracle.key(1, 0) != oracle.key(1, 1)
    assert oracle.key(5, 9) == _mix_py(5 ^ _mix_py(9))


# ---------------------------------------------------------------- tables --
@pytest.mark.parametrize("m", [2, 3, 5, 256, 4096])
def test_tables_closed_forms(m):
    beta, gamma, dgamma, lam, (lam3, c3, inv3, delta) = oracle.tables(m)
    assert gamma[0] == 0.0 and gamma[1] == 1.0                 # gamma_1 = lambda_1/lambda_1
    assert lam3 == pytest.approx(math.log(m / (m - 1)), rel=1e-14)
    assert delta == pytest.approx(1.0 / lam3, rel=1e-15)
    for i in range(1, m + 1):
        assert beta[i] == pytest.approx(m / (m - i + 1), rel=1e-15)
    for i in range(1, m):
        # boundaries of the correlated generation: gamma_i = log(m/(m-i))/lambda_1
        assert gamma[i] == pytest.approx(math.log(m / (m - i)) / lam3, rel=1e-12)
        # every interval [gamma_{i-1}, gamma_i) carries probability 1/m under Exp(lambda_1)
        p = math.exp(-lam3 * gamma[i - 1]) - math.exp(-lam3 * gamma[i])
        assert p == pytest.approx(1.0 / m, rel=1e-9)
        # rate of the i-th truncated exponential: lambda_1 * (gamma_i - gamma_{i-1}) = lambda_i
        assert lam3 * dgamma[i] == pytest.approx(lam[i], rel=1e-9)


@pytest.mark.parametrize("m", [2, 16, 1024])
def test_pmh3_intervals_match_first_occurrence_law(m):
    # With replacement the i-th label is the first k with probability (1/m)(1-1/m)^(i-1)
    # (Eq. correlated_probabilities, r -> inf); the interval [i-1, i) carries exactly that
    # mass under Exp(lambda) with lambda = log(1 + 1/(m-1)).
    lam = oracle.tables(m)[4][0]
    for i in (1, 2, 5, 50):
        p_int = math.exp(-lam * (i - 1)) - math.exp(-lam * i)
        assert p_int == pytest.approx((1 / m) * (1 - 1 / m) ** (i - 1), rel=1e-9)


# ------------------------------------------------------------ track_max --
@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 7, 8, 16, 33, 100])
def test_track_max_matches_linear_max(m):
    rng = np.random.default_rng(m)
    cnt = 40 * m
    leaves = rng.integers(0, m, size=cnt)
    vals = rng.exponential(1.0, size=cnt)
    roots = oracle.track_max_run(m, vals, leaves)
    q = np.full(m, np.inf)
    for t in range(cnt):
        q[leaves[t]] = min(q[leaves[t]], vals[t])
        assert roots[t] == q.max()


def test_ties_keep_smallest_id_in_any_order():
    # Reading of the tie rule: lexicographic (value, id) minimum per component.
    vals = [2.0, 1.0, 1.0, 1.0, 3.0]
    ids = [50, 40, 30, 35, 10]
    for perm in ([0, 1, 2, 3, 4], [4, 3, 2, 1, 0], [2, 0, 4, 1, 3]):
        q, z = oracle.offer_run(1, [vals[i] for i in perm], [ids[i] for i in perm], [0] * 5)
        assert q[0] == 1.0 and z[0] == 30


# ---------------------------------------------------------- permutation --
@pytest.mark.parametrize("m", [1, 2, 5, 64, 300])
def test_lazy_permutation_is_fisher_yates(m):
    for e in range(20):
        k = oracle.key(e, 77)
        lab = oracle.perm_labels(m, k, m)
        assert sorted(lab.tolist()) == list(range(m))
        # eager Fisher-Yates with the same draws
        p = list(range(m))
        ref = []
        for t in range(m):
            r = t + oracle.uint(oracle.word(k, 2 * t + 1), m - t)
            ref.append(p[r])
            p[r], p[t] = p[t], p[r]
        assert lab.tolist() == ref


def test_lazy_permutation_first_label_uniform():
    m = 6
    first = [int(oracle.perm_labels(m, oracle.key(e, 3), 1)[0]) for e in range(6000)]
    assert stats.chisquare(np.bincount(first, minlength=m)).pvalue > 1e-4


# ---------------------------------------------- definition & invariants --
def _rand_set(rng, n, weight="uniform"):
    ids = W.distinct_ids(int(rng.integers(0, 2**40)), n, int(rng.integers(0, 2**32)))
    if weight == "uniform":
        w = 1.0 - rng.random(n)
    elif weight == "pareto":
        w = (1.0 - rng.random(n)) ** (-1 / 1.5)
    elif weight == "lognormal":
        w = rng.lognormal(0, 2, n)
    else:
        w = np.ones(n)
    return ids, w


@pytest.mark.parametrize("variant", VARS)
def test_early_stop_equals_brute_force(variant):
    rng = np.random.default_rng(100 + VARS.index(variant))
    for trial in range(40):
        n = int(rng.integers(1, 80))
        m = int(rng.integers(2, 70))
        ids, w = _rand_set(rng, n, ["uniform", "pareto", "lognormal", "unit"][trial % 4])
        q, z, _ = oracle.sketch(variant, ids, w, m, seed=trial)
        qb, zb, _ = oracle.sketch(variant, ids, w, m, seed=trial, brute=True)
        assert np.array_equal(z, zb) and np.array_equal(q, qb)


@pytest.mark.parametrize("pair", [("1", "1a"), ("3", "3a")])
def test_interleaved_equals_sequential(pair):
    rng = np.random.default_rng(7)
    for trial in range(30):
        n = int(rng.integers(1, 3000))
        m = int(rng.choice([2, 16, 128, 256]))
        ids, w = _rand_set(rng, n, ["uniform", "pareto", "lognormal"][trial % 3])
        qa, za, _ = oracle.sketch(pair[0], ids, w, m, seed=trial)
        qb, zb, _ = oracle.sketch(pair[1], ids, w, m, seed=trial)
        assert np.array_equal(za, zb) and np.array_equal(qa, qb)


@pytest.mark.parametrize("variant", VARS)
def test_order_independence(variant):
    rng = np.random.default_rng(11)
    for trial in range(10):
        n = int(rng.integers(1, 500))
        ids, w = _rand_set(rng, n)
        q, z, _ = oracle.sketch(variant, ids, w, 64, seed=3)
        perm = rng.permutation(n)
        q2, z2, _ = oracle.sketch(variant, ids[perm], w[perm], 64, seed=3)
        assert np.array_equal(z, z2) and np.array_equal(q, q2)


@pytest.mark.parametrize("variant", VARS)
def test_scale_invariance(variant):
    rng = np.random.default_rng(12)
    for trial in range(8):
        ids, w = _rand_set(rng, int(rng.integers(1, 400)), "lognormal")
        q, z, _ = oracle.sketch(variant, ids, w, 64, seed=5)
        q2, z2, _ = oracle.sketch(variant, ids, w * 8.0, 64, seed=5)      # exact power-of-two scaling
        assert np.array_equal(z, z2) and np.array_equal(q2, q / 8.0)
        q3, z3, _ = oracle.sketch(variant, ids, w * 3.7, 64, seed=5)      # general factor
        assert np.array_equal(z, z3)


@pytest.mark.parametrize("variant", VARS)
def test_single_element(variant):
    for m in (2, 17, 256):
        q, z, st = oracle.sketch(variant, np.array([42], dtype=np.uint64), np.array([0.3]), m, seed=1)
        assert (z == 42).all() and np.isfinite(q).all()
        if variant == "2":
            assert st["points"] == m          # exactly m points when n = 1
        if variant == "4":
            assert st["points"] <= m


def test_zero_weights_skipped_and_empty_sets():
    ids = np.array([1, 2, 3], dtype=np.uint64)
    for v in VARS:
        q, z, _ = oracle.sketch(v, ids, np.array([0.0, 1.0, 0.0]), 8, seed=0)
        assert (z == 2).all()
        q, z, _ = oracle.sketch(v, ids, np.zeros(3), 8, seed=0)
        assert (z == 0).all() and np.isinf(q).all()
        q, z, _ = oracle.sketch(v, ids[:0], np.zeros(0), 8, seed=0)
        assert (z == 0).all() and np.isinf(q).all()


def test_error_codes():
    ids = np.array([1, 2], dtype=np.uint64)
    for bad in (-1.0, np.nan, np.inf, 1e-320):
        assert oracle.sketch_status("1", ids, np.array([1.0, bad]), 8) == oracle.ERR_BAD_WEIGHT
    for v in ("3", "3a", "4"):
        assert oracle.sketch_status(v, ids, np.array([1.0, 2.0]), 1) == oracle.ERR_INVALID_ARG
    for v in ("1", "1a", "2"):
        assert oracle.sketch_status(v, ids, np.array([1.0, 2.0]), 1) == oracle.OK


# ------------------------------------------------------------- marginals --
@pytest.mark.parametrize("variant", VARS)
def test_marginals_exponential_race(variant):
    # P(z_k = d) = w(d) / sum(w): the exponential race behind Eq. def_hash_jp.
    ids = np.array([11, 22, 33, 44], dtype=np.uint64)
    w = np.array([1.0, 2.0, 3.0, 4.0])
    m = 32
    counts = np.zeros(4)
    for seed in range(400):
        _, z, _ = oracle.sketch(variant, ids, w, m, seed=seed)
        for j, d in enumerate(ids):
            counts[j] += np.count_nonzero(z == d)
    expected = w / w.sum() * counts.sum()
    # components within one signature are dependent for 3/3a/4; use a wide acceptance
    assert stats.chisquare(counts, expected).pvalue > 1e-6


@pytest.mark.parametrize("variant", VARS)
def test_hash_values_are_exponential(variant):
    # h_k(d) ~ Exp(lambda * w(d)) with lambda = 1/m (ProbMinHash1/2) or log(1+1/(m-1)) (3/4).
    m, w = 16, 2.5
    lam = 1.0 / m if variant in ("1", "1a", "2") else math.log1p(1.0 / (m - 1))
    vals = []
    for seed in range(3000):
        q, _, _ = oracle.sketch(variant, np.array([9], dtype=np.uint64), np.array([w]), m, seed=seed)
        vals.append(q[seed % m] * lam * w)
    assert stats.kstest(vals, "expon").pvalue > 1e-4


# ----------------------------------------------------------------- J_P --
def _golden_jp():
    rows = []
    with open(os.path.join(GOLDEN, "jp_examples.txt")) as f:
        for ln in f:
            if not ln.strip() or ln.startswith("#"):
                continue
            pairs, frac = ln.split(";")
            ws = [tuple(float(x) for x in p.split(",")) for p in pairs.split()]
            rows.append((ws, Fraction(frac.strip())))
    return rows


def test_jp_golden_examples():
    rng = np.random.default_rng(0)
    for ws, frac in _golden_jp():
        a, wa, b, wb = W.pair_from_weight_pairs(rng, ws)
        assert oracle.jp(a, wa, b, wb) == pytest.approx(float(frac), rel=1e-14)
        assert oracle.jp(b, wb, a, wa) == pytest.approx(float(frac), rel=1e-14)


def test_jp_properties():
    rng = np.random.default_rng(1)
    for t in range(20):
        a, wa, b, wb, p = W.constructed_pair(rng, t / 19.0, n_total=int(rng.integers(10, 300)))
        closed = p["w_s"] / (p["w_s"] + p["a"] + p["b"] / p["c"]) if p["w_s"] > 0 else 0.0
        assert oracle.jp(a, wa, b, wb) == pytest.approx(closed, rel=1e-12, abs=1e-15)
        assert oracle.jp(a, wa * 3.0, b, wb) == pytest.approx(closed, rel=1e-12, abs=1e-15)
    ids, w = _rand_set(rng, 50, "lognormal")
    assert oracle.jp(ids, w, ids, w) == pytest.approx(1.0, rel=1e-14)
    ids2, w2 = _rand_set(rng, 30)
    assert oracle.jp(ids, w, ids2, w2) == 0.0
    # binary weights: J_P equals the Jaccard similarity
    u = W.distinct_ids(0, 40, 9)
    a, b = u[:25], u[10:]
    assert oracle.jp(a, np.ones(25), b, np.ones(30)) == pytest.approx(15 / 40, rel=1e-14)


# ---------------------------------------------------- estimator & error --
def _mse_zscore(est, jp, m):
    c = len(est)
    mse = float(np.mean((np.asarray(est) - jp) ** 2))
    mean = jp * (1 - jp) / m
    var = (jp**2 * (1 - jp) ** 2 / (m**2 * c)) * (2 - 6 / m) + jp * (1 - jp) / (m**3 * c)
    return mse / mean, (mse - mean) / math.sqrt(var)


@pytest.mark.parametrize("example", [[(3, 20), (30, 7)], [(0, 1), (1, 0), (1, 1)]])
def test_relative_mse_on_paper_examples(example):
    # Sec. Verification: relative MSE ~ 1 for the uncorrelated variants (independent
    # components, Eq. jaccard_variance) and <= 1 for the correlated ones; z-score of the
    # empirical MSE from the variance formula printed there.
    m, c = 32, 1500
    rng = np.random.default_rng(2)
    pairs = [W.pair_from_weight_pairs(rng, example) for _ in range(c)]
    jp = oracle.jp(*pairs[0])
    for variant in ("1", "2", "3", "4"):
        est = []
        for t, (a, wa, b, wb) in enumerate(pairs):
            _, za, _ = oracle.sketch(variant, a, wa, m, seed=t)
            _, zb, _ = oracle.sketch(variant, b, wb, m, seed=t)
            est.append(oracle.count_equal(za, zb) / m)
        rel, z = _mse_zscore(est, jp, m)
        if variant in ("1", "2"):
            assert abs(z) < 4.5, (variant, rel, z)
        else:
            # correlated generation: the error is significantly reduced for n < m
            assert rel < 0.9 and z < -3.0, (variant, rel, z)
    # P-MinHash reference
    est = []
    for t, (a, wa, b, wb) in enumerate(pairs):
        _, za = oracle.pminhash(a, wa, m, seed=t)
        _, zb = oracle.pminhash(b, wb, m, seed=t)
        est.append(oracle.count_equal(za, zb) / m)
    assert abs(_mse_zscore(est, jp, m)[1]) < 4.5


def _alpha(m, u):
    """SuperMinHash improvement factor, Eq. improvement_factor (exact rational)."""
    s = sum(Fraction(l) ** u * ((l + 1) ** u + (l - 1) ** u - 2 * l**u) for l in range(1, m))
    return 1 - s / (Fraction(m - 1) ** (u - 1) * Fraction(m) ** u * (u - 1))


def test_pmh4_unit_weights_matches_superminhash_variance():
    # With binary weights ProbMinHash4 is logically SuperMinHash (Sec. Conventional Jaccard
    # Similarity); its estimator variance is alpha(m,u) J(1-J)/m (Eq. superminhash_variance).
    m, c = 16, 4000
    u_ids = W.distinct_ids(0, 4, 5)
    rng = np.random.default_rng(3)
    a_idx, b_idx = [0, 1, 2], [1, 2, 3]     # J = 2/4, u = 4
    jp = 0.5
    alpha = float(_alpha(m, 4))
    est = []
    for t in range(c):
        ids = W.distinct_ids(int(rng.integers(0, 2**40)), 4, t)
        _, za, _ = oracle.sketch("4", ids[a_idx], np.ones(3), m, seed=t)
        _, zb, _ = oracle.sketch("4", ids[b_idx], np.ones(3), m, seed=t)
        est.append(oracle.count_equal(za, zb) / m)
    mse = float(np.mean((np.array(est) - jp) ** 2))
    predicted = alpha * jp * (1 - jp) / m
    assert mse / predicted == pytest.approx(1.0, abs=0.12)
    assert alpha < 0.8       # the improvement is real at u < m


def test_count_equal_and_allpairs():
    rng = np.random.default_rng(4)
    sig = rng.integers(0, 5, size=(7, 64)).astype(np.uint64)
    cnt = oracle.count_allpairs(sig)
    ref = (sig[:, None, :] == sig[None, :, :]).sum(-1)
    assert np.array_equal(cnt, ref)
    assert oracle.count_equal(sig[0], sig[1]) == ref[0, 1]


# -------------------------------------------------------- work counters --
def test_work_counters_match_paper_analysis():
    m = 128
    hm = sum(1 / k for k in range(1, m + 1))
    rng = np.random.default_rng(5)
    for n in (1, 10, 1000):
        pts, buf1 = [], []
        for t in range(30):
            ids, w = _rand_set(rng, n)
            pts.append(oracle.sketch("1", ids, w, m, seed=t)[2]["points"])
            buf1.append(oracle.sketch("1a", ids, w, m, seed=t)[2]["buffer_max"])
        hn = sum(1 / k for k in range(1, n + 1))
        # total points ~ m H_m H_n (Sec. ProbMinHash1) for n <~ m H_m; each element costs >= 1
        assert np.mean(pts) == pytest.approx(max(m * hm * hn, n), rel=0.35)
        # expected maximum buffer of 1a: sum_j min(1, m H_m / j) (Sec. Interleaved Element Processing)
        eb = sum(min(1.0, m * hm / j) for j in range(1, n + 1))
        assert np.mean(buf1) == pytest.approx(eb, rel=0.35)
    # 3a, unit weights: buffer after pass 1 ~ min(n, m H_m) (plateau)
    n = 5000
    b3 = [oracle.sketch("3a", *_rand_set(rng, n, "unit"), m, seed=t)[2]["buffer_max"] for t in range(10)]
    assert np.mean(b3) == pytest.approx(min(n, m * hm), rel=0.35)


def test_near_tie_scan_consistency():
    rng = np.random.default_rng(6)
    for v in VARS:
        ids, w = _rand_set(rng, 300, "pareto")
        q, z, _ = oracle.sketch(v, ids, w, 64, seed=1)
        flags, ru = oracle.near_ties(v, ids, w, 64, 1, q, z, 1e-12)
        assert flags.sum() == 0
        assert (ru >= q).all()
        # a huge relative gap flags every component with a runner-up
        flags, ru = oracle.near_ties(v, ids, w, 64, 1, q, z, 1e6)
        assert flags.sum() == np.isfinite(ru).sum()


def _singleton_hashes(variant, ids, w, m, seed):
    """h_k(d) for every element d and component k: the signature of the one-element set {d} holds
    exactly d's first point with each label (Eq. def_new_exp), computed by the pinned algorithm."""
    return np.array([oracle.sketch(variant, ids[j:j + 1], w[j:j + 1], m, seed=seed)[0] for j in range(len(ids))])


@pytest.mark.parametrize("variant", VARS + ["3u", "3au", "4u"])
def test_near_tie_scan_runner_up_equals_singletons(variant):
    # The near-tie scan decides which GPU/oracle id mismatches are forgiven, so its runner-up is
    # pinned to an independent computation: per component the second smallest h_k(d) over the
    # set's elements (Eq. signature_def ranks (h_k(d), d) lexicographically), taken from the
    # singleton signatures.  The scan only sees points up to q_max (1 + rel); wide windows
    # (rel = 0.3, 3) put runner-ups of the maximum component above q_max inside it.
    rng = np.random.default_rng(810 + (VARS + ["3u", "3au", "4u"]).index(variant))
    for trial, m in enumerate([7, 16, 33, 64]):
        n = int(rng.integers(2, 60))
        ids, w = _rand_set(rng, n, ["uniform", "pareto", "lognormal", "unit"][trial])
        seed = 40 + trial
        h = _singleton_hashes(variant, ids, w, m, seed)
        q, z, _ = oracle.sketch(variant, ids, w, m, seed=seed)
        for rel in (1e-12, 0.3, 3.0):
            flags, ru = oracle.near_ties(variant, ids, w, m, seed, q, z, rel)
            bound = q.max() * (1.0 + rel)
            for k in range(m):
                order = np.lexsort((ids, h[:, k]))
                assert ids[order[0]] == z[k] and h[order[0], k] == q[k]
                second = h[order[1], k]
                expect = second if second <= bound else np.inf
                assert ru[k] == expect, (variant, m, rel, k)
                assert bool(flags[k]) == bool(np.isfinite(expect) and expect - q[k] < rel * q[k])


@pytest.mark.parametrize("variant", VARS)
@pytest.mark.parametrize("where", ["first", "max"])
def test_near_tie_scan_flags_a_planted_tie(variant, where):
    # Two elements A and B.  B's weight is chosen so that its point with label k lies within
    # 3e-13 relative above A's (all of B's points scale with 1/w_B), so A wins component k by
    # less than 1e-12 relative: a near tie the scan must flag with B's value as runner-up.
    # where = "first": k = the label of A's first point.  where = "max": k = A's largest
    # component, which stays the set's maximum component (every component is at most A's
    # value), so B's point lies above q_max and is found only through the widened window.
    m, seed = 16, 9
    pool = W.distinct_ids(1 << 33, 400, 77)
    a, wa = pool[:1], np.array([1.0])
    ha = oracle.sketch(variant, a, wa, m, seed=seed)[0]
    k = int(np.argmin(ha)) if where == "first" else int(np.argmax(ha))
    for b in pool[1:]:
        hb1 = oracle.sketch(variant, np.array([b], dtype=np.uint64), np.array([1.0]), m, seed=seed)[0]
        wb = hb1[k] / (ha[k] * (1.0 + 3e-13))
        hb = oracle.sketch(variant, np.array([b], dtype=np.uint64), np.array([wb]), m, seed=seed)[0]
        gap = (hb[k] - ha[k]) / ha[k]
        if not 0.0 < gap < 1e-12:
            continue
        # A must win every other component comfortably (B's values elsewhere well above A's)
        others = np.delete(np.arange(m), k)
        if where == "max" and not (hb[others] > ha[others] * 1.01).all():
            continue
        ids = np.array([a[0], b], dtype=np.uint64)
        w = np.array([wa[0], wb])
        q, z, _ = oracle.sketch(variant, ids, w, m, seed=seed)
        assert z[k] == a[0] and q[k] == ha[k]
        if where == "max":
            assert q[k] == q.max()
        flags, ru = oracle.near_ties(variant, ids, w, m, seed, q, z, 1e-12)
        assert flags[k] == 1 and ru[k] == hb[k]
        assert flags.sum() == 1
        return
    pytest.fail("no element found to plant a near tie")


# --------------------------------------------------------------- b-bit signatures
# Algorithm "Reduction to a b-bit signature": each component becomes b bits of a hash of
# (component, index); the estimator must account for collisions of different elements.

def test_bbit_64_preserves_equality_exactly():
    # b = 64 keeps the whole hash: a bijection of the id for each index, so equal-component
    # counts of the codes are those of the ids
    rng = np.random.default_rng(70)
    m, n = 48, 30
    base = rng.integers(0, 2**63, size=(6, m), dtype=np.uint64)
    sigs = base[rng.integers(0, 6, size=n)].copy()
    noise = rng.random((n, m)) < 0.4
    sigs[noise] = rng.integers(0, 2**63, size=int(noise.sum()), dtype=np.uint64)
    codes = oracle.bbit_reduce(sigs, 64, seed=3)
    assert np.array_equal(oracle.count_allpairs(codes), oracle.count_allpairs(sigs))
    assert np.array_equal(codes[0, :5], [oracle.bbit_code(int(sigs[0, k]), k, 64, 3) for k in range(5)])


@pytest.mark.parametrize("b", [1, 2, 4, 8])
def test_bbit_codes_uniform_and_collision_rate(b):
    # different ids collide with probability 2^-b; codes are uniform on {0..2^b-1}
    rng = np.random.default_rng(71 + b)
    m, n = 512, 400
    sigs = rng.integers(0, 2**64, size=(n, m), dtype=np.uint64)
    codes = oracle.bbit_reduce(sigs, b, seed=9)
    assert codes.max() < 2**b
    counts = np.bincount(codes.ravel().astype(np.int64), minlength=2**b)
    expected = codes.size / 2**b
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 2**b + 6 * np.sqrt(2 * 2**b)          # chi-square with 2^b - 1 dof, far tail
    a, c = codes[0::2], codes[1::2]
    p = 2.0 ** -b
    matches = (a == c).sum()
    trials = a.size
    assert abs(matches - trials * p) < 5 * np.sqrt(trials * p * (1 - p))


def test_bbit_index_enters_the_hash():
    # two signatures made of one id each, repeated over all components: with the index in the
    # hash their codes match at rate 2^-b per component, not all-or-nothing
    m, b = 4096, 1
    za = np.full((1, m), 0x1234567890ABCDEF, dtype=np.uint64)
    zb = np.full((1, m), 0x0FEDCBA098765432, dtype=np.uint64)
    ca = oracle.bbit_reduce(za, b, seed=1)
    cb = oracle.bbit_reduce(zb, b, seed=1)
    matches = int((ca == cb).sum())
    assert abs(matches - m / 2) < 5 * np.sqrt(m / 4)
    assert len(np.unique(ca)) == 2                        # one id, both code values over the components


@pytest.mark.parametrize("b", [1, 4, 8])
def test_bbit_estimator_is_unbiased(b):
    # pairs with exactly j*m equal components and the rest distinct: the corrected estimate
    # averages to j (E[count/m] = J + (1 - J) 2^-b)
    rng = np.random.default_rng(80 + b)
    m = 256
    for j in (0.0, 0.3, 0.8, 1.0):
        est = []
        for t in range(200):
            a = rng.integers(0, 2**64, size=(1, m), dtype=np.uint64)
            c = rng.integers(0, 2**64, size=(1, m), dtype=np.uint64)
            eq = rng.permutation(m)[: int(round(j * m))]
            c[0, eq] = a[0, eq]
            ca, cc = oracle.bbit_reduce(a, b, 5), oracle.bbit_reduce(c, b, 5)
            est.append(oracle.bbit_estimate(int((ca == cc).sum()), m, b))
        p = 2.0 ** -b
        jj = round(j * m) / m                              # the exact fraction planted
        sd = np.sqrt((1 - jj) * p * (1 - p) / m) / (1 - p) / np.sqrt(len(est))
        assert abs(np.mean(est) - jj) < 5 * sd + 1e-12, (jj, np.mean(est))
    assert oracle.bbit_estimate(m, m, b) == 1.0


# --------------------------------------------------- binary-weight specialisations
# Sec. Conventional Jaccard Similarity: with weights in {0, 1} all elements share the interval
# boundaries of ProbMinHash3/4, so the truncated exponentials become Uniform([0,1)) and
# gamma_i = i; ProbMinHash4 then is SuperMinHash.
UVARS = ["3u", "3au", "4u"]


@pytest.mark.parametrize("variant", UVARS)
def test_unweighted_early_stop_equals_brute_force(variant):
    rng = np.random.default_rng(300 + UVARS.index(variant))
    for trial in range(40):
        n = int(rng.integers(1, 80))
        m = int(rng.integers(1, 70))
        ids, _ = _rand_set(rng, n, "unit")
        w = np.ones(n)
        q, z, _ = oracle.sketch(variant, ids, w, m, seed=trial)
        qb, zb, _ = oracle.sketch(variant, ids, w, m, seed=trial, brute=True)
        assert np.array_equal(z, zb) and np.array_equal(q, qb)


def test_unweighted_interleaved_equals_sequential_and_ignores_weight_values():
    rng = np.random.default_rng(310)
    for trial in range(20):
        n = int(rng.integers(1, 2000))
        m = int(rng.choice([1, 2, 16, 256]))
        ids, w = _rand_set(rng, n, "pareto")
        q, z, _ = oracle.sketch("3u", ids, w, m, seed=trial)
        qa, za, _ = oracle.sketch("3au", ids, w, m, seed=trial)
        assert np.array_equal(z, za) and np.array_equal(q, qa)
        # only w > 0 matters: the same set with unit weights has the same signature
        q1, z1, _ = oracle.sketch("3u", ids, np.ones(n), m, seed=trial)
        assert np.array_equal(z, z1) and np.array_equal(q, q1)
        q4, z4, _ = oracle.sketch("4u", ids, w, m, seed=trial)
        q41, z41, _ = oracle.sketch("4u", ids, np.ones(n), m, seed=trial)
        assert np.array_equal(z4, z41) and np.array_equal(q4, q41)


@pytest.mark.parametrize("variant", UVARS)
def test_unweighted_marginals_are_uniform(variant):
    # binary weights: every element wins a component with probability 1/n
    ids = np.array([11, 22, 33, 44, 55], dtype=np.uint64)
    m = 32
    counts = np.zeros(len(ids))
    for seed in range(400):
        _, z, _ = oracle.sketch(variant, ids, np.ones(len(ids)), m, seed=seed)
        for j, d in enumerate(ids):
            counts[j] += np.count_nonzero(z == d)
    assert counts.sum() == 400 * m
    assert stats.chisquare(counts).pvalue > 1e-6


def test_unweighted_points_are_uniform_plus_index():
    # x_i = (i-1) + U_i: the fractional parts of the first points are Uniform([0,1))
    rng = np.random.default_rng(320)
    ids = W.distinct_ids(5, 2000, 5)
    for variant in ("3u", "4u"):
        q, _, _ = oracle.sketch(variant, ids[:1], np.ones(1), 4096, seed=9)   # one element: all its points
        frac = q[np.isfinite(q)] % 1.0
        assert stats.kstest(frac, "uniform").pvalue > 1e-4
    # 4u draws labels without replacement: point i lands in its own component, so the integer
    # parts of a single element's signature are a permutation of 0..m-1
    q, _, _ = oracle.sketch("4u", ids[:1], np.ones(1), 4096, seed=9)
    assert np.array_equal(np.sort(np.floor(q)), np.arange(4096))


def test_pmh4u_is_superminhash():
    # the binary-weight ProbMinHash4 has SuperMinHash's estimator variance alpha(m,u) J(1-J)/m
    m, c = 16, 4000
    rng = np.random.default_rng(330)
    a_idx, b_idx = [0, 1, 2], [1, 2, 3]
    jp = 0.5
    alpha = float(_alpha(m, 4))
    est = []
    for t in range(c):
        ids = W.distinct_ids(int(rng.integers(0, 2**40)), 4, t)
        _, za, _ = oracle.sketch("4u", ids[a_idx], np.ones(3), m, seed=t)
        _, zb, _ = oracle.sketch("4u", ids[b_idx], np.ones(3), m, seed=t)
        est.append(oracle.count_equal(za, zb) / m)
    mse = float(np.mean((np.array(est) - jp) ** 2))
    assert mse / (alpha * jp * (1 - jp) / m) == pytest.approx(1.0, abs=0.12)


def test_pmh3u_estimator_unbiased_for_jaccard():
    # E[count/m] = J for binary weights (J_P = J, Sec. Probability Jaccard Similarity)
    rng = np.random.default_rng(340)
    m = 64
    est = []
    for t in range(600):
        ids = W.distinct_ids(int(rng.integers(0, 2**40)), 30, t)
        a, b = ids[:20], ids[10:]          # |A & B| = 10, |A | B| = 30: J = 1/3
        _, za, _ = oracle.sketch("3u", a, np.ones(20), m, seed=t)
        _, zb, _ = oracle.sketch("3u", b, np.ones(20), m, seed=t)
        est.append(oracle.count_equal(za, zb) / m)
    assert abs(np.mean(est) - 1 / 3) < 5 * np.std(est) / np.sqrt(len(est))


# ------------------------------------------------- rejection sampler for Exp(lambda;0,1) --
# Sec. Truncated Exponential Sampling: Exp(lambda;0,1) (density proportional to e^{-lambda x} on
# [0,1)) drawn without a logarithm: a first uniform scaled by c1 is returned when below 1,
# otherwise a rejection loop over the region between e^{-lambda} and the density.

RATES = [1e-3, 0.1, 0.5, math.log(2.0)]


def _rej_samples(lam, n, salt):
    xs, att = np.empty(n), np.empty(n, dtype=int)
    for j in range(n):
        k = oracle.key(j, salt)
        xs[j], att[j] = oracle.texp_rej(k, 1 + j % 7, oracle.word(k, 2 * (j % 7)), lam)
    return xs, att


def _te_cdf(lam):
    return lambda x: -np.expm1(-lam * np.asarray(x)) / -math.expm1(-lam)


@pytest.mark.parametrize("lam", RATES)
def test_texp_rejection_distribution(lam):
    # the variates follow Exp(lam;0,1): F(x) = (1 - e^{-lam x}) / (1 - e^{-lam})
    xs, _ = _rej_samples(lam, 20000, 91)
    assert ((xs >= 0) & (xs < 1)).all()
    assert stats.kstest(xs, _te_cdf(lam)).pvalue > 1e-4


@pytest.mark.parametrize("lam", [0.5, math.log(2.0)])
def test_texp_rejection_loop_distribution(lam):
    # the draws that went through the rejection loop follow the region between e^{-lam} and the
    # density: density proportional to e^{-lam x} - e^{-lam}, CDF
    # ((1 - e^{-lam x})/lam - x e^{-lam}) / ((1 - e^{-lam})/lam - e^{-lam})
    xs, att = _rej_samples(lam, 60000, 92)
    loop = xs[att > 0]
    assert len(loop) > 5000
    el = math.exp(-lam)
    norm = -math.expm1(-lam) / lam - el
    cdf = lambda x: (-np.expm1(-lam * np.asarray(x)) / lam - np.asarray(x) * el) / norm  # noqa: E731
    assert stats.kstest(loop, cdf).pvalue > 1e-4


@pytest.mark.parametrize("lam", RATES)
def test_texp_rejection_first_draw_and_attempt_rates(lam):
    # P(first draw below 1) = lam / (e^lam - 1) (Sec. Truncated Exponential Sampling); one loop
    # attempt succeeds with the area under the density above e^{-lam} (rescaled to [0,1] in y)
    # over the sampled rectangle's 1/2, so attempts are geometric with that success rate
    n = 40000
    _, att = _rej_samples(lam, n, 93)
    p1 = lam / math.expm1(lam)
    hit = np.count_nonzero(att == 0)
    assert abs(hit - n * p1) < 5 * math.sqrt(n * p1 * (1 - p1)) + 1
    loop = att[att > 0]
    if len(loop) > 500:
        el = math.exp(-lam)
        p_acc = 2.0 * (-math.expm1(-lam) / lam - el) / (1.0 - el)
        mean = loop.mean()
        sd = math.sqrt((1 - p_acc) / p_acc**2 / len(loop))
        assert abs(mean - 1 / p_acc) < 5 * sd


@pytest.mark.parametrize("lam", RATES)
def test_rejection_constants_fit_the_geometry(lam):
    # c1 = |A1 u A2| / |A1| (the first draw lands in A1 = [0,1) x [0, e^-lam) with P = 1/c1);
    # at x = c2 the density, rescaled y~ = (y - e^-lam)/(1 - e^-lam), is exactly 1/2; the
    # tangent of the rescaled density at 0 meets y~ = 0 at x = c3
    c1, c2, c3 = oracle.rej_consts(lam)
    el = math.exp(-lam)
    area = (1 - el) / lam            # integral of e^{-lam x} over [0, 1)
    assert c1 == pytest.approx(area / el, rel=1e-13)
    ytil = lambda x: (math.exp(-lam * x) - el) / (1 - el)  # noqa: E731
    assert ytil(c2) == pytest.approx(0.5, rel=1e-12)
    h = 1e-6
    slope0 = (ytil(h) - ytil(0.0)) / h
    assert 1.0 / -slope0 == pytest.approx(c3, rel=1e-5)


@pytest.mark.parametrize("variant", ["3", "3a", "4"])
def test_rejection_sampler_early_stop_equals_brute_force(variant):
    rng = np.random.default_rng(140 + ["3", "3a", "4"].index(variant))
    for trial in range(30):
        n = int(rng.integers(1, 80))
        m = int(rng.integers(2, 70))
        ids, w = _rand_set(rng, n, ["uniform", "pareto", "lognormal", "unit"][trial % 4])
        q, z, _ = oracle.sketch(variant, ids, w, m, seed=trial, te_rejection=True)
        qb, zb, _ = oracle.sketch(variant, ids, w, m, seed=trial, brute=True, te_rejection=True)
        assert np.array_equal(z, zb) and np.array_equal(q, qb)


def test_rejection_sampler_interleaved_equals_sequential_and_order_free():
    rng = np.random.default_rng(150)
    for trial in range(12):
        ids, w = _rand_set(rng, int(rng.integers(1, 2000)), ["uniform", "pareto", "lognormal"][trial % 3])
        m = int(rng.choice([2, 16, 256]))
        qa, za, _ = oracle.sketch("3", ids, w, m, seed=trial, te_rejection=True)
        qb, zb, _ = oracle.sketch("3a", ids, w, m, seed=trial, te_rejection=True)
        assert np.array_equal(za, zb) and np.array_equal(qa, qb)
        perm = rng.permutation(len(ids))
        qc, zc, _ = oracle.sketch("3", ids[perm], w[perm], m, seed=trial, te_rejection=True)
        assert np.array_equal(za, zc) and np.array_equal(qa, qc)


@pytest.mark.parametrize("variant", ["3", "4"])
def test_rejection_sampler_marginals_and_hash_values(variant):
    # the exponential race and h_k(d) ~ Exp(lambda w) hold with any exact Exp(lambda;0,1) sampler
    ids = np.array([11, 22, 33, 44], dtype=np.uint64)
    w = np.array([1.0, 2.0, 3.0, 4.0])
    counts = np.zeros(4)
    for seed in range(400):
        _, z, _ = oracle.sketch(variant, ids, w, 32, seed=seed, te_rejection=True)
        for j, d in enumerate(ids):
            counts[j] += np.count_nonzero(z == d)
    assert stats.chisquare(counts, w / w.sum() * counts.sum()).pvalue > 1e-6
    m, wt = 16, 2.5
    lam = math.log1p(1.0 / (m - 1))
    vals = [oracle.sketch(variant, np.array([9], dtype=np.uint64), np.array([wt]), m, seed=s,
                          te_rejection=True)[0][s % m] * lam * wt for s in range(3000)]
    assert stats.kstest(vals, "expon").pvalue > 1e-4


@pytest.mark.parametrize("variant", ["3", "4"])
def test_rejection_sampler_changes_signatures_and_scan_matches_singletons(variant):
    # the sampler draws other variates than inversion; the near-tie scan follows the sampler
    rng = np.random.default_rng(160)
    ids, w = _rand_set(rng, 40, "pareto")
    m, seed = 33, 4
    q0, z0, _ = oracle.sketch(variant, ids, w, m, seed=seed)
    q, z, _ = oracle.sketch(variant, ids, w, m, seed=seed, te_rejection=True)
    assert not np.array_equal(q, q0)
    h = np.array([oracle.sketch(variant, ids[j:j + 1], w[j:j + 1], m, seed=seed, te_rejection=True)[0]
                  for j in range(len(ids))])
    flags, ru = oracle.near_ties(variant, ids, w, m, seed, q, z, 3.0, te_rejection=True)
    bound = q.max() * 4.0
    for k in range(m):
        order = np.lexsort((ids, h[:, k]))
        assert ids[order[0]] == z[k] and h[order[0], k] == q[k]
        second = h[order[1], k]
        assert ru[k] == (second if second <= bound else np.inf)


# ------------------------------------------------------------------ P-MinHash --
# Algorithm P-MinHash: h_k(d) = Exp(1)/w(d) independently per component (no early stop); the
# reference method the ProbMinHash algorithms are compared with, also built on the GPU.

def test_pminhash_exponential_race_and_hash_values():
    ids = np.array([11, 22, 33, 44], dtype=np.uint64)
    w = np.array([1.0, 2.0, 3.0, 4.0])
    counts = np.zeros(4)
    for seed in range(300):
        _, z = oracle.pminhash(ids, w, 32, seed=seed)
        for j, d in enumerate(ids):
            counts[j] += np.count_nonzero(z == d)
    assert stats.chisquare(counts, w / w.sum() * counts.sum()).pvalue > 1e-4
    # a single element: every component holds an independent Exp(1)/w
    q, z = oracle.pminhash(np.array([9], dtype=np.uint64), np.array([2.5]), 4000, seed=1)
    assert (z == 9).all()
    assert stats.kstest(q * 2.5, "expon").pvalue > 1e-4
    assert abs(np.corrcoef(q[:-1], q[1:])[0, 1]) < 0.06


def test_pminhash_invariants():
    rng = np.random.default_rng(170)
    for trial in range(8):
        ids, w = _rand_set(rng, int(rng.integers(1, 300)), ["uniform", "pareto", "lognormal", "unit"][trial % 4])
        q, z = oracle.pminhash(ids, w, 64, seed=trial)
        perm = rng.permutation(len(ids))
        q2, z2 = oracle.pminhash(ids[perm], w[perm], 64, seed=trial)
        assert np.array_equal(q, q2) and np.array_equal(z, z2)
        q3, z3 = oracle.pminhash(ids, w * 4.0, 64, seed=trial)
        assert np.array_equal(z, z3) and np.array_equal(q3, q / 4.0)
        # the signature of a disjoint union is the lexicographic minimum of the parts' (Eq. signature_def)
        cut = len(ids) // 2
        qa, za = oracle.pminhash(ids[:cut], w[:cut], 64, seed=trial)
        qb, zb = oracle.pminhash(ids[cut:], w[cut:], 64, seed=trial)
        take_b = (qb < qa) | ((qb == qa) & (zb < za))
        assert np.array_equal(np.where(take_b, zb, za), z) and np.array_equal(np.where(take_b, qb, qa), q)


def test_sketch_batch_is_the_per_set_sketch():
    """The oracle's CSR batch loop: each row is that set's own signature (offsets, empty sets),
    and a set with a bad weight reports its status with zero ids and +inf q."""
    rng = np.random.default_rng(99)
    sizes = [5, 0, 40, 3, 17]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    ids = rng.permutation(10_000)[: off[-1]].astype(np.uint64) * np.uint64(2654435761) + np.uint64(12345)
    w = rng.uniform(0.1, 2.0, off[-1])
    w[off[3] + 1] = -1.0                       # set 3: a negative weight
    for v in ("1", "2", "3a", "4"):
        q, z, st = oracle.sketch_batch(v, ids, w, off, 16, seed=4)
        for s in range(len(sizes)):
            sid, sw = ids[off[s]:off[s + 1]], w[off[s]:off[s + 1]]
            code = oracle.sketch_status(v, sid, sw, 16, seed=4)
            assert st[s] == code
            if code == 0:
                qs, zs, _ = oracle.sketch(v, sid, sw, 16, seed=4)
                assert np.array_equal(z[s], zs) and np.array_equal(q[s], qs)
            else:
                assert (z[s] == 0).all() and np.isinf(q[s]).all()
        assert st[3] != 0 and st[1] == 0 and np.isinf(q[1]).all()   # bad weight; empty set
