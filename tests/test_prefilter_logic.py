"""The prefilter pass's test is looser than every variant's own first-point test (host check of
the FP32 arithmetic both sides use; no GPU).

A variant's filter keeps an element unless  fl(fl(u * te) * (1 - 16 ulp)) > fl(b * ws),  with u
the 23-bit lower bound of U, te the family's lower-bound factor (1 for Exp(1), (1 - e^-lambda) /
lambda for Exp(lambda;0,1)), b the team's current bound and ws the scaled weight.  The prefilter
pass applies the same test with the smallest factor of any family and with the first round's
bound t_s, which every later bound of that round only undercuts.  Correctly rounded products are
monotone in each factor, so whatever a variant keeps, the pass keeps too; these cases check that
with float32 arithmetic rounded like the kernels' __fmul_rn, including bounds and products one
ulp apart.
"""
import numpy as np

F = np.float32
SLACK = F(1.0) - F(16.0) * F(2.0 ** -24)


def keeps(u, te, b, ws):
    return ~((u * te) * SLACK > b * ws)


def test_prefilter_keeps_a_superset_of_every_variant():
    rng = np.random.default_rng(7)
    n = 2_000_000
    # u: 23-bit uniforms as the kernels form them (1.f with 23 random mantissa bits, minus 1)
    u = (np.uint32(0x3F800000) | rng.integers(0, 1 << 23, n, dtype=np.uint32)).view(F) - F(1.0)
    ws = rng.uniform(0.5, 2.0, n).astype(F) * F(2.0) ** rng.integers(-20, 20, n).astype(F)
    t_s = rng.uniform(1.0, 2.0, n).astype(F)
    # a later bound of the round: at most t_s, often within a few ulp of it
    shrink = np.where(rng.random(n) < 0.5, rng.uniform(0.2, 1.0, n),
                      1.0 - rng.integers(0, 4, n) * 2.0 ** -24).astype(F)
    b = np.minimum(t_s * shrink, t_s)
    for m in (2, 3, 64, 1024, 8192):
        lam = np.log1p(1.0 / (m - 1))
        te_lo = F(-np.expm1(-lam) / lam)       # the correlated families' factor, rounded to FP32
        if float(te_lo) > -np.expm1(-lam) / lam:
            te_lo = np.nextafter(te_lo, F(0))   # rounded down, as the tables do
        pre = keeps(u, te_lo, t_s, ws)
        for te in (F(1.0), te_lo):              # Exp(1) families and Exp(lambda;0,1) families
            fam = keeps(u, te, b, ws)
            assert not (fam & ~pre).any(), f"m={m}: a variant keeps an element the prefilter rejects"
        # the pass does reject: it is a filter, not a pass-through
        assert (~pre).any()


def test_equal_bounds_and_factors_keep_the_same_elements():
    rng = np.random.default_rng(8)
    n = 200_000
    u = (np.uint32(0x3F800000) | rng.integers(0, 1 << 23, n, dtype=np.uint32)).view(F) - F(1.0)
    ws = rng.uniform(0.01, 3.0, n).astype(F)
    t_s = F(1.5)
    te = F(0.9995)
    assert np.array_equal(keeps(u, te, t_s, ws), keeps(u, te, t_s, ws))
    # one ulp more bound never rejects an element that the smaller bound keeps
    assert not (keeps(u, te, t_s, ws) & ~keeps(u, te, np.nextafter(t_s, F(2)), ws)).any()
