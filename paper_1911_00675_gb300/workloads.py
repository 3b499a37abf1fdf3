"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws inputs: 64-bit element ids, FP64 weights and CSR
offsets.  It holds none of the sketching arithmetic, so both the CUDA path's
tests/benchmarks and the CPU oracle's tests can use it.

The paper evaluates on synthetic sets of random 64-bit integers (Sec.
Experiments): "sets of randomly generated 64-bit integers".  Ids here are
distinct by construction: id = B(counter) with B a fixed 64-bit bijection
(odd multiplications and xor-shifts), so no two elements of a batch collide.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_M1 = np.uint64(0xD1342543DE82EF95)
_M2 = np.uint64(0xAF251AF3B0F025B5)


def distinct_ids(start: int, count: int, salt: int) -> np.ndarray:
    """`count` distinct uniform-looking uint64 ids (a bijection of start..start+count-1)."""
    x = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x ^= np.uint64(salt & 0xFFFFFFFFFFFFFFFF)
        x *= _M1
        x ^= x >> np.uint64(32)
        x *= _M2
        x ^= x >> np.uint64(29)
    return x


@dataclass
class Batch:
    """CSR batch of weighted sets: set s owns ids[offsets[s]:offsets[s+1]]."""
    ids: np.ndarray          # uint64[N]
    weights: np.ndarray      # float64[N]
    offsets: np.ndarray      # int64[S+1]
    m: int
    variants: tuple = ("1",)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def num_sets(self) -> int:
        return len(self.offsets) - 1

    @property
    def num_elements(self) -> int:
        return int(self.offsets[-1])

    def set(self, s: int):
        b, e = int(self.offsets[s]), int(self.offsets[s + 1])
        return self.ids[b:e], self.weights[b:e]


def _offsets(sizes: np.ndarray) -> np.ndarray:
    off = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=off[1:])
    return off


def batch_c1(seed: int = 0xC0FFEE01, num_sets: int = 1000, n: int = 1000, m: int = 256) -> Batch:
    """1,000 sets of n=1,000 distinct ids, weights Exp(1) normalised to sum 1 per set; m=256."""
    rng = np.random.default_rng(seed)
    sizes = np.full(num_sets, n, dtype=np.int64)
    off = _offsets(sizes)
    ids = distinct_ids(0, int(off[-1]), seed)
    w = rng.exponential(1.0, size=int(off[-1]))
    sums = np.add.reduceat(w, off[:-1]) if num_sets else np.zeros(0)
    w /= np.repeat(sums, sizes)
    return Batch(ids, w, off, m, ("1", "3"), "c1: 1000 sets n=1000 Exp(1)-normalised m=256")


def batch_c2(seed: int = 0xC0FFEE02, num_sets: int = 20000, n_max: float = 1e5, m: int = 1024) -> Batch:
    """20,000 sets, n = floor(10^(5U)) log-uniform over [1, 1e5], weights Uniform(0,1]; m=1024, six variants."""
    rng = np.random.default_rng(seed)
    u = rng.random(num_sets)
    sizes = np.floor(np.power(n_max, u)).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    off = _offsets(sizes)
    ids = distinct_ids(0, int(off[-1]), seed)
    w = 1.0 - rng.random(int(off[-1]))     # (0, 1]
    return Batch(ids, w, off, m, ("1", "1a", "2", "3", "3a", "4"),
                 f"c2: {num_sets} sets n log-uniform [1,{int(n_max)}] Uniform(0,1] m={m}")


def batch_c3(seed: int = 0xC0FFEE03, num_sets: int = 10000, n: int = 10000, m: int = 4096,
             tail: float = 1.5) -> Batch:
    """10,000 sets of n=10,000, weights Pareto(x_m=1, tail 1.5): w = U^(-1/1.5), U in (0,1]; m=4096."""
    rng = np.random.default_rng(seed)
    sizes = np.full(num_sets, n, dtype=np.int64)
    off = _offsets(sizes)
    ids = distinct_ids(0, int(off[-1]), seed)
    u = 1.0 - rng.random(int(off[-1]))
    w = np.power(u, -1.0 / tail)
    return Batch(ids, w, off, m, ("2", "4"), f"c3: {num_sets} sets n={n} Pareto({tail}) m={m}")


def batch_c4_sets(seed: int = 0xC0FFEE04, num_base: int = 512, n: int = 5000, variants_per_base: int = 32,
                  m: int = 1024) -> Batch:
    """512 base sets (n=5,000, Exp(1) weights), each perturbed into 32 variants v: every element is
    dropped with probability v/40 and surviving weights are multiplied by exp(sigma_v * N(0,1)),
    sigma_v = v/16.  Sketched with ProbMinHash3a at m=1024 for all-pairs estimation."""
    rng = np.random.default_rng(seed)
    base_ids = distinct_ids(0, num_base * n, seed).reshape(num_base, n)
    base_w = rng.exponential(1.0, size=(num_base, n))
    ids_l, w_l, sizes = [], [], []
    for b in range(num_base):
        for v in range(variants_per_base):
            keep = rng.random(n) >= v / 40.0
            jitter = np.exp((v / 16.0) * rng.standard_normal(n))
            ids_l.append(base_ids[b][keep])
            w_l.append((base_w[b] * jitter)[keep])
            sizes.append(int(keep.sum()))
    off = _offsets(np.array(sizes, dtype=np.int64))
    return Batch(np.concatenate(ids_l), np.concatenate(w_l), off, m, ("3a",),
                 f"c4: {num_base}x{variants_per_base} perturbed sets n={n} m={m}")


def batch_c5(seed: int = 0xC0FFEE05, n: int = 100_000_000, m: int = 4096, sigma: float = 2.0) -> Batch:
    """One set of n=1e8 distinct ids, weights lognormal(0, 2); m=4096, ProbMinHash3a."""
    rng = np.random.default_rng(seed)
    ids = distinct_ids(0, n, seed)
    w = rng.lognormal(0.0, sigma, size=n)
    return Batch(ids, w, np.array([0, n], dtype=np.int64), m, ("3a",), f"c5: one set n={n} lognormal(0,{sigma}) m={m}")


def random_batch(seed: int, sizes, m: int, weight: str = "uniform", variants=("1",)) -> Batch:
    """Small CSR batch with the given set sizes (tests)."""
    rng = np.random.default_rng(seed)
    sizes = np.asarray(sizes, dtype=np.int64)
    off = _offsets(sizes)
    total = int(off[-1])
    ids = distinct_ids(int(rng.integers(0, 2**40)), total, seed)
    if weight == "uniform":
        w = 1.0 - rng.random(total)
    elif weight == "exp":
        w = rng.exponential(1.0, size=total)
    elif weight == "pareto":
        w = np.power(1.0 - rng.random(total), -1.0 / 1.5)
    elif weight == "lognormal":
        w = rng.lognormal(0.0, 2.0, size=total)
    elif weight == "unit":
        w = np.ones(total)
    else:
        raise ValueError(weight)
    return Batch(ids, w, off, m, tuple(variants), f"random sizes={list(sizes[:8])}... weight={weight}")


def pair_from_weight_pairs(rng: np.random.Generator, pairs, salt: int = 0):
    """Two weighted sets whose union has exactly the given (w_A, w_B) weight pairs (Sec. Verification):
    one fresh random element per pair, added to A if w_A > 0 and to B if w_B > 0."""
    pairs = np.asarray(pairs, dtype=np.float64).reshape(-1, 2)
    ids = distinct_ids(int(rng.integers(0, 2**62)), len(pairs), salt)
    a = pairs[:, 0] > 0
    b = pairs[:, 1] > 0
    return ids[a], pairs[a, 0], ids[b], pairs[b, 1]


def constructed_pair(rng: np.random.Generator, target_jp: float, n_total: int = 1000, salt: int = 0):
    """A pair from the family: shared part S with w_B = c*w_A on S, extra A-only elements of total mass
    a and B-only elements of total mass b.  Their J_P has a closed form in (W_S, a, b, c), returned
    as `params`; the mass split is chosen so that J_P is near `target_jp`.
    Returns (ids_a, w_a, ids_b, w_b, params)."""
    c = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
    j = float(min(max(target_jp, 0.0), 1.0))
    n_s = min(max(int(round(j * n_total)), 1), n_total) if j > 0 else 0
    n_rest = n_total - n_s
    n_a = n_rest // 2
    n_b = n_rest - n_a
    ids = distinct_ids(int(rng.integers(0, 2**62)), n_s + n_a + n_b, salt)
    ws = rng.exponential(1.0, size=n_s)
    w_s = float(ws.sum())
    rest = 1.0 if j <= 0.0 else (0.0 if j >= 1.0 else w_s * (1.0 / j - 1.0))   # = a + b/c
    f = rng.uniform(0.2, 0.8)
    if n_a and n_b:
        a, b = f * rest, (1.0 - f) * rest * c
    elif n_b:
        a, b = 0.0, rest * c
    elif n_a:
        a, b = rest, 0.0
    else:
        a, b = 0.0, 0.0
    wa_only = rng.exponential(1.0, size=n_a)
    wb_only = rng.exponential(1.0, size=n_b)
    if n_a:
        wa_only *= a / wa_only.sum()
    if n_b:
        wb_only *= b / wb_only.sum()
    ids_s, ids_a, ids_b = ids[:n_s], ids[n_s:n_s + n_a], ids[n_s + n_a:]
    a_ids = np.concatenate([ids_s, ids_a])
    a_w = np.concatenate([ws, wa_only])
    b_ids = np.concatenate([ids_s, ids_b])
    b_w = np.concatenate([c * ws, wb_only])
    ka, kb = a_w > 0, b_w > 0
    params = dict(w_s=w_s, a=float(wa_only.sum()), b=float(wb_only.sum()), c=c)
    return a_ids[ka], a_w[ka], b_ids[kb], b_w[kb], params
