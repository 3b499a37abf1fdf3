"""Grid mode (sets spread over every SM) and the threshold schedule, on the
GPU through the C ABI, against the CPU oracle.

The thresholds only decide how much work a call does (which points are
generated in which round); the signature is the paper's (Eq. signature_def)
whatever they are.  So every test here compares with the oracle under the
same rules as the batch tests: winning ids bit-exact except oracle near ties,
q within 1e-10 relative.
"""
import numpy as np
import pytest
import torch

from paper_1911_00675_gb300 import workloads as W
from parity_util import VARS, assert_near_tie_rate, check_sets, run, to_dev

pytestmark = pytest.mark.gpu
GRID_MIN = 40_000


@pytest.fixture(scope="module")
def H():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    return pmh.Handle(0)


@pytest.fixture
def grid(H):
    H.set_thresholds(grid_min=GRID_MIN)
    yield H
    H.set_thresholds()


def _status_ok(st):
    assert (st == 0).all(), np.unique(st)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_grid_items_match_oracle(grid, precision):
    # two grid sets (one ragged), small sets beside them, an empty set
    b = W.random_batch(31, [45_000, 3, 1000, 70_001, 0, 1], 256, "lognormal")
    z, q, st = run(grid, b, VARS, precision, seed=5)
    _status_ok(st)
    for vi, v in enumerate(VARS):
        check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=5)


@pytest.mark.parametrize("m", [2, 1024, 4096])
def test_grid_equals_oracle_large_m(grid, m):
    b = W.random_batch(32 + m, [GRID_MIN + 17], m, "pareto")
    for precision in (0, 1):
        z, q, st = run(grid, b, ["1", "2", "3a", "4"], precision, seed=1)
        _status_ok(st)
        for vi, v in enumerate(["1", "2", "3a", "4"]):
            check_sets(b, v, z[vi], q[vi], [0], seed=1)


def test_grid_finalize_rerun_when_components_stay_empty(H):
    # ln m + t_c_grid = 0.05: the grid round leaves most components empty, so the
    # last CTA redoes the item on its own with the ordinary threshold rounds
    m = 512
    H.set_thresholds(t_c_grid=0.05 - np.log(m), grid_min=GRID_MIN)
    try:
        b = W.random_batch(33, [50_000, 10], m, "uniform")
        for precision in (0, 1):
            z, q, st = run(H, b, ["1", "2", "3", "4"], precision, seed=2)
            _status_ok(st)
            for vi, v in enumerate(["1", "2", "3", "4"]):
                check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=2)
    finally:
        H.set_thresholds()


@pytest.mark.parametrize("shape", [0, 3, 1], ids=["warp", "pair", "cta8"])
@pytest.mark.parametrize("t_c,rounds", [(0.02, 5), (0.02, 0), (0.5, 1), (30.0, 5)])
def test_threshold_schedule_does_not_change_results(H, t_c, rounds, shape):
    # t_c is given as ln m + t_c: tiny first thresholds force retry rounds; rounds=0
    # goes straight to the unbounded loop of the paper's algorithms, where a team's
    # bound stays infinite until its signature is full
    m = 300
    H.set_team_shape(0, shape)
    H.set_thresholds(t_c=t_c - np.log(m), rounds=rounds, grid_min=0)
    try:
        b = W.random_batch(34, [1, 2, 7, 100, 999, 5000], m, "lognormal")
        for precision in (0, 1):
            z, q, st = run(H, b, VARS, precision, seed=9)
            _status_ok(st)
            for vi, v in enumerate(VARS):
                check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=9)
    finally:
        H.set_thresholds()
        H.set_team_shape(0, -1)


def test_more_grid_items_than_slots(H):
    # 20 sets above grid_min: 16 per family run in grid mode, the rest the usual way
    H.set_thresholds(grid_min=3_000)
    try:
        b = W.random_batch(35, [3_500] * 20 + [12], 128, "exp")
        z, q, st = run(H, b, ["1", "3a"], 1, seed=4)
        _status_ok(st)
        for vi, v in enumerate(["1", "3a"]):
            check_sets(b, v, z[vi], q[vi], range(b.num_sets), seed=4)
    finally:
        H.set_thresholds()


def test_grid_bad_and_zero_weight_sets(grid):
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(36, [GRID_MIN + 5, GRID_MIN + 6, GRID_MIN + 7, 50], 64, "uniform")
    w = b.weights.copy()
    w[b.offsets[0] + 12345] = -1.0                       # set 0: a negative weight
    w[b.offsets[1]:b.offsets[2]] = 0.0                   # set 1: all weights zero
    bb = W.Batch(b.ids, w, b.offsets, b.m)
    for precision in (0, 1):
        z, q, st = run(grid, bb, ["1", "4"], precision, seed=3)
        assert (st[:, 0] == pmh.ERR_BAD_WEIGHT).all() and (z[:, 0] == 0).all()
        assert (st[:, 1:] == 0).all()
        assert (z[:, 1] == 0).all() and np.isinf(q[:, 1]).all()       # empty signature
        for vi, v in enumerate(["1", "4"]):
            check_sets(bb, v, z[vi], q[vi], [2, 3], seed=3)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_grid_inputs_off_the_16_byte_grid(grid, precision):
    # 16-byte aligned ids and weights take the trimmed grid-mode filter (two elements per load),
    # inputs at an 8-byte offset the general one: the same signatures, q and statuses; grid sets
    # that start at an odd element, a ragged end and every variant family
    b = W.random_batch(39, [GRID_MIN + 3, 5, 2 * GRID_MIN + 1, GRID_MIN + 64], 512, "lognormal")
    ids, w, off = to_dev(b)
    ids_u = torch.empty(ids.numel() + 1, dtype=ids.dtype, device=ids.device)[1:]
    w_u = torch.empty(w.numel() + 1, dtype=w.dtype, device=w.device)[1:]
    ids_u.copy_(ids)
    w_u.copy_(w)
    assert ids.data_ptr() % 16 == 0 and w.data_ptr() % 16 == 0
    assert ids_u.data_ptr() % 16 == 8 and w_u.data_ptr() % 16 == 8
    za, qa, sa = grid.sketch_batch(ids, w, off, b.m, VARS, precision, 6, with_q=True)
    zb, qb, sb = grid.sketch_batch(ids_u, w_u, off, b.m, VARS, precision, 6, with_q=True)
    torch.cuda.synchronize()
    assert int(sa.abs().sum()) == 0
    assert torch.equal(za, zb) and torch.equal(qa, qb) and torch.equal(sa, sb)
    from paper_1911_00675_gb300 import pmh
    z, q = pmh.to_u64(za), qa.cpu().numpy()
    for vi, v in enumerate(VARS):
        check_sets(b, v, z[vi], q[vi], [0, 2, 3], seed=6)


def test_grid_counters_count_every_element_once(grid):
    # the grid pass counts each element with w > 0 once per variant (a zero weight not at all),
    # and the elements it rejected without a logarithm among them
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(40, [GRID_MIN + 11, 2 * GRID_MIN + 3], 256, "lognormal")
    w = b.weights.copy()
    w[b.offsets[0] + 5] = 0.0
    w[b.offsets[1] + 7] = 0.0
    bb = W.Batch(b.ids, w, b.offsets, b.m)
    cnt = torch.zeros(len(pmh.COUNTERS), dtype=torch.int64, device="cuda")
    z, q, st = run(grid, bb, ["1", "3a"], 1, seed=2, counters=cnt)
    _status_ok(st)
    c = dict(zip(pmh.COUNTERS, cnt.cpu().tolist()))
    npos = int((w > 0).sum())
    assert c["rounds"] > 0 or c["elements"] == 2 * npos
    assert 0 < c["prefiltered"] < c["elements"] and c["points32"] > 0
    for vi, v in enumerate(["1", "3a"]):
        check_sets(bb, v, z[vi], q[vi], [0, 1], seed=2)


def test_launch_count_reported(H):
    b = W.random_batch(37, [10, 20], 64, "uniform")
    H.set_thresholds(grid_min=0)
    run(H, b, ["1", "2", "3", "4"], 1)
    # queue (3) + statistics (2) + prefilter pass (2: set selection, hashing) + per family one
    # sketch kernel and one FP64 redo kernel
    assert H.last_launches() == 5 + 2 + 4 + 4
    run(H, b, ["1", "2", "3", "4"], 0)
    assert H.last_launches() == 5 + 2 + 4                 # FP64 calls have no redo kernels
    H.set_prefilter(0.0)
    run(H, b, ["1", "2", "3", "4"], 0)
    assert H.last_launches() == 5 + 4                     # no prefilter pass
    H.set_prefilter()
    H.set_thresholds()
    run(H, b, ["1", "3a"], 1)
    assert H.last_launches() == 5 + 2 + 2 + 2 + 1 + 2     # + grid reset + one grid kernel per family


@pytest.mark.slow
@pytest.mark.parametrize("precision", [1, 0], ids=["fp32", "fp64"])
def test_c5_full_size(H, precision):
    # one set of 1e8 elements, lognormal(0, 2) weights, m = 4096, ProbMinHash3a: every component
    H.set_thresholds()
    b = W.batch_c5()
    z, q, st = run(H, b, ["3a"], precision, seed=0)
    _status_ok(st)
    stats = {"near": 0, "components": 0}
    check_sets(b, "3a", z[0], q[0], [0], seed=0, stats=stats, scan=True)
    assert_near_tie_rate(stats, f"c5 ({'fp32' if precision else 'fp64'}, one set of 1e8, m=4096)")


def test_profiling_history_records_each_call(H):
    b = W.random_batch(38, [100, 2000, 5], 64, "uniform")
    H.set_profiling(True)
    try:
        for _ in range(5):
            run(H, b, ["1", "3"], 1)
        q, k = H.kernel_ms_history(8)
        assert len(q) == 5 and len(k) == 5
        assert all(x > 0 for x in k) and all(x >= 0 for x in q)
        q1, k1 = H.last_kernel_ms()
        assert k1 == k[-1] and q1 == q[-1]
    finally:
        H.set_profiling(False)
    run(H, b, ["1"], 1)
    from paper_1911_00675_gb300 import pmh
    with pytest.raises(pmh.PmhError):
        H.last_kernel_ms()
