"""The allocation-free batch sketch against the allocating one.

Some callers cannot allocate GPU memory: they run under another runtime's
fixed memory budget, or inside a framework that forbids cudaMalloc on its hot
path.  pmh_sketch_batch_noalloc serves them from one fixed device array that
the library holds while it is loaded.  Its results must equal those of
pmh_sketch_batch (same kernels, same tables) on consecutive calls that reuse
the array, with the tolerances of the other GPU tests: ids bit-exact, q within
1e-10 relative.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
VARS = ["1", "1a", "2", "3", "3a", "4"]


def _dev(b):
    dev = torch.device("cuda", 0)
    return (torch.from_numpy(b.ids.view(np.int64).copy()).to(dev), torch.from_numpy(b.weights.copy()).to(dev),
            torch.from_numpy(b.offsets.copy()).to(dev))


def _same(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    fa, fb = np.isfinite(a), np.isfinite(b)
    assert np.array_equal(fa, fb)
    np.testing.assert_allclose(a[fa], b[fb], rtol=1e-10, atol=0)


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls():
    # m alternates 256 -> 33 -> 256 (the shared array's tables change between calls), and the
    # first batch holds a set of 300,000 elements, whose weight statistics are split over all
    # blocks (the path for sets above 262,144 elements)
    from paper_1911_00675_gb300 import build, pmh
    from paper_1911_00675_gb300 import workloads as W
    build.build()
    h = pmh.Handle(0)
    cases = ((256, [0, 1, 3, 64, 700, 5000, 300000], "pareto"), (33, [2, 40, 1000], "lognormal"),
             (256, [5, 90, 2500], "uniform"))
    for m, sizes, weight in cases:
        b = W.random_batch(4242 + m + len(sizes), sizes, m, weight)
        ids, w, off = _dev(b)
        for prec in (pmh.FP32_RECHECK, pmh.FP64):
            z_ref, q_ref, st_ref = h.sketch_batch(ids, w, off, m, VARS, prec, seed=7, with_q=True)
            torch.cuda.synchronize()
            assert int(st_ref.abs().sum()) == 0
            for _ in range(2):   # the second call reuses the array left by the first
                z, q, st = pmh.sketch_batch_noalloc(ids, w, off, m, VARS, prec, seed=7, with_q=True)
                torch.cuda.synchronize()
                assert torch.equal(st, st_ref)
                assert torch.equal(z, z_ref)
                _same(q, q_ref)
    h.close()


def test_noalloc_call_allocates_no_device_memory():
    # With the outputs passed in, a call changes neither the device's free memory nor PyTorch's
    # allocations.  The first call may load kernel code, so the memory is read after it.
    from paper_1911_00675_gb300 import build, pmh
    from paper_1911_00675_gb300 import workloads as W
    build.build()
    b = W.random_batch(77, [3, 300, 4000, 20000], 512, "uniform")
    ids, w, off = _dev(b)
    z = torch.empty((len(VARS), b.num_sets, b.m), dtype=torch.int64, device="cuda")
    q = torch.empty(z.shape, dtype=torch.float64, device="cuda")
    st = torch.empty((len(VARS), b.num_sets), dtype=torch.int32, device="cuda")
    pmh.sketch_batch_noalloc(ids, w, off, b.m, VARS, pmh.FP32_RECHECK, seed=1, out_ids=z, out_q=q, status=st)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        pmh.sketch_batch_noalloc(ids, w, off, b.m, VARS, pmh.FP32_RECHECK, seed=1, out_ids=z, out_q=q, status=st)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0
    assert int(st.abs().sum()) == 0


def test_noalloc_rejects_batches_beyond_its_limit():
    from paper_1911_00675_gb300 import pmh
    dev = torch.device("cuda", 0)
    n_sets = 65536 + 1                     # PMH_NOALLOC_MAX_SETS + 1
    off = torch.zeros(n_sets + 1, dtype=torch.int64, device=dev)
    ids = torch.zeros(1, dtype=torch.int64, device=dev)
    w = torch.ones(1, dtype=torch.float64, device=dev)
    with pytest.raises(pmh.PmhError) as err:
        pmh.sketch_batch_noalloc(ids, w, off, 64, ["1"], pmh.FP32_RECHECK)
    assert err.value.code == pmh.ERR_UNSUPPORTED
    assert "limit" in str(err.value)


def test_noalloc_refuses_a_stream_being_captured():
    # The tables are staged through a host buffer that later calls rewrite, so a captured call
    # could replay with another call's tables: the entry point refuses while its stream captures.
    from paper_1911_00675_gb300 import pmh
    from paper_1911_00675_gb300 import workloads as W
    b = W.random_batch(78, [10, 20], 64, "uniform")
    ids, w, off = _dev(b)
    z = torch.empty((1, b.num_sets, b.m), dtype=torch.int64, device="cuda")
    st = torch.empty((1, b.num_sets), dtype=torch.int32, device="cuda")
    pmh.sketch_batch_noalloc(ids, w, off, b.m, ["1"], pmh.FP32_RECHECK, out_ids=z, status=st)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(g, stream=side):
        try:
            pmh.sketch_batch_noalloc(ids, w, off, b.m, ["1"], pmh.FP32_RECHECK, out_ids=z, status=st, stream=side)
        except pmh.PmhError as e:
            err = e
        z.add_(0)   # the captured graph is not empty
    assert err is not None and err.code == pmh.ERR_UNSUPPORTED
    torch.cuda.synchronize()
