"""pmh_sketch_batch_host: the sketch of a batch held in host memory, copied, sketched and copied
back in a chunked pipeline.  Results must equal the device entry point's bit for bit (the same
kernels on the same inputs), and those are checked against the oracle in test_sketch_gpu.py; a
sample of sets is checked against the oracle here as well."""
import numpy as np
import pytest
import torch

from paper_1911_00675_gb300 import workloads as W
from parity_util import check_sets, run

pytestmark = pytest.mark.gpu
VARS = ["1", "2", "3a", "4"]


@pytest.fixture(scope="module")
def H():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    return pmh.Handle(0)


def _host(b, pin=True):
    ids = torch.from_numpy(b.ids.view(np.int64).copy())
    w = torch.from_numpy(b.weights.copy())
    off = torch.from_numpy(b.offsets.copy())
    if pin:
        ids, w, off = ids.pin_memory(), w.pin_memory(), off.pin_memory()
    return ids, w, off


@pytest.mark.parametrize("chunks", [1, 3, 0])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_host_path_equals_device_path(H, chunks, precision):
    from paper_1911_00675_gb300 import pmh
    sizes = np.floor(10 ** (4 * np.random.default_rng(chunks).random(300))).astype(np.int64)
    b = W.random_batch(60 + chunks, sizes, 256, "uniform")
    zd, qd, sd = run(H, b, VARS, precision, with_q=True, seed=8)
    z, q, st = H.sketch_batch_host(*_host(b), 256, VARS, precision, 8, with_q=True, chunks=chunks)
    assert np.array_equal(pmh.to_u64(z), zd)
    assert np.array_equal(q.numpy(), qd)
    assert np.array_equal(st.numpy(), sd) and (st.numpy() == 0).all()
    check_sets(b, "3a", pmh.to_u64(z)[2], q.numpy()[2], [0, 7, 150, 299], seed=8)


def test_host_path_pageable_and_offset_start(H):
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(70, [10, 0, 500, 3, 2000], 64, "pareto")
    # offsets not starting at 0: the elements before offsets[0] are never read as set members
    ids, w, off = _host(b, pin=False)
    pad_ids = torch.cat([torch.zeros(5, dtype=torch.int64), ids])
    pad_w = torch.cat([torch.full((5,), -1.0, dtype=torch.float64), w])    # would be a bad weight if read
    z, q, st = H.sketch_batch_host(pad_ids, pad_w, off + 5, 64, ["1", "4"], 1, 2, with_q=True, chunks=2)
    assert (st.numpy() == 0).all()
    for vi, v in enumerate(["1", "4"]):
        check_sets(b, v, pmh.to_u64(z)[vi], q.numpy()[vi], range(b.num_sets), seed=2)


def test_host_path_rejects_decreasing_offsets(H):
    from paper_1911_00675_gb300 import pmh
    b = W.random_batch(71, [10, 20, 30], 32, "uniform")
    ids, w, off = _host(b, pin=False)
    off = off.clone()
    off[2] = 5
    with pytest.raises(pmh.PmhError) as ei:
        H.sketch_batch_host(ids, w, off, 32, ["1"], 1, 0)
    assert ei.value.code == pmh.ERR_INVALID_ARG
