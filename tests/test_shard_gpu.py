"""The sharded huge-set path on one GPU: k element-range shards emulated in sequence, partial
signatures gathered, merged by pmh_merge; the result equals the oracle's whole-set signature
(Eq. signature_def over a disjoint union) under the batch parity rules."""
import numpy as np
import pytest
import torch

from paper_1911_00675_gb300 import shard
from paper_1911_00675_gb300 import workloads as W
from parity_util import check_sets

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_1911_00675_gb300 import build, pmh
    build.build()
    return pmh.Handle(0)


@pytest.mark.parametrize("variant,prec", [("1", 1), ("2", 0), ("3a", 1), ("4", 1)])
def test_sketch_set_sharded_emulated_ranks(H, variant, prec):
    from paper_1911_00675_gb300 import pmh
    world, m = 4, 512
    b = W.random_batch(41, [20_000], m, "lognormal")
    ids, w = b.set(0)
    eb = shard.partition_elements(len(ids), world)
    dev = torch.device("cuda", 0)
    parts = [(torch.from_numpy(ids[eb[r]:eb[r + 1]].view(np.int64).copy()).to(dev),
              torch.from_numpy(w[eb[r]:eb[r + 1]].copy()).to(dev)) for r in range(world)]
    partials = []
    for pid, pw in parts:
        off = torch.tensor([0, pid.numel()], dtype=torch.int64, device=dev)
        z, q, st = H.sketch_batch(pid, pw, off, m, [variant], prec, 3, with_q=True)
        assert int(st.abs().max()) == 0
        partials.append((q[0, 0], z[0, 0]))
    Q = torch.stack([p[0] for p in partials])
    Z = torch.stack([p[1] for p in partials])
    for r in range(world):   # every emulated rank sees the same gathered partials
        qm, zm = shard.sketch_set_sharded(H, *parts[r], m, variant, prec, 3, gather=lambda q, z, g: (Q, Z))
        torch.cuda.synchronize()
        zn = pmh.to_u64(zm.unsqueeze(0))
        check_sets(b, variant, zn, qm.unsqueeze(0).cpu().numpy(), [0], seed=3)
