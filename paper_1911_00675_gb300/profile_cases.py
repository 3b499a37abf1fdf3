"""Small, self-contained cases of every kernel of libpmh, for profilers (ncu).

    python -m paper_1911_00675_gb300.profile_cases CASE [REPS]

Each case builds its inputs (seeded, synthetic), runs the call REPS times (default 2) on cuda:0
and checks the statuses; a profiler then captures the launches of one repetition.  Team shapes
are pinned and autotuning is off, so every repetition launches the same kernels.

Cases (kernels launched per repetition):
  fp32      c2-shaped batch of 2,000 sets, six variants, FP32 + recheck: queue build, statistics,
            four family sketch kernels, each followed by its (empty) FP64 redo kernel
  fp64      the same batch with PMH_FP64: four family sketch kernels
  rej       the same batch, ProbMinHash3/3a/4 with the rejection sampler for Exp(lambda;0,1)
  grid      one set of 1e7 elements (lognormal(0, 2) weights), m = 4096, ProbMinHash3a, FP32:
            split statistics and the grid-mode kernel
  grid64    the same with PMH_FP64
  allpairs  all-pairs counts of 16,384 signatures of m = 1024 (upper triangle)
  bbit      8-bit reduction of the same signatures and their all-pairs counts
  pairs     counts of 1e6 listed pairs of the same signatures
  merge     merge of 128 partial signatures of m = 131,072
  pminhash  P-MinHash of 2,000 sets of n = 1,000 at m = 1024
  status    status reduction of 1e7 items
"""
from __future__ import annotations

import sys


def main(argv=None) -> int:
    import numpy as np
    import torch

    from . import build, pmh
    from . import workloads as W

    argv = sys.argv[1:] if argv is None else argv
    case = argv[0]
    reps = int(argv[1]) if len(argv) > 1 else 2
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    h = pmh.Handle(0)
    h.set_autotune(0)

    def up(b):
        return (torch.from_numpy(b.ids.view(np.int64)).to(dev), torch.from_numpy(b.weights).to(dev),
                torch.from_numpy(b.offsets).to(dev))

    def check(st):
        torch.cuda.synchronize()
        if int((st != 0).sum()) != 0:
            raise RuntimeError(f"{case}: a status is not PMH_OK")

    if case in ("fp32", "fp64", "rej"):
        b = W.batch_c2(num_sets=2000)
        ids, w, off = up(b)
        variants = ["1", "1a", "2", "3", "3a", "4"]
        if case == "fp64":
            shapes = ((1, 3), (2, 5), (3, 3), (4, 3))
            prec = pmh.FP64
        else:
            shapes = ((1, 3), (2, 4), (3, 3), (4, 4))
            prec = pmh.FP32_RECHECK
        if case == "rej":
            variants = ["3", "3a", "4"]
            h.set_te_sampler(pmh.TE_REJECTION)
        for f, s in shapes:
            h.set_team_shape(f, s)
        out = torch.empty((len(variants), b.num_sets, b.m), dtype=torch.int64, device=dev)
        st = torch.empty((len(variants), b.num_sets), dtype=torch.int32, device=dev)
        for _ in range(reps):
            h.sketch_batch(ids, w, off, b.m, variants, prec, 0, out_ids=out, status=st)
        check(st)
    elif case in ("grid", "grid64"):
        b = W.batch_c5(n=10_000_000)
        ids, w, off = up(b)
        out = torch.empty((1, 1, 4096), dtype=torch.int64, device=dev)
        st = torch.empty((1, 1), dtype=torch.int32, device=dev)
        prec = pmh.FP64 if case == "grid64" else pmh.FP32_RECHECK
        for _ in range(reps):
            h.sketch_batch(ids, w, off, 4096, ["3a"], prec, 0, out_ids=out, status=st)
        check(st)
    elif case in ("allpairs", "bbit", "pairs"):
        g = torch.Generator(device="cpu").manual_seed(7)
        sigs = torch.randint(0, 1 << 20, (16384, 1024), generator=g, dtype=torch.int64).to(dev)
        counts = torch.empty((16384, 16384), dtype=torch.int16, device=dev)
        if case == "allpairs":
            for _ in range(reps):
                h.estimate_jp(sigs, upper_only=True, counts=counts)
        elif case == "bbit":
            packed = h.bbit_reduce(sigs, 8, seed=1)
            for _ in range(reps):
                h.bbit_reduce(sigs, 8, seed=1, packed=packed)
                h.bbit_allpairs(packed, 1024, 8, upper_only=True, counts=counts)
        else:
            pa = torch.randint(0, 16384, (1_000_000,), generator=g, dtype=torch.int64).to(dev)
            pb = torch.randint(0, 16384, (1_000_000,), generator=g, dtype=torch.int64).to(dev)
            for _ in range(reps):
                h.estimate_pairs(sigs, sigs, pa, pb)
        torch.cuda.synchronize()
    elif case == "merge":
        g = torch.Generator(device="cpu").manual_seed(8)
        q = torch.rand((128, 131072), generator=g, dtype=torch.float64).to(dev)
        z = torch.randint(0, 1 << 40, (128, 131072), generator=g, dtype=torch.int64).to(dev)
        oq = torch.empty(131072, dtype=torch.float64, device=dev)
        oz = torch.empty(131072, dtype=torch.int64, device=dev)
        for _ in range(reps):
            h.merge(q, z, out_q=oq, out_z=oz)
        torch.cuda.synchronize()
    elif case == "pminhash":
        b = W.random_batch(9, [1000] * 2000, 1024, "uniform")
        ids, w, off = up(b)
        for _ in range(reps):
            _, _, st = h.pminhash_batch(ids, w, off, 1024, 0)
        check(st)
    elif case == "status":
        st = torch.zeros(10_000_000, dtype=torch.int32, device=dev)
        for _ in range(reps):
            rc, counts, first = h.sync_status(st)
            if rc != pmh.OK or counts[0] != st.numel() or first != -1:
                raise RuntimeError("status reduction disagrees")
    else:
        raise SystemExit(f"unknown case {case!r}; see the module docstring")
    h.close()
    print(case, "ok")
    return 0


if __name__ == "__main__":
    sys.exit(main())
