"""Batched EMD solve (independent problems of mixed sizes in one CUDA graph
per chunk) through the C ABI.

* Against the FP64 oracle: a mixed batch (33^2 on the dense path, 64^2 to
  512^2 on the fast transforms) run for a fixed number of iterations; every
  problem's m and p element by element and its P and D against the oracle's
  run of the same length (section 3.2 iteration, zero start), with the bars of
  the one-problem EMD tests: P 1e-5 and D 1e-4 relative, m 1e-3 relative L2,
  p 3e-4 absolute.
* Against the one-at-a-time solve: same kernels in the same order, so the
  same iterates bit for bit, and each problem stops at its own tolerance.
"""
import numpy as np
import pytest
import torch

from oracle import gprox_oracle as O
from paper_1805_09453_gb300 import synth
from tests.gpu_common import rel_l2

pytestmark = pytest.mark.gpu


def test_batched_matches_oracle_on_a_mixed_batch():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    h = gprox.Handle(0)
    sizes = [33, 256, 512, 64, 128]
    iters = 40
    pairs = [synth.gaussian_mixture_pair(N, 200 + b) for b, N in enumerate(sizes)]
    f0s = [torch.from_numpy(a).cuda() for a, _ in pairs]
    f1s = [torch.from_numpy(b).cuda() for _, b in pairs]
    ms = [torch.full((2, N, N), float("nan"), device="cuda") for N in sizes]
    ps = [torch.full((2, N, N), float("nan"), device="cuda") for N in sizes]
    opts = gprox.default_opts(max_iters=iters, tol_rel_gap=0.0, gap_every=20)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        st, reps = gprox.emd_solve_batched(h, f0s, f1s, ms, opts, ps=ps)
        stream.synchronize()
    assert st == gprox.GP_OK
    for b, N in enumerate(sizes):
        f0, f1 = pairs[b]
        ref = O.emd_solve(f0, f1, n_iters=iters)
        assert reps[b]["iters"] == iters
        assert abs(reps[b]["primal"] - ref["primal"]) < 1e-5 * ref["primal"], (N, reps[b], ref["primal"])
        assert abs(reps[b]["dual"] - ref["dual"]) < 1e-4 * abs(ref["dual"]), (N, reps[b], ref["dual"])
        m = ms[b].cpu().numpy()
        p = ps[b].cpu().numpy()
        assert rel_l2(m, np.stack([ref["mx"], ref["my"]])) < 1e-3, N
        assert np.abs(p[0] - ref["px"]).max() < 3e-4 and np.abs(p[1] - ref["py"]).max() < 3e-4, N
    h.close()


def test_batched_equals_individual_solves():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    h = gprox.Handle(0)
    sizes = [64, 32, 128, 33, 64, 256]
    pairs = [synth.gaussian_mixture_pair(N, 100 + b) for b, N in enumerate(sizes)]
    f0s = [torch.from_numpy(a).cuda() for a, _ in pairs]
    f1s = [torch.from_numpy(b).cuda() for _, b in pairs]
    ms = [torch.empty((2, N, N), device="cuda") for N in sizes]
    ps = [torch.empty((2, N, N), device="cuda") for N in sizes]
    opts = gprox.default_opts(max_iters=3000, tol_rel_gap=1e-4)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        st, reps = gprox.emd_solve_batched(h, f0s, f1s, ms, opts, ps=ps)
        stream.synchronize()
        assert st in (gprox.GP_OK, gprox.GP_ERR_MAXITER)
        for b, N in enumerate(sizes):
            m1 = torch.empty((2, N, N), device="cuda")
            p1 = torch.empty((2, N, N), device="cuda")
            st1, rep1 = gprox.emd_solve(h, f0s[b], f1s[b], m1, p1, opts=opts)
            stream.synchronize()
            assert reps[b]["iters"] == rep1["iters"], (b, reps[b], rep1)
            assert reps[b]["status"] == st1
            assert abs(reps[b]["primal"] - rep1["primal"]) <= 1e-12 * abs(rep1["primal"])
            assert torch.equal(ms[b], m1)
            assert torch.equal(ps[b], p1)
    # problems stop independently: not all at the same iteration count
    assert len({r["iters"] for r in reps}) > 1
    h.close()


def test_batched_split_bf16_equals_individual_and_oracle():
    """The batched solve with the split-precision (BF16 tensor-core) transform:
    each problem equals its one-at-a-time solve bit for bit (the branches
    share no scratch) and sits within the split mode's bars of the FP64
    oracle after a fixed number of iterations (m 1e-3 relative L2, P 1e-4)."""
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    h = gprox.Handle(0)
    sizes, iters = [128, 256, 128], 60
    pairs = [synth.gaussian_mixture_pair(N, 300 + b) for b, N in enumerate(sizes)]
    f0s = [torch.from_numpy(a).cuda() for a, _ in pairs]
    f1s = [torch.from_numpy(b).cuda() for _, b in pairs]
    ms = [torch.empty((2, N, N), device="cuda") for N in sizes]
    opts = gprox.default_opts(max_iters=iters, tol_rel_gap=0.0, gap_every=20, prec="split_bf16")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        st, reps = gprox.emd_solve_batched(h, f0s, f1s, ms, opts)
        stream.synchronize()
        h.check(st)
        for b, N in enumerate(sizes):
            m1 = torch.empty((2, N, N), device="cuda")
            h.check(gprox.emd_solve(h, f0s[b], f1s[b], m1, None, opts=opts)[0])
            stream.synchronize()
            assert torch.equal(ms[b], m1)
            ref = O.emd_solve(pairs[b][0], pairs[b][1], n_iters=iters)
            assert rel_l2(ms[b].cpu().numpy(), np.stack([ref["mx"], ref["my"]])) < 1e-3
            assert abs(reps[b]["primal"] - ref["primal"]) < 1e-4 * ref["primal"]
    o16 = gprox.default_opts(max_iters=10, tol_rel_gap=0.0, prec="split_fp16")
    with torch.cuda.stream(stream):
        st, _ = gprox.emd_solve_batched(h, f0s, f1s, ms, o16)
    assert st == gprox.GP_ERR_UNSUPPORTED
    h.close()
