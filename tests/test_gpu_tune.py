"""Autotuner of the fused kernels' tile shape (row-block height): it picks a
valid height, persists it in a JSON cache that a second handle reads back,
and changes no iterate (the kernels compute the same values per point)."""
import json

import numpy as np
import pytest
import torch

from paper_1805_09453_gb300 import synth

pytestmark = pytest.mark.gpu


def test_autotune_cache_and_identical_iterates(tmp_path):
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    N = 256
    path = str(tmp_path / "tune.json")
    h1 = gprox.Handle(0)
    I = torch.from_numpy(synth.rof_image(N, 4)).cuda()
    u_ref = torch.empty_like(I)
    p_ref = torch.empty((2, N, N), device="cuda")
    opts = gprox.default_opts(max_iters=40, tol_rel_gap=0.0)
    st, rep_ref = gprox.rof_solve(h1, I, u_ref, p_ref, 8.0, opts)
    h1.check(st)
    h1.check(gprox.autotune(h1, N, path))
    rows = {k: gprox.tuned_row_block(h1, k, N) for k in ("rof_fused", "emd_fused")}
    assert all(v in (4, 8, 16, 32) for v in rows.values()), rows
    cache = json.load(open(path))
    assert len(cache) == 2 and sorted(cache.values()) == sorted(rows.values())
    u = torch.empty_like(I)
    p = torch.empty((2, N, N), device="cuda")
    st, rep = gprox.rof_solve(h1, I, u, p, 8.0, opts)
    h1.check(st)
    assert torch.equal(u, u_ref) and torch.equal(p, p_ref)
    assert abs(rep["primal"] - rep_ref["primal"]) <= 1e-12 * abs(rep_ref["primal"])
    h2 = gprox.Handle(0)
    h2.check(gprox.autotune(h2, N, path))  # read back, no re-timing needed
    assert {k: gprox.tuned_row_block(h2, k, N) for k in rows} == rows
    h1.close()
    h2.close()
