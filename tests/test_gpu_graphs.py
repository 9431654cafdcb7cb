"""CUDA-graph replay across calls (use_graph, non-default stream): a state's
captured chunk graphs read only the state's own buffers, so solving new
inputs -- in new buffers or in the same ones -- replays them; every result
must equal the graph-free solve of the same input on a fresh handle, bit for
bit (same kernels, same order)."""
import numpy as np
import pytest
import torch

from paper_1805_09453_gb300 import synth

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_graph_replay_follows_new_inputs():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    N = 128
    h = gprox.Handle(0)
    imgs = [synth.rof_image(N, s) for s in (0, 1)]
    pairs = [synth.gaussian_mixture_pair(N, s) for s in (2, 3)]
    og = gprox.default_opts(max_iters=40, tol_rel_gap=0.0, gap_every=10, use_graph=1)
    od = gprox.default_opts(max_iters=40, tol_rel_gap=0.0, gap_every=10, use_graph=0)
    stream = torch.cuda.Stream()
    got_u, got_m = [], []
    with torch.cuda.stream(stream):
        # A, B, then A again from a new buffer: the second A replays graphs captured for B
        for I in (imgs[0], imgs[1], imgs[0]):
            u = torch.empty((N, N), device="cuda")
            st, rep = gprox.rof_solve(h, _t(I), u, None, 8.0, og)
            h.check(st)
            got_u.append(u)
        for f0, f1 in (pairs[0], pairs[1], pairs[0]):
            m = torch.empty((2, N, N), device="cuda")
            st, rep = gprox.emd_solve(h, _t(f0), _t(f1), m, None, None, og)
            h.check(st)
            got_m.append(m)
        stream.synchronize()
    h2 = gprox.Handle(0)
    for k, I in enumerate((imgs[0], imgs[1], imgs[0])):
        u = torch.empty((N, N), device="cuda")
        h2.check(gprox.rof_solve(h2, _t(I), u, None, 8.0, od)[0])
        assert torch.equal(u, got_u[k]), k
    for k, (f0, f1) in enumerate((pairs[0], pairs[1], pairs[0])):
        m = torch.empty((2, N, N), device="cuda")
        h2.check(gprox.emd_solve(h2, _t(f0), _t(f1), m, None, None, od)[0])
        assert torch.equal(m, got_m[k]), k
    assert not torch.equal(got_u[0], got_u[1])
    h.close()
    h2.close()
