"""The fused step kernels (one iteration's stencil run by the CTAs of the next
solve's forward row pass) against the unfused kernels and the FP64 oracle.

Within a chunk of k steps every step but the last runs its stencil fused with
the next row pass, the right-hand side handed on as row spectra; a chunk of
one step runs the plain stencil kernel and then, in the next chunk, the
separate row pass.  So `step(S)` takes S - 1 fused steps and S x `step(1)`
none.  Both evaluate the same formulas, but the compiler may contract a
multiply-add differently in the two kernels, and on a random (non-smooth)
state the 1/h of the gradient amplifies such FP32 rounding differences over
the steps (at 512^2 after 6 ROF steps both runs sit ~3e-5 from the oracle).
So the oracle decides: the fused run must be as close to the FP64 oracle as
the unfused run (within 1.5x plus a rounding floor), and the two runs no
further apart than twice the unfused run's distance to the oracle.  Sizes:
the fast-path classes (16 and 64: one thread group per transform; 512 and
1024: parallel syntheses in the other passes; 4096: the benchmark size, 3
steps there to keep the oracle run short).  ROF: section 3.1, EMD: section
3.2.
"""
import numpy as np
import pytest
import torch

from oracle import gprox_oracle as O
from paper_1805_09453_gb300 import synth
from tests.gpu_common import random_unit_field, rel_l2, zero_slots

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    from paper_1805_09453_gb300 import build, gprox

    build.build()
    hh = gprox.Handle(0)
    yield hh
    hh.close()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rof_state(h, N, I, u0, p0, pb0):
    from paper_1805_09453_gb300 import gprox

    return gprox.State(h, "rof", N, I=_t(I), lam=8.0, tau=2.0, sigma=0.5, primal0=_t(u0), p0=_t(np.stack(p0)),
                       pbar0=_t(np.stack(pb0)))


def _emd_state(h, N, f0, f1, m0, p0, pb0):
    from paper_1805_09453_gb300 import gprox

    return gprox.State(h, "emd", N, f0=_t(f0), f1=_t(f1), tau=1.3, sigma=0.7, primal0=_t(np.stack(m0)),
                       p0=_t(np.stack(p0)), pbar0=_t(np.stack(pb0)))


def _run(make, steps):
    a = make()
    a.step(steps)
    prim_a, p_a = a.read()
    b = make()
    for _ in range(steps):
        b.step(1)
    prim_b, p_b = b.read()
    a.close()
    b.close()
    return (prim_a.cpu().numpy(), p_a.cpu().numpy()), (prim_b.cpu().numpy(), p_b.cpu().numpy())


def _judge(fa, fb, ref_prim, ref_p, what):
    pmax = lambda p: max(np.abs(p[0] - ref_p[0]).max(), np.abs(p[1] - ref_p[1]).max())
    d_fo, d_po, d_fp = rel_l2(fa[0], ref_prim), rel_l2(fb[0], ref_prim), rel_l2(fa[0], fb[0])
    q_fo, q_po, q_fp = pmax(fa[1]), pmax(fb[1]), float(np.abs(fa[1] - fb[1]).max())
    print(f"{what}: primal fused-oracle {d_fo:.2e} plain-oracle {d_po:.2e} fused-plain {d_fp:.2e} | "
          f"p {q_fo:.2e} {q_po:.2e} {q_fp:.2e}")
    assert d_fo <= 1.5 * d_po + 1e-6 and d_fp <= 2 * d_po + 1e-6, (d_fo, d_po, d_fp)
    assert q_fo <= 1.5 * q_po + 1e-5 and q_fp <= 2 * q_po + 1e-5, (q_fo, q_po, q_fp)


def _steps(N):
    return 3 if N >= 4096 else 6


@pytest.mark.parametrize("N", [16, 64, 512, 1024, 4096])
def test_rof_fused_steps(h, N):
    rng = np.random.default_rng(7 * N)
    I = synth.rof_image(N, 3) if N >= 512 else rng.uniform(0, 1, (N, N)).astype(np.float32)
    u0 = rng.uniform(0, 1, (N, N)).astype(np.float32)
    p0 = random_unit_field(N, N + 1)
    pb0 = random_unit_field(N, N + 2, scale=2.0)
    S = _steps(N)
    fa, fb = _run(lambda: _rof_state(h, N, I, u0, p0, pb0), S)
    ref = O.rof_init(I, u0, p0, pb0)
    O.rof_iterate(ref, I, 8.0, 2.0, 0.5, S)
    _judge(fa, fb, ref["u"], (ref["px"], ref["py"]), f"ROF {N}, {S} steps")


@pytest.mark.parametrize("N", [16, 64, 512, 1024, 4096])
def test_emd_fused_steps(h, N):
    f0, f1 = synth.gaussian_mixture_pair(N, N)
    rng = np.random.default_rng(N)
    m0 = zero_slots(rng.normal(size=(N, N)), rng.normal(size=(N, N)))
    p0 = random_unit_field(N, N + 1)
    pb0 = random_unit_field(N, N + 2, scale=2.0)
    S = _steps(N)
    fa, fb = _run(lambda: _emd_state(h, N, f0, f1, m0, p0, pb0), S)
    # the library keeps m on {div m = f0 - f1}: the oracle starts from the
    # projection of m0 onto that set (the library's first step does the same)
    hh = 1.0 / N
    c = O.helmholtz_solve(-(f0.astype(np.float64) - f1 - O.div(m0[0].astype(np.float64),
                                                               m0[1].astype(np.float64), hh)), 0.0, hh)
    gx, gy = O.grad(c, hh)
    ref = O.emd_init(f0, f1, (m0[0] + gx, m0[1] + gy), p0, pb0)
    O.emd_iterate(ref, 1.3, 0.7, S)
    _judge(fa, fb, np.stack([ref["mx"], ref["my"]]), (ref["px"], ref["py"]), f"EMD {N}, {S} steps")


def test_fused_chunk_then_split_precision_step(h):
    """A chunk always ends with the right-hand side itself written, so a
    split-precision step (which has no row-spectra input) may follow an FP32
    chunk: same iterate as FP32 chunks throughout, to the split mode's error."""
    N = 512
    f0, f1 = synth.gaussian_mixture_pair(N, 5)
    z = np.zeros((N, N), np.float32)
    a = _emd_state(h, N, f0, f1, (z, z), (z, z), (z, z))
    b = _emd_state(h, N, f0, f1, (z, z), (z, z), (z, z))
    a.step(5)
    a.step(1, prec="split_bf16")
    a.step(4)
    b.step(10)
    ma, _ = a.read()
    mb, _ = b.read()
    e = rel_l2(ma.cpu().numpy(), mb.cpu().numpy())
    print(f"FP32 chunks with one split-precision step vs FP32 only: {e:.2e}")
    assert e < 1e-3
    a.close()
    b.close()
