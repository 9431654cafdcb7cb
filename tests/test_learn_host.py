"""Host-side data handling of the warm-start training driver (no GPU): the
symmetry augmentation and the crop windows used to train on large grids."""
import numpy as np
import torch

from paper_1805_09453_gb300 import learn


def _sample(N, seed):
    g = torch.Generator().manual_seed(seed)
    return [torch.rand((N, N), generator=g) for _ in range(4)]


def test_crop_sample_takes_the_window_and_centres_the_target():
    f0, f1, phi, prior = _sample(32, 0)
    c0, c1, cphi, cpri = learn.crop_sample(f0, f1, phi, prior, 8, 16, 16)
    assert torch.equal(c0, f0[8:24, 16:32]) and torch.equal(c1, f1[8:24, 16:32])
    assert torch.equal(cpri, prior[8:24, 16:32])
    # the target is the window minus its own mean (the network's output is mean-free)
    w = phi[8:24, 16:32].double()
    assert torch.allclose(cphi.double(), w - w.mean(), atol=1e-6)
    assert abs(cphi.double().mean().item()) < 1e-7


def test_augment_group_is_the_16_symmetries():
    f0, f1, phi, prior = _sample(8, 1)
    seen = set()
    for g in range(16):
        a0, a1, aphi, apri = learn.augment(f0, f1, phi, prior, g)
        assert all(t.is_contiguous() for t in (a0, a1, aphi, apri))
        if g & 8:  # the swap exchanges the densities and negates the potentials
            b0, _, bphi, _ = learn.augment(f0, f1, phi, prior, g & 7)
            assert torch.equal(a1, b0) and torch.equal(aphi, -bphi)
        seen.add(a0.numpy().tobytes() + a1.numpy().tobytes())
    assert len(seen) == 16
    # transposition alone
    t0, _, tphi, _ = learn.augment(f0, f1, phi, prior, 1)
    assert torch.equal(t0, f0.T) and torch.equal(tphi, phi.T)
    assert np.array_equal(learn.augment(f0, f1, phi, prior, 0)[2].numpy(), phi.numpy())
