"""FP64 oracle of the learned warm-start network (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module; the library never does.

The paper has no learned component.  What is fixed by the paper is the object
the network predicts: the dual of the Beckmann problem (section 4.2) is a
potential phi with |grad phi| <= 1, and the dual iterate p of the G-prox
PDHG iteration (Algorithm 2, section 3.2) converges to its gradient, so a
predicted potential phi_0 gives the dual start p_0 = proj(grad phi_0).

Everything else here is the definition of the network written out plainly,
in float64, with no blocking or fusion:

* 3x3 convolution (cross-correlation) with zero padding,
      y[b, o, i, j] = bias[o] + sum_c sum_{di, dj in -1..1} W[o, c, di+1, dj+1] x[b, c, i+di, j+dj];
* ReLU after every convolution but the last;
* 2x2 average pooling; nearest 2x upsampling; skip connections by channel
  concatenation [upsampled, skip];
* widths 3 -> C -> C | C -> 2C -> 2C | 2C -> 4C -> 4C | 4C -> 8C -> 8C |
  12C -> 4C -> 4C | 6C -> 2C -> 2C | 3C -> C -> C | C -> 1;
* inputs (f0 - f1)/16, (f0 + f1)/16 and a prior potential (zero if none);
* output phi = prior + head output, with its mean removed;
* loss per sample |e|^2/|t|^2 + |D e|^2/|D t|^2 (e = phi - t, both
  mean-free, D the forward difference without 1/h, zero last slots),
  averaged over the batch;
* Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected).

The prior used by the library is the coarse-grid start: the densities'
block means on an (N/k)^2 grid, the EMD solved there (the oracle's own
iteration), and its potential interpolated bilinearly between cell centres
(clamped at the outermost centres) -- ``coarse_start`` below.

The backward pass is derived by hand (the adjoint of each linear map and
the ReLU mask); tests pin it against central finite differences of the loss.

``bf16=True`` reproduces the storage precision of the GPU's BF16 mode: the
inputs, the compute copy of the weights, every stored activation (ReLU
outputs, pooled fields) are rounded to bfloat16 (round to nearest even);
biases, the head's output, all gradients stay in full precision.
"""
from __future__ import annotations

import numpy as np

from oracle import gprox_oracle as O


# ------------------------------------------------------------------ layout
def conv_specs(C: int):
    """(cin, cout) of the 15 convolutions in forward order."""
    return [(3, C), (C, C), (C, 2 * C), (2 * C, 2 * C), (2 * C, 4 * C), (4 * C, 4 * C), (4 * C, 8 * C),
            (8 * C, 8 * C), (12 * C, 4 * C), (4 * C, 4 * C), (6 * C, 2 * C), (2 * C, 2 * C), (3 * C, C), (C, C),
            (C, 1)]


def num_params(C: int) -> int:
    return sum(ci * co * 9 + co for ci, co in conv_specs(C))


def unpack(w, C: int):
    """Flat parameter vector -> list of (W (cout, cin, 3, 3), b (cout,)) in float64."""
    w = np.asarray(w, np.float64)
    out, off = [], 0
    for ci, co in conv_specs(C):
        W = w[off:off + ci * co * 9].reshape(co, ci, 3, 3)
        off += ci * co * 9
        b = w[off:off + co]
        off += co
        out.append((W, b))
    assert off == w.size, (off, w.size)
    return out


def pack(grads):
    return np.concatenate([np.concatenate([dW.ravel(), db.ravel()]) for dW, db in grads])


# ------------------------------------------------------------ bf16 rounding
def round_bf16(x):
    """Round float64 values to bfloat16 (via float32, round to nearest even)."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).astype(np.float64)
    return np.where(np.isfinite(f), out, f.astype(np.float64))


# ------------------------------------------------------------ linear pieces
def conv3x3(x, W, b):
    """Zero-padded 3x3 cross-correlation, x (B, cin, H, W) -> (B, cout, H, W)."""
    B, ci, H, Wd = x.shape
    xp = np.zeros((B, ci, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((B, W.shape[0], H, Wd))
    for di in range(3):
        for dj in range(3):
            y += np.einsum("oc,bchw->bohw", W[:, :, di, dj], xp[:, :, di:di + H, dj:dj + Wd])
    if b is not None:
        y += b[None, :, None, None]
    return y


def conv3x3_adjoint(dy, W, x_shape):
    """Adjoint of x -> conv3x3(x, W, 0): the input gradient."""
    B, ci, H, Wd = x_shape
    dxp = np.zeros((B, ci, H + 2, Wd + 2))
    for di in range(3):
        for dj in range(3):
            dxp[:, :, di:di + H, dj:dj + Wd] += np.einsum("oc,bohw->bchw", W[:, :, di, dj], dy)
    return dxp[:, :, 1:-1, 1:-1]


def conv3x3_wgrad(dy, x):
    """Gradient of <dy, conv3x3(x, W, b)> with respect to W and b."""
    B, ci, H, Wd = x.shape
    xp = np.zeros((B, ci, H + 2, Wd + 2))
    xp[:, :, 1:-1, 1:-1] = x
    dW = np.zeros((dy.shape[1], ci, 3, 3))
    for di in range(3):
        for dj in range(3):
            dW[:, :, di, dj] = np.einsum("bohw,bchw->oc", dy, xp[:, :, di:di + H, dj:dj + Wd])
    return dW, dy.sum(axis=(0, 2, 3))


def pool2(x):
    """2x2 average pooling."""
    return 0.25 * ((x[:, :, 0::2, 0::2] + x[:, :, 0::2, 1::2]) + (x[:, :, 1::2, 0::2] + x[:, :, 1::2, 1::2]))


def pool2_adjoint(dy):
    return 0.25 * np.repeat(np.repeat(dy, 2, axis=2), 2, axis=3)


def up2(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(x, 2, axis=2), 2, axis=3)


def up2_adjoint(dy):
    return (dy[:, :, 0::2, 0::2] + dy[:, :, 0::2, 1::2]) + (dy[:, :, 1::2, 0::2] + dy[:, :, 1::2, 1::2])


# ------------------------------------------------------------------ inputs
def features(f0, f1, prior=None):
    """(3, N, N) input channels of one density pair."""
    f0 = np.asarray(f0, np.float64)
    f1 = np.asarray(f1, np.float64)
    pr = np.zeros_like(f0) if prior is None else np.asarray(prior, np.float64)
    return np.stack([(f0 - f1) / 16.0, (f0 + f1) / 16.0, pr])


def restrict_mean(f, k: int):
    """Block means over k x k blocks (an (N/k)^2 density of the same mass)."""
    n = f.shape[0] // k
    return np.asarray(f, np.float64).reshape(n, k, n, k).mean(axis=(1, 3))


def upsample_bilinear(c, k: int):
    """Cell-centred bilinear interpolation from n x n to nk x nk: fine centre j
    sits at coarse coordinate (j + 1/2)/k - 1/2, clamped to [0, n - 1]."""
    c = np.asarray(c, np.float64)
    n = c.shape[0]
    x = np.clip((np.arange(n * k) + 0.5) / k - 0.5, 0.0, n - 1.0)
    i0 = np.minimum(np.floor(x).astype(int), n - 1)
    i1 = np.minimum(i0 + 1, n - 1)
    t = x - i0
    rows = c[i0] * (1 - t)[:, None] + c[i1] * t[:, None]       # interpolate along y
    return rows[:, i0] * (1 - t)[None, :] + rows[:, i1] * t[None, :]


def coarse_start(f0, f1, k: int, n_iters: int):
    """Potential of the EMD on the k-times coarser grid after n_iters
    iterations of the oracle's iteration (from zero), interpolated to N x N."""
    c0, c1 = restrict_mean(f0, k), restrict_mean(f1, k)
    st = O.emd_solve(c0, c1, n_iters=n_iters)
    _, phi, _ = O.emd_dual(st["px"], st["py"], c0, c1)
    return upsample_bilinear(phi, k)


# ----------------------------------------------------------------- network
def forward(w, x, C: int, bf16: bool = False):
    """Network on inputs x (B, 3, N, N), channel 2 the prior; returns
    (phi (B, N, N) mean-free, cache)."""
    rnd = round_bf16 if bf16 else (lambda a: a)
    P = unpack(w, C)
    Wc = [(rnd(W), b) for W, b in P]  # compute copy of the weights; biases stay FP32
    cache = {"W": Wc, "C": C}

    def conv(i, a, relu=True):
        y = conv3x3(a, *Wc[i])
        return rnd(np.maximum(y, 0.0)) if relu else y

    x0 = rnd(np.asarray(x, np.float64))
    a1 = conv(0, x0)
    s1 = conv(1, a1)
    p1 = rnd(pool2(s1))
    a2 = conv(2, p1)
    s2 = conv(3, a2)
    p2 = rnd(pool2(s2))
    a3 = conv(4, p2)
    s3 = conv(5, a3)
    p3 = rnd(pool2(s3))
    m1 = conv(6, p3)
    m2 = conv(7, m1)
    k3 = np.concatenate([up2(m2), s3], axis=1)
    d3a = conv(8, k3)
    d3b = conv(9, d3a)
    k2 = np.concatenate([up2(d3b), s2], axis=1)
    d2a = conv(10, k2)
    d2b = conv(11, d2a)
    k1 = np.concatenate([up2(d2b), s1], axis=1)
    d1a = conv(12, k1)
    d1b = conv(13, d1a)
    raw = conv(14, d1b, relu=False)[:, 0] + np.asarray(x, np.float64)[:, 2]  # the prior, unrounded
    phi = raw - raw.mean(axis=(1, 2), keepdims=True)
    cache.update(x0=x0, a1=a1, s1=s1, p1=p1, a2=a2, s2=s2, p2=p2, a3=a3, s3=s3, p3=p3, m1=m1, m2=m2, k3=k3,
                 d3a=d3a, d3b=d3b, k2=k2, d2a=d2a, d2b=d2b, k1=k1, d1a=d1a, d1b=d1b)
    return phi, cache


def backward(cache, dphi):
    """Parameter gradient (flat) for dL/dphi (B, N, N) of a mean-free output."""
    C, Wc = cache["C"], cache["W"]
    c = cache
    grads = [None] * 15
    dphi = np.asarray(dphi, np.float64)
    draw = dphi - dphi.mean(axis=(1, 2), keepdims=True)  # adjoint of the mean removal

    def conv_back(i, dy, x, want_dx=True):
        grads[i] = conv3x3_wgrad(dy, x)
        return conv3x3_adjoint(dy, Wc[i][0], x.shape) if want_dx else None

    def relu_mask(d, y):
        return d * (y > 0)

    d = conv_back(14, draw[:, None], c["d1b"])
    d = conv_back(13, relu_mask(d, c["d1b"]), c["d1a"])
    dk1 = conv_back(12, relu_mask(d, c["d1a"]), c["k1"])
    n2 = 2 * C
    d = conv_back(11, relu_mask(up2_adjoint(dk1[:, :n2]), c["d2b"]), c["d2a"])
    dk2 = conv_back(10, relu_mask(d, c["d2a"]), c["k2"])
    n4 = 4 * C
    d = conv_back(9, relu_mask(up2_adjoint(dk2[:, :n4]), c["d3b"]), c["d3a"])
    dk3 = conv_back(8, relu_mask(d, c["d3a"]), c["k3"])
    n8 = 8 * C
    d = conv_back(7, relu_mask(up2_adjoint(dk3[:, :n8]), c["m2"]), c["m1"])
    dp3 = conv_back(6, relu_mask(d, c["m1"]), c["p3"])
    ds3 = dk3[:, n8:] + pool2_adjoint(dp3)
    d = conv_back(5, relu_mask(ds3, c["s3"]), c["a3"])
    dp2 = conv_back(4, relu_mask(d, c["a3"]), c["p2"])
    ds2 = dk2[:, n4:] + pool2_adjoint(dp2)
    d = conv_back(3, relu_mask(ds2, c["s2"]), c["a2"])
    dp1 = conv_back(2, relu_mask(d, c["a2"]), c["p1"])
    ds1 = dk1[:, n2:] + pool2_adjoint(dp1)
    d = conv_back(1, relu_mask(ds1, c["s1"]), c["a1"])
    conv_back(0, relu_mask(d, c["a1"]), c["x0"], want_dx=False)
    return pack(grads)


# -------------------------------------------------------------------- loss
def _fdiff(e):
    """Forward differences without 1/h, zero last slots."""
    dx = np.zeros_like(e)
    dy = np.zeros_like(e)
    dx[..., :, :-1] = e[..., :, 1:] - e[..., :, :-1]
    dy[..., :-1, :] = e[..., 1:, :] - e[..., :-1, :]
    return dx, dy


def loss(phi, t):
    """Batch-mean of |e|^2/|t|^2 + |D e|^2/|D t|^2 (phi, t: (B, N, N))."""
    phi = np.asarray(phi, np.float64)
    t = np.asarray(t, np.float64)
    t = t - t.mean(axis=(1, 2), keepdims=True)
    phi = phi - phi.mean(axis=(1, 2), keepdims=True)
    e = phi - t
    ex, ey = _fdiff(e)
    tx, ty = _fdiff(t)
    per = (e ** 2).sum(axis=(1, 2)) / (t ** 2).sum(axis=(1, 2)) + \
        (ex ** 2 + ey ** 2).sum(axis=(1, 2)) / (tx ** 2 + ty ** 2).sum(axis=(1, 2))
    return float(per.mean())


def loss_grad_phi(phi, t):
    """dL/dphi for mean-free phi: 2 e/|t|^2 + 2 D^T D e/|D t|^2, over B."""
    phi = np.asarray(phi, np.float64)
    t = np.asarray(t, np.float64)
    t = t - t.mean(axis=(1, 2), keepdims=True)
    e = phi - t
    ex, ey = _fdiff(e)
    tx, ty = _fdiff(t)
    # D^T applied to (ex, ey): the adjoint of the forward difference
    dtd = np.zeros_like(e)
    dtd[..., :, :-1] -= ex[..., :, :-1]
    dtd[..., :, 1:] += ex[..., :, :-1]
    dtd[..., :-1, :] -= ey[..., :-1, :]
    dtd[..., 1:, :] += ey[..., :-1, :]
    s0 = (t ** 2).sum(axis=(1, 2))[:, None, None]
    s1 = (tx ** 2 + ty ** 2).sum(axis=(1, 2))[:, None, None]
    return (2.0 * e / s0 + 2.0 * dtd / s1) / e.shape[0]


def loss_and_grad(w, x, t, C: int, bf16: bool = False):
    phi, cache = forward(w, x, C, bf16)
    return loss(phi, t), backward(cache, loss_grad_phi(phi, t)), phi


def adam_step(w, m, v, g, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (step counts from 1)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    w = w - lr * (m / (1 - b1 ** step)) / (np.sqrt(v / (1 - b2 ** step)) + eps)
    return w, m, v


def warm_dual(phi):
    """p_0 = proj(grad phi) with the oracle's forward-difference gradient (h = 1/N)."""
    N = phi.shape[-1]
    gx, gy = O.grad(np.asarray(phi, np.float64), 1.0 / N)
    return O.project(gx, gy)
