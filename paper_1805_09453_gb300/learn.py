"""Training and evaluation driver of the learned warm starts (EMD, and ROF
with ``--problem rof``).

Every step runs in the library: the training targets come from the library's
own EMD solve (the converged dual potential phi* = Lap^{-1} div p*), the
network's prior is the library's coarse-grid start (``emd_coarse_start``),
the network's forward pass, loss, backward pass and Adam step are the
library's kernels (``gp_cnn_*``), and the evaluation compares three arms to
the same relative gap: ``emd_solve`` from zero, the prior alone (a network
whose head is zero returns its prior), and ``emd_solve_learned`` (the start
with the smallest duality gap at n = 0 among learned, prior and zero).

    python -m paper_1805_09453_gb300.learn --N 512 --C 32 --train 512 --test 64 \
        --steps 2000 --out warm.npz --report warm.json

Inputs are seeded Gaussian-mixture density pairs (``synth.gaussian_mixture_pair``);
training seeds are 0.., held-out seeds start at 1_000_000.  ``--problem rof``
trains the same network on ROF images (``synth.rof_image``, fidelity weight
``--lam``) against u* - mean(I) and evaluates ``rof_solve_learned``:

    python -m paper_1805_09453_gb300.learn --problem rof --N 512 --train 256 --test 32 \
        --steps 1500 --report rof_warm.json
"""
from __future__ import annotations

import argparse
import json
import statistics
import time

import numpy as np
import torch

from . import gprox, synth

TEST_SEED0 = 1_000_000


def pairs(N: int, seeds, device="cuda"):
    """(f0, f1) stacks (S, N, N) on the device for the given seeds."""
    f0 = torch.empty((len(seeds), N, N), device=device)
    f1 = torch.empty_like(f0)
    for i, s in enumerate(seeds):
        a, b = synth.gaussian_mixture_pair(N, int(s))
        f0[i].copy_(torch.from_numpy(a))
        f1[i].copy_(torch.from_numpy(b))
    return f0, f1


def coarse_opts(tol: float = 1e-4, max_iters: int = 100000, gap_every: int = 50):
    return gprox.default_opts(max_iters=max_iters, tol_rel_gap=tol, gap_every=gap_every, use_graph=1)


def generate(h: gprox.Handle, N: int, seeds, tol: float = 1e-6, max_iters: int = 40000, gap_every: int = 50,
             coarse_factor: int = 4, coarse_tol: float = 1e-4, verbose: bool = False, warm: bool = False):
    """Solve each pair and compute its coarse-grid prior; returns f0, f1,
    phi*, prior (S, N, N), the iteration counts and the gaps.  The solve
    starts from zero, or with warm from the prior (emd_solve_learned with a
    network whose output is its prior: the same certified stop, fewer
    iterations on large grids)."""
    f0, f1 = pairs(N, seeds)
    phi = torch.empty_like(f0)
    prior = torch.zeros_like(f0)
    torch.cuda.synchronize()
    with torch.cuda.stream(torch.cuda.Stream()):  # a non-default stream: the solves replay CUDA graphs
        out = _generate(h, N, f0, f1, phi, prior, tol, max_iters, gap_every, coarse_factor, coarse_tol, verbose,
                        warm)
    torch.cuda.synchronize()
    return out


def _generate(h, N, f0, f1, phi, prior, tol, max_iters, gap_every, coarse_factor, coarse_tol, verbose, warm):
    seeds = range(f0.shape[0])
    m = torch.empty((2, N, N), device=f0.device)
    p = torch.empty((2, N, N), device=f0.device)
    o = gprox.default_opts(max_iters=max_iters, tol_rel_gap=tol, gap_every=gap_every, use_graph=1)
    oc = coarse_opts(coarse_tol)
    base = None
    if warm and coarse_factor:
        base = gprox.Cnn(h, 1, seed=0)
        base.set_params(np.zeros(base.num_params, np.float32))  # output = prior
    iters, gaps = [], []
    for i in range(len(seeds)):
        if base is not None:
            st, rep = gprox.emd_solve_learned(h, base, f0[i], f1[i], m, p, phi[i], o, coarse_factor, oc)
        else:
            st, rep = gprox.emd_solve(h, f0[i], f1[i], m, p, phi[i], o)
        h.check(st, allow=(gprox.GP_OK, gprox.GP_ERR_MAXITER))
        iters.append(rep["iters"])
        gaps.append(rep["rel_gap"])
        if coarse_factor:
            st, _, _ = gprox.emd_coarse_start(h, f0[i], f1[i], coarse_factor, oc, phi=prior[i])
            h.check(st, allow=(gprox.GP_OK, gprox.GP_ERR_MAXITER))
        if verbose and ((i + 1) % 32 == 0 or (base is not None and (i + 1) % 4 == 0)):
            print(f"generated {i + 1}/{len(seeds)} pairs (median iterations {statistics.median(iters)})", flush=True)
    torch.cuda.synchronize()
    if base is not None:
        base.close()
    return f0, f1, phi, prior, iters, gaps


# --------------------------------------------------------------------- ROF
# The same network proposes the ROF primal iterate (rof_solve_learned): the
# inputs are a = 8 (I - mean), b = -a (channels I - mean and 0), the prior
# u_prior - mean, and the target u* - mean (a fidelity minimiser keeps the
# mean).  Swapping a and b negates I, and the ROF minimiser is odd in I, so
# the symmetries of `augment` hold for these samples too.

def images(N: int, seeds, device="cuda"):
    """ROF images (S, N, N) on the device (``synth.rof_image``)."""
    out = torch.empty((len(seeds), N, N), device=device)
    for i, s in enumerate(seeds):
        out[i].copy_(torch.from_numpy(synth.rof_image(N, int(s))))
    return out


def generate_rof(h: gprox.Handle, N: int, seeds, lam: float = 8.0, tol: float = 1e-6, max_iters: int = 20000,
                 gap_every: int = 10, coarse_factor: int = 4, coarse_tol: float = 1e-4):
    """Solve each image with the plain method; returns the network's inputs
    (a, b), targets u* - mean, priors u_prior - mean (S, N, N), the images,
    the iteration counts and the gaps."""
    I = images(N, seeds)
    tgt = torch.empty_like(I)
    prior = torch.zeros_like(I)
    u = torch.empty((N, N), device=I.device)
    o = gprox.default_opts(max_iters=max_iters, tol_rel_gap=tol, gap_every=gap_every, use_graph=1)
    oc = coarse_opts(coarse_tol)
    iters, gaps = [], []
    torch.cuda.synchronize()
    with torch.cuda.stream(torch.cuda.Stream()):
        for i in range(I.shape[0]):
            st, rep = gprox.rof_solve(h, I[i], u, None, lam, o)
            h.check(st, allow=(gprox.GP_OK, gprox.GP_ERR_MAXITER))
            iters.append(rep["iters"])
            gaps.append(rep["rel_gap"])
            mean = I[i].double().mean().float()
            tgt[i].copy_(u - mean)
            if coarse_factor:
                st, uc, _, _ = gprox.rof_coarse_start(h, I[i], coarse_factor, lam, oc)
                h.check(st, allow=(gprox.GP_OK, gprox.GP_ERR_MAXITER))
                prior[i].copy_(uc - mean)
    torch.cuda.synchronize()
    c = I - I.double().mean(dim=(1, 2), keepdim=True).float()
    return 8.0 * c, -8.0 * c, tgt, prior, I, iters, gaps


def evaluate_rof(h: gprox.Handle, net: gprox.Cnn, I, lam: float = 8.0, tol: float = 1e-5, max_iters: int = 20000,
                 gap_every: int = 10, coarse_factor: int = 4, coarse_tol: float = 1e-4):
    """Per image: iterations, seconds, status and primal to `tol` from zero, from
    the prior alone and from the learned start (rof_solve_learned)."""
    N = I.shape[-1]
    u = torch.empty((N, N), device=I.device)
    o = gprox.default_opts(max_iters=max_iters, tol_rel_gap=tol, gap_every=gap_every, use_graph=1)
    oc = coarse_opts(coarse_tol)
    base = gprox.Cnn(h, 1, seed=0)
    base.set_params(np.zeros(base.num_params, np.float32))  # output = prior
    name = gprox.STATUS_NAMES
    rows = []
    torch.cuda.synchronize()
    with torch.cuda.stream(torch.cuda.Stream()):
        for i in range(I.shape[0]):
            (st, rz), tz = _timed(lambda: gprox.rof_solve(h, I[i], u, None, lam, o))
            row = {"zero_iters": rz["iters"], "zero_s": tz, "zero_gap": rz["rel_gap"], "zero_status": name[st],
                   "zero_primal": rz["primal"]}
            if coarse_factor:
                (st, rp), tp = _timed(lambda: gprox.rof_solve_learned(h, base, I[i], u, None, lam, o,
                                                                       coarse_factor, oc))
                row.update(prior_iters=rp["iters"], prior_s=tp, prior_gap=rp["rel_gap"], prior_status=name[st],
                           prior_start=rp["start"], prior_primal=rp["primal"])
            (st, rw), tw = _timed(lambda: gprox.rof_solve_learned(h, net, I[i], u, None, lam, o, coarse_factor, oc))
            row.update(warm_iters=rw["iters"], warm_s=tw, warm_gap=rw["rel_gap"], warm_status=name[st],
                       warm_start=rw["start"], warm_primal=rw["primal"])
            rows.append(row)
    torch.cuda.synchronize()
    base.close()
    return rows


def augment(f0, f1, phi, prior, g: int):
    """Symmetry g in [0, 16) of a training sample: bit 0 transposes, bits 1-2
    flip rows / columns, bit 3 swaps f0 and f1 (which negates the potentials).
    Transposition and the swap map solutions to solutions exactly; a flip
    turns forward into backward differences, so its targets are approximate."""
    out = [f0, f1, phi, prior]
    if g & 1:
        out = [t.transpose(-2, -1) for t in out]
    dims = [d for d, bit in ((-2, 2), (-1, 4)) if g & bit]
    if dims:
        out = [torch.flip(t, dims) for t in out]
    if g & 8:
        out = [out[1], out[0], -out[2], -out[3]]
    return [t.contiguous() for t in out]


def crop_sample(f0, f1, phi, prior, y: int, x: int, c: int):
    """The c x c window at (y, x) of one sample.  The network's inputs are
    pointwise in (f0, f1, prior) and its output is made mean-free, so a window
    of a large grid is a sample with that grid's local statistics (features
    as many cells wide as there); the target is made mean-free in the window."""
    out = [t[y:y + c, x:x + c] for t in (f0, f1, phi, prior)]
    out[2] = out[2] - out[2].double().mean().float()
    return out


def train(net: gprox.Cnn, f0, f1, phi, prior, steps: int, batch: int, lr: float, seed: int = 0,
          log_every: int = 50, lr_final: float | None = None, augment_data: bool = True, crop: int = 0):
    """Adam on random mini-batches (random symmetries when augment_data; with
    crop, random crop x crop windows at multiples of 8); cosine decay of the
    step size to lr_final."""
    rng = np.random.default_rng(seed)
    S, N = f0.shape[0], f0.shape[-1]
    lr_final = lr * 0.05 if lr_final is None else lr_final
    hist = []
    for k in range(steps):
        idx = rng.choice(S, size=min(batch, S), replace=False) if not crop else rng.integers(0, S, size=batch)
        gs = rng.integers(0, 16, size=len(idx)) if augment_data else np.zeros(len(idx), int)
        if crop:
            yx = rng.integers(0, (N - crop) // 8 + 1, size=(len(idx), 2)) * 8
            smp = [augment(*crop_sample(f0[i], f1[i], phi[i], prior[i], int(y), int(x), crop), int(g))
                   for i, g, (y, x) in zip(idx, gs, yx)]
        else:
            smp = [augment(f0[i], f1[i], phi[i], prior[i], int(g)) for i, g in zip(idx, gs)]
        want = (k % log_every == 0) or k == steps - 1
        L, _ = net.loss_grad([a[0] for a in smp], [a[1] for a in smp], [a[2] for a in smp], [a[3] for a in smp],
                             want_loss=want)
        if want:
            hist.append((k, L))
        a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * k / max(1, steps)))
        net.adam_step(a)
    torch.cuda.synchronize()
    return hist


def test_loss(net: gprox.Cnn, f0, f1, phi, prior, batch: int = 8):
    out = []
    for i in range(0, f0.shape[0], batch):
        j = range(i, min(i + batch, f0.shape[0]))
        L, _ = net.loss_grad([f0[k] for k in j], [f1[k] for k in j], [phi[k] for k in j], [prior[k] for k in j])
        out.append(L * len(j))
    return sum(out) / f0.shape[0]


def _timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def evaluate(h: gprox.Handle, net: gprox.Cnn, f0, f1, tol: float = 1e-5, max_iters: int = 40000,
             gap_every: int = 10, coarse_factor: int = 4, coarse_tol: float = 1e-4, prior_arm: bool = True):
    """Per pair: iterations, seconds and status to `tol` from the zero start,
    from the prior alone and from the learned start (seconds include the
    coarse solve, the network and the start probes).  Runs on a non-default
    stream, so every arm replays CUDA graphs."""
    torch.cuda.synchronize()
    with torch.cuda.stream(torch.cuda.Stream()):
        return _evaluate(h, net, f0, f1, tol, max_iters, gap_every, coarse_factor, coarse_tol, prior_arm)


def _evaluate(h, net, f0, f1, tol, max_iters, gap_every, coarse_factor, coarse_tol, prior_arm):
    N = f0.shape[-1]
    m = torch.empty((2, N, N), device=f0.device)
    o = gprox.default_opts(max_iters=max_iters, tol_rel_gap=tol, gap_every=gap_every, use_graph=1)
    oc = coarse_opts(coarse_tol)
    base = None
    if prior_arm and coarse_factor:
        base = gprox.Cnn(h, 1, seed=0)
        base.set_params(np.zeros(base.num_params, np.float32))  # output = prior
    name = gprox.STATUS_NAMES
    rows = []
    for i in range(f0.shape[0]):
        (st, rz), tz = _timed(lambda: gprox.emd_solve(h, f0[i], f1[i], m, None, None, o))
        row = {"zero_iters": rz["iters"], "zero_s": tz, "zero_gap": rz["rel_gap"], "zero_status": name[st]}
        if base is not None:
            (st, rp), tp = _timed(lambda: gprox.emd_solve_learned(h, base, f0[i], f1[i], m, None, None, o,
                                                                   coarse_factor, oc))
            row.update(prior_iters=rp["iters"], prior_s=tp, prior_gap=rp["rel_gap"], prior_status=name[st],
                       prior_start=rp["start"])
        (st, rw), tw = _timed(lambda: gprox.emd_solve_learned(h, net, f0[i], f1[i], m, None, None, o,
                                                               coarse_factor, oc))
        row.update(warm_iters=rw["iters"], warm_s=tw, warm_gap=rw["rel_gap"], warm_status=name[st],
                   warm_start=rw["start"])
        rows.append(row)
    if base is not None:
        base.close()
    return rows


def network_cost(net: gprox.Cnn, f0, f1, prior, reps: int = 10):
    """Mean seconds of one forward pass (B = 1) on the device."""
    net.forward([f0[0]], [f1[0]], [prior[0]])
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        net.forward([f0[0]], [f1[0]], [prior[0]])
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / 1e3 / reps


def summarize(rows):
    med = statistics.median
    out = {"pairs": len(rows)}
    for arm in ("zero", "prior", "warm"):
        if f"{arm}_iters" not in rows[0]:
            continue
        out[f"median_{arm}_iters"] = med([r[f"{arm}_iters"] for r in rows])
        out[f"median_{arm}_s"] = med([r[f"{arm}_s"] for r in rows])
        out[f"{arm}_not_ok"] = sum(r[f"{arm}_status"] != "GP_OK" for r in rows)
    out["median_iter_ratio"] = med([r["warm_iters"] / max(r["zero_iters"], 1) for r in rows])
    out["median_time_ratio"] = med([r["warm_s"] / max(r["zero_s"], 1e-12) for r in rows])
    out["fallback_rate"] = sum(r["warm_start"] != "learned" for r in rows) / len(rows)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--problem", default="emd", choices=["emd", "rof"])
    ap.add_argument("--lam", type=float, default=8.0, help="ROF fidelity weight")
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--C", type=int, default=32)
    ap.add_argument("--fp32", action="store_true", help="FP32 storage instead of BF16")
    ap.add_argument("--train", type=int, default=512, help="training pairs (seeds 0..)")
    ap.add_argument("--test", type=int, default=64, help="held-out pairs (seeds 1e6..)")
    ap.add_argument("--data-tol", type=float, default=1e-6)
    ap.add_argument("--data-max-iters", type=int, default=40000)
    ap.add_argument("--data-warm", action="store_true", help="solve the training pairs from the coarse start")
    ap.add_argument("--crop", type=int, default=0, help="train on random crop x crop windows (0: whole grids)")
    ap.add_argument("--eval-gap-every", type=int, default=10, help="gap checks of the evaluation (0: adaptive)")
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--tol", type=float, default=1e-5, help="evaluation gap")
    ap.add_argument("--coarse", type=int, default=4, help="coarse-grid factor of the prior (0: none)")
    ap.add_argument("--coarse-tol", type=float, default=1e-4)
    ap.add_argument("--eval-N", type=int, default=0, help="also evaluate on pairs of this size (0: no)")
    ap.add_argument("--eval-pairs", type=int, default=1)
    ap.add_argument("--eval-coarse", type=int, default=8)
    ap.add_argument("--eval-coarse-tol", type=float, default=1e-6)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--init", default=None, help="start from these weights (.npz)")
    ap.add_argument("--out", default=None, help="write the trained weights (.npz)")
    ap.add_argument("--report", default=None, help="write the JSON report")
    a = ap.parse_args(argv)
    gprox.lib()
    h = gprox.Handle(0)
    net = gprox.Cnn(h, a.C, bf16=not a.fp32, seed=a.seed)
    if a.init:
        net.set_params(np.load(a.init)["w"])
    rep = {"N": a.N, "C": a.C, "bf16": not a.fp32, "params": net.num_params, "problem": a.problem}
    if a.problem == "rof":
        return _main_rof(a, h, net, rep)
    t0 = time.perf_counter()
    dge = 0 if a.data_warm else 50
    f0, f1, phi, pri, it, gaps = generate(h, a.N, range(a.train), a.data_tol, a.data_max_iters, dge,
                                          coarse_factor=a.coarse, coarse_tol=a.coarse_tol, verbose=True,
                                          warm=a.data_warm)
    rep["data"] = {"pairs": a.train, "seconds": time.perf_counter() - t0, "median_iters": statistics.median(it),
                   "max_gap": max(gaps), "warm": a.data_warm, "crop": a.crop}
    g0, g1, gphi, gpri, _, _ = generate(h, a.N, range(TEST_SEED0, TEST_SEED0 + a.test), a.data_tol,
                                        a.data_max_iters, dge, coarse_factor=a.coarse, coarse_tol=a.coarse_tol,
                                        warm=a.data_warm)
    tb = 1 if a.N > 1024 else 8
    rep["test_loss_init"] = test_loss(net, g0, g1, gphi, gpri, tb)
    t0 = time.perf_counter()
    hist = train(net, f0, f1, phi, pri, a.steps, a.batch, a.lr, a.seed, crop=a.crop)
    print(f"trained {a.steps} steps in {time.perf_counter() - t0:.1f} s, loss {hist[-1][1]:.4g}", flush=True)
    rep["train"] = {"steps": a.steps, "batch": a.batch, "lr": a.lr, "seconds": time.perf_counter() - t0,
                    "loss": hist[-1][1], "history": hist}
    rep["test_loss"] = test_loss(net, g0, g1, gphi, gpri, tb)
    rep["network_seconds"] = network_cost(net, g0, g1, gpri)
    if a.out:
        np.savez(a.out, w=net.get_params(), C=a.C, N=a.N, coarse=a.coarse, crop=a.crop)
    rows = evaluate(h, net, g0, g1, a.tol, max_iters=max(40000, a.data_max_iters), gap_every=a.eval_gap_every,
                    coarse_factor=a.coarse, coarse_tol=a.coarse_tol)
    rep["eval"] = summarize(rows)
    rep["eval"]["tol"] = a.tol
    rep["rows"] = rows
    if a.eval_N:
        e0, e1 = pairs(a.eval_N, range(TEST_SEED0, TEST_SEED0 + a.eval_pairs))
        big = evaluate(h, net, e0, e1, a.tol, max_iters=200000, coarse_factor=a.eval_coarse,
                       coarse_tol=a.eval_coarse_tol)
        rep["eval_large"] = {"N": a.eval_N, "coarse": a.eval_coarse, "coarse_tol": a.eval_coarse_tol,
                             "summary": summarize(big), "rows": big}
        print(json.dumps(rep["eval_large"]["summary"]), flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps({k: v for k, v in rep.items() if k not in ("rows", "eval_large")}, default=str))
    return rep


def _main_rof(a, h, net, rep):
    t0 = time.perf_counter()
    f0, f1, tgt, pri, _, it, gaps = generate_rof(h, a.N, range(a.train), a.lam, a.data_tol,
                                                  coarse_factor=a.coarse, coarse_tol=a.coarse_tol)
    rep["data"] = {"images": a.train, "lambda": a.lam, "seconds": time.perf_counter() - t0,
                   "median_iters": statistics.median(it), "max_gap": max(gaps)}
    g0, g1, gt, gp, gI, _, _ = generate_rof(h, a.N, range(TEST_SEED0, TEST_SEED0 + a.test), a.lam, a.data_tol,
                                            coarse_factor=a.coarse, coarse_tol=a.coarse_tol)
    rep["test_loss_init"] = test_loss(net, g0, g1, gt, gp)
    t0 = time.perf_counter()
    hist = train(net, f0, f1, tgt, pri, a.steps, a.batch, a.lr, a.seed)
    rep["train"] = {"steps": a.steps, "batch": a.batch, "lr": a.lr, "seconds": time.perf_counter() - t0,
                    "loss": hist[-1][1], "history": hist}
    rep["test_loss"] = test_loss(net, g0, g1, gt, gp)
    rep["network_seconds"] = network_cost(net, g0, g1, gp)
    if a.out:
        np.savez(a.out, w=net.get_params(), C=a.C, N=a.N, coarse=a.coarse, problem="rof", lam=a.lam)
    rows = evaluate_rof(h, net, gI, a.lam, a.tol, coarse_factor=a.coarse, coarse_tol=a.coarse_tol)
    rep["eval"] = summarize(rows)
    rep["eval"]["tol"] = a.tol
    rep["rows"] = rows
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps({k: v for k, v in rep.items() if k != "rows"}, default=str))
    return rep


if __name__ == "__main__":
    main()
