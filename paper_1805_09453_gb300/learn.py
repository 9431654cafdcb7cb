"""Training and evaluation driver of the learned EMD warm start.

Every step runs in the library: the training targets come from the library's
own EMD solve (the converged dual potential phi* = Lap^{-1} div p*), the
network's forward pass, loss, backward pass and Adam step are the library's
kernels (``gp_cnn_*``), and the evaluation compares ``emd_solve`` from the
zero start with ``emd_solve_learned`` (learned start with the zero-start
fallback decided by the duality gap at n = 0).

    python -m paper_1805_09453_gb300.learn --N 512 --C 32 --train 512 --test 64 \
        --steps 2000 --out warm.npz --report warm.json

Inputs are seeded Gaussian-mixture density pairs (``synth.gaussian_mixture_pair``);
training seeds are 0.., held-out seeds start at 1_000_000.
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


def generate(h: gprox.Handle, N: int, seeds, tol: float = 1e-6, max_iters: int = 40000, gap_every: int = 50,
             verbose: bool = False):
    """Solve each pair with the plain method; returns f0, f1, phi* (S, N, N), the iteration counts and gaps."""
    f0, f1 = pairs(N, seeds)
    phi = torch.empty_like(f0)
    m = torch.empty((2, N, N), device=f0.device)
    p = torch.empty((2, N, N), device=f0.device)
    o = gprox.default_opts(max_iters=max_iters, tol_rel_gap=tol, gap_every=gap_every, use_graph=1)
    iters, gaps = [], []
    for i in range(len(seeds)):
        st, rep = gprox.emd_solve(h, f0[i], f1[i], m, p, phi[i], o)
        h.check(st, allow=(gprox.GP_OK, gprox.GP_ERR_MAXITER))
        iters.append(rep["iters"])
        gaps.append(rep["rel_gap"])
        if verbose and (i + 1) % 32 == 0:
            print(f"generated {i + 1}/{len(seeds)} pairs (median iterations {statistics.median(iters)})", flush=True)
    torch.cuda.synchronize()
    return f0, f1, phi, iters, gaps


def train(net: gprox.Cnn, f0, f1, phi, steps: int, batch: int, lr: float, seed: int = 0, log_every: int = 50,
          lr_final: float | None = None):
    """Adam on random mini-batches; cosine decay of the step size to lr_final."""
    rng = np.random.default_rng(seed)
    S = f0.shape[0]
    lr_final = lr * 0.05 if lr_final is None else lr_final
    hist = []
    for k in range(steps):
        idx = rng.choice(S, size=min(batch, S), replace=False)
        want = (k % log_every == 0) or k == steps - 1
        L, _ = net.loss_grad([f0[i] for i in idx], [f1[i] for i in idx], [phi[i] for i in idx], want_loss=want)
        if want:
            hist.append((k, L))
        a = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * k / max(1, steps)))
        net.adam_step(a)
    torch.cuda.synchronize()
    return hist


def test_loss(net: gprox.Cnn, f0, f1, phi, batch: int = 8):
    out = []
    for i in range(0, f0.shape[0], batch):
        j = range(i, min(i + batch, f0.shape[0]))
        L, _ = net.loss_grad([f0[k] for k in j], [f1[k] for k in j], [phi[k] for k in j])
        out.append(L * len(j))
    return sum(out) / f0.shape[0]


def evaluate(h: gprox.Handle, net: gprox.Cnn, f0, f1, tol: float = 1e-5, max_iters: int = 40000,
             gap_every: int = 10):
    """Per pair: iterations and seconds to `tol` from the zero start and from the learned start."""
    N = f0.shape[-1]
    m = torch.empty((2, N, N), device=f0.device)
    o = gprox.default_opts(max_iters=max_iters, tol_rel_gap=tol, gap_every=gap_every, use_graph=1)
    rows = []
    for i in range(f0.shape[0]):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, rz = gprox.emd_solve(h, f0[i], f1[i], m, None, None, o)
        torch.cuda.synchronize()
        tz = time.perf_counter() - t0
        h.check(st, allow=(gprox.GP_OK, gprox.GP_ERR_MAXITER))
        t0 = time.perf_counter()
        st, rw = gprox.emd_solve_learned(h, net, f0[i], f1[i], m, None, None, o)
        torch.cuda.synchronize()
        tw = time.perf_counter() - t0
        net.check(st, allow=(gprox.GP_OK, gprox.GP_ERR_MAXITER))
        rows.append({"zero_iters": rz["iters"], "zero_s": tz, "zero_gap": rz["rel_gap"],
                     "warm_iters": rw["iters"], "warm_s": tw, "warm_gap": rw["rel_gap"],
                     "used_warm": rw["used_warm"]})
    return rows


def network_cost(net: gprox.Cnn, f0, f1, reps: int = 10):
    """Mean seconds of one forward pass (B = 1) on the device."""
    net.forward([f0[0]], [f1[0]])
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        net.forward([f0[0]], [f1[0]])
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / 1e3 / reps


def summarize(rows):
    zi = [r["zero_iters"] for r in rows]
    wi = [r["warm_iters"] for r in rows]
    zs = [r["zero_s"] for r in rows]
    ws = [r["warm_s"] for r in rows]
    return {"pairs": len(rows), "median_zero_iters": statistics.median(zi), "median_warm_iters": statistics.median(wi),
            "median_zero_s": statistics.median(zs), "median_warm_s": statistics.median(ws),
            "median_iter_ratio": statistics.median([w / max(z, 1) for w, z in zip(wi, zi)]),
            "fallback_rate": sum(not r["used_warm"] for r in rows) / len(rows)}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--N", type=int, default=512)
    ap.add_argument("--C", type=int, default=32)
    ap.add_argument("--fp32", action="store_true", help="FP32 storage instead of BF16")
    ap.add_argument("--train", type=int, default=512, help="training pairs (seeds 0..)")
    ap.add_argument("--test", type=int, default=64, help="held-out pairs (seeds 1e6..)")
    ap.add_argument("--data-tol", type=float, default=1e-6)
    ap.add_argument("--data-max-iters", type=int, default=40000)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--tol", type=float, default=1e-5, help="evaluation gap")
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
    rep = {"N": a.N, "C": a.C, "bf16": not a.fp32, "params": net.num_params}
    t0 = time.perf_counter()
    f0, f1, phi, it, gaps = generate(h, a.N, range(a.train), a.data_tol, a.data_max_iters, verbose=True)
    rep["data"] = {"pairs": a.train, "seconds": time.perf_counter() - t0, "median_iters": statistics.median(it),
                   "max_gap": max(gaps)}
    g0, g1, gphi, _, _ = generate(h, a.N, range(TEST_SEED0, TEST_SEED0 + a.test), a.data_tol, a.data_max_iters)
    rep["test_loss_init"] = test_loss(net, g0, g1, gphi)
    t0 = time.perf_counter()
    hist = train(net, f0, f1, phi, a.steps, a.batch, a.lr, a.seed)
    print(f"trained {a.steps} steps in {time.perf_counter() - t0:.1f} s, loss {hist[-1][1]:.4g}", flush=True)
    rep["train"] = {"steps": a.steps, "batch": a.batch, "lr": a.lr, "seconds": time.perf_counter() - t0,
                    "loss": hist[-1][1], "history": hist}
    rep["test_loss"] = test_loss(net, g0, g1, gphi)
    rep["network_seconds"] = network_cost(net, g0, g1)
    rows = evaluate(h, net, g0, g1, a.tol)
    rep["eval"] = summarize(rows)
    rep["eval"]["tol"] = a.tol
    rep["rows"] = rows
    if a.out:
        np.savez(a.out, w=net.get_params(), C=a.C, N=a.N)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(rep, f, indent=1)
    print(json.dumps({k: v for k, v in rep.items() if k not in ("rows",)}, default=str))
    return rep


if __name__ == "__main__":
    main()
