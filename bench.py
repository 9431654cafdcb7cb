"""Benchmark of the G-prox PDHG hot path on one GB300 (or N replicas).

Workload: the 4096 x 4096 ROF problem (noisy disks + rectangle, sigma = 0.1,
lambda = 8) and the 4096 x 4096 L1-EMD problem (two 8-Gaussian mixtures with a
1e-3 floor), FP32 state, FP64 gap reductions.  One step = 10 G-prox PDHG
iterations of each problem including one duality-gap check each (the chunk a
solve runs between stopping tests).  value = grid-point-iterations per second
over the whole job (all ranks), inputs resident in HBM.  Every plane is 64 MB
and each problem's working set is ~1 GB, larger than the 129 MB L2, so no L2
flush is needed between steps.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU (torchrun): independent replicas,
one per GPU, timed between barriers (max over ranks).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grid-pt-iters/s + time to rel. gap 1e-5 at 4096² (frac. of HBM roofline)"
UNIT = "grid-pt-iters/s"
N_DEFAULT = 4096
ITERS_PER_STEP = 10
LAMBDA = 8.0

# Algorithmic DRAM bytes per grid point for one launch of each kernel class
# (FP32 words read + written, each operand touched once).
BYTES_PER_POINT = {
    "dct_rows_fwd": 8,     # read b, write row spectrum
    "dct_cols_solve": 8,   # read + write the plane in place
    "dct_rows_inv": 8,     # read spectrum, write x
    "dct_cols_grad": 12,   # read row spectrum, write A and B
    "dct_rows_grad": 16,   # read A, B; write grad x (2)   (gap checks also write phi)
    "dct_tc_split": 32,    # four GEMMs, each reads two N^2 operands and writes one (contraction-bound)
    "rof_fused": 32,       # read grad u(2), p(2), I; write p(2), r   (gap steps also read u)
    "emd_fused": 48,       # read grad q(2), s(2), p(2), g; write s(2), p(2), d  (gap steps add m(2), e)
    # N = 4096: one kernel per non-gap step = the solve's row syntheses + the step + the next
    # forward row pass (other sizes: the step + the next forward row pass, grad u / grad q read)
    "rof_step_fwd": 32,    # read A, B (column syntheses), p(2), I; write p(2), row spectrum of r
    "emd_step_fwd": 48,    # read A, B, s(2), p(2), g; write s(2), p(2), row spectrum of d
    "cp2_dual": 20,        # CP2 (section 4.1 comparison): read ubar, p(2); write p(2)
    "cp2_primal": 24,      # read u, p(2), I; write u, ubar
}

# The same per-kernel figures as the scope table of the method counts them
# (FP32 words per grid point, one read or write of each operand): every
# pass of the cosine solve 2 words; the ROF stencil step u, p(2), I in and
# p(2), r out; the EMD stencil step q, m(2), p(2), pbar(2) in and m(2),
# p(2), pbar(2), d out; a stencil step fused with the next forward row pass
# counts all of them (at N = 4096 the step kernel also runs the solve's row
# syntheses: step + two row passes).  Per iteration: ROF 13 words = 52 B, EMD
# 20 words = 80 B.
SCOPE_BYTES_PER_POINT = {
    "dct_rows_fwd": 8, "dct_cols_solve": 8, "dct_rows_inv": 8, "dct_cols_grad": 8, "dct_rows_grad": 8,
    "rof_fused": 28, "emd_fused": 56, "rof_step_fwd": 44, "emd_step_fwd": 72,
}
SCOPE_BYTES_PER_ITER = {"rof": 52, "emd": 80}

# ncu DRAM traffic (read + write bytes per launch) of the dominant kernel at
# 4096^2 (the column pass k_cols_grad_4k), from the committed summary named in
# "profile"; valid only while the source file holding that kernel is unchanged
# (sha256 prefix), else the line reports traffic null.
NCU_TRAFFIC = {
    "dct_cols_grad": {"bytes": 157.2e6, "file": "fftreg.cu", "src": "7d76152a3ad6b054",
                      "profile": "profiles/fftreg_cols_4096.md",
                      "ncu": {"dram_pct_of_peak": 14.3, "issue_active_pct": 51.5, "fma_pipe_pct": 40.5,
                              "note": "bound by FP32 issue and the shared-memory exchanges, not DRAM"}},
}


def _config(N, ws):
    """The workload both arms report (the reference arm times a bounded sample of it)."""
    return {"workload": f"ROF (lambda=8, noisy shapes) + L1-EMD (8-Gaussian mixtures) G-prox PDHG, "
                        f"{N}x{N}, {ITERS_PER_STEP} iterations of each per step incl. one gap check",
            "N": N, "iters_per_step": ITERS_PER_STEP, "parallelism": f"replicas{ws}",
            "l2": "no flush: inputs and working set (~1 GB per problem) exceed the 129 MB L2"}


def _src_hash(fname):
    path = os.path.join(ROOT, "paper_1805_09453_gb300", "csrc", fname)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.idx)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _helmholtz64(b, alpha):
    """x = (alpha - Lap_h)^{-1} b in FP64 through scipy's orthonormal DCT-II (the
    5-point Neumann Laplacian's eigenbasis, eigenvalues mu_k + mu_l,
    mu_k = 4 N^2 sin^2(pi k / 2N)): the reference of the precision study."""
    import numpy as np
    import scipy.fft as sfft

    N = b.shape[0]
    mu = 4.0 * N * N * np.sin(np.pi * np.arange(N) / (2.0 * N)) ** 2
    den = alpha + mu[:, None] + mu[None, :]
    return sfft.idctn(sfft.dctn(b.astype(np.float64), type=2, norm="ortho", workers=-1) / den,
                      type=2, norm="ortho", workers=-1)


def _bench_3d(h, dev, stream, N3, peak, cap3=5000):
    """The d = 3 instance (rof_solve3d / emd_solve3d) at N3^3: per-iteration time from two
    fixed-length solves, the line-transform pass against HBM, and the time to a gap."""
    import numpy as np
    import torch

    from paper_1805_09453_gb300 import gprox, synth

    rng = np.random.default_rng(0)
    I3 = (synth.ball_image3(N3) + 0.1 * rng.normal(size=(N3, N3, N3))).astype(np.float32)
    a0, a1 = synth.translated_balls3(N3)
    Id = torch.from_numpy(I3).to(dev)
    f0 = torch.from_numpy(a0).to(dev)
    f1 = torch.from_numpy(a1).to(dev)
    u = torch.empty_like(Id)
    m = torch.empty((3, N3, N3, N3), device=dev)
    n3 = N3 ** 3
    out = {"N": N3, "what": "rof_solve3d (noisy ball, lambda=20) and emd_solve3d (balls translated by "
                             "(1/4,1/4,1/4)); 12 line passes + 2 stencil kernels per iteration"}

    def run(kind, iters, tol=0.0, gap_every=100000):
        o = gprox.default_opts(max_iters=iters, tol_rel_gap=tol, gap_every=gap_every)
        t0 = time.perf_counter()
        if kind == "rof":
            st, rep = gprox.rof_solve3d(h, Id, u, None, 20.0, o)
        else:
            st, rep = gprox.emd_solve3d(h, f0, f1, m, None, o)
        stream.synchronize()
        return time.perf_counter() - t0, st, rep

    with torch.cuda.stream(stream):
        for kind in ("rof", "emd"):
            run(kind, 2)
            t10 = run(kind, 10)[0]
            gprox.profile(h, True)
            t40, st, rep = run(kind, 40)
            stream.synchronize()
            gprox.profile(h, False)
            pc = gprox.profile_read(h)
            it_s = (t40 - t10) / 30
            lms, ln = pc["dct3_lines"]
            avg = lms / 1e3 / max(ln, 1)
            gbs = 8 * n3 / avg / 1e9
            tol, cap = 1e-4, cap3
            tg, st, rep = run(kind, cap, tol, 0)
            out[kind] = {"value": n3 / it_s, "unit": UNIT, "ms_per_iter": it_s * 1e3,
                         "dct3_lines": {"avg_us": avg * 1e6, "launches": ln, "achieved_gbs": gbs,
                                        "frac": gbs / peak, "bytes_per_point": 8},
                         "stencil3_ms_per_iter": pc["stencil3"][0] / 40,
                         "to_gap": {"tol": tol, "seconds": tg, "iters": rep["iters"], "rel_gap": rep["rel_gap"],
                                    "primal": rep["primal"], "status": rep["status_name"], "cap": cap}}
    out["emd"]["to_gap"]["translation_length"] = float(np.sqrt(3) / 4)
    return out


def _inputs(N):
    from paper_1805_09453_gb300 import synth

    I = synth.rof_image(N, 0)
    f0, f1 = synth.gaussian_mixture_pair(N, 1)
    return I, f0, f1


def cpu_baseline_oracle(N, n_iter=1):
    """The FP64 oracle as it stands, one iteration of each problem at N (bounded sample)."""
    import numpy as np

    from oracle import gprox_oracle as O

    I, f0, f1 = _inputs(N)
    t0 = time.perf_counter()
    tau, sigma, _ = O.rof_step_rule(I, LAMBDA)
    st = O.rof_init(I)
    t1 = time.perf_counter()
    O.rof_iterate(st, I.astype(np.float64), LAMBDA, tau, sigma, n_iter)
    t2 = time.perf_counter()
    se = O.emd_init(f0, f1)
    t3 = time.perf_counter()
    O.emd_iterate(se, 1.0, 1.0, n_iter)
    t4 = time.perf_counter()
    secs = (t2 - t1) + (t4 - t3)
    return {"value": 2 * n_iter * N * N / secs, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n_iter} FP64 oracle iteration(s) of ROF and of EMD at {N}x{N} (setup excluded), "
                      f"scipy.fft with all {os.cpu_count()} host threads",
            "seconds": secs}


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle as it stands, on the host cores."""
    import numpy as np

    from oracle import gprox_oracle as O

    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    N = args.size
    I, f0, f1 = _inputs(N)
    I64 = I.astype(np.float64)
    tau, sigma, _ = O.rof_step_rule(I, LAMBDA)
    sr = O.rof_init(I64)
    se = O.emd_init(f0, f1)

    def step():
        t0 = time.perf_counter()
        O.rof_iterate(sr, I64, LAMBDA, tau, sigma, 1)
        O.emd_iterate(se, 1.0, 1.0, 1)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        step()
    t = sum(step() for _ in range(args.steps))
    value = args.steps * 2 * N * N / t
    sample = (f"each step 1 ROF + 1 EMD FP64 oracle iteration at {N}x{N} (no gap check) instead of 10 + 10; "
              f"{args.steps} steps; value per grid-point-iteration")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(N, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1805_09453_gb300 import build, gprox

    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        build.build()
    if ws > 1:
        dist.barrier()
    N = args.size
    I, f0, f1 = _inputs(N)
    Id = torch.from_numpy(I).to(dev)
    f0d = torch.from_numpy(f0).to(dev)
    f1d = torch.from_numpy(f1).to(dev)
    h = gprox.Handle(local)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        # step sizes: ROF rule (sections 3.1 / 4.1), EMD tau = sigma = 1 (section 4.2)
        u0 = torch.empty((N, N), device=dev)
        st, rep = gprox.rof_solve(h, Id, u0, None, LAMBDA, gprox.default_opts(max_iters=0, tol_rel_gap=0.0))
        h.check(st)
        tau_rof = rep["tau"]
        srof = gprox.State(h, "rof", N, I=Id, lam=LAMBDA, tau=tau_rof)
        semd = gprox.State(h, "emd", N, f0=f0d, f1=f1d, tau=1.0)

        def step():
            srof.step(ITERS_PER_STEP)
            g1 = srof.gap()
            semd.step(ITERS_PER_STEP)
            g2 = semd.gap()
            return g1, g2

        for _ in range(args.warmup):
            step()
        stream.synchronize()
        clocks = ClockSampler(local) if rank == 0 else None
        if clocks:
            clocks.start()
            time.sleep(0.3)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            g_rof, g_emd = step()
        e1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        cl = clocks.stop() if clocks else None
        ms = e0.elapsed_time(e1)
        # per-kernel device times: the same steps again with the library's launch
        # profiler on (CUDA events around every launch; it disables graph replay,
        # which costs ~3 % of the step time, so it stays out of the timed window)
        prof_steps = max(1, min(args.steps, 20))
        gprox.profile(h, True)
        for _ in range(prof_steps):
            step()
        torch.cuda.synchronize()
        gprox.profile(h, False)
        prof = gprox.profile_read(h)
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if ws > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    units = ws * args.steps * 2 * ITERS_PER_STEP * N * N
    value = units / (ms_max / 1e3)

    # roofline of the dominant kernel (largest summed device time)
    peak, peak_kind = _peaks()
    name = max((k for k in prof if k in BYTES_PER_POINT), key=lambda k: prof[k][0])
    kms, kn = prof[name]
    avg_s = kms / 1e3 / max(kn, 1)
    bytes_launch = BYTES_PER_POINT[name] * N * N
    achieved = bytes_launch / avg_s / 1e9
    tr = NCU_TRAFFIC.get(name)
    fresh = bool(tr and tr.get("src") == _src_hash(tr["file"]))
    traffic = tr["bytes"] if fresh else None
    scope_launch = SCOPE_BYTES_PER_POINT[name] * N * N
    roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                "bytes_per_launch": bytes_launch, "avg_launch_ms": avg_s * 1e3,
                "scope_bytes_per_launch": scope_launch,
                "frac_scope_bytes": scope_launch / avg_s / 1e9 / peak,
                "timing": f"CUDA events around every launch over {prof_steps} steps run right after the timed window"}
    if fresh and "ncu" in tr:  # the same capture's view of what bounds the kernel
        roofline["ncu"] = dict(tr["ncu"], source=tr["profile"])
    kernels = {k: {"ms_total": v[0], "launches": v[1], "avg_us": 1e3 * v[0] / v[1]} for k, v in prof.items() if v[1]}
    # kernels launched inside the timed window: the profiled pass runs the same steps (the timed
    # window replays them from CUDA graphs, kernel for kernel)
    launches = int(round(sum(v[1] for v in prof.values()) * args.steps / prof_steps))

    # whole-step HBM fraction: algorithmic bytes of every pass the step launches (profiled pass,
    # per step) over the step time
    step_bytes = sum(BYTES_PER_POINT[k] * v[1] for k, v in prof.items() if k in BYTES_PER_POINT) * N * N / prof_steps
    whole_frac = (step_bytes * args.steps / (ms_max / 1e3) / 1e9) / peak
    # the same over the scope table's per-iteration bytes (ROF 52 B, EMD 80 B per point)
    scope_step = (SCOPE_BYTES_PER_ITER["rof"] + SCOPE_BYTES_PER_ITER["emd"]) * ITERS_PER_STEP * N * N
    whole_frac_scope = (scope_step * args.steps / (ms_max / 1e3) / 1e9) / peak

    # end to end through the public solve calls with host (pinned) buffers: every step copies
    # its inputs in and its results out; the copies run on their own streams into / out of
    # double-buffered device arrays, so that step k+1's inputs arrive and step k's results
    # leave while the solves compute
    e2e = None
    if not args.no_e2e:
        Ih = torch.from_numpy(I).pin_memory()
        f0h = torch.from_numpy(f0).pin_memory()
        f1h = torch.from_numpy(f1).pin_memory()
        uh = torch.empty((N, N), dtype=torch.float32).pin_memory()
        mh = torch.empty((2, N, N), dtype=torch.float32).pin_memory()
        dbuf = [{"I": torch.empty_like(Id), "f0": torch.empty_like(f0d), "f1": torch.empty_like(f1d),
                 "u": torch.empty((N, N), device=dev), "m": torch.empty((2, N, N), device=dev)} for _ in range(2)]
        h2d, d2h = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        opts = gprox.default_opts(max_iters=ITERS_PER_STEP, gap_every=ITERS_PER_STEP, tol_rel_gap=0.0, use_graph=1)
        ke = max(1, min(args.steps, 20))

        def load(k):  # step k's inputs -> buffer set k % 2; event marks arrival
            b = dbuf[k % 2]
            with torch.cuda.stream(h2d):
                if "free" in b:  # the previous results of this set have left
                    h2d.wait_event(b["free"])
                b["I"].copy_(Ih, non_blocking=True)
                b["f0"].copy_(f0h, non_blocking=True)
                b["f1"].copy_(f1h, non_blocking=True)
                b["in"] = torch.cuda.Event()
                b["in"].record(h2d)

        def e2e_run(steps):
            load(0)
            for k in range(steps):
                b = dbuf[k % 2]
                if k + 1 < steps:
                    load(k + 1)
                stream.wait_event(b["in"])
                with torch.cuda.stream(stream):
                    h.check(gprox.rof_solve(h, b["I"], b["u"], None, LAMBDA, opts)[0])
                    eu = torch.cuda.Event()
                    eu.record(stream)
                    with torch.cuda.stream(d2h):
                        d2h.wait_event(eu)
                        uh.copy_(b["u"], non_blocking=True)
                    h.check(gprox.emd_solve(h, b["f0"], b["f1"], b["m"], None, None, opts)[0])
                    em = torch.cuda.Event()
                    em.record(stream)
                with torch.cuda.stream(d2h):
                    d2h.wait_event(em)
                    mh.copy_(b["m"], non_blocking=True)
                    b["free"] = torch.cuda.Event()
                    b["free"].record(d2h)
            torch.cuda.synchronize()

        e2e_run(2)
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_run(ke)
        te = torch.tensor([time.perf_counter() - t0], device=dev, dtype=torch.float64)
        if ws > 1:
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
        e2e = {"value": ws * ke * 2 * ITERS_PER_STEP * N * N / float(te.item()), "unit": UNIT,
               "h2d_bytes_per_step": 3 * N * N * 4, "d2h_bytes_per_step": 3 * N * N * 4,
               "steps": ke, "what": "rof_solve + emd_solve (10 iterations each, setup included, CUDA graphs on) "
                                    "from pinned host inputs, u and m copied back; copies overlapped with the "
                                    "solves through double-buffered device arrays"}

    # time to relative gap 1e-5 (solve calls from device inputs, CUDA graphs on, the adaptive
    # gap-check schedule: checks thin out far from the tolerance)
    ttg = None
    if not args.no_ttg:
        ttg = {}
        cert = ("stops once the corrected flux m + grad Lap^-1((f0-f1) - div m), feasible to "
                "mass_residual_feasible, is within rel. 1e-5 of the best dual bound met (the iterates' p at "
                "the checks and windowed averages of them)")

        def emd_row(rep, sec):
            return {"seconds": sec, "iters": rep["iters"], "status": rep["status_name"],
                    "rel_gap_feasible": rep["rel_gap_feasible"], "primal": rep["primal"],
                    "primal_feasible": rep["primal_feasible"], "dual": rep["dual"], "rel_gap": rep["rel_gap"],
                    "mass_residual": rep["mass_residual"], "mass_residual_feasible": rep["mass_residual_feasible"]}

        with torch.cuda.stream(stream):
            m = torch.empty((2, N, N), device=dev)
            o = gprox.default_opts(max_iters=args.ttg_cap, tol_rel_gap=1e-5, gap_every=0, use_graph=1)
            u = torch.empty((N, N), device=dev)
            # ROF: a check every 10 iterations (its gap terms come with the fused step: no extra solve)
            o10 = gprox.default_opts(max_iters=args.ttg_cap, tol_rel_gap=1e-5, gap_every=10, use_graph=1)
            stream.synchronize()
            t0 = time.perf_counter()
            st, rep = gprox.rof_solve(h, Id, u, None, LAMBDA, o10)
            ttg["rof"] = {"seconds": time.perf_counter() - t0, "iters": rep["iters"], "rel_gap": rep["rel_gap"],
                          "status": rep["status_name"], "tau": rep["tau"]}
            t0 = time.perf_counter()
            st, rep = gprox.emd_solve(h, f0d, f1d, m, None, None, o)
            ttg["emd"] = dict(emd_row(rep, time.perf_counter() - t0), certificate=cert, cap=args.ttg_cap)
            for tol, key in ((1e-4, "emd_1e-4"), (2e-5, "emd_2e-5")):  # the looser tolerances
                o4 = gprox.default_opts(max_iters=args.ttg_cap, tol_rel_gap=tol, gap_every=0, use_graph=1)
                t0 = time.perf_counter()
                st, rep = gprox.emd_solve(h, f0d, f1d, m, None, None, o4)
                ttg[key] = emd_row(rep, time.perf_counter() - t0)
            if N % 64 == 0:
                # warm-started form: the EMD solved 4x coarser to gap 1e-5, interpolated, as the start
                # (emd_solve_learned with a network whose output is its prior; the duality gap at
                # n = 0 picks between that start and zero)
                base = gprox.Cnn(h, 1, seed=0)
                base.set_params(np.zeros(base.num_params, np.float32))
                oc = gprox.default_opts(max_iters=200000, tol_rel_gap=1e-5, gap_every=0, use_graph=1)
                stream.synchronize()
                t0 = time.perf_counter()
                st, rep = gprox.emd_solve_learned(h, base, f0d, f1d, m, None, None, o, 4, oc)
                sec = time.perf_counter() - t0
                # the network's output is exactly its prior here, so a start it wins is the prior's
                start = "prior" if rep["start"] in ("learned", "prior") else rep["start"]
                ttg["emd_coarse_start"] = dict(emd_row(rep, sec), start=start, coarse_factor=4, coarse_tol=1e-5,
                                               speedup=ttg["emd"]["seconds"] / sec)
                base.close()

    # batched solve: 64 independent EMD pairs of sizes drawn from {256, 512, 1024, 2048}^2,
    # 200 iterations each (set-up included), one emd_solve_batched call against the same
    # pairs solved one at a time
    batched = None
    if not args.no_batched and rank == 0:
        import numpy as np

        from paper_1805_09453_gb300 import synth

        rng = np.random.default_rng(3)
        sizes = [int(x) for x in rng.choice([256, 512, 1024, 2048], size=64)]
        bf0, bf1, bm = [], [], []
        for b, Nb in enumerate(sizes):
            a0, a1 = synth.gaussian_mixture_pair(Nb, 5000 + b)
            bf0.append(torch.from_numpy(a0).to(dev))
            bf1.append(torch.from_numpy(a1).to(dev))
            bm.append(torch.empty((2, Nb, Nb), device=dev))
        ob = gprox.default_opts(max_iters=200, tol_rel_gap=0.0, gap_every=10, use_graph=1)
        pts = sum(Nb * Nb for Nb in sizes) * 200
        with torch.cuda.stream(stream):
            gprox.emd_solve_batched(h, bf0, bf1, bm, ob)  # captures the chunk graph
            stream.synchronize()
            t0 = time.perf_counter()
            st, reps = gprox.emd_solve_batched(h, bf0, bf1, bm, ob)
            stream.synchronize()
            tb = time.perf_counter() - t0
            for b in range(len(sizes)):  # first use of each size: plans, states, graphs
                gprox.emd_solve(h, bf0[b], bf1[b], bm[b], None, None, ob)
            stream.synchronize()
            t0 = time.perf_counter()
            for b in range(len(sizes)):
                gprox.emd_solve(h, bf0[b], bf1[b], bm[b], None, None, ob)
            stream.synchronize()
            ts = time.perf_counter() - t0
            # the same batch to relative gap 1e-5: every pair stops at its own gap; the call
            # returns when the slowest pair is done
            og = gprox.default_opts(max_iters=40000, tol_rel_gap=1e-5, gap_every=10, use_graph=1)
            t0 = time.perf_counter()
            stg, reps_g = gprox.emd_solve_batched(h, bf0, bf1, bm, og)
            stream.synchronize()
            tg = time.perf_counter() - t0
        slow = max(range(len(sizes)), key=lambda b: reps_g[b]["iters"])
        to_gap = {"seconds": tg, "status": gprox.STATUS_NAMES[stg],
                  "slowest_pair": {"N": sizes[slow], "iters": reps_g[slow]["iters"]},
                  "median_iters": {str(n): statistics.median([r["iters"] for b, r in enumerate(reps_g) if sizes[b] == n])
                                   for n in (256, 512, 1024, 2048) if n in sizes},
                  "not_ok": sum(r["status"] != gprox.GP_OK for r in reps_g)}
        batched = {"pairs": len(sizes), "sizes": {str(n): sizes.count(n) for n in (256, 512, 1024, 2048)},
                   "iters": 200, "status": gprox.STATUS_NAMES[st], "seconds": tb,
                   "value": pts / tb, "unit": UNIT, "sequential_seconds": ts, "sequential_value": pts / ts,
                   "speedup": ts / tb, "to_gap_1e-5": to_gap,
                   "what": "emd_solve_batched (one CUDA graph per chunk, a branch per "
                           "problem) vs emd_solve per pair; set-up included"}
        del bf0, bf1, bm

    # CP2, the accelerated PDHG the paper compares with (section 4.1): the same ROF problem,
    # no linear solve, two stencil passes per iteration; throughput and its roofline, and the
    # gap it reaches in a fixed budget of iterations against the G-prox solve's time to 1e-5
    cp2 = None
    if not args.no_cp2 and rank == 0:
        u2 = torch.empty((N, N), device=dev)
        with torch.cuda.stream(stream):
            o2 = gprox.default_opts(max_iters=50, tol_rel_gap=0.0, gap_every=50)
            h.check(gprox.rof_solve_cp2(h, Id, u2, None, LAMBDA, o2)[0])
            stream.synchronize()
            gprox.profile(h, True)
            o2 = gprox.default_opts(max_iters=200, tol_rel_gap=0.0, gap_every=200)
            st, rep = gprox.rof_solve_cp2(h, Id, u2, None, LAMBDA, o2)
            stream.synchronize()
            gprox.profile(h, False)
            pc = gprox.profile_read(h)
            kern = {}
            for k in ("cp2_dual", "cp2_primal"):
                kms, kn = pc[k]
                avg = kms / 1e3 / max(kn, 1)
                gbs = BYTES_PER_POINT[k] * N * N / avg / 1e9
                kern[k] = {"avg_us": avg * 1e6, "achieved_gbs": gbs, "frac": gbs / peak}
            it_s = (pc["cp2_dual"][0] + pc["cp2_primal"][0]) / 1e3 / max(pc["cp2_dual"][1], 1)
            o2 = gprox.default_opts(max_iters=args.cp2_iters, tol_rel_gap=1e-5, gap_every=100)
            t0 = time.perf_counter()
            st, rep = gprox.rof_solve_cp2(h, Id, u2, None, LAMBDA, o2)
            stream.synchronize()
            sec = time.perf_counter() - t0
        cp2 = {"kernels": kern, "value": N * N / it_s, "unit": UNIT, "bytes_per_point_iteration": 44,
               "to_gap_1e-5": {"seconds": sec, "iters": rep["iters"], "rel_gap": rep["rel_gap"],
                               "status": rep["status_name"], "cap": args.cp2_iters},
               "gprox_to_gap_1e-5": ttg.get("rof") if ttg else None,
               "what": "rof_solve_cp2 (section 4.1 comparison method) on the bench's ROF image, lambda=8"}

    # split-precision study (FP32 fast transform vs hi+lo BF16 tensor-core GEMMs): the FP64
    # residual of the discrete equation (alpha - Lap_h) x = b for each solve, and the split
    # solve's distance from the FP32 one
    prec_study = None
    if not args.no_prec and rank == 0:
        bp = np.ascontiguousarray(I[:, :], dtype=np.float32)
        bd = torch.from_numpy(bp).to(dev)
        xo = torch.empty_like(bd)
        prec_study = {"solve": f"(50 - Lap)^-1 I at {N}x{N}",
                      "error": "relative L2 distance from an FP64 scipy DCT-II solve of the same system"}
        x64 = _helmholtz64(bp, 50.0)
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {"bf16_tflops": 1900.0}
        x32 = None
        with torch.cuda.stream(stream):
            for prec in ("fp32", "split_bf16", "split_fp16", "split_bf16_refined", "split_fp16_refined"):
                for _ in range(2):
                    h.check(gprox.dct2_poisson(h, bd, xo, 50.0, prec=prec))
                stream.synchronize()
                a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                for _ in range(3):
                    gprox.dct2_poisson(h, bd, xo, 50.0, prec=prec)
                a1.record(stream)
                stream.synchronize()
                ms_s = a0.elapsed_time(a1) / 3
                x = xo.cpu().numpy().astype(np.float64)
                row = {"ms": ms_s, "rel_l2_err": float(np.linalg.norm(x - x64) / np.linalg.norm(x64))}
                if prec == "fp32":
                    x32 = x
                else:
                    gemms = 4 * (2 if prec.endswith("refined") else 1)
                    tf = gemms * 3 * 2.0 * N ** 3 / (ms_s / 1e3) / 1e12
                    row.update({"rel_l2_vs_fp32": float(np.linalg.norm(x - x32) / np.linalg.norm(x32)),
                                "tflops": tf, "bf16_peak_tflops": float(pk.get("bf16_tflops", 1900.0)),
                                "tensor_frac": tf / float(pk.get("bf16_tflops", 1900.0))})
                prec_study[prec] = row
            # the ROF solve to relative gap 1e-5 with each transform (config 2's time to gap)
            u3 = torch.empty((N, N), device=dev)
            ttg_prec = {}
            for prec in ("fp32", "split_bf16", "split_fp16", "split_bf16_refined", "split_fp16_refined"):
                o3 = gprox.default_opts(max_iters=3000, tol_rel_gap=1e-5, gap_every=10, prec=prec)
                t0 = time.perf_counter()
                st3, r3 = gprox.rof_solve(h, Id, u3, None, LAMBDA, o3)
                stream.synchronize()
                ttg_prec[prec] = {"seconds": time.perf_counter() - t0, "iters": r3["iters"],
                                  "rel_gap": r3["rel_gap"], "primal": r3["primal"], "status": r3["status_name"]}
            prec_study["rof_time_to_gap_1e-5"] = ttg_prec

    three_d = None
    if not args.no_3d and rank == 0:
        three_d = _bench_3d(h, dev, stream, args.size3, peak, args.ttg3_cap)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": _config(N, ws),
            "roofline": roofline, "whole_iteration_hbm_frac": whole_frac,
            "whole_iteration_hbm_frac_scope_bytes": whole_frac_scope, "kernels": kernels,
            "gpu_launches": launches, "clocks": cl, "e2e": e2e, "time_to_gap": ttg, "batched": batched,
            "precision_study": prec_study, "cp2": cp2, "three_d": three_d,
            "last_gap": {"rof": g_rof["rel_gap"], "emd": g_emd["rel_gap"]}}
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_oracle(N, 1)
        line["cpu_baseline"].pop("seconds", None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    srof.close()
    semd.close()
    h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=N_DEFAULT)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ttg", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-prec", action="store_true")
    ap.add_argument("--no-cp2", action="store_true")
    ap.add_argument("--cp2-iters", type=int, default=20000)
    ap.add_argument("--ttg-cap", type=int, default=200000)
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--size3", type=int, default=256)
    ap.add_argument("--ttg3-cap", type=int, default=5000, help="iteration cap of the 3-D runs to a gap")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
