"""Thin ctypes binding of the C ABI in ``include/gprox.h``.

Argument marshalling only: every step of the method runs in the CUDA library
``_lib/libgprox.so``.  Arrays are torch CUDA tensors (float32, contiguous);
their device pointers and the current torch stream are passed through.  If the
library is missing, loading fails loudly -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libgprox.so")
_lib = None

GP_OK, GP_ERR_ARG, GP_ERR_CUDA, GP_ERR_MAXITER, GP_ERR_NONFINITE, GP_ERR_DIVERGED, GP_ERR_MASS, GP_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = {0: "GP_OK", 1: "GP_ERR_ARG", 2: "GP_ERR_CUDA", 3: "GP_ERR_MAXITER", 4: "GP_ERR_NONFINITE",
                5: "GP_ERR_DIVERGED", 6: "GP_ERR_MASS", 7: "GP_ERR_UNSUPPORTED"}
PREC = {"fp32": 0, "split_bf16": 1, "split_fp16": 2, "split_bf16_refined": 3, "split_fp16_refined": 4}
ABI_VERSION = 2  # GP_ABI_VERSION of include/gprox.h that these signatures follow

EXPORTS = ["gp_abi_version", "gp_default_opts", "gp_create", "gp_destroy", "gp_last_error", "dct2_poisson",
           "rof_solve", "emd_solve", "gp_state_create_rof", "gp_state_create_emd", "pd_step", "gp_state_read",
           "gp_state_gap", "gp_state_destroy", "gp_profile", "gp_profile_kernels", "gp_profile_query",
           "dct2_poisson_static", "dct2_poisson_grad", "emd_solve_batched", "gp_autotune", "gp_tuned_row_block",
           "gp_cnn_create", "gp_cnn_destroy", "gp_cnn_last_error", "gp_cnn_num_params", "gp_cnn_get_params",
           "gp_cnn_set_params", "gp_cnn_forward", "gp_cnn_loss_grad", "gp_cnn_adam_step", "emd_solve_learned",
           "emd_coarse_start", "gp_gap_schedule_next", "gp_rof_image_stats", "gp_state_average",
           "gp_state_read_average", "rof_solve_cp2", "rof_solve3d", "emd_solve3d", "gp_state_certify",
           "rof_coarse_start", "rof_solve_learned", "gp_rof_step_tau", "gp_emd_delta_tau"]


class Opts(C.Structure):
    _fields_ = [("max_iters", C.c_int), ("gap_every", C.c_int), ("tol_rel_gap", C.c_double),
                ("tau", C.c_double), ("sigma", C.c_double), ("tau_scale", C.c_double), ("eps", C.c_double),
                ("prec", C.c_int), ("use_graph", C.c_int), ("warm_start", C.c_int)]


class Report(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("primal", C.c_double), ("dual", C.c_double),
                ("rel_gap", C.c_double), ("mass_residual", C.c_double), ("tau", C.c_double),
                ("sigma", C.c_double), ("seconds", C.c_double), ("primal_feasible", C.c_double),
                ("rel_gap_feasible", C.c_double), ("mass_residual_feasible", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class GproxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """Load libgprox.so (built by ``paper_1805_09453_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with `python -m paper_1805_09453_gb300.build`")
    L = C.CDLL(_LIB_PATH)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    L.gp_abi_version.restype = i
    if L.gp_abi_version() != ABI_VERSION:
        raise RuntimeError(f"{_LIB_PATH} has ABI {L.gp_abi_version()}, the binding expects {ABI_VERSION}: rebuild it")
    L.gp_default_opts.argtypes = [C.POINTER(Opts)]
    L.gp_create.argtypes = [C.POINTER(vp), i]
    L.gp_destroy.argtypes = [vp]
    L.gp_last_error.argtypes = [vp]
    L.gp_last_error.restype = C.c_char_p
    L.dct2_poisson.argtypes = [vp, vp, vp, i, d, i, vp]
    L.rof_solve.argtypes = [vp, vp, vp, vp, i, d, C.POINTER(Opts), C.POINTER(Report), vp]
    L.rof_solve_cp2.argtypes = [vp, vp, vp, vp, i, d, C.POINTER(Opts), C.POINTER(Report), vp]
    L.emd_solve.argtypes = [vp, vp, vp, vp, vp, vp, i, C.POINTER(Opts), C.POINTER(Report), vp]
    L.gp_state_create_rof.argtypes = [vp, C.POINTER(vp), vp, i, d, d, d, vp, vp, vp, vp]
    L.gp_state_create_emd.argtypes = [vp, C.POINTER(vp), vp, vp, i, d, d, vp, vp, vp, vp]
    L.pd_step.argtypes = [vp, vp, i, i, vp]
    L.gp_state_read.argtypes = [vp, vp, vp, vp, vp]
    L.gp_state_gap.argtypes = [vp, vp, C.POINTER(Report), vp]
    L.gp_state_certify.argtypes = [vp, vp, C.POINTER(Report), vp]
    L.gp_state_destroy.argtypes = [vp]
    L.dct2_poisson_static.argtypes = [vp, vp, i, d, vp]
    L.dct2_poisson_grad.argtypes = [vp, vp, vp, i, d, i, vp]
    L.gp_autotune.argtypes = [vp, i, C.c_char_p, vp]
    L.gp_tuned_row_block.argtypes = [vp, C.c_char_p, i]
    L.gp_tuned_row_block.restype = i
    L.emd_solve_batched.argtypes = [vp, i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp),
                                    C.POINTER(i), C.POINTER(Opts), C.POINTER(Report), vp]
    L.gp_profile.argtypes = [vp, i]
    L.gp_cnn_create.argtypes = [vp, i, i, C.c_ulonglong, C.POINTER(vp)]
    L.gp_cnn_destroy.argtypes = [vp]
    L.gp_cnn_last_error.argtypes = [vp]
    L.gp_cnn_last_error.restype = C.c_char_p
    L.gp_cnn_num_params.argtypes = [vp]
    L.gp_cnn_num_params.restype = C.c_longlong
    L.gp_cnn_get_params.argtypes = [vp, vp]
    L.gp_cnn_set_params.argtypes = [vp, vp]
    L.gp_cnn_forward.argtypes = [vp, i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), i, vp, vp]
    L.gp_cnn_loss_grad.argtypes = [vp, i, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), i,
                                   C.POINTER(d), vp, vp]
    L.gp_cnn_adam_step.argtypes = [vp, d, vp]
    L.emd_solve_learned.argtypes = [vp, vp, vp, vp, vp, vp, vp, i, i, C.POINTER(Opts), C.POINTER(Opts),
                                    C.POINTER(Report), C.POINTER(i), vp]
    L.emd_coarse_start.argtypes = [vp, vp, vp, i, i, C.POINTER(Opts), vp, C.POINTER(Report), vp]
    L.rof_coarse_start.argtypes = [vp, vp, i, i, d, C.POINTER(Opts), vp, vp, C.POINTER(Report), vp]
    L.rof_solve_learned.argtypes = [vp, vp, vp, vp, vp, i, d, i, C.POINTER(Opts), C.POINTER(Opts),
                                    C.POINTER(Report), C.POINTER(i), vp]
    L.gp_gap_schedule_next.argtypes = [i, d, i, d, d]
    L.gp_state_average.argtypes = [vp, vp, i, vp]
    L.gp_state_read_average.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_longlong), vp]
    L.gp_rof_image_stats.argtypes = [vp, vp, i, C.POINTER(d), vp]
    L.rof_solve3d.argtypes = [vp, vp, vp, vp, i, d, C.POINTER(Opts), C.POINTER(Report), vp]
    L.emd_solve3d.argtypes = [vp, vp, vp, vp, vp, i, C.POINTER(Opts), C.POINTER(Report), vp]
    L.gp_rof_step_tau.argtypes = [C.POINTER(d), d, d, i]
    L.gp_emd_delta_tau.argtypes = [i, d, i]
    L.gp_profile_kernels.restype = i
    L.gp_profile_query.argtypes = [vp, i, C.POINTER(C.c_char_p), C.POINTER(d), C.POINTER(C.c_longlong)]
    for name in EXPORTS:
        if name not in ("gp_abi_version", "gp_default_opts", "gp_last_error", "gp_profile_kernels",
                        "gp_tuned_row_block", "gp_cnn_last_error", "gp_cnn_num_params", "gp_rof_step_tau",
                        "gp_emd_delta_tau"):
            getattr(L, name).restype = i
    L.gp_rof_step_tau.restype = d
    L.gp_emd_delta_tau.restype = d
    _lib = L
    return L


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("expected a contiguous float32 tensor")
    return C.c_void_p(t.data_ptr())


def _side(t, name="array"):
    """Grid side N of an (N, N) tensor (ValueError for any other shape)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if t.dim() != 2 or t.shape[0] != t.shape[1]:
        raise ValueError(f"{name}: expected an (N, N) grid, got shape {tuple(t.shape)}")
    return int(t.shape[-1])


def _shape(t, shape, name):
    """Require t (if given) to have exactly `shape`: the library reads and
    writes N*N (or 2*N*N) floats through the pointer, so a smaller tensor
    would be overrun."""
    if t is None:
        return
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().gp_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = PREC[v]
        setattr(o, k, v)
    return o


class Handle:
    """Owns a gp_handle (workspace, cosine-transform tables, scratch)."""

    def __init__(self, device: int | None = None):
        if device is None:
            device = torch.cuda.current_device()
        self._h = C.c_void_p()
        st = lib().gp_create(C.byref(self._h), int(device))
        if st != GP_OK:
            raise GproxError(st, "gp_create failed")
        self.device = device

    @property
    def ptr(self):
        return self._h

    def last_error(self) -> str:
        return lib().gp_last_error(self._h).decode()

    def check(self, st, allow=(GP_OK,)):
        if st not in allow:
            raise GproxError(st, self.last_error())
        return st

    def close(self):
        if self._h:
            lib().gp_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dct2_poisson(h: Handle, b, x, alpha: float, prec="fp32", stream=None) -> int:
    """x = (alpha - Lap)^{-1} b (Neumann) -- see include/gprox.h."""
    N = _side(b, "b")
    _shape(x, (N, N), "x")
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    return lib().dct2_poisson(h.ptr, _ptr(b), _ptr(x), int(N), float(alpha), p, _stream(stream))


def dct2_poisson_grad(h: Handle, b, g, alpha: float, prec="fp32", stream=None) -> int:
    """g (2, N, N) = forward-difference gradient of (alpha - Lap)^{-1} b -- see include/gprox.h."""
    N = _side(b, "b")
    _shape(g, (2, N, N), "g")
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    return lib().dct2_poisson_grad(h.ptr, _ptr(b), _ptr(g), int(N), float(alpha), p, _stream(stream))


def dct2_poisson_static(b, x, alpha: float, stream=None) -> int:
    """dct2_poisson without device allocation (static scratch, N <= 1024) -- see include/gprox.h."""
    N = _side(b, "b")
    _shape(x, (N, N), "x")
    return lib().dct2_poisson_static(_ptr(b), _ptr(x), N, float(alpha), _stream(stream))


def static_last_error() -> str:
    """Error text of the last failed handle-free call on this thread."""
    return lib().gp_last_error(None).decode()


def rof_solve(h: Handle, I, u, p=None, lam: float = 8.0, opts: Opts | None = None, stream=None):
    """ROF G-prox PDHG solve; returns (status, report dict)."""
    N = _side(I, "I")
    _shape(u, (N, N), "u")
    _shape(p, (2, N, N), "p")
    rep = Report()
    st = lib().rof_solve(h.ptr, _ptr(I), _ptr(u), _ptr(p), N, float(lam),
                         C.byref(opts) if opts is not None else None, C.byref(rep), _stream(stream))
    return st, rep.as_dict()


def rof_solve_cp2(h: Handle, I, u, p=None, lam: float = 8.0, opts: Opts | None = None, stream=None):
    """ROF by the accelerated PDHG comparison method (CP2) of section 4.1; returns (status, report dict)."""
    N = _side(I, "I")
    _shape(u, (N, N), "u")
    _shape(p, (2, N, N), "p")
    rep = Report()
    st = lib().rof_solve_cp2(h.ptr, _ptr(I), _ptr(u), _ptr(p), N, float(lam),
                             C.byref(opts) if opts is not None else None, C.byref(rep), _stream(stream))
    return st, rep.as_dict()


def emd_solve(h: Handle, f0, f1, m, p=None, phi=None, opts: Opts | None = None, stream=None):
    """L1 EMD G-prox PDHG solve; returns (status, report dict)."""
    N = _side(f0, "f0")
    _shape(f1, (N, N), "f1")
    _shape(m, (2, N, N), "m")
    _shape(p, (2, N, N), "p")
    _shape(phi, (N, N), "phi")
    rep = Report()
    st = lib().emd_solve(h.ptr, _ptr(f0), _ptr(f1), _ptr(m), _ptr(p), _ptr(phi), N,
                         C.byref(opts) if opts is not None else None, C.byref(rep), _stream(stream))
    return st, rep.as_dict()


def _side3(t, name="array"):
    """Grid side N of an (N, N, N) tensor (ValueError for any other shape)."""
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch tensor")
    if t.dim() != 3 or not (t.shape[0] == t.shape[1] == t.shape[2]):
        raise ValueError(f"{name}: expected an (N, N, N) volume, got shape {tuple(t.shape)}")
    return int(t.shape[-1])


def rof_solve3d(h: Handle, I, u, p=None, lam: float = 8.0, opts: Opts | None = None, stream=None):
    """ROF G-prox PDHG on an (N, N, N) volume (z, y, x); p is (3, N, N, N); returns (status, report dict)."""
    N = _side3(I, "I")
    _shape(u, (N, N, N), "u")
    _shape(p, (3, N, N, N), "p")
    rep = Report()
    st = lib().rof_solve3d(h.ptr, _ptr(I), _ptr(u), _ptr(p), N, float(lam),
                           C.byref(opts) if opts is not None else None, C.byref(rep), _stream(stream))
    return st, rep.as_dict()


def emd_solve3d(h: Handle, f0, f1, m, p=None, opts: Opts | None = None, stream=None):
    """L1 EMD G-prox PDHG on (N, N, N) densities; m and p are (3, N, N, N); returns (status, report dict)."""
    N = _side3(f0, "f0")
    _shape(f1, (N, N, N), "f1")
    _shape(m, (3, N, N, N), "m")
    _shape(p, (3, N, N, N), "p")
    rep = Report()
    st = lib().emd_solve3d(h.ptr, _ptr(f0), _ptr(f1), _ptr(m), _ptr(p), N,
                           C.byref(opts) if opts is not None else None, C.byref(rep), _stream(stream))
    return st, rep.as_dict()


def emd_solve_batched(h: Handle, f0s, f1s, ms, opts: Opts | None = None, stream=None, ps=None):
    """Batched EMD solve of independent problems; returns (status, [report dicts]).
    ms[b] (and ps[b] when ps is given) receive each problem's last m (and p).

    `stream` (or the current torch stream) must not be the default stream."""
    B = len(f0s)
    if len(f1s) != B or len(ms) != B or (ps is not None and len(ps) != B):
        raise ValueError("f0s, f1s, ms (and ps) must have one entry per problem")
    sides = []
    for b in range(B):
        N = _side(f0s[b], f"f0s[{b}]")
        _shape(f1s[b], (N, N), f"f1s[{b}]")
        _shape(ms[b], (2, N, N), f"ms[{b}]")
        if ps is not None:
            _shape(ps[b], (2, N, N), f"ps[{b}]")
        sides.append(N)
    P = C.c_void_p * B
    reps = (Report * B)()
    Ns = (C.c_int * B)(*sides)
    st = lib().emd_solve_batched(h.ptr, B, P(*[_ptr(x) for x in f0s]), P(*[_ptr(x) for x in f1s]),
                                 P(*[_ptr(x) for x in ms]), P(*[_ptr(x) for x in ps]) if ps is not None else None,
                                 Ns, C.byref(opts) if opts is not None else None, reps, _stream(stream))
    return st, [r.as_dict() for r in reps]


class State:
    """An explicit G-prox PDHG state (gp_state) for step-by-step driving."""

    def __init__(self, h: Handle, kind: str, N: int, *, I=None, lam=None, f0=None, f1=None, tau=1.0, sigma=None,
                 primal0=None, p0=None, pbar0=None, stream=None):
        self.h = h
        self.kind = kind
        self.N = N
        self._s = C.c_void_p()
        sigma = 1.0 / tau if sigma is None else sigma
        self._keep = (I, f0, f1)  # inputs must outlive the state
        for t, nm in ((I, "I"), (f0, "f0"), (f1, "f1")):
            _shape(t, (N, N), nm)
        for t, nm in ((p0, "p0"), (pbar0, "pbar0")):
            _shape(t, (2, N, N), nm)
        _shape(primal0, (N, N) if kind == "rof" else (2, N, N), "primal0")
        if kind == "rof":
            st = lib().gp_state_create_rof(h.ptr, C.byref(self._s), _ptr(I), int(N), float(lam), float(tau),
                                           float(sigma), _ptr(primal0), _ptr(p0), _ptr(pbar0), _stream(stream))
        elif kind == "emd":
            st = lib().gp_state_create_emd(h.ptr, C.byref(self._s), _ptr(f0), _ptr(f1), int(N), float(tau),
                                           float(sigma), _ptr(primal0), _ptr(p0), _ptr(pbar0), _stream(stream))
        else:
            raise ValueError(kind)
        h.check(st)

    def step(self, n: int, prec="fp32", stream=None) -> int:
        p = PREC[prec] if isinstance(prec, str) else int(prec)
        return self.h.check(lib().pd_step(self.h.ptr, self._s, int(n), p, _stream(stream)))

    def read(self, stream=None):
        N = self.N
        dev = torch.device("cuda", self.h.device)
        prim = torch.empty((N, N) if self.kind == "rof" else (2, N, N), device=dev, dtype=torch.float32)
        p = torch.empty((2, N, N), device=dev, dtype=torch.float32)
        self.h.check(lib().gp_state_read(self.h.ptr, self._s, _ptr(prim), _ptr(p), _stream(stream)))
        return prim, p

    def average(self, enable: bool = True, stream=None) -> int:
        """Start (restart) or stop the ergodic averages of this state's iterates."""
        return self.h.check(lib().gp_state_average(self.h.ptr, self._s, int(bool(enable)), _stream(stream)))

    def read_average(self, stream=None):
        """(primal average, p average, number of averaged steps)."""
        N = self.N
        dev = torch.device("cuda", self.h.device)
        prim = torch.empty((N, N) if self.kind == "rof" else (2, N, N), device=dev, dtype=torch.float32)
        p = torch.empty((2, N, N), device=dev, dtype=torch.float32)
        n = C.c_longlong(0)
        self.h.check(lib().gp_state_read_average(self.h.ptr, self._s, _ptr(prim), _ptr(p), C.byref(n),
                                                 _stream(stream)))
        return prim, p, int(n.value)

    def gap(self, stream=None):
        rep = Report()
        self.h.check(lib().gp_state_gap(self.h.ptr, self._s, C.byref(rep), _stream(stream)))
        return rep.as_dict()

    def certify(self, stream=None):
        """gap() plus, for EMD, the feasibility certificate of the current flux."""
        rep = Report()
        self.h.check(lib().gp_state_certify(self.h.ptr, self._s, C.byref(rep), _stream(stream)))
        return rep.as_dict()

    def close(self):
        if self._s:
            lib().gp_state_destroy(self._s)
            self._s = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(h: Handle, N: int, cache_path: str | None = None, stream=None) -> int:
    """Time the fused kernels' row-block heights for size N; later solves on h use the fastest."""
    return lib().gp_autotune(h.ptr, int(N), cache_path.encode() if cache_path else None, _stream(stream))


def tuned_row_block(h: Handle, kernel: str, N: int) -> int:
    return lib().gp_tuned_row_block(h.ptr, kernel.encode(), int(N))


def rof_image_stats(h: Handle, I, stream=None):
    """(||I||_TV, ||grad I||_L2, ||I - mean I||^2_L2), reduced on the GPU."""
    out = (C.c_double * 3)()
    h.check(lib().gp_rof_image_stats(h.ptr, _ptr(I), _side(I, "I"), out, _stream(stream)))
    return float(out[0]), float(out[1]), float(out[2])


RULE_GRID_CAP, RULE_FIDELITY_BOUND = 1, 2


def rof_step_tau(stats, lam: float, eps: float, grid_cap: bool = True, fidelity_bound: bool = False) -> float:
    """Section 4.1's ROF step rule from (||I||_TV, ||grad I||_L2, ||I - mean I||^2) -- see include/gprox.h."""
    arr = (C.c_double * 3)(*[float(x) for x in stats])
    flags = (RULE_GRID_CAP if grid_cap else 0) | (RULE_FIDELITY_BOUND if fidelity_bound else 0)
    return float(lib().gp_rof_step_tau(arr, float(lam), float(eps), flags))


def emd_delta_tau(N: int, eps: float, m_points: bool = True) -> float:
    """Section 4.2's step rule for delta measures -- see include/gprox.h."""
    return float(lib().gp_emd_delta_tau(int(N), float(eps), 1 if m_points else 0))


def gap_schedule_next(n_prev: int, g_prev: float, n: int, g: float, tol: float) -> int:
    """Iterations to the next gap check of the adaptive schedule (gap_every = 0)."""
    return int(lib().gp_gap_schedule_next(int(n_prev), float(g_prev), int(n), float(g), float(tol)))


def profile(h: Handle, enable: bool) -> int:
    """Start (clearing the counters) or stop the library's launch profiler."""
    return lib().gp_profile(h.ptr, 1 if enable else 0)


def profile_read(h: Handle):
    """{kernel class: (total device ms, launches)} recorded by the profiler."""
    out = {}
    for k in range(lib().gp_profile_kernels()):
        name, ms, n = C.c_char_p(), C.c_double(), C.c_longlong()
        h.check(lib().gp_profile_query(h.ptr, k, C.byref(name), C.byref(ms), C.byref(n)))
        out[name.value.decode()] = (ms.value, n.value)
    return out


def pd_step(state: State, n_steps: int, prec="fp32", stream=None) -> int:
    """Run n_steps G-prox PDHG iterations on an explicit state."""
    return state.step(n_steps, prec, stream)


def _ptr_array(ts, shape=None, name="arrays"):
    if ts is None:
        return None
    if shape is not None:
        for b, t in enumerate(ts):
            _shape(t, shape, f"{name}[{b}]")
    P = C.c_void_p * len(ts)
    return P(*[_ptr(t) for t in ts])


class Cnn:
    """The learned warm-start network (gp_cnn): 4-level encoder-decoder of base
    width C mapping (f0, f1) to a dual potential -- see include/gprox.h."""

    def __init__(self, h: Handle, C_base: int = 32, bf16: bool = True, seed: int = 0):
        self.h = h
        self._n = C.c_void_p()
        st = lib().gp_cnn_create(h.ptr, int(C_base), 1 if bf16 else 0, C.c_ulonglong(seed), C.byref(self._n))
        if st != GP_OK:
            raise GproxError(st, "gp_cnn_create failed")
        self.C = C_base
        self.bf16 = bf16

    def last_error(self) -> str:
        return lib().gp_cnn_last_error(self._n).decode()

    def check(self, st, allow=(GP_OK,)):
        if st not in allow:
            raise GproxError(st, self.last_error())
        return st

    @property
    def num_params(self) -> int:
        return int(lib().gp_cnn_num_params(self._n))

    def get_params(self):
        import numpy as np

        w = np.empty(self.num_params, np.float32)
        self.check(lib().gp_cnn_get_params(self._n, w.ctypes.data_as(C.c_void_p)))
        return w

    def set_params(self, w):
        import numpy as np

        w = np.ascontiguousarray(w, np.float32)
        if w.size != self.num_params:
            raise ValueError(f"expected {self.num_params} parameters, got {w.size}")
        self.check(lib().gp_cnn_set_params(self._n, w.ctypes.data_as(C.c_void_p)))

    def forward(self, f0s, f1s, priors=None, stream=None):
        """phi (B, N, N), mean-free, for lists of (N, N) device tensors (priors: list or None)."""
        B, N = len(f0s), _side(f0s[0], "f0s[0]")
        if len(f1s) != B or (priors is not None and len(priors) != B):
            raise ValueError("f0s, f1s (and priors) must have one entry per sample")
        phi = torch.empty((B, N, N), device=f0s[0].device, dtype=torch.float32)
        self.check(lib().gp_cnn_forward(self._n, B, _ptr_array(f0s, (N, N), "f0s"), _ptr_array(f1s, (N, N), "f1s"),
                                        _ptr_array(priors, (N, N), "priors"), N, _ptr(phi), _stream(stream)))
        return phi

    def loss_grad(self, f0s, f1s, targets, priors=None, want_grad=False, want_loss=True, stream=None):
        """Forward + loss + backward; returns (loss or None, gradient (numpy) or None)."""
        import numpy as np

        B, N = len(f0s), _side(f0s[0], "f0s[0]")
        if len(f1s) != B or len(targets) != B or (priors is not None and len(priors) != B):
            raise ValueError("f0s, f1s, targets (and priors) must have one entry per sample")
        for nm, ts in (("f0s", f0s), ("f1s", f1s), ("targets", targets), ("priors", priors)):
            _ptr_array(ts, (N, N), nm)
        loss = C.c_double(float("nan"))
        g = np.empty(self.num_params, np.float32) if want_grad else None
        self.check(lib().gp_cnn_loss_grad(self._n, B, _ptr_array(f0s), _ptr_array(f1s), _ptr_array(priors),
                                          _ptr_array(targets), N, C.byref(loss) if want_loss else None,
                                          g.ctypes.data_as(C.c_void_p) if g is not None else None, _stream(stream)))
        return (loss.value if want_loss else None), g

    def adam_step(self, lr: float, stream=None):
        self.check(lib().gp_cnn_adam_step(self._n, float(lr), _stream(stream)))

    def close(self):
        if self._n:
            lib().gp_cnn_destroy(self._n)
            self._n = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def emd_solve_learned(h: Handle, net: Cnn, f0, f1, m, p=None, phi=None, opts: Opts | None = None,
                      coarse_factor: int = 4, coarse_opts: Opts | None = None, stream=None):
    """EMD solve from the best (by the gap at n = 0) of the learned, prior and zero
    starts; returns (status, report dict with 'start': 'zero' | 'learned' | 'prior')."""
    N = _side(f0, "f0")
    _shape(f1, (N, N), "f1")
    _shape(m, (2, N, N), "m")
    _shape(p, (2, N, N), "p")
    _shape(phi, (N, N), "phi")
    rep = Report()
    used = C.c_int(0)
    st = lib().emd_solve_learned(h.ptr, net._n, _ptr(f0), _ptr(f1), _ptr(m), _ptr(p), _ptr(phi),
                                 N, int(coarse_factor),
                                 C.byref(coarse_opts) if coarse_opts is not None else None,
                                 C.byref(opts) if opts is not None else None, C.byref(rep), C.byref(used),
                                 _stream(stream))
    d = rep.as_dict()
    d["start"] = ("zero", "learned", "prior")[used.value]
    return st, d


def rof_solve_learned(h: Handle, net: Cnn, I, u, p=None, lam: float = 8.0, opts: Opts | None = None,
                      coarse_factor: int = 4, coarse_opts: Opts | None = None, stream=None):
    """ROF solve from the best (by the gap at n = 0) of the learned, prior and zero
    starts; returns (status, report dict with 'start': 'zero' | 'learned' | 'prior')."""
    N = _side(I, "I")
    _shape(u, (N, N), "u")
    _shape(p, (2, N, N), "p")
    rep = Report()
    used = C.c_int(0)
    st = lib().rof_solve_learned(h.ptr, net._n, _ptr(I), _ptr(u), _ptr(p), N, float(lam), int(coarse_factor),
                                 C.byref(coarse_opts) if coarse_opts is not None else None,
                                 C.byref(opts) if opts is not None else None, C.byref(rep), C.byref(used),
                                 _stream(stream))
    d = rep.as_dict()
    d["start"] = ("zero", "learned", "prior")[used.value]
    return st, d


def rof_coarse_start(h: Handle, I, factor: int, lam: float = 8.0, opts: Opts | None = None, u=None, p=None,
                     stream=None):
    """ROF (u, p) solved on an N/factor grid, interpolated to N x N (p made
    feasible); returns (status, u, p, coarse report dict)."""
    N = _side(I, "I")
    _shape(u, (N, N), "u")
    _shape(p, (2, N, N), "p")
    if u is None:
        u = torch.empty((N, N), device=I.device, dtype=torch.float32)
    if p is None:
        p = torch.empty((2, N, N), device=I.device, dtype=torch.float32)
    rep = Report()
    st = lib().rof_coarse_start(h.ptr, _ptr(I), N, int(factor), float(lam),
                                C.byref(opts) if opts is not None else None, _ptr(u), _ptr(p), C.byref(rep),
                                _stream(stream))
    return st, u, p, rep.as_dict()


def emd_coarse_start(h: Handle, f0, f1, factor: int, opts: Opts | None = None, phi=None, stream=None):
    """Potential of the EMD solved on an N/factor grid, interpolated to N x N;
    returns (status, phi, coarse report dict)."""
    N = _side(f0, "f0")
    _shape(f1, (N, N), "f1")
    _shape(phi, (N, N), "phi")
    if phi is None:
        phi = torch.empty((N, N), device=f0.device, dtype=torch.float32)
    rep = Report()
    st = lib().emd_coarse_start(h.ptr, _ptr(f0), _ptr(f1), N, int(factor),
                                C.byref(opts) if opts is not None else None, _ptr(phi), C.byref(rep),
                                _stream(stream))
    return st, phi, rep.as_dict()
