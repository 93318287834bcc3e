"""Thin ctypes binding of ``liblift_gb300.so`` (C ABI in ``include/lift.h``).

The functions below carry the names of the C entry points and only marshal
arguments; every step of the solver runs in the library's CUDA kernels.
Device buffers may be passed as ``torch`` CUDA tensors (their data pointers
are used) and host buffers as numpy arrays.  There is no CPU fallback: if the
library is missing, loading fails with an error naming the build step.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

LIFT_QUAD, LIFT_TRUNC_QUAD, LIFT_PL_SAMPLED, LIFT_PERIODIC_QUAD = 0, 1, 2, 3
LIFT_OK, LIFT_ERR_SPEC, LIFT_ERR_OOM, LIFT_ERR_CUDA = 0, 1, 2, 3
LIFT_ERR_NAN, LIFT_ERR_NOT_CONVERGED, LIFT_ERR_ARG, LIFT_ERR_TIMEOUT = 4, 5, 6, 7
LIFT_MAX_K = 64
LIFT_HALO_PRIMAL, LIFT_HALO_DUAL = 0, 1

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liblift_gb300.so")

EXPORTED = (
    "lift_create", "lift_destroy", "lift_set_data", "lift_reset", "lift_iterate", "lift_solve",
    "lift_dual_step", "lift_primal_step",
    "lift_energy", "lift_gap", "lift_unlift", "lift_state_bytes", "lift_get_state",
    "lift_set_state", "lift_proj_epi", "lift_envelope", "lift_strerror",
    "lift_energy_noalloc",
    "lift_create_batch", "lift_batch_destroy", "lift_batch_size", "lift_batch_reset",
    "lift_batch_iterate", "lift_batch_solve", "lift_batch_energy", "lift_batch_unlift",
    "lift_batch_get_state", "lift_batch_autotune", "lift_batch_schedule",
    "lift_batch_set_schedule",
    "lift_set_params", "lift_unrolled_forward", "lift_unrolled_backward",
    "lift_get_balance", "lift_set_resident", "lift_set_bands", "lift_unrolled_generation",
    "lift_create_band", "lift_band_halo_bytes", "lift_band_export", "lift_band_import",
    "lift_cuda_error", "lift_batch_streams",
    "lift_average", "lift_average_count", "lift_energy_average", "lift_unlift_average",
    "lift_average_restart", "lift_solve_averaged",
)


class lift_spec(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("H", C.c_int), ("W", C.c_int), ("L", C.c_int),
        ("gamma_min", C.c_double), ("gamma_max", C.c_double), ("lambda_", C.c_double),
        ("alpha", C.c_double), ("nu", C.c_double),
        ("f", C.c_void_p), ("cost", C.c_void_p), ("n_samples", C.c_int),
        ("sample_min", C.c_double), ("sample_max", C.c_double),
        ("data_on_host", C.c_int), ("check_every", C.c_int), ("step_balance", C.c_double),
        ("adaptive_balance", C.c_int), ("tv_anisotropic", C.c_int), ("D", C.c_int),
    ]


class LiftError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        detail = ""
        if code == LIFT_ERR_CUDA:
            detail = f" [{load().lift_cuda_error().decode()}]"
        super().__init__(f"{where}: {strerror(code)} (code {code}){detail}")


_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    sig = {
        "lift_create": (C.c_int, [C.POINTER(lift_spec), vp, C.POINTER(vp)]),
        "lift_destroy": (None, [vp]),
        "lift_set_data": (C.c_int, [vp, vp, C.c_int]),
        "lift_reset": (C.c_int, [vp]),
        "lift_iterate": (C.c_int, [vp, C.c_int]),
        "lift_solve": (C.c_int, [vp, C.c_int, C.c_double, ip]),
        "lift_dual_step": (C.c_int, [vp]),
        "lift_primal_step": (C.c_int, [vp]),
        "lift_energy": (C.c_int, [vp, dp, dp, dp]),
        "lift_gap": (C.c_int, [vp, dp]),
        "lift_unlift": (C.c_int, [vp, vp, C.c_int]),
        "lift_average": (C.c_int, [vp, C.c_int]),
        "lift_average_count": (C.c_longlong, [vp]),
        "lift_energy_average": (C.c_int, [vp, dp, dp, dp]),
        "lift_unlift_average": (C.c_int, [vp, vp, C.c_int]),
        "lift_average_restart": (C.c_int, [vp]),
        "lift_solve_averaged": (C.c_int, [vp, C.c_int, C.c_double, C.c_int, C.c_int, ip, dp]),
        "lift_state_bytes": (C.c_size_t, [vp]),
        "lift_get_state": (C.c_int, [vp, vp, C.c_size_t, C.c_int]),
        "lift_set_state": (C.c_int, [vp, vp, C.c_size_t, C.c_int]),
        "lift_proj_epi": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, C.c_int]),
        "lift_envelope": (C.c_int, [vp, vp, vp, vp, vp, C.c_int]),
        "lift_strerror": (C.c_char_p, [C.c_int]),
        "lift_energy_noalloc": (C.c_int, [C.POINTER(lift_spec), vp, vp, vp]),
        "lift_create_batch": (C.c_int, [C.POINTER(lift_spec), C.c_int, vp, C.POINTER(vp)]),
        "lift_batch_destroy": (None, [vp]),
        "lift_batch_size": (C.c_int, [vp]),
        "lift_batch_reset": (C.c_int, [vp]),
        "lift_batch_iterate": (C.c_int, [vp, C.c_int]),
        "lift_batch_solve": (C.c_int, [vp, C.c_int, C.c_double, ip, ip]),
        "lift_batch_energy": (C.c_int, [vp, dp]),
        "lift_batch_unlift": (C.c_int, [vp, C.c_int, vp, C.c_int]),
        "lift_batch_get_state": (C.c_int, [vp, C.c_int, vp, C.c_size_t, C.c_int]),
        "lift_batch_autotune": (C.c_int, [vp, C.c_int, ip]),
        "lift_batch_schedule": (C.c_int, [vp, ip, ip, ip]),
        "lift_batch_set_schedule": (C.c_int, [vp, C.c_int, C.c_int]),
        "lift_set_params": (C.c_int, [vp, C.c_double, C.c_double, C.c_double]),
        "lift_unrolled_forward": (C.c_int, [vp, C.c_int, C.c_int]),
        "lift_unrolled_backward": (C.c_int, [vp, vp, vp, dp]),
        "lift_get_balance": (C.c_int, [vp, dp]),
        "lift_set_resident": (C.c_int, [vp, C.c_int, ip]),
        "lift_set_bands": (C.c_int, [vp, C.c_int, ip]),
        "lift_unrolled_generation": (C.c_int, [vp, C.POINTER(C.c_ulonglong)]),
        "lift_create_band": (C.c_int, [C.POINTER(lift_spec), C.c_int, C.c_int, vp, C.POINTER(vp)]),
        "lift_band_halo_bytes": (C.c_int, [vp, C.c_int, C.POINTER(C.c_size_t)]),
        "lift_band_export": (C.c_int, [vp, C.c_int, vp, C.c_int]),
        "lift_band_import": (C.c_int, [vp, C.c_int, vp, C.c_int]),
        "lift_cuda_error": (C.c_char_p, []),
        "lift_batch_streams": (C.c_int, [vp, C.c_int, ip]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().lift_strerror(code).decode()


def _check(rc: int, where: str):
    if rc != LIFT_OK:
        raise LiftError(rc, where)


def _ptr(a) -> tuple[int, int]:
    """(address, on_host) of a torch tensor or numpy array."""
    if a is None:
        return 0, 1
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data, 1
    # torch.Tensor
    assert a.is_contiguous()
    return a.data_ptr(), 0 if a.is_cuda else 1


def current_stream() -> int:
    """cudaStream_t of torch's current stream (0 if torch is unavailable)."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


# ---------------------------------------------------------------------------
# One function per C entry point.
# ---------------------------------------------------------------------------
def lift_create(spec: lift_spec, stream: int | None = None) -> int:
    h = C.c_void_p()
    s = current_stream() if stream is None else stream
    _check(load().lift_create(C.byref(spec), C.c_void_p(s), C.byref(h)), "lift_create")
    return h.value


def lift_destroy(h: int) -> None:
    load().lift_destroy(C.c_void_p(h))


def lift_set_data(h: int, data) -> None:
    p, on_host = _ptr(data)
    _check(load().lift_set_data(C.c_void_p(h), C.c_void_p(p), on_host), "lift_set_data")


def lift_reset(h: int) -> None:
    _check(load().lift_reset(C.c_void_p(h)), "lift_reset")


def lift_iterate(h: int, iters: int) -> None:
    _check(load().lift_iterate(C.c_void_p(h), iters), "lift_iterate")


def lift_create_band(spec: lift_spec, row0: int, row1: int, stream: int | None = None) -> int:
    h = C.c_void_p()
    s = current_stream() if stream is None else stream
    _check(load().lift_create_band(C.byref(spec), row0, row1, C.c_void_p(s), C.byref(h)),
           "lift_create_band")
    return h.value


def lift_band_halo_bytes(h: int, which: int) -> int:
    n = C.c_size_t()
    _check(load().lift_band_halo_bytes(C.c_void_p(h), which, C.byref(n)), "lift_band_halo_bytes")
    return int(n.value)


def lift_band_export(h: int, which: int, dst) -> None:
    p, on_host = _ptr(dst)
    _check(load().lift_band_export(C.c_void_p(h), which, C.c_void_p(p), on_host), "lift_band_export")


def lift_band_import(h: int, which: int, src) -> None:
    p, on_host = _ptr(src)
    _check(load().lift_band_import(C.c_void_p(h), which, C.c_void_p(p), on_host), "lift_band_import")


def lift_dual_step(h: int) -> None:
    _check(load().lift_dual_step(C.c_void_p(h)), "lift_dual_step")


def lift_primal_step(h: int) -> None:
    _check(load().lift_primal_step(C.c_void_p(h)), "lift_primal_step")


def lift_solve(h: int, max_iters: int, rel_gap_tol: float) -> tuple[int, int]:
    """Returns (status code, iterations done); NOT_CONVERGED is not raised."""
    n = C.c_int()
    rc = load().lift_solve(C.c_void_p(h), max_iters, rel_gap_tol, C.byref(n))
    if rc not in (LIFT_OK, LIFT_ERR_NOT_CONVERGED):
        raise LiftError(rc, "lift_solve")
    return rc, n.value


def lift_get_balance(h: int) -> float:
    t = C.c_double()
    _check(load().lift_get_balance(C.c_void_p(h), C.byref(t)), "lift_get_balance")
    return t.value


def lift_set_bands(h: int, bands: int) -> int:
    """Bands of the iteration graph (0 automatic, 1 off); returns the number used."""
    u = C.c_int()
    _check(load().lift_set_bands(C.c_void_p(h), bands, C.byref(u)), "lift_set_bands")
    return u.value


def lift_set_resident(h: int, enable: bool) -> bool:
    """Prefer (or not) the cluster-resident iteration for small problems;
    returns whether lift_iterate now takes it."""
    a = C.c_int()
    _check(load().lift_set_resident(C.c_void_p(h), 1 if enable else 0, C.byref(a)),
           "lift_set_resident")
    return bool(a.value)


def lift_energy(h: int) -> tuple[float, float, float]:
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(load().lift_energy(C.c_void_p(h), C.byref(a), C.byref(b), C.byref(c)), "lift_energy")
    return a.value, b.value, c.value


def lift_gap(h: int) -> float:
    g = C.c_double()
    _check(load().lift_gap(C.c_void_p(h), C.byref(g)), "lift_gap")
    return g.value


def lift_unlift(h: int, out) -> None:
    p, on_host = _ptr(out)
    _check(load().lift_unlift(C.c_void_p(h), C.c_void_p(p), on_host), "lift_unlift")


def lift_average(h: int, accumulate: bool) -> None:
    _check(load().lift_average(C.c_void_p(h), 1 if accumulate else 0), "lift_average")


def lift_average_count(h: int) -> int:
    return int(load().lift_average_count(C.c_void_p(h)))


def lift_energy_average(h: int) -> tuple[float, float, float]:
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    _check(load().lift_energy_average(C.c_void_p(h), C.byref(a), C.byref(b), C.byref(c)),
           "lift_energy_average")
    return a.value, b.value, c.value


def lift_unlift_average(h: int, out) -> None:
    p, on_host = _ptr(out)
    _check(load().lift_unlift_average(C.c_void_p(h), C.c_void_p(p), on_host),
           "lift_unlift_average")


def lift_average_restart(h: int) -> None:
    _check(load().lift_average_restart(C.c_void_p(h)), "lift_average_restart")


def lift_solve_averaged(h: int, max_iters: int, rel_gap_tol: float, first_epoch: int = 1000,
                        every: int = 10) -> tuple[int, int, float]:
    """(return code LIFT_OK or LIFT_ERR_NOT_CONVERGED, iterations, final gap)."""
    n, g = C.c_int(0), C.c_double(float("nan"))
    rc = load().lift_solve_averaged(C.c_void_p(h), max_iters, rel_gap_tol, first_epoch, every,
                                    C.byref(n), C.byref(g))
    if rc not in (LIFT_OK, LIFT_ERR_NOT_CONVERGED):
        _check(rc, "lift_solve_averaged")
    return rc, n.value, g.value


def lift_state_bytes(h: int) -> int:
    return load().lift_state_bytes(C.c_void_p(h))


def lift_get_state(h: int, dst) -> None:
    p, on_host = _ptr(dst)
    nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
    _check(load().lift_get_state(C.c_void_p(h), C.c_void_p(p), nbytes, on_host), "lift_get_state")


def lift_set_state(h: int, src) -> None:
    p, on_host = _ptr(src)
    nbytes = src.nbytes if isinstance(src, np.ndarray) else src.numel() * src.element_size()
    _check(load().lift_set_state(C.c_void_p(h), C.c_void_p(p), nbytes, on_host), "lift_set_state")


def lift_proj_epi(h: int, pix, interval, y0, h0, y, hout) -> None:
    n = int(y0.numel())
    args = [C.c_void_p(t.data_ptr()) for t in (pix, interval, y0, h0, y, hout)]
    _check(load().lift_proj_epi(C.c_void_p(h), *args, n), "lift_proj_epi")


def lift_envelope(h: int, pix, interval, t, out) -> None:
    n = int(t.numel())
    args = [C.c_void_p(a.data_ptr()) for a in (pix, interval, t, out)]
    _check(load().lift_envelope(C.c_void_p(h), *args, n), "lift_envelope")


def lift_energy_noalloc(spec: lift_spec, state, out, stream: int | None = None) -> None:
    """Energies of a caller-held device state into out[3] (device), with no
    allocation (see include/lift.h).  The C entry point cannot see buffer
    sizes, so they are checked here: out must be a CUDA float64 tensor of at
    least 3 elements, state a CUDA tensor holding at least the primal and dual
    records of the problem (H*W*(L-1) * 32 bytes, the x, xbar and y parts of
    the lift_get_state layout)."""
    import torch
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
            and out.numel() >= 3 and out.is_contiguous()):
        raise LiftError(LIFT_ERR_ARG, "lift_energy_noalloc: out must be a contiguous CUDA "
                                      "float64 tensor of at least 3 elements")
    need = spec.H * spec.W * (spec.L - 1) * 32
    if not (isinstance(state, torch.Tensor) and state.is_cuda and state.is_contiguous()
            and state.numel() * state.element_size() >= need):
        raise LiftError(LIFT_ERR_ARG, f"lift_energy_noalloc: state must be a contiguous CUDA "
                                      f"tensor of at least {need} bytes")
    s = current_stream() if stream is None else stream
    _check(load().lift_energy_noalloc(C.byref(spec), C.c_void_p(state.data_ptr()),
                                      C.c_void_p(out.data_ptr()), C.c_void_p(s)),
           "lift_energy_noalloc")


# ---------------------------------------------------------------------------
# Convenience wrapper holding a handle and the buffers it was created from.
# ---------------------------------------------------------------------------
def make_spec(kind: int, H: int, W: int, L: int, gamma_min: float, gamma_max: float,
              lam: float, alpha: float = 1.0, nu: float = 0.0, f=None, cost=None,
              sample_min: float = 0.0, sample_max: float = 1.0,
              check_every: int = 100, step_balance: float = 1.0,
              adaptive_balance: bool = False, anisotropic: bool = False,
              depth: int = 1) -> lift_spec:
    data = f if kind != LIFT_PL_SAMPLED else cost
    p, on_host = _ptr(data)
    n_samples = 0
    if cost is not None:
        n_samples = int(cost.shape[-1])
    return lift_spec(kind, H, W, L, gamma_min, gamma_max, lam, alpha, nu,
                     p if kind != LIFT_PL_SAMPLED else 0, p if kind == LIFT_PL_SAMPLED else 0,
                     n_samples, sample_min, sample_max, on_host, check_every, step_balance,
                     1 if adaptive_balance else 0, 1 if anisotropic else 0, depth)


def state_arrays(h: int, k: int, depth: int = 1) -> dict:
    """Host copy of a handle's iterate as numpy arrays (the lift_get_state
    layout: x, xbar, y records, q, and pz on a volume); the pixel count
    follows from lift_state_bytes (a band handle: its local rows)."""
    nb = lift_state_bytes(h)
    per = 32 * k + 4 + (4 * k if depth > 1 else 0)
    N = nb // per
    assert N * per == nb
    buf = np.empty(nb, dtype=np.uint8)
    lift_get_state(h, buf)
    f = buf.view(np.float32)
    o = 0
    x = f[o:o + 2 * N * k].reshape(N, k, 2); o += 2 * N * k
    xb = f[o:o + 2 * N * k].reshape(N, k, 2); o += 2 * N * k
    y = f[o:o + 4 * N * k].reshape(N, k, 4); o += 4 * N * k
    q = f[o:o + N]; o += N
    st = {"u": x[..., 0], "s": x[..., 1], "ubar": xb[..., 0], "sbar": xb[..., 1],
          "v": y[..., 0], "z": y[..., 1], "px": y[..., 2], "py": y[..., 3], "q": q}
    if depth > 1:
        st["pz"] = f[o:o + N * k].reshape(N, k)
    return st


class Solver:
    """A lifted problem on the GPU: ``Solver(kind, H, W, L, ...)``; depth > 1
    makes it a depth x H x W volume."""

    def __init__(self, kind: int, H: int, W: int, L: int, gamma_min: float = 0.0,
                 gamma_max: float = 1.0, lam: float = 0.0, alpha: float = 1.0,
                 nu: float = 0.0, f=None, cost=None, sample_min: float = 0.0,
                 sample_max: float = 1.0, check_every: int = 100, stream: int | None = None,
                 step_balance: float = 1.0, adaptive_balance: bool = False,
                 anisotropic: bool = False, depth: int = 1, resident: bool = True):
        self.kind, self.H, self.W, self.L, self.k = kind, H, W, L, L - 1
        self.D = max(int(depth), 1)
        self.spec = make_spec(kind, H, W, L, gamma_min, gamma_max, lam, alpha, nu, f, cost,
                              sample_min, sample_max, check_every, step_balance, adaptive_balance,
                              anisotropic, depth)
        self._keep = (f, cost)
        self.h = lift_create(self.spec, stream)
        self._keep = None
        if not resident:
            lift_set_resident(self.h, False)

    def close(self):
        if getattr(self, "h", None):
            lift_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self):
        lift_reset(self.h)

    def set_data(self, data):
        lift_set_data(self.h, data)

    def iterate(self, n: int):
        lift_iterate(self.h, n)

    def solve(self, max_iters: int, rel_gap_tol: float):
        return lift_solve(self.h, max_iters, rel_gap_tol)

    def energy(self):
        return lift_energy(self.h)

    def gap(self):
        return lift_gap(self.h)

    def average_reset(self):
        lift_average(self.h, False)

    def average_add(self):
        """Add the current iterate to the running average."""
        lift_average(self.h, True)

    def average_count(self) -> int:
        return lift_average_count(self.h)

    def energy_average(self):
        return lift_energy_average(self.h)

    def solve_averaged(self, max_iters: int, rel_gap_tol: float, first_epoch: int = 1000,
                       every: int = 10):
        return lift_solve_averaged(self.h, max_iters, rel_gap_tol, first_epoch, every)

    def average_restart(self):
        """Restart the iteration from the averaged point (and empty the average)."""
        lift_average_restart(self.h)

    def unlift_average(self, out=None) -> np.ndarray:
        if out is None:
            shape = (self.H, self.W) if self.D == 1 else (self.D, self.H, self.W)
            out = np.empty(shape, dtype=np.float32)
        lift_unlift_average(self.h, out)
        return out

    @property
    def N(self) -> int:
        return self.D * self.H * self.W

    def unlift(self, out=None) -> np.ndarray:
        if out is None:
            shape = (self.H, self.W) if self.D == 1 else (self.D, self.H, self.W)
            out = np.empty(shape, dtype=np.float32)
        lift_unlift(self.h, out)
        return out

    def state(self) -> dict:
        """Host copy of the iterate as numpy arrays (layout of include/lift.h)."""
        return state_arrays(self.h, self.k, self.D)

    def set_state(self, st: dict):
        N, k = self.N, self.k
        x = np.stack([st["u"], st["s"]], -1).astype(np.float32).reshape(-1)
        xb = np.stack([st["ubar"], st["sbar"]], -1).astype(np.float32).reshape(-1)
        y = np.stack([st["v"], st["z"], st["px"], st["py"]], -1).astype(np.float32).reshape(-1)
        q = np.asarray(st["q"], dtype=np.float32).reshape(N)
        parts = [x, xb, y, q]
        if self.D > 1:
            parts.append(np.asarray(st["pz"], dtype=np.float32).reshape(-1))
        buf = np.ascontiguousarray(np.concatenate(parts))
        assert buf.size * 4 == lift_state_bytes(self.h) and N * k > 0
        lift_set_state(self.h, buf)


# ---------------------------------------------------------------------------
# Batches
# ---------------------------------------------------------------------------
def lift_create_batch(specs: list, stream: int | None = None) -> int:
    arr = (lift_spec * len(specs))(*specs)
    h = C.c_void_p()
    s = current_stream() if stream is None else stream
    _check(load().lift_create_batch(arr, len(specs), C.c_void_p(s), C.byref(h)),
           "lift_create_batch")
    return h.value


def lift_batch_destroy(b: int) -> None:
    load().lift_batch_destroy(C.c_void_p(b))


def lift_batch_size(b: int) -> int:
    return load().lift_batch_size(C.c_void_p(b))


def lift_batch_reset(b: int) -> None:
    _check(load().lift_batch_reset(C.c_void_p(b)), "lift_batch_reset")


def lift_batch_iterate(b: int, iters: int) -> None:
    _check(load().lift_batch_iterate(C.c_void_p(b), iters), "lift_batch_iterate")


def lift_batch_solve(b: int, max_iters: int, rel_gap_tol: float):
    """(status, per-instance iterations, number converged)."""
    n = lift_batch_size(b)
    it = (C.c_int * n)()
    nc = C.c_int()
    rc = load().lift_batch_solve(C.c_void_p(b), max_iters, rel_gap_tol, it, C.byref(nc))
    if rc not in (LIFT_OK, LIFT_ERR_NOT_CONVERGED):
        raise LiftError(rc, "lift_batch_solve")
    return rc, list(it), nc.value


def lift_batch_energy(b: int) -> np.ndarray:
    n = lift_batch_size(b)
    out = np.empty(3 * n, dtype=np.float64)
    _check(load().lift_batch_energy(C.c_void_p(b), out.ctypes.data_as(C.POINTER(C.c_double))),
           "lift_batch_energy")
    return out.reshape(n, 3)


def lift_batch_unlift(b: int, i: int, out) -> None:
    p, on_host = _ptr(out)
    _check(load().lift_batch_unlift(C.c_void_p(b), i, C.c_void_p(p), on_host), "lift_batch_unlift")


def lift_batch_get_state(b: int, i: int, dst) -> None:
    p, on_host = _ptr(dst)
    nbytes = dst.nbytes if isinstance(dst, np.ndarray) else dst.numel() * dst.element_size()
    _check(load().lift_batch_get_state(C.c_void_p(b), i, C.c_void_p(p), nbytes, on_host),
           "lift_batch_get_state")


def lift_batch_autotune(b: int, iters: int) -> int:
    t = C.c_int()
    _check(load().lift_batch_autotune(C.c_void_p(b), iters, C.byref(t)), "lift_batch_autotune")
    return t.value


def lift_batch_set_schedule(b: int, threads: int, big_tiles: int) -> None:
    _check(load().lift_batch_set_schedule(C.c_void_p(b), threads, big_tiles),
           "lift_batch_set_schedule")


def lift_batch_streams(b: int, set_to: int = 0) -> int:
    """Set (1..4) and return the number of streams the big instances share."""
    n = C.c_int()
    _check(load().lift_batch_streams(C.c_void_p(b), set_to, C.byref(n)), "lift_batch_streams")
    return n.value


def lift_batch_schedule(b: int) -> tuple[int, int, int]:
    """(merged tile width, big-instance threshold in 256-thread tiles, number
    of instances on the single-instance kernels)."""
    t, g, n = C.c_int(), C.c_int(), C.c_int()
    _check(load().lift_batch_schedule(C.c_void_p(b), C.byref(t), C.byref(g), C.byref(n)),
           "lift_batch_schedule")
    return t.value, g.value, n.value


# ---------------------------------------------------------------------------
# Differentiable unrolled solve
# ---------------------------------------------------------------------------
def lift_set_params(h: int, lam: float, alpha: float, nu: float) -> None:
    _check(load().lift_set_params(C.c_void_p(h), lam, alpha, nu), "lift_set_params")


def lift_unrolled_forward(h: int, iters: int, checkpoint_every: int) -> None:
    _check(load().lift_unrolled_forward(C.c_void_p(h), iters, checkpoint_every),
           "lift_unrolled_forward")


def lift_unrolled_generation(h: int) -> int:
    """The handle's forward-pass generation (changes with every unrolled
    forward, parameter, data or reset call)."""
    g = C.c_ulonglong(0)
    _check(load().lift_unrolled_generation(C.c_void_p(h), C.byref(g)), "lift_unrolled_generation")
    return int(g.value)


def lift_unrolled_backward(h: int, grad_u, grad_f=None) -> tuple[float, float, float]:
    """grad_u, grad_f: device tensors (H*W float32); returns dL/d(lambda, alpha, nu)."""
    out = (C.c_double * 3)()
    gf = C.c_void_p(grad_f.data_ptr()) if grad_f is not None else C.c_void_p(0)
    _check(load().lift_unrolled_backward(C.c_void_p(h), C.c_void_p(grad_u.data_ptr()), gf, out),
           "lift_unrolled_backward")
    return out[0], out[1], out[2]
