"""ctypes binding of the FP64 oracle (``lift_oracle.c``).

Test infrastructure only: callers are ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py``.  The library is compiled from source with
gcc on first use (or by ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

QUAD, TRUNC, PL, PERIODIC = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lift_oracle.c")
_SO = os.path.join(_HERE, "liblift_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)


class _Problem(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("H", C.c_int), ("W", C.c_int), ("L", C.c_int),
        ("gmin", C.c_double), ("gmax", C.c_double), ("lam", C.c_double),
        ("alpha", C.c_double), ("nu", C.c_double),
        ("f", _dp), ("cost", _dp), ("ns", C.c_int),
        ("smin", C.c_double), ("smax", C.c_double), ("theta", C.c_double),
        ("aniso", C.c_int), ("D", C.c_int),
    ]


class _State(C.Structure):
    _fields_ = [(n, _dp) for n in ("u", "s", "ubar", "sbar", "v", "z", "px", "py", "q", "pz")]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P, S = C.POINTER(_Problem), C.POINTER(_State)
        lib.orc_rho.restype = C.c_double
        lib.orc_rho.argtypes = [P, C.c_int, C.c_double]
        lib.orc_conj.restype = C.c_double
        lib.orc_conj.argtypes = [P, C.c_int, C.c_int, C.c_double, _dp]
        lib.orc_lifted_conj.restype = C.c_double
        lib.orc_lifted_conj.argtypes = [P, C.c_int, _dp]
        lib.orc_proj_epi.restype = None
        lib.orc_proj_epi.argtypes = [P, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp]
        lib.orc_biconj.restype = C.c_double
        lib.orc_biconj.argtypes = [P, C.c_int, C.c_int, C.c_double]
        lib.orc_grad.restype = None
        lib.orc_grad.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
        lib.orc_div.restype = None
        lib.orc_div.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _dp, _dp]
        lib.orc_grad3.restype = None
        lib.orc_grad3.argtypes = [C.c_int] * 4 + [_dp] * 4
        lib.orc_div3.restype = None
        lib.orc_div3.argtypes = [C.c_int] * 4 + [_dp] * 4
        lib.orc_rof_direct3.restype = C.c_double
        lib.orc_rof_direct3.argtypes = [C.c_int] * 3 + [_dp] + [C.c_double] * 4 + [C.c_int] * 2 + [_dp]
        lib.orc_rof_energy3.restype = C.c_double
        lib.orc_rof_energy3.argtypes = [C.c_int] * 3 + [_dp, _dp, C.c_double, C.c_double, C.c_int]
        lib.orc_steps_get.restype = None
        lib.orc_steps_get.argtypes = [P, _dp, _dp, _dp, _dp, _dp]
        lib.orc_pdhg.restype = C.c_int
        lib.orc_pdhg.argtypes = [P, S, C.c_int]
        lib.orc_half_step.restype = C.c_int
        lib.orc_half_step.argtypes = [P, S, C.c_int]
        lib.orc_unlift.restype = None
        lib.orc_unlift.argtypes = [P, _dp, _dp]
        lib.orc_monotone_proj.restype = None
        lib.orc_monotone_proj.argtypes = [C.c_int, _dp, _dp]
        lib.orc_energy.restype = None
        lib.orc_energy.argtypes = [P, S, _dp, _dp, _dp]
        lib.orc_rof_direct.restype = C.c_double
        lib.orc_rof_direct.argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_double,
                                       C.c_double, C.c_double, C.c_int, _dp]
        lib.orc_unrolled_grad.restype = C.c_int
        lib.orc_unrolled_grad.argtypes = [P, C.c_int, _dp, _dp, _dp]
        for nm in ("orc_rof_direct_aniso",):
            getattr(lib, nm).restype = C.c_double
            getattr(lib, nm).argtypes = [C.c_int, C.c_int, _dp, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_int, _dp]
        lib.orc_rof_energy_aniso.restype = C.c_double
        lib.orc_rof_energy_aniso.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_double, C.c_double]
        lib.orc_rof_energy.restype = C.c_double
        lib.orc_rof_energy.argtypes = [C.c_int, C.c_int, _dp, _dp, C.c_double, C.c_double]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    if a is None:
        return C.cast(None, _dp)
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def labels(L: int, gmin: float, gmax: float) -> np.ndarray:
    """Equidistant labels gamma_1 < ... < gamma_L on [gmin, gmax] (Sec. 3)."""
    k = L - 1
    return gmin + (gmax - gmin) * np.arange(L, dtype=np.float64) / k


@dataclass
class Problem:
    """Lifted problem: data term, label grid and TV weight (eq. general_energy)."""
    kind: int
    H: int
    W: int
    L: int
    gmin: float = 0.0
    gmax: float = 1.0
    lam: float = 0.0
    alpha: float = 1.0
    nu: float = 0.0
    f: np.ndarray | None = None
    cost: np.ndarray | None = None
    smin: float = 0.0
    smax: float = 1.0
    theta: float = 1.0
    aniso: int = 0
    D: int = 1                  # depth: D > 1 makes a D x H x W volume
    _c: _Problem = field(default=None, repr=False)

    def __post_init__(self):
        if self.f is not None:
            self.f = np.ascontiguousarray(self.f, dtype=np.float64).reshape(self.N)
        if self.cost is not None:
            self.cost = np.ascontiguousarray(self.cost, dtype=np.float64).reshape(self.N, -1)
        ns = 0 if self.cost is None else self.cost.shape[1]
        self._c = _Problem(self.kind, self.H, self.W, self.L, self.gmin, self.gmax, self.lam,
                           self.alpha, self.nu, _ptr(self.f), _ptr(self.cost), ns,
                           self.smin, self.smax, self.theta, self.aniso, self.D)

    @property
    def k(self) -> int:
        return self.L - 1

    @property
    def N(self) -> int:
        return max(self.D, 1) * self.H * self.W

    def with_theta(self, theta: float) -> "Problem":
        return Problem(self.kind, self.H, self.W, self.L, self.gmin, self.gmax, lam=self.lam,
                       alpha=self.alpha, nu=self.nu, f=self.f, cost=self.cost, smin=self.smin,
                       smax=self.smax, theta=theta, aniso=self.aniso, D=self.D)

    def ref(self):
        return C.byref(self._c)


class State:
    """PDHG iterate, all variables zero at the start (arrays [pixel, i]);
    pz, the third component of p_i, is used on volumes only (stays 0)."""
    names = ("u", "s", "ubar", "sbar", "v", "z", "px", "py")

    def __init__(self, P: Problem):
        for n in self.names:
            setattr(self, n, np.zeros((P.N, P.k), dtype=np.float64))
        self.q = np.zeros(P.N, dtype=np.float64)
        self.pz = np.zeros((P.N, P.k), dtype=np.float64)

    def _c(self):
        return _State(*[_ptr(getattr(self, n)) for n in self.names], _ptr(self.q), _ptr(self.pz))

    def copy(self, P: Problem) -> "State":
        o = State(P)
        for n in self.names + ("q", "pz"):
            getattr(o, n)[...] = getattr(self, n)
        return o


def rho(P: Problem, pix: int, t: float) -> float:
    return _load().orc_rho(P.ref(), pix, t)


def conj(P: Problem, pix: int, i: int, y: float) -> tuple[float, float]:
    """(rho_i^*(y), a maximiser t) for interval i (0-based) at pixel pix."""
    t = C.c_double()
    val = _load().orc_conj(P.ref(), pix, i, y, C.byref(t))
    return val, t.value


def lifted_conj(P: Problem, pix: int, v: np.ndarray) -> float:
    v = np.ascontiguousarray(v, dtype=np.float64)
    return _load().orc_lifted_conj(P.ref(), pix, _ptr(v))


def proj_epi(P: Problem, pix: int, i: int, y0: float, h0: float) -> tuple[float, float]:
    y, h = C.c_double(), C.c_double()
    _load().orc_proj_epi(P.ref(), pix, i, y0, h0, C.byref(y), C.byref(h))
    return y.value, h.value


def biconj(P: Problem, pix: int, i: int, t: float) -> float:
    return _load().orc_biconj(P.ref(), pix, i, t)


def grad(H: int, W: int, k: int, u: np.ndarray):
    u = np.ascontiguousarray(u, dtype=np.float64)
    gx, gy = np.empty_like(u), np.empty_like(u)
    _load().orc_grad(H, W, k, _ptr(u), _ptr(gx), _ptr(gy))
    return gx, gy


def div(H: int, W: int, k: int, px: np.ndarray, py: np.ndarray):
    px = np.ascontiguousarray(px, dtype=np.float64)
    py = np.ascontiguousarray(py, dtype=np.float64)
    d = np.empty_like(px)
    _load().orc_div(H, W, k, _ptr(px), _ptr(py), _ptr(d))
    return d


def grad3(D: int, H: int, W: int, k: int, u: np.ndarray):
    """Forward differences (x, y, z) on a D x H x W volume, Neumann."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    gx, gy, gz = np.empty_like(u), np.empty_like(u), np.empty_like(u)
    _load().orc_grad3(D, H, W, k, _ptr(u), _ptr(gx), _ptr(gy), _ptr(gz))
    return gx, gy, gz


def div3(D: int, H: int, W: int, k: int, px: np.ndarray, py: np.ndarray, pz: np.ndarray):
    px, py, pz = (np.ascontiguousarray(a, dtype=np.float64) for a in (px, py, pz))
    d = np.empty_like(px)
    _load().orc_div3(D, H, W, k, _ptr(px), _ptr(py), _ptr(pz), _ptr(d))
    return d


def steps(P: Problem) -> dict:
    tu, sq, sp = C.c_double(), C.c_double(), C.c_double()
    ts, svz = np.zeros(P.k), np.zeros(P.k)
    _load().orc_steps_get(P.ref(), C.byref(tu), C.byref(sq), C.byref(sp), _ptr(ts), _ptr(svz))
    return {"tau_u": tu.value, "sigma_q": sq.value, "sigma_p": sp.value,
            "tau_s": ts, "sigma_vz": svz}


def pdhg(P: Problem, X: State, iters: int) -> State:
    """Run ``iters`` PDHG iterations in place on X."""
    cs = X._c()
    rc = _load().orc_pdhg(P.ref(), C.byref(cs), iters)
    if rc != 0:
        raise MemoryError("oracle pdhg: allocation failed")
    return X


def half_step(P: Problem, X: State, half: int) -> State:
    """One half-step of the iteration alone: half = 0 the dual step, 1 the
    primal step (with the extrapolation)."""
    cs = X._c()
    rc = _load().orc_half_step(P.ref(), C.byref(cs), half)
    if rc != 0:
        raise RuntimeError(f"orc_half_step failed ({rc})")
    return X


def unlift(P: Problem, u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.empty(P.N)
    _load().orc_unlift(P.ref(), _ptr(u), _ptr(out))
    return out


def monotone_proj(u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.empty_like(u)
    _load().orc_monotone_proj(u.size, _ptr(u), _ptr(w))
    return w


def energy(P: Problem, X: State) -> tuple[float, float, float]:
    """(P_hat, D, E_nc): primal bound, dual bound, nonconvex energy."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    cs = X._c()
    _load().orc_energy(P.ref(), C.byref(cs), C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def rof_direct(f: np.ndarray, alpha: float, lam: float, lo: float, hi: float,
               iters: int, aniso: bool = False) -> tuple[np.ndarray, float]:
    """Unlifted box-constrained ROF by accelerated primal-dual; (u, gap).
    aniso: |grad u|_1 instead of |grad u|_2."""
    H, W = f.shape
    fd = np.ascontiguousarray(f, dtype=np.float64)
    u = np.empty_like(fd)
    fn = _load().orc_rof_direct_aniso if aniso else _load().orc_rof_direct
    gap = fn(H, W, _ptr(fd), alpha, lam, lo, hi, iters, _ptr(u))
    return u, gap


def rof_direct3(f: np.ndarray, alpha: float, lam: float, lo: float, hi: float,
                iters: int, aniso: bool = False) -> tuple[np.ndarray, float]:
    """The same on a D x H x W volume f; (u, gap)."""
    D, H, W = f.shape
    fd = np.ascontiguousarray(f, dtype=np.float64)
    u = np.empty_like(fd)
    gap = _load().orc_rof_direct3(D, H, W, _ptr(fd), alpha, lam, lo, hi, iters, int(aniso), _ptr(u))
    return u, gap


def rof_energy3(u: np.ndarray, f: np.ndarray, alpha: float, lam: float,
                aniso: bool = False) -> float:
    D, H, W = f.shape
    u = np.ascontiguousarray(u, dtype=np.float64)
    fd = np.ascontiguousarray(f, dtype=np.float64)
    return _load().orc_rof_energy3(D, H, W, _ptr(u), _ptr(fd), alpha, lam, int(aniso))


def rof_energy(u: np.ndarray, f: np.ndarray, alpha: float, lam: float,
               aniso: bool = False) -> float:
    H, W = f.shape
    u = np.ascontiguousarray(u, dtype=np.float64)
    fd = np.ascontiguousarray(f, dtype=np.float64)
    fn = _load().orc_rof_energy_aniso if aniso else _load().orc_rof_energy
    return fn(H, W, _ptr(u), _ptr(fd), alpha, lam)


def unrolled_grad(P: Problem, iters: int, g_u: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Reverse pass through `iters` iterations from zero: given dL/du~ of the
    final unlifted image, (dL/df [N], dL/d(lambda, alpha, nu) [3])."""
    g = np.ascontiguousarray(g_u, dtype=np.float64).reshape(P.N)
    gf, gs = np.zeros(P.N), np.zeros(3)
    rc = _load().orc_unrolled_grad(P.ref(), iters, _ptr(g), _ptr(gf), _ptr(gs))
    if rc != 0:
        raise RuntimeError(f"oracle unrolled_grad failed ({rc})")
    return gf, gs


def movement(P: Problem, X: State, Xp: State) -> tuple[float, float]:
    """Squared movement of the primal and the dual iterate between two states
    in the metric of the theta = 1 steps: (sum |dx|^2/tau, sum |dy|^2/sigma)."""
    S = steps(P.with_theta(1.0))
    dx = (np.sum((X.u - Xp.u) ** 2) / S["tau_u"]
          + np.sum((X.s - Xp.s) ** 2 / S["tau_s"][None, :]))
    dy = (np.sum(((X.v - Xp.v) ** 2 + (X.z - Xp.z) ** 2) / S["sigma_vz"][None, :])
          + np.sum((X.px - Xp.px) ** 2 + (X.py - Xp.py) ** 2 + (X.pz - Xp.pz) ** 2) / S["sigma_p"]
          + np.sum((X.q - Xp.q) ** 2) / S["sigma_q"])
    return float(dx), float(dy)


def pdhg_adaptive(P: Problem, X: State, checks: int, every: int) -> float:
    """`checks` rounds of `every` iterations; after each round log theta moves
    a fraction w toward log(dx/dy), dx/dy the ratio of the primal to the dual
    movement in the theta = 1 metric; w starts at 1/2 and shrinks by 0.95 per
    round.  Returns the final theta."""
    th = P.theta if P.theta > 0 else 1.0
    w = 0.5
    for _ in range(checks):
        Pc = P.with_theta(th)
        Xp = X.copy(Pc)
        pdhg(Pc, X, every)
        dx, dy = movement(Pc, X, Xp)
        if dx > 0 and dy > 0 and np.isfinite(dx) and np.isfinite(dy):
            th = float(np.exp((1.0 - w) * np.log(th) + w * np.log(np.sqrt(dx / dy))))
            th = min(max(th, 1e-4), 1e6)
            w *= 0.95
    return th


def pdhg_averaged(P: Problem, X: State, iters: int, every: int = 1) -> State:
    """Run ``iters`` iterations in place on X and return the uniform average
    of the iterates after iterations every, 2 every, ... (u, s and the dual
    v, z, p, q; the average's extrapolated point is its own x).  Every iterate
    is feasible (u in [0,1]^k after the clamp, p_i in its ball, (v_i, z_i) in
    the scaled epigraph after the projection), all three sets are convex, so
    the average is feasible and P_hat and D evaluated at it bound the
    relaxation's optimum as those of any iterate do."""
    names = ("u", "s", "v", "z", "px", "py", "pz", "q")
    acc = {n: np.zeros_like(getattr(X, n)) for n in names}
    cnt = 0
    done = 0
    while done + every <= iters:
        pdhg(P, X, every)
        done += every
        for n in names:
            acc[n] += getattr(X, n)
        cnt += 1
    if done < iters:
        pdhg(P, X, iters - done)
    A = State(P)
    if cnt:
        for n in names:
            getattr(A, n)[...] = acc[n] / cnt
    A.ubar[...] = A.u
    A.sbar[...] = A.s
    return A


def solve_restarted(P: Problem, X: State, max_iters: int, rel_gap_tol: float, beta: float = 0.5,
                    every: int = 10, check: int = 500):
    """Primal-dual iterations with restarts from the averaged iterate.  The
    iterate is added to a running average every `every` iterations; every
    `check` iterations the relative gaps (P_hat - D) / max(|P_hat|, |D|, 1)
    of the average and of the last iterate are compared, and once the
    smaller is at most beta times the gap at the previous restart, the
    better point becomes the iterate (its extrapolated point its own x) and
    the average starts afresh.  Stops when that smaller gap is <= rel_gap_tol.
    Returns (X, iterations done, the best gap, restarts)."""
    names = ("u", "s", "v", "z", "px", "py", "pz", "q")

    def rel_gap(S):
        p, d, _ = energy(P, S)
        return (p - d) / max(abs(p), abs(d), 1.0)

    acc = {n: np.zeros_like(getattr(X, n)) for n in names}
    cnt, done, restarts = 0, 0, 0
    g_restart, best = float("inf"), float("inf")
    while done < max_iters:
        for _ in range(max(check // every, 1)):
            if done >= max_iters:
                break
            step = min(every, max_iters - done)
            pdhg(P, X, step)
            done += step
            for n in names:
                acc[n] += getattr(X, n)
            cnt += 1
        A = State(P)
        for n in names:
            getattr(A, n)[...] = acc[n] / cnt
        A.ubar[...] = A.u
        A.sbar[...] = A.s
        ga, gl = rel_gap(A), rel_gap(X)
        g = min(ga, gl)
        best = min(best, g)
        if g <= rel_gap_tol or g <= beta * g_restart:
            if ga < gl:
                X = A
            g_restart = g
            restarts += 1
            for n in names:
                acc[n][...] = 0.0
            cnt = 0
            if g <= rel_gap_tol:
                break
    return X, done, best, restarts
