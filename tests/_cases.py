"""Shared test helpers: identical seeded problems for the oracle and the GPU."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_1512_01383_gb300 import synth

KIND_ORACLE = {0: O.QUAD, 1: O.TRUNC, 2: O.PL, 3: O.PERIODIC}


def case(kind: int, H: int, W: int, L: int, seed: int, **kw) -> dict:
    """A problem description with float32 inputs (what the GPU sees)."""
    if kind == 0:
        f = synth.as_f32(synth.gaussian_blobs(H, W, seed))
        d = dict(kind=0, H=H, W=W, L=L, gamma_min=0.0, gamma_max=1.0, lam=0.2, alpha=1.0, f=f)
    elif kind == 1:
        f = synth.as_f32(synth.voronoi_ramps(H, W, seed)[0])
        d = dict(kind=1, H=H, W=W, L=L, gamma_min=0.0, gamma_max=1.0, lam=0.25, alpha=25.0,
                 nu=0.1, f=f)
    elif kind == 3:
        f = synth.as_f32(synth.wrapped_phase(H, W, seed)[0])
        d = dict(kind=3, H=H, W=W, L=L, gamma_min=0.0, gamma_max=float(4 * np.pi), lam=0.05,
                 alpha=1.0, nu=float(2 * np.pi), f=f)
    else:
        ndisp = kw.pop("ndisp", 17)
        cost = synth.as_f32(synth.stereo_cost(H, W, seed, ndisp=ndisp)[0])
        d = dict(kind=2, H=H, W=W, L=L, gamma_min=0.0, gamma_max=float(ndisp - 1), lam=0.05,
                 cost=cost, sample_min=0.0, sample_max=float(ndisp - 1))
    d.update(kw)
    return d


def oracle_problem(c: dict) -> O.Problem:
    """The same problem in the oracle's FP64 types (inputs widened exactly)."""
    return O.Problem(KIND_ORACLE[c["kind"]], c["H"], c["W"], c["L"], c["gamma_min"],
                     c["gamma_max"], lam=c["lam"], alpha=c.get("alpha", 1.0), nu=c.get("nu", 0.0),
                     f=None if c.get("f") is None else c["f"].astype(np.float64),
                     cost=None if c.get("cost") is None else c["cost"].astype(np.float64),
                     smin=c.get("sample_min", 0.0), smax=c.get("sample_max", 1.0),
                     theta=c.get("theta", 1.0), aniso=int(c.get("aniso", 0)))


def crop(c: dict, y0: int, y1: int, x0: int, x1: int) -> dict:
    d = dict(c)
    d["H"], d["W"] = y1 - y0, x1 - x0
    if d.get("f") is not None:
        d["f"] = np.ascontiguousarray(c["f"][y0:y1, x0:x1])
    if d.get("cost") is not None:
        d["cost"] = np.ascontiguousarray(c["cost"][y0:y1, x0:x1])
    return d


def gpu_solver(c: dict, device_inputs: bool = True, **kw):
    """Create the GPU solver for case c (inputs uploaded from torch tensors)."""
    import torch

    from paper_1512_01383_gb300 import lift as G
    f = cost = None
    if c.get("f") is not None:
        f = torch.from_numpy(c["f"]).cuda() if device_inputs else c["f"]
    if c.get("cost") is not None:
        cost = torch.from_numpy(c["cost"]).cuda() if device_inputs else c["cost"]
    return G.Solver(c["kind"], c["H"], c["W"], c["L"], c["gamma_min"], c["gamma_max"], c["lam"],
                    c.get("alpha", 1.0), c.get("nu", 0.0), f=f, cost=cost,
                    sample_min=c.get("sample_min", 0.0), sample_max=c.get("sample_max", 1.0),
                    step_balance=c.get("theta", 1.0), anisotropic=bool(c.get("aniso", 0)), **kw)


def oracle_run(c: dict, iters: int):
    P = oracle_problem(c)
    X = O.State(P)
    O.pdhg(P, X, iters)
    return P, X


def crop_oracle_pixel(job):
    """Worker for parity at full size: run the oracle on a crop and return
    the unlifted value and the state rows of one pixel of it.  job = (case,
    (y0, y1, x0, x1), iters, (py, px)) with (py, px) in image coordinates."""
    c, (y0, y1, x0, x1), iters, (py_, px_) = job
    P, X = oracle_run(crop(c, y0, y1, x0, x1), iters)
    j = (py_ - y0) * (x1 - x0) + (px_ - x0)
    rows = {name: np.array(getattr(X, name)[j]) for name in ("u", "s", "v", "z", "px", "py")}
    return float(O.unlift(P, X.u)[j]), rows
