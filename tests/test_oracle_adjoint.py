"""Pins of the oracle's reverse pass through the unrolled solve: FP64 central
finite differences (eps = 1e-6) of the oracle's own forward map, for lambda,
alpha, nu and random directions in f."""
import numpy as np
import pytest

import oracle as O
from paper_1512_01383_gb300 import synth


def loss_of(kind, f, clean, L, lam, alpha, nu, iters, theta=1.0, aniso=0):
    H, W = f.shape
    P = O.Problem(kind, H, W, L, 0.0, 1.0, lam=lam, alpha=alpha, nu=nu, f=f, theta=theta,
                  aniso=aniso)
    X = O.State(P)
    O.pdhg(P, X, iters)
    u = O.unlift(P, X.u)
    return float(((u - clean.reshape(-1)) ** 2).sum()), u, P


@pytest.mark.parametrize("kind,L,lam,alpha,nu,theta,aniso", [
    (O.TRUNC, 5, 0.25, 25.0, 0.1, 1.0, 0),
    (O.QUAD, 4, 0.2, 1.5, 0.0, 1.0, 0),
    (O.TRUNC, 5, 0.25, 25.0, 0.1, 16.0, 0),
    (O.TRUNC, 5, 0.25, 25.0, 0.1, 1.0, 1),
    (O.PERIODIC, 6, 0.2, 1.5, 0.4, 1.0, 0),
])
def test_reverse_pass_matches_central_differences(kind, L, lam, alpha, nu, theta, aniso):
    H, W, iters, eps = 5, 4, 30, 1e-6
    noisy, clean = synth.voronoi_ramps(H, W, 71, cells=3)
    f = synth.as_f32(noisy).astype(np.float64)
    loss, u, P = loss_of(kind, f, clean, L, lam, alpha, nu, iters, theta, aniso)
    gf, gs = O.unrolled_grad(P, iters, 2.0 * (u - clean.reshape(-1)))

    def fd(**kw):
        args = dict(lam=lam, alpha=alpha, nu=nu)
        hi, lo = dict(args), dict(args)
        (name, h), = kw.items()
        hi[name] += h
        lo[name] -= h
        return (loss_of(kind, f, clean, L, **hi, iters=iters, theta=theta, aniso=aniso)[0] -
                loss_of(kind, f, clean, L, **lo, iters=iters, theta=theta, aniso=aniso)[0]) / (2 * h)

    names = ["lam", "alpha"] + (["nu"] if kind == O.TRUNC else [])
    if kind == O.PERIODIC:
        names = ["lam", "alpha"]     # the period moves the pieces only by jumps
    for j, name in enumerate(["lam", "alpha", "nu"]):
        if name not in names:
            assert abs(gs[j]) <= 1e-6
            continue
        want = fd(**{name: eps})
        assert abs(gs[j] - want) <= 1e-4 * abs(want) + 1e-8, (name, gs[j], want)
    rng = np.random.default_rng(3)
    for _ in range(4):
        d = rng.standard_normal(f.shape)
        want = (loss_of(kind, f + eps * d, clean, L, lam, alpha, nu, iters, theta, aniso)[0] -
                loss_of(kind, f - eps * d, clean, L, lam, alpha, nu, iters, theta, aniso)[0]) / (2 * eps)
        got = float((gf.reshape(f.shape) * d).sum())
        assert abs(got - want) <= 1e-4 * abs(want) + 1e-8, (got, want)
