"""Worked examples with hand-derived values (tests/golden/, each file citing
the passage it follows): the oracle must reproduce them.  The same
two-pixel problems run on the GPU in test_gpu_parity."""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden(name: str) -> np.ndarray:
    return np.atleast_2d(np.loadtxt(os.path.join(GOLDEN, name), comments="#"))


@pytest.mark.parametrize("row", list(golden("rof_two_pixel.txt")))
def test_two_pixel_rof_closed_form(row):
    """L = 2 (Prop. 3) on two pixels: at convergence the lifted iterate
    unlifts to the soft-thresholded pair and every energy bound meets the
    closed-form optimum."""
    f1, f2, lam, u1, u2, E = row
    P = O.Problem(O.QUAD, 1, 2, 2, 0.0, 1.0, lam=lam, alpha=1.0, f=np.array([f1, f2]))
    X = O.State(P)
    O.pdhg(P, X, 20000)
    ut = O.unlift(P, X.u)
    assert np.abs(ut - [u1, u2]).max() <= 1e-7, ut
    Ph, D, Enc = O.energy(P, X)
    assert D <= E + 1e-9 and Ph >= E - 1e-9          # weak duality around the optimum
    for v in (Ph, D, Enc):
        assert abs(v - E) <= 1e-7, (v, E)


@pytest.mark.parametrize("row", list(golden("quad_piece_conjugate.txt")))
def test_quadratic_piece_conjugate(row):
    f, alpha, L, i, y, c, t = row
    P = O.Problem(O.QUAD, 1, 1, int(L), 0.0, 1.0, alpha=alpha, f=np.array([f]))
    val, arg = O.conj(P, 0, int(i), y)
    assert abs(val - c) <= 1e-12, (val, c)
    assert abs(arg - t) <= 1e-12, (arg, t)


@pytest.mark.parametrize("row", list(golden("trunc_chain.txt")))
def test_truncated_chain_closed_form(row):
    """Truncated-quadratic data (Sec. 5.2) on 1-D chains of two and three
    pixels: at convergence the unlifted image is the hand-derived optimum and
    P, D and the nonconvex energy E_nc all meet its energy."""
    _, L, lam, f1, f2, f3, u1, u2, u3, E = row
    f = np.array([f1, f2, f3] if f3 >= 0 else [f1, f2])
    want = np.array([u1, u2, u3] if f3 >= 0 else [u1, u2])
    P = O.Problem(O.TRUNC, 1, len(f), int(L), 0.0, 1.0, lam=lam, alpha=25.0, nu=0.1, f=f)
    X = O.State(P)
    O.pdhg(P, X, 60000)
    ut = O.unlift(P, X.u)
    assert np.abs(ut - want).max() <= 1e-7, ut
    Ph, D, Enc = O.energy(P, X)
    assert D <= E + 1e-9 and Ph >= E - 1e-9
    for v in (Ph, D, Enc):
        assert abs(v - E) <= 1e-7, (v, E)


PL_COSTS = np.array([[3.0, 1.0, 0.0, 1.0, 3.0], [0.0, 1.5, 3.0, 4.5, 6.0]])


@pytest.mark.parametrize("row", list(golden("pl_two_pixel.txt")))
def test_pl_two_pixel_closed_form(row):
    """Sampled (piecewise-linear) costs (Sec. 5.4) on two pixels at L = 2
    (Prop. 3): at convergence the unlifted pair is the hand-derived optimum
    and P, D and the nonconvex E_nc all meet its energy."""
    lam, u1, u2, E = row
    P = O.Problem(O.PL, 1, 2, 2, 0.0, 4.0, lam=lam, cost=PL_COSTS, smin=0.0, smax=4.0)
    X = O.State(P)
    O.pdhg(P, X, 20000)
    ut = O.unlift(P, X.u)
    assert np.abs(ut - [u1, u2]).max() <= 1e-7, ut
    Ph, D, Enc = O.energy(P, X)
    assert D <= E + 1e-9 and Ph >= E - 1e-9
    for v in (Ph, D, Enc):
        assert abs(v - E) <= 1e-7, (v, E)


@pytest.mark.parametrize("row", list(golden("periodic_two_pixel.txt")))
def test_periodic_two_pixel_closed_form(row):
    """Wrapped phases on either side of the wrap (Sec. 5.5) on two pixels:
    at convergence the unlifted pair is the hand-derived unwrapped optimum,
    and P, D and the nonconvex E_nc (the squared circular distance) all meet
    its energy."""
    L, lam, alpha, u1, u2, E = row
    two_pi = 2 * np.pi
    f = np.array([two_pi - 0.3, 0.3])
    P = O.Problem(O.PERIODIC, 1, 2, int(L), 0.0, 2 * two_pi, lam=lam, alpha=alpha, nu=two_pi, f=f)
    X = O.State(P)
    O.pdhg(P, X, 40000)
    ut = O.unlift(P, X.u)
    assert np.abs(ut - [u1, u2]).max() <= 1e-7, ut
    Ph, D, Enc = O.energy(P, X)
    assert D <= E + 1e-9 and Ph >= E - 1e-9
    for v in (Ph, D, Enc):
        assert abs(v - E) <= 1e-7, (v, E)
