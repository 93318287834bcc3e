"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks one oracle function against something other than itself:
brute force over fine grids, the variational characterisation of a
projection, closed forms stated by the propositions of arXiv 1512.01383, or an
independent solver.  A plausible slip (a dropped term of c_i, a wrong sign
in the primal update, a transposed difference) fails at least one of them.
"""
import numpy as np
import pytest

import oracle as O
from paper_1512_01383_gb300 import synth


def lower_hull_values(ts, vals, tq):
    """Brute-force lower convex envelope of the points (ts, vals), at tq.

    Independent of the oracle: monotone-chain lower hull, then linear
    interpolation along the hull."""
    hx, hy = [], []
    for x, y in zip(ts, vals):
        while len(hx) >= 2:
            x1, y1, x2, y2 = hx[-2], hy[-2], hx[-1], hy[-1]
            if (x2 - x1) * (y - y1) - (y2 - y1) * (x - x1) <= 0.0:
                hx.pop(); hy.pop()
            else:
                break
        hx.append(x); hy.append(y)
    return np.interp(tq, hx, hy)


def make_problems():
    """One small problem of each data-term kind, inputs rounded to float32."""
    H, W = 3, 4
    f = synth.as_f32(synth.voronoi_ramps(H, W, 11)[0]).astype(np.float64)
    cost, _ = synth.stereo_cost(H, W, 12, ndisp=17, tau=0.2)
    cost = synth.as_f32(cost).astype(np.float64)
    return [
        O.Problem(O.QUAD, H, W, 4, 0.0, 1.0, lam=0.2, alpha=1.7, f=f),
        O.Problem(O.TRUNC, H, W, 5, 0.0, 1.0, lam=0.25, alpha=25.0, nu=0.1, f=f),
        O.Problem(O.TRUNC, H, W, 3, -0.5, 1.5, lam=0.25, alpha=25.0, nu=0.1, f=f),
        O.Problem(O.PL, H, W, 6, 0.0, 16.0, lam=0.05, cost=cost, smin=0.0, smax=16.0),
    ]


def brute_rho(P, pix, t):
    t = np.asarray(t, dtype=np.float64)
    if P.kind == O.QUAD:
        return 0.5 * P.alpha * (t - P.f[pix]) ** 2
    if P.kind == O.TRUNC:
        return np.minimum(P.alpha * (t - P.f[pix]) ** 2, P.nu)
    xs = np.linspace(P.smin, P.smax, P.cost.shape[1])
    return np.interp(t, xs, P.cost[pix])


# --------------------------------------------------------------------------
# rho and rho_i^* (Prop. 1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pi", range(4))
def test_rho_matches_definition(pi):
    P = make_problems()[pi]
    ts = np.linspace(P.gmin, P.gmax, 37)
    for pix in (0, 5, P.N - 1):
        got = np.array([O.rho(P, pix, t) for t in ts])
        np.testing.assert_allclose(got, brute_rho(P, pix, ts), rtol=0, atol=1e-12)


@pytest.mark.parametrize("pi", range(4))
def test_conj_brute_force(pi):
    """rho_i^*(y) = sup_{t in Gamma_i} t y - rho(t) against a 10^6-point grid."""
    P = make_problems()[pi]
    lab = O.labels(P.L, P.gmin, P.gmax)
    r = synth.Rng(7, pi)
    for pix in (0, 7, P.N - 1):
        for i in range(P.k):
            l, rr = lab[i], lab[i + 1]
            grid = np.linspace(l, rr, 1_000_001)
            if P.kind == O.PL:   # include the sample positions exactly
                xs = np.linspace(P.smin, P.smax, P.cost.shape[1])
                grid = np.union1d(grid, xs[(xs > l) & (xs < rr)])
            rv = brute_rho(P, pix, grid)
            scale = 3.0 * (abs(P.alpha) + 1.0) * (P.gmax - P.gmin + 1.0)
            for y in r.uniform(9, -scale, scale):
                val, t = O.conj(P, pix, i, y)
                bf = np.max(grid * y - rv)
                assert val >= bf - 1e-12
                assert val <= bf + 1e-9 * (1 + abs(bf))
                # the reported maximiser attains the value
                assert abs(t * y - O.rho(P, pix, t) - val) < 1e-12 * (1 + abs(val))


@pytest.mark.parametrize("pi", range(4))
def test_lifted_conj_prop1_appendix_form(pi):
    """Prop. 1: the conjugate of the lifted data term, sup over graph points
    1_i^alpha of <1_i^alpha, v> - rho(gamma_i^alpha), equals
    max_i c_i(v) + rho_i^*(v_i/Delta_i) with c_i(v) = <1_{i-1},v> - gamma_i v_i/Delta_i.
    Brute force over all pieces and 20001 values of alpha each."""
    P = make_problems()[pi]
    lab = O.labels(P.L, P.gmin, P.gmax)
    r = synth.Rng(9, pi)
    al = np.linspace(0.0, 1.0, 20001)
    for pix in (1, P.N - 2):
        for _ in range(6):
            v = r.uniform(P.k, -3.0, 3.0) * (P.gmax - P.gmin)
            best = -np.inf
            for i in range(P.k):
                pts = lab[i] + al * (lab[i + 1] - lab[i])
                inner = v[:i].sum() + al * v[i]          # <1_i^alpha, v>
                best = max(best, np.max(inner - brute_rho(P, pix, pts)))
            got = O.lifted_conj(P, pix, v)
            assert abs(got - best) <= 1e-6 * (1 + abs(best))


# --------------------------------------------------------------------------
# Projection onto epi(rho_i^*)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pi", range(4))
def test_proj_epi_variational(pi):
    """Projection onto a convex set: the result lies in the set, points of the
    set are fixed, and <x - P(x), w - P(x)> <= 0 for every w in the set
    (checked on dense samples of the graph and of points above it)."""
    P = make_problems()[pi]
    r = synth.Rng(13, pi)
    scale = 2.0 * (abs(P.alpha) + 1.0) * (P.gmax - P.gmin + 1.0)
    for pix in (0, 6, P.N - 1):
        for i in range(P.k):
            ys = np.linspace(-4 * scale, 4 * scale, 4001)
            phis = np.array([O.conj(P, pix, i, y)[0] for y in ys])
            for _ in range(8):
                y0 = r.uniform(1, -2 * scale, 2 * scale)[0]
                phi0 = O.conj(P, pix, i, y0)[0]
                h0 = phi0 + r.uniform(1, -3 * scale, 1.0)[0]
                yp, hp = O.proj_epi(P, pix, i, y0, h0)
                assert hp >= O.conj(P, pix, i, yp)[0] - 1e-10 * (1 + abs(hp))
                if h0 >= phi0:
                    assert (yp, hp) == (y0, h0)
                # variational inequality against graph points and points above
                for lift in (0.0, 1.0):
                    ip = (y0 - yp) * (ys - yp) + (h0 - hp) * (phis + lift - hp)
                    assert ip.max() <= 1e-8 * (1 + scale * scale)
                # idempotence
                y2, h2 = O.proj_epi(P, pix, i, yp, hp + 1e-12 * (1 + abs(hp)))
                assert abs(y2 - yp) <= 1e-9 * (1 + abs(yp))


def test_proj_epi_brute_nearest():
    """Distance to the graph computed by brute force over 2*10^5 graph points."""
    P = make_problems()[1]
    r = synth.Rng(17, 0)
    for pix in (2, 9):
        for i in range(P.k):
            ys = np.linspace(-60, 60, 200001)
            phis = np.array([O.conj(P, pix, i, y)[0] for y in ys[::50]])
            phis = np.interp(ys, ys[::50], phis)  # phi is piecewise smooth
            for _ in range(5):
                y0 = r.uniform(1, -20, 20)[0]
                h0 = O.conj(P, pix, i, y0)[0] - r.uniform(1, 0.01, 5)[0]
                yp, hp = O.proj_epi(P, pix, i, y0, h0)
                dbf = np.sqrt(((ys - y0) ** 2 + (phis - h0) ** 2).min())
                d = np.hypot(yp - y0, hp - h0)
                assert d <= dbf + 1e-6
                assert d >= dbf - 1e-3


# --------------------------------------------------------------------------
# rho_i^** (the convexified pieces)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("pi", range(4))
def test_biconj_is_lower_convex_envelope(pi):
    """rho_i^** on Gamma_i equals the lower convex hull of rho restricted to
    Gamma_i (brute force hull of a dense sampling; exact at PL samples)."""
    P = make_problems()[pi]
    lab = O.labels(P.L, P.gmin, P.gmax)
    for pix in (0, 4, P.N - 1):
        for i in range(P.k):
            l, rr = lab[i], lab[i + 1]
            ts = np.linspace(l, rr, 20001)
            if P.kind == O.PL:
                xs = np.linspace(P.smin, P.smax, P.cost.shape[1])
                ts = np.union1d(ts, xs[(xs > l) & (xs < rr)])
            hull_t = np.linspace(l, rr, 23)
            want = lower_hull_values(ts, brute_rho(P, pix, ts), hull_t)
            got = np.array([O.biconj(P, pix, i, t) for t in hull_t])
            tol = 1e-9 if P.kind == O.PL else 2e-6 * (1 + P.alpha)
            np.testing.assert_allclose(got, want, rtol=0, atol=tol)


def test_biconj_keeps_minimum():
    """The envelope keeps the minimum value of each piece."""
    for P in make_problems():
        lab = O.labels(P.L, P.gmin, P.gmax)
        for pix in range(P.N):
            for i in range(P.k):
                ts = np.linspace(lab[i], lab[i + 1], 4001)
                rv = brute_rho(P, pix, ts)
                # a minimiser of rho on the piece lies on its lower hull
                got = O.biconj(P, pix, i, ts[np.argmin(rv)])
                assert abs(got - rv.min()) <= 1e-9 * (1 + abs(rv.min()))


# --------------------------------------------------------------------------
# grad / div, monotone projection, unlifting
# --------------------------------------------------------------------------
def test_grad_div_adjoint():
    r = synth.Rng(21)
    for H, W, k in ((1, 1, 1), (1, 7, 2), (5, 1, 3), (6, 9, 4)):
        u = r.uniform(H * W * k, -1, 1)
        px, py = r.uniform(H * W * k, -1, 1), r.uniform(H * W * k, -1, 1)
        gx, gy = O.grad(H, W, k, u)
        d = O.div(H, W, k, px, py)
        assert abs((gx * px + gy * py).sum() + (u * d).sum()) < 1e-12
        # Neumann: no difference across the last column / row
        g = gx.reshape(H, W, k)
        assert np.all(g[:, -1, :] == 0)
        g = gy.reshape(H, W, k)
        assert np.all(g[-1, :, :] == 0)
        # forward difference in the interior
        U = u.reshape(H, W, k)
        if W > 1:
            np.testing.assert_allclose(gx.reshape(H, W, k)[:, :-1], U[:, 1:] - U[:, :-1])
        if H > 1:
            np.testing.assert_allclose(gy.reshape(H, W, k)[:-1], U[1:] - U[:-1])


def test_monotone_projection_bruteforce():
    """clamp(PAV) is the Euclidean projection onto {1>=w_1>=...>=w_k>=0}:
    its residual satisfies the variational inequality against many feasible
    points, and it equals brute force on k=2."""
    r = synth.Rng(23)
    for k in (1, 2, 3, 7):
        for _ in range(30):
            u = r.uniform(k, -0.5, 1.5)
            w = O.monotone_proj(u)
            assert np.all(np.diff(w) <= 1e-15) and w.min() >= 0 and w.max() <= 1
            feas = np.sort(r.uniform(200 * k, 0, 1).reshape(200, k), axis=1)[:, ::-1]
            assert ((u - w)[None, :] * (feas - w[None, :])).sum(1).max() <= 1e-12
    g = np.linspace(0, 1, 401)
    A, B = np.meshgrid(g, g, indexing="ij")
    m = A >= B
    for _ in range(10):
        u = r.uniform(2, -0.5, 1.5)
        d = (A - u[0]) ** 2 + (B - u[1]) ** 2
        d[~m] = np.inf
        j = np.unravel_index(np.argmin(d), d.shape)
        w = O.monotone_proj(u)
        assert abs(w[0] - g[j[0]]) <= 2.5e-3 and abs(w[1] - g[j[1]]) <= 2.5e-3


def test_unlift_layer_cake():
    """Layer-cake formula of Sec. 3 on graph vectors 1_i^alpha."""
    P = O.Problem(O.QUAD, 1, 5, 5, -1.0, 3.0, f=np.zeros(5))
    lab = O.labels(5, -1.0, 3.0)
    u = np.zeros((5, 4))
    want = []
    for pix, (i, a) in enumerate([(0, 0.0), (0, 0.3), (1, 1.0), (2, 0.5), (3, 1.0)]):
        vec = np.zeros(4)
        vec[:i] = 1.0
        vec[i] = a
        u[pix] = vec
        want.append(lab[i] + a * (lab[i + 1] - lab[i]))
    np.testing.assert_allclose(O.unlift(P, u), want, atol=1e-15)


# --------------------------------------------------------------------------
# TV set K (Props. 4 and 5)
# --------------------------------------------------------------------------
def test_projected_p_satisfies_infinite_constraints():
    """After PDHG steps, p lies in the ball product of Prop. 5; sampling the
    infinitely many constraints of Prop. 4 (scaled by lambda) finds no
    violation, and a p with one ball violated breaks Prop. 4 at i=j."""
    f = synth.voronoi_ramps(5, 6, 31)[0]
    P = O.Problem(O.TRUNC, 5, 6, 6, 0.0, 1.0, lam=0.3, alpha=25.0, nu=0.1, f=f)
    X = O.State(P)
    O.pdhg(P, X, 40)
    lab = O.labels(P.L, 0, 1)
    r = synth.Rng(33)
    p = np.stack([X.px, X.py], axis=-1)        # [N, k, 2]
    assert np.abs(p).max() > 0
    for pix in range(P.N):
        for _ in range(60):
            j, i = sorted(r.integers(2, 0, P.k - 1))
            a, b = r.uniform(2)
            vec = p[pix, j:i].sum(0) + a * p[pix, i] - b * p[pix, j]
            rhs = abs((lab[i] + a * (lab[i + 1] - lab[i])) - (lab[j] + b * (lab[j + 1] - lab[j])))
            assert np.linalg.norm(vec) <= P.lam * rhs + 1e-12
    pb = p[0].copy()
    pb[2] *= 1.001 * P.lam * (lab[3] - lab[2]) / max(np.linalg.norm(pb[2]), 1e-30)
    vec = 1.0 * pb[2] - 0.0 * pb[2]
    assert np.linalg.norm(vec) > P.lam * (lab[3] - lab[2])


# --------------------------------------------------------------------------
# Whole-solver pins
# --------------------------------------------------------------------------
def test_steps_are_reciprocal_abs_sums():
    """Preconditioners: reciprocal absolute row/column sums of the operator
    assembled explicitly as a dense matrix for one interior pixel's block."""
    P = O.Problem(O.TRUNC, 1, 1, 5, -0.4, 2.0, f=np.zeros(1), alpha=1, nu=1)
    k = P.k
    lab = O.labels(P.L, P.gmin, P.gmax)
    d = np.diff(lab)
    # rows: v (k), z (k), q (1); columns: u (k), s (k)
    K = np.zeros((2 * k + 1, 2 * k))
    for l in range(k):
        K[l, l] = 1.0
        K[l, k + l] = -lab[l]
        for j in range(l + 1, k):
            K[l, k + j] = d[j]
        K[k + l, k + l] = 1.0
        K[2 * k, k + l] = -d[l]
    st = O.steps(P)
    col = np.abs(K).sum(0)
    row = np.abs(K).sum(1)
    np.testing.assert_allclose(st["tau_s"], 1.0 / col[k:], rtol=1e-14)
    # u columns also carry the 4 entries of the 2-D forward difference
    assert st["tau_u"] == pytest.approx(1.0 / (col[0] + 4))
    np.testing.assert_allclose(st["sigma_vz"], 1.0 / np.maximum(row[:k], row[k:2 * k]), rtol=1e-14)
    assert st["sigma_q"] == pytest.approx(1.0 / row[2 * k])
    assert st["sigma_p"] == 0.5


def test_step_balance_keeps_step_products():
    """theta multiplies the primal steps and divides the dual ones, so every
    product tau*sigma (and the convergence condition) is unchanged."""
    base = O.Problem(O.TRUNC, 1, 1, 7, -0.3, 1.4, f=np.zeros(1), alpha=1, nu=1)
    for th in (0.25, 1.0, 49.0):
        P = O.Problem(O.TRUNC, 1, 1, 7, -0.3, 1.4, f=np.zeros(1), alpha=1, nu=1, theta=th)
        a, b = O.steps(base), O.steps(P)
        np.testing.assert_allclose(b["tau_s"], th * a["tau_s"], rtol=1e-15)
        np.testing.assert_allclose(b["sigma_vz"], a["sigma_vz"] / th, rtol=1e-15)
        assert b["tau_u"] == pytest.approx(th * a["tau_u"])
        assert b["sigma_q"] == pytest.approx(a["sigma_q"] / th)
        assert b["sigma_p"] == pytest.approx(a["sigma_p"] / th)


@pytest.mark.parametrize("theta", [0.3, 4.0])
def test_step_balance_reaches_the_same_optimum(theta):
    """Any balance converges to the same optimum: L = 2 ROF against the
    independent direct solver."""
    f = synth.gaussian_blobs(9, 8, 45)
    u_dir, gap = O.rof_direct(f, 1.0, 0.2, 0.0, 1.0, 100000)
    Er = O.rof_energy(u_dir, f, 1.0, 0.2)
    P = O.Problem(O.QUAD, 9, 8, 2, 0.0, 1.0, lam=0.2, alpha=1.0, f=f, theta=theta)
    X = O.State(P)
    O.pdhg(P, X, 6000)
    Ph, D, _ = O.energy(P, X)
    assert D <= Er + 1e-12 and abs(Ph - Er) < 1e-8 * Er and abs(D - Er) < 1e-8 * Er
    assert np.abs(O.unlift(P, X.u).reshape(9, 8) - u_dir).max() < 2e-5


@pytest.mark.parametrize("alpha", [1.0, 2.5])
def test_L2_equals_direct_rof(alpha):
    """Prop. 3: with L = 2 the relaxation is the unlifted problem; for the
    quadratic data term it is box-constrained ROF, solved here independently
    by the accelerated primal-dual method."""
    f = synth.gaussian_blobs(10, 9, 41)
    P = O.Problem(O.QUAD, 10, 9, 2, 0.0, 1.0, lam=0.2, alpha=alpha, f=f)
    X = O.State(P)
    O.pdhg(P, X, 4000)
    u_dir, gap = O.rof_direct(f, alpha, 0.2, 0.0, 1.0, 100000)
    assert gap < 1e-9
    Er = O.rof_energy(u_dir, f, alpha, 0.2)
    Ph, D, E = O.energy(P, X)
    ut = O.unlift(P, X.u).reshape(10, 9)
    Eu = O.rof_energy(ut, f, alpha, 0.2)
    # weak duality across the two solvers, and both at the same optimum
    assert D <= Er + 1e-12 and D <= Eu + 1e-12
    assert abs(Ph - Er) < 1e-8 * Er and abs(D - Er) < 1e-8 * Er
    # strong convexity (modulus alpha): |u - u*|^2 <= 2 (E(u) - D) / alpha
    assert np.sqrt(2 * (Eu - D) / alpha) < 1e-4
    assert np.abs(ut - u_dir).max() < 2e-5


def test_convex_data_tight_for_more_labels():
    """For a convex data term the relaxation is tight at any label count
    (Sec. 5.1).  On a 1-D signal the lifted TV of a graph function equals the
    TV of the unlifted signal, so L = 3 must reach the direct ROF optimum and
    L = 6 must never certify a lower bound above it.  (On a 2-D grid the
    discrete lifted TV sum_i Delta_i |grad u_i| exceeds the isotropic TV of
    the unlifted image wherever the x and y differences cross different
    intervals, so the two discrete problems differ for L > 2.)"""
    f = synth.gaussian_blobs(1, 40, 43, noise=0.05)
    u_dir, gap = O.rof_direct(f, 1.0, 0.15, 0.0, 1.0, 100000)
    assert gap < 1e-9
    Er = O.rof_energy(u_dir, f, 1.0, 0.15)
    P = O.Problem(O.QUAD, 1, 40, 3, 0.0, 1.0, lam=0.15, alpha=1.0, f=f)
    X = O.State(P)
    O.pdhg(P, X, 12000)
    Ph, D, E = O.energy(P, X)
    assert abs(Ph - Er) < 1e-8 and abs(D - Er) < 1e-8
    assert np.abs(O.unlift(P, X.u) - u_dir.ravel()).max() < 1e-5
    P6 = O.Problem(O.QUAD, 1, 40, 6, 0.0, 1.0, lam=0.15, alpha=1.0, f=f)
    X6 = O.State(P6)
    for _ in range(4):
        O.pdhg(P6, X6, 1500)
        Ph, D, E = O.energy(P6, X6)
        assert D <= Er + 1e-9 and Ph >= Er - 1e-9


@pytest.mark.parametrize("kind", [O.QUAD, O.TRUNC])
def test_lambda0_pixelwise_minimum(kind):
    """lambda = 0 decouples pixels; the optimum is the per-pixel minimum of rho
    on Gamma (the envelope keeps the minimum), attained at clamp(f)."""
    f = synth.gaussian_blobs(4, 5, 47)
    P = O.Problem(kind, 4, 5, 5, 0.0, 1.0, lam=0.0, alpha=3.0, nu=0.2, f=f)
    X = O.State(P)
    tc = np.clip(f.reshape(-1), 0, 1)
    opt = sum(O.rho(P, j, tc[j]) for j in range(P.N))
    gaps, errs = [], []
    for _ in range(8):
        O.pdhg(P, X, 2000)
        Ph, D, E = O.energy(P, X)
        # the closed-form optimum lies between the two certified bounds
        assert D <= opt + 1e-9 and Ph >= opt - 1e-9
        gaps.append(Ph - D)
        errs.append(np.abs(O.unlift(P, X.u) - tc).max())
    assert gaps[-1] < 0.1 * gaps[0] and gaps[-1] < 2e-3
    assert errs[-1] < 0.6 * errs[0] and errs[-1] < 1e-2


def test_prop2_linear_pieces_closed_form():
    """Prop. 2: if rho is linear on each interval, the relaxed data term of a
    monotone u is rho(gamma_1) + <u, r>, r_i = rho(gamma_{i+1}) - rho(gamma_i),
    whatever decomposition the energy evaluation picks (lambda = 0)."""
    L = 5
    cost = synth.Rng(51).uniform(3 * L, 0, 2).reshape(3, L)
    P = O.Problem(O.PL, 1, 3, L, 0.0, 4.0, lam=0.0, cost=cost, smin=0.0, smax=4.0)
    X = O.State(P)
    r = synth.Rng(52)
    X.u[...] = np.sort(r.uniform(3 * (L - 1)).reshape(3, L - 1), axis=1)[:, ::-1]
    X.s[...] = r.uniform(3 * (L - 1), -1, 0.2).reshape(3, L - 1)
    Ph, _, _ = O.energy(P, X)
    want = sum(cost[j, 0] + X.u[j] @ np.diff(cost[j]) for j in range(3))
    assert abs(Ph - want) < 1e-12 * (1 + abs(want))


def test_gap_nonnegative_and_decreasing():
    """Weak duality: P_hat >= D at every check; the gap shrinks."""
    f = synth.voronoi_ramps(7, 6, 53)[0]
    P = O.Problem(O.TRUNC, 7, 6, 5, 0.0, 1.0, lam=0.25, alpha=25.0, nu=0.1, f=f)
    X = O.State(P)
    gaps = []
    for _ in range(8):
        O.pdhg(P, X, 250)
        Ph, D, _ = O.energy(P, X)
        assert Ph >= D - 1e-10
        gaps.append(Ph - D)
    assert gaps[-1] < 0.2 * gaps[0]


def test_monotone_label_order_at_convergence():
    f = synth.voronoi_ramps(5, 5, 55)[0]
    P = O.Problem(O.TRUNC, 5, 5, 4, 0.0, 1.0, lam=0.25, alpha=25.0, nu=0.1, f=f)
    X = O.State(P)
    O.pdhg(P, X, 6000)
    assert np.diff(X.u, axis=1).max() <= 1e-4


def viterbi_1d(costs, lam, h):
    """Exact min over a label grid of sum_x c_x(t_x) + lam sum |t_{x+1}-t_x|
    (distance-transform DP)."""
    m = costs[0].copy()
    j = np.arange(costs.shape[1]) * h
    for c in costs[1:]:
        fwd = np.minimum.accumulate(m - lam * j) + lam * j
        bwd = (np.minimum.accumulate((m + lam * j)[::-1]) - lam * j[::-1])[::-1]
        m = np.minimum(fwd, bwd) + c
    return m.min()


@pytest.mark.parametrize("seed", [61, 62, 63])
def test_1d_dynamic_programming_bound(seed):
    """1-D nonconvex signals: the relaxed energy of graph functions is
    sum_x rho_i^**(t_x) + lam |t_{x+1} - t_x|; DP over a 4001-label grid with
    the brute-force per-interval envelopes bounds the relaxed optimum from
    above, so the oracle's dual bound must not exceed it, and the oracle's
    primal bound must approach it when the relaxation is tight."""
    n, L = 20, 5
    f = synth.voronoi_ramps(1, n, seed, cells=3)[0]
    P = O.Problem(O.TRUNC, 1, n, L, 0.0, 1.0, lam=0.15, alpha=25.0, nu=0.1, f=f)
    lab = O.labels(L, 0, 1)
    G = 4001
    grid = np.linspace(0, 1, G)
    env = np.zeros((n, G))
    for x in range(n):
        for i in range(P.k):
            m = (grid >= lab[i]) & (grid <= lab[i + 1])
            ts = np.linspace(lab[i], lab[i + 1], 8001)
            env[x, m] = lower_hull_values(ts, brute_rho(P, x, ts), grid[m])
    E_dp = viterbi_1d(env, P.lam, grid[1] - grid[0])
    X = O.State(P)
    O.pdhg(P, X, 20000)
    Ph, D, _ = O.energy(P, X)
    assert D <= E_dp + 1e-9
    assert Ph >= D
    if Ph - D < 1e-6:
        # converged; the relaxed optimum E* lies in [D, P_hat] and the DP on a
        # grid of step 2.5e-4 overestimates the graph optimum only slightly
        assert E_dp - D < 2e-3


def test_adaptive_balance_converges_like_tuned_balance():
    """The movement-balancing rule, started from theta = 1, reaches a gap
    within a small factor of the hand-tuned constant balance and far below
    the plain preconditioner's (truncated quadratic, L = 10)."""
    f = synth.voronoi_ramps(16, 16, 57)[0]

    def gap_after(theta, adaptive):
        P = O.Problem(O.TRUNC, 16, 16, 10, 0.0, 1.0, lam=0.25, alpha=25.0, nu=0.1, f=f,
                      theta=theta)
        X = O.State(P)
        if adaptive:
            O.pdhg_adaptive(P, X, 20, 100)
        else:
            O.pdhg(P, X, 2000)
        Ph, D, _ = O.energy(P, X)
        assert Ph >= D - 1e-10
        return (Ph - D) / max(abs(Ph), abs(D), 1.0)

    ga, gt, g1 = gap_after(1.0, True), gap_after(81.0, False), gap_after(1.0, False)
    assert ga < 0.1 * g1 and ga < 5.0 * gt, (ga, gt, g1)


def test_movement_is_weighted_squared_change():
    P = O.Problem(O.TRUNC, 3, 4, 5, 0.0, 1.0, lam=0.25, alpha=25.0, nu=0.1,
                  f=synth.voronoi_ramps(3, 4, 58)[0], theta=7.0)
    X, Y = O.State(P), O.State(P)
    Y.u[1, 2] = 0.5
    Y.q[3] = 2.0
    st = O.steps(O.Problem(O.TRUNC, 3, 4, 5, 0.0, 1.0, lam=0.25, alpha=25.0, nu=0.1, f=P.f))
    dx, dy = O.movement(P, Y, X)
    assert dx == pytest.approx(0.25 / st["tau_u"])
    assert dy == pytest.approx(4.0 / st["sigma_q"])


# --------------------------------------------------------------------------
# Anisotropic TV (Sec. 5.3: Props. 4-5 hold for phi = |.|_1)
# --------------------------------------------------------------------------
def test_anisotropic_L2_equals_direct_anisotropic_rof():
    """With phi = |.|_1 and L = 2 the relaxation is box-constrained ROF with
    the anisotropic TV |grad u|_1, solved independently."""
    f = synth.gaussian_blobs(10, 9, 141)
    P = O.Problem(O.QUAD, 10, 9, 2, 0.0, 1.0, lam=0.2, alpha=1.0, f=f, aniso=1)
    X = O.State(P)
    O.pdhg(P, X, 5000)
    u_dir, gap = O.rof_direct(f, 1.0, 0.2, 0.0, 1.0, 100000, aniso=True)
    assert gap < 1e-8
    Er = O.rof_energy(u_dir, f, 1.0, 0.2, aniso=True)
    Ph, D, E = O.energy(P, X)
    assert D <= Er + 1e-12 and abs(Ph - Er) < 1e-7 * Er and abs(D - Er) < 1e-7 * Er
    assert np.abs(O.unlift(P, X.u).reshape(10, 9) - u_dir).max() < 1e-4
    # and the isotropic optimum differs (the two TVs are different energies)
    Eiso = O.rof_energy(O.rof_direct(f, 1.0, 0.2, 0.0, 1.0, 20000)[0], f, 1.0, 0.2)
    assert abs(Eiso - Er) > 1e-3 * Er


def test_anisotropic_p_satisfies_infinite_constraints():
    """Prop. 4 with phi = |.|_1: |q^T (1_i^a - 1_j^b)|_inf <= lambda |gamma_i^a - gamma_j^b|
    on sampled (i, j, a, b) for the box-projected p."""
    f = synth.voronoi_ramps(5, 6, 143)[0]
    P = O.Problem(O.TRUNC, 5, 6, 6, 0.0, 1.0, lam=0.3, alpha=25.0, nu=0.1, f=f, aniso=1)
    X = O.State(P)
    O.pdhg(P, X, 40)
    lab = O.labels(P.L, 0, 1)
    p = np.stack([X.px, X.py], axis=-1)
    assert np.abs(p).max() > 0
    # box-projected: the l2 norm of some p_i exceeds the ball radius
    assert (np.linalg.norm(p, axis=-1) > P.lam * np.diff(lab)[None, :] * (1 + 1e-9)).any()
    r = synth.Rng(144)
    for pix in range(P.N):
        for _ in range(40):
            j, i = sorted(r.integers(2, 0, P.k - 1))
            a, b = r.uniform(2)
            vec = p[pix, j:i].sum(0) + a * p[pix, i] - b * p[pix, j]
            rhs = abs((lab[i] + a * (lab[i + 1] - lab[i])) - (lab[j] + b * (lab[j + 1] - lab[j])))
            assert np.abs(vec).max() <= P.lam * rhs + 1e-12


# --------------------------------------------------------------------------
# Phase unwrapping (Sec. 5.5): quadratic pieces of the periodic data
# --------------------------------------------------------------------------
def _periodic_piece(f, per, alpha, l, r, t):
    c = f + per * np.floor((0.5 * (l + r) - f) / per + 0.5)
    return 0.5 * alpha * (t - c) ** 2


def test_periodic_pieces_conjugate_and_envelope():
    """Each interval sees the parabola of the periodic copy of f nearest to
    its midpoint: conjugate by brute force, envelope = the parabola itself."""
    w, _ = synth.wrapped_phase(2, 3, 151)
    per = 2 * np.pi
    P = O.Problem(O.PERIODIC, 2, 3, 8, 0.0, 4 * np.pi, lam=0.005, alpha=1.0, nu=per, f=w)
    lab = O.labels(8, 0.0, 4 * np.pi)
    r = synth.Rng(152)
    for pix in range(P.N):
        for i in range(P.k):
            grid = np.linspace(lab[i], lab[i + 1], 200001)
            vals = _periodic_piece(P.f[pix], per, 1.0, lab[i], lab[i + 1], grid)
            for y in r.uniform(5, -15, 15):
                val, _ = O.conj(P, pix, i, y)
                bf = np.max(grid * y - vals)
                assert bf - 1e-12 <= val <= bf + 1e-7 * (1 + abs(bf))
            for t in np.linspace(lab[i], lab[i + 1], 7):
                want = _periodic_piece(P.f[pix], per, 1.0, lab[i], lab[i + 1], t)
                assert abs(O.biconj(P, pix, i, t) - want) <= 1e-9 * (1 + want)
    # at an interior point rho is the interval's piece; the pieces match the
    # squared circular distance where the nearest copy does not change
    t = 0.5 * (lab[2] + lab[3])
    d = np.abs(((t - P.f[0]) + np.pi) % per - np.pi)
    assert O.rho(P, 0, t) == pytest.approx(0.5 * d * d)


def test_periodic_rho_is_the_squared_circular_distance():
    """rho of the phase-unwrapping term (Sec. 5.5) is alpha/2 times the
    squared circular distance to f: against the minimum over 21 copies
    f + 2 pi m, at random points, exactly at the labels, one rounding step
    to either side of them, and half a period from f (the two nearest copies
    tie there)."""
    per, alpha = 2 * np.pi, 1.7
    w, _ = synth.wrapped_phase(3, 4, 159)
    L = 8
    P = O.Problem(O.PERIODIC, 3, 4, L, 0.0, 4 * np.pi, lam=0.1, alpha=alpha, nu=per, f=w)
    lab = O.labels(L, 0.0, 4 * np.pi)
    r = synth.Rng(160)
    ms = np.arange(-10, 11)
    for pix in range(P.N):
        f = P.f[pix]
        pts = list(r.uniform(40, -1.0, 4 * np.pi + 1.0)) + list(lab)
        pts += [np.nextafter(x, -np.inf) for x in lab] + [np.nextafter(x, np.inf) for x in lab]
        pts += [f + 0.5 * per, f + 1.5 * per, f - 0.5 * per]
        for t in pts:
            want = 0.5 * alpha * np.min((t - f - per * ms) ** 2)
            assert abs(O.rho(P, pix, t) - want) <= 1e-12 * (1.0 + want), (pix, t)


def test_phase_unwrapping_recovers_the_ramp():
    """A wrapped 1-D phase ramp from 1 to 11 rad (wraps twice) is unwrapped by
    the relaxation with 8 labels on [0, 4 pi]: errors far below pi."""
    w, true = synth.wrapped_phase(1, 48, 5)
    P = O.Problem(O.PERIODIC, 1, 48, 8, 0.0, 4 * np.pi, lam=0.05, alpha=1.0, nu=2 * np.pi, f=w)
    X = O.State(P)
    O.pdhg(P, X, 4000)
    err = np.abs(O.unlift(P, X.u) - true.ravel())
    assert err.mean() < 0.15 and err.max() < 0.5, (err.mean(), err.max())
    # wrapping only would leave errors of about 2 pi
    assert np.abs(w.ravel() - true.ravel()).max() > 5.0


def test_periodic_lambda0_circular_distance():
    """lambda = 0 with labels on [1, 3] (less than one period): the optimum is
    the per-pixel alpha/2 * (circular distance of f to [1, 3])^2, the textbook
    distance over the copies f + 2 pi m, attained at the point of [1, 3]
    nearest to the nearest copy."""
    per, alpha = 2 * np.pi, 3.0
    w, _ = synth.wrapped_phase(4, 5, 157)
    P = O.Problem(O.PERIODIC, 4, 5, 5, 1.0, 3.0, lam=0.0, alpha=alpha, nu=per, f=w)
    X = O.State(P)
    copies = w.reshape(-1)[:, None] + per * np.array([-1.0, 0.0, 1.0])[None, :]
    near = np.clip(copies, 1.0, 3.0)
    dist = np.abs(copies - near)
    m = np.argmin(dist, axis=1)
    d = dist[np.arange(P.N), m]
    tc = near[np.arange(P.N), m]
    opt = 0.5 * alpha * float((d * d).sum())
    assert opt > 1.0          # most pixels lie outside [1, 3]
    gaps, errs = [], []
    for _ in range(8):
        O.pdhg(P, X, 2000)
        Ph, D, E = O.energy(P, X)
        assert D <= opt + 1e-9 and Ph >= opt - 1e-9
        gaps.append(Ph - D)
        errs.append(np.abs(O.unlift(P, X.u) - tc).max())
    assert gaps[-1] < 0.1 * gaps[0] and gaps[-1] < 2e-3 * max(opt, 1.0)
    assert errs[-1] < 1e-2, errs
    # the nonconvex energy of the unlifted image (rho itself, the squared
    # circular distance; no TV at lambda = 0) reaches the same optimum
    assert abs(E - opt) <= 2e-3 * max(opt, 1.0), (E, opt)
