"""Volumes (the d = 3 Cartesian grid of Sec. 4) on the GPU against the FP64
oracle: iterates including the z component of p, energies, edge shapes, the
adaptive balance, the state image, and sampled voxels at the bench size."""
import numpy as np
import pytest

import oracle as O
from paper_1512_01383_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_TOL = 1e-4       # unlifted volume, normalised by the label range
E_TOL = 1e-5       # energies, relative


def _require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def vcase(kind, D, H, W, L, seed, **kw):
    """A volume problem with float32 inputs (what the GPU sees)."""
    if kind in (0, 1):
        f = synth.as_f32(synth.voronoi_ramps_3d(D, H, W, seed, cells=6)[0])
        c = dict(kind=kind, D=D, H=H, W=W, L=L, gmin=0.0, gmax=1.0, f=f,
                 lam=0.2 if kind == 0 else 0.25, alpha=1.0 if kind == 0 else 25.0,
                 nu=0.0 if kind == 0 else 0.1)
    elif kind == 3:
        f = synth.as_f32(np.stack([synth.wrapped_phase(H, W, seed + z)[0] for z in range(D)]))
        c = dict(kind=3, D=D, H=H, W=W, L=L, gmin=0.0, gmax=float(4 * np.pi), f=f, lam=0.05,
                 alpha=1.0, nu=float(2 * np.pi))
    else:
        cost = synth.as_f32(synth.Rng(seed).uniform(D * H * W * 9, 0.0, 1.0).reshape(D, H, W, 9))
        c = dict(kind=2, D=D, H=H, W=W, L=L, gmin=0.0, gmax=8.0, cost=cost, lam=0.05,
                 smin=0.0, smax=8.0)
    c.update(kw)
    return c


def oproblem(c):
    return O.Problem({0: O.QUAD, 1: O.TRUNC, 2: O.PL, 3: O.PERIODIC}[c["kind"]], c["H"], c["W"],
                     c["L"], c["gmin"], c["gmax"], lam=c["lam"], alpha=c.get("alpha", 1.0),
                     nu=c.get("nu", 0.0),
                     f=None if c.get("f") is None else c["f"].astype(np.float64),
                     cost=None if c.get("cost") is None else c["cost"].astype(np.float64),
                     smin=c.get("smin", 0.0), smax=c.get("smax", 1.0), theta=c.get("theta", 1.0),
                     aniso=c.get("aniso", 0), D=c["D"])


def gsolver(c, **kw):
    from paper_1512_01383_gb300 import lift as G
    f = torch.from_numpy(c["f"]).cuda() if c.get("f") is not None else None
    cost = torch.from_numpy(c["cost"]).cuda() if c.get("cost") is not None else None
    return G.Solver(c["kind"], c["H"], c["W"], c["L"], c["gmin"], c["gmax"], c["lam"],
                    c.get("alpha", 1.0), c.get("nu", 0.0), f=f, cost=cost,
                    sample_min=c.get("smin", 0.0), sample_max=c.get("smax", 1.0),
                    step_balance=c.get("theta", 1.0), anisotropic=bool(c.get("aniso", 0)),
                    depth=c["D"], **kw)


def _compare_state(st, X, P, tol):
    for name in ("u", "s", "v", "z", "px", "py", "pz"):
        a, b = st[name].reshape(P.N, P.k), getattr(X, name)
        err = np.abs(a - b).max()
        assert err <= tol * (1.0 + np.abs(b).max()), (name, err)
    assert np.abs(st["q"] - X.q).max() <= tol * (1.0 + np.abs(X.q).max())


def _check(c, iters, etol=E_TOL):
    P = oproblem(c)
    X = O.State(P)
    O.pdhg(P, X, iters)
    with gsolver(c) as s:
        s.iterate(iters)
        ut = s.unlift()
        st = s.state()
        Pg, Dg, Eg = s.energy()
    assert ut.shape == (c["D"], c["H"], c["W"])
    rng = c["gmax"] - c["gmin"]
    assert np.abs(ut.reshape(-1) - O.unlift(P, X.u)).max() / rng <= U_TOL
    _compare_state(st, X, P, 2e-3)
    assert np.abs(X.pz).max() > 0 or c["D"] == 1
    Po, Do, Eo = O.energy(P, X)
    for g, o in ((Pg, Po), (Dg, Do), (Eg, Eo)):
        assert abs(g - o) <= etol * max(abs(o), 1.0), (g, o)


@pytest.mark.parametrize("kind,D,H,W,L,iters,aniso", [
    # several 256-thread blocks, slices that do not align with tiles, ragged tail
    (1, 5, 9, 11, 5, 150, 0),
    (0, 4, 13, 7, 2, 200, 0),
    (2, 3, 8, 9, 5, 100, 0),
    (1, 6, 7, 5, 10, 100, 0),
    (1, 5, 6, 7, 5, 150, 1),
    (3, 3, 10, 9, 8, 100, 0),
])
def test_volume_iterations_match_oracle(kind, D, H, W, L, iters, aniso):
    _require_gpu()
    c = vcase(kind, D, H, W, L, 2000 + 7 * D + L, aniso=aniso)
    _check(c, iters, E_TOL)


@pytest.mark.parametrize("D,H,W,L", [(2, 1, 37, 5), (9, 1, 1, 4), (3, 5, 1, 6), (7, 2, 3, 3)])
def test_volume_edge_shapes(D, H, W, L):
    """Lines along each axis and slabs of one row or column."""
    _require_gpu()
    _check(vcase(1, D, H, W, L, 2100 + D * H * W), 120)


def test_volume_energy_kernel_on_oracle_state():
    """The energy kernels evaluate an oracle state (loaded through the state
    image, z component included) to the oracle's own energies."""
    _require_gpu()
    c = vcase(1, 4, 9, 10, 6, 2200)
    P = oproblem(c)
    X = O.State(P)
    O.pdhg(P, X, 80)
    with gsolver(c) as s:
        s.set_state({n: getattr(X, n) for n in ("u", "s", "ubar", "sbar", "v", "z", "px", "py",
                                                "q", "pz")})
        Pg, Dg, Eg = s.energy()
    for g, o in zip((Pg, Dg, Eg), O.energy(P, X)):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (g, o)


def test_volume_adaptive_balance_matches_oracle():
    """The movement behind the adaptive balance includes the z component."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = vcase(1, 4, 10, 9, 6, 2300)
    P = oproblem(c)
    X = O.State(P)
    th_o = O.pdhg_adaptive(P, X, 5, 100)
    with gsolver(c, check_every=100, adaptive_balance=True) as s:
        rc, n = s.solve(500, 1e-15)
        assert rc == G.LIFT_ERR_NOT_CONVERGED and n == 500
        th_g = G.lift_get_balance(s.h)
        ut = s.unlift()
    assert abs(th_g - th_o) <= 1e-3 * th_o, (th_g, th_o)
    assert np.abs(ut.reshape(-1) - O.unlift(P, X.u)).max() <= U_TOL


def test_volume_state_image_roundtrip_and_size():
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = vcase(1, 3, 6, 7, 5, 2400)
    N, k = 3 * 6 * 7, 4
    with gsolver(c) as a, gsolver(c) as b:
        assert G.lift_state_bytes(a.h) == N * k * (8 + 8 + 16 + 4) + N * 4
        a.iterate(37)
        b.set_state(a.state())
        a.iterate(20)
        b.iterate(20)
        sa, sb = a.state(), b.state()
        for n in sa:
            np.testing.assert_array_equal(sa[n], sb[n])
        b.reset()
        assert not np.any(b.state()["pz"])


def test_volume_rejected_where_images_only():
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = vcase(1, 3, 5, 6, 4, 2500)
    with gsolver(c) as s:
        with pytest.raises(G.LiftError) as e:
            G.lift_unrolled_forward(s.h, 10, 5)
        assert e.value.code == G.LIFT_ERR_SPEC


def test_full_size_volume_128():
    """The bench's 128^3, L = 8 truncated-quadratic volume: after n
    iterations a voxel depends only on inputs within 2n voxels per axis, so an
    oracle crop with that margin (clipped at the border) reproduces it."""
    _require_gpu()
    n, D = 2, 128
    f = synth.as_f32(synth.voronoi_ramps_3d(D, D, D, 1512013837)[0])
    c = dict(kind=1, D=D, H=D, W=D, L=8, gmin=0.0, gmax=1.0, f=f, lam=0.25, alpha=25.0, nu=0.1)
    with gsolver(c) as s:
        s.iterate(n)
        ut = s.unlift()
        st = s.state()
    m = 2 * n + 2
    rng = np.random.default_rng(5)
    pts = [(0, 0, 0), (D - 1, D - 1, D - 1), (0, D - 1, 0)] + [
        tuple(int(v) for v in rng.integers(0, D, 3)) for _ in range(4)]
    for (z, y, x) in pts:
        z0, z1 = max(0, z - m), min(D, z + m + 1)
        y0, y1 = max(0, y - m), min(D, y + m + 1)
        x0, x1 = max(0, x - m), min(D, x + m + 1)
        cc = dict(c, D=z1 - z0, H=y1 - y0, W=x1 - x0,
                  f=np.ascontiguousarray(f[z0:z1, y0:y1, x0:x1]))
        P = oproblem(cc)
        X = O.State(P)
        O.pdhg(P, X, n)
        j = ((z - z0) * (y1 - y0) + (y - y0)) * (x1 - x0) + (x - x0)
        assert abs(ut[z, y, x] - O.unlift(P, X.u)[j]) <= U_TOL
        g = (z * D + y) * D + x
        for name in ("u", "s", "v", "z", "px", "py", "pz"):
            a, b = st[name][g], getattr(X, name)[j]
            assert np.abs(a - b).max() <= 2e-3 * (1 + np.abs(b).max()), (name, a, b)
