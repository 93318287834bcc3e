"""Oracle pins for volumes (the d = 3 Cartesian grid of Sec. 4: Omega in R^d,
p_i in R^{k x d}, three forward differences).  CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_1512_01383_gb300 import synth


def test_grad3_div3_adjoint_neumann_and_axes():
    r = synth.Rng(301)
    for D, H, W, k in ((1, 4, 5, 2), (3, 1, 1, 1), (2, 3, 4, 3), (4, 5, 3, 2)):
        n = D * H * W * k
        u = r.uniform(n, -1, 1)
        px, py, pz = (r.uniform(n, -1, 1) for _ in range(3))
        gx, gy, gz = O.grad3(D, H, W, k, u)
        d = O.div3(D, H, W, k, px, py, pz)
        assert abs((gx * px + gy * py + gz * pz).sum() + (u * d).sum()) < 1e-12
        U = u.reshape(D, H, W, k)
        GZ = gz.reshape(D, H, W, k)
        # Neumann: no difference across the last slice; forward differences
        # between slices along the slowest axis
        assert np.all(GZ[-1] == 0)
        np.testing.assert_allclose(GZ[:-1], U[1:] - U[:-1])
        np.testing.assert_allclose(gy.reshape(D, H, W, k)[:, :-1], U[:, 1:] - U[:, :-1])
        np.testing.assert_allclose(gx.reshape(D, H, W, k)[:, :, :-1], U[:, :, 1:] - U[:, :, :-1])
        # each slice's x/y differences are the image operator's
        for z in range(D):
            ix, iy = O.grad(H, W, k, U[z].reshape(-1))
            np.testing.assert_array_equal(gx.reshape(D, H, W, k)[z].reshape(-1), ix)
            np.testing.assert_array_equal(gy.reshape(D, H, W, k)[z].reshape(-1), iy)


def test_volume_steps_from_dense_operator():
    """tau_u is the reciprocal of the largest column sum of |[I; grad]| on a
    3x3x3 volume (interior voxel: 1 + 6); every gradient row sums to 2."""
    D = H = W = 3
    N = D * H * W
    G = []
    for ax in range(3):
        for v in range(N):
            z, rem = divmod(v, H * W)
            y, x = divmod(rem, W)
            c = [z, y, x]
            lim = [D, H, W][ax]
            row = np.zeros(N)
            if c[ax] + 1 < lim:
                c2 = list(c)
                c2[ax] += 1
                row[(c2[0] * H + c2[1]) * W + c2[2]] = 1.0
                row[v] = -1.0
            G.append(row)
    K = np.vstack([np.eye(N), np.array(G)])
    col = np.abs(K).sum(0).max()
    P = O.Problem(O.QUAD, H, W, 2, f=np.zeros(N), D=D)
    st = O.steps(P)
    assert col == 7.0 and st["tau_u"] == pytest.approx(1.0 / col)
    assert np.abs(np.array(G)).sum(1).max() == 2.0 and st["sigma_p"] == 0.5
    # an image keeps 1 + 4
    assert O.steps(O.Problem(O.QUAD, H, W, 2, f=np.zeros(H * W)))["tau_u"] == pytest.approx(0.2)


@pytest.mark.parametrize("aniso", [0, 1])
def test_volume_L2_equals_direct_rof(aniso):
    """Prop. 3 on a volume: L = 2 is box-constrained ROF with the 3-D TV
    (|grad u|_2, or |grad u|_1), solved by the independent unlifted solver."""
    f = synth.voronoi_ramps_3d(4, 6, 5, 303, cells=5)[0]
    P = O.Problem(O.QUAD, 6, 5, 2, 0.0, 1.0, lam=0.15, alpha=1.0, f=f, aniso=aniso, D=4)
    X = O.State(P)
    O.pdhg(P, X, 6000)
    u_dir, gap = O.rof_direct3(f, 1.0, 0.15, 0.0, 1.0, 100000, aniso=bool(aniso))
    assert gap < 1e-8
    Er = O.rof_energy3(u_dir, f, 1.0, 0.15, aniso=bool(aniso))
    Ph, Dl, E = O.energy(P, X)
    assert Dl <= Er + 1e-10 and abs(Ph - Er) < 1e-6 * Er and abs(Dl - Er) < 1e-6 * Er
    assert np.abs(O.unlift(P, X.u) - u_dir.reshape(-1)).max() < 2e-4
    # the z coupling matters: the slices solved as separate images differ
    Es = sum(O.rof_energy(O.rof_direct(f[z], 1.0, 0.15, 0.0, 1.0, 30000, aniso=bool(aniso))[0],
                          f[z], 1.0, 0.15, aniso=bool(aniso)) for z in range(4))
    assert Es < Er - 1e-3 * Er


@pytest.mark.parametrize("kind", [O.TRUNC, O.PL])
def test_identical_slices_reduce_to_the_image(kind):
    """A volume of D identical slices has no z differences at the optimum:
    the converged relaxation per slice is the image's (energies D times the
    image's), whichever kind of data term."""
    H, W, L, D = 6, 7, 5, 3
    if kind == O.TRUNC:
        img = synth.voronoi_ramps(H, W, 305)[0]
        kw = dict(alpha=25.0, nu=0.1, lam=0.25)
        P2 = O.Problem(kind, H, W, L, 0.0, 1.0, f=img, **kw)
        P3 = O.Problem(kind, H, W, L, 0.0, 1.0, f=np.stack([img] * D), D=D, **kw)
    else:
        cost = synth.Rng(305).uniform(H * W * 9, 0.0, 1.0).reshape(H, W, 9)
        kw = dict(lam=0.05, smin=0.0, smax=8.0)
        P2 = O.Problem(kind, H, W, L, 0.0, 8.0, cost=cost, **kw)
        P3 = O.Problem(kind, H, W, L, 0.0, 8.0, cost=np.stack([cost] * D), D=D, **kw)
    X2, X3 = O.State(P2), O.State(P3)
    O.pdhg(P2, X2, 8000)
    O.pdhg(P3, X3, 8000)
    a2, b2, _ = O.energy(P2, X2)
    a3, b3, _ = O.energy(P3, X3)
    # both bracket their optimum; the volume's optimum is D times the image's
    assert b3 <= D * a2 + 1e-9 and D * b2 <= a3 + 1e-9
    assert a2 > 1.0 and (a2 - b2) / a2 < 1e-3 and (a3 - b3) / a3 < 1e-3
    u3 = O.unlift(P3, X3.u).reshape(D, H, W)
    u2 = O.unlift(P2, X2.u).reshape(H, W)
    rng = P2.gmax - P2.gmin
    assert np.abs(u3 - u2[None]).max() / rng < 2e-2
    assert np.abs(u3[1:] - u3[:-1]).max() / rng < 1e-3


def test_volume_p_satisfies_infinite_constraints():
    """Prop. 4 with p_i in R^3: sampled constraints hold for the projected p."""
    f = synth.voronoi_ramps_3d(3, 4, 5, 307)[0]
    P = O.Problem(O.TRUNC, 4, 5, 6, 0.0, 1.0, lam=0.3, alpha=25.0, nu=0.1, f=f, D=3)
    X = O.State(P)
    O.pdhg(P, X, 40)
    lab = O.labels(P.L, 0, 1)
    p = np.stack([X.px, X.py, X.pz], axis=-1)
    assert np.abs(X.pz).max() > 0
    r = synth.Rng(308)
    for pix in range(P.N):
        for _ in range(30):
            j, i = sorted(r.integers(2, 0, P.k - 1))
            a, b = r.uniform(2)
            vec = p[pix, j:i].sum(0) + a * p[pix, i] - b * p[pix, j]
            rhs = abs((lab[i] + a * (lab[i + 1] - lab[i])) - (lab[j] + b * (lab[j + 1] - lab[j])))
            assert np.linalg.norm(vec) <= P.lam * rhs + 1e-12


def test_volume_gap_nonnegative_and_decreasing():
    f = synth.voronoi_ramps_3d(4, 5, 6, 309)[0]
    P = O.Problem(O.TRUNC, 5, 6, 5, 0.0, 1.0, lam=0.25, alpha=25.0, nu=0.1, f=f, theta=16.0, D=4)
    X = O.State(P)
    gaps = []
    for _ in range(6):
        O.pdhg(P, X, 300)
        a, b, _ = O.energy(P, X)
        assert a >= b - 1e-10
        gaps.append(a - b)
    assert gaps[-1] < 0.2 * gaps[0]
