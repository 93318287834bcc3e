"""The running average of the iterate (lift_average, lift_energy_average,
lift_unlift_average) against the oracle's average of the same iterates, and
its edge cases.  Every iterate is feasible and the feasible set is convex, so
the averaged point's energies are bounds of the relaxation too; on the
sampled costs of Sec. 5.4 they close where the last iterate's do not."""
import numpy as np
import pytest

import oracle as O
from _cases import case, gpu_solver, oracle_run

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_TOL = 1e-4       # unlifted image, normalised by (gamma_max - gamma_min)
E_TOL = 1e-5       # energies, relative


def _require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


@pytest.mark.parametrize("kind,H,W,L", [(1, 19, 23, 5), (2, 17, 21, 6), (0, 24, 31, 3)])
def test_average_matches_oracle(kind, H, W, L):
    """Iterations 1..20 unaveraged, then the average of iterates 21..60 on
    both sides: energies at the average within E_TOL, its unlifted image
    within U_TOL of the label range."""
    _require_gpu()
    c = case(kind, H, W, L, 2100 + 10 * kind + L)
    P, X = oracle_run(c, 20)
    A = O.pdhg_averaged(P, X, 40)
    with gpu_solver(c) as s:
        s.iterate(20)
        s.average_reset()
        for _ in range(40):
            s.iterate(1)
            s.average_add()
        assert s.average_count() == 40
        eg = s.energy_average()
        ug = s.unlift_average().reshape(-1).astype(np.float64)
    eo = O.energy(P, A)
    for g, o in zip(eg, eo):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (eg, eo)
    rng = c["gamma_max"] - c["gamma_min"]
    assert np.abs(ug - O.unlift(P, A.u)).max() / rng <= U_TOL


def test_average_edge_cases():
    """Empty average: LIFT_ERR_ARG.  One iterate: the average is that
    iterate (its energies equal lift_energy's bit for bit).  Adding to the
    average leaves the iterate unchanged.  average_reset and lift_reset
    empty it."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(1, 13, 11, 4, 2201)
    with gpu_solver(c) as s:
        with pytest.raises(G.LiftError) as e:
            s.energy_average()
        assert e.value.code == G.LIFT_ERR_ARG
        s.iterate(7)
        before = s.state()
        s.average_add()
        after = s.state()
        for n in before:
            assert np.array_equal(before[n], after[n]), n
        assert s.energy_average() == s.energy()
        assert np.array_equal(s.unlift_average(), s.unlift())
        s.average_reset()
        assert s.average_count() == 0
        with pytest.raises(G.LiftError):
            s.unlift_average()
        # a fresh start empties the average
        s.average_add()
        assert s.average_count() == 1
        s.reset()
        assert s.average_count() == 0


def test_average_of_a_volume():
    """On a volume the third dual component is averaged too: after one
    iterate the averaged energies equal lift_energy's, and after a restart
    the iterate's energies equal those of the average it was given."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G, synth
    f = torch.from_numpy(synth.as_f32(synth.voronoi_ramps_3d(4, 9, 10, 2301)[0])).cuda()
    with G.Solver(G.LIFT_TRUNC_QUAD, 9, 10, 5, 0.0, 1.0, 0.25, 25.0, 0.1, f=f, depth=4) as s:
        s.iterate(12)
        s.average_add()
        assert s.energy_average() == s.energy()
        s.iterate(1)
        s.average_add()
        Pa, Da, Ea = s.energy_average()
        assert np.isfinite([Pa, Da, Ea]).all()
        # a restart makes the averaged point (pz included) the iterate
        s.average_restart()
        assert s.energy() == (Pa, Da, Ea)
        s.iterate(5)
        assert np.isfinite(s.energy()).all()


@pytest.mark.parametrize("kind,H,W,L", [(2, 17, 21, 6), (1, 19, 23, 5)])
def test_restart_from_average_matches_oracle(kind, H, W, L):
    """Ten iterations, two epochs of fifteen iterations each averaged and
    followed by a restart from the average, then ten plain iterations, on
    both sides (the oracle restarts by taking its averaged state as the
    iterate): energies within E_TOL, the unlifted image within U_TOL."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(kind, H, W, L, 2400 + 10 * kind + L)
    P, X = oracle_run(c, 10)
    for _ in range(2):
        X = O.pdhg_averaged(P, X, 15)
    O.pdhg(P, X, 10)
    with gpu_solver(c) as s:
        with pytest.raises(G.LiftError) as e:
            s.average_restart()                  # empty average
        assert e.value.code == G.LIFT_ERR_ARG
        s.iterate(10)
        for _ in range(2):
            s.average_reset()
            for _ in range(15):
                s.iterate(1)
                s.average_add()
            s.average_restart()
            assert s.average_count() == 0
        s.iterate(10)
        eg = s.energy()
        ug = s.unlift().reshape(-1).astype(np.float64)
    eo = O.energy(P, X)
    for g, o in zip(eg, eo):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (eg, eo)
    rng = c["gamma_max"] - c["gamma_min"]
    assert np.abs(ug - O.unlift(P, X.u)).max() / rng <= U_TOL


def test_solve_averaged_certifies_in_fp64():
    """An 8 x 8 crop of the stereo cost volume (65 disparities, L = 8,
    balance 0.1), where the last iterate's gap stalls near 0.08:
    lift_solve_averaged reaches gap 5e-3, the gap it returns is the iterate's
    own (lift_gap agrees bit for bit), and the oracle's FP64 energies of the
    final state certify it; lift_solve on the last iterate needs more
    iterations or does not get there."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G, synth
    cost, _ = synth.stereo_cost(480, 640, synth.BASE_SEED + 3, ndisp=65)
    c32 = np.ascontiguousarray(synth.as_f32(cost)[:8, :8])
    cd = torch.from_numpy(c32).cuda()
    tol, cap = 5e-3, 200000
    kw = dict(cost=cd, sample_min=0.0, sample_max=64.0, step_balance=0.1)
    with G.Solver(G.LIFT_PL_SAMPLED, 8, 8, 8, 0.0, 64.0, 0.05, **kw) as s:
        rc, n, g = s.solve_averaged(cap, tol, first_epoch=1000, every=10)
        assert rc == G.LIFT_OK, (rc, n, g)
        assert g <= tol and s.gap() == g
        st = s.state()
    with G.Solver(G.LIFT_PL_SAMPLED, 8, 8, 8, 0.0, 64.0, 0.05, **kw) as s:
        rc_plain, n_plain = s.solve(cap, tol)
    assert rc_plain != G.LIFT_OK or n_plain > n, (n, n_plain)
    P = O.Problem(O.PL, 8, 8, 8, 0.0, 64.0, lam=0.05, cost=c32.astype(np.float64),
                  smin=0.0, smax=64.0, theta=0.1)
    X = O.State(P)
    for name in ("u", "s", "v", "z", "px", "py"):
        getattr(X, name)[...] = st[name].reshape(P.N, P.k)
    X.q[...] = st["q"].reshape(P.N)
    Ph, D, _ = O.energy(P, X)
    assert (Ph - D) / max(abs(Ph), abs(D), 1.0) <= tol + 1e-4, (Ph, D)
