"""The cluster-resident iteration of small problems (resident.cu): which
problems take it, agreement with the oracle and with the per-half-step
kernels, and calls that compose (the state goes through global memory
between them)."""
import numpy as np
import pytest

import oracle as O
from _cases import case, gpu_solver, oracle_run
from paper_1512_01383_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_TOL = 1e-4
E_TOL = 1e-5


def _require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def _compare_state(st, X, P, tol):
    for name in ("u", "s", "v", "z", "px", "py"):
        a, b = st[name].reshape(P.N, P.k), getattr(X, name)
        assert np.abs(a - b).max() <= tol * (1.0 + np.abs(b).max()), name
    assert np.abs(st["q"] - X.q).max() <= tol * (1.0 + np.abs(X.q).max())


@pytest.mark.parametrize("kind,H,W,L,want", [
    (0, 64, 64, 2, True),        # the ROF configuration: 16 tiles, one per CTA
    (1, 40, 40, 6, True),        # 32 tiles, two per CTA
    (1, 19, 17, 20, True),
    (2, 21, 19, 5, True),
    (1, 512, 512, 20, False),    # far beyond one cluster
])
def test_which_problems_are_resident(kind, H, W, L, want):
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(kind, H, W, L, 2700)
    with gpu_solver(c) as s:
        assert G.lift_set_resident(s.h, True) == want
        assert G.lift_set_resident(s.h, False) is False


def test_volumes_are_never_resident():
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    f = torch.from_numpy(synth.as_f32(synth.voronoi_ramps_3d(3, 8, 9, 2701)[0])).cuda()
    with G.Solver(1, 8, 9, 5, 0.0, 1.0, 0.25, 25.0, 0.1, f=f, depth=3) as s:
        assert G.lift_set_resident(s.h, True) is False


@pytest.mark.parametrize("kind,H,W,L,iters,extra", [
    (0, 64, 64, 2, 300, {}),
    (1, 40, 40, 6, 200, {}),
    (1, 40, 40, 6, 200, {"aniso": 1}),
    (1, 19, 17, 20, 120, {"theta": 361.0}),
    (2, 21, 19, 5, 150, {}),
    (3, 27, 23, 8, 150, {}),
])
def test_resident_matches_oracle_and_per_step_kernels(kind, H, W, L, iters, extra):
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(kind, H, W, L, 2800 + L, **extra)
    P, X = oracle_run(c, iters)
    with gpu_solver(c) as a, gpu_solver(c, resident=False) as b:
        assert G.lift_set_resident(a.h, True)
        a.iterate(iters)
        b.iterate(iters)
        ua, ub = a.unlift(), b.unlift()
        sa = a.state()
        ea, eb = a.energy(), b.energy()
    rng = c["gamma_max"] - c["gamma_min"]
    assert np.abs(ua.reshape(-1) - O.unlift(P, X.u)).max() / rng <= U_TOL
    assert np.abs(ua - ub).max() / rng <= U_TOL
    _compare_state(sa, X, P, 2e-3)
    for g, h, o in zip(ea, eb, O.energy(P, X)):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (g, o)
        assert abs(g - h) <= E_TOL * max(abs(h), 1.0), (g, h)


def test_resident_calls_compose():
    """37 + 63 iterations in two calls equal 100 in one (bitwise)."""
    _require_gpu()
    c = case(1, 40, 40, 6, 2900)
    with gpu_solver(c) as a, gpu_solver(c) as b:
        a.iterate(37)
        a.iterate(63)
        b.iterate(100)
        sa, sb = a.state(), b.state()
    for n in sa:
        np.testing.assert_array_equal(sa[n], sb[n])


def test_resident_solve_reaches_gap():
    """The ROF configuration (64 x 64, L = 2) solved to relative gap 1e-5 in
    the resident form, as in the per-half-step form."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    f = torch.from_numpy(synth.as_f32(synth.gaussian_blobs(64, 64, synth.BASE_SEED))).cuda()
    its = []
    for resident in (True, False):
        with G.Solver(0, 64, 64, 2, 0.0, 1.0, 0.2, 1.0, 0.0, f=f, check_every=100,
                      resident=resident) as s:
            rc, n = s.solve(100000, 1e-5)
            assert rc == G.LIFT_OK and s.gap() <= 1e-5
            its.append(n)
    assert abs(its[0] - its[1]) <= 200, its


def test_resident_handles_of_different_sizes_alternate():
    """Handles with different shared-memory needs, created in turn and then
    iterated alternately, all take the resident path and match their
    per-half-step twins."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    shapes = [(64, 64, 2), (19, 17, 20), (40, 40, 6), (13, 11, 3)]
    cases = [case(1 if L > 2 else 0, H, W, L, 3300 + j) for j, (H, W, L) in enumerate(shapes)]
    res = [gpu_solver(c) for c in cases]
    ref = [gpu_solver(c, resident=False) for c in cases]
    try:
        assert all(G.lift_set_resident(s.h, True) for s in res)
        for _ in range(3):
            for s, r in zip(res, ref):
                s.iterate(20)
                r.iterate(20)
        for s, r, c in zip(res, ref, cases):
            rng = c["gamma_max"] - c["gamma_min"]
            assert np.abs(s.unlift() - r.unlift()).max() / rng <= U_TOL
    finally:
        for s in res + ref:
            s.close()
