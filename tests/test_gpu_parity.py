"""GPU (CUDA, FP32) against the FP64 oracle on identical seeded inputs.

Tolerances: the unlifted image within 1e-4 max-abs after normalising by the
label range, energies within 1e-5 relative, after a fixed iteration count;
single projections and envelopes within a few FP32 ulps of the point's scale.
"""
import os

import numpy as np
import pytest

import oracle as O
from _cases import case, crop, gpu_solver, oracle_problem, oracle_run
from paper_1512_01383_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_TOL = 1e-4       # unlifted image, normalised by (gamma_max - gamma_min)
E_TOL = 1e-5       # energies, relative


def _require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


# ---------------------------------------------------------------------------
# Single projections and envelopes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind,L", [(0, 4), (1, 5), (1, 3), (2, 6)])
def test_projection_matches_oracle(kind, L):
    _require_gpu()
    c = case(kind, 6, 7, L, 101 + kind)
    P = oracle_problem(c)
    rng = np.random.default_rng(5)
    n = 3000
    pix = rng.integers(0, P.N, n).astype(np.int32)
    itv = rng.integers(0, P.k, n).astype(np.int32)
    scale = (c.get("alpha", 1.0) + 1.0) * (c["gamma_max"] - c["gamma_min"])
    y0 = rng.uniform(-3 * scale, 3 * scale, n).astype(np.float32)
    h0 = np.empty(n, np.float32)
    for j in range(n):
        phi = O.conj(P, int(pix[j]), int(itv[j]), float(y0[j]))[0]
        h0[j] = phi + rng.uniform(-4 * scale, 0.5 * scale)
    with gpu_solver(c) as s:
        t = lambda a: torch.from_numpy(a).cuda()
        yo, ho = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
        from paper_1512_01383_gb300 import lift as G
        G.lift_proj_epi(s.h, t(pix), t(itv), t(y0), t(h0), yo, ho)
        torch.cuda.synchronize()
        yo, ho = yo.cpu().numpy(), ho.cpu().numpy()
    for j in range(n):
        ry, rh = O.proj_epi(P, int(pix[j]), int(itv[j]), float(y0[j]), float(h0[j]))
        mag = 1.0 + abs(y0[j]) + abs(h0[j])
        assert abs(yo[j] - ry) <= 2e-5 * mag, (j, yo[j], ry)
        assert abs(ho[j] - rh) <= 2e-5 * mag, (j, ho[j], rh)


@pytest.mark.parametrize("kind,L", [(0, 4), (1, 5), (1, 2), (2, 6)])
def test_envelope_matches_oracle(kind, L):
    _require_gpu()
    c = case(kind, 5, 4, L, 201 + kind)
    P = oracle_problem(c)
    lab = O.labels(c["L"], c["gamma_min"], c["gamma_max"])
    rng = np.random.default_rng(7)
    n = 2000
    pix = rng.integers(0, P.N, n).astype(np.int32)
    itv = rng.integers(0, P.k, n).astype(np.int32)
    tt = (lab[itv] + rng.uniform(0, 1, n) * (lab[itv + 1] - lab[itv])).astype(np.float32)
    with gpu_solver(c) as s:
        from paper_1512_01383_gb300 import lift as G
        t = lambda a: torch.from_numpy(a).cuda()
        out = torch.empty(n, device="cuda")
        G.lift_envelope(s.h, t(pix), t(itv), t(tt), out)
        got = out.cpu().numpy()
    want = np.array([O.biconj(P, int(pix[j]), int(itv[j]), float(tt[j])) for j in range(n)])
    scale = 1.0 + np.abs(want)
    assert np.all(np.abs(got - want) <= 2e-5 * scale * (1 + c.get("alpha", 1.0)))


# ---------------------------------------------------------------------------
# Whole iterations
# ---------------------------------------------------------------------------
def _compare_state(st, X, P, tol):
    for name in ("u", "s", "v", "z", "px", "py"):
        a, b = st[name].reshape(P.N, P.k), getattr(X, name)
        err = np.abs(a - b).max()
        assert err <= tol * (1.0 + np.abs(b).max()), (name, err)
    assert np.abs(st["q"] - X.q).max() <= tol * (1.0 + np.abs(X.q).max())


PARITY_CASES = [
    # kind, H, W, L, iters: several 256-thread blocks plus a ragged tail
    (0, 37, 29, 2, 300),
    (1, 37, 29, 5, 300),
    (1, 23, 31, 10, 200),
    (1, 19, 17, 20, 120),
    (2, 21, 19, 5, 150),
    (2, 13, 11, 17, 80),
]
BALANCED_CASES = [
    # the same with the primal/dual balance of the time-to-gap runs
    (1, 37, 29, 5, 300, 16.0),
    (1, 19, 17, 20, 120, 361.0),
    (0, 25, 23, 2, 200, 0.3),
]


@pytest.mark.parametrize("kind,H,W,L,iters,theta", BALANCED_CASES)
def test_balanced_steps_match_oracle(kind, H, W, L, iters, theta):
    _require_gpu()
    c = case(kind, H, W, L, 350 + H + L, theta=theta)
    P, X = oracle_run(c, iters)
    with gpu_solver(c) as s:
        s.iterate(iters)
        ut = s.unlift()
        Pg, Dg, Eg = s.energy()
    ur = O.unlift(P, X.u).reshape(H, W)
    assert np.abs(ut - ur).max() <= U_TOL
    Po, Do, Eo = O.energy(P, X)
    for g, o in ((Pg, Po), (Dg, Do), (Eg, Eo)):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (g, o)


@pytest.mark.parametrize("resident", [True, False])
@pytest.mark.parametrize("kind,H,W,L,iters", PARITY_CASES)
def test_iterations_match_oracle(kind, H, W, L, iters, resident):
    """Both ways lift_iterate runs small problems: inside one thread-block
    cluster (the default where the problem fits) and as per-half-step
    kernels."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(kind, H, W, L, 300 + H + L)
    P, X = oracle_run(c, iters)
    with gpu_solver(c, resident=resident) as s:
        assert G.lift_set_resident(s.h, resident) == resident
        s.iterate(iters)
        ut = s.unlift()
        st = s.state()
        Pg, Dg, Eg = s.energy()
    rng = c["gamma_max"] - c["gamma_min"]
    ur = O.unlift(P, X.u).reshape(H, W)
    assert np.abs(ut - ur).max() / rng <= U_TOL
    _compare_state(st, X, P, 2e-3)
    Po, Do, Eo = O.energy(P, X)
    for g, o in ((Pg, Po), (Dg, Do), (Eg, Eo)):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (g, o)


@pytest.mark.parametrize("kind,L", [(0, 2), (1, 5), (2, 5), (3, 8)])
def test_energy_kernel_on_oracle_state(kind, L):
    """The energy reduction alone: load the oracle's iterate (rounded to
    float32) into the GPU and evaluate both sides on the same state."""
    _require_gpu()
    c = case(kind, 33, 27, L, 400 + kind)
    P, X = oracle_run(c, 60)
    names = ("u", "s", "ubar", "sbar", "v", "z", "px", "py")
    for n in names:
        getattr(X, n)[...] = getattr(X, n).astype(np.float32).astype(np.float64)
    X.q[...] = X.q.astype(np.float32).astype(np.float64)
    with gpu_solver(c) as s:
        s.set_state({n: getattr(X, n) for n in names} | {"q": X.q})
        Pg, Dg, Eg = s.energy()
        ug = s.unlift()
    Po, Do, Eo = O.energy(P, X)
    for g, o in ((Pg, Po), (Dg, Do), (Eg, Eo)):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (g, o)
    np.testing.assert_allclose(ug.reshape(-1), O.unlift(P, X.u), atol=1e-6 * (c["gamma_max"] + 1))


EDGE_CASES = [
    (1, 1, 1, 5, 50),     # a single pixel
    (1, 1, 33, 4, 80),    # one row (1-D)
    (1, 29, 1, 4, 80),    # one column
    (0, 3, 5, 2, 100),
    (1, 9, 7, 65, 30),    # k = 64, the largest supported
    (1, 11, 13, 33, 40),  # k = 32 (a pixel straddles no warp boundary)
]


@pytest.mark.parametrize("kind,H,W,L,iters", EDGE_CASES)
def test_edge_shapes(kind, H, W, L, iters):
    _require_gpu()
    c = case(kind, H, W, L, 500 + H * W + L)
    P, X = oracle_run(c, iters)
    with gpu_solver(c) as s:
        s.iterate(iters)
        ut = s.unlift()
        Pg, Dg, Eg = s.energy()
    ur = O.unlift(P, X.u).reshape(H, W)
    assert np.abs(ut - ur).max() <= U_TOL
    Po, Do, Eo = O.energy(P, X)
    for g, o in ((Pg, Po), (Dg, Do), (Eg, Eo)):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (g, o)


def test_lambda_zero_and_zero_iterations():
    _require_gpu()
    c = case(1, 12, 10, 5, 601, lam=0.0)
    P, X = oracle_run(c, 100)
    with gpu_solver(c) as s:
        z = s.unlift()
        assert np.all(z == 0.0)           # all-zero start: u~ = gamma_1
        s.iterate(0)
        s.iterate(100)
        ut = s.unlift()
    assert np.abs(ut.reshape(-1) - O.unlift(P, X.u)).max() <= U_TOL


# ---------------------------------------------------------------------------
# Full-size workloads: sampled pixels against oracle crops.  After n
# iterations a pixel depends only on inputs within 2n pixels (each half-step
# reads one neighbour per axis), so a crop with a margin of 2n+2 around it
# (clipped at the true image border) reproduces it exactly.
# ---------------------------------------------------------------------------
def _sampled_parity(c, iters, samples, seed):
    """The full-size problem on the GPU, as the bench runs it (the iteration
    graph, banded where the size asks for it), against the oracle on crops
    around sampled pixels: the three corners, `samples` random pixels, the
    first and last pixel of every band of the graph, and pixels on both sides
    of a dual-step strip boundary.  One iteration spreads a pixel's influence
    one pixel along each axis (the dual step reads x+1, y+1, the primal step
    x-1, y-1), so a crop margin of 2 iters + 2 pixels leaves the sampled
    pixel's iterate exactly that of the full image.  The crops run in
    parallel processes (started with spawn)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    from _cases import crop_oracle_pixel
    from paper_1512_01383_gb300 import lift as G
    H, W, L = c["H"], c["W"], c["L"]
    k = L - 1
    with gpu_solver(c, check_every=iters // 2) as s:
        bands = G.lift_set_bands(s.h, 0)
        s.iterate(iters)
        ut = s.unlift()
        st = s.state()
    # band boundaries of the graph (tiles of 256 // k pixels, cut at even tiles)
    ppb = 256 // k
    T = (H * W + ppb - 1) // ppb
    cuts = [(T * j // bands) // 2 * 2 * ppb for j in range(1, bands)]
    rng = np.random.default_rng(seed)
    flat = [0, H * W - 1, W - 1, 64 * 37 - 1, 64 * 37]
    for b in cuts:
        flat += [b - 1, b]
    flat += [int(v) for v in rng.integers(0, H * W, samples)]
    pts = sorted({(p // W, p % W) for p in flat})
    m = 2 * iters + 2
    jobs = []
    for (py_, px_) in pts:
        box = (max(0, py_ - m), min(H, py_ + m + 1), max(0, px_ - m), min(W, px_ + m + 1))
        jobs.append((c, box, iters, (py_, px_)))
    with ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1),
                             mp_context=mp.get_context("spawn")) as ex:
        results = list(ex.map(crop_oracle_pixel, jobs))
    rngl = c["gamma_max"] - c["gamma_min"]
    for (py_, px_), (ur, rows) in zip(pts, results):
        assert abs(ut[py_, px_] - ur) / rngl <= U_TOL, (py_, px_, ut[py_, px_], ur)
        g = py_ * W + px_
        for name, b in rows.items():
            a = st[name][g]
            assert np.abs(a - b).max() <= 2e-3 * (1 + np.abs(b).max()), (name, a, b)
    return len(pts)


@pytest.mark.parametrize("L", [5, 10, 20])
def test_full_size_truncated_512(L):
    """512 x 512 truncated quadratic (the bench's workload at L = 20), 50
    iterations, in the banded graph."""
    _require_gpu()
    c = case(1, 512, 512, L, 1512013832)
    assert _sampled_parity(c, 50, 8, L) >= 11


@pytest.mark.parametrize("L", [8, 32])
def test_full_size_stereo_640x480(L):
    """640 x 480 stereo costs (PL pieces), 50 iterations."""
    _require_gpu()
    c = case(2, 480, 640, L, 1512013834, ndisp=65)
    assert _sampled_parity(c, 50, 8, L) >= 11


# ---------------------------------------------------------------------------
# API behaviour on the GPU
# ---------------------------------------------------------------------------
def test_host_inputs_and_state_roundtrip():
    _require_gpu()
    c = case(1, 20, 18, 5, 701)
    with gpu_solver(c, device_inputs=False) as a, gpu_solver(c) as b:
        a.iterate(40)
        b.iterate(40)
        np.testing.assert_array_equal(a.unlift(), b.unlift())
        st = a.state()
        b.reset()
        b.set_state(st)
        a.iterate(10)
        b.iterate(10)
        np.testing.assert_array_equal(a.unlift(), b.unlift())
        # device output buffer
        out = torch.empty((20, 18), device="cuda")
        a.unlift(out)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(out.cpu().numpy(), a.unlift())


def test_solve_reaches_gap_and_reports_iterations():
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(0, 24, 24, 2, 801)
    with gpu_solver(c, check_every=50) as s:
        rc, n = s.solve(20000, 1e-5)
        assert rc == G.LIFT_OK and 0 < n < 20000 and n % 50 == 0
        assert s.gap() <= 1e-5
    with gpu_solver(c, check_every=10) as s:
        rc, n = s.solve(20, 1e-12)
        assert rc == G.LIFT_ERR_NOT_CONVERGED and n == 20


def test_nan_input_reports_nan():
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(1, 8, 8, 5, 901)
    c["f"] = c["f"].copy()
    c["f"][3, 3] = np.nan
    with gpu_solver(c) as s:
        s.iterate(5)
        with pytest.raises(G.LiftError) as e:
            s.energy()
        assert e.value.code == G.LIFT_ERR_NAN


def test_graph_replay_equals_direct_launches():
    """lift_iterate replays whole check intervals from a CUDA graph; the
    iterate must equal that of the same half-steps launched one by one."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(1, 23, 19, 6, 951)
    with gpu_solver(c, check_every=40, resident=False) as a, \
            gpu_solver(c, check_every=40, resident=False) as b:
        a.iterate(130)                     # 3 graph replays + 10 direct iterations
        for _ in range(130):
            G.lift_dual_step(b.h)
            G.lift_primal_step(b.h)
        sa, sb = a.state(), b.state()
        for k in sa:
            np.testing.assert_array_equal(sa[k], sb[k])
        # parameters are baked into the graph: a change must be picked up
        G.lift_set_params(a.h, 0.4, 25.0, 0.1)
        G.lift_set_params(b.h, 0.4, 25.0, 0.1)
        a.iterate(40)
        for _ in range(40):
            G.lift_dual_step(b.h)
            G.lift_primal_step(b.h)
        np.testing.assert_array_equal(a.unlift(), b.unlift())


@pytest.mark.parametrize("resident", [True, False])
@pytest.mark.parametrize("L", [5, 10])
def test_adaptive_balance_matches_oracle(L, resident):
    """lift_solve with adaptive_balance re-balances theta at every check from
    the movement since the previous check; the same rule on the oracle gives
    the same theta sequence and iterate."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(1, 21, 18, L, 990 + L)
    P = oracle_problem(c)
    X = O.State(P)
    th_o = O.pdhg_adaptive(P, X, 5, 100)
    with gpu_solver(c, check_every=100, adaptive_balance=True, resident=resident) as s:
        rc, n = s.solve(500, 1e-15)
        assert rc == G.LIFT_ERR_NOT_CONVERGED and n == 500
        th_g = G.lift_get_balance(s.h)
        ut = s.unlift()
    assert abs(th_g - th_o) <= 1e-3 * th_o, (th_g, th_o)
    assert np.abs(ut.reshape(-1) - O.unlift(P, X.u)).max() <= U_TOL


@pytest.mark.parametrize("kind,H,W,L,iters", [(1, 29, 23, 5, 250), (0, 25, 21, 2, 250), (2, 17, 15, 6, 100)])
def test_anisotropic_tv_matches_oracle(kind, H, W, L, iters):
    """phi = |.|_1: box projection of p_i and l1 norms in the energies."""
    _require_gpu()
    c = case(kind, H, W, L, 1700 + L, aniso=1)
    P, X = oracle_run(c, iters)
    with gpu_solver(c) as s:
        s.iterate(iters)
        ut = s.unlift()
        st = s.state()
        Pg, Dg, Eg = s.energy()
    rng = c["gamma_max"] - c["gamma_min"]
    assert np.abs(ut.reshape(-1) - O.unlift(P, X.u)).max() / rng <= U_TOL
    _compare_state(st, X, P, 2e-3)
    Po, Do, Eo = O.energy(P, X)
    for g, o in ((Pg, Po), (Dg, Do), (Eg, Eo)):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (g, o)


@pytest.mark.parametrize("H,W,L,iters", [(27, 23, 8, 300), (13, 40, 5, 200)])
def test_phase_unwrapping_matches_oracle(H, W, L, iters):
    """Periodic quadratic pieces (Sec. 5.5) on wrapped synthetic phase."""
    _require_gpu()
    c = case(3, H, W, L, 1800 + L)
    P, X = oracle_run(c, iters)
    with gpu_solver(c) as s:
        s.iterate(iters)
        ut = s.unlift()
        st = s.state()
        Pg, Dg, Eg = s.energy()
    rng = c["gamma_max"] - c["gamma_min"]
    assert np.abs(ut.reshape(-1) - O.unlift(P, X.u)).max() / rng <= U_TOL
    _compare_state(st, X, P, 2e-3)
    Po, Do, Eo = O.energy(P, X)
    for g, o in ((Pg, Po), (Dg, Do), (Eg, Eo)):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (g, o)


@pytest.mark.parametrize("L,iters", [(5, 200), (12, 150)])
def test_baseline_lifting_matches_oracle(L, iters):
    """The baseline lifting (Prop. 2): the PL kind with the cost sampled only
    at the labels, so every interval holds no interior sample and rho_i** is
    the chord.  Samples of the truncated quadratic of the denoising workload."""
    _require_gpu()
    H, W = 19, 26
    f = synth.voronoi_ramps(H, W, 1900 + L)[0]
    lab = O.labels(L, 0.0, 1.0)
    cost = synth.as_f32(np.minimum(25.0 * (lab[None, None, :] - f[:, :, None]) ** 2, 0.1))
    c = dict(kind=2, H=H, W=W, L=L, gamma_min=0.0, gamma_max=1.0, lam=0.25, cost=cost,
             sample_min=0.0, sample_max=1.0)
    P, X = oracle_run(c, iters)
    with gpu_solver(c) as s:
        s.iterate(iters)
        ut = s.unlift()
        st = s.state()
        Pg, Dg, Eg = s.energy()
    assert np.abs(ut.reshape(-1) - O.unlift(P, X.u)).max() <= U_TOL
    _compare_state(st, X, P, 2e-3)
    Po, Do, Eo = O.energy(P, X)
    for g, o in ((Pg, Po), (Dg, Do), (Eg, Eo)):
        assert abs(g - o) <= E_TOL * max(abs(o), 1.0), (g, o)


@pytest.mark.parametrize("resident", [True, False])
def test_two_pixel_rof_golden(resident):
    """The hand-derived two-pixel closed forms of tests/golden/rof_two_pixel.txt
    (L = 2, Prop. 3) on the GPU: after 20 000 iterations the unlifted pair
    and the energies meet them within FP32 rounding."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    from test_golden import golden
    for f1, f2, lam, u1, u2, E in golden("rof_two_pixel.txt"):
        f = torch.tensor([[f1, f2]], dtype=torch.float32, device="cuda")
        with G.Solver(G.LIFT_QUAD, 1, 2, 2, 0.0, 1.0, lam, 1.0, 0.0, f=f,
                      resident=resident) as s:
            s.iterate(20000)
            ut = s.unlift().reshape(-1)
            Pg, Dg, Eg = s.energy()
        assert np.abs(ut - [u1, u2]).max() <= 2e-6, (ut, u1, u2)
        for v in (Pg, Dg, Eg):
            assert abs(v - E) <= 1e-6, (v, E)


@pytest.mark.parametrize("resident", [True, False])
def test_truncated_chain_golden(resident):
    """The hand-derived truncated-quadratic chains of tests/golden/trunc_chain.txt
    (Sec. 5.2) on the GPU: after 60 000 iterations the unlifted image and the
    energies meet them within FP32 rounding."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    from test_golden import golden
    for _, L, lam, f1, f2, f3, u1, u2, u3, E in golden("trunc_chain.txt"):
        fv = [f1, f2, f3] if f3 >= 0 else [f1, f2]
        want = [u1, u2, u3] if f3 >= 0 else [u1, u2]
        f = torch.tensor([fv], dtype=torch.float32, device="cuda")
        with G.Solver(G.LIFT_TRUNC_QUAD, 1, len(fv), int(L), 0.0, 1.0, lam, 25.0, 0.1, f=f,
                      resident=resident) as s:
            s.iterate(60000)
            ut = s.unlift().reshape(-1)
            Pg, Dg, Eg = s.energy()
        assert np.abs(ut - want).max() <= 2e-6, (ut, want)
        for v in (Pg, Dg, Eg):
            assert abs(v - E) <= 1e-6, (v, E)


@pytest.mark.parametrize("resident", [True, False])
def test_pl_two_pixel_golden(resident):
    """The hand-derived sampled-cost pairs of tests/golden/pl_two_pixel.txt
    (Sec. 5.4 costs, L = 2, Prop. 3) on the GPU: after 20 000 iterations the
    unlifted pair meets them within FP32 rounding of labels on [0, 4], and the
    energies within the stated relative bar (FP32 rounding of u on [0, 4],
    times cost slopes up to 2, is about 2e-6 of the energy)."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    from test_golden import PL_COSTS, golden
    cost = torch.tensor(PL_COSTS.reshape(1, 2, 5), dtype=torch.float32, device="cuda")
    for lam, u1, u2, E in golden("pl_two_pixel.txt"):
        with G.Solver(G.LIFT_PL_SAMPLED, 1, 2, 2, 0.0, 4.0, lam, 0.0, 0.0, cost=cost,
                      sample_min=0.0, sample_max=4.0, resident=resident) as s:
            s.iterate(20000)
            ut = s.unlift().reshape(-1)
            Pg, Dg, Eg = s.energy()
        assert np.abs(ut - [u1, u2]).max() <= 4 * 2e-6, (ut, u1, u2)
        for v in (Pg, Dg, Eg):
            assert abs(v - E) <= E_TOL * max(abs(E), 1.0), (v, E)


@pytest.mark.parametrize("resident", [True, False])
def test_periodic_two_pixel_golden(resident):
    """The hand-derived unwrapped pairs of tests/golden/periodic_two_pixel.txt
    (Sec. 5.5, L = 2 and 9) on the GPU: after 40 000 iterations the unlifted
    pair and the energies meet them within the parity bar (U_TOL of the label
    range, E_TOL).  The FP32 iterate settles further from the optimum here than
    on labels in [0, 1] (larger values on a 4 pi range, larger rounding per
    step): observed 1.6e-5 of the range at L = 2."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    from test_golden import golden
    two_pi = 2 * np.pi
    f = torch.tensor([[two_pi - 0.3, 0.3]], dtype=torch.float32, device="cuda")
    for L, lam, alpha, u1, u2, E in golden("periodic_two_pixel.txt"):
        with G.Solver(G.LIFT_PERIODIC_QUAD, 1, 2, int(L), 0.0, 2 * two_pi, lam, alpha, two_pi,
                      f=f, resident=resident) as s:
            s.iterate(40000)
            ut = s.unlift().reshape(-1)
            Pg, Dg, Eg = s.energy()
        assert np.abs(ut - [u1, u2]).max() <= U_TOL * 2 * two_pi, (ut, u1, u2)
        for v in (Pg, Dg, Eg):
            assert abs(v - E) <= E_TOL * max(abs(E), 1.0), (v, E)
