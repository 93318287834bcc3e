"""The hand-written reverse pass of the unrolled solve (adjoint.cu) against
the oracle's FP64 reverse pass, checkpoint invariance, the autograd.Function,
and a first-order Taylor check at the 256x256, L=16, 500-iteration size."""
import numpy as np
import pytest

import oracle as O
from paper_1512_01383_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def _solver(kind, f, L, lam, alpha, nu, theta=1.0, aniso=0):
    from paper_1512_01383_gb300 import lift as G
    H, W = f.shape
    return G.Solver(kind, H, W, L, 0.0, 1.0, lam, alpha, nu, f=torch.from_numpy(f).cuda(),
                    step_balance=theta, anisotropic=bool(aniso))


def _gpu_grads(s, iters, every, clean):
    from paper_1512_01383_gb300 import lift as G
    G.lift_unrolled_forward(s.h, iters, every)
    u = torch.empty((s.H, s.W), device="cuda")
    G.lift_unlift(s.h, u)
    cl = torch.from_numpy(clean.astype(np.float32)).cuda()
    gu = (2.0 * (u - cl)).contiguous()
    gf = torch.empty_like(u)
    sc = G.lift_unrolled_backward(s.h, gu, gf)
    return u.cpu().numpy(), gf.cpu().numpy(), np.array(sc)


CASES = [
    (1, 5, 0.25, 25.0, 0.1, 1.0, 0),
    (0, 4, 0.2, 1.5, 0.0, 1.0, 0),
    (1, 9, 0.3, 20.0, 0.08, 1.0, 0),
    (1, 5, 0.25, 25.0, 0.1, 16.0, 0),
    (1, 5, 0.25, 25.0, 0.1, 1.0, 1),
    (3, 6, 0.2, 1.5, 0.4, 1.0, 0),      # periodic pieces, period 0.4 on [0, 1]
]


@pytest.mark.parametrize("H,W,iters,df_tol,sc_tol", [
    # observed on a GB300: dL/df within 4.7e-6 of its maximum and the
    # scalars within 1.7e-3 (11 x 9), 3.3e-4 and 3.9e-4 (32 x 32)
    (11, 9, 30, 1e-4, 5e-3),
    (32, 32, 100, 1e-3, 2e-3),
])
@pytest.mark.parametrize("kind,L,lam,alpha,nu,theta,aniso", CASES)
def test_gradients_match_oracle_reverse_pass(kind, L, lam, alpha, nu, theta, aniso, H, W, iters,
                                             df_tol, sc_tol):
    _require_gpu()
    noisy, clean = synth.voronoi_ramps(H, W, 81 + L, cells=4)
    f = synth.as_f32(noisy)
    with _solver(kind, f, L, lam, alpha, nu, theta, aniso) as s:
        u, gf, gs = _gpu_grads(s, iters, 7, clean)
    okind = {0: O.QUAD, 1: O.TRUNC, 3: O.PERIODIC}[kind]
    P = O.Problem(okind, H, W, L, 0.0, 1.0, lam=lam, alpha=alpha,
                  nu=nu, f=f.astype(np.float64), theta=theta, aniso=aniso)
    X = O.State(P)
    O.pdhg(P, X, iters)
    uo = O.unlift(P, X.u)
    assert np.abs(u.reshape(-1) - uo).max() <= 1e-4
    gfo, gso = O.unrolled_grad(P, iters, 2.0 * (uo - clean.reshape(-1)))
    scale = np.abs(gfo).max()
    assert scale > 1e-3
    assert np.abs(gf.reshape(-1) - gfo).max() <= df_tol * scale
    # the unrolled map is piecewise smooth: where an FP32 and an FP64 branch
    # choice differ near a region boundary the one-sided derivatives differ,
    # which the scalar sums over all records collect
    for g, o in zip(gs, gso):
        assert abs(g - o) <= sc_tol * max(abs(o), 1e-2), (gs, gso)


def test_checkpoint_spacing_does_not_change_gradients():
    _require_gpu()
    H, W, L, iters = 14, 12, 6, 40
    noisy, clean = synth.voronoi_ramps(H, W, 91)
    f = synth.as_f32(noisy)
    res = []
    with _solver(1, f, L, 0.25, 25.0, 0.1) as s:
        for every in (1, 7, 40):
            res.append(_gpu_grads(s, iters, every, clean))
    for r in res[1:]:
        np.testing.assert_array_equal(r[0], res[0][0])
        np.testing.assert_array_equal(r[1], res[0][1])
        np.testing.assert_array_equal(r[2], res[0][2])


def test_autograd_function():
    _require_gpu()
    from paper_1512_01383_gb300.autograd import unrolled_solve
    H, W, L, iters = 12, 10, 5, 25
    noisy, clean = synth.voronoi_ramps(H, W, 95)
    f = torch.from_numpy(synth.as_f32(noisy)).cuda().requires_grad_(True)
    lam = torch.tensor(0.25, dtype=torch.float64, requires_grad=True)
    al = torch.tensor(25.0, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    with _solver(1, synth.as_f32(noisy), L, 0.25, 25.0, 0.1) as s:
        u = unrolled_solve(f, lam, al, nu, s, iters, 5)
        loss = ((u - torch.from_numpy(clean.astype(np.float32)).cuda()) ** 2).sum()
        loss.backward()
        u2, gf2, gs2 = _gpu_grads(s, iters, 5, clean)
    np.testing.assert_allclose(u.detach().cpu().numpy(), u2)
    np.testing.assert_allclose(f.grad.cpu().numpy(), gf2)
    np.testing.assert_allclose([lam.grad.item(), al.grad.item(), nu.grad.item()], gs2)


def test_mid_size_many_segments_match_oracle_reverse_pass():
    """32 x 32, L = 16, 200 iterations with checkpoints every 50: the
    reverse pass recomputes four segments, the regime of the 256 x 256
    configuration, against the oracle's FP64 reverse pass (the observed
    errors are printed next to the tolerances)."""
    _require_gpu()
    H, W, L, iters = 32, 32, 16, 200
    noisy, clean = synth.voronoi_ramps(H, W, 97)
    f = synth.as_f32(noisy)
    with _solver(1, f, L, 0.25, 25.0, 0.1) as s:
        u, gf, gs = _gpu_grads(s, iters, 50, clean)
    P = O.Problem(O.TRUNC, H, W, L, 0.0, 1.0, lam=0.25, alpha=25.0, nu=0.1, f=f.astype(np.float64))
    X = O.State(P)
    O.pdhg(P, X, iters)
    uo = O.unlift(P, X.u)
    assert np.abs(u.reshape(-1) - uo).max() <= 1e-4
    gfo, gso = O.unrolled_grad(P, iters, 2.0 * (uo - clean.reshape(-1)))
    scale = np.abs(gfo).max()
    ef = np.abs(gf.reshape(-1) - gfo).max() / scale
    es = [abs(g - o) / max(abs(o), 1e-2) for g, o in zip(gs, gso)]
    print(f"mid-size adjoint: max|dL/df - oracle| / max = {ef:.2e}; "
          f"scalar relative errors {es[0]:.2e} {es[1]:.2e} {es[2]:.2e}")
    # observed on a GB300: 1.4e-3 and 1e-5..3e-5 (the scalar sums over many
    # records average out the branch differences that dominate tiny images)
    assert ef <= 2e-3
    for e in es:
        assert e <= 1e-3, (gs, gso)


def test_backward_refuses_a_replaced_forward_pass():
    """The handle keeps one forward pass: a second unrolled_solve on the
    same solver, or new parameters, data or a reset, make the reverse pass of
    the first one fail loudly (the autograd wrapper and the C entry point)."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    from paper_1512_01383_gb300.autograd import unrolled_solve
    H, W, L, iters = 12, 10, 5, 20
    noisy, clean = synth.voronoi_ramps(H, W, 96)
    f = torch.from_numpy(synth.as_f32(noisy)).cuda().requires_grad_(True)
    cl = torch.from_numpy(clean.astype(np.float32)).cuda()
    with _solver(1, synth.as_f32(noisy), L, 0.25, 25.0, 0.1) as s:
        u1 = unrolled_solve(f, 0.25, 25.0, 0.1, s, iters, 5)
        u2 = unrolled_solve(f, 0.3, 25.0, 0.1, s, iters, 5)
        with pytest.raises(G.LiftError):
            ((u1 - cl) ** 2).sum().backward()
        ((u2 - cl) ** 2).sum().backward()          # the stored pass is u2's
        assert f.grad is not None and torch.isfinite(f.grad).all()
        gu = torch.zeros((H, W), device="cuda")
        for change in (lambda: G.lift_set_params(s.h, 0.2, 25.0, 0.1),
                       lambda: G.lift_set_data(s.h, torch.from_numpy(synth.as_f32(noisy)).cuda()),
                       lambda: G.lift_reset(s.h)):
            G.lift_unrolled_forward(s.h, iters, 5)
            g0 = G.lift_unrolled_generation(s.h)
            G.lift_unrolled_backward(s.h, gu)
            change()
            assert G.lift_unrolled_generation(s.h) != g0
            with pytest.raises(G.LiftError) as e:
                G.lift_unrolled_backward(s.h, gu)
            assert e.value.code == G.LIFT_ERR_ARG


def test_full_size_taylor_check():
    """256x256, L=16, 500 unrolled iterations, checkpoints every 50: the
    gradient is finite, equals that of a single-segment reverse pass, and
    predicts the change of the loss when single pixels of f move (FP32
    central differences, step 1e-3; a move of one pixel leaves the rounding
    of all distant pixels unchanged, so the quotient is not drowned in the
    loss's rounding noise as a move of every pixel would be)."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    H = W = 256
    L, iters = 16, 500
    noisy, clean = synth.voronoi_ramps(H, W, synth.BASE_SEED + 4)
    f = synth.as_f32(noisy)
    s = G.Solver(1, H, W, L, 0.0, 1.0, 0.25, 25.0, 0.1, f=torch.from_numpy(f).cuda())
    try:
        u, gf, gs = _gpu_grads(s, iters, 50, clean)
        assert np.all(np.isfinite(gf)) and np.all(np.isfinite(gs))
        u1, gf1, gs1 = _gpu_grads(s, iters, 500, clean)
        np.testing.assert_array_equal(gf, gf1)
        np.testing.assert_array_equal(gs, gs1)

        def loss_at(fv):
            G.lift_set_data(s.h, torch.from_numpy(fv).cuda())
            G.lift_unrolled_forward(s.h, iters, 50)
            return float(((s.unlift().astype(np.float64) - clean) ** 2).sum())

        # pixels whose gradient is well above the rounding floor; a pixel
        # passes if either step (1e-3 or 3e-4) stays clear of the map's kinks
        order = np.argsort(-np.abs(gf).reshape(-1))
        rel = []
        for j in order[:40:5]:
            e = np.zeros_like(f)
            e.reshape(-1)[j] = 1.0
            pred = float(gf.reshape(-1)[j])
            best = np.inf
            for eps in (1e-3, 3e-4):
                fd = (loss_at(f + eps * e) - loss_at(f - eps * e)) / (2 * eps)
                best = min(best, abs(fd - pred) / abs(pred))
            rel.append(best)
        rel = np.array(rel)
        assert np.median(rel) <= 0.05 and (rel <= 0.1).sum() >= 6, rel
    finally:
        s.close()
