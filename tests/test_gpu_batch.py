"""Batched solves: many instances of different sizes and label counts in one
launch per half-step (CUDA graph per check interval) against single-instance
handles and against the oracle."""
import numpy as np
import pytest

import oracle as O
from _cases import case, gpu_solver, oracle_run

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(37, 29, 5), (20, 64, 9), (64, 20, 3), (13, 13, 17), (50, 41, 33), (1, 70, 4)]


def _require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def _batch(cases, check_every=50):
    from paper_1512_01383_gb300 import lift as G
    keep = [torch.from_numpy(c["f"]).cuda() for c in cases]
    specs = [G.make_spec(c["kind"], c["H"], c["W"], c["L"], c["gamma_min"], c["gamma_max"],
                         c["lam"], c.get("alpha", 1.0), c.get("nu", 0.0), f=f,
                         check_every=check_every, step_balance=c.get("theta", 1.0))
             for c, f in zip(cases, keep)]
    b = G.lift_create_batch(specs, torch.cuda.current_stream().cuda_stream)
    return b, keep


# big-instance thresholds in 256-thread tiles: 0 merges every instance, 1 runs
# every instance on the single-instance kernels, 17 splits SHAPES 3 / 3
# (their tile counts are 17, 40, 10, 11, 257, 1)
SCHEDULES = [(0, 0), (1, len(SHAPES)), (17, 3)]


@pytest.mark.parametrize("big_tiles,n_big", SCHEDULES)
def test_batch_equals_single_handles_bitwise(big_tiles, n_big):
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    cases = [case(1, H, W, L, 1200 + j) for j, (H, W, L) in enumerate(SHAPES)]
    b, keep = _batch(cases)
    try:
        G.lift_batch_set_schedule(b, 256, big_tiles)
        assert G.lift_batch_schedule(b) == (256, big_tiles, n_big)
        G.lift_batch_iterate(b, 130)          # two graph replays + 30 direct iterations
        e = G.lift_batch_energy(b)
        for j, c in enumerate(cases):
            with gpu_solver(c, resident=False) as s:
                s.iterate(130)
                ut = s.unlift()
                Pg, Dg, Eg = s.energy()
                nb = G.lift_state_bytes(s.h)
                a = np.empty(nb, np.uint8)
                G.lift_get_state(s.h, a)
            ub = np.empty((c["H"], c["W"]), np.float32)
            G.lift_batch_unlift(b, j, ub)
            np.testing.assert_array_equal(ub, ut)
            sb = np.empty(nb, np.uint8)
            G.lift_batch_get_state(b, j, sb)
            np.testing.assert_array_equal(sb, a)
            assert tuple(e[j]) == (Pg, Dg, Eg)
    finally:
        G.lift_batch_destroy(b)


def test_batch_instance_matches_oracle():
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    cases = [case(1, 31, 23, 5, 1300), case(1, 17, 19, 2, 1301), case(1, 12, 40, 9, 1302)]
    b, keep = _batch(cases, check_every=40)
    try:
        G.lift_batch_iterate(b, 120)
        e = G.lift_batch_energy(b)
        for j, c in enumerate(cases):
            P, X = oracle_run(c, 120)
            ub = np.empty((c["H"], c["W"]), np.float32)
            G.lift_batch_unlift(b, j, ub)
            assert np.abs(ub.reshape(-1) - O.unlift(P, X.u)).max() <= 1e-4
            Po, Do, Eo = O.energy(P, X)
            for g, o in zip(e[j], (Po, Do, Eo)):
                assert abs(g - o) <= 1e-5 * max(abs(o), 1.0)
    finally:
        G.lift_batch_destroy(b)


@pytest.mark.parametrize("big_tiles", [0, 1])
def test_batch_solve_stops_converged_instances(big_tiles):
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    cases = [case(1, H, W, L, 1400 + j, theta=float((L - 1) ** 2))
             for j, (H, W, L) in enumerate([(24, 24, 3), (40, 32, 5), (16, 48, 9)])]
    b, keep = _batch(cases, check_every=100)
    try:
        G.lift_batch_set_schedule(b, 256, big_tiles)
        rc, iters, nconv = G.lift_batch_solve(b, 40000, 1e-4)
        assert rc == G.LIFT_OK and nconv == len(cases)
        assert all(i > 0 and i % 100 == 0 for i in iters)
        assert len(set(iters)) > 1                     # instances stopped at different times
        e = G.lift_batch_energy(b)
        for p, d, _ in e:
            assert (p - d) / max(abs(p), abs(d), 1.0) <= 1e-4 and p >= d - 1e-9
        # converged instances no longer move
        snaps = []
        for j, c in enumerate(cases):
            N, k = c["H"] * c["W"], c["L"] - 1
            a = np.empty(N * k * 32 + N * 4, np.uint8)
            G.lift_batch_get_state(b, j, a)
            snaps.append(a)
        G.lift_batch_iterate(b, 50)
        torch.cuda.synchronize()
        for j, c in enumerate(cases):
            a = np.empty_like(snaps[j])
            G.lift_batch_get_state(b, j, a)
            np.testing.assert_array_equal(a, snaps[j])
    finally:
        G.lift_batch_destroy(b)


def test_batch_autotune_keeps_results():
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    cases = [case(1, H, W, L, 1500 + j) for j, (H, W, L) in enumerate(SHAPES)]
    b, keep = _batch(cases)
    try:
        t = G.lift_batch_autotune(b, 5)
        assert t in (128, 256, 512) and G.lift_batch_schedule(b)[0] == t
        G.lift_batch_iterate(b, 80)
        for j, c in enumerate(cases):
            P, X = oracle_run(c, 80)
            ub = np.empty((c["H"], c["W"]), np.float32)
            G.lift_batch_unlift(b, j, ub)
            assert np.abs(ub.reshape(-1) - O.unlift(P, X.u)).max() <= 1e-4
    finally:
        G.lift_batch_destroy(b)


def test_batch_rejects_mixed_or_pl_kinds():
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    a, c2 = case(1, 8, 8, 5, 1600), case(0, 8, 8, 2, 1601)
    fa, fc = torch.from_numpy(a["f"]).cuda(), torch.from_numpy(c2["f"]).cuda()
    specs = [G.make_spec(1, 8, 8, 5, 0, 1, 0.25, 25, 0.1, f=fa),
             G.make_spec(0, 8, 8, 2, 0, 1, 0.2, 1.0, 0.0, f=fc)]
    with pytest.raises(G.LiftError) as e:
        G.lift_create_batch(specs)
    assert e.value.code == G.LIFT_ERR_SPEC


def test_batch_schedule_rejects_invalid_arguments():
    """A tile width other than 128/256/512 or a negative threshold is an
    argument error and leaves the schedule as it was."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    cases = [case(1, 9, 11, 5, 1600), case(1, 10, 7, 3, 1601)]
    b, keep = _batch(cases)
    try:
        before = G.lift_batch_schedule(b)
        with pytest.raises(G.LiftError):
            G.lift_batch_set_schedule(b, 200, 0)
        with pytest.raises(G.LiftError):
            G.lift_batch_set_schedule(b, 256, -1)
        assert G.lift_batch_schedule(b) == before
    finally:
        G.lift_batch_destroy(b)
