"""lift_energy_noalloc: energies of a caller-held state without any allocation.

Some callers cannot call cudaMalloc: their device memory all belongs to
another allocator (a framework's caching pool, a fixed budget), or they must
not trigger an allocation that can synchronise the device.  The allocation-
free entry point keeps its per-block partial sums in one fixed array of the
library instead.  This file checks it, through the C ABI, against the
handle-based lift_energy on the same state, on two calls in a row (the second
on a different state, so stale contents of the shared array would show).
It is named to be collected last.
"""
import numpy as np
import pytest

from _cases import case, gpu_solver

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

E_TOL = 1e-5   # relative, as for every energy comparison in the GPU tests


@pytest.mark.parametrize("kind,H,W,L", [(1, 37, 29, 5), (0, 24, 31, 3), (1, 130, 70, 20)])
def test_noalloc_energy_matches_lift_energy(kind, H, W, L):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1512_01383_gb300 import lift as G
    c = case(kind, H, W, L, 1100 + H + L)
    f_dev = torch.from_numpy(c["f"]).cuda()
    spec = G.make_spec(c["kind"], H, W, L, c["gamma_min"], c["gamma_max"], c["lam"],
                       c.get("alpha", 1.0), c.get("nu", 0.0), f=f_dev)
    stream = torch.cuda.current_stream().cuda_stream
    with gpu_solver(c, stream=stream) as s:
        state = torch.empty(G.lift_state_bytes(s.h), dtype=torch.uint8, device="cuda")
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        for iters in (40, 25):                  # two calls in a row, different states
            s.iterate(iters)
            want = s.energy()
            G.lift_get_state(s.h, state)
            G.lift_energy_noalloc(spec, state, out, stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            for g, w in zip(got, want):
                assert np.isfinite(g)
                assert abs(g - w) <= E_TOL * max(abs(w), 1.0), (iters, got, want)


def test_noalloc_rejects_oversized_and_host_inputs():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1512_01383_gb300 import lift as G
    f_dev = torch.zeros(4, device="cuda")
    state = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    big = G.make_spec(G.LIFT_TRUNC_QUAD, 1025, 1024, 5, 0.0, 1.0, 0.25, 25.0, 0.1, f=f_dev)
    with pytest.raises(G.LiftError) as e:
        G.lift_energy_noalloc(big, state, out)
    assert e.value.code == G.LIFT_ERR_ARG
    host = G.make_spec(G.LIFT_TRUNC_QUAD, 2, 2, 5, 0.0, 1.0, 0.25, 25.0, 0.1,
                       f=np.zeros(4, np.float32))
    with pytest.raises(G.LiftError) as e:
        G.lift_energy_noalloc(host, state, out)
    assert e.value.code == G.LIFT_ERR_ARG
    # buffers the wrapper checks before the C call (which cannot see sizes)
    ok = G.make_spec(G.LIFT_TRUNC_QUAD, 2, 2, 5, 0.0, 1.0, 0.25, 25.0, 0.1, f=f_dev)
    bad_outs = [torch.zeros(3, dtype=torch.float32, device="cuda"),    # not float64
                torch.zeros(2, dtype=torch.float64, device="cuda"),    # too short
                torch.zeros(3, dtype=torch.float64)]                   # on the host
    for bad in bad_outs:
        with pytest.raises(G.LiftError) as e:
            G.lift_energy_noalloc(ok, state, bad)
        assert e.value.code == G.LIFT_ERR_ARG
    small = torch.zeros(2 * 2 * 4 * 32 - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(G.LiftError) as e:
        G.lift_energy_noalloc(ok, small, out)
    assert e.value.code == G.LIFT_ERR_ARG
