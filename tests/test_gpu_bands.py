"""The banded iteration graph (lift_set_bands): each band's half-steps follow
only those of the adjacent bands they read from, so the iterate must equal
the one-stream graph's bitwise."""
import numpy as np
import pytest

from _cases import case, gpu_solver
from paper_1512_01383_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")


def _same(a, b, iters):
    a.iterate(iters)
    b.iterate(iters)
    sa, sb = a.state(), b.state()
    for n in sa:
        np.testing.assert_array_equal(sa[n], sb[n])
    np.testing.assert_array_equal(a.unlift(), b.unlift())


@pytest.mark.parametrize("kind,H,W,L,bands,want", [
    (1, 512, 512, 10, 0, 4),     # automatic: 4 bands, dual steps in tile pairs
    (1, 512, 512, 5, 3, 3),      # forced, unequal band sizes
    (0, 300, 257, 2, 8, 8),      # single-tile dual steps, ragged width
    (2, 240, 320, 8, 0, 1),      # too few tiles for the automatic choice
    (2, 240, 320, 8, 4, 4),      # sampled costs, forced
    (1, 40, 40, 6, 8, 8),        # small, but every band longer than a row
    (0, 4, 2000, 2, 8, 3),       # rows of 2000 pixels: only 3 bands are long enough
])
def test_banded_graph_equals_one_stream(kind, H, W, L, bands, want):
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(kind, H, W, L, 3100 + L, ndisp=33) if kind == 2 else case(kind, H, W, L, 3100 + L)
    with gpu_solver(c, check_every=40, resident=False) as a, \
            gpu_solver(c, check_every=40, resident=False) as b:
        assert G.lift_set_bands(a.h, bands) == want
        assert G.lift_set_bands(b.h, 1) == 1
        _same(a, b, 130)             # 3 graph replays + 10 direct iterations


def test_banded_volume_equals_one_stream():
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    D = 40
    f = torch.from_numpy(synth.as_f32(synth.voronoi_ramps_3d(D, 48, 44, 3200)[0])).cuda()
    kw = dict(f=f, depth=D, check_every=30)
    with G.Solver(1, 48, 44, 6, 0.0, 1.0, 0.25, 25.0, 0.1, **kw) as a, \
            G.Solver(1, 48, 44, 6, 0.0, 1.0, 0.25, 25.0, 0.1, **kw) as b:
        assert G.lift_set_bands(a.h, 4) == 4
        assert G.lift_set_bands(b.h, 1) == 1
        _same(a, b, 70)


def test_banded_graph_follows_a_changing_balance():
    """The adaptive balance changes theta at every check without rebuilding
    the graph (the step kernels read the steps from device memory): banded
    and one-stream solves stay bitwise equal, theta included."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(1, 512, 512, 10, 3400)
    with gpu_solver(c, check_every=100, adaptive_balance=True, resident=False) as a, \
            gpu_solver(c, check_every=100, adaptive_balance=True, resident=False) as b:
        assert G.lift_set_bands(a.h, 0) == 4
        assert G.lift_set_bands(b.h, 1) == 1
        ra, na = a.solve(600, 1e-15)
        rb, nb = b.solve(600, 1e-15)
        assert na == nb == 600
        ta, tb = G.lift_get_balance(a.h), G.lift_get_balance(b.h)
        assert ta == tb and ta != 1.0
        np.testing.assert_array_equal(a.unlift(), b.unlift())
