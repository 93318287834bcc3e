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


@pytest.mark.parametrize("kind,H,W,L,nb", [
    (1, 512, 512, 20, 4),        # the bench's workload, four bands
    (1, 61, 47, 6, 3),           # rows not divisible by the band count
    (2, 48, 64, 8, 2),           # sampled costs (PL pieces)
    (0, 40, 33, 2, 5),           # one interval per pixel
    (3, 37, 41, 7, 2),           # periodic pieces
])
def test_band_handles_equal_one_handle(kind, H, W, L, nb):
    """The spatial decomposition of Sec. 4's grid over band handles on one
    GPU (one handle per band of rows, halo rows exchanged by device copies
    before each half-step): after the iterations the bands' own rows equal
    the single handle's state bit for bit, and the bands' energies add up to
    the single handle's (FP64 sums in another order)."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    from paper_1512_01383_gb300.bands import LocalBands
    c = case(kind, H, W, L, 3500 + L, ndisp=17) if kind == 2 else case(kind, H, W, L, 3500 + L)
    iters = 60
    data = {n: torch.from_numpy(c[n]).cuda() for n in ("f", "cost") if c.get(n) is not None}
    spec = G.make_spec(c["kind"], H, W, L, c["gamma_min"], c["gamma_max"], c["lam"],
                       c.get("alpha", 1.0), c.get("nu", 0.0), f=data.get("f"),
                       cost=data.get("cost"), sample_min=c.get("sample_min", 0.0),
                       sample_max=c.get("sample_max", 1.0))
    with gpu_solver(c, resident=False) as a:
        bands = LocalBands(spec, nb)          # reads the data through spec (kept alive above)
        try:
            for _ in range(iters):
                G.lift_dual_step(a.h)
                G.lift_primal_step(a.h)
            bands.iterate(iters)
            sa = a.state()
            ua = a.unlift()
            ea = a.energy()
            np.testing.assert_array_equal(bands.unlift(), ua)
            for b in bands.bands:
                sb = G.state_arrays(b.h, b.k)
                up = 0 if b.first else 1
                own = slice(up * W, (up + b.row1 - b.row0) * W)
                glob = slice(b.row0 * W, b.row1 * W)
                for n in ("u", "s", "ubar", "sbar", "v", "z", "px", "py"):
                    np.testing.assert_array_equal(sb[n][own], sa[n][glob], err_msg=n)
                np.testing.assert_array_equal(sb["q"][own], sa["q"][glob])
            eb = bands.energy()
            for x, y in zip(eb, ea):
                assert abs(x - y) <= 1e-12 * max(abs(y), 1.0), (eb, ea)
        finally:
            bands.close()


def test_band_handles_refuse_whole_image_calls():
    """A band runs only under the exchange schedule: lift_iterate, lift_solve
    and lift_gap return LIFT_ERR_ARG; exports and imports that have no
    neighbour do too."""
    _require_gpu()
    from paper_1512_01383_gb300 import lift as G
    c = case(1, 20, 16, 5, 3600)
    f = torch.from_numpy(c["f"]).cuda()
    spec = G.make_spec(1, 20, 16, 5, 0.0, 1.0, c["lam"], c["alpha"], c["nu"], f=f)
    top = G.lift_create_band(spec, 0, 10)
    try:
        for fn in (lambda: G.lift_iterate(top, 5), lambda: G.lift_gap(top),
                   lambda: G.lift_solve(top, 10, 1e-5)):
            with pytest.raises(G.LiftError) as e:
                fn()
            assert e.value.code == G.LIFT_ERR_ARG
        buf = torch.empty(G.lift_band_halo_bytes(top, G.LIFT_HALO_PRIMAL), dtype=torch.uint8,
                          device="cuda")
        with pytest.raises(G.LiftError):
            G.lift_band_export(top, G.LIFT_HALO_PRIMAL, buf)     # no band above
        with pytest.raises(G.LiftError):
            G.lift_band_import(top, G.LIFT_HALO_DUAL, buf)       # no halo row above
        with pytest.raises(G.LiftError):
            G.lift_create_band(spec, 10, 25)                     # beyond the image
    finally:
        G.lift_destroy(top)
