"""The seeded input generators (paper_1512_01383_gb300/synth.py) that the
GPU path, the oracle checks and the bench all draw from: the random stream
is SplitMix64 (pinned to its reference outputs), the draws do not depend on
how they are chunked, and each workload stand-in has the shape, value
ranges and structure its recipe states."""
import numpy as np
import pytest

from paper_1512_01383_gb300 import synth


def test_splitmix64_reference_outputs():
    """SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) from state 1234567: its
    first five outputs are the generator's standard reference values."""
    r = synth.Rng(0)
    r.key = np.uint64(1234567)
    r.counter = 0
    assert [int(v) for v in r._bits(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


def test_draws_do_not_depend_on_chunking():
    a, b = synth.Rng(42, 3), synth.Rng(42, 3)
    whole = a._bits(10)
    parts = np.concatenate([b._bits(3), b._bits(7)])
    np.testing.assert_array_equal(whole, parts)
    # other seeds and streams give other sequences
    assert not np.array_equal(synth.Rng(42, 4)._bits(10), whole)
    assert not np.array_equal(synth.Rng(43, 3)._bits(10), whole)


def test_uniform_and_normal_moments():
    r = synth.Rng(7)
    u = r.uniform(200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12.0) < 0.002
    g = r.normal(200000, 2.0)
    assert abs(g.mean()) < 0.02 and abs(g.std() - 2.0) < 0.02
    k = r.integers(100000, 4, 9)
    assert k.min() == 4 and k.max() == 9 and set(np.unique(k)) == set(range(4, 10))


def test_voronoi_ramps_recipe():
    """Truncated-quadratic stand-in: clean ramps in [0, 1], N(0, 0.05^2)
    noise, 10 % of pixels replaced by U[0, 1]; deterministic in the seed."""
    noisy, clean = synth.voronoi_ramps(256, 192, 11)
    assert noisy.shape == clean.shape == (256, 192)
    assert clean.min() >= 0.0 and clean.max() <= 1.0
    dev = np.abs(noisy - clean)
    # only outliers deviate by more than 6 sigma; about half of them do
    far = (dev > 0.3).mean()
    assert 0.02 < far < 0.1, far
    near = (noisy - clean)[dev < 0.15]
    assert 0.045 < near.std() < 0.06, near.std()
    n2, c2 = synth.voronoi_ramps(256, 192, 11)
    np.testing.assert_array_equal(n2, noisy)
    np.testing.assert_array_equal(c2, clean)
    assert not np.array_equal(synth.voronoi_ramps(256, 192, 12)[0], noisy)


def test_gaussian_blobs_recipe():
    f = synth.gaussian_blobs(64, 64, 5)
    assert f.shape == (64, 64)
    # min-max normalised blobs in [0, 1] plus N(0, 0.1^2)
    assert -0.6 < f.min() < 0.0 and 1.0 < f.max() < 1.6
    np.testing.assert_array_equal(f, synth.gaussian_blobs(64, 64, 5))


def test_stereo_cost_recipe():
    """Truncated absolute differences in [0, tau]; at the true disparity
    the cost is far below its mean over all disparities."""
    cost, disp = synth.stereo_cost(48, 96, 3, ndisp=33, tau=0.2)
    assert cost.shape == (48, 96, 33) and disp.shape == (48, 96)
    assert cost.min() >= 0.0 and cost.max() <= 0.2
    assert disp.min() >= 0.0 and disp.max() <= 32.0
    H, W = disp.shape
    inner = (np.arange(W)[None, :] + disp) < W - 2           # no clamping at the right edge
    d0 = np.floor(disp).astype(np.int64)
    rows, cols = np.nonzero(inner)
    at_true = np.minimum(cost[rows, cols, d0[rows, cols]], cost[rows, cols, np.minimum(d0[rows, cols] + 1, 32)])
    assert at_true.mean() < 0.25 * cost[inner].mean(), (at_true.mean(), cost[inner].mean())


def test_wrapped_phase_recipe():
    w, true = synth.wrapped_phase(64, 80, 9)
    assert w.min() >= 0.0 and w.max() < 2 * np.pi
    assert abs(true.min() - 1.0) < 1e-12 and abs(true.max() - 11.0) < 1e-12
    d = np.angle(np.exp(1j * (w - true)))                      # circular difference
    assert abs(d.mean()) < 0.01 and abs(d.std() - 0.1) < 0.01


@pytest.mark.parametrize("n", [1, 64, 256])
def test_batch_instances_recipe(n):
    inst = synth.batch_instances(n, synth.BASE_SEED + 2)
    assert len(inst) == n
    assert all(128 <= s <= 1024 and L in (4, 8, 16, 32) for s, L in inst)
    assert inst == synth.batch_instances(n, synth.BASE_SEED + 2)


def test_as_f32_rounds_to_contiguous_float32():
    a = np.arange(12, dtype=np.float64).reshape(3, 4)[:, ::2]
    b = synth.as_f32(a)
    assert b.dtype == np.float32 and b.flags["C_CONTIGUOUS"]
    np.testing.assert_array_equal(b, a.astype(np.float32))
