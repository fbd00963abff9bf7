"""Checks of the seeded scene / right-hand-side generators (no GPU)."""
import numpy as np

from paper_2310_00177_b300 import synth


def test_pool_scene_structure_and_determinism():
    lab = synth.pool_scene(32, 1000)
    assert lab.shape == (32, 32, 32) and lab.dtype == np.uint8
    assert (lab[0] == synth.SOLID).all() and (lab[:, :, -1] == synth.SOLID).all()
    inner = lab[1:-1, 1:-1, 1:-1]
    assert ((inner[23:] == synth.AIR) | (inner[23:] == synth.SOLID)).all()
    assert (inner[:23] != synth.AIR).all()
    np.testing.assert_array_equal(lab, synth.pool_scene(32, 1000))
    assert not np.array_equal(lab, synth.pool_scene(32, 1001))


def test_slosh_scene_surface_and_frames():
    lab = synth.slosh_scene(64, 7)
    counts = np.bincount(lab.ravel(), minlength=3)
    assert counts.min() > 0
    # air only above the lowest possible surface height, fluid only below the highest
    z_air = np.argwhere(lab == synth.AIR)[:, 0]
    z_flu = np.argwhere(lab == synth.FLUID)[:, 0]
    assert z_air.min() >= 40 - 8 - 1 and z_flu.max() <= 40 + 8 + 1
    nxt = synth.slosh_scene(64, 7, frame=1)
    assert not np.array_equal(lab, nxt)


def test_rhs_is_zero_off_fluid_and_mean_free_on_neumann_components():
    lab = synth.slosh_scene(32, 3)
    lab[3:9, 3:9, 3:9] = synth.SOLID
    lab[4:8, 4:8, 4:8] = synth.FLUID  # a sealed pocket
    b = synth.rhs_normal(lab, 4)
    assert not b[lab != synth.FLUID].any()
    comp, pure = synth.neumann_components(lab)
    assert len(pure) >= 1
    for c in pure:
        assert abs(b[comp == c].sum()) < 1e-10


def test_init_weights_layout():
    w = synth.init_weights(4, 0)
    assert w.size == 15990
    per = 2 * synth.CCONV_PARAMS + 2 * synth.AFF_PARAMS
    assert w[2187 + 13] > 0.9  # CConv1 level-1 centre bias
    assert w[(4 - 1) * per + 2187 + 13] > 10.0  # coarsest CConv1 centre bias (4^3/6)


def test_serving_requests_are_poisson_and_mixed():
    reqs = synth.serving_requests(512, 200.0, seed=5000)
    t = np.array([r["t_arrival"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert 1.5 < t[-1] < 3.5  # mean inter-arrival 5 ms
    sizes = {r["n"] for r in reqs}
    assert sizes == {64, 128, 192, 256}
