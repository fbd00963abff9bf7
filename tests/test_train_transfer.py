"""The network transfer of the training driver (Sec. 4.2.3: a 5-level network
initialises a 6-level one): the (L+1)-level network built from an L-level one
must compute exactly what the L-level network computes (FP64 oracle), and
differ from it once the new level's Aff2 is non-zero."""
import numpy as np

import oracle
from paper_2310_00177_b300 import synth
from paper_2310_00177_b300.train import AFF_PARAMS, CCONV_PARAMS, PER_LEVEL, transfer_weights


def test_transfer_preserves_the_network():
    lab = synth.slosh_scene(32, 11)
    r = np.random.default_rng(12).standard_normal(lab.shape)
    for L in (3, 4, 5):
        w = synth.init_weights(L, 20 + L, spread=0.05)
        w2 = transfer_weights(w.astype(np.float32), L)
        assert w2.size == oracle.weight_count(L + 1)
        z = oracle.network(lab, L, w.astype(np.float32).astype(np.float64), r)
        z2 = oracle.network(lab, L + 1, w2.astype(np.float64), r)
        np.testing.assert_allclose(z2, z, rtol=0, atol=1e-12 * np.abs(z).max())
        # the new coarse path enters through Aff2 of level L: switching it on changes the output
        w3 = w2.astype(np.float64).copy()
        w3[(L - 1) * PER_LEVEL + 2 * CCONV_PARAMS + 2 * AFF_PARAMS - 1] = 0.5
        z3 = oracle.network(lab, L + 1, w3, r)
        assert np.linalg.norm(z3 - z) > 1e-3 * np.linalg.norm(z)
