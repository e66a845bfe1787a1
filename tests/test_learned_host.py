"""Host-side logic of the learned lane change that runs without a GPU: the class weights of
the training loss, the initial network, and the mix of logged scenarios."""
import collections
import math

import numpy as np
import torch

from oracle import mlp
from paper_2405_12520_b300 import learned, moss


def test_class_weights_are_softened_inverse_frequencies_with_mean_one():
    y = torch.tensor([0] * 60 + [1] * 30 + [2] * 10, dtype=torch.int32)
    w, cnt = learned.class_weights(y, power=0.25)
    assert cnt.tolist() == [60.0, 30.0, 10.0]
    raw = np.array([(100 / 60) ** 0.25, (100 / 30) ** 0.25, (100 / 10) ** 0.25])
    np.testing.assert_allclose(w, raw / raw.mean(), rtol=1e-6)
    assert abs(float(w.mean()) - 1.0) < 1e-6
    # a class that never occurs counts as one sample, not as a division by zero
    w0, cnt0 = learned.class_weights(torch.tensor([0, 0, 1], dtype=torch.int32))
    assert cnt0.tolist() == [2.0, 1.0, 0.0] and np.all(np.isfinite(w0))


def test_initial_network_has_the_abi_layout_he_uniform_weights_and_zero_biases():
    th = learned.init_params(3)
    assert th.dtype == np.float32 and th.shape == (moss.MLP_NPARAM,) == (mlp.N_PARAMS,)
    p = mlp.unpack(th.astype(np.float64))
    for name, shape in mlp.SHAPES:
        a = p[name]
        assert a.shape == shape
        if name.startswith("b"):
            assert np.all(a == 0.0), name
        else:
            lim = math.sqrt(6.0 / shape[1])
            assert np.all(np.abs(a) <= lim) and np.abs(a).max() > 0.9 * lim, name
    assert np.array_equal(th, learned.init_params(3)) and not np.array_equal(th, learned.init_params(4))


def test_scenario_mix_follows_its_shares_with_distinct_seeds():
    n = 256
    specs = learned.mixed_specs(n)
    assert specs == learned.mixed_specs(n)                      # deterministic
    assert len({s for s, _, _ in specs}) == len(specs)          # one seed per scenario
    got = collections.Counter((t, p) for _, t, p in specs)
    for trips, placed, share in learned.MIX:
        assert got[(trips, placed)] == int(round(n * share))
