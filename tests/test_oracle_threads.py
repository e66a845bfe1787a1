"""The oracle's update phase on several OpenMP threads gives the single-threaded oracle's
results bit for bit (every vehicle's update reads only the snapshot and writes only its own
outputs, Sec. III-A's two phases), with the rule, with the learned lane change (R19) and
under max-pressure signals (R13), including every per-vehicle debug record."""
import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2405_12520_b300 import synth

P = synth.default_params()


@pytest.mark.parametrize("mode", ["rule", "learned", "maxpressure"])
def test_threaded_oracle_is_bit_identical(mode):
    net = synth.grid_network(8, 8, 3, 250.0, 30, 3, "wave")
    dem = synth.merge_demands(synth.place_vehicles(net, 4000, seed=5, min_spacing=7.0, internal_frac=0.3),
                              synth.uniform_trips(net, 1500, 120, seed=6))
    params = dict(P, signal_mode=1, mp_interval=10) if mode == "maxpressure" else P
    one = oracle.Oracle(net, dem, params, n_windows=2)
    many = oracle.Oracle(net, dem, params, n_windows=2, threads=8)
    if mode == "learned":
        theta = (mlp.init(2) + np.random.default_rng(0).normal(scale=0.05, size=mlp.N_PARAMS)).astype(np.float32)
        for o in (one, many):
            o.set_lc_model(theta, 0.1)
    n_learn = 0
    for k in range(40):
        dbg = k % 5 == 0
        e1, d1 = one.step(debug=dbg)
        e2, d2 = many.step(debug=dbg)
        assert e1 == e2
        if dbg:
            for f in d1:
                assert np.array_equal(d1[f], d2[f]), (k, f)
            n_learn += int((d1["lc_learn"] == 1).sum())
    a, b = one.state(), many.state()
    for f in ("status", "lane", "x", "v", "rp", "t_arr"):
        assert np.array_equal(a[f], b[f]), f
    ma, mb = one.metrics(), many.metrics()
    for f in ("vsum", "vcnt"):
        assert np.array_equal(ma[f], mb[f]), f
    assert (ma["inserted"], ma["arrived"], ma["sum_tt"]) == (mb["inserted"], mb["arrived"], mb["sum_tt"])
    if mode == "maxpressure":
        assert np.array_equal(one.ctrl_state(), many.ctrl_state())
    if mode == "learned":
        assert n_learn > 100
