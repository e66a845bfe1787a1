"""Batched scenarios (disjoint union in one step launch sequence) and the autotuner.

The batch must equal (bit-exact) the same union loaded as one network, and every scenario
simulated on its own (with its trip-id base so the lane-change gate draws the same
numbers); single steps of the union match the FP64 oracle like any network."""
import numpy as np
import pytest

import oracle
import parity
from paper_2405_12520_b300 import learned, moss, synth

pytestmark = pytest.mark.gpu
P = synth.default_params()


def _scen():
    return synth.batch_scenarios(7, seed=3, side=(3, 8), n_range=(60, 1500))


@pytest.mark.parametrize("learned_model", [False, True])
def test_batch_equals_union_and_standalone(learned_model):
    """learned_model: an untrained surrogate with margin 0.05 decides most discretionary
    changes on every side (each network row depends on its own inputs only, so the learned
    decisions do not depend on which other candidates share a tensor-core tile)."""
    sc = _scen()
    nets, dems = [n for n, _ in sc], [d for _, d in sc]
    b = moss.Sim(P, n_windows=1)
    b.load_network_batch(nets)
    b.add_vehicles_batch(dems)
    lane_off, trip_off = b.batch_offsets()
    unet, udem = synth.union(nets, dems)
    assert lane_off[-1] == unet.n_lanes and trip_off[-1] == udem.n
    u = parity.gpu_sim(unet, udem, P, debug=False)
    solo = []
    for k, (n, d) in enumerate(sc):
        s = moss.Sim(P, id_base=int(trip_off[k]))
        s.load_network(n)
        s.add_vehicles(d)
        solo.append(s)
    if learned_model:
        theta = learned.init_params(7)
        for s in [b, u] + solo:
            s.set_lc_model(theta, 0.05)
    for rnd in range(3):
        b.step(40)
        u.step(40)
        for s in solo:
            s.step(40)
        sb, su = b.read_state(), u.read_state()
        for f in ("id", "lane", "x", "v", "route_idx", "t_arr"):
            np.testing.assert_array_equal(sb[f], su[f])
        for k, s in enumerate(solo):
            ss = s.read_state()
            m = (sb["id"] >= trip_off[k]) & (sb["id"] < trip_off[k + 1])
            np.testing.assert_array_equal(sb["id"][m] - trip_off[k], ss["id"])
            np.testing.assert_array_equal(sb["lane"][m] - lane_off[k], ss["lane"])
            np.testing.assert_array_equal(sb["x"][m], ss["x"])
            np.testing.assert_array_equal(sb["v"][m], ss["v"])
            np.testing.assert_array_equal(sb["t_arr"][trip_off[k]:trip_off[k + 1]], ss["t_arr"])
    assert b.read_metrics(lanes=False)["err"] == 0
    if learned_model:
        st = b.read_lc_stats()
        assert st["candidates"] > 100 and st["fallbacks"] < st["candidates"]


def test_batch_single_steps_match_oracle():
    sc = _scen()
    unet, udem = synth.union([n for n, _ in sc], [d for _, d in sc])
    sim = parity.gpu_sim(unet, udem, P)
    orc = oracle.Oracle(unet, udem, P)
    rep = []
    for _ in range(6):
        _, gd, gs, od, os_ = parity.step_pair(sim, orc)
        parity.compare_step(gd, gs, od, os_, udem.n, report=rep)
    assert sum(r["compared"] for r in rep) > 0.9 * sum(r["active"] for r in rep)


def test_autotune_keeps_results_and_picks_a_candidate():
    sc = _scen()
    nets, dems = [n for n, _ in sc], [d for _, d in sc]
    a = moss.Sim(P)
    a.load_network_batch(nets)
    a.add_vehicles_batch(dems)
    b = moss.Sim(P)
    b.load_network_batch(nets)
    b.add_vehicles_batch(dems)
    a.step(20)
    b.step(20)
    ms, cfg = b.autotune(trial_steps=3)
    assert ms > 0 and cfg[0] in (128, 256, 512) and cfg[1] in (1, 2, 4) and cfg[2] in (1, 2, 4)
    assert cfg[3] in (128, 256, 512) and cfg[4] in (128, 256, 512) and cfg[5] in (1, 2)
    sa, sb = a.read_state(), b.read_state()
    assert sa["t"] == sb["t"] == 20   # the trials left no trace
    a.step(60)
    b.step(60)
    sa, sb = a.read_state(), b.read_state()
    for f in ("id", "lane", "x", "v", "route_idx", "t_arr"):
        np.testing.assert_array_equal(sa[f], sb[f])
