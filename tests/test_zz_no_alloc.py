"""ms_step_noalloc: the allocation-free step, checked against ms_step through the C ABI.

Some callers cannot call cudaMalloc once their simulation exists -- a loop that runs inside
a device-memory budget reserved in advance, or a component without the right to allocate on
a shared GPU.  For them ms_step_noalloc runs the same step with the lane scan's per-tile
status in one static device array instead of memory it would otherwise need.  These tests
step two identical simulations, one with each entry point, and require identical states
after each of two calls in a row; a network larger than the static array's limit must be
refused with a clear error.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _sim(net, dem, params):
    from paper_2405_12520_b300 import moss
    s = moss.Sim(params, n_windows=2)
    s.load_network(net)
    s.add_vehicles(dem)
    return s


def test_noalloc_step_matches_step_on_two_calls():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2405_12520_b300 import synth
    net = synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave")   # ~6.6k lanes: 4 scan tiles
    dem = synth.merge_demands(synth.place_vehicles(net, 6000, seed=21, min_spacing=7.0, internal_frac=0.3),
                              synth.uniform_trips(net, 1500, 60, seed=22))
    p = synth.default_params()
    ref = _sim(net, dem, p)
    alt = _sim(net, dem, p)
    for call in range(2):
        ref.step(25)
        alt.step_noalloc(25)
        ref.sync()
        alt.sync()
        a, b = ref.read_state(), alt.read_state()
        assert a["t"] == b["t"] == 25 * (call + 1)
        for k in ("id", "lane", "x", "v", "route_idx", "t_arr", "trip_status"):
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"call {call}: {k}")
        ma, mb = ref.read_metrics(), alt.read_metrics()
        for k in ("inserted", "arrived", "sum_tt", "n_active", "err"):
            assert ma[k] == mb[k], (call, k)
        np.testing.assert_array_equal(ma["vsum"], mb["vsum"])
        np.testing.assert_array_equal(ma["vcnt"], mb["vcnt"])
        assert ma["err"] == 0


def test_noalloc_step_refuses_networks_beyond_its_limit():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2405_12520_b300 import moss, synth
    lib_max = 3072 * 1024   # MS_NOALLOC_MAX_TILES * MS_NOALLOC_TILE_LANES
    E = lib_max + 1         # one-lane roads, no junctions: just over the limit
    z = np.zeros(E, np.int32)
    net = synth.Network(
        node_xy=np.zeros((1, 2)), edge_from=z, edge_to=z, edge_len=np.full(E, 30.0, np.float32),
        edge_nlanes=np.ones(E, np.int32), edge_lane0=np.arange(E, dtype=np.int32),
        lane_len=np.full(E, 30.0, np.float32), lane_edge=np.arange(E, dtype=np.int32), lane_index=z,
        lane_left=np.full(E, -1, np.int32), lane_right=np.full(E, -1, np.int32),
        succ_off=np.zeros(E + 1, np.int32), succ_lane=np.zeros(0, np.int32), succ_edge=np.zeros(0, np.int32),
        lane_ctrl=np.full(E, -1, np.int32), lane_group=z, ctrl_node=np.zeros(0, np.int32),
        ctrl_offset=np.zeros(0, np.int32), ctrl_green=np.zeros(0, np.int32), ctrl_yellow=np.zeros(0, np.int32),
        ctrl_nphase=np.zeros(0, np.int32))
    dem = synth._pack(np.zeros(1, np.int32), np.full(1, 13.9), np.array([0, 1]), np.array([0], np.int32))
    s = _sim(net, dem, synth.default_params())
    with pytest.raises(moss.MossError) as e:
        s.step_noalloc(1)
    assert e.value.code == moss.MS_ERR_CAPACITY
    assert "at most" in str(e.value)
    s.step(1)   # the allocating entry point has no such limit
    s.sync()
