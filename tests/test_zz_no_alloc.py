"""ms_step_noalloc: the allocation-free step, checked against ms_step through the C ABI.

Some callers cannot call cudaMalloc once their simulation exists -- a loop that runs inside
a device-memory budget reserved in advance, or a component without the right to allocate on
a shared GPU.  For them ms_step_noalloc runs the same step with the lane scan's per-tile
status in one static device array instead of memory it would otherwise need.  These tests
step two identical simulations, one with each entry point, and require identical states
after each of two calls in a row, with the rule and with a learned lane-change model, and
the device's free memory unchanged across the allocation-free calls; a network larger than
the static array's limit must be refused with a clear error and leave the simulation as it
was (a later export still copies the current state).
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


@pytest.mark.parametrize("learned", [False, True])
def test_noalloc_step_matches_step_on_two_calls(learned):
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2405_12520_b300 import learned as lrn, synth
    net = synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave")   # ~6.6k lanes: 4 scan tiles
    dem = synth.merge_demands(synth.place_vehicles(net, 6000, seed=21, min_spacing=7.0, internal_frac=0.3),
                              synth.uniform_trips(net, 1500, 60, seed=22))
    p = synth.default_params()
    ref = _sim(net, dem, p)
    alt = _sim(net, dem, p)
    if learned:   # an untrained network decides (margin 0.05): many changes, all by the model
        theta = lrn.init_params(7)
        for s in (ref, alt):
            s.set_lc_model(theta, 0.05)
    # set-up: the first step of each simulation goes through ms_step (its graphs, the
    # kernels' first loads); from here on the allocation-free calls must not allocate
    for s in (ref, alt):
        s.step(1)
        s.sync()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for call in range(2):
        ref.step(25)
        alt.step_noalloc(25)
        alt.sync()
        assert torch.cuda.mem_get_info()[0] == free0, f"call {call}: device free memory changed"
        ref.sync()
        a, b = ref.read_state(), alt.read_state()
        assert a["t"] == b["t"] == 1 + 25 * (call + 1)
        for k in ("id", "lane", "x", "v", "route_idx", "t_arr", "trip_status"):
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"call {call}: {k}")
        ma, mb = ref.read_metrics(), alt.read_metrics()
        for k in ("inserted", "arrived", "sum_tt", "n_active", "err"):
            assert ma[k] == mb[k], (call, k)
        np.testing.assert_array_equal(ma["vsum"], mb["vsum"])
        np.testing.assert_array_equal(ma["vcnt"], mb["vcnt"])
        assert ma["err"] == 0
    if learned:
        sa, sb = ref.read_lc_stats(), alt.read_lc_stats()
        assert sa == sb and sa["candidates"] > 0 and sa["fallbacks"] < sa["candidates"]


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
    # the refused call changed nothing: an export now copies the state after that one step
    st = s.read_state()
    assert st["t"] == 1 and st["n_active"] == 1
    bufs = dict(x=torch.zeros(4, dtype=torch.float32, pin_memory=True),
                v=torch.zeros(4, dtype=torch.float32, pin_memory=True),
                lane=torch.full((4,), -7, dtype=torch.int32, pin_memory=True),
                vid=torch.full((4,), -7, dtype=torch.int32, pin_memory=True))
    s.read_state_async(**bufs)
    n, t = s.read_wait()
    assert (n, t) == (1, 1)
    assert bufs["x"][0].item() == st["x"][0] and bufs["v"][0].item() == st["v"][0]
    assert bufs["lane"][0].item() == st["lane"][0] and bufs["vid"][0].item() == st["id"][0]
