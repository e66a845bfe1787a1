"""GPU route planner (ms_route_trips, reading R15) against the CPU reference: identical
routes, edge for edge, for random trips on grid and Delaunay networks, across destination
batches, with unreachable trips; the routes drive a simulation as they are."""
import numpy as np
import pytest

from paper_2405_12520_b300 import synth
import netkit
from oracle import routing

pytestmark = pytest.mark.gpu


def _sim(net):
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_2405_12520_b300 import moss
    s = moss.Sim(synth.default_params())
    s.load_network(net)
    return s


@pytest.mark.parametrize("kind", ["grid12x3", "delaunay"])
def test_routes_match_the_reference(kind):
    net = synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave") if kind == "grid12x3" else \
        synth.delaunay_network(120, box=3000.0, seed=7)
    rng = np.random.default_rng(5)
    o = rng.integers(0, net.n_edges, 3000).astype(np.int32)
    d = rng.integers(0, net.n_edges, 3000).astype(np.int32)
    d[:10] = o[:10]   # origin = destination
    s = _sim(net)
    off, edges, bad = s.route_trips(o, d)
    ro, re, rb = routing.routes(net, o, d)
    assert bad == rb
    np.testing.assert_array_equal(off, ro)
    np.testing.assert_array_equal(edges, re)


def test_routes_across_destination_batches():
    """More distinct destinations (5000) than one batch holds (4096)."""
    net = synth.grid_network(40, 40, 1, 150.0, 30, 3, "zero")
    rng = np.random.default_rng(6)
    d = rng.permutation(net.n_edges)[:5000].astype(np.int32)
    d = np.concatenate([d, rng.choice(d, 1000)]).astype(np.int32)
    o = rng.integers(0, net.n_edges, d.size).astype(np.int32)
    s = _sim(net)
    off, edges, bad = s.route_trips(o, d)
    ro, re, rb = routing.routes(net, o, d)
    assert bad == rb == 0
    np.testing.assert_array_equal(off, ro)
    np.testing.assert_array_equal(edges, re)


def test_unreachable_trips_and_empty_input():
    a = netkit.line(3, 300.0, 1)
    b = netkit.line(3, 300.0, 2)
    net, _ = synth.union([a, b], [netkit.vehicles([-1], [0.0], [0.0], [[0]])] * 2)
    s = _sim(net)
    off, edges, bad = s.route_trips([0, 0, a.n_edges], [a.n_edges, 1, a.n_edges + 1])
    ro, re, rb = routing.routes(net, [0, 0, a.n_edges], [a.n_edges, 1, a.n_edges + 1])
    assert bad == rb == 1
    np.testing.assert_array_equal(off, ro)
    np.testing.assert_array_equal(edges, re)
    off, edges, bad = s.route_trips(np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert off.tolist() == [0] and edges.size == 0 and bad == 0


def test_gpu_routes_drive_a_simulation():
    from paper_2405_12520_b300 import moss
    net = synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave")
    rng = np.random.default_rng(8)
    n = 4000
    o = rng.integers(0, net.n_edges, n).astype(np.int32)
    d = rng.integers(0, net.n_edges, n).astype(np.int32)
    router = _sim(net)
    off, edges, bad = router.route_trips(o, d)
    assert bad == 0
    dem = synth.Demand(t_dep=rng.integers(0, 300, n).astype(np.int32), v0=np.full(n, 13.9, np.float32),
                       route_off=off, route_edges=edges, lane=np.full(n, -1, np.int32),
                       x=np.zeros(n, np.float32), v=np.zeros(n, np.float32))
    s = moss.Sim(synth.default_params(), n_windows=1)
    s.load_network(net)
    s.add_vehicles(dem)   # validates that consecutive route edges are lane-linked
    s.step(400)
    s.sync()
    m = s.read_metrics(lanes=False)
    assert m["err"] == 0 and m["inserted"] > 0.9 * n and m["arrived"] > 0


@pytest.mark.parametrize("gamma", [0, 2])
def test_gravity_sampling_matches_the_reference(gamma):
    """ms_sample_trips draws the same trips (origin, destination, departure) as the CPU
    reference, bit for bit, on a 12x12 grid with 64 zones."""
    import oracle
    net = synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave")
    rng = np.random.default_rng(9)
    zones = rng.choice(net.n_edges, 64, replace=False).astype(np.int32)
    A = rng.lognormal(0.0, 1.0, 64).astype(np.float32)
    s = _sim(net)
    o, d, t = s.sample_trips(zones, A, gamma, 20000, 900, 1234)
    ro, rd, rt = routing.gravity_trips(net, zones, A, gamma, 20000, 900, 1234, oracle.splitmix64)
    np.testing.assert_array_equal(o, ro)
    np.testing.assert_array_equal(d, rd)
    np.testing.assert_array_equal(t, rt)


def test_gravity_sampling_with_an_isolated_zone_and_into_a_simulation():
    import oracle
    from paper_2405_12520_b300 import moss
    a = synth.grid_network(6, 6, 2, 200.0, 30, 3, "zero")
    b = netkit.line(3, 300.0, 1)
    net, _ = synth.union([a, b], [netkit.vehicles([-1], [0.0], [0.0], [[0]])] * 2)
    zones = np.array([0, 5, 17, 40, a.n_edges], np.int32)   # the last zone is on the other network
    A = np.array([1.0, 2.0, 1.0, 3.0, 5.0], np.float32)
    s = _sim(net)
    o, d, t = s.sample_trips(zones, A, 1, 3000, 300, 99)
    ro, rd, rt = routing.gravity_trips(net, zones, A, 1, 3000, 300, 99, oracle.splitmix64)
    np.testing.assert_array_equal(o, ro)
    np.testing.assert_array_equal(d, rd)
    np.testing.assert_array_equal(t, rt)
    home = o == a.n_edges
    assert home.any() and np.all(d[home] == a.n_edges)   # reaches no other zone: stays
    off, edges, bad = s.route_trips(o, d)
    assert bad == 0
    dem = synth.Demand(t_dep=t, v0=np.full(o.size, 13.9, np.float32), route_off=off, route_edges=edges,
                       lane=np.full(o.size, -1, np.int32), x=np.zeros(o.size, np.float32),
                       v=np.zeros(o.size, np.float32))
    sim = moss.Sim(synth.default_params())
    sim.load_network(net)
    sim.add_vehicles(dem)
    sim.step(600)
    sim.sync()
    assert sim.read_metrics(lanes=False)["err"] == 0


@pytest.mark.parametrize("kind,n_zones", [("grid", 64), ("delaunay", 300), ("grid", 4096)])
def test_radiation_sampling_matches_the_reference(kind, n_zones):
    """ms_sample_trips_radiation draws the same trips as the CPU reference (R18), bit for
    bit: a 12x12 grid (many equal route costs, so tie groups matter), an irregular network,
    and the 4096-zone maximum (a full-width bitonic sort per origin)."""
    import oracle
    if kind == "grid":
        net = synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave") if n_zones <= 64 else \
            synth.grid_network(40, 40, 2, 200.0, 30, 3, "wave")
    else:
        net = synth.delaunay_network(400, box=8000.0, seed=5)
    rng = np.random.default_rng(n_zones)
    zones = rng.choice(net.n_edges, n_zones, replace=False).astype(np.int32)
    m = rng.lognormal(0.0, 1.0, n_zones).astype(np.float32)
    s = _sim(net)
    n = 20000 if n_zones <= 300 else 5000
    o, d, t = s.sample_trips_radiation(zones, m, n, 900, 4321)
    ro, rd, rt = routing.radiation_trips(net, zones, m, n, 900, 4321, oracle.splitmix64)
    np.testing.assert_array_equal(o, ro)
    np.testing.assert_array_equal(d, rd)
    np.testing.assert_array_equal(t, rt)
    assert len(np.unique(d)) > min(20, n_zones // 4)
