"""Input generators: seeded determinism and structural validity (CPU)."""
import numpy as np
import pytest

from paper_2405_12520_b300 import synth


def _check_net(net):
    L = net.n_lanes
    assert net.succ_off[0] == 0 and np.all(np.diff(net.succ_off) >= 0)
    internal = net.lane_edge < 0
    assert np.all(np.diff(net.succ_off)[internal] == 1)
    # left/right consistent within an edge
    for l in np.nonzero(net.lane_left >= 0)[0]:
        assert net.lane_right[net.lane_left[l]] == l and net.lane_edge[net.lane_left[l]] == net.lane_edge[l]
    # every internal lane's target is on its recorded exit edge
    tg = net.succ_lane[net.succ_off[:-1][internal]]
    assert np.all(net.lane_edge[tg] == net.succ_edge[net.succ_off[:-1][internal]])
    assert np.all(net.lane_len > 20.0)


def _check_routes(net, dem):
    E = net.n_edges
    pairs = set()
    for l in np.nonzero(net.lane_edge >= 0)[0]:
        for k in range(net.succ_off[l], net.succ_off[l + 1]):
            pairs.add((int(net.lane_edge[l]), int(net.succ_edge[k])))
    for i in range(dem.n):
        r = dem.route_edges[dem.route_off[i]:dem.route_off[i + 1]]
        assert r.size >= 1 and np.all((r >= 0) & (r < E))
        for a, b in zip(r[:-1], r[1:]):
            assert (int(a), int(b)) in pairs


@pytest.mark.parametrize("maker", [lambda: synth.grid_network(4, 4, 2, 200.0),
                                   lambda: synth.grid_network(5, 3, 3, 300.0, offset="wave"),
                                   lambda: synth.delaunay_network(60, box=2500.0, seed=2)])
def test_networks_are_valid(maker):
    _check_net(maker())


def test_generators_are_deterministic():
    a = synth.small_grid_workload(4)
    b = synth.small_grid_workload(4)
    for f in ("t_dep", "v0", "route_off", "route_edges"):
        np.testing.assert_array_equal(getattr(a[1], f), getattr(b[1], f))
    net = synth.grid_network(6, 6, 3, 200.0)
    p1 = synth.place_vehicles(net, 500, seed=9, internal_frac=0.3)
    p2 = synth.place_vehicles(net, 500, seed=9, internal_frac=0.3)
    for f in ("lane", "x", "v", "v0", "route_edges"):
        np.testing.assert_array_equal(getattr(p1, f), getattr(p2, f))


def test_trips_and_placements_are_consistent():
    net, dem = synth.small_grid_workload(2)
    _check_routes(net, dem)
    d2 = synth.place_vehicles(net, 400, seed=3, min_spacing=6.0, internal_frac=0.4)
    _check_routes(net, d2)
    assert d2.n == 400
    o = np.lexsort((d2.x, d2.lane))
    la, xa = d2.lane[o], d2.x[o]
    same = la[1:] == la[:-1]
    assert np.all((xa[1:] - xa[:-1])[same] >= 6.0 - 1e-4)
    assert np.all((d2.x > 0) & (d2.x <= net.lane_len[d2.lane]))


def test_union_offsets():
    sc = synth.batch_scenarios(3, seed=1, side=(3, 5), n_range=(30, 200))
    net, dem = synth.union([n for n, _ in sc], [d for _, d in sc])
    _check_net(net)
    _check_routes(net, dem)
    assert net.n_lanes == sum(n.n_lanes for n, _ in sc) and dem.n == sum(d.n for _, d in sc)


def test_pareto_trip_lengths():
    """Truncated Pareto(1.5, 1 km, 40 km) draws follow their CDF, and placed vehicles routed
    to the zone closest to a draw get heavy-tailed route lengths near the draws'."""
    rng = np.random.default_rng(5)
    ell = synth._pareto_lengths(rng, 200_000)
    assert ell.min() >= synth.PARETO_XM and ell.max() <= synth.PARETO_XMAX
    a, xm, xmax = synth.PARETO_ALPHA, synth.PARETO_XM, synth.PARETO_XMAX
    for q in (1500.0, 3000.0, 10000.0):   # truncated CDF at q vs the empirical fraction
        cdf = (1 - (xm / q) ** a) / (1 - (xm / xmax) ** a)
        assert abs(np.mean(ell <= q) - cdf) < 0.005
    net = synth.delaunay_network(1500, box=12000.0, seed=4)
    dem = synth.place_vehicles(net, 4000, seed=2, min_spacing=7.0, dest="pareto")
    _check_routes(net, dem)
    lens = np.array([net.edge_len[dem.route_edges[dem.route_off[i] + 1:dem.route_off[i + 1]]].sum()
                     for i in range(dem.n)])
    med = np.median(lens)
    assert 0.6 * xm * 2 ** (1 / a) < med < 1.6 * xm * 2 ** (1 / a)   # Pareto median 1.59 km
    assert 0.01 < np.mean(lens > 6000.0) < 0.15                      # the tail is there
    uni = synth.place_vehicles(net, 4000, seed=2, min_spacing=7.0, dest="uniform")
    ulens = np.array([net.edge_len[uni.route_edges[uni.route_off[i] + 1:uni.route_off[i + 1]]].sum()
                      for i in range(uni.n)])
    assert np.median(ulens) > 2 * med                                # uniform zones: long trips
