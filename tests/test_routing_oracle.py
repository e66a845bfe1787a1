"""Pins of the route planner's CPU reference (oracle/routing.py, reading R15) against
brute force and invariants that do not come from it: on small networks every simple path
is enumerated and the least-cost, then lexicographically smallest, one must be the route;
routes are lane-linked, end at the destination and cost exactly the Dijkstra distance;
trips between disjoint networks are unreachable."""
import numpy as np
import pytest

from paper_2405_12520_b300 import synth
import netkit
from oracle import routing


def _linked(net, e, f):
    for q in range(int(net.edge_nlanes[e])):
        l = int(net.edge_lane0[e]) + q
        if f in net.succ_edge[net.succ_off[l]:net.succ_off[l + 1]]:
            return True
    return False


def _brute_route(succ, c, o, d):
    """Every simple path from o to d, depth first with branch and bound (a partial path
    costing more than the best complete one is dropped): the least-cost path, then the
    lexicographically smallest by edge ids; None if d is unreachable."""
    import sys
    sys.setrecursionlimit(10000)
    best = [None, None]

    def dfs(e, cost, path, seen):
        if best[0] is not None and cost > best[0]:
            return
        if e == d:
            t = tuple(path)
            if best[0] is None or cost < best[0] or t < best[1]:
                best[0], best[1] = cost, t
            return
        for f in succ[e]:
            if f in seen:
                continue
            seen.add(f)
            path.append(f)
            dfs(f, cost + int(c[f]), path, seen)
            path.pop()
            seen.remove(f)

    dfs(o, 0, [o], {o})
    return best[1]


@pytest.mark.parametrize("kind", ["grid3", "delaunay"])
def test_routes_are_the_lexicographically_smallest_least_cost_paths(kind):
    net = synth.grid_network(3, 3, 2, 200.0, 30, 3, "zero") if kind == "grid3" else \
        synth.delaunay_network(9, box=900.0, seed=4)
    src, dst = routing.edge_graph(net)
    c = routing.edge_cost(net)
    succ = [sorted(dst[src == e].tolist()) for e in range(net.n_edges)]
    rng = np.random.default_rng(1)
    pairs = [(int(a), int(b)) for a, b in rng.integers(0, net.n_edges, size=(25, 2))]
    pairs.append((pairs[0][0], pairs[0][0]))   # origin = destination
    off, edges, bad = routing.routes(net, [p[0] for p in pairs], [p[1] for p in pairs])
    for i, (o, d) in enumerate(pairs):
        got = edges[off[i]:off[i + 1]].tolist()
        want = _brute_route(succ, c, o, d)
        assert (tuple(got) if got else None) == want, (o, d)


def test_routes_are_linked_and_cost_the_distance():
    net = synth.grid_network(12, 12, 3, 200.0, 30, 3, "wave")
    rng = np.random.default_rng(2)
    o = rng.integers(0, net.n_edges, 300)
    d = rng.integers(0, net.n_edges, 300)
    off, edges, bad = routing.routes(net, o, d)
    assert bad == 0
    c = routing.edge_cost(net)
    dist = routing.distances_to(net, np.unique(d))
    col = {int(x): k for k, x in enumerate(np.unique(d))}
    for i in range(300):
        r = edges[off[i]:off[i + 1]]
        assert r[0] == o[i] and r[-1] == d[i]
        assert all(_linked(net, int(a), int(b)) for a, b in zip(r[:-1], r[1:]))
        assert int(c[r[1:]].sum()) == dist[col[int(d[i])], o[i]]
    # the grid is uniform: a least-cost route enters exactly as many edges as the fewest
    # lane-linked hops
    assert np.all((c == c[0]))


def test_unreachable_trips_get_empty_routes():
    a = netkit.line(3, 300.0, 1)
    b = netkit.line(3, 300.0, 1)
    net, _ = synth.union([a, b], [netkit.vehicles([-1], [0.0], [0.0], [[0]]), netkit.vehicles([-1], [0.0], [0.0], [[0]])])
    off, edges, bad = routing.routes(net, [0, 0], [a.n_edges, 1])
    assert bad == 1
    assert off[1] - off[0] == 0 and off[2] - off[1] == 2


# ---------------------------------------------------------------------------------------
# gravity OD sampling (R16)
# ---------------------------------------------------------------------------------------

def _sm(z):
    import oracle
    return oracle.splitmix64(z)   # the published generator (pinned by its vector)


def test_gravity_origins_and_destinations_follow_the_weights():
    """gamma = 0: P(O = i) = A_i / sum A and P(D = j | O = i) = A_j / sum_{k != i} A_k; the
    sampled shares agree within 4 binomial standard deviations; departures are uniform."""
    net = synth.grid_network(6, 6, 1, 200.0, 30, 3, "zero")
    rng = np.random.default_rng(3)
    zones = rng.choice(net.n_edges, 6, replace=False)
    A = np.array([1.0, 2.0, 4.0, 0.5, 3.0, 1.5], np.float32)
    n = 6000
    o, d, t = routing.gravity_trips(net, zones, A, 0, n, 600, 77, _sm)
    zi = {int(z): k for k, z in enumerate(zones)}
    oi = np.array([zi[int(x)] for x in o])
    di = np.array([zi[int(x)] for x in d])
    assert np.all(oi != di)
    p_o = A / A.sum()
    f_o = np.bincount(oi, minlength=6) / n
    assert np.all(np.abs(f_o - p_o) <= 4 * np.sqrt(p_o * (1 - p_o) / n))
    sel = oi == 2   # destinations of zone 2's trips
    p_d = np.where(np.arange(6) == 2, 0.0, A) / (A.sum() - A[2])
    f_d = np.bincount(di[sel], minlength=6) / sel.sum()
    assert np.all(np.abs(f_d - p_d) <= 4 * np.sqrt(p_d * (1 - p_d) / sel.sum()) + 1e-12)
    assert t.min() >= 0 and t.max() < 600 and abs(t.mean() - 299.5) < 4 * 600 / np.sqrt(12 * n)


def test_gravity_decays_with_route_distance():
    """gamma = 2, equal attractions, on a one-lane line road: from the zone at one end the
    destination shares are proportional to 1 / (route distance)^2 (closed form over the
    zones' distances along the line)."""
    net = netkit.line(8, 500.0, 1)
    zones = np.array([0, 2, 4, 6], np.int64)   # eastbound edges 0 -> 1, 2 -> 3, ...
    A = np.ones(4, np.float32)
    n = 8000
    o, d, t = routing.gravity_trips(net, zones, A, 2, n, 60, 5, _sm)
    sel = o == 0
    dist = routing.distances_to(net, zones)[:, 0]   # cost from edge 0 to each zone edge
    # the route costs are the line's: zone k is 2k edges of 500 m further along
    np.testing.assert_array_equal(dist, [0.0, 1.0e6, 2.0e6, 3.0e6])
    w = np.zeros(4)
    w[1:] = 1.0 / dist[1:] ** 2
    p = w / w.sum()
    f = np.array([(d[sel] == z).mean() for z in zones])
    assert np.all(np.abs(f - p) <= 4 * np.sqrt(p * (1 - p) / sel.sum()) + 1e-12)


def test_radiation_weights_closed_form_on_a_line():
    """R18 with equal populations m: the k-th closest zone (no ties) has
    w = m^2 / ((m + (k-1) m)(2m + (k-1) m)) = 1 / (k (k + 1)); with unequal populations the
    weights from the line's end follow the formula with s = the populations in between."""
    net = netkit.line(10, 500.0, 1)
    zones = np.array([0, 2, 4, 6, 8], np.int64)
    cost = routing.distances_to(net, zones)[:, zones].T
    W = routing.radiation_weights(cost, np.full(5, 3.0, np.float32))
    k = np.arange(1, 5)
    np.testing.assert_allclose(W[0, 1:], 1.0 / (k * (k + 1)), rtol=1e-6)
    assert W[0, 0] == 0
    m = np.array([2.0, 1.0, 4.0, 0.5, 3.0], np.float32)
    W = routing.radiation_weights(cost, m)
    m64 = m.astype(np.float64)
    for j in range(1, 5):
        s = m64[1:j].sum()
        want = m64[0] * m64[j] / ((m64[0] + s) * (m64[0] + m64[j] + s))
        assert W[0, j] == pytest.approx(want, rel=1e-6)
    # ties: zones at equal distance count for neither; unreachable zones for nobody
    c = np.full((5, 5), 7.0)
    np.fill_diagonal(c, 0.0)
    c[0] = [0.0, 5.0, 5.0, 9.0, np.inf]
    mm = np.array([1.0, 2.0, 3.0, 4.0, 8.0], np.float32)
    W = routing.radiation_weights(c, mm)
    want = [0.0, 1 * 2 / ((1 + 0) * (1 + 2 + 0)), 1 * 3 / ((1 + 0) * (1 + 3 + 0)),
            1 * 4 / ((1 + 5) * (1 + 4 + 5)), 0.0]
    np.testing.assert_allclose(W[0], want, rtol=1e-6)


def test_radiation_sampling_follows_the_weights_and_is_scale_free():
    """Sampled origins follow the populations and the destinations of one origin the
    normalised weights (4 binomial standard deviations each); scaling every population by 2^3 (exact in float32) or every road length by 2
    (same distance ranks) draws exactly the same trips: the model has no free parameter and
    uses distances only through their order."""
    net = netkit.line(10, 500.0, 1)
    zones = np.array([0, 2, 4, 6, 8], np.int64)
    m = np.array([2.0, 1.0, 4.0, 0.5, 3.0], np.float32)
    n = 8000
    o, d, t = routing.radiation_trips(net, zones, m, n, 600, 31, _sm)
    cost = routing.distances_to(net, zones)[:, zones].T
    W = routing.radiation_weights(cost, m).astype(np.float64)
    sel = o == zones[0]
    p = W[0] / W[0].sum()
    f = np.array([(d[sel] == z).mean() for z in zones])
    assert np.all(np.abs(f - p) <= 4 * np.sqrt(p * (1 - p) / sel.sum()) + 1e-12)
    # origins: drawn as the gravity model draws them, by population share
    po = m.astype(np.float64) / m.sum()
    fo = np.array([(o == z).mean() for z in zones])
    assert np.all(np.abs(fo - po) <= 4 * np.sqrt(po * (1 - po) / n) + 1e-12)
    o2, d2, t2 = routing.radiation_trips(net, zones, m * np.float32(8.0), n, 600, 31, _sm)
    np.testing.assert_array_equal(d, d2)
    np.testing.assert_array_equal(o, o2)
    net2 = netkit.line(10, 1000.0, 1)
    o3, d3, t3 = routing.radiation_trips(net2, zones, m, n, 600, 31, _sm)
    np.testing.assert_array_equal(d, d3)
    np.testing.assert_array_equal(t, t3)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_radiation_weights_vectorised_form_equals_the_loop(seed):
    """radiation_weights_vec (used for thousands of zones) gives the zone-by-zone loop of
    R18 bit for bit: random populations (some equal), integer costs with many ties, zones
    unreachable from some origins, zero-cost neighbours."""
    rng = np.random.default_rng(seed)
    Z = 150
    m = rng.choice(np.array([1.0, 2.5, 7.0, 1e3, 3.3e4], np.float32), size=Z) * rng.integers(1, 4, Z).astype(np.float32)
    cost = rng.integers(0, 25, size=(Z, Z)).astype(np.float64) * 1000.0
    cost[rng.random((Z, Z)) < 0.1] = np.inf
    np.fill_diagonal(cost, 0.0)
    a = routing.radiation_weights(cost, m)
    b = routing.radiation_weights_vec(cost, m)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert (a > 0).sum() > Z * Z // 2


def test_departure_times_scale_with_the_span():
    """A departure time is the trip's uniform draw scaled to the span and rounded down, so
    the same seed with twice the span gives every trip 2 t or 2 t + 1 (gravity and
    radiation), and every time lies in [0, span)."""
    net = netkit.line(10, 500.0, 1)
    zones = np.array([0, 2, 4, 6, 8], np.int64)
    m = np.array([2.0, 1.0, 4.0, 0.5, 3.0], np.float32)
    n = 3000
    for draw in (lambda T: routing.gravity_trips(net, zones, m, 2, n, T, 5, _sm),
                 lambda T: routing.radiation_trips(net, zones, m, n, T, 5, _sm)):
        _, _, t1 = draw(600)
        _, _, t2 = draw(1200)
        assert t1.min() >= 0 and t1.max() < 600 and t2.max() < 1200
        assert np.all((t2 == 2 * t1) | (t2 == 2 * t1 + 1))
        assert (t2 == 2 * t1).any() and (t2 == 2 * t1 + 1).any()

