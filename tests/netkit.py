"""Small hand-built networks and placements for pin tests (inputs only, no model code)."""
from __future__ import annotations

import numpy as np

from paper_2405_12520_b300 import synth


def ring(edge_len: float = 200.0, n_lanes: int = 1) -> synth.Network:
    """Two nodes, one road each way: A->B, junction at B (U-turn is the only exit), B->A,
    junction at A.  A closed loop of two edge lanes and two internal lanes."""
    xy = np.array([[0.0, 0.0], [edge_len, 0.0]])
    return synth._assemble(xy, np.array([0, 1]), np.array([1, 0]), np.array([edge_len, edge_len]),
                           np.array([n_lanes, n_lanes]), [], 30, 3, 0, name="ring")


def line(n_nodes: int = 3, edge_len: float = 300.0, n_lanes: int = 2) -> synth.Network:
    """Straight road of n_nodes-1 links each way, no signals."""
    xy = np.stack([np.arange(n_nodes) * edge_len, np.zeros(n_nodes)], 1)
    ef = np.concatenate([np.arange(n_nodes - 1), np.arange(1, n_nodes)])
    et = np.concatenate([np.arange(1, n_nodes), np.arange(n_nodes - 1)])
    return synth._assemble(xy, ef, et, np.full(ef.shape[0], edge_len), np.full(ef.shape[0], n_lanes),
                           [], 30, 3, 0, name="line")


def ring_path(net: synth.Network):
    """Lane sequence around the ring starting at A->B lane 0, with cumulative starts."""
    e0 = 0
    l0 = int(net.edge_lane0[e0])
    seq = []
    cur = l0
    for _ in range(4):
        seq.append(cur)
        s0 = net.succ_off[cur]
        cur = int(net.succ_lane[s0])
    lens = net.lane_len[seq].astype(np.float64)
    starts = np.concatenate([[0.0], np.cumsum(lens)[:-1]])
    return seq, starts, float(lens.sum())


def ring_demand(net: synth.Network, u_front: np.ndarray, v: np.ndarray, v0: float,
                n_laps: int = 400) -> synth.Demand:
    """Vehicles on the single-lane ring with fronts at ring coordinates u_front (ring lane
    sequence from ring_path), all going round for n_laps laps."""
    seq, starts, total = ring_path(net)
    n = u_front.shape[0]
    lane = np.empty(n, np.int64)
    x = np.empty(n)
    first_edge = np.empty(n, np.int64)
    for i, u in enumerate(np.mod(u_front, total)):
        k = int(np.searchsorted(starts, u, side="right") - 1)
        xx = u - starts[k]
        if xx <= 0.0 and k > 0:   # a front exactly on a boundary belongs to the earlier lane
            k -= 1
            xx = u - starts[k]
        if xx <= 0.0 and k == 0:
            k = 3
            xx = u + total - starts[3]
        lane[i] = seq[k]
        x[i] = xx
        # route starts at the edge of the lane (edge lane) or the approach edge (internal)
        first_edge[i] = 0 if k in (0, 1) else 1
    offs = np.arange(n + 1, dtype=np.int64) * (2 * n_laps)
    edges = np.empty(int(offs[-1]), np.int32)
    for i in range(n):
        e = first_edge[i]
        edges[offs[i]:offs[i + 1]] = np.tile([e, 1 - e], n_laps)
    return synth._pack(np.zeros(n, np.int32), np.full(n, v0), offs, edges, lane=lane, x=x, v=v)


def single(net: synth.Network, lane: int, x: float, v: float, route, v0: float = 13.9) -> synth.Demand:
    r = np.asarray(route, np.int32)
    return synth._pack(np.zeros(1, np.int32), np.full(1, v0), np.array([0, r.shape[0]]), r,
                       lane=np.array([lane]), x=np.array([x]), v=np.array([v]))


def vehicles(lanes, xs, vs, routes, v0=13.9, t_dep=None) -> synth.Demand:
    n = len(lanes)
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum([len(r) for r in routes])
    edges = np.concatenate([np.asarray(r, np.int32) for r in routes]) if n else np.zeros(0, np.int32)
    v0a = np.full(n, v0) if np.isscalar(v0) else np.asarray(v0)
    td = np.zeros(n, np.int32) if t_dep is None else np.asarray(t_dep, np.int32)
    return synth._pack(td, v0a, offs, edges, lane=np.asarray(lanes), x=np.asarray(xs, np.float64),
                       v=np.asarray(vs, np.float64))


def closable_links(net, dem, rng, frac):
    return synth.closable_link_masks(net, dem, rng, frac)
