"""Seeded synthetic inputs: lane-level road networks, signal plans and travel demand.

This module builds the *inputs* of the per-step vehicle update and nothing else: node
and edge geometry, lane connectivity through junctions (the map builder's job, Sec. III-C
"Map Builder"), fixed-time signal plans, trips with host-computed shortest-path routes (the
OD-to-demand converter's job, Sec. III-C "Converter from OD matrix to travel demand") and
pre-placed vehicle states for steady-state workloads.  It holds none of the simulation
arithmetic (signal state at a time, sensing, car following, lane changing, motion); both
the CPU oracle and the CUDA path consume what it returns and derive their own tables.

The workloads stand in for the paper's evaluation networks (Sec. IV-A: six real cities and
nine grids with 16 to 93,564 grids, up to about 2.46M vehicles), which are not available.

All arrays are numpy; every generator takes an explicit seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Lane id layout: lanes of edge e are edge_lane0[e] + idx (idx 0 = rightmost lane), all
# edge lanes first, then junction-internal lanes grouped by junction node.

INTERNAL_MIN_LEN = 21.0  # m; longer than v_max*dt so no vehicle crosses one in a step
MIN_EDGE_LEN = 25.0      # m; same reason for edge lanes


@dataclass
class Network:
    node_xy: np.ndarray      # [V,2] float64, metres
    edge_from: np.ndarray    # [E] int32
    edge_to: np.ndarray      # [E] int32
    edge_len: np.ndarray     # [E] float32
    edge_nlanes: np.ndarray  # [E] int32
    edge_lane0: np.ndarray   # [E] int32
    lane_len: np.ndarray     # [Λ] float32
    lane_edge: np.ndarray    # [Λ] int32, -1 for junction-internal lanes
    lane_index: np.ndarray   # [Λ] int32, 0 = rightmost (0 for internal lanes)
    lane_left: np.ndarray    # [Λ] int32, -1 none
    lane_right: np.ndarray   # [Λ] int32, -1 none
    succ_off: np.ndarray     # [Λ+1] int32 CSR
    succ_lane: np.ndarray    # [S] int32: internal lane (edge lanes) / target lane (internal)
    succ_edge: np.ndarray    # [S] int32: exit edge reached through that successor
    lane_ctrl: np.ndarray    # [Λ] int32, -1 = no signal at the lane end
    lane_group: np.ndarray   # [Λ] int32 phase group served (valid when ctrl >= 0)
    ctrl_node: np.ndarray    # [C] int32
    ctrl_offset: np.ndarray  # [C] int32, s
    ctrl_green: np.ndarray   # [C] int32, s
    ctrl_yellow: np.ndarray  # [C] int32, s
    ctrl_nphase: np.ndarray  # [C] int32
    name: str = ""
    grid_shape: tuple | None = None   # (nx, ny) for grids

    @property
    def n_lanes(self) -> int:
        return int(self.lane_len.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.edge_len.shape[0])

    @property
    def n_ctrl(self) -> int:
        return int(self.ctrl_node.shape[0])

    @property
    def n_edge_lanes(self) -> int:
        return int(self.edge_nlanes.sum())


@dataclass
class Demand:
    """Trips.  Trip i departs at t_dep[i] on route_edges[route_off[i]:route_off[i+1]].

    If lane[i] >= 0 the vehicle is already on the network at (lane[i], x[i], v[i]) at
    t = 0 (steady-state workloads); its route then starts at the edge it is on, or, for a
    junction-internal lane, at the approach edge the internal lane leaves from.
    """
    t_dep: np.ndarray        # [n] int32
    v0: np.ndarray           # [n] float32 desired speed
    route_off: np.ndarray    # [n+1] int64
    route_edges: np.ndarray  # [R] int32
    lane: np.ndarray         # [n] int32
    x: np.ndarray            # [n] float32
    v: np.ndarray            # [n] float32

    @property
    def n(self) -> int:
        return int(self.t_dep.shape[0])


def default_params(**over) -> dict:
    """Model parameters of the small plain-method configuration (IDM and MOBIL values as
    the workload fixes them; readings for the values the paper leaves open)."""
    p = dict(dt=1.0, veh_len=5.0,
             idm_a=2.0, idm_b=4.5, idm_T=1.5, idm_s0=2.0,
             mobil_p=0.1, mobil_th=0.2, mobil_bsafe=4.0,
             p_lc=1.0, a_min=-9.0, v_max=20.0, d_look=200.0,
             x_lc_min=25.0, x_lc_end=20.0, window=300, seed=1,
             mobil_th_jitter=0.0)   # R12 threshold jitter (a randomized-MOBIL variant), off
    p.update(over)
    return p


# ----------------------------------------------------------------------------------------
# junction builder (lane connectivity + signal groups), shared by all network shapes
# ----------------------------------------------------------------------------------------

def _turn_angle(din, dout):
    return math.atan2(din[0] * dout[1] - din[1] * dout[0], din[0] * dout[0] + din[1] * dout[1])


def _assemble(node_xy, edge_from, edge_to, edge_len, edge_nlanes, signal_nodes,
              green, yellow, offset, name, grid_shape=None) -> Network:
    V = node_xy.shape[0]
    E = edge_from.shape[0]
    edge_lane0 = np.zeros(E, np.int64)
    edge_lane0[1:] = np.cumsum(edge_nlanes)[:-1]
    n_edge_lanes = int(edge_nlanes.sum())
    lane_edge = np.repeat(np.arange(E), edge_nlanes)
    lane_index = np.arange(n_edge_lanes) - edge_lane0[lane_edge]
    lane_left = np.where(lane_index + 1 < edge_nlanes[lane_edge], np.arange(n_edge_lanes) + 1, -1)
    lane_right = np.where(lane_index > 0, np.arange(n_edge_lanes) - 1, -1)

    order_in = np.argsort(edge_to, kind="stable")
    order_out = np.argsort(edge_from, kind="stable")
    in_off = np.searchsorted(edge_to[order_in], np.arange(V + 1))
    out_off = np.searchsorted(edge_from[order_out], np.arange(V + 1))

    # successors of edge lanes: list of (internal lane, exit edge); internal lane records
    succ_of_edge_lane = [[] for _ in range(n_edge_lanes)]
    int_from, int_to, int_edge, int_len = [], [], [], []
    n_int = 0
    for n in range(V):
        ins = order_in[in_off[n]:in_off[n + 1]]
        outs = order_out[out_off[n]:out_off[n + 1]]
        for a in ins:
            u = edge_from[a]
            din = node_xy[n] - node_xy[u]
            exits = [x for x in outs if edge_to[x] != u]
            if not exits:
                exits = list(outs)  # dead end: the U-turn is the only way on
            th = [_turn_angle(din, node_xy[edge_to[x]] - node_xy[n]) for x in exits]
            srt = np.argsort(th, kind="stable")  # rightmost exit first
            k = int(edge_nlanes[a])
            m = len(exits)
            for j, s in enumerate(srt):
                x = exits[s]
                lo = (j * k) // m
                hi = -(-((j + 1) * k) // m) - 1
                hi = max(hi, lo)
                c = hi - lo + 1
                ne = int(edge_nlanes[x])
                length = INTERNAL_MIN_LEN + 9.0 * abs(th[s]) / math.pi
                for q in range(lo, hi + 1):
                    uu = q - lo
                    tt = (ne - c + uu) if (j == m - 1 and m > 1) else uu
                    tt = min(max(tt, 0), ne - 1)
                    src = int(edge_lane0[a] + q)
                    # fan-out: one internal lane to every lane of the exit edge, the natural
                    # target (right-aligned, left-aligned for the leftmost exit) first, then by
                    # distance from it (lower index first on ties)
                    for t2 in sorted(range(ne), key=lambda z: (abs(z - tt), z)):
                        dst = int(edge_lane0[x] + t2)
                        lid = n_edge_lanes + n_int
                        n_int += 1
                        int_from.append(src)
                        int_to.append(dst)
                        int_edge.append(int(x))
                        int_len.append(length)
                        succ_of_edge_lane[src].append((lid, int(x)))

    L = n_edge_lanes + n_int
    lane_len = np.concatenate([edge_len[lane_edge], np.asarray(int_len, np.float64)]).astype(np.float32)
    succ_cnt = np.zeros(L, np.int64)
    succ_cnt[:n_edge_lanes] = [len(s) for s in succ_of_edge_lane]
    succ_cnt[n_edge_lanes:] = 1
    succ_off = np.zeros(L + 1, np.int64)
    succ_off[1:] = np.cumsum(succ_cnt)
    succ_lane = np.empty(int(succ_off[-1]), np.int64)
    succ_edge = np.empty(int(succ_off[-1]), np.int64)
    pos = 0
    for s in succ_of_edge_lane:
        for (lid, x) in s:
            succ_lane[pos] = lid
            succ_edge[pos] = x
            pos += 1
    succ_lane[pos:] = np.asarray(int_to, np.int64)
    succ_edge[pos:] = np.asarray(int_edge, np.int64)

    # fixed-time signals: approaches sorted by heading, P = ceil(deg/2) phases, approach a
    # served in phase (rank mod P)
    lane_ctrl = np.full(L, -1, np.int64)
    lane_group = np.zeros(L, np.int64)
    ctrl_node, ctrl_nphase = [], []
    for n in signal_nodes:
        ins = order_in[in_off[n]:in_off[n + 1]]
        if len(ins) < 3:
            continue
        c = len(ctrl_node)
        ang = [math.atan2(*(node_xy[n] - node_xy[edge_from[a]])[::-1]) for a in ins]
        P = (len(ins) + 1) // 2
        for r, s in enumerate(np.argsort(ang, kind="stable")):
            a = ins[s]
            l0 = int(edge_lane0[a])
            lane_ctrl[l0:l0 + int(edge_nlanes[a])] = c
            lane_group[l0:l0 + int(edge_nlanes[a])] = r % P
        ctrl_node.append(n)
        ctrl_nphase.append(P)
    C = len(ctrl_node)
    ctrl_node = np.asarray(ctrl_node, np.int64)
    ctrl_nphase = np.asarray(ctrl_nphase, np.int64)
    g = np.broadcast_to(np.asarray(green(ctrl_node) if callable(green) else green), (C,))
    y = np.broadcast_to(np.asarray(yellow), (C,))
    cyc = ctrl_nphase * (g + y)
    off = np.asarray(offset(ctrl_node, cyc) if callable(offset) else np.broadcast_to(offset, (C,)))
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    return Network(
        node_xy=node_xy.astype(np.float64), edge_from=i32(edge_from), edge_to=i32(edge_to),
        edge_len=edge_len.astype(np.float32), edge_nlanes=i32(edge_nlanes), edge_lane0=i32(edge_lane0),
        lane_len=lane_len, lane_edge=i32(np.concatenate([lane_edge, np.full(n_int, -1)])),
        lane_index=i32(np.concatenate([lane_index, np.zeros(n_int, np.int64)])),
        lane_left=i32(np.concatenate([lane_left, np.full(n_int, -1)])),
        lane_right=i32(np.concatenate([lane_right, np.full(n_int, -1)])),
        succ_off=i32(succ_off), succ_lane=i32(succ_lane), succ_edge=i32(succ_edge),
        lane_ctrl=i32(lane_ctrl), lane_group=i32(lane_group),
        ctrl_node=i32(ctrl_node), ctrl_offset=i32(np.mod(off, np.maximum(cyc, 1))),
        ctrl_green=i32(g), ctrl_yellow=i32(y), ctrl_nphase=i32(ctrl_nphase),
        name=name, grid_shape=grid_shape)


def grid_network(nx: int, ny: int, n_lanes: int = 2, link_len: float = 200.0,
                 green: int = 30, yellow: int = 3, offset: str = "zero",
                 seed: int = 0, signals: bool = True) -> Network:
    """nx*ny signalised grid, bidirectional links of n_lanes lanes.

    offset: "zero" (all controllers in phase), "wave" ((i+j)*22 s, a green wave at about
    300 m / 13.9 m/s), or "random" (uniform in the cycle, from seed; green then drawn
    U{20..40} per node)."""
    assert link_len >= MIN_EDGE_LEN
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    node_xy = np.stack([ii.ravel() * link_len, jj.ravel() * link_len], 1).astype(np.float64)
    ef, et = [], []
    for j in range(ny):
        for i in range(nx):
            n = j * nx + i
            for di, dj in ((1, 0), (0, 1), (-1, 0), (0, -1)):
                a, b = i + di, j + dj
                if 0 <= a < nx and 0 <= b < ny:
                    ef.append(n)
                    et.append(b * nx + a)
    ef = np.asarray(ef, np.int64)
    et = np.asarray(et, np.int64)
    E = ef.shape[0]
    rng = np.random.default_rng(seed)
    g: object = green
    if offset == "zero":
        off: object = 0
    elif offset == "wave":
        off = lambda nodes, cyc: ((nodes % nx) + (nodes // nx)) * 22
    elif offset == "random":
        gg = rng.integers(20, 41, size=nx * ny)
        g = lambda nodes: gg[nodes]
        uu = rng.random(nx * ny)
        off = lambda nodes, cyc: np.floor(uu[nodes] * cyc).astype(np.int64)
    else:
        raise ValueError(offset)
    sig_nodes = range(nx * ny) if signals else []
    return _assemble(node_xy, ef, et, np.full(E, link_len), np.full(E, n_lanes, np.int64),
                     sig_nodes, g, yellow, off, name=f"grid{nx}x{ny}x{n_lanes}", grid_shape=(nx, ny))


def delaunay_network(n_pts: int, box: float = 30000.0, seed: int = 0, r_min: float = 30.0,
                     green: int = 30, yellow: int = 3) -> Network:
    """Random planar network: Delaunay triangulation of n_pts points (hard-core distance
    r_min) in a box x box m square; every triangulation edge is a road in both directions;
    1-4 lanes per road by length quartile (shortest quarter 1 lane, longest 4); signals
    at nodes with 3 or more approaches."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    cell = r_min / math.sqrt(2.0)
    ncell = int(math.ceil(box / cell))
    occ = {}
    pts = []
    while len(pts) < n_pts:
        cand = rng.random((n_pts, 2)) * box
        for p in cand:
            ci, cj = int(p[0] // cell), int(p[1] // cell)
            ok = True
            for a in range(ci - 2, ci + 3):
                for b in range(cj - 2, cj + 3):
                    q = occ.get((a, b))
                    if q is not None and (q[0] - p[0]) ** 2 + (q[1] - p[1]) ** 2 < r_min * r_min:
                        ok = False
                        break
                if not ok:
                    break
            if ok:
                occ[(ci, cj)] = p
                pts.append(p)
                if len(pts) == n_pts:
                    break
    del ncell
    xy = np.asarray(pts, np.float64)
    tri = Delaunay(xy)
    s = tri.simplices
    und = np.concatenate([s[:, [0, 1]], s[:, [1, 2]], s[:, [2, 0]]])
    und = np.sort(und, 1)
    und = np.unique(und, axis=0)
    ef = np.concatenate([und[:, 0], und[:, 1]])
    et = np.concatenate([und[:, 1], und[:, 0]])
    o = np.lexsort((et, ef))
    ef, et = ef[o], et[o]
    el = np.linalg.norm(xy[et] - xy[ef], axis=1)
    q = np.quantile(el, [0.25, 0.5, 0.75])
    nl = 1 + (el > q[0]).astype(np.int64) + (el > q[1]) + (el > q[2])
    return _assemble(xy, ef, et, el, nl, range(xy.shape[0]), green, yellow, 0,
                     name=f"delaunay{n_pts}")


# ----------------------------------------------------------------------------------------
# routing (host-side shortest paths; demand conversion, not the simulation)
# ----------------------------------------------------------------------------------------

def _edge_lookup(net: Network):
    V = net.node_xy.shape[0]
    key = net.edge_from.astype(np.int64) * V + net.edge_to
    o = np.argsort(key)
    return key[o], o, V


def _eid(lut, a, b):
    keys, o, V = lut
    k = a.astype(np.int64) * V + b
    p = np.searchsorted(keys, k)
    p = np.minimum(p, keys.shape[0] - 1)
    ok = keys[p] == k
    return np.where(ok, o[p], -1)


def _grid_routes(net: Network, start_edge: np.ndarray, start_node: np.ndarray, dest: np.ndarray):
    """Shortest (Manhattan) routes on a grid: the x moves first, unless the first x move
    would be a U-turn back along start_edge, then the y moves first.  Returns
    (route_off, route_edges, ok) where routes begin with start_edge if >= 0."""
    nx, ny = net.grid_shape
    n = dest.shape[0]
    ci, cj = start_node % nx, start_node // nx
    di, dj = dest % nx, dest // nx
    dx, dy = di - ci, dj - cj
    prev = np.where(start_edge >= 0, net.edge_from[np.maximum(start_edge, 0)], -1)
    # first hop under x-first
    fx = np.where(dx != 0, start_node + np.sign(dx), np.where(dy != 0, start_node + np.sign(dy) * nx, -1))
    yfirst = (fx == prev) & (fx >= 0)
    fy = np.where(dy != 0, start_node + np.sign(dy) * nx, np.where(dx != 0, start_node + np.sign(dx), -1))
    bad = yfirst & (fy == prev)
    hops = np.abs(dx) + np.abs(dy)
    has0 = (start_edge >= 0).astype(np.int64)
    lens = hops + has0
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(lens)
    out = np.empty(int(off[-1]), np.int32)
    out[off[:-1][has0 == 1]] = start_edge[has0 == 1]
    lut = _edge_lookup(net)
    cur = start_node.astype(np.int64).copy()
    rx, ry = np.abs(dx).copy(), np.abs(dy).copy()
    sx, sy = np.sign(dx), np.sign(dy)
    for h in range(int(hops.max()) if n else 0):
        act = np.nonzero(h < hops)[0]
        if act.size == 0:
            break
        usex = np.where(yfirst[act], ry[act] == 0, rx[act] > 0)
        nxt = np.where(usex, cur[act] + sx[act], cur[act] + sy[act] * nx)
        e = _eid(lut, cur[act], nxt)
        out[off[act] + has0[act] + h] = e
        rx[act] -= usex
        ry[act] -= ~usex
        cur[act] = nxt
    return off, out, ~bad


def _tree_routes(net: Network, start_edge, start_node, dest_zone, zones, pred):
    """Routes following reverse shortest-path trees (pred[z, v] = next node from v toward
    zones[z]).  ok=False where the first hop would be a U-turn."""
    n = dest_zone.shape[0]
    prev = np.where(start_edge >= 0, net.edge_from[np.maximum(start_edge, 0)], -1)
    first = np.where(start_node == zones[dest_zone], -1, pred[dest_zone, start_node])
    ok = ~((first == prev) & (first >= 0))
    lut = _edge_lookup(net)
    # hop counts
    hops = np.zeros(n, np.int64)
    cur = start_node.astype(np.int64).copy()
    tgt = zones[dest_zone]
    act = np.nonzero(cur != tgt)[0]
    while act.size:
        hops[act] += 1
        cur[act] = pred[dest_zone[act], cur[act]]
        act = act[cur[act] != tgt[act]]
    has0 = (start_edge >= 0).astype(np.int64)
    lens = hops + has0
    off = np.zeros(n + 1, np.int64)
    off[1:] = np.cumsum(lens)
    out = np.empty(int(off[-1]), np.int32)
    out[off[:-1][has0 == 1]] = start_edge[has0 == 1]
    cur = start_node.astype(np.int64).copy()
    for h in range(int(hops.max()) if n else 0):
        act = np.nonzero(h < hops)[0]
        nxt = pred[dest_zone[act], cur[act]]
        out[off[act] + has0[act] + h] = _eid(lut, cur[act], nxt)
        cur[act] = nxt
    return off, out, ok


def _zone_trees(net: Network, zones: np.ndarray):
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    V = net.node_xy.shape[0]
    # reversed graph: an edge u->v becomes v->u, so trees from a zone give next hops to it
    g = csr_matrix((net.edge_len.astype(np.float64), (net.edge_to, net.edge_from)), shape=(V, V))
    dist, pred = dijkstra(g, directed=True, indices=zones, return_predecessors=True)
    return dist, pred.astype(np.int64)


# ----------------------------------------------------------------------------------------
# demand
# ----------------------------------------------------------------------------------------

def _pack(t_dep, v0, off, edges, lane=None, x=None, v=None) -> Demand:
    n = t_dep.shape[0]
    return Demand(t_dep=np.ascontiguousarray(t_dep, np.int32), v0=np.ascontiguousarray(v0, np.float32),
                  route_off=np.ascontiguousarray(off, np.int64), route_edges=np.ascontiguousarray(edges, np.int32),
                  lane=np.ascontiguousarray(np.full(n, -1) if lane is None else lane, np.int32),
                  x=np.ascontiguousarray(np.zeros(n) if x is None else x, np.float32),
                  v=np.ascontiguousarray(np.zeros(n) if v is None else v, np.float32))


def _select(off, edges, keep):
    lens = (off[1:] - off[:-1])[keep]
    noff = np.zeros(lens.shape[0] + 1, np.int64)
    noff[1:] = np.cumsum(lens)
    idx = np.repeat(off[:-1][keep], lens) + (np.arange(int(noff[-1])) - np.repeat(noff[:-1], lens))
    return noff, edges[idx]


def uniform_trips(net: Network, n: int, t_span: int = 600, v0: float = 13.9, seed: int = 1) -> Demand:
    """Uniform-random origin and destination edges (O != D), departures uniform in
    [0, t_span) s, shortest-path routes from the head of the origin edge to the tail of the
    destination edge.  Trips whose route would begin with a U-turn are redrawn."""
    rng = np.random.default_rng(seed)
    E = net.n_edges
    o_all, d_all = [], []
    need = n
    while need > 0:
        o = rng.integers(0, E, size=2 * need)
        d = rng.integers(0, E, size=2 * need)
        keep = o != d
        o_all.append(o[keep])
        d_all.append(d[keep])
        need -= int(keep.sum())
    o = np.concatenate(o_all)
    d = np.concatenate(d_all)
    # route: o + path(head(o) -> tail(d)) + d
    head = net.edge_to[o].astype(np.int64)
    tail = net.edge_from[d].astype(np.int64)
    if net.grid_shape is not None:
        off, edges, ok = _grid_routes(net, o, head, tail)
    else:
        zones = np.unique(tail)
        _, pred = _zone_trees(net, zones)
        off, edges, ok = _tree_routes(net, o, head, np.searchsorted(zones, tail), zones, pred)
    # last hop arrives at tail(d); it must not be a U-turn into d either
    last = np.where(off[1:] > off[:-1], edges[np.maximum(off[1:] - 1, 0)], o)
    ok &= ~(net.edge_from[last] == net.edge_to[d])
    ok &= last != d  # never happens, kept for clarity
    keep = np.nonzero(ok)[0][:n]
    if keep.shape[0] < n:
        return uniform_trips(net, n, t_span, v0, seed + 7919)
    off, edges = _select(off, edges, keep)
    # append destination edge
    lens = off[1:] - off[:-1] + 1
    noff = np.zeros(n + 1, np.int64)
    noff[1:] = np.cumsum(lens)
    out = np.empty(int(noff[-1]), np.int32)
    pos = np.repeat(noff[:-1], lens - 1) + (np.arange(int(off[-1])) - np.repeat(off[:-1], lens - 1))
    out[pos] = edges
    out[noff[1:] - 1] = d[keep]
    t_dep = np.sort(rng.integers(0, t_span, size=n))
    return _pack(t_dep, np.full(n, v0), noff, out)


def _gravity_dest(rng, nx, ny, origins, attract, chunk=512):
    """Destination node per origin: P(D=j|O=i) ∝ A_j / d_ij^2, d = Manhattan distance in
    links, j != i."""
    V = nx * ny
    jx = np.arange(V) % nx
    jy = np.arange(V) // nx
    dest = np.empty(origins.shape[0], np.int64)
    order = np.argsort(origins, kind="stable")
    so = origins[order]
    uo, st = np.unique(so, return_index=True)
    en = np.append(st[1:], so.shape[0])
    for c0 in range(0, uo.shape[0], chunk):
        us = uo[c0:c0 + chunk]
        d = np.abs(jx[None, :] - (us % nx)[:, None]) + np.abs(jy[None, :] - (us // nx)[:, None])
        w = np.where(d > 0, attract[None, :] / np.maximum(d, 1) ** 2, 0.0)
        cw = np.cumsum(w, 1)
        for r, u in enumerate(us):
            k = c0 + r
            cnt = en[k] - st[k]
            uu = rng.random(cnt) * cw[r, -1]
            dest[order[st[k]:en[k]]] = np.searchsorted(cw[r], uu, side="right")
    return np.minimum(dest, V - 1)


def gravity_trips(net: Network, n: int, t_span: int = 3600, seed: int = 2) -> Demand:
    """Gravity-model OD on a grid: attraction A_i ~ LogNormal(0,1) per node,
    P(O=i) ∝ A_i, P(D=j|O=i) ∝ A_j/d_ij^2 (Manhattan links); departures of a Poisson
    process over t_span s (uniform order statistics); v0 ~ N(13.9, 1.5) clipped to
    [8, 20] m/s; routes x-then-y shortest paths."""
    assert net.grid_shape is not None
    nx, ny = net.grid_shape
    rng = np.random.default_rng(seed)
    A = rng.lognormal(0.0, 1.0, size=nx * ny)
    o = rng.choice(nx * ny, size=n, p=A / A.sum())
    d = _gravity_dest(rng, nx, ny, o, A)
    off, edges, ok = _grid_routes(net, np.full(n, -1), o, d)
    assert ok.all()
    t_dep = np.sort(rng.integers(0, t_span, size=n))
    v0 = np.clip(rng.normal(13.9, 1.5, size=n), 8.0, 20.0)
    return _pack(t_dep, v0, off, edges)


def _spaced_positions(rng, lane_len, counts, min_spacing, veh_len):
    """Sorted front positions in (veh_len, len] with consecutive fronts >= min_spacing
    apart, uniform among such configurations."""
    total = int(counts.sum())
    lane_of = np.repeat(np.arange(counts.shape[0]), counts)
    slack = lane_len[lane_of] - veh_len - (counts[lane_of] - 1) * min_spacing
    u = rng.random(total) * np.maximum(slack, 0.0)
    o = np.lexsort((u, lane_of))
    u = u[o]
    start = np.zeros(counts.shape[0] + 1, np.int64)
    start[1:] = np.cumsum(counts)
    rank = np.arange(total) - start[lane_of]
    return lane_of, (veh_len + u + rank * min_spacing)


def _gather_csr(parts, which, idx_in_part, n):
    """Assemble per-vehicle routes from several CSR parts: vehicle i takes route
    idx_in_part[i] of part which[i]."""
    lens = np.empty(n, np.int64)
    src = np.empty(n, np.int64)
    base = 0
    bases = []
    for k, (off, _) in enumerate(parts):
        m = which == k
        lens[m] = (off[1:] - off[:-1])[idx_in_part[m]]
        src[m] = base + off[:-1][idx_in_part[m]]
        bases.append(base)
        base += int(off[-1])
    allr = np.concatenate([e for _, e in parts]) if parts else np.zeros(0, np.int32)
    noff = np.zeros(n + 1, np.int64)
    noff[1:] = np.cumsum(lens)
    pos = np.repeat(src - noff[:-1], lens) + np.arange(int(noff[-1]))
    return noff, allr[pos].astype(np.int32)


PARETO_ALPHA, PARETO_XM, PARETO_XMAX = 1.5, 1000.0, 40000.0


class _ZoneLengths:
    """Trip-length destinations over zone nodes: per node, the zones' shortest-path
    distances sorted ascending (unreachable ones last), as one flat sorted key array."""
    ROW = 1e9   # row offset of a node's keys (route lengths stay far below 1e8 m)

    def __init__(self, zdist: np.ndarray):
        Z, V = zdist.shape
        d = np.where(np.isfinite(zdist), zdist, 1e8).T          # [V, Z]
        self.order = np.argsort(d, axis=1, kind="stable")
        ds = np.take_along_axis(d, self.order, axis=1)
        self.keys = (ds + np.arange(V, dtype=np.float64)[:, None] * self.ROW).ravel()
        self.ds = ds
        self.Z = Z

    def pick(self, node: np.ndarray, ell: np.ndarray) -> np.ndarray:
        """Zone whose distance from node is closest to ell (reachable zones only)."""
        Z = self.Z
        lo = node * Z
        k = np.searchsorted(self.keys, ell + node * self.ROW)
        k = np.clip(k, lo + 1, lo + Z - 1)
        a, b = k - 1, k
        da = np.abs(self.keys[a] - node * self.ROW - ell)
        db = np.abs(self.keys[b] - node * self.ROW - ell)
        fin_b = self.ds.ravel()[b] < 1e8
        j = np.where(fin_b & (db < da), b, a)
        return self.order.ravel()[j]


def _pareto_lengths(rng, n: int) -> np.ndarray:
    """Trip lengths ~ Pareto(alpha 1.5, x_m 1 km) truncated at 40 km (inverse CDF)."""
    u = rng.random(n)
    c = 1.0 - (PARETO_XM / PARETO_XMAX) ** PARETO_ALPHA
    return PARETO_XM * (1.0 - u * c) ** (-1.0 / PARETO_ALPHA)


def _route_many(net, rng, se, snode, dest, A, zs, pred, max_tries=50, zlen=None):
    """Route vehicles starting on edge se (head node snode); redraw destinations whose
    route would begin with a U-turn.  Returns CSR (off, edges)."""
    n = se.shape[0]
    V = net.node_xy.shape[0]
    parts = []
    which = np.full(n, -1, np.int64)
    idx = np.zeros(n, np.int64)
    pending = np.arange(n)
    for k in range(max_tries):
        if pending.size == 0:
            break
        if dest == "gravity":
            nx, ny = net.grid_shape
            d = _gravity_dest(rng, nx, ny, snode[pending], A)
            off, e, ok = _grid_routes(net, se[pending], snode[pending], d)
        elif net.grid_shape is not None:
            d = rng.integers(0, V, size=pending.shape[0])
            off, e, ok = _grid_routes(net, se[pending], snode[pending], d)
        elif dest == "pareto":
            d = zlen.pick(snode[pending], _pareto_lengths(rng, pending.shape[0]))
            off, e, ok = _tree_routes(net, se[pending], snode[pending], d, zs, pred)
        else:
            d = rng.integers(0, zs.shape[0], size=pending.shape[0])
            off, e, ok = _tree_routes(net, se[pending], snode[pending], d, zs, pred)
        parts.append((off, e))
        good = np.nonzero(ok)[0]
        which[pending[good]] = len(parts) - 1
        idx[pending[good]] = good
        pending = pending[~ok]
    # leftovers (destination straight behind): end the trip on the current edge
    if pending.size:
        off = np.arange(pending.size + 1, dtype=np.int64)
        parts.append((off, se[pending].astype(np.int32)))
        which[pending] = len(parts) - 1
        idx[pending] = np.arange(pending.size)
    return _gather_csr(parts, which, idx, n)


def place_vehicles(net: Network, n: int, seed: int = 3, min_spacing: float = 9.0,
                   veh_len: float = 5.0, v0_mean: float = 13.9, v0_sd: float = 1.5,
                   internal_frac: float = 0.0, dest: str = "gravity", zones: int = 256) -> Demand:
    """Steady-state workload: n vehicles already on the network at t = 0.

    Vehicles are spread over edges in proportion to lane length (and, if internal_frac > 0,
    also over junction-internal lanes with that relative weight), routed from the edge
    they are on (gravity destinations on grids, else uniform over `zones` zone nodes, or
    with dest="pareto" the zone whose shortest-path distance from the edge's head node is
    closest to a trip length drawn from Pareto(1.5, 1 km) truncated at 40 km),
    then put on a lane of their edge that serves their next route edge; consecutive fronts
    on a lane are at least min_spacing apart; speed uniform in [0, v0];
    v0 ~ N(v0_mean, v0_sd) clipped to [8, 20]."""
    rng = np.random.default_rng(seed)
    nel = net.n_edge_lanes
    L = net.n_lanes
    E = net.n_edges
    V = net.node_xy.shape[0]
    lane_cap = np.floor((net.lane_len.astype(np.float64) - veh_len) / min_spacing).astype(np.int64) + 1
    use_gravity = net.grid_shape is not None and dest == "gravity"
    A = rng.lognormal(0.0, 1.0, size=V) if use_gravity else None
    zs = pred = zlen = None
    if not use_gravity and net.grid_shape is None:
        zs = np.unique(rng.integers(0, V, size=zones))
        zd, pred = _zone_trees(net, zs)
        if dest == "pareto":
            zlen = _ZoneLengths(zd)
    gdest = "gravity" if use_gravity else ("pareto" if zlen is not None else "uniform")
    # internal lanes: (approach edge, exit edge, target lane)
    int_src = np.full(L, -1, np.int64)
    int_dst = np.full(L, -1, np.int64)
    src_l = np.repeat(np.arange(nel), np.diff(net.succ_off[:nel + 1]))
    sl = net.succ_lane[:net.succ_off[nel]]
    int_src[sl] = net.lane_edge[src_l]
    int_dst[sl] = net.succ_edge[:net.succ_off[nel]]
    int_tgt = np.full(L, -1, np.int64)
    int_tgt[nel:] = net.succ_lane[net.succ_off[nel:L]]
    # how many on internal lanes vs edges
    w_edge = net.edge_len.astype(np.float64) * net.edge_nlanes
    w_int = net.lane_len[nel:].astype(np.float64) * internal_frac
    tot = w_edge.sum() + w_int.sum()
    n_int = int(round(n * w_int.sum() / tot)) if internal_frac > 0 else 0
    cnt_i = None
    if n_int:
        wi = net.lane_len[nel:].astype(np.float64)
        cnt_i = np.minimum(rng.multinomial(n_int, wi / wi.sum()), lane_cap[nel:])
        n_int = int(cnt_i.sum())
    n_edge = n - n_int
    # --- edge vehicles: draw an edge, route from it, take a lane of it that serves the next
    # route edge; vehicles that find their serving lanes full are drawn again elsewhere
    conn_key = np.unique(src_l.astype(np.int64) * E + net.succ_edge[:net.succ_off[nel]])
    lane_fill = np.zeros(L, np.int64)
    e_cap = net.edge_nlanes.astype(np.int64) * lane_cap[net.edge_lane0]
    if n_edge > int(e_cap.sum()):
        raise ValueError(f"{n_edge} vehicles do not fit")
    acc_parts, acc_lane = [], []
    pending = n_edge
    for attempt in range(200):
        if pending == 0:
            break
        e_room = (e_cap - np.bincount(net.lane_edge[:nel], weights=lane_fill[:nel], minlength=E)).astype(np.float64)
        w = w_edge * (e_room > 0)
        se = rng.choice(E, size=pending, p=w / w.sum())
        snode = net.edge_to[se].astype(np.int64)
        off, edges = _route_many(net, rng, se, snode, gdest, A, zs, pred, zlen=zlen)
        nxt = np.where(off[1:] - off[:-1] >= 2, edges[np.minimum(off[:-1] + 1, max(edges.shape[0] - 1, 0))], -1)
        kmax = int(net.edge_nlanes.max())
        ok_mask = np.zeros((pending, kmax), bool)
        for q in range(kmax):
            lq = net.edge_lane0[se] + q
            key = lq.astype(np.int64) * E + np.maximum(nxt, 0)
            pos = np.minimum(np.searchsorted(conn_key, key), conn_key.shape[0] - 1)
            ok_mask[:, q] = (q < net.edge_nlanes[se]) & ((nxt < 0) | (conn_key[pos] == key))
        nok = ok_mask.sum(1)
        pick = np.floor(rng.random(pending) * np.maximum(nok, 1)).astype(np.int64)
        q_sel = np.argmax(np.cumsum(ok_mask, 1) > pick[:, None], axis=1)
        lane_e = net.edge_lane0[se] + q_sel
        # accept up to the remaining capacity of each lane
        o = np.argsort(lane_e, kind="stable")
        ls = lane_e[o]
        rank = np.arange(pending) - np.searchsorted(ls, ls, side="left")
        acc = np.zeros(pending, bool)
        acc[o] = rank < (lane_cap[ls] - lane_fill[ls])
        acc &= nok > 0
        ai = np.nonzero(acc)[0]
        lane_fill += np.bincount(lane_e[ai], minlength=L)
        acc_parts.append(_gather_csr([(off, edges)], np.zeros(ai.size, np.int64), ai, ai.size))
        acc_lane.append(lane_e[ai])
        pending -= ai.size
    else:
        raise RuntimeError("could not place all vehicles; lower the density")
    lane_e = np.concatenate(acc_lane)
    off, edges = _gather_csr(acc_parts, np.concatenate([np.full(l.shape[0], k) for k, l in enumerate(acc_lane)]),
                             np.concatenate([np.arange(l.shape[0]) for l in acc_lane]), n_edge)
    parts = [(off, edges)]
    lanes_all = [lane_e]
    # --- internal-lane vehicles (tests of junction logic)
    if n_int:
        lane_i = nel + np.repeat(np.arange(L - nel), cnt_i)
        m = lane_i.shape[0]
        se_i = int_dst[lane_i]
        sn_i = net.edge_to[se_i].astype(np.int64)
        off_i, edges_i = _route_many(net, rng, se_i, sn_i, gdest, A, zs, pred, zlen=zlen)
        # keep those whose target lane serves the route's next edge, else end at the exit edge
        nx_i = np.where(off_i[1:] - off_i[:-1] >= 2, edges_i[np.minimum(off_i[:-1] + 1, max(edges_i.shape[0] - 1, 0))], -1)
        key = int_tgt[lane_i] * E + np.maximum(nx_i, 0)
        pos = np.minimum(np.searchsorted(conn_key, key), conn_key.shape[0] - 1)
        good = (nx_i < 0) | (conn_key[pos] == key)
        one = np.arange(m + 1, dtype=np.int64)
        short_parts = [(off_i, edges_i), (one, se_i.astype(np.int32))]
        off_i, edges_i = _gather_csr(short_parts, np.where(good, 0, 1), np.arange(m), m)
        # prepend the approach edge
        lens = off_i[1:] - off_i[:-1] + 1
        o2 = np.zeros(m + 1, np.int64)
        o2[1:] = np.cumsum(lens)
        e2 = np.empty(int(o2[-1]), np.int32)
        e2[o2[:-1]] = int_src[lane_i]
        pos2 = np.repeat(o2[:-1] + 1 - off_i[:-1], off_i[1:] - off_i[:-1]) + np.arange(int(off_i[-1]))
        e2[pos2] = edges_i
        parts.append((o2, e2))
        lanes_all.append(lane_i)
    lane_of = np.concatenate(lanes_all)
    which = np.concatenate([np.full(a.shape[0], k) for k, a in enumerate(lanes_all)])
    idx = np.concatenate([np.arange(a.shape[0]) for a in lanes_all])
    off, edges = _gather_csr(parts, which, idx, n)
    # positions: per lane, sorted uniform with spacing
    order = np.argsort(lane_of, kind="stable")
    counts = np.bincount(lane_of, minlength=L)
    lane_sorted, x_sorted = _spaced_positions(rng, net.lane_len.astype(np.float64), counts, min_spacing, veh_len)
    x = np.empty(n)
    x[order] = x_sorted
    v0 = np.clip(rng.normal(v0_mean, v0_sd, size=n), 8.0, 20.0)
    v = rng.random(n) * v0
    return _pack(np.zeros(n, np.int32), v0, off, edges, lane=lane_of, x=x, v=v)


def merge_demands(a: Demand, b: Demand) -> Demand:
    off = np.concatenate([a.route_off[:-1], b.route_off + a.route_off[-1]])
    return Demand(t_dep=np.concatenate([a.t_dep, b.t_dep]), v0=np.concatenate([a.v0, b.v0]),
                  route_off=off, route_edges=np.concatenate([a.route_edges, b.route_edges]),
                  lane=np.concatenate([a.lane, b.lane]), x=np.concatenate([a.x, b.x]),
                  v=np.concatenate([a.v, b.v]))


def union(nets, dems):
    """Disjoint union of several scenarios as one network and one demand: scenario k's
    lanes, edges, controllers and trips are offset by the totals of scenarios 0..k-1."""
    lo = np.cumsum([0] + [n.n_lanes for n in nets])
    eo = np.cumsum([0] + [n.n_edges for n in nets])
    co = np.cumsum([0] + [n.n_ctrl for n in nets])
    so = np.cumsum([0] + [int(n.succ_off[-1]) for n in nets])
    vo = np.cumsum([0] + [n.node_xy.shape[0] for n in nets])
    sh = lambda a, o: np.where(a >= 0, a + o, a)
    cat = lambda f: np.concatenate(f)
    net = Network(
        node_xy=cat([n.node_xy for n in nets]),
        edge_from=cat([n.edge_from + vo[k] for k, n in enumerate(nets)]).astype(np.int32),
        edge_to=cat([n.edge_to + vo[k] for k, n in enumerate(nets)]).astype(np.int32),
        edge_len=cat([n.edge_len for n in nets]), edge_nlanes=cat([n.edge_nlanes for n in nets]),
        edge_lane0=cat([n.edge_lane0 + lo[k] for k, n in enumerate(nets)]).astype(np.int32),
        lane_len=cat([n.lane_len for n in nets]),
        lane_edge=cat([sh(n.lane_edge, eo[k]) for k, n in enumerate(nets)]).astype(np.int32),
        lane_index=cat([n.lane_index for n in nets]),
        lane_left=cat([sh(n.lane_left, lo[k]) for k, n in enumerate(nets)]).astype(np.int32),
        lane_right=cat([sh(n.lane_right, lo[k]) for k, n in enumerate(nets)]).astype(np.int32),
        succ_off=np.concatenate([n.succ_off[:-1] + so[k] for k, n in enumerate(nets)] + [[so[-1]]]).astype(np.int32),
        succ_lane=cat([n.succ_lane + lo[k] for k, n in enumerate(nets)]).astype(np.int32),
        succ_edge=cat([n.succ_edge + eo[k] for k, n in enumerate(nets)]).astype(np.int32),
        lane_ctrl=cat([sh(n.lane_ctrl, co[k]) for k, n in enumerate(nets)]).astype(np.int32),
        lane_group=cat([n.lane_group for n in nets]),
        ctrl_node=cat([n.ctrl_node + vo[k] for k, n in enumerate(nets)]).astype(np.int32),
        ctrl_offset=cat([n.ctrl_offset for n in nets]), ctrl_green=cat([n.ctrl_green for n in nets]),
        ctrl_yellow=cat([n.ctrl_yellow for n in nets]), ctrl_nphase=cat([n.ctrl_nphase for n in nets]),
        name="union")
    ro = np.cumsum([0] + [int(d.route_off[-1]) for d in dems])
    dem = Demand(
        t_dep=cat([d.t_dep for d in dems]), v0=cat([d.v0 for d in dems]),
        route_off=np.concatenate([d.route_off[:-1] + ro[k] for k, d in enumerate(dems)] + [[ro[-1]]]).astype(np.int64),
        route_edges=cat([d.route_edges + eo[k] for k, d in enumerate(dems)]).astype(np.int32),
        lane=cat([sh(d.lane, lo[k]) for k, d in enumerate(dems)]).astype(np.int32),
        x=cat([d.x for d in dems]), v=cat([d.v for d in dems]))
    return net, dem


def batch_scenarios(n_scen: int = 256, seed: int = 7, side=(4, 32), n_range=(500, 200_000),
                    n_lanes: int = 2, link_len: float = 200.0):
    """Independent scenarios of uneven size for batched runs: grid side ~ U{side}, vehicle
    count ~ log-uniform n_range (capped at 60% of the grid's jam capacity), distinct seeds
    and random signal plans (offsets uniform in the cycle, green U{20..40} s); vehicles are
    pre-placed (steady state) with uniform destinations."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_scen):
        a = int(rng.integers(side[0], side[1] + 1))
        net = grid_network(a, a, n_lanes, link_len, 30, 3, "random", seed=seed * 1000 + k)
        cap = int(0.6 * net.n_edge_lanes * (link_len - 5.0) / 9.0)
        n = int(min(cap, np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1])))))
        dem = place_vehicles(net, max(n, 1), seed=seed * 1000 + k, dest="uniform")
        out.append((net, dem))
    return out


# ----------------------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------------------

def small_grid_workload(seed: int = 1):
    """4x4 signalised grid, 2 lanes per direction, 200 m links, 30 s green / 3 s yellow,
    zero offsets; 500 trips, uniform OD edges, departures uniform over 600 s, v0 = 13.9."""
    net = grid_network(4, 4, 2, 200.0, 30, 3, "zero")
    dem = uniform_trips(net, 500, 600, 13.9, seed=seed)
    return net, dem


def large_grid_network():
    """100x100 signalised grid, 3 lanes per direction, 300 m links, green-wave offsets."""
    return grid_network(100, 100, 3, 300.0, 30, 3, "wave")


def closable_link_masks(net: Network, dem: Demand, rng, frac: float) -> dict:
    """Open-link masks per edge lane with about frac of the links closed, every route still
    lane-connected: a link closes only if each pair of consecutive route edges leaving its
    edge keeps an open link from some lane of that edge."""
    re = np.asarray(dem.route_edges, np.int64)
    last = np.zeros(re.shape[0], bool)   # route entries that end a route (no pair after them)
    last[np.asarray(dem.route_off[1:], np.int64) - 1] = True
    idx = np.nonzero(~last[:-1])[0]
    pairs = np.unique(re[idx] * net.n_edges + re[idx + 1])
    exits = {}
    for pr in pairs.tolist():
        exits.setdefault(pr // net.n_edges, set()).add(pr % net.n_edges)
    el = np.nonzero(net.lane_edge >= 0)[0]
    deg = {int(l): int(net.succ_off[l + 1] - net.succ_off[l]) for l in el}
    mask = {l: (1 << d) - 1 for l, d in deg.items()}

    def connected(e, b):
        for q in range(int(net.edge_nlanes[e])):
            l = int(net.edge_lane0[e]) + q
            for j in range(deg[l]):
                if (mask[l] >> j) & 1 and int(net.succ_edge[net.succ_off[l] + j]) == b:
                    return True
        return False

    for l in rng.permutation(el):
        l = int(l)
        e = int(net.lane_edge[l])
        for j in range(deg[l]):
            if rng.random() >= frac:
                continue
            mask[l] &= ~(1 << j)
            if not all(connected(e, b) for b in exits.get(e, ())):
                mask[l] |= 1 << j
    return mask
