"""FP64 / integer CPU reference of the GPU route planner -- TEST INFRASTRUCTURE.

Reading R15 (demand generation: routes of trips; the paper builds trips with routes from
OD matrices on the host, Sec. III-C "Converter from OD matrix to travel demand", and its
GPU simulator needs them at scale).  Only tests/, __graft_entry__.smoke() and bench.py may
import this module.  Plain numpy / scipy; shares no code with the CUDA library.

R15  The route graph has one node per road edge and an arc e -> f wherever some lane of e
     has a lane link whose exit edge is f.  Entering f costs c(f) = round(1000 * length of
     f) integer millimetres.  d_D(e) is the least total cost of the edges entered on a path
     from e to the destination edge D (d_D(D) = 0).  A trip from o to D follows, from e = o,
     the lowest-id successor f with c(f) + d_D(f) = d_D(e) until it reaches D; this is the
     lexicographically smallest (by edge ids) of its least-cost routes.  A trip whose
     destination cannot be reached gets an empty route.
"""
from __future__ import annotations

import numpy as np


def edge_graph(net):
    """Arcs of the route graph: (src, dst) pairs, unique, sorted by (src, dst)."""
    E = net.n_edges
    src, dst = [], []
    for e in range(E):
        outs = set()
        for q in range(int(net.edge_nlanes[e])):
            l = int(net.edge_lane0[e]) + q
            outs.update(int(x) for x in net.succ_edge[net.succ_off[l]:net.succ_off[l + 1]])
        for f in sorted(outs):
            src.append(e)
            dst.append(f)
    return np.asarray(src, np.int64), np.asarray(dst, np.int64)


def edge_cost(net) -> np.ndarray:
    """c(f): rounded length of edge f in millimetres (the float32 lane length times 1000)."""
    lens = np.asarray(net.lane_len, np.float32)[np.asarray(net.edge_lane0, np.int64)].astype(np.float64)
    return np.rint(lens * 1000.0).astype(np.int64)


def distances_to(net, dests) -> np.ndarray:
    """d_D(e) for every destination D in dests: [len(dests), E] (inf where unreachable), by
    Dijkstra (a library routine) on the reversed route graph, arc f -> e weighted c(f).
    Integer-valued weights below 2^53 keep the float64 sums exact."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import dijkstra
    E = net.n_edges
    src, dst = edge_graph(net)
    c = edge_cost(net)
    g = csr_matrix((c[dst].astype(np.float64), (dst, src)), shape=(E, E))
    return dijkstra(g, directed=True, indices=np.asarray(dests, np.int64))


def routes(net, orig, dest):
    """Routes of the trips (orig[i] -> dest[i]): CSR (off, edges) and the unreachable count."""
    orig = np.asarray(orig, np.int64)
    dest = np.asarray(dest, np.int64)
    src, dst = edge_graph(net)
    c = edge_cost(net)
    off_s = np.searchsorted(src, np.arange(net.n_edges + 1))
    uniq, inv = np.unique(dest, return_inverse=True)
    d = distances_to(net, uniq)
    off = [0]
    out = []
    bad = 0
    for i in range(orig.shape[0]):
        row = d[inv[i]]
        e, D = int(orig[i]), int(dest[i])
        if not np.isfinite(row[e]):
            bad += 1
            off.append(len(out))
            continue
        out.append(e)
        while e != D:
            nxt = -1
            for k in range(off_s[e], off_s[e + 1]):   # successors in increasing id
                f = int(dst[k])
                if np.isfinite(row[f]) and c[f] + row[f] == row[e]:
                    nxt = f
                    break
            assert nxt >= 0, "no successor on a least-cost route"
            e = nxt
            out.append(e)
        off.append(len(out))
    return np.asarray(off, np.int64), np.asarray(out, np.int32), bad


# ---------------------------------------------------------------------------------------
# R16  Gravity OD sampling.  Zone z has a representative edge zone_edge[z] and attraction
#      A_z > 0.  Trip k draws three 24-bit uniforms u = (SplitMix64(seed ^ salt ^ k) >> 40)
#      / 2^24 with salts 0x5851F42D4C957F2D (origin), 0x14057B7EF767814F (destination) and
#      0x2545F4914F6CDD1D (departure).  Origin zone: the first i whose cumulative attraction
#      exceeds u * sum(A).  Destination zone: with w_j = A_j / dkm_ij^gamma for j != i
#      (dkm_ij = float32(route cost from zone_edge[i] to zone_edge[j] in mm) * 1e-6, raised
#      by gamma float32 products; 0 if unreachable), the first j whose cumulative weight
#      exceeds u * sum(w).  Departure step: floor(u24 * t_span / 2^24) in integers.  Weights
#      and sums are float32, accumulated in index order (so the draw is exact on both sides).
#      An origin zone that reaches no other zone keeps the trip at home (destination = origin).
# ---------------------------------------------------------------------------------------

SALT_ORIGIN, SALT_DEST, SALT_TIME = 0x5851F42D4C957F2D, 0x14057B7EF767814F, 0x2545F4914F6CDD1D


def _u24(splitmix64, seed, salt, k):
    return splitmix64((seed ^ salt ^ k) % 2 ** 64) >> 40


def _first_above(cdf, target):
    """First index whose cumulative value exceeds target (float32 compare)."""
    i = int(np.searchsorted(cdf, target, side="right"))
    return min(i, cdf.shape[0] - 1)


def gravity_trips(net, zone_edge, attract, gamma, n, t_span, seed, splitmix64):
    """Trips (orig_edge, dest_edge, t_dep) of R16; splitmix64 is the published generator
    (the oracle's C implementation, pinned by its published vector)."""
    zone_edge = np.asarray(zone_edge, np.int64)
    A = np.asarray(attract, np.float32)
    Z = zone_edge.shape[0]
    d = distances_to(net, zone_edge)            # [Z dest, E]: d[j, e] = cost e -> zone j
    cost = d[:, zone_edge].T                    # cost[i, j] = zone i -> zone j
    cdf_o = np.cumsum(A, dtype=np.float32)
    W = np.zeros((Z, Z), np.float32)
    for i in range(Z):
        for j in range(Z):
            if j == i or not np.isfinite(cost[i, j]):
                continue
            dkm = np.float32(np.float32(cost[i, j]) * np.float32(1e-6))
            p = np.float32(1.0)
            for _ in range(gamma):
                p = np.float32(p * dkm)
            W[i, j] = np.float32(A[j] / p)
    cdf_d = np.cumsum(W, axis=1, dtype=np.float32)
    o = np.zeros(n, np.int32)
    de = np.zeros(n, np.int32)
    td = np.zeros(n, np.int32)
    for k in range(n):
        uo = np.float32(_u24(splitmix64, seed, SALT_ORIGIN, k)) * np.float32(2.0 ** -24)
        i = _first_above(cdf_o, np.float32(uo * cdf_o[-1]))
        ud = np.float32(_u24(splitmix64, seed, SALT_DEST, k)) * np.float32(2.0 ** -24)
        j = _first_above(cdf_d[i], np.float32(ud * cdf_d[i, -1])) if cdf_d[i, -1] > 0 else i
        o[k], de[k] = zone_edge[i], zone_edge[j]
        td[k] = (_u24(splitmix64, seed, SALT_TIME, k) * int(t_span)) >> 24
    return o, de, td


# ---------------------------------------------------------------------------------------
# R18  Radiation OD sampling (Simini, Gonzalez, Maritan and Barabasi 2012, "A universal
#      model for mobility and migration patterns").  Zone z has a representative edge and a
#      population m_z > 0.  The origin draw is R16's with the populations as attractions.
#      For origin i, with d_ij the route cost from zone i's edge to zone j's (R15, mm) and
#      s_ij the population of the zones strictly closer to i than j (neither i nor j), the
#      destination weight of j != i is
#          w_ij = (m_i * m_j) / ((m_i + s_ij) * ((m_i + m_j) + s_ij)),
#      0 if j is unreachable.  s_ij is the float32 running sum of populations over the zones
#      in order of (d_ik, k), i excluded, taken before the first zone at distance d_ij; every
#      operation is one IEEE float32 operation in the order written.  Destination and
#      departure draws are R16's (same salts, cumulative weights in index order).
# ---------------------------------------------------------------------------------------

def radiation_weights(cost, pop):
    """w[i, j] of R18 from the zone-to-zone route costs cost[i, j] (inf: unreachable), zone
    by zone as R18 states it: walk the zones in order of (distance, index), give each group
    of equal distance the running population sum of the zones before the group, then add
    the group's populations (zone i's excepted) one float32 addition at a time."""
    m = np.asarray(pop, np.float32)
    Z = m.shape[0]
    W = np.zeros((Z, Z), np.float32)
    for i in range(Z):
        d = np.asarray(cost[i], np.float64)
        order = np.lexsort((np.arange(Z), d))           # by (distance, zone index)
        run = np.float32(0.0)
        s = np.zeros(Z, np.float32)
        q = 0
        while q < Z:                                     # groups of equal distance
            r = q
            while r < Z and d[order[r]] == d[order[q]]:
                r += 1
            for k in order[q:r]:
                s[k] = run                               # zones strictly closer
            for k in order[q:r]:
                if k != i:
                    run = np.float32(run + m[k])
            q = r
        for j in range(Z):
            if j == i or not np.isfinite(d[j]):
                continue
            num = np.float32(m[i] * m[j])
            den = np.float32(np.float32(m[i] + s[j]) * np.float32(np.float32(m[i] + m[j]) + s[j]))
            W[i, j] = np.float32(num / den)
    return W


def radiation_weights_vec(cost, pop):
    """radiation_weights with each origin's row in array operations (for thousands of
    zones): the running sum is a sequential float32 cumulative sum in the same order (zone
    i adds 0, which leaves a float32 sum unchanged), each group takes the sum before its
    first zone, and the weight is the same three IEEE float32 operations.  Pinned against
    radiation_weights on random inputs with ties and unreachable zones."""
    m = np.asarray(pop, np.float32)
    Z = m.shape[0]
    W = np.zeros((Z, Z), np.float32)
    for i in range(Z):
        d = np.asarray(cost[i], np.float64)
        order = np.lexsort((np.arange(Z), d))                 # by (distance, zone index)
        ds = d[order]
        run = np.cumsum(np.where(order == i, np.float32(0.0), m[order]), dtype=np.float32)
        start = np.r_[0, np.nonzero(ds[1:] != ds[:-1])[0] + 1]   # first position of each
        grp = np.searchsorted(start, np.arange(Z), side="right") - 1   # equal-distance group
        before = np.where(start[grp] > 0, run[np.maximum(start[grp] - 1, 0)], np.float32(0.0))
        s_ij = np.empty(Z, np.float32)
        s_ij[order] = before                                  # zones strictly closer
        ok = (np.arange(Z) != i) & np.isfinite(d)
        num = m[i] * m                                        # float32 elementwise, IEEE
        den = (m[i] + s_ij) * ((m[i] + m) + s_ij)
        W[i] = np.where(ok, num / np.where(ok, den, np.float32(1.0)), np.float32(0.0))
    return W


def radiation_trips(net, zone_edge, pop, n, t_span, seed, splitmix64):
    """Trips (orig_edge, dest_edge, t_dep) of R18."""
    zone_edge = np.asarray(zone_edge, np.int64)
    m = np.asarray(pop, np.float32)
    d = distances_to(net, zone_edge)            # [Z dest, E]
    cost = d[:, zone_edge].T                    # cost[i, j] = zone i -> zone j
    W = (radiation_weights if m.shape[0] <= 256 else radiation_weights_vec)(cost, m)
    cdf_o = np.cumsum(m, dtype=np.float32)
    cdf_d = np.cumsum(W, axis=1, dtype=np.float32)
    o = np.zeros(n, np.int32)
    de = np.zeros(n, np.int32)
    td = np.zeros(n, np.int32)
    for k in range(n):
        uo = np.float32(_u24(splitmix64, seed, SALT_ORIGIN, k)) * np.float32(2.0 ** -24)
        i = _first_above(cdf_o, np.float32(uo * cdf_o[-1]))
        ud = np.float32(_u24(splitmix64, seed, SALT_DEST, k)) * np.float32(2.0 ** -24)
        j = _first_above(cdf_d[i], np.float32(ud * cdf_d[i, -1])) if cdf_d[i, -1] > 0 else i
        o[k], de[k] = zone_edge[i], zone_edge[j]
        td[k] = (_u24(splitmix64, seed, SALT_TIME, k) * int(t_span)) >> 24
    return o, de, td
