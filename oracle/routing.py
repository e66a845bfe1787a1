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
