// route_kernels.cuh -- least-cost lane-linked routes for trips (demand generation, sm_103a).
//
// The route graph has one node per road edge and an arc e -> f wherever a lane of e links
// to exit edge f; entering f costs c(f) integer millimetres.  For a batch of B destinations
// the distances d[e * B + b] = least cost from e to destination b are relaxed in place by
// pull iterations (thread (e, b): d = min(d, min over successors f of c(f) + d[f][b])), which
// reach the exact least costs once nothing changes (only that thread writes d[e][b], and the
// minimum does not depend on the order of updates).  The B destinations of one edge are
// contiguous, so a warp reads each successor's row of 32 distances in one coalesced load.
// A trip then walks from its origin along the lowest-id successor that stays on a
// least-cost route.
#pragma once
#include <cstdint>

namespace moss {

constexpr long long ROUTE_INF = 0x3fffffffffffffffLL;

struct RouteGraph {
  const int *off;          // [E + 1] successor ranges
  const int *dst;          // successors of each edge, increasing id
  const long long *cost;   // [E] c(f), mm
  int E;
};

__global__ void k_route_init(long long *d, int E, int B, const int *dest, int nb) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)E * B) return;
  const int e = (int)(i / B), b = (int)(i % B);
  d[i] = (b < nb && dest[b] == e) ? 0 : ROUTE_INF;
}

__global__ void k_route_relax(long long *d, RouteGraph g, int B, int *changed) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)g.E * B) return;
  const int e = (int)(i / B), b = (int)(i % B);
  const long long cur = d[i];
  long long best = cur;
  for (int k = g.off[e]; k < g.off[e + 1]; ++k) {
    const int f = g.dst[k];
    const long long v = d[(long long)f * B + b];
    if (v < ROUTE_INF) best = min(best, g.cost[f] + v);
  }
  if (best < cur) {
    d[i] = best;
    *changed = 1;
  }
}

// next edge on the route from e toward destination column b (-1 if none)
__device__ __forceinline__ int route_next(const long long *d, const RouteGraph &g, int B, int e, int b) {
  const long long de = d[(long long)e * B + b];
  for (int k = g.off[e]; k < g.off[e + 1]; ++k) {
    const int f = g.dst[k];
    const long long v = d[(long long)f * B + b];
    if (v < ROUTE_INF && g.cost[f] + v == de) return f;
  }
  return -1;
}

// trips of one destination batch: tr[j] = {trip index, origin, destination, column}
// pass 0 (out == nullptr) counts each route's length into len[j] (0: unreachable, at most
// max_hops: least-cost routes are simple paths since every c(f) > 0); pass 1 writes exactly
// len[j] edges at off[j]
__global__ void k_route_walk(const long long *d, RouteGraph g, int B, const int4 *tr, int n, const long long *off,
                             int *len, int *out, int max_hops, int *err) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int4 t = tr[j];
  int e = t.y;
  if (!out) {
    if (d[(long long)e * B + t.w] >= ROUTE_INF) {
      len[j] = 0;
      return;
    }
    int cnt = 1;
    while (e != t.z) {
      e = route_next(d, g, B, e, t.w);
      if (e < 0 || cnt >= max_hops) {   // never expected on converged distances
        atomicOr(err, 1);
        break;
      }
      ++cnt;
    }
    len[j] = cnt;
    return;
  }
  const int L = len[j];
  if (L == 0) return;
  int *o = out + off[j];
  o[0] = e;
  for (int k = 1; k < L; ++k) {
    const int f = route_next(d, g, B, e, t.w);
    if (f < 0) {
      atomicOr(err, 1);
      o[k] = t.z;
      continue;
    }
    e = f;
    o[k] = e;
  }
}

}  // namespace moss
