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

// Gravity OD sampling.  Per origin zone i (one thread, index order, float32): the
// cumulative destination weights cdf[i][j] of w_ij = A_j / dkm_ij^gamma (j != i; 0 where
// unreachable), dkm_ij = float(cost i -> j in mm) * 1e-6 raised by gamma products; the
// origin CDF of the attractions in thread 0.  IEEE division (no fast math), so the
// table matches a float32 CPU computation bit for bit.
__global__ void k_od_cdf(const long long *d, int B, const int *zone_edge, const float *attract, int Z, int gamma,
                         float *cdf_d, float *cdf_o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Z) return;
  if (i == 0) {
    float acc = 0.f;
    for (int z = 0; z < Z; ++z) {
      acc = __fadd_rn(acc, attract[z]);
      cdf_o[z] = acc;
    }
  }
  const long long row = (long long)zone_edge[i] * B;   // distances from zone i's edge
  float acc = 0.f;
  for (int j = 0; j < Z; ++j) {
    const long long c = d[row + j];
    if (j != i && c < ROUTE_INF) {
      const float dkm = __fmul_rn((float)c, 1e-6f);
      float p = 1.f;
      for (int g = 0; g < gamma; ++g) p = __fmul_rn(p, dkm);
      acc = __fadd_rn(acc, __fdiv_rn(attract[j], p));
    }
    cdf_d[(long long)i * Z + j] = acc;
  }
}

// Radiation OD weights (Simini et al. 2012): block i handles origin zone i.  The zones are
// sorted by (route cost from zone i, zone index) with a bitonic sort in shared memory (cost
// and index packed into one 64-bit key; unreachable zones last); one thread then walks the
// sorted order, giving every zone s = the float32 running sum of the populations of the
// zones strictly closer (i excluded, equal costs in one group), and the block forms
// w_ij = (m_i m_j) / ((m_i + s_ij)((m_i + m_j) + s_ij)) with IEEE float32 operations; the
// cumulative weights in index order follow (as for the gravity model), and block 0 also
// writes the origin CDF of the populations.  Shared memory: 8 P + 8 Z bytes (P = Z rounded
// up to a power of two).  A reachable cost of 2^40 mm or more sets *err (never expected).
constexpr int OD_RAD_THREADS = 1024;
constexpr unsigned long long OD_RAD_FAR = (1ull << 40) - 1;

__global__ void __launch_bounds__(OD_RAD_THREADS) k_od_radiation_cdf(const long long *d, int B, const int *zone_edge,
                                                                     const float *pop, int Z, int P, float *cdf_d,
                                                                     float *cdf_o, int *err) {
  extern __shared__ __align__(16) unsigned char rsm[];
  unsigned long long *key = reinterpret_cast<unsigned long long *>(rsm);
  float *m = reinterpret_cast<float *>(key + P);
  float *sc = m + Z;
  const int i = blockIdx.x;
  const long long row = (long long)zone_edge[i] * B;   // costs from zone i's edge
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    unsigned long long kk = ~0ull;   // padding sorts last
    if (k < Z) {
      const long long c = d[row + k];
      unsigned long long cd = OD_RAD_FAR;
      if (c < ROUTE_INF) {
        if ((unsigned long long)c >= OD_RAD_FAR) atomicOr(err, 1);
        cd = (unsigned long long)c < OD_RAD_FAR ? (unsigned long long)c : OD_RAD_FAR - 1;
      }
      kk = (cd << 12) | (unsigned long long)k;
      m[k] = pop[k];
    }
    key[k] = kk;
  }
  __syncthreads();
  for (int w = 2; w <= P; w <<= 1)
    for (int j = w >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < P; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const unsigned long long a = key[t], b = key[u];
          if ((a > b) == ((t & w) == 0)) {
            key[t] = b;
            key[u] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) {
    float run = 0.f;
    int q = 0;
    while (q < Z) {   // groups of equal cost
      const unsigned long long cq = key[q] >> 12;
      int r = q;
      while (r < Z && (key[r] >> 12) == cq) ++r;
      for (int x = q; x < r; ++x) sc[(int)(key[x] & 0xfff)] = run;
      for (int x = q; x < r; ++x) {
        const int k = (int)(key[x] & 0xfff);
        if (k != i) run = __fadd_rn(run, m[k]);
      }
      q = r;
    }
  }
  __syncthreads();
  const float mi = m[i];
  float *out = cdf_d + (long long)i * Z;
  for (int j = threadIdx.x; j < Z; j += blockDim.x) {   // weights first, then the running sum
    float w = 0.f;
    if (j != i && d[row + j] < ROUTE_INF) {
      const float num = __fmul_rn(mi, m[j]);
      const float den = __fmul_rn(__fadd_rn(mi, sc[j]), __fadd_rn(__fadd_rn(mi, m[j]), sc[j]));
      w = __fdiv_rn(num, den);
    }
    out[j] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float acc = 0.f;
    for (int j = 0; j < Z; ++j) {
      acc = __fadd_rn(acc, out[j]);
      out[j] = acc;
    }
    if (i == 0) {
      float ao = 0.f;
      for (int z = 0; z < Z; ++z) {
        ao = __fadd_rn(ao, m[z]);
        cdf_o[z] = ao;
      }
    }
  }
}

__device__ __forceinline__ unsigned long long od_mix(unsigned long long z) {   // SplitMix64
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// first index whose cumulative value exceeds target (the last one if none does)
__device__ __forceinline__ int od_first_above(const float *cdf, int Z, float target) {
  int lo = 0, hi = Z;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cdf[mid] > target) hi = mid; else lo = mid + 1;
  }
  return lo < Z ? lo : Z - 1;
}

__global__ void k_od_sample(const float *cdf_d, const float *cdf_o, const int *zone_edge, int Z, int n, int t_span,
                            unsigned long long seed, int *orig, int *dest, int *tdep) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const unsigned long long kk = (unsigned long long)(unsigned)k;
  const float uo = __fmul_rn((float)(uint32_t)(od_mix(seed ^ 0x5851F42D4C957F2DULL ^ kk) >> 40), 0x1p-24f);
  const int i = od_first_above(cdf_o, Z, __fmul_rn(uo, cdf_o[Z - 1]));
  const float *row = cdf_d + (long long)i * Z;
  int j = i;   // no reachable destination: the trip stays at home
  if (row[Z - 1] > 0.f) {
    const float ud = __fmul_rn((float)(uint32_t)(od_mix(seed ^ 0x14057B7EF767814FULL ^ kk) >> 40), 0x1p-24f);
    j = od_first_above(row, Z, __fmul_rn(ud, row[Z - 1]));
  }
  const unsigned long long ut = od_mix(seed ^ 0x2545F4914F6CDD1DULL ^ kk) >> 40;
  orig[k] = zone_edge[i];
  dest[k] = zone_edge[j];
  tdep[k] = (int)((ut * (unsigned long long)t_span) >> 24);
}

}  // namespace moss
