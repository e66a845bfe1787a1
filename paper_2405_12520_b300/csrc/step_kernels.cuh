// step_kernels.cuh -- CUDA kernels of one simulation step (sm_103a).
//
// The step of Sec. III-A (prepare phase + update phase) is laid out for HBM as four
// kernels over a vehicle state that is kept physically sorted by (lane, x):
//
//   k_decide  (update phase, pass 1)  one thread per vehicle in sorted order: sense the
//             own-path leader and the target-lane neighbours from the read-only snapshot,
//             IDM + randomized MOBIL + stop lines + ballistic advance + transfer; emit a
//             leave bit per vehicle (warp ballot) and a record per vehicle that changes
//             lane; per-lane window metrics by the first vehicle of each lane.
//   k_lanes   (prepare phase for t+1)  decoupled look-back scan over lanes: new per-lane
//             counts = stayers + arrivals + departures, new segment starts, arrival bucket
//             starts; departure FIFOs admit their head vehicle.
//   k_bucket  place each arrival record into its lane's bucket with its rank among the
//             lane's stayers.
//   k_apply   (update phase, pass 2) recompute the same update (bit-identical) and write
//             each vehicle straight to its sorted slot of the t+1 buffer.
//
// Stayers keep their relative order (no overtaking within a lane), so the t+1 order is a
// merge of the stayers with the few arrivals; no full sort is needed.
#pragma once
#include <cstdint>
#include <cuda/atomic>
#include <cuda_runtime.h>

namespace moss {

enum { SIG_G = 0, SIG_Y = 1, SIG_R = 2 };
enum { K_FREE = 0, K_VEH = 1, K_OBST = 2 };
enum { U_STAY = 0, U_CHANGE = 1, U_TRANSFER = 2, U_RETIRE = 3 };
constexpr int HOP_CAP = 12;          // lanes searched ahead for a leader
constexpr float FLAG_EPS = 1e-3f;    // decision margins closer than this are flagged
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr int SPIN_LIMIT = 1 << 22;  // bounded wait of the look-back
constexpr int AMIN_NONE = 0x7fffffff;

constexpr unsigned DEV_HOP = 1u, DEV_SCAN = 2u, DEV_ORDER = 4u, DEV_BUCKET = 8u;

// Static lane record, one 32-byte sector per lane.
struct __align__(32) LaneInfo {
  float len;
  int edge;     // -1 for junction-internal lanes
  int left;     // -1 none
  int right;    // -1 none
  int succ;     // edge lane: first entry in succ[]; internal lane: its target lane
  int pred;     // first entry in pred[] of the internal lanes feeding this lane
  int ctrl;     // signal controller at the lane end, -1 none
  unsigned char n_succ, n_pred, group, idx;
};

struct DevParams {
  float dt, L, a, b, T, s0, p, th, bsafe, a_min, v_max, d_look, x_lc_min, x_lc_end;
  float inv2sqrtab;      // 1 / (2 sqrt(a b))
  uint32_t lc_thresh;    // floor(p_lc * 2^24)
  unsigned long long seed;
  int window, n_windows, debug, n_lanes;
};

struct Soa {
  float *x, *v, *v0;
  int *lane, *rp, *nxt, *id;
};

struct DevCtrl {
  int t;             // step the next k_decide computes
  int t_apply;       // step being applied (set by k_lanes, read by k_bucket / k_apply)
  int n_active[2];   // vehicles in buffer 0 / 1
  int n_movers;
  int tile_ticket;
  unsigned err;
  int movers_last;
  unsigned long long inserted, arrived, sum_tt;
};

struct Mover {
  int i, lane;
  float xnew, xold;
  int k, kind;
};

struct DebugOut {
  int *id, *lead_kind, *lead_id, *lc_dir, *lc_cand, *tau_lead, *tau_foll, *old_foll, *flag;
  float *s_own, *vl_own, *a_own, *incentive, *a_use;
  int *trip_ins, *trip_flag;   // step stamps (t+1) per trip id
  int *arr_flag;               // per lane: a flagged vehicle enters it this step
};

struct StepArgs {
  const LaneInfo *li;
  const int2 *succ;    // {internal lane, exit edge}
  const int *pred;
  const int4 *ctrl4;   // {offset, green, yellow, nphase}
  const int *routes;   // per trip: its edges then -1
  Soa A[2];
  int2 *dyn[2];        // per lane {segment start, count} for buffer 0 / 1
  DevCtrl *ctrl;
  unsigned *leave;
  int *arr_cnt, *amin, *arr_start;
  Mover *movers;
  int4 *bucket;        // {r, x bits, id, old index}
  int *tile_flag;
  unsigned long long *tile_agg, *tile_pre;
  const int *q_off, *q_trip;
  int *q_head;
  const int *trip_tdep, *trip_route0;
  const float *trip_v0;
  int *t_arr;
  float *vsum;
  int *vcnt;
  DebugOut dbg;
  DevParams P;
};

// ------------------------------------------------------------------------------------
// model (FP32)
// ------------------------------------------------------------------------------------

__device__ __forceinline__ void mark(int &f, float m) {
  if (fabsf(m) < FLAG_EPS) f = 1;
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// order-preserving int key of a float (for atomicMin on possibly negative values)
__device__ __forceinline__ int fkey(float f) {
  int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float unfkey(int k) {
  return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
}

__device__ __forceinline__ float idm(const DevParams &P, float v, float v0, bool has, float gap,
                                     float vl) {
  float r = v / v0;
  float r2 = r * r;
  float fr = 1.f - r2 * r2;
  float acc;
  if (!has) {
    acc = P.a * fr;
  } else {
    float dv = v - vl;
    float ss = P.s0 + fmaxf(0.f, v * P.T + v * dv * P.inv2sqrtab);
    float q = ss / fmaxf(gap, 0.01f);
    acc = P.a * (fr - q * q);
  }
  return fmaxf(acc, P.a_min);
}

__device__ __forceinline__ int sig_state(const StepArgs &a, const LaneInfo &li, int t) {
  if (li.ctrl < 0) return SIG_G;
  int4 c = a.ctrl4[li.ctrl];
  int gy = c.y + c.z;
  int cyc = c.w * gy;
  int tau = ((t + c.x) % cyc + cyc) % cyc;
  if (tau / gy != (int)li.group) return SIG_R;
  return (tau % gy) < c.y ? SIG_G : SIG_Y;
}

// edge lane l has a link toward edge en (en < 0: route ends, always true)
__device__ __forceinline__ bool connects(const StepArgs &a, const LaneInfo &li, int en) {
  if (en < 0) return true;
  for (int k = 0; k < li.n_succ; ++k)
    if (a.succ[li.succ + k].y == en) return true;
  return false;
}

// fan-out link of edge lane l toward en: the first whose target lane serves en2
__device__ __forceinline__ int choose_succ(const StepArgs &a, const LaneInfo &li, int en, int en2) {
  int first = -1;
  for (int k = 0; k < li.n_succ; ++k) {
    int2 s = a.succ[li.succ + k];
    if (s.y != en) continue;
    if (first < 0) first = s.x;
    if (en2 < 0) return s.x;
    int tg = a.li[s.x].succ;
    if (connects(a, a.li[tg], en2)) return s.x;
  }
  return first;
}

struct Lead {
  int kind;
  float gap, vl;
  int j;          // sorted index of the leader, -1 none / obstacle
  int end_obst;   // obstacle at the end of the own lane
};

struct LC {
  int dir, cand, tl, tf, of;
  float inc;
  int tkind;
  float tgap, tvl, anew;
};

struct Upd {
  int kind, lane, rp, nxt;
  float x, v, a_use, a_own;
  Lead own;
  LC lc;
  int flag;
};

__device__ __forceinline__ Lead own_leader(const StepArgs &a, const Soa &S, const int2 *dyn, int i,
                                           int l, const LaneInfo &li, float x, float v, int rp,
                                           int en, int myid, int t, int &flag) {
  const DevParams &P = a.P;
  Lead r{K_FREE, 0.f, 0.f, -1, 0};
  int2 d = dyn[l];
  if (i + 1 < d.x + d.y) {
    int j = i + 1;
    r = Lead{K_VEH, (S.x[j] - x) - P.L, S.v[j], j, 0};
  } else {
    float dist = li.len - x;
    int ri = rp, e_next = en;
    LaneInfo lc = li;
    for (int hop = 0;; ++hop) {
      mark(flag, dist - P.d_look);
      if (dist >= P.d_look) break;
      int nxt;
      if (lc.edge >= 0) {
        if (e_next < 0) break;   // destination edge: open end
        nxt = choose_succ(a, lc, e_next, a.routes[ri + 2]);
        bool stop = nxt < 0;
        if (!stop) {
          int sg = sig_state(a, lc, t);
          if (sg == SIG_R) {
            stop = true;
          } else if (sg == SIG_Y) {
            float m = dist - v * v / (2.f * P.b);
            mark(flag, m);
            stop = m >= 0.f;
          }
        }
        if (stop) {
          r = Lead{K_OBST, dist, 0.f, -1, hop == 0};
          break;
        }
      } else {
        nxt = lc.succ;
        ri += 1;
        e_next = a.routes[ri + 1];
      }
      if (hop + 1 >= HOP_CAP) {
        r = Lead{K_OBST, dist, 0.f, -1, hop == 0};
        break;
      }
      int2 dn = dyn[nxt];
      if (dn.y > 0) {
        int j = dn.x;
        r = Lead{K_VEH, (dist + S.x[j]) - P.L, S.v[j], j, 0};
        break;
      }
      lc = a.li[nxt];
      dist += lc.len;
    }
  }
  // merge projection (vehicle on an internal lane feeding a multi-feeder lane)
  if (li.edge < 0) {
    LaneInfo lt = a.li[li.succ];
    if (lt.n_pred > 1) {
      float dc = li.len - x;
      for (int q = 0; q < lt.n_pred; ++q) {
        int f = a.pred[lt.pred + q];
        if (f == l) continue;
        int2 df = dyn[f];
        float lf = a.li[f].len;
        int found = -1;
        for (int jj = 0; jj < df.y; ++jj) {
          int j = df.x + jj;
          float dj = lf - S.x[j];
          mark(flag, dc - dj);
          if (dj < dc || (dj == dc && S.id[j] < myid)) {
            found = j;
            break;
          }
        }
        if (found >= 0) {
          float dj = lf - S.x[found];
          float g = (dc - dj) - P.L;
          if (r.kind != K_FREE) mark(flag, g - r.gap);
          if (r.kind == K_FREE || g < r.gap) r = Lead{K_VEH, g, S.v[found], found, 0};
        }
      }
    }
  }
  return r;
}

// target lane end blocks a vehicle at (x, v) heading for edge en
__device__ __forceinline__ bool end_blocks(const StepArgs &a, const LaneInfo &lt, int en, float x,
                                           float v, int t, int &flag) {
  if (en < 0) return false;
  if (!connects(a, lt, en)) return true;
  int sg = sig_state(a, lt, t);
  if (sg == SIG_R) return true;
  if (sg == SIG_Y) {
    float m = (lt.len - x) - v * v / (2.f * a.P.b);
    mark(flag, m);
    return m >= 0.f;
  }
  return false;
}

__device__ __forceinline__ LC lane_change(const StepArgs &a, const Soa &S, const int2 *dyn, int i,
                                          int l, const LaneInfo &li, float x, float v, float v0,
                                          int en, int myid, int t, const Lead &own, float a_c,
                                          int &flag) {
  const DevParams &P = a.P;
  LC r{};
  r.tl = r.tf = r.of = -1;
  if (li.edge < 0) return r;
  int step_dir = (t % 2 == 0) ? 1 : -1;
  int tau = step_dir > 0 ? li.left : li.right;
  if (tau < 0) return r;
  bool mand = !connects(a, li, en);
  if (mand) {
    int dr = 1 << 30, dl = 1 << 30, k = 1;
    for (int q = li.right; q >= 0; q = a.li[q].right, ++k)
      if (connects(a, a.li[q], en)) { dr = k; break; }
    k = 1;
    for (int q = li.left; q >= 0; q = a.li[q].left, ++k)
      if (connects(a, a.li[q], en)) { dl = k; break; }
    if (dr == (1 << 30) && dl == (1 << 30)) return r;
    int want = dr <= dl ? -1 : +1;
    if (want != step_dir) return r;
  }
  mark(flag, x - P.x_lc_min);
  if (x < P.x_lc_min) return r;
  const LaneInfo lt = a.li[tau];
  if (!mand) {
    if (!connects(a, lt, en)) return r;
    mark(flag, (li.len - x) - P.x_lc_end);
    if (li.len - x < P.x_lc_end) return r;
    unsigned long long h = splitmix64(P.seed ^ ((unsigned long long)(unsigned)t << 32) ^
                                      (unsigned long long)(unsigned)myid);
    if ((uint32_t)(h >> 40) >= P.lc_thresh) return r;
  }
  r.cand = 1;
  int2 dt = dyn[tau];
  int lo = dt.x, hi = dt.x + dt.y;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (S.x[mid] > x) hi = mid; else lo = mid + 1;
  }
  int Lt = lo < dt.x + dt.y ? lo : -1;
  int Ft = lo > dt.x ? lo - 1 : -1;
  r.tl = Lt;
  r.tf = Ft;
  if (Lt >= 0) {
    r.tkind = K_VEH;
    r.tgap = (S.x[Lt] - x) - P.L;
    r.tvl = S.v[Lt];
  } else if (end_blocks(a, lt, en, x, v, t, flag)) {
    r.tkind = K_OBST;
    r.tgap = li.len - x;
    r.tvl = 0.f;
  } else {
    r.tkind = K_FREE;
  }
  if (r.tkind == K_VEH) {
    mark(flag, r.tgap);
    if (r.tgap <= 0.f) return r;
  }
  float aF_new = 0.f, xF = 0.f, vF = 0.f, v0F = 1.f;
  if (Ft >= 0) {
    xF = S.x[Ft];
    vF = S.v[Ft];
    v0F = S.v0[Ft];
    float gF = (x - xF) - P.L;
    float guard = vF * P.dt + 0.5f * P.a * P.dt * P.dt;
    mark(flag, gF - guard);
    if (gF < guard) return r;
    aF_new = idm(P, vF, v0F, true, gF, v);
    mark(flag, aF_new + P.bsafe);
    if (aF_new < -P.bsafe) return r;
  }
  r.anew = idm(P, v, v0, r.tkind != K_FREE, r.tgap, r.tvl);
  if (!mand) {
    float delta = r.anew - a_c;
    if (Ft >= 0) {
      float aF_old;
      if (Lt >= 0)
        aF_old = idm(P, vF, v0F, true, (S.x[Lt] - xF) - P.L, S.v[Lt]);
      else if (end_blocks(a, lt, en, xF, vF, t, flag))
        aF_old = idm(P, vF, v0F, true, li.len - xF, 0.f);
      else
        aF_old = idm(P, vF, v0F, false, 0.f, 0.f);
      delta += P.p * (aF_new - aF_old);
    }
    int2 d = dyn[l];
    if (i > d.x) {
      int O = i - 1;
      r.of = O;
      float xO = S.x[O], vO = S.v[O], v0O = S.v0[O];
      float aO_old = idm(P, vO, v0O, true, (x - xO) - P.L, v);
      float aO_new = own.kind != K_FREE ? idm(P, vO, v0O, true, own.gap + (x - xO), own.vl)
                                        : idm(P, vO, v0O, false, 0.f, 0.f);
      delta += P.p * (aO_new - aO_old);
    }
    r.inc = delta;
    mark(flag, delta - P.th);
    if (!(delta > P.th)) return r;
  }
  r.dir = step_dir;
  return r;
}

// The update of vehicle i (snapshot index) at step t.  Pure function of the snapshot.
__device__ __forceinline__ Upd vehicle_update(const StepArgs &a, const Soa &S, const int2 *dyn, int i,
                                              int t) {
  const DevParams &P = a.P;
  Upd u;
  u.flag = 0;
  const int l = S.lane[i];
  const float x = S.x[i], v = S.v[i], v0 = S.v0[i];
  const int rp = S.rp[i], en = S.nxt[i], myid = S.id[i];
  const LaneInfo li = a.li[l];
  u.own = own_leader(a, S, dyn, i, l, li, x, v, rp, en, myid, t, u.flag);
  u.a_own = idm(P, v, v0, u.own.kind != K_FREE, u.own.gap, u.own.vl);
  u.lc = lane_change(a, S, dyn, i, l, li, x, v, v0, en, myid, t, u.own, u.a_own, u.flag);
  const int dir = u.lc.dir;
  u.a_use = dir ? fminf(u.a_own, u.lc.anew) : u.a_own;
  float vraw = v + u.a_use * P.dt;
  float vn, d;
  if (vraw > 0.f) {
    vn = fminf(vraw, P.v_max);
    d = 0.5f * (v + vn) * P.dt;
  } else {
    vn = 0.f;
    d = v > 0.f ? (v * v) / (-2.f * u.a_use) : 0.f;
  }
  float gmin = __int_as_float(0x7f800000);
  if (u.own.kind != K_FREE) gmin = u.own.gap;
  if (dir) {
    if (u.lc.tkind != K_FREE) gmin = fminf(gmin, u.lc.tgap);
    gmin = fminf(gmin, li.len - x);
  }
  float dmax = fmaxf(0.f, gmin);
  if (d > dmax) {
    d = dmax;
    vn = fminf(vn, d / P.dt);
  }
  float xn = x + d;
  if (u.own.end_obst || dir) xn = fminf(xn, li.len);
  u.kind = dir ? U_CHANGE : U_STAY;
  u.lane = dir ? (dir > 0 ? li.left : li.right) : l;
  u.rp = rp;
  u.nxt = en;
  if (!dir) {
    mark(u.flag, xn - li.len);
    if (xn > li.len) {
      if (li.edge >= 0 && en < 0) {
        u.kind = U_RETIRE;
      } else {
        xn -= li.len;
        u.kind = U_TRANSFER;
        int nl;
        if (li.edge >= 0) {
          nl = choose_succ(a, li, en, a.routes[rp + 2]);
        } else {
          nl = li.succ;
          u.rp = rp + 1;
          u.nxt = a.routes[rp + 2];
        }
        if (nl < 0 || xn > a.li[nl].len) {
          atomicOr(&a.ctrl->err, DEV_HOP);
          nl = l;
          xn = li.len;
          u.kind = U_STAY;
          u.rp = rp;
          u.nxt = en;
        }
        u.lane = nl;
      }
    }
  }
  u.x = xn;
  u.v = vn;
  return u;
}

// number of set bits of b in [s, e)
__device__ __forceinline__ int count_bits(const unsigned *b, int s, int e) {
  if (s >= e) return 0;
  int ws = s >> 5, we = (e - 1) >> 5;
  unsigned lo = 0xffffffffu << (s & 31);
  unsigned hi = 0xffffffffu >> (31 - ((e - 1) & 31));
  if (ws == we) return __popc(b[ws] & lo & hi);
  int c = __popc(b[ws] & lo);
  for (int w = ws + 1; w < we; ++w) c += __popc(b[w]);
  return c + __popc(b[we] & hi);
}

// ------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------

__global__ void k_decide(StepArgs a) {
  const int t = a.ctrl->t;
  const int p = t & 1;
  const Soa S = a.A[p];
  const int2 *dyn = a.dyn[p];
  const int n = a.ctrl->n_active[p];
  const int w = t / a.P.window;
  const bool rec = a.vsum != nullptr && w < a.P.n_windows;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const int i = base + threadIdx.x;
    int leave = 0;
    if (i < n) {
      Upd u = vehicle_update(a, S, dyn, i, t);
      const int l = S.lane[i];
      leave = u.kind != U_STAY;
      if (rec) {
        int2 d = dyn[l];
        if (i == d.x) {
          float s = 0.f;
          for (int j = d.x; j < d.x + d.y; ++j) s += S.v[j];
          size_t o = (size_t)w * a.P.n_lanes + l;
          a.vsum[o] += s;
          a.vcnt[o] += d.y;
        }
      }
      if (u.kind == U_CHANGE || u.kind == U_TRANSFER) {
        int k = atomicAdd(&a.arr_cnt[u.lane], 1);
        int slot = atomicAdd(&a.ctrl->n_movers, 1);
        a.movers[slot] = Mover{i, u.lane, u.x, S.x[i], k, u.kind};
        atomicMin(&a.amin[u.lane], fkey(u.x - a.P.L));
        if (a.P.debug && u.flag) a.dbg.arr_flag[u.lane] = 1;
      }
      if (a.P.debug) {
        a.dbg.id[i] = S.id[i];
        a.dbg.lead_kind[i] = u.own.kind;
        a.dbg.lead_id[i] = u.own.j >= 0 ? S.id[u.own.j] : -1;
        a.dbg.s_own[i] = u.own.gap;
        a.dbg.vl_own[i] = u.own.vl;
        a.dbg.a_own[i] = u.a_own;
        a.dbg.lc_dir[i] = u.lc.dir;
        a.dbg.lc_cand[i] = u.lc.cand;
        a.dbg.tau_lead[i] = u.lc.tl >= 0 ? S.id[u.lc.tl] : -1;
        a.dbg.tau_foll[i] = u.lc.tf >= 0 ? S.id[u.lc.tf] : -1;
        a.dbg.old_foll[i] = u.lc.of >= 0 ? S.id[u.lc.of] : -1;
        a.dbg.incentive[i] = u.lc.inc;
        a.dbg.a_use[i] = u.a_use;
        a.dbg.flag[i] = u.flag;
      }
    }
    unsigned m = __ballot_sync(0xffffffffu, leave);
    if ((threadIdx.x & 31) == 0) a.leave[(base + threadIdx.x) >> 5] = m;
  }
}

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += y;
  }
  return v;
}

// Lane pass: new per-lane counts, decoupled look-back scan, departures.
__global__ void __launch_bounds__(SCAN_THREADS) k_lanes(StepArgs a) {
  __shared__ int s_tile;
  __shared__ unsigned long long s_warp[SCAN_THREADS / 32];
  __shared__ unsigned long long s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(&a.ctrl->tile_ticket, 1);
  __syncthreads();
  const int tile = s_tile;
  const int t = a.ctrl->t;
  const int p = t & 1;
  const Soa S = a.A[p];
  const Soa D = a.A[p ^ 1];
  const int2 *dyn = a.dyn[p];
  int2 *ndyn = a.dyn[p ^ 1];
  const int nl = a.P.n_lanes;
  const float room_need = a.P.L + a.P.s0;
  const int l0 = tile * SCAN_TILE + threadIdx.x * SCAN_ITEMS;

  int cnt[SCAN_ITEMS], arr[SCAN_ITEMS], ins[SCAN_ITEMS];
  unsigned long long run = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int l = l0 + k;
    cnt[k] = arr[k] = ins[k] = 0;
    if (l < nl) {
      int2 d = dyn[l];
      int leavers = count_bits(a.leave, d.x, d.x + d.y);
      arr[k] = a.arr_cnt[l];
      int qh = a.q_head[l];
      if (qh < a.q_off[l + 1]) {
        int trip = a.q_trip[qh];
        if (a.trip_tdep[trip] <= t) {
          int fl = 0;
          bool room = true;
          if (d.y > 0) {
            float m = (S.x[d.x] - a.P.L) - room_need;
            mark(fl, m);
            room = m >= 0.f;
          }
          int ak = a.amin[l];
          if (ak != AMIN_NONE) {
            float m = unfkey(ak) - room_need;
            mark(fl, m);
            if (m < 0.f) room = false;
          }
          if (a.P.debug && (fl || a.dbg.arr_flag[l])) a.dbg.trip_flag[trip] = t + 1;
          ins[k] = room ? 1 : 0;
        }
      }
      cnt[k] = d.y - leavers + arr[k] + ins[k];
      run += ((unsigned long long)cnt[k] << 32) | (unsigned)(arr[k] + ins[k]);
    }
  }
  // block-wide exclusive scan of the packed (count, arrivals) pairs
  unsigned long long incl = warp_incl_scan(run);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long wv = lane < SCAN_THREADS / 32 ? s_warp[lane] : 0ull;
    unsigned long long wi = warp_incl_scan(wv);
    if (lane < SCAN_THREADS / 32) s_warp[lane] = wi - wv;   // exclusive warp offsets
    if (lane == SCAN_THREADS / 32 - 1) {
      // decoupled look-back for the tile prefix
      const unsigned long long agg = wi;
      cuda::atomic_ref<int, cuda::thread_scope_device> myflag(a.tile_flag[tile]);
      unsigned long long excl = 0;
      if (tile == 0) {
        a.tile_pre[0] = agg;
        myflag.store(2, cuda::memory_order_release);
      } else {
        a.tile_agg[tile] = agg;
        myflag.store(1, cuda::memory_order_release);
        int j = tile - 1, spins = 0;
        while (j >= 0) {
          cuda::atomic_ref<int, cuda::thread_scope_device> f(a.tile_flag[j]);
          int fv = f.load(cuda::memory_order_acquire);
          if (fv == 0) {
            if (++spins > SPIN_LIMIT) {
              atomicOr(&a.ctrl->err, DEV_SCAN);
              break;
            }
            continue;
          }
          if (fv == 2) {
            excl += a.tile_pre[j];
            break;
          }
          excl += a.tile_agg[j];
          --j;
        }
        a.tile_pre[tile] = excl + agg;
        myflag.store(2, cuda::memory_order_release);
      }
      s_excl = excl;
    }
  }
  __syncthreads();
  unsigned long long pre = s_excl + s_warp[warp] + (incl - run);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int l = l0 + k;
    if (l >= nl) break;
    const int nstart = (int)(pre >> 32);
    const int astart = (int)(pre & 0xffffffffu);
    ndyn[l] = make_int2(nstart, cnt[k]);
    a.arr_start[l] = astart;
    if (ins[k]) {
      int qh = a.q_head[l];
      int trip = a.q_trip[qh];
      a.q_head[l] = qh + 1;
      int r0 = a.trip_route0[trip];
      D.x[nstart] = a.P.L;
      D.v[nstart] = 0.f;
      D.v0[nstart] = a.trip_v0[trip];
      D.lane[nstart] = l;
      D.rp[nstart] = r0;
      D.nxt[nstart] = a.routes[r0 + 1];
      D.id[nstart] = trip;
      a.bucket[astart + arr[k]] = make_int4(0, __float_as_int(a.P.L), trip, -1);
      atomicAdd(&a.ctrl->inserted, 1ull);
      if (a.P.debug) a.dbg.trip_ins[trip] = t + 1;
    }
    a.arr_cnt[l] = 0;
    a.amin[l] = AMIN_NONE;
    if (a.P.debug) a.dbg.arr_flag[l] = 0;
    pre += ((unsigned long long)cnt[k] << 32) | (unsigned)(arr[k] + ins[k]);
    if (l == nl - 1) {
      a.ctrl->n_active[p ^ 1] = (int)(pre >> 32);
      a.arr_start[nl] = (int)(pre & 0xffffffffu);
      a.ctrl->t_apply = t;
    }
  }
}

// Arrival records -> lane buckets with their rank among the lane's stayers.
__global__ void k_bucket(StepArgs a, int n_tiles) {
  const int t = a.ctrl->t_apply;
  const int p = t & 1;
  const Soa S = a.A[p];
  const int2 *dyn = a.dyn[p];
  const int nm = a.ctrl->n_movers;
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  for (int m = gid; m < nm; m += stride) {
    Mover mv = a.movers[m];
    int r = 0;
    if (mv.kind == U_CHANGE) {
      int2 d = dyn[mv.lane];
      int lo = d.x, hi = d.x + d.y;
      while (lo < hi) {   // first vehicle of the target lane not behind the changer
        int mid = (lo + hi) >> 1;
        if (S.x[mid] < mv.xold) lo = mid + 1; else hi = mid;
      }
      r = (lo - d.x) - count_bits(a.leave, d.x, lo);
    }
    a.bucket[a.arr_start[mv.lane] + mv.k] = make_int4(r, __float_as_int(mv.xnew), S.id[mv.i], mv.i);
  }
  for (int k = gid; k < n_tiles; k += stride) a.tile_flag[k] = 0;
  if (gid == 0) {
    a.ctrl->movers_last = nm;
    a.ctrl->t = t + 1;
    a.ctrl->tile_ticket = 0;
  }
}

__device__ __forceinline__ bool bucket_less(int4 f, int4 e) {
  if (f.x != e.x) return f.x < e.x;
  float fx = __int_as_float(f.y), ex = __int_as_float(e.y);
  if (fx != ex) return fx < ex;
  return f.z < e.z;
}

// Recompute the update and write each vehicle to its sorted slot of the t+1 buffer.
__global__ void k_apply(StepArgs a) {
  const int t = a.ctrl->t_apply;
  const int p = t & 1;
  const Soa S = a.A[p];
  const Soa D = a.A[p ^ 1];
  const int2 *dyn = a.dyn[p];
  const int2 *ndyn = a.dyn[p ^ 1];
  const int n = a.ctrl->n_active[p];
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  if (gid == 0) a.ctrl->n_movers = 0;
  for (int i = gid; i < n; i += stride) {
    Upd u = vehicle_update(a, S, dyn, i, t);
    const int id = S.id[i];
    if (u.kind == U_RETIRE) {
      a.t_arr[id] = t + 1;
      atomicAdd(&a.ctrl->arrived, 1ull);
      atomicAdd(&a.ctrl->sum_tt, (unsigned long long)(t + 1 - a.trip_tdep[id]));
      continue;
    }
    int pos;
    if (u.kind == U_STAY) {
      const int l = u.lane;
      int2 d = dyn[l];
      int k = (i - d.x) - count_bits(a.leave, d.x, i);
      int bs = a.arr_start[l], be = a.arr_start[l + 1];
      int m = 0;
      for (int q = bs; q < be; ++q) m += a.bucket[q].x <= k;
      pos = ndyn[l].x + k + m;
    } else {
      int bs = a.arr_start[u.lane], be = a.arr_start[u.lane + 1];
      int4 me = make_int4(0, 0, 0, -2);
      for (int q = bs; q < be; ++q) {
        int4 f = a.bucket[q];
        if (f.w == i) { me = f; break; }
      }
      if (me.w != i) {
        atomicOr(&a.ctrl->err, DEV_BUCKET);
        continue;
      }
      int rank = 0;
      for (int q = bs; q < be; ++q) rank += bucket_less(a.bucket[q], me);
      pos = ndyn[u.lane].x + me.x + rank;
    }
    D.x[pos] = u.x;
    D.v[pos] = u.v;
    D.v0[pos] = S.v0[i];
    D.lane[pos] = u.lane;
    D.rp[pos] = u.rp;
    D.nxt[pos] = u.nxt;
    D.id[pos] = id;
  }
}

// Debug check of the t+1 buffer: sorted by (lane, x), gap >= 0 (up to float rounding).
__global__ void k_check(StepArgs a) {
  const int t = a.ctrl->t;   // already advanced
  const int p = t & 1;
  const Soa S = a.A[p];
  const int n = a.ctrl->n_active[p];
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = gid; i + 1 < n; i += gridDim.x * blockDim.x) {
    int la = S.lane[i], lb = S.lane[i + 1];
    if (la > lb || (la == lb && (S.x[i + 1] - a.P.L) - S.x[i] < -1e-3f))
      atomicOr(&a.ctrl->err, DEV_ORDER);
  }
}

__global__ void k_route_idx(const int *rp, const int *id, const int *route0, int *out, const int *n_ptr,
                            int n_fixed) {
  int n = n_ptr ? *n_ptr : n_fixed;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = rp[i] - route0[id[i]];
}

}  // namespace moss
