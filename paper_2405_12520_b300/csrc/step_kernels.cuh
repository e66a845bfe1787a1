// step_kernels.cuh -- CUDA kernels of one simulation step (sm_103a).
//
// The step of Sec. III-A (prepare phase + update phase) is laid out for HBM as four
// kernels over a vehicle state that is kept physically sorted by (lane, x):
//
//   k_decide  (update phase)  one thread per vehicle in sorted order: sense the own-path
//             leader and the target-lane neighbours from the read-only snapshot, IDM +
//             randomized MOBIL + stop lines + ballistic advance + transfer; store the
//             vehicle's result (x', v', new lane and kind: 12 B), a leave bit per vehicle
//             (warp ballot), per-lane arrival counts and rearmost arrival (fire-and-forget
//             atomics); per-lane window metrics by the first vehicle of each lane.
//   k_lanes   (prepare phase for t+1)  a scan over lanes in two launches: pass 0 writes each
//             tile's aggregate, pass 1 sums its predecessors' and writes the new per-lane
//             counts = stayers + arrivals + departures, segment starts, arrival bucket
//             starts; departure FIFOs admit their head; the signal table of step t+1.
//   k_bucket  place each arrival record into its lane's bucket with its rank among the
//             lane's stayers.
//   k_apply   stream every vehicle with its stored result to its sorted slot of the t+1
//             buffer (no sensing repeated).
//
// Stayers keep their relative order (no overtaking within a lane), so the t+1 order is a
// merge of the stayers with the few arrivals; no full sort is needed.
#pragma once
#include <climits>
#include <cstdint>
#include <cuda/atomic>
#include <cuda_runtime.h>

#include "mlp_kernels.cuh"
#include "tma.cuh"

namespace moss {

enum { SIG_G = 0, SIG_Y = 1, SIG_R = 2 };
enum { K_FREE = 0, K_VEH = 1, K_OBST = 2 };
enum { U_STAY = 0, U_CHANGE = 1, U_TRANSFER = 2, U_RETIRE = 3 };
constexpr int HOP_CAP = 12;          // lanes searched ahead for a leader
constexpr float FLAG_EPS = 1e-3f;    // decision margins closer than this are flagged
// lane pass: tiles of LANE_TILE lanes, LANE_THREADS threads with LANE_ITEMS lanes each
constexpr int LANE_THREADS = 256;
constexpr int LANE_ITEMS = 4;
constexpr int LANE_TILE = LANE_THREADS * LANE_ITEMS;
constexpr int LANE_WARPS = LANE_THREADS / 32;

constexpr int AMIN_NONE = 0x7fffffff;

constexpr unsigned DEV_HOP = 1u, DEV_SCAN = 2u, DEV_ORDER = 4u, DEV_BUCKET = 8u, DEV_TIMEOUT = 16u;
constexpr int LEAVE_ONE = 1 << 16;   // a leaver in the per-lane arrival word

// Static lane record, one 32-byte sector per lane.
struct __align__(32) LaneInfo {
  float len;
  int edge;     // -1 for junction-internal lanes
  int left;     // edge lane: lane to the left, -1 none; internal lane: tsucc, the first
                // successor entry of its target lane
  int right;    // edge lane: lane to the right, -1 none; internal lane: tn_succ, the
                // number of successor entries of its target lane
  int succ;     // edge lane: first entry in succ[]; internal lane: its target lane
  int pred;     // first entry in pred[] of the internal lanes feeding this lane
  int ctrl;     // signal controller at the lane end, -1 none
  unsigned char n_succ, n_pred, group;
  unsigned char idx;   // edge lane: position across its edge (0 = rightmost, by the right
                       // links); internal lane: its target lane's position
};

struct DevParams {
  float dt, L, a, b, T, s0, p, th, bsafe, a_min, v_max, d_look, x_lc_min, x_lc_end;
  float inv2sqrtab;      // 1 / (2 sqrt(a b))
  float inv2b;           // 1 / (2 b): braking distance v^2 / (2 b) as a product
  uint32_t lc_thresh;    // floor(p_lc * 2^24)
  unsigned long long seed;
  int window, n_windows, debug, n_lanes;
  int id_base;           // added to trip ids in the lane-change gate hash
  float th_jitter;       // half-width of each trip's incentive-threshold offset (0: off)
  int signal_mode;       // 0 fixed-time plans, 1 max pressure
  int mp_interval;       // steps between max-pressure decisions
  int lane_mods;         // some lane has a speed limit or is closed
  int fifo;              // some trip enters through a departure queue
  int test_withhold;     // test of the timeout path: k_apply issues no bulk copy, so its
                         // waits run out (after a short limit) and report MS_DEV_TIMEOUT
};

// Link plan of a route entry r (edge e = routes[r]), one 64-bit word built at load time:
// field q (bits 6q..6q+5) is, for the lane at position q of e, the index among that lane's
// successor entries of the link the trip takes toward routes[r + 1] (the first such link
// whose target lane serves routes[r + 2], else the first one), PLAN_NONE if the lane has no
// link toward it; bit 63 (PLAN_END) is set when the route ends on e.  It turns every
// link search of the step (next-lane choice, mandatory and discretionary lane-change
// checks, look-ahead hops) into one field extract and at most one successor load.
constexpr int PLAN_BITS = 6;
constexpr unsigned PLAN_NONE = (1u << PLAN_BITS) - 1u;   // also bounds a lane's link count
constexpr unsigned long long PLAN_END = 1ull << 63;
constexpr int PLAN_LANES = 10;                            // lanes per edge
__host__ __device__ __forceinline__ unsigned plan_nib(unsigned long long pl, int q) {
  return (unsigned)(pl >> (PLAN_BITS * q)) & PLAN_NONE;
}
// lane at position q of the plan's edge can continue the route (the route ends here, or
// the lane has a link toward the next edge)
__device__ __forceinline__ bool plan_ok(unsigned long long pl, int q) {
  return (pl & PLAN_END) || plan_nib(pl, q) != PLAN_NONE;
}

// Vehicle state, sorted by (lane, x).  rp: index into routes[] of the current edge (the
// approach edge on an internal lane); pl = plan[rp]; nl: the lane the vehicle will enter at
// the end of its current edge lane (for an internal lane: at the end of its target lane);
// NL_END (-1) if the route ends on that edge, NL_NONE (-2) if that lane has no link toward
// the next route edge -- cached so that sensing needs no route or link lookups.
constexpr int NL_END = -1, NL_NONE = -2;
struct Soa {
  float *x, *v, *v0;
  int *lane, *rp;
  unsigned long long *pl;
  int *nl, *id;
};

struct DevCtrl {
  int t;             // step the next k_decide computes
  int t_apply;       // step being applied (set by k_lanes, read by k_bucket / k_apply)
  int n_active[2];   // vehicles in buffer 0 / 1
  int n_movers;      // arrivals of the last step (count only)
  unsigned err;
  int movers_last;
  int n_cand;        // discretionary candidates listed for k_learn this step (reset by k_apply)
  unsigned long long inserted, arrived, sum_tt;
};

struct DebugOut {
  int *id, *lead_kind, *lead_id, *lc_dir, *lc_cand, *tau_lead, *tau_foll, *old_foll, *flag;
  float *s_own, *vl_own, *a_own, *incentive, *a_use;
  int *trip_ins, *trip_flag;   // step stamps (t+1) per trip id
  int *arr_flag;               // per lane: a flagged vehicle enters it this step
  // learned lane change: 1 where the network decided; its softmax margin, logits [3 per
  // vehicle] and BF16 inputs [16 per vehicle]
  int *lc_learn;
  float *lc_margin, *lc_logit, *lc_feat;
};

// Per-vehicle result of k_decide, consumed by k_apply: new x, new v, and a code word
// (new lane in bits 0..28, kind in bits 29..31).
constexpr int CODE_LANE_BITS = 29;
constexpr int CODE_LANE_MASK = (1 << CODE_LANE_BITS) - 1;
enum { C_STAY = 0, C_CHANGE = 1, C_TRANSFER = 2, C_TRANSFER_ROUTE = 3, C_RETIRE = 4 };

// learned lane change: decision log (training data), model, agreement statistics
enum { MODE_PLAIN = 0, MODE_LOG = 1, MODE_LEARN = 2 };
enum { ST_CAND = 0, ST_FALLBACK = 1, ST_AGREE = 2, ST_CONF = 3 };   // ST_CONF + 3*rule + final
constexpr int LC_STATS = 12;

struct LcAux {
  __nv_bfloat16 *log_x;   // [cap][16]
  int *log_y;             // [cap]
  int log_cap;
  int *log_n;             // samples offered (may exceed cap; extra ones are dropped)
  const MlpDev *model;
  float margin;           // softmax top1 - top2 below which the rule decides
  unsigned long long *stats;
  int *cand;              // [cand_cap] vehicles whose update k_learn finishes
  void *rec_u, *rec_c;    // [cand_cap] sensing results (Upd) and fields (VCtx), by vehicle index
  int cand_cap;
};

struct StepArgs {
  const LaneInfo *li;
  const int2 *succ;    // {internal lane, exit edge}
  const unsigned char *link_off;   // per successor entry: 1 = closed (dynamic lanes)
  const int *pred;
  const int4 *ctrl4;   // {offset, green, yellow, nphase}
  int *sig[2];         // per controller, for the steps of parity 0 / 1: 2 * phase + yellow
  int n_ctrl;
  int4 *mp;            // max-pressure controllers: {green phase, pending phase or -1, step
                       // the pending phase turns green, 0}
  const int *ctrl_loff, *ctrl_lanes;   // approach edge lanes of each controller (CSR)
  const float *lane_vmax;              // per lane speed limit (+inf: none)
  const unsigned char *lane_closed;    // per lane: closed to entering vehicles
  const int *routes;   // per trip: its edges then -1
  const unsigned long long *plan;   // link plan per routes[] entry
  Soa A[2];
  int4 *dyn[2];        // per lane {first index, count, tail x, tail v} for buffer 0 / 1
  DevCtrl *ctrl;
  unsigned *leave;
  int *arr_cnt;        // per lane: arrivals (bits 0..15) + leavers (bits 16..30) of the step
  int *amin, *arr_start;
  int4 *bucket;        // {r, x bits, id, old index}
  float *res_x, *res_v;
  int *res_code;
  int *arr_fill;       // per lane: arrival slots handed out by k_bucket (reset by k_apply)
  int *res_code_nl;    // next-lane choice of arrivals, written by k_decide (sparse)
  int2 *res_pos;       // lane changers: {target segment start, first target index not
                       // behind the changer}, written by k_decide (sparse)
  unsigned long long *tile_agg;    // per lane tile: {new vehicles, arrivals} packed
  const int *q_off, *q_trip;
  int2 *q_hd;          // per lane: {FIFO head entry, its departure step (INT_MAX if empty)}
  const int4 *q_ent;   // per FIFO entry: {trip, route start, next-lane choice, v0 bits}
  const int4 *q_ent2;  // per FIFO entry: {plan of the first edge (lo, hi), departure step
                       // of the lane's next entry or INT_MAX, 0}
  const int *trip_tdep;
  int *t_arr;
  unsigned long long *vsum;   // per window x lane: sum of speeds in units of 2^-24 m/s
  int *vcnt;
  DebugOut dbg;
  LcAux lc;
  DevParams P;
};

// Programmatic dependent launch: the step's kernels are launched so that each may start
// while the previous one drains.  A kernel first waits here until the previous kernel has
// completed and its writes are visible (everything before that point touches nothing it
// wrote), then lets its own dependents launch; they can only start once all of its blocks
// have started, so they never take a slot a block of this kernel still needs.  Both are
// no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

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

// free-road term of the IDM, 1 - (v/v0)^4 (shared by the IDM calls of one vehicle at one
// desired speed).  Fast division (2 ulp): the FP32 path is compared with the FP64 oracle at
// 1e-4, and decisions this close to a threshold are flagged either way.
__device__ __forceinline__ float idm_free(float v, float v0) {
  const float r = __fdividef(v, v0);
  const float r2 = r * r;
  return 1.f - r2 * r2;
}

// IDM acceleration from the free-road term fr
__device__ __forceinline__ float idm_fr(const DevParams &P, float fr, float v, bool has, float gap, float vl) {
  float acc;
  if (!has) {
    acc = P.a * fr;
  } else {
    float dv = v - vl;
    float ss = P.s0 + fmaxf(0.f, v * P.T + v * dv * P.inv2sqrtab);
    float q = __fdividef(ss, fmaxf(gap, 0.01f));
    acc = P.a * (fr - q * q);
  }
  return fmaxf(acc, P.a_min);
}

__device__ __forceinline__ float idm(const DevParams &P, float v, float v0, bool has, float gap, float vl) {
  return idm_fr(P, idm_free(v, v0), v, has, gap, vl);
}

// Fixed-time signal of controller c at step t (Sec. III-A, traffic lights): the cycle of
// nphase phases of green + yellow seconds, shifted by offset; phase index and whether its
// yellow is on, packed as 2 * phase + yellow.
__host__ __device__ __forceinline__ int sig_pack(int4 c, int t) {
  const int gy = c.y + c.z;
  const int cyc = c.w * gy;
  const int tau = ((t + c.x) % cyc + cyc) % cyc;
  return 2 * (tau / gy) + ((tau % gy) >= c.y ? 1 : 0);
}
// state of the signal group `group` of controller ctrl at step t, from the table of that
// step's parity (k_lanes of step t - 1 or the host wrote it)
__device__ __forceinline__ int sig_state(const StepArgs &a, int ctrl, int group, int t) {
  if (ctrl < 0) return SIG_G;
  const int pk = a.sig[t & 1][ctrl];
  if ((pk >> 1) != group) return SIG_R;
  return (pk & 1) ? SIG_Y : SIG_G;
}
__device__ __forceinline__ int sig_state(const StepArgs &a, const LaneInfo &li, int t) {
  return sig_state(a, li.ctrl, (int)li.group, t);
}

// Lane entered at the end of the edge lane at plan position q with successor entries from
// sb, following plan word pl: NL_END if the route ends there, NL_NONE if it has no link.
__device__ __forceinline__ int plan_next(const StepArgs &a, unsigned long long pl, int q, int sb) {
  if (pl & PLAN_END) return NL_END;
  const unsigned k = plan_nib(pl, q);
  return k == PLAN_NONE ? NL_NONE : a.succ[sb + k].x;
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
  int safe, mand, step_dir;   // safety passed; mandatory change; direction allowed this step
  float gF, vF, aFn;          // new follower: gap, speed, acceleration behind the changer
  int tfirst, pos;            // target segment start; first target index with x' >= x
};

// Neighbours in the sorted order, exchanged within the warp: vehicle i + 1 (the own-lane
// leader when it is on the same lane) and vehicle i - 1 (the old follower when it is).
struct Nbr {
  float xL, vL, xF, vF, v0F;
  int sameL, sameF;
};

// Records of lane l + step direction, loaded together with the own lane's: the lane-change
// target when the own lane has a neighbour on that side (an edge's lanes are consecutive,
// numbered from the right, and equally long).
struct Tgt {
  int first, count;   // its segment of the snapshot
  int ctrl, group;    // the signal at its end
  float vmax;         // its speed limit (+inf: none)
  int closed;         // closed to entering vehicles
};

struct Upd {
  int kind, lane, rp;
  float x, v, a_use, a_own;
  Lead own;
  LC lc;
  int flag;
};

// Lane records per step: {first index, count, tail x bits, tail v bits}; the tail fields
// (rearmost vehicle of the lane) are valid when count > 0.  MODS: lane closures in effect.
template <bool MODS>
__device__ __forceinline__ Lead own_leader(const StepArgs &a, const Soa &S, const int4 *dyn, int i,
                                           int l, const LaneInfo &li, const Nbr &nb, float x, float v,
                                           int rp, int nlc, int4 pf_dyn, const LaneInfo &pf_li,
                                           int myid, int t, int &flag) {
  const DevParams &P = a.P;
  Lead r{K_FREE, 0.f, 0.f, -1, 0};
  if (nb.sameL) {
    r = Lead{K_VEH, (nb.xL - x) - P.L, nb.vL, i + 1, 0};
  } else {
    float dist = li.len - x;
    int ri = rp;
    bool cached = true;   // the first edge-lane hop uses the vehicle's cached choice
    LaneInfo lc = li;
    for (int hop = 0;; ++hop) {
      mark(flag, dist - P.d_look);
      if (dist >= P.d_look) break;
      int nxt;
      bool pre = false;
      if (lc.edge >= 0) {
        if (cached) {
          cached = false;
          if (nlc == NL_END) break;   // destination edge: open end
          nxt = nlc;
          pre = nxt >= 0;
        } else {
          nxt = plan_next(a, a.plan[ri], lc.idx, lc.succ);
          if (nxt == NL_END) break;   // destination edge: open end
        }
        bool stop = nxt < 0;
        if (!stop) {
          int sg = sig_state(a, lc, t);
          if (sg == SIG_R) {
            stop = true;
          } else if (sg == SIG_Y) {
            float m = dist - v * v * P.inv2b;
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
      }
      if (MODS && a.lane_closed[nxt]) {   // a closed lane ends the path
        r = Lead{K_OBST, dist, 0.f, -1, hop == 0};
        break;
      }
      if (hop + 1 >= HOP_CAP) {
        r = Lead{K_OBST, dist, 0.f, -1, hop == 0};
        break;
      }
      const int4 dn = pre ? pf_dyn : dyn[nxt];
      if (dn.y > 0) {
        r = Lead{K_VEH, (dist + __int_as_float(dn.z)) - P.L, __int_as_float(dn.w), dn.x, 0};
        break;
      }
      lc = pre ? pf_li : a.li[nxt];
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
        int4 df = dyn[f];
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

// end of the target lane (length len, plan position q) blocks a vehicle at (x, v)
// following plan word pl
__device__ __forceinline__ bool end_blocks(const StepArgs &a, const Tgt &tg, float len, int q,
                                           unsigned long long pl, float x, float v, int t, int &flag) {
  if (pl & PLAN_END) return false;
  if (plan_nib(pl, q) == PLAN_NONE) return true;
  int sg = sig_state(a, tg.ctrl, tg.group, t);
  if (sg == SIG_R) return true;
  if (sg == SIG_Y) {
    float m = (len - x) - v * v * a.P.inv2b;
    mark(flag, m);
    return m >= 0.f;
  }
  return false;
}

__device__ __forceinline__ LC lane_change(const StepArgs &a, const Soa &S, const int4 *dyn, int i,
                                          int l, const LaneInfo &li, float x, float v, float v0,
                                          unsigned long long pl, int nlc, const Nbr &nb, const Tgt &tg,
                                          float vmax_own, float fr_own, int myid, int t, const Lead &own,
                                          float a_c, int &flag) {
  const DevParams &P = a.P;
  LC r{};
  r.tl = r.tf = r.of = -1;
  if (li.edge < 0) return r;
  int step_dir = (t % 2 == 0) ? 1 : -1;
  r.step_dir = step_dir;
  int tau = step_dir > 0 ? li.left : li.right;
  if (tau < 0) return r;
  if (tg.closed) return r;   // a closed lane is never a target
  const bool mand = nlc == NL_NONE;   // own lane has no link toward the next edge
  r.mand = mand;
  if (mand) {   // nearest lane on each side with a link toward the next edge
    const int q = li.idx;
    int dr = 1 << 30, dl = 1 << 30;
    for (int k = 1; k <= q; ++k)
      if (plan_nib(pl, q - k) != PLAN_NONE) { dr = k; break; }
    for (int k = 1; q + k < PLAN_LANES; ++k)
      if (plan_nib(pl, q + k) != PLAN_NONE) { dl = k; break; }
    if (dr == (1 << 30) && dl == (1 << 30)) return r;
    int want = dr <= dl ? -1 : +1;
    if (want != step_dir) return r;
  }
  mark(flag, x - P.x_lc_min);
  if (x < P.x_lc_min) return r;
  const int tq = li.idx + step_dir;   // the target's plan position (tau == l + step_dir)
  if (!mand) {
    if (!plan_ok(pl, tq)) return r;
    mark(flag, (li.len - x) - P.x_lc_end);
    if (li.len - x < P.x_lc_end) return r;
    if (P.lc_thresh < (1u << 24)) {   // p_lc = 1: the gate always passes
      unsigned long long h = splitmix64(P.seed ^ ((unsigned long long)(unsigned)t << 32) ^
                                        (unsigned long long)(unsigned)(myid + P.id_base));
      if ((uint32_t)(h >> 40) >= P.lc_thresh) return r;
    }
  }
  r.cand = 1;
  int lo = tg.first, hi = tg.first + tg.count;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (S.x[mid] > x) hi = mid; else lo = mid + 1;
  }
  int Lt = lo < tg.first + tg.count ? lo : -1;
  int Ft = lo > tg.first ? lo - 1 : -1;
  r.tfirst = tg.first;
  r.pos = lo;   // first with x' > x; moved onto the follower below if it is level with x
  r.tl = Lt;
  r.tf = Ft;
  if (Lt >= 0) {
    r.tkind = K_VEH;
    r.tgap = (S.x[Lt] - x) - P.L;
    r.tvl = S.v[Lt];
  } else if (end_blocks(a, tg, li.len, tq, pl, x, v, t, flag)) {
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
  float aF_new = 0.f, xF = 0.f, vF = 0.f, v0F = 1.f, frF = 1.f;
  if (Ft >= 0) {
    xF = S.x[Ft];
    vF = S.v[Ft];
    v0F = fminf(S.v0[Ft], tg.vmax);   // the new follower drives under the target's limit
    frF = idm_free(vF, v0F);
    float gF = (x - xF) - P.L;
    float guard = vF * P.dt + 0.5f * P.a * P.dt * P.dt;
    mark(flag, gF - guard);
    if (gF < guard) return r;
    if (xF == x) r.pos = Ft;   // at most one vehicle of a lane can be level with x
    aF_new = idm_fr(P, frF, vF, true, gF, v);
    mark(flag, aF_new + P.bsafe);
    if (aF_new < -P.bsafe) return r;
    r.gF = gF;
    r.vF = vF;
    r.aFn = aF_new;
  }
  r.safe = 1;
  // the changer's free-road term: its own lane's unless the target lane's limit differs
  const float fr_new = tg.vmax == vmax_own ? fr_own : idm_free(v, fminf(v0, tg.vmax));
  r.anew = idm_fr(P, fr_new, v, r.tkind != K_FREE, r.tgap, r.tvl);
  if (!mand) {
    float delta = r.anew - a_c;
    if (Ft >= 0) {
      float aF_old;
      if (Lt >= 0)
        aF_old = idm_fr(P, frF, vF, true, (S.x[Lt] - xF) - P.L, S.v[Lt]);
      else if (end_blocks(a, tg, li.len, tq, pl, xF, vF, t, flag))
        aF_old = idm_fr(P, frF, vF, true, li.len - xF, 0.f);
      else
        aF_old = idm_fr(P, frF, vF, false, 0.f, 0.f);
      delta += P.p * (aF_new - aF_old);
    }
    if (nb.sameF) {
      r.of = i - 1;
      const float xO = nb.xF, vO = nb.vF, v0O = fminf(nb.v0F, vmax_own);
      const float frO = idm_free(vO, v0O);
      float aO_old = idm_fr(P, frO, vO, true, (x - xO) - P.L, v);
      float aO_new = own.kind != K_FREE ? idm_fr(P, frO, vO, true, own.gap + (x - xO), own.vl)
                                        : idm_fr(P, frO, vO, false, 0.f, 0.f);
      delta += P.p * (aO_new - aO_old);
    }
    r.inc = delta;
    // incentive threshold: mobil_th, offset per trip when the jitter variant is on (the
    // salted draw is fixed for the trip; its low 32 bits never equal the gate draw's)
    float th = P.th;
    if (P.th_jitter > 0.f) {
      const unsigned long long hj = splitmix64(P.seed ^ 0x9E3779B97F4A7C15ULL ^
                                               (unsigned long long)(unsigned)(myid + P.id_base));
      th += P.th_jitter * (2.f * ((float)(uint32_t)(hj >> 40) * 0x1p-24f) - 1.f);
    }
    mark(flag, delta - th);
    if (!(delta > th)) return r;
  }
  r.dir = step_dir;
  return r;
}

// Per-vehicle context of one step (snapshot values the update reuses)
struct VCtx {
  int l, rp, nlc, id;
  unsigned long long pl;
  float x, v, v0;
  LaneInfo li;
  Nbr nb;
};

// The vehicle's own fields (coalesced) and its sorted-order neighbours: warp shuffles, with
// the vehicles just outside the warp loaded by its edge lanes.  Called by the whole warp.
__device__ __forceinline__ void load_vehicle(const Soa &S, int n, int i, VCtx &c) {
  const bool act = i < n;
  c.l = -1;
  c.x = c.v = 0.f;
  c.v0 = 1.f;
  c.rp = c.nlc = c.id = 0;
  c.pl = 0;
  if (act) {
    c.l = S.lane[i];
    c.x = S.x[i];
    c.v = S.v[i];
    c.v0 = S.v0[i];
    c.rp = S.rp[i];
    c.pl = S.pl[i];
    c.nlc = S.nl[i];
    c.id = S.id[i];
  }
  const unsigned full = 0xffffffffu;
  const int wl = threadIdx.x & 31;
  float xL = __shfl_down_sync(full, c.x, 1), vL = __shfl_down_sync(full, c.v, 1);
  int lL = __shfl_down_sync(full, c.l, 1);
  float xF = __shfl_up_sync(full, c.x, 1), vF = __shfl_up_sync(full, c.v, 1), v0F = __shfl_up_sync(full, c.v0, 1);
  int lF = __shfl_up_sync(full, c.l, 1);
  if (wl == 31) {
    lL = -1;
    if (i + 1 < n) {
      xL = S.x[i + 1];
      vL = S.v[i + 1];
      lL = S.lane[i + 1];
    }
  }
  if (wl == 0) {
    lF = -1;
    if (act && i > 0) {
      xF = S.x[i - 1];
      vF = S.v[i - 1];
      v0F = S.v0[i - 1];
      lF = S.lane[i - 1];
    }
  }
  c.nb = Nbr{xL, vL, xF, vF, v0F, act && lL == c.l, act && lF == c.l};
}

// Sensing, car following and the rule's lane-change decision of vehicle i at step t (own
// fields and neighbours already in c).  MODS: lane speed limits / closures in effect.
template <bool MODS>
__device__ __forceinline__ Upd vehicle_sense(const StepArgs &a, const Soa &S, const int4 *dyn, int i, int t,
                                             VCtx &c) {
  const DevParams &P = a.P;
  Upd u;
  u.flag = 0;
  // every record the vehicle may need is loaded here, together with the own lane's: the
  // cached next lane's (only the lane's front vehicle looks ahead) and the possible target
  // lane's (lane l + step direction, only at or past the lane-change start)
  c.li = a.li[c.l];
  int4 pf_dyn = make_int4(0, 0, 0, 0);
  LaneInfo pf_li{};
  if (!c.nb.sameL && c.nlc >= 0) {
    pf_dyn = dyn[c.nlc];
    pf_li = a.li[c.nlc];
  }
  const float inf = __int_as_float(0x7f800000);
  Tgt tg{0, 0, -1, 0, inf, 0};
  const int tl = c.l + ((t & 1) == 0 ? 1 : -1);
  if (c.x >= P.x_lc_min && tl >= 0 && tl < P.n_lanes) {
    const int2 d2 = reinterpret_cast<const int2 *>(dyn)[2 * tl];
    const int2 c2 = reinterpret_cast<const int2 *>(a.li)[4 * tl + 3];   // {ctrl, packed bytes}
    tg = Tgt{d2.x, d2.y, c2.x, (c2.y >> 16) & 0xff, inf, 0};
    if (MODS) {
      tg.vmax = a.lane_vmax[tl];
      tg.closed = a.lane_closed[tl];
    }
  }
  // lane speed limits cap the desired speed: v0_eff = min(v0, vmax of the lane)
  const float vmax_own = MODS ? a.lane_vmax[c.l] : inf;
  u.own = own_leader<MODS>(a, S, dyn, i, c.l, c.li, c.nb, c.x, c.v, c.rp, c.nlc, pf_dyn, pf_li, c.id, t, u.flag);
  const float fr_own = idm_free(c.v, fminf(c.v0, vmax_own));
  u.a_own = idm_fr(P, fr_own, c.v, u.own.kind != K_FREE, u.own.gap, u.own.vl);
  u.lc = lane_change(a, S, dyn, i, c.l, c.li, c.x, c.v, c.v0, c.pl, c.nlc, c.nb, tg, vmax_own, fr_own, c.id, t,
                     u.own, u.a_own, u.flag);
  return u;
}

// Motion, safety clamp and lane transfer for the lane-change direction dir.
__device__ __forceinline__ void vehicle_move(const StepArgs &a, Upd &u, const VCtx &c, int dir) {
  const DevParams &P = a.P;
  const LaneInfo &li = c.li;
  const float x = c.x, v = c.v;
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
  // the lane end is tested as d > len - x (len - x is exact when x >= len / 2) and a
  // transferred position is d - (len - x), rounded at its own magnitude: x + d - len would
  // carry the rounding of x + d (2.4e-4 m on a 3 km lane) onto the next lane
  const float rem = li.len - x;
  float xn = x + d;
  if (u.own.end_obst || dir) xn = fminf(xn, li.len);
  u.kind = dir ? U_CHANGE : U_STAY;
  u.lane = dir ? (dir > 0 ? li.left : li.right) : c.l;
  u.rp = c.rp;
  if (!dir) {
    mark(u.flag, d - rem);
    if (!(d > rem)) {
      xn = fminf(xn, li.len);   // x + d may round past the end when d is within an ulp of rem
    } else if (li.edge >= 0 && (c.pl & PLAN_END)) {
      u.kind = U_RETIRE;
    } else {
      xn = d - rem;
      u.kind = U_TRANSFER;
      int nl;
      if (li.edge >= 0) {
        nl = c.nlc;
      } else {
        nl = li.succ;
        u.rp = c.rp + 1;
      }
      if (nl < 0 || xn > a.li[nl].len) {
        atomicOr(&a.ctrl->err, DEV_HOP);
        nl = c.l;
        xn = li.len;
        u.kind = U_STAY;
        u.rp = c.rp;
      }
      u.lane = nl;
    }
  }
  u.x = xn;
  u.v = vn;
}

// The rest of vehicle i's update once its lane-change direction dir is known: motion, its
// result record and the count of vehicles leaving its lane.  Returns whether it leaves its
// slot (changes lane, transfers or retires).
template <bool DBG>
__device__ __forceinline__ int vehicle_finish(const StepArgs &a, const Soa &S, int i, Upd &u, const VCtx &c,
                                              int dir) {
  vehicle_move(a, u, c, dir);
  const int leave = u.kind != U_STAY;
  if (leave) atomicAdd(&a.arr_cnt[c.l], LEAVE_ONE);   // fire-and-forget, like the arrivals
  int kind = u.kind == U_STAY ? C_STAY
           : u.kind == U_CHANGE ? C_CHANGE
           : u.kind == U_RETIRE ? C_RETIRE
           : (u.rp != c.rp ? C_TRANSFER_ROUTE : C_TRANSFER);
  a.res_x[i] = u.x;
  a.res_v[i] = u.v;
  a.res_code[i] = (kind << CODE_LANE_BITS) | (u.kind == U_RETIRE ? 0 : u.lane);
  if constexpr (DBG) {
    a.dbg.id[i] = c.id;
    a.dbg.lead_kind[i] = u.own.kind;
    a.dbg.lead_id[i] = u.own.j >= 0 ? S.id[u.own.j] : -1;
    a.dbg.s_own[i] = u.own.gap;
    a.dbg.vl_own[i] = u.own.vl;
    a.dbg.a_own[i] = u.a_own;
    a.dbg.lc_dir[i] = dir;   // the direction taken (the network's where it decided)
    a.dbg.lc_cand[i] = u.lc.cand;
    a.dbg.tau_lead[i] = u.lc.tl >= 0 ? S.id[u.lc.tl] : -1;
    a.dbg.tau_foll[i] = u.lc.tf >= 0 ? S.id[u.lc.tf] : -1;
    a.dbg.old_foll[i] = u.lc.of >= 0 ? S.id[u.lc.of] : -1;
    a.dbg.incentive[i] = u.lc.inc;
    a.dbg.a_use[i] = u.a_use;
    a.dbg.flag[i] = u.flag;
    a.dbg.lc_learn[i] = 0;   // k_learn marks the vehicles its network decided
  }
  return leave;
}

// The records of a vehicle arriving on a new lane (lane change or transfer): the lane's
// arrival count and rearmost arrival (no value returned, so nothing waits on these atomics;
// slots are handed out by k_bucket), and the arrival's cached next-lane choice for its new
// lane (internal -> edge lane keeps the choice it already made for that target lane): a
// lane change follows the plan of its own edge, an internal lane the plan of its target
// lane's edge.
template <bool DBG>
__device__ __forceinline__ void arrival_records(const StepArgs &a, int i, const Upd &u, const VCtx &c) {
  atomicAdd(&a.arr_cnt[u.lane], 1);
  if (a.P.fifo) atomicMin(&a.amin[u.lane], fkey(u.x - a.P.L));   // read only by the entry test
  if (u.kind == U_CHANGE) a.res_pos[i] = make_int2(u.lc.tfirst, u.lc.pos);
  if (u.rp == c.rp) {
    const LaneInfo ln = a.li[u.lane];
    const unsigned long long pn = a.plan[c.rp + 1];
    a.res_code_nl[i] = ln.edge >= 0 ? plan_next(a, c.pl, ln.idx, ln.succ) : plan_next(a, pn, ln.idx, ln.left);
  }
  if constexpr (DBG) {
    if (u.flag) a.dbg.arr_flag[u.lane] = 1;
  }
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

// Per-lane window metrics over the snapshot: sum of speeds and count.  A lane's vehicles are
// consecutive, so each warp sums the run of every lane within it (segmented scan from the
// right, a fixed order) and the run's first vehicle adds it to the lane's accumulators: the
// count as an integer, the sum in integer units of 2^-24 m/s, so the per-lane totals are
// exact sums of the runs whatever the order of the atomics (deterministic).  Called by all
// 32 threads.
__device__ __forceinline__ void lane_speed_sums(const StepArgs &a, int w, const VCtx &c) {
  const unsigned full = 0xffffffffu;
  const int wl = threadIdx.x & 31;
  const bool act = c.l >= 0;
  const int l = act ? c.l : -1 - wl;
  float v = act ? c.v : 0.f;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float y = __shfl_down_sync(full, v, o);
    const int ly = __shfl_down_sync(full, l, o);
    if (wl + o < 32 && ly == l) v += y;
  }
  // bit k: vehicle k + 1 of the warp continues vehicle k's run (never past the warp)
  const unsigned cont = __ballot_sync(full, __shfl_down_sync(full, l, 1) == l) & 0x7fffffffu;
  const bool head = act && (wl == 0 || !((cont >> (wl - 1)) & 1u));
  if (!head) return;
  const size_t o = (size_t)w * a.P.n_lanes + l;
  atomicAdd(&a.vsum[o], __float2ull_rn(v * 16777216.f));
  atomicAdd(&a.vcnt[o], __ffs(~(cont >> wl)));   // the run's length
}

// The 16 inputs of the learned lane-change decision (scaled to O(1)): own speed and desired
// speed, own-path gap and closing speed, current acceleration, allowed direction, target
// lane gap and closing speed, new follower gap / speed / acceleration, prospective
// acceleration, old follower speed, distance to the lane end, leader speed, old follower gap.
__device__ __forceinline__ void lc_features(const StepArgs &a, const Soa &S, int i, const Upd &u, const VCtx &c,
                                            float f[MLP_IN]) {
  const float L = a.P.L;
  f[0] = c.v / 20.f;
  f[1] = c.v0 / 20.f;
  f[2] = u.own.kind != K_FREE ? fminf(u.own.gap, 200.f) / 100.f : 2.f;
  f[3] = u.own.kind == K_VEH ? (c.v - u.own.vl) / 10.f : (u.own.kind == K_OBST ? c.v / 10.f : 0.f);
  f[4] = u.a_own / a.P.a;
  f[5] = (float)u.lc.step_dir;
  f[6] = u.lc.tkind != K_FREE ? fminf(u.lc.tgap, 200.f) / 100.f : 2.f;
  f[7] = u.lc.tkind == K_VEH ? (c.v - u.lc.tvl) / 10.f : (u.lc.tkind == K_OBST ? c.v / 10.f : 0.f);
  f[8] = u.lc.tf >= 0 ? fminf(u.lc.gF, 200.f) / 100.f : 2.f;
  f[9] = u.lc.tf >= 0 ? u.lc.vF / 20.f : 0.f;
  f[10] = u.lc.tf >= 0 ? u.lc.aFn / a.P.a : 0.f;
  f[11] = u.lc.anew / a.P.a;
  f[12] = c.nb.sameF ? c.nb.vF / 20.f : 0.f;
  f[13] = fminf(c.li.len - c.x, 200.f) / 100.f;
  f[14] = u.own.kind == K_VEH ? u.own.vl / 20.f : (u.own.kind == K_OBST ? 0.f : 1.f);
  f[15] = c.nb.sameF ? fminf((c.x - c.nb.xF) - L, 200.f) / 100.f : 2.f;
}

__device__ __forceinline__ int lc_class(int dir) { return dir > 0 ? 1 : (dir < 0 ? 2 : 0); }
__device__ __forceinline__ int lc_dir(int cls) { return cls == 1 ? 1 : (cls == 2 ? -1 : 0); }

// shared memory of the learned step: the model plus, per warp, 32 feature rows, one 16-row
// hidden buffer and 32 x 3 logits
constexpr int LEARN_WARP_SMEM = 32 * MLP_IN * 2 + 16 * MLP_H * 2 + 32 * MLP_OUT * 4;
constexpr int LEARN_THREADS = 256;   // k_learn block
constexpr unsigned DEC_WAIT_LIMIT = 1u << 20;   // polls of a tile's copy barrier before giving up
__host__ __device__ constexpr int learn_smem(int threads) {
  return (int)sizeof(MlpDev) + (threads / 32) * LEARN_WARP_SMEM;
}

// DBG: record per-vehicle sensing and decisions (tests); a separate instance, so that the
// production kernel keeps none of those values alive.  MODS: lane speed limits or closures
// are set (also a separate instance: without them the step does no work for them).  The plain
// production instance is capped at 48 registers: 5 blocks of 256 per SM instead of 4 outweigh
// its few spills (the kernel is bound by the latency of dependent gathers, so resident warps
// decide its speed).  The learned instance is the plain one that lists its discretionary
// candidates with their sensing records instead of finishing them (k_learn does); it gets
// 64 registers, since the records keep more values live (48 spilled 272 B).
template <int MODE, bool DBG, bool MODS>
__global__ void __launch_bounds__(512, 2) __maxnreg__((MODE == MODE_PLAIN && !DBG) ? 48 : 64)
    k_decide_t(StepArgs a) {
  pdl_enter();
  const int t = a.ctrl->t;
  const int p = t & 1;
  const Soa S = a.A[p];
  const int4 *dyn = a.dyn[p];
  const int n = a.ctrl->n_active[p];
  const int w = t / a.P.window;
  const bool rec = a.vsum != nullptr && w < a.P.n_windows;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n; base += stride) {
    const int i = base + threadIdx.x;
    int leave = 0, moving = 0;
    Upd u;
    VCtx c;
    int dir = 0;
    bool defer = false;   // learned instance: k_learn finishes this vehicle
    load_vehicle(S, n, i, c);
    if (i < n) {
      u = vehicle_sense<MODS>(a, S, dyn, i, t, c);
      dir = u.lc.dir;
    }
    if constexpr (MODE != MODE_PLAIN) {
      // discretionary candidates that passed the safety criteria: the decision to learn
      const bool cand = i < n && u.lc.cand && u.lc.safe && !u.lc.mand;
      if (MODE == MODE_LEARN && cand) {   // k_learn continues from these (slot = index)
        reinterpret_cast<Upd *>(a.lc.rec_u)[i] = u;
        reinterpret_cast<VCtx *>(a.lc.rec_c)[i] = c;
      }
      const int rule = cand ? lc_class(u.lc.dir) : 0;
      const unsigned cm = __ballot_sync(0xffffffffu, cand);
      const int wl = threadIdx.x & 31;
      if constexpr (MODE == MODE_LOG) {
        if (cm) {
          int slot0 = 0;
          const int leader = __ffs(cm) - 1;
          if (wl == leader) slot0 = atomicAdd(a.lc.log_n, __popc(cm));
          slot0 = __shfl_sync(0xffffffffu, slot0, leader);
          if (cand) {
            const int slot = slot0 + __popc(cm & ((1u << wl) - 1u));
            if (slot < a.lc.log_cap) {
              float f[MLP_IN];
              lc_features(a, S, i, u, c, f);
              for (int q = 0; q < MLP_IN; ++q) a.lc.log_x[(size_t)slot * MLP_IN + q] = __float2bfloat16_rn(f[q]);
              a.lc.log_y[slot] = rule;
            }
          }
        }
      } else {   // MODE_LEARN: the candidates are listed and their update left to k_learn
        if (cm) {
          int slot0 = 0;
          const int leader = __ffs(cm) - 1;
          if (wl == leader) slot0 = atomicAdd(&a.ctrl->n_cand, __popc(cm));
          slot0 = __shfl_sync(0xffffffffu, slot0, leader);
          const int slot = slot0 + __popc(cm & ((1u << wl) - 1u));
          if (cand && slot < a.lc.cand_cap) {
            a.lc.cand[slot] = i;
            defer = true;
          }
        }
      }
    }
    if (i < n && !defer) {
      leave = vehicle_finish<DBG>(a, S, i, u, c, dir);
      moving = u.kind == U_CHANGE || u.kind == U_TRANSFER;
    }
    const unsigned lm = __ballot_sync(0xffffffffu, leave);
    if ((threadIdx.x & 31) == 0) a.leave[(base + threadIdx.x) >> 5] = lm;
    if (rec) lane_speed_sums(a, w, c);
    if (moving) arrival_records<DBG>(a, i, u, c);
  }
}

// Learned lane change: the decisions of the step's discretionary candidates, listed by the
// decide kernel with their sensing results and their update left undone.  Each warp takes
// 16 listed vehicles, evaluates the surrogate network on their features as one 16-row
// tensor-core tile (rows past the list are zero; each output row depends on its own input
// row only), takes the network's class unless its softmax margin is below lc.margin (then
// the rule's), and finishes their update with that direction.  Launched right after the
// decide kernel.
template <bool DBG>
__global__ void __launch_bounds__(LEARN_THREADS) k_learn(StepArgs a) {
  extern __shared__ __align__(16) unsigned char lsm[];
  pdl_enter();
  const int p = a.ctrl->t & 1;
  const int nc = min(a.ctrl->n_cand, a.lc.cand_cap);
  {   // the model into shared memory: every 16-byte load of the block in flight at once
    static_assert(sizeof(MlpDev) % 16 == 0, "model copied in 16-byte words");
    constexpr int NV = (int)(sizeof(MlpDev) / 16), PER = (NV + LEARN_THREADS - 1) / LEARN_THREADS;
    const uint4 *src = reinterpret_cast<const uint4 *>(a.lc.model);
    uint4 *dst = reinterpret_cast<uint4 *>(lsm);
    uint4 r[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k)
      if (threadIdx.x + k * LEARN_THREADS < NV) r[k] = src[threadIdx.x + k * LEARN_THREADS];
#pragma unroll
    for (int k = 0; k < PER; ++k)
      if (threadIdx.x + k * LEARN_THREADS < NV) dst[threadIdx.x + k * LEARN_THREADS] = r[k];
    __syncthreads();
  }
  const MlpDev &w = *reinterpret_cast<const MlpDev *>(lsm);
  unsigned char *ws = lsm + sizeof(MlpDev) + (threadIdx.x >> 5) * LEARN_WARP_SMEM;
  __nv_bfloat16 *X = reinterpret_cast<__nv_bfloat16 *>(ws);
  __nv_bfloat16 *H1 = X + 32 * MLP_IN;
  float *Z = reinterpret_cast<float *>(H1 + 16 * MLP_H);
  const Soa S = a.A[p];
  const int n = a.ctrl->n_active[p];
  const int wl = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  // 16 candidates per warp (lanes 0..15), one tensor-core tile each: the network's three
  // layers are a serial chain, so two tiles per warp would double its latency
  for (int cb = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 16; cb < nc; cb += nw * 16) {   // warp-uniform
    const bool listed = wl < 16 && cb + wl < nc;
    const int i = listed ? a.lc.cand[cb + wl] : n;
    VCtx c;
    Upd u;
    int dir = 0;
    bool cand = false;
    int rule = 0;
    if (listed) {
      u = reinterpret_cast<const Upd *>(a.lc.rec_u)[i];
      c = reinterpret_cast<const VCtx *>(a.lc.rec_c)[i];
      dir = u.lc.dir;
      cand = true;
      rule = lc_class(u.lc.dir);
    }
    if (cand) {
      float f[MLP_IN];
      lc_features(a, S, i, u, c, f);
      for (int q = 0; q < MLP_IN; ++q) X[wl * MLP_IN + q] = __float2bfloat16_rn(f[q]);
      if constexpr (DBG)
        for (int q = 0; q < MLP_IN; ++q) a.dbg.lc_feat[(size_t)i * MLP_IN + q] = __bfloat162float(X[wl * MLP_IN + q]);
    } else {
      for (int q = 0; q < MLP_IN; ++q) X[wl * MLP_IN + q] = __float2bfloat16_rn(0.f);
    }
    __syncwarp();
    mlp_forward_tile(w, X, H1, nullptr, [&](int m, int q, float v) { Z[m * MLP_OUT + q] = v; });
    __syncwarp();
    int fin = rule;
    bool fb = false;
    if (cand) {
      const float z0 = Z[wl * 3], z1 = Z[wl * 3 + 1], z2 = Z[wl * 3 + 2];
      const float mx = fmaxf(z0, fmaxf(z1, z2));
      const float e0 = __expf(z0 - mx), e1 = __expf(z1 - mx), e2 = __expf(z2 - mx);
      const float sum = e0 + e1 + e2;
      const float p0 = e0 / sum, p1 = e1 / sum, p2 = e2 / sum;
      int cls = 0;
      float top = p0, sec = fmaxf(p1, p2);
      if (p1 > top) { cls = 1; sec = fmaxf(p0, p2); top = p1; }
      if (p2 > top) { cls = 2; sec = fmaxf(p0, p1); top = p2; }
      fb = top - sec < a.lc.margin;
      if (!fb) fin = (cls != 0 && lc_dir(cls) != u.lc.step_dir) ? 0 : cls;
      dir = lc_dir(fin);
      if constexpr (DBG) {
        mark(u.flag, (top - sec) - a.lc.margin);
        a.dbg.lc_margin[i] = top - sec;
        a.dbg.lc_logit[(size_t)i * 3] = z0;
        a.dbg.lc_logit[(size_t)i * 3 + 1] = z1;
        a.dbg.lc_logit[(size_t)i * 3 + 2] = z2;
      }
    }
    __syncwarp();   // the next chunk overwrites X and Z
    if (a.lc.stats) {
      const unsigned cm = __ballot_sync(0xffffffffu, cand);
      const unsigned fbm = __ballot_sync(0xffffffffu, cand && fb);
      const unsigned agm = __ballot_sync(0xffffffffu, cand && fin == rule);
      unsigned conf[9];
      for (int q = 0; q < 9; ++q) conf[q] = __ballot_sync(0xffffffffu, cand && rule * 3 + fin == q);
      if (wl == 0 && cm) {
        atomicAdd(&a.lc.stats[ST_CAND], (unsigned long long)__popc(cm));
        if (fbm) atomicAdd(&a.lc.stats[ST_FALLBACK], (unsigned long long)__popc(fbm));
        if (agm) atomicAdd(&a.lc.stats[ST_AGREE], (unsigned long long)__popc(agm));
        for (int q = 0; q < 9; ++q)
          if (conf[q]) atomicAdd(&a.lc.stats[ST_CONF + q], (unsigned long long)__popc(conf[q]));
      }
    }
    if (listed) {
      if (vehicle_finish<DBG>(a, S, i, u, c, dir)) atomicOr(&a.leave[i >> 5], 1u << (i & 31));
      if (u.kind == U_CHANGE || u.kind == U_TRANSFER) arrival_records<DBG>(a, i, u, c);
      if constexpr (DBG) a.dbg.lc_learn[i] = 1;
    }
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

// Lane pass: new per-lane counts, a scan over lanes, departures.  A tile of LANE_TILE lanes
// is processed by TH threads in LANE_TILE / TH striped slices (lane k * TH + thread), so every load is coalesced and the loads of all slices are issued before any
// is used.  Two launches: pass 0 computes every tile's aggregate and writes it; pass 1
// computes the same per-lane counts again (its inputs are read-only here), sums the
// aggregates of all its predecessors, one per thread (with a few hundred tiles the
// quadratic number of reads is small), and writes the results.  The launch boundary makes
// the aggregates visible; a single launch that waited on its predecessors' flags spent
// several microseconds before those stores became visible to the waiting blocks.
// TH threads per tile (LANE_TILE / TH lanes each): the autotuner picks among 128, 256, 512.
// Whether the due head of lane l's departure FIFO enters this step: room behind the lane's
// tail (d: its lane record) and behind every arrival (amk: their rearmost key).  fl: a
// margin within the flag distance (debug records).
__device__ __forceinline__ int lane_entry(const StepArgs &a, int4 d, int amk, int &fl) {
  const float room_need = a.P.L + a.P.s0;
  bool room = true;
  if (d.y > 0) {
    float m = (__int_as_float(d.z) - a.P.L) - room_need;
    mark(fl, m);
    room = m >= 0.f;
  }
  if (amk != AMIN_NONE) {
    float m = unfkey(amk) - room_need;
    mark(fl, m);
    if (m < 0.f) room = false;
  }
  return room ? 1 : 0;
}

template <int PASS, int TH = LANE_THREADS>
__global__ void __launch_bounds__(TH, LANE_TILE / TH) k_lanes_t(StepArgs a) {
  constexpr int LANE_THREADS = TH, LANE_ITEMS = LANE_TILE / TH, LANE_WARPS = TH / 32;
  static_assert(LANE_ITEMS * TH == LANE_TILE && LANE_WARPS <= 32, "lane tile shape");
  __shared__ unsigned long long s_wsum[LANE_ITEMS][LANE_WARPS];
  __shared__ unsigned long long s_part[LANE_WARPS];
  pdl_enter();
  const int tile = blockIdx.x;
  const int t = a.ctrl->t;
  const int p = t & 1;
  const Soa D = a.A[p ^ 1];
  const int4 *dyn = a.dyn[p];
  int4 *ndyn = a.dyn[p ^ 1];
  const int nlanes = a.P.n_lanes;
  const int lbase = tile * LANE_TILE + threadIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (PASS == 0 && !a.P.fifo) {
    // without departure queues the tile's aggregate {new vehicles, arrivals} needs only the
    // arrival words: its lanes hold the vehicles between two lane starts (every lane's
    // start is the count of the vehicles before it), to which the arrivals are added and
    // the leavers taken away (with queues the general path below also tests the entries)
    long long dv = 0;
    unsigned na = 0;
    int first0 = 0, first1 = 0;   // the tile's lane starts, loaded with the lanes' words
    if (threadIdx.x == 0) {
      const int l0 = tile * LANE_TILE, l1 = l0 + LANE_TILE;
      first0 = dyn[l0].x;
      first1 = l1 < nlanes ? dyn[l1].x : a.ctrl->n_active[p];
    }
#pragma unroll
    for (int k = 0; k < LANE_ITEMS; ++k) {
      const int l = lbase + k * LANE_THREADS;
      if (l < nlanes) {
        const int w = a.arr_cnt[l];
        const int arr = w & (LEAVE_ONE - 1);
        dv += arr - (w >> 16);
        na += arr;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dv += __shfl_xor_sync(0xffffffffu, dv, o);
      na += __shfl_xor_sync(0xffffffffu, na, o);
    }
    __shared__ long long s_dv[LANE_WARPS];
    __shared__ unsigned s_na[LANE_WARPS];
    if (lane == 0) {
      s_dv[warp] = dv;
      s_na[warp] = na;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long cnt = first1 - first0;
      unsigned arr = 0;
      for (int w2 = 0; w2 < LANE_WARPS; ++w2) {
        cnt += s_dv[w2];
        arr += s_na[w2];
      }
      a.tile_agg[tile] = ((unsigned long long)cnt << 32) | arr;   // read by pass 1
    }
    return;
  }
  // the general path (both passes): per-lane counts and their scan over the tile; pass 1
  // loads the predecessors' aggregates first, with the lane records
  unsigned long long part = 0;
  if (PASS == 1)
    for (int j = threadIdx.x; j < tile; j += LANE_THREADS) part += a.tile_agg[j];

  int4 d[LANE_ITEMS];
  int arr[LANE_ITEMS], lv[LANE_ITEMS], amk[LANE_ITEMS];
  int2 qhd[LANE_ITEMS];
#pragma unroll
  for (int k = 0; k < LANE_ITEMS; ++k) {
    const int l = lbase + k * LANE_THREADS;
    if (l < nlanes) {
      d[k] = dyn[l];
      const int w = a.arr_cnt[l];
      arr[k] = w & (LEAVE_ONE - 1);
      lv[k] = w >> 16;
      if (a.P.fifo) {   // queue heads and rearmost arrivals matter to entries only
        amk[k] = a.amin[l];
        qhd[k] = a.q_hd[l];
      } else {
        amk[k] = AMIN_NONE;
        qhd[k] = make_int2(0, 0x7fffffff);
      }
    } else {
      d[k] = make_int4(0, 0, 0, 0);
      arr[k] = lv[k] = 0;
      amk[k] = AMIN_NONE;
      qhd[k] = make_int2(0, 0x7fffffff);
    }
  }
  int cnt[LANE_ITEMS], ins[LANE_ITEMS];
  unsigned long long val[LANE_ITEMS], incl[LANE_ITEMS];
#pragma unroll
  for (int k = 0; k < LANE_ITEMS; ++k) {
    const int leavers = lv[k];
    ins[k] = 0;
    if (qhd[k].y <= t) {   // (a closed lane's head is parked at INT_MAX by the host)
      if (PASS == 1) {   // the head's record is read after the scan: start bringing it in now
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.q_ent + qhd[k].x));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a.q_ent2 + qhd[k].x));
      }
      int fl = 0;
      ins[k] = lane_entry(a, d[k], amk[k], fl);
      if (PASS == 1 && a.P.debug) {
        const int l = lbase + k * LANE_THREADS;
        if (fl || a.dbg.arr_flag[l]) a.dbg.trip_flag[a.q_trip[qhd[k].x]] = t + 1;
      }
    }
    cnt[k] = d[k].y - leavers + arr[k] + ins[k];
    val[k] = ((unsigned long long)cnt[k] << 32) | (unsigned)(arr[k] + ins[k]);
    incl[k] = warp_incl_scan(val[k]);
    if (lane == 31) s_wsum[k][warp] = incl[k];
  }
  __syncthreads();
  if (warp == 0) {
    // exclusive offsets of every warp of every slice, in lane order
    unsigned long long run = 0;
#pragma unroll
    for (int k = 0; k < LANE_ITEMS; ++k) {
      const unsigned long long wv = lane < LANE_WARPS ? s_wsum[k][lane] : 0ull;
      const unsigned long long wi = warp_incl_scan(wv);
      if (lane < LANE_WARPS) s_wsum[k][lane] = run + wi - wv;
      run += __shfl_sync(0xffffffffu, wi, LANE_WARPS - 1);
    }
    if (PASS == 0 && lane == 0) a.tile_agg[tile] = run;   // read by pass 1
  }
  if constexpr (PASS == 0) {
    return;
  } else {
    // sum of the predecessors' aggregates
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) s_part[warp] = part;
    __syncthreads();
    unsigned long long tile_excl = 0;
#pragma unroll
    for (int w = 0; w < LANE_WARPS; ++w) tile_excl += s_part[w];

    int n_ins = 0;
#pragma unroll
    for (int k = 0; k < LANE_ITEMS; ++k) {
      const int l = lbase + k * LANE_THREADS;
      if (l >= nlanes) break;
      const unsigned long long pre = tile_excl + s_wsum[k][warp] + (incl[k] - val[k]);
      const int nstart = (int)(pre >> 32);
      const int astart = (int)(pre & 0xffffffffu);
      // tail fields: the departing vehicle if one enters, else set by k_apply
      ndyn[l] = make_int4(nstart, cnt[k], ins[k] ? __float_as_int(a.P.L) : 0, 0);
      a.arr_start[l] = astart;
      if (ins[k]) {   // the entry's record was built at load time
        const int4 e = a.q_ent[qhd[k].x];
        const int4 e2 = a.q_ent2[qhd[k].x];
        a.q_hd[l] = make_int2(qhd[k].x + 1, e2.z);
        D.x[nstart] = a.P.L;
        D.v[nstart] = 0.f;
        D.v0[nstart] = __int_as_float(e.w);
        D.lane[nstart] = l;
        D.rp[nstart] = e.y;
        D.pl[nstart] = (unsigned long long)(unsigned)e2.x | ((unsigned long long)(unsigned)e2.y << 32);
        D.nl[nstart] = e.z;
        D.id[nstart] = e.x;
        a.bucket[astart + arr[k]] = make_int4(0, __float_as_int(a.P.L), e.x, -1);
        ++n_ins;
        if (a.P.debug) a.dbg.trip_ins[e.x] = t + 1;
      }
      if (arr[k] | lv[k]) a.arr_cnt[l] = 0;
      if (amk[k] != AMIN_NONE) a.amin[l] = AMIN_NONE;
      if (a.P.debug) a.dbg.arr_flag[l] = 0;
      if (l == nlanes - 1) {
        const unsigned long long tot = pre + val[k];
        a.ctrl->n_active[p ^ 1] = (int)(tot >> 32);
        a.arr_start[nlanes] = (int)(tot & 0xffffffffu);
        a.ctrl->t_apply = t;
      }
    }
    // signal table of step t + 1 (the next k_decide reads it); max-pressure controllers
    // are advanced by k_signals instead
    if (a.P.signal_mode == 0)
      for (int c = tile * LANE_THREADS + threadIdx.x; c < a.n_ctrl; c += gridDim.x * LANE_THREADS)
        a.sig[(t + 1) & 1][c] = sig_pack(a.ctrl4[c], t + 1);
    n_ins = __reduce_add_sync(0xffffffffu, n_ins);
    if (lane == 0 && n_ins) atomicAdd(&a.ctrl->inserted, (unsigned long long)n_ins);
  }
}

// Arrivals -> lane buckets with their rank among the lane's stayers.  Arrivals are found
// by streaming the result codes of the snapshot's vehicles; each arrival issues its loads
// and its slot atomic together, so an arrival costs two dependent round trips (three for
// a lane change, whose rank needs the leave words).
__global__ void k_bucket(StepArgs a) {
  __shared__ int s_cnt;
  if (threadIdx.x == 0) s_cnt = 0;
  pdl_enter();
  const int t = a.ctrl->t_apply;
  const int p = t & 1;
  const Soa S = a.A[p];
  const int n = a.ctrl->n_active[p];
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  int mine = 0;
  // four result codes per thread and load (the code buffer is padded to a multiple of 4)
  const int ng = (n + 3) >> 2;
  for (int g = gid; g < ng; g += stride) {
    const int4 c4 = reinterpret_cast<const int4 *>(a.res_code)[g];
    const int cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = 4 * g + q;
      if (i >= n) break;
      const int code = cs[q];
      const int kind = (unsigned)code >> CODE_LANE_BITS;
      if (kind != C_CHANGE && kind != C_TRANSFER && kind != C_TRANSFER_ROUTE) continue;
      const int nl = code & CODE_LANE_MASK;
      const int2 fp = kind == C_CHANGE ? a.res_pos[i] : make_int2(0, 0);
      const int xb = __float_as_int(a.res_x[i]);
      const int id = S.id[i];
      const int s0 = a.arr_start[nl], s1 = a.arr_start[nl + 1];
      const int slot = s0 + atomicAdd(&a.arr_fill[nl], 1);
      // rank among the target lane's stayers (k_decide found the segment); 0 for transfers
      const int r = (fp.y - fp.x) - count_bits(a.leave, fp.x, fp.y);
      if (slot >= s1) {   // never expected: more arrivals than counted
        atomicOr(&a.ctrl->err, DEV_BUCKET);
        continue;
      }
      a.bucket[slot] = make_int4(r, xb, id, i);
      ++mine;
    }
  }
  __syncthreads();   // s_cnt is set
  mine = __reduce_add_sync(0xffffffffu, mine);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(&s_cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0 && s_cnt) atomicAdd(&a.ctrl->n_movers, s_cnt);
  if (gid == 0) a.ctrl->t = t + 1;
}

__device__ __forceinline__ bool bucket_less(int4 f, int4 e) {
  if (f.x != e.x) return f.x < e.x;
  float fx = __int_as_float(f.y), ex = __int_as_float(e.y);
  if (fx != ex) return fx < ex;
  return f.z < e.z;
}

// Tile of the apply kernel in shared memory: per vehicle of a tile of T its plan word, result
// code, id, route pointer, next-lane choice, v0, x', v' and lane, the lane from 4 vehicles
// before the tile (the vehicle before its first warp); every part 16-byte aligned.
__host__ __device__ constexpr int app_buf_bytes(int T) { return 40 * T + 16; }
__host__ __device__ constexpr int app_smem(int T) { return 2 * app_buf_bytes(T) + 16; }

// Issue the copies of apply tile `tile` into buffer buf (one thread).  Extents are multiples
// of four elements: the arrays are allocated to a multiple of four.
__device__ __forceinline__ void app_issue(const StepArgs &a, const Soa &S, int n, int T, int tile, unsigned char *buf,
                                          uint64_t *bar) {
  const int npad = (n + 3) & ~3;
  const int base = tile * T;
  const unsigned c = (unsigned)(min(base + T, npad) - base);
  const int lo = max(0, base - 4), hi = min(base + T, npad);
  const unsigned bl = 4u * (unsigned)(hi - lo);
  mbar_expect_tx(bar, 36u * c + bl);
  tma_load_1d(buf, S.pl + base, 8u * c, bar);
  unsigned char *q = buf + 8 * T;
  tma_load_1d(q, a.res_code + base, 4u * c, bar);
  tma_load_1d(q + 4 * T, S.id + base, 4u * c, bar);
  tma_load_1d(q + 8 * T, S.rp + base, 4u * c, bar);
  tma_load_1d(q + 12 * T, S.nl + base, 4u * c, bar);
  tma_load_1d(q + 16 * T, S.v0 + base, 4u * c, bar);
  tma_load_1d(q + 20 * T, a.res_x + base, 4u * c, bar);
  tma_load_1d(q + 24 * T, a.res_v + base, 4u * c, bar);
  tma_load_1d(q + 28 * T + 4 * (lo - (base - 4)), S.lane + lo, bl, bar);
}

// Write each vehicle, with the result k_decide computed for it, to its sorted slot of the
// t+1 buffer: stayers by their rank among the lane's stayers plus the arrivals ranked
// before them, arrivals by their bucket rank.  Each block walks tiles of blockDim.x
// consecutive vehicles (grid stride); a tile's inputs arrive in shared memory by bulk
// asynchronous copies (TMA), the next tile's while this one is written (two buffers), so
// each warp's chain starts at its lane's new start and arrival bucket.  A stayer's rank
// among its lane's stayers comes from the warp's leave word (same-lane threads by a
// match), and only the lane that continues from the previous warp reads its lane record and
// earlier words.  Waits are bounded (MS_DEV_TIMEOUT).
__global__ void k_apply(StepArgs a) {
  extern __shared__ __align__(128) unsigned char ssm[];
  const int T = blockDim.x;
  const int bsz = app_buf_bytes(T);
  uint64_t *bar = reinterpret_cast<uint64_t *>(ssm + 2 * bsz);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async();
  }
  __syncthreads();
  pdl_enter();
  const int t = a.ctrl->t_apply;
  const int p = t & 1;
  const Soa S = a.A[p];
  const Soa D = a.A[p ^ 1];
  const int4 *dyn = a.dyn[p];
  int4 *ndyn = a.dyn[p ^ 1];
  const int n = a.ctrl->n_active[p];
  const int G = gridDim.x;
  const int wl = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    a.ctrl->movers_last = a.ctrl->n_movers;
    a.ctrl->n_movers = 0;
    a.ctrl->n_cand = 0;
  }
  const bool issue = !a.P.test_withhold;
  const unsigned limit = issue ? DEC_WAIT_LIMIT : 4096u;
  if (issue && threadIdx.x == 0 && blockIdx.x * T < n) app_issue(a, S, n, T, blockIdx.x, ssm, &bar[0]);
  for (int j = 0;; ++j) {
    const int tile = blockIdx.x + j * G;
    const int base = tile * T;
    if (base >= n) break;   // block-uniform
    const int b = j & 1;
    if (issue && threadIdx.x == 0 && base + G * T < n) {   // the other buffer was released by the last barrier
      fence_proxy_async();
      app_issue(a, S, n, T, tile + G, ssm + (b ^ 1) * bsz, &bar[b ^ 1]);
    }
    const bool ok = __all_sync(full, mbar_wait(&bar[b], (j >> 1) & 1, limit));
    const int ws = base + (threadIdx.x & ~31);   // this warp's first vehicle
    if (ok && ws < n) do {
      const unsigned char *buf = ssm + b * bsz;
      const unsigned long long *tl_pl = reinterpret_cast<const unsigned long long *>(buf);
      const int *tl = reinterpret_cast<const int *>(buf + 8 * T);
      const int *tl_lane = tl + 7 * T;   // lane of vehicle base - 4 + k at k
      const int i = ws + wl;
      const int q = i - base;
      const bool act = i < n;
      int code = C_RETIRE << CODE_LANE_BITS, id = 0, lane = -1 - wl, rp = 0, nlc = 0;
      unsigned long long pl = 0;
      float v0 = 0.f, xn = 0.f, vn = 0.f;
      if (act) {
        code = tl[q];
        id = tl[T + q];
        rp = tl[2 * T + q];
        nlc = tl[3 * T + q];
        v0 = __int_as_float(tl[4 * T + q]);
        xn = __int_as_float(tl[5 * T + q]);
        vn = __int_as_float(tl[6 * T + q]);
        lane = tl_lane[q + 4];
        pl = tl_pl[q];
      }
      const unsigned lw = a.leave[ws >> 5];
      const int prev = ws > 0 ? tl_lane[ws - base + 3] : -1;   // the vehicle before this warp
      const int kind = (unsigned)code >> CODE_LANE_BITS;
      const int nl = code & CODE_LANE_MASK;
      const unsigned same = __match_any_sync(full, lane);
      // retirements: arrival step per trip, counters summed per warp
      const bool ret = act && kind == C_RETIRE;
      const unsigned rm = __ballot_sync(full, ret);
      if (rm) {
        const unsigned tt = ret ? (unsigned)(t + 1 - a.trip_tdep[id]) : 0u;
        const unsigned tsum = __reduce_add_sync(full, tt);
        if (ret) a.t_arr[id] = t + 1;
        if (wl == 0) {
          atomicAdd(&a.ctrl->arrived, (unsigned long long)__popc(rm));
          atomicAdd(&a.ctrl->sum_tt, (unsigned long long)tsum);
        }
      }
      if (!act || kind == C_RETIRE) break;
      const int bs = a.arr_start[nl], be = a.arr_start[nl + 1];
      const int nfirst = ndyn[nl].x;
      if (kind == C_TRANSFER_ROUTE) {   // internal lane -> edge lane: next route edge; the
        rp += 1;                        // cached choice was made for this target lane
        pl = a.plan[rp];
      } else if (kind != C_STAY) {      // lane change or edge lane -> internal lane
        nlc = a.res_code_nl[i];
      }
      int pos;
      if (kind == C_STAY) {
        // rank among the lane's stayers: same-lane stayers earlier in this warp, plus those
        // before the warp when the lane continues from the previous one
        int k = __popc(~lw & same & ((1u << wl) - 1u));
        if (prev == lane) {
          const int dx = dyn[lane].x;
          k += (ws - dx) - count_bits(a.leave, dx, ws);
        }
        int m = 0;
        for (int q = bs; q < be; ++q) m += a.bucket[q].x <= k;
        pos = nfirst + k + m;
      } else {
        int4 me = make_int4(0, 0, 0, -2);
        for (int q = bs; q < be; ++q) {
          int4 f = a.bucket[q];
          if (f.w == i) { me = f; break; }
        }
        if (me.w != i) {
          atomicOr(&a.ctrl->err, DEV_BUCKET);
          break;
        }
        int rank = 0;
        for (int q = bs; q < be; ++q) rank += bucket_less(a.bucket[q], me);
        pos = nfirst + me.x + rank;
        a.arr_fill[nl] = 0;   // every arrival resets it; k_bucket is done
      }
      if (pos == nfirst)   // rearmost vehicle of its lane: the lane record's tail fields
        reinterpret_cast<int2 *>(&ndyn[nl])[1] = make_int2(__float_as_int(xn), __float_as_int(vn));
      D.x[pos] = xn;
      D.v[pos] = vn;
      D.v0[pos] = v0;
      D.lane[pos] = nl;
      D.rp[pos] = rp;
      D.pl[pos] = pl;
      D.nl[pos] = nlc;
      D.id[pos] = id;
    } while (0);
    // every thread is done with buffer b (refilled two tiles on); a warp whose copies did not
    // arrive in time stops the block
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicOr(&a.ctrl->err, DEV_TIMEOUT);
        if (base + G * T < n) mbar_wait(&bar[b ^ 1], ((j + 1) >> 1) & 1, limit);   // in flight
      }
      return;
    }
  }
}

// Debug check of the t+1 buffer: sorted by (lane, x), gap >= 0 (up to float rounding).
__global__ void k_check(StepArgs a) {
  pdl_enter();
  const int t = a.ctrl->t;   // already advanced
  const int p = t & 1;
  const Soa S = a.A[p];
  const int n = a.ctrl->n_active[p];
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  for (int i = gid; i + 1 < n; i += gridDim.x * blockDim.x) {
    int la = S.lane[i], lb = S.lane[i + 1];
    if (la > lb || (la == lb && (S.x[i + 1] - a.P.L) - S.x[i] < -fmaxf(1e-3f, 5e-7f * S.x[i + 1])))
      atomicOr(&a.ctrl->err, DEV_ORDER);
  }
}

// Max-pressure controllers (Varaiya 2013 with unit saturation flows, at lane level),
// advanced to step t = ctrl->t on that step's lane counts; writes the signal table of step
// t.  One warp per controller.  Advancing twice to the same step changes nothing, so the
// host can also run it after every state upload.  At step t a pending phase whose time has
// come turns green; at a decision step (t mod mp_interval = 0) with nothing pending, the
// pressure of phase q is the sum over its approach lanes' links of (vehicles on the
// approach lane - vehicles on the link's target lane); the green phase wins a tie it is
// in, else the lowest index; a different winner first shows the green phase yellow for the
// controller's yellow time (or turns green at once when that is 0).
__global__ void k_signals(StepArgs a) {
  pdl_enter();
  const int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (c >= a.n_ctrl) return;   // whole warps
  const int lane = threadIdx.x & 31;
  const int t = a.ctrl->t;
  const int p = t & 1;
  const int4 *dyn = a.dyn[p];
  const int4 cc = a.ctrl4[c];   // {offset, green, yellow, nphase}
  int4 st = a.mp[c];
  if (st.y >= 0 && t >= st.z) {
    st.x = st.y;
    st.y = -1;
  }
  if (t % a.P.mp_interval == 0 && st.y < 0) {
    // phase q's pressure ends up in warp lane q
    long long mine = 0;
    const int b = a.ctrl_loff[c], e = a.ctrl_loff[c + 1];
    for (int j0 = b; j0 < e; j0 += 32) {
      const int j = j0 + lane;
      long long contrib = 0;
      int grp = -1;
      if (j < e) {
        const int l = a.ctrl_lanes[j];
        const LaneInfo li = a.li[l];
        const int ql = dyn[l].y;
        grp = li.group;
        for (int k = 0; k < li.n_succ; ++k) {
          if (a.link_off[li.succ + k]) continue;   // a closed link is no link
          const int tg = a.li[a.succ[li.succ + k].x].succ;   // internal lane's target
          contrib += ql - dyn[tg].y;
        }
      }
      for (int q = 0; q < cc.w; ++q) {
        long long v = grp == q ? contrib : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == q) mine += v;
      }
    }
    // highest pressure, lowest phase index on ties
    long long bv = lane < cc.w ? mine : LLONG_MIN;
    int bi = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    const long long gv = __shfl_sync(0xffffffffu, mine, st.x & 31);
    if (gv == bv) bi = st.x;
    if (bi != st.x) {
      if (cc.z > 0) {
        st.y = bi;
        st.z = t + cc.z;
      } else {
        st.x = bi;
      }
    }
  }
  if (lane == 0) {
    a.mp[c] = st;
    a.sig[p][c] = 2 * st.x + (st.y >= 0 ? 1 : 0);
  }
}

// Vehicle count and step of the state at step t, written into mapped host memory: the host
// learns how many entries to copy without a device-to-host copy that would queue behind
// an export in flight on the copy engine.  Step t + 1 does not write n_active[t & 1].
__global__ void k_export_meta(const DevCtrl *ctrl, int t, int *meta) {
  meta[0] = ctrl->n_active[t & 1];
  meta[1] = t;
}

__global__ void k_route_idx(const int *rp, const int *id, const int *route0, int *out, const int *n_ptr,
                            int n_fixed) {
  int n = n_ptr ? *n_ptr : n_fixed;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = rp[i] - route0[id[i]];
}

}  // namespace moss
