/*
 * moss_oracle.c -- FP64 CPU oracle of one simulation step (TEST INFRASTRUCTURE ONLY).
 *
 * Plain, obviously-correct restatement of the model, single-threaded unless or_set_threads
 * asks for more (then the update phase, where every vehicle reads only the snapshot and
 * writes only its own outputs, runs its vehicles on OpenMP threads; the results do not
 * depend on the thread count).  Only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline may load this library.
 *
 * What the paper fixes (Sec. III-A): two phases per step -- a prepare phase that indexes
 * vehicles by lane and position and takes a read-only copy of their motion state, and an
 * update phase in which each vehicle senses its neighbours (the vehicle ahead first),
 * computes IDM car following (Treiber, Hennecke & Helbing 2000) and a randomized MOBIL
 * lane-change decision (Kesting, Treiber & Helbing 2007), then advances by Newton's
 * equations; dt = 1 s (Sec. III-A, IV-A); fixed-time signals at junctions (Sec. III-C map
 * builder, Sec. IV-E "FP").  Everything else below is a reading of what the paper leaves
 * open, numbered R1, R2, ... and stated where it applies.
 *
 * Parity unpinned against the paper: the form of MOBIL's randomization (the R4 gate and
 * the R12 threshold jitter), which the paper does not give; those draws are pinned by the
 * published SplitMix64 vector, by CPU/GPU identity, and by the statistics the readings fix
 * (a gate passed with probability p_lc, drawn afresh per trip and step; a jitter uniform
 * over trips), not by the paper.
 *
 *  R1  IDM: a = a_max [1 - (v/v0)^4 - (ss/s)^2], ss = s0 + max(0, vT + v dv/(2 sqrt(a_max b))),
 *      dv = v - v_lead, s = bumper gap floored at 0.01 m; (v/v0)^4 by two squarings; no
 *      leader within d_look: the interaction term is dropped; result clamped to >= a_min.
 *  R2  Sensing: own-lane leader = next vehicle in the lane by position; if none, look ahead
 *      along the route through the lane's successor toward the next route edge, the
 *      internal junction lane and its target lane, up to d_look metres and 12 lanes; the
 *      first vehicle found is the leader (gap measured along the path).  A stopped virtual
 *      obstacle sits at a lane end when (a) the lane has no successor toward the next route
 *      edge, (b) the signal is red, (c) it is yellow and the vehicle can stop,
 *      dist >= v^2/(2b), (d) the 12-lane cap is reached.  On the destination edge the lane
 *      end is open (the vehicle leaves there).
 *  R3  Merges: a vehicle on an internal lane whose target lane has several feeding internal
 *      lanes also treats, on every other feeder f, the vehicle with the largest distance
 *      to the merge point d_f = len_f - x that is still below its own d (ties: lower id
 *      goes first) as a leader with gap d - d_f - L.  Internal lanes are >= 21 m and edge
 *      lanes >= 25 m, both longer than v_max dt, so only vehicles already on a feeder can
 *      reach a merge point within a step.
 *  R4  Randomized MOBIL: even steps only allow moves to the left lane, odd steps only to the
 *      right; a discretionary change is considered only if SplitMix64(seed ^ t<<32 ^ id)>>40
 *      < floor(p_lc 2^24); incentive a~_c - a_c + p[(a~_n - a_n) + (a~_o - a_o)] > th;
 *      safety a~_n >= -b_safe, new follower gap >= v_n dt + a_max dt^2/2, new leader gap > 0;
 *      no change on internal lanes or with x < x_lc_min; no discretionary change with
 *      len - x < x_lc_end or from a lane connecting to the next route edge into one that
 *      does not; if the own lane does not connect, the change toward the nearest connecting
 *      lane is mandatory (no incentive, no random gate, safety still applies).  The
 *      target-lane leader is searched in that lane only; past its end the same obstacle
 *      rules as R2 apply, evaluated from the vehicle's (or follower's) own position.
 *  R5  A changer accelerates with min(a_c, a~_c) and may not pass its own-lane leader, its
 *      new leader, or the lane end in the step it changes.
 *  R6  Motion (ballistic): v' = min(v + a dt, v_max) if positive, else v' = 0 and the
 *      distance is the stopping distance v^2/(-2a); otherwise d = (v+v')dt/2.  Safety clamp:
 *      d <= max(0, g_min) over the gaps of R5/R2; if clamped, v' = min(v', d/dt).  A vehicle
 *      whose own-lane end holds an obstacle (or that changes lane) stays at x' <= len.
 *  R7  Transfer: x' > len moves the vehicle to the successor toward the next route edge
 *      (edge lane -> internal lane) or to the internal lane's target (internal -> edge lane,
 *      route index + 1) with x' -= len; on the destination edge it arrives instead.
 *  R8  Departures: a trip waits in the FIFO (t_dep, id) of its departure lane, the
 *      lowest-index lane of its first edge connecting to its second edge; at step t the
 *      head with t_dep <= t enters at x = L, v = 0 if the lane's first vehicle in the
 *      snapshot has rear >= L + s0 and every vehicle entering the lane this step has
 *      rear >= L + s0.
 *  R9  Signals: state of group g of controller c at step t: tau = (t + offset) mod cycle,
 *      cycle = P (green + yellow); phase k = tau div (green + yellow); green if k == g and
 *      tau mod (green+yellow) < green, yellow if k == g otherwise, red if k != g.
 *  R10 Metrics: per lane and window w = t div window, the sum of speeds and the count of
 *      vehicles in the snapshot of each step.
 *  R11 Lane links fan out (every turning lane links to every lane of its exit edge, in a
 *      preferred order); a vehicle takes the first link whose target lane serves the route
 *      edge after the exit edge, so it enters each edge on a lane that serves its next turn.
 *  R13 Max-pressure signals (signal_mode 1; Varaiya 2013 with unit saturation flows, at
 *      lane level).  Each controller keeps a green phase g, a pending phase and the step
 *      at which it turns green.  At the start of step t, a pending phase whose time has
 *      come becomes g.  Then, at a decision step (t mod mp_interval = 0) with nothing
 *      pending, every phase's pressure is summed over the lane links of its approach
 *      lanes: the vehicles on the approach lane minus the vehicles on the link's target
 *      lane (snapshot counts at t).  The phase of highest pressure wins; g wins a tie it
 *      is in, else the lowest phase index.  A winner other than g turns g yellow for the
 *      controller's yellow time (then the winner is green), or at once when that is 0.
 *      Lanes of phase g are green, or yellow while a phase is pending; all others red.
 *      Controllers start with phase 0 green and nothing pending.
 *  R14 Lane modifications (set between steps): a lane's speed limit caps the desired
 *      speed of every vehicle on it, v0_eff = min(v0, vmax_lane), in all IDM terms -- the
 *      changer's prospective acceleration and the new follower's use the target lane's
 *      limit, the old follower's its own lane's.  A closed lane cannot be entered: a path
 *      that reaches it ends in a stopped obstacle at the end of the lane before it, it is
 *      never a lane-change target, and its departure queue waits.  Vehicles already on it
 *      drive on.
 *  R17 Dynamic lanes (set between steps): each lane link of an edge lane (one successor
 *      entry: the junction-internal lane of one movement) is open or closed.  A closed
 *      link is no link: the fan-out choice (R11), every test of whether a lane links
 *      toward an edge (mandatory changes, the lanes a discretionary change may target, the
 *      obstacle at a lane end) and the max-pressure sums (R13) skip it.  Vehicles already
 *      on its internal lane finish the movement; waiting trips keep the departure lanes
 *      assigned at load.  The caller keeps every remaining route lane-connected.
 *  R12 Threshold jitter (a randomized-MOBIL variant, off when th_jitter = 0): trip c's
 *      incentive threshold is th + th_jitter (2u - 1), u = (SplitMix64(seed ^ 0x9E3779B97F4A7C15
 *      ^ c) >> 40) / 2^24, fixed for the trip (driver heterogeneity); the salt keeps these
 *      draws apart from the per-step gate draws of R4 (whose low 32 bits are c alone).
 *  R19 Learned lane change (the surrogate of the learned form; not in the paper, off unless a
 *      model is set): for a discretionary candidate of R4 that passed every safety test, a
 *      16 -> 64 -> 64 -> 3 network (ReLU; softmax over stay / left / right) replaces the
 *      incentive test.  BF16 with FP32 accumulation fixes where values are rounded: the 16
 *      inputs, the weights, and both hidden layers after bias and ReLU are rounded to BF16
 *      (round to nearest even); biases stay as given; sums here are FP64.  Its class is
 *      taken when the softmax margin (top1 - top2) is >= margin, else the rule's decision;
 *      a left or right class against the step's allowed direction means stay.  Inputs:
 *      v/20, v0/20, own gap min(s,200)/100 (2 free), own closing speed (v-vl)/10 (v/10 at an
 *      obstacle, 0 free), a_c/a_max, the allowed direction, target gap and closing speed
 *      (same forms), new follower gap min(g,200)/100 (2 none), its speed /20 and its
 *      acceleration behind the changer /a_max (0 none), a~_c/a_max, old follower speed /20
 *      (0 none), distance to the lane end min(len-x,200)/100, leader speed /20 (0 obstacle,
 *      1 free), old follower gap min(g,200)/100 (2 none).
 *      Flag (the FP32 path rounds its own FP32 values, so a value whose FP64 form lies
 *      within the FP32 path's error of a BF16 rounding boundary may round the other way
 *      there): an input or hidden value within delta of a boundary is near; the decision is
 *      recomputed with each near value rounded the other way, and the candidate is flagged
 *      when any such change alters the decision, or when |margin - threshold| < 1e-3 plus
 *      the summed margin changes.  delta: inputs 2^-22 |f| plus 1e-5 (gap and distance
 *      inputs: FP32 gaps are within 1e-3 m) or 5e-5 (acceleration inputs: within 1e-4
 *      m/s^2); hidden units (K + 1) 2^-22 (sum of |terms| + |bias|), K the fan-in, four
 *      times the round-to-nearest bound of an FP32 sum of K products.
 */
#include "moss_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { SIG_GREEN = 0, SIG_YELLOW = 1, SIG_RED = 2 };
enum { K_FREE = 0, K_VEH = 1, K_OBST = 2 };
#define HOP_CAP 12
#define FLAG_EPS 1e-3
#define ST_WAIT 0
#define ST_ACTIVE 1
#define ST_DONE 2

struct or_sim {
  or_net net;
  or_params p;
  int n;             /* trips */
  const int *t_dep;
  const float *v0;
  const int64_t *route_off;
  const int *route_edges;
  /* dynamic per trip */
  int *status, *lane, *rp, *t_arr;
  double *x, *v;
  int t;
  /* derived: departure lane per trip, FIFO per lane */
  int *dep_lane;
  int *q_off, *q_ids, *q_head; /* CSR over lanes of trip ids sorted by (t_dep, id) */
  /* derived: feeders (internal lanes) of each lane */
  int *pred_off, *pred_ids;
  /* snapshot index */
  int n_act;
  int *order;       /* active trip ids sorted by (lane, x, id) */
  int *seg_start, *seg_cnt;
  int *pos;         /* trip id -> position in order */
  /* metrics */
  double *vsum;
  int64_t *vcnt;
  int64_t counters[4]; /* inserted, arrived, sum of travel times, errors */
  /* step outputs */
  int *n_lane, *n_rp, *n_status, *n_flag;
  double *n_x, *n_v;
  int threads;      /* threads of the update phase (OpenMP); 1: serial */
  /* R13 controllers */
  int *mp_g, *mp_pend, *mp_yend;
  int64_t *mp_pres;   /* per controller x phase pressure (scratch) */
  int *mp_poff;       /* phase offsets into mp_pres */
  /* R14 lane modifications */
  double *lane_vmax;  /* speed limit per lane, INFINITY = none */
  int *lane_closed;
  /* R17 dynamic lanes */
  unsigned char *link_off;   /* per successor entry: 1 = closed */
  /* R19 learned lane change (NULL: the rule alone) */
  struct or_mlp *mlp;
};

/* R19 network: weights rounded to BF16, biases as given, all held as doubles */
struct or_mlp {
  double w1[64][16], b1[64], w2[64][64], b2[64], w3[3][64], b3[3];
  double margin;
};

/* ------------------------------------------------------------------------------------ */
/* helpers                                                                               */
/* ------------------------------------------------------------------------------------ */

uint64_t or_splitmix64(uint64_t z) {
  /* SplitMix64 output function (Steele, Lea & Flood 2014): one increment by the golden
     gamma, then the two xor-shift-multiply rounds and a final xor-shift. */
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* R12: incentive threshold of trip c */
static double trip_threshold(const or_params *p, int c) {
  if (!(p->th_jitter > 0.0)) return p->th;
  const uint64_t h = or_splitmix64(p->seed ^ 0x9E3779B97F4A7C15ull ^ (uint64_t)(uint32_t)c);
  const double u = (double)(h >> 40) / 16777216.0;
  return p->th + p->th_jitter * (2.0 * u - 1.0);
}

static int is_internal(const or_sim *s, int l) { return s->net.lane_edge[l] < 0; }

static int connects(const or_sim *s, int l, int en) {
  if (en < 0) return 1;
  for (int k = s->net.succ_off[l]; k < s->net.succ_off[l + 1]; ++k)
    if (s->net.succ_edge[k] == en && !s->link_off[k]) return 1;   /* R17: open links only */
  return 0;
}

/* R11: successor of edge lane l toward edge en: among the internal lanes of l that lead to
   en (CSR order), the first whose target lane connects to the edge after, en2; the first
   one if none does or the route ends at en; -1 if l has none toward en. */
static int choose_succ(const or_sim *s, int l, int en, int en2) {
  int first = -1;
  for (int k = s->net.succ_off[l]; k < s->net.succ_off[l + 1]; ++k) {
    if (s->net.succ_edge[k] != en || s->link_off[k]) continue;   /* R17 */
    int il = s->net.succ_lane[k];
    if (first < 0) first = il;
    if (en2 < 0) return il;
    int tg = s->net.succ_lane[s->net.succ_off[il]];
    if (connects(s, tg, en2)) return il;
  }
  return first;
}

static int route_len(const or_sim *s, int id) {
  return (int)(s->route_off[id + 1] - s->route_off[id]);
}

static int route_at(const or_sim *s, int id, int k) {
  if (k < 0 || k >= route_len(s, id)) return -1;
  return s->route_edges[s->route_off[id] + k];
}

/* R13 */
static void mp_reset(or_sim *s) {
  for (int c = 0; c < s->net.n_ctrl; ++c) {
    s->mp_g[c] = 0;
    s->mp_pend[c] = -1;
    s->mp_yend[c] = 0;
  }
}

/* advance every controller to step s->t on the prepared snapshot (seg_cnt) */
static void mp_advance(or_sim *s) {
  const int t = s->t, C = s->net.n_ctrl;
  const int decide = (t % s->p.mp_interval) == 0;
  if (decide) {
    memset(s->mp_pres, 0, sizeof(int64_t) * (size_t)s->mp_poff[C]);
    for (int l = 0; l < s->net.n_lanes; ++l) {
      const int c = s->net.lane_ctrl[l];
      if (c < 0 || is_internal(s, l)) continue;
      int64_t sum = 0;
      for (int k = s->net.succ_off[l]; k < s->net.succ_off[l + 1]; ++k) {
        if (s->link_off[k]) continue;   /* R17 */
        const int il = s->net.succ_lane[k];
        const int m = s->net.succ_lane[s->net.succ_off[il]];
        sum += s->seg_cnt[l] - s->seg_cnt[m];
      }
      s->mp_pres[s->mp_poff[c] + s->net.lane_group[l]] += sum;
    }
  }
  for (int c = 0; c < C; ++c) {
    if (s->mp_pend[c] >= 0 && t >= s->mp_yend[c]) {
      s->mp_g[c] = s->mp_pend[c];
      s->mp_pend[c] = -1;
    }
    if (!decide || s->mp_pend[c] >= 0) continue;
    const int64_t *pr = s->mp_pres + s->mp_poff[c];
    const int np = s->net.ctrl_nphase[c];
    int best = 0;
    for (int ph = 1; ph < np; ++ph)
      if (pr[ph] > pr[best]) best = ph;
    if (pr[s->mp_g[c]] == pr[best]) best = s->mp_g[c];
    if (best == s->mp_g[c]) continue;
    if (s->net.ctrl_yellow[c] > 0) {
      s->mp_pend[c] = best;
      s->mp_yend[c] = t + s->net.ctrl_yellow[c];
    } else {
      s->mp_g[c] = best;
    }
  }
}

int or_signal_state(const or_sim *s, int l, int t) {
  int c = s->net.lane_ctrl[l];
  if (c < 0) return SIG_GREEN;
  if (s->p.signal_mode == 1) {   /* R13: the controllers' current state */
    if (s->net.lane_group[l] != s->mp_g[c]) return SIG_RED;
    return s->mp_pend[c] >= 0 ? SIG_YELLOW : SIG_GREEN;
  }
  int g = s->net.ctrl_green[c], y = s->net.ctrl_yellow[c], P = s->net.ctrl_nphase[c];
  int cyc = P * (g + y);
  int tau = ((t + s->net.ctrl_offset[c]) % cyc + cyc) % cyc;
  int k = tau / (g + y);
  if (k != s->net.lane_group[l]) return SIG_RED;
  return (tau % (g + y)) < g ? SIG_GREEN : SIG_YELLOW;
}

static void mark(int *flag, double margin) {
  if (fabs(margin) < FLAG_EPS) *flag = 1;
}

/* R14: desired speed of trip c on lane l */
static double v0_on(const or_sim *s, int c, int l) {
  return fmin((double)s->v0[c], s->lane_vmax[l]);
}

/* R1 */
static double idm(const or_sim *s, double v, double v0, int has_leader, double gap, double vl) {
  const or_params *p = &s->p;
  double r = v / v0;
  double r2 = r * r;
  double freeterm = 1.0 - r2 * r2;
  double a;
  if (!has_leader) {
    a = p->a * freeterm;
  } else {
    double dv = v - vl;
    double ss = p->s0 + fmax(0.0, v * p->T + v * dv / (2.0 * sqrt(p->a * p->b)));
    double q = ss / fmax(gap, 0.01);
    a = p->a * (freeterm - q * q);
  }
  return fmax(a, p->a_min);
}

/* ------------------------------------------------------------------------------------ */
/* prepare phase: index by (lane, position, id)                                          */
/* ------------------------------------------------------------------------------------ */

static const or_sim *g_sort_sim;
static int cmp_lane_x(const void *pa, const void *pb) {
  const or_sim *s = g_sort_sim;
  int a = *(const int *)pa, b = *(const int *)pb;
  if (s->lane[a] != s->lane[b]) return s->lane[a] < s->lane[b] ? -1 : 1;
  if (s->x[a] != s->x[b]) return s->x[a] < s->x[b] ? -1 : 1;
  return a < b ? -1 : (a > b);
}

static void prepare(or_sim *s) {
  int m = 0;
  for (int i = 0; i < s->n; ++i)
    if (s->status[i] == ST_ACTIVE) s->order[m++] = i;
  s->n_act = m;
  g_sort_sim = s;
  qsort(s->order, (size_t)m, sizeof(int), cmp_lane_x);
  memset(s->seg_cnt, 0, sizeof(int) * (size_t)s->net.n_lanes);
  for (int k = 0; k < m; ++k) s->seg_cnt[s->lane[s->order[k]]]++;
  int acc = 0;
  for (int l = 0; l < s->net.n_lanes; ++l) {
    s->seg_start[l] = acc;
    acc += s->seg_cnt[l];
  }
  for (int k = 0; k < m; ++k) s->pos[s->order[k]] = k;
}

/* first index in lane l's segment whose position is > x (segment-relative), by bisection */
static int seg_upper(const or_sim *s, int l, double x) {
  int lo = 0, hi = s->seg_cnt[l];
  const int *o = s->order + s->seg_start[l];
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (s->x[o[mid]] > x) hi = mid; else lo = mid + 1;
  }
  return lo;
}

/* ------------------------------------------------------------------------------------ */
/* update phase                                                                          */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  int kind;
  double gap, vl;
  int lead_id;
  int end_obstacle; /* obstacle at the end of the vehicle's own lane */
} leader_t;

/* R2 + R3: own-path leader of trip c */
static leader_t own_leader(const or_sim *s, int c, int *flag) {
  const double L = s->p.veh_len;
  leader_t r = {K_FREE, 0.0, 0.0, -1, 0};
  int l = s->lane[c];
  double x = s->x[c], v = s->v[c];
  int k = s->pos[c] - s->seg_start[l];
  if (k + 1 < s->seg_cnt[l]) {
    int j = s->order[s->seg_start[l] + k + 1];
    r.kind = K_VEH; r.gap = (s->x[j] - x) - L; r.vl = s->v[j]; r.lead_id = j;
  } else {
    double dist = (double)s->net.lane_len[l] - x;
    int cur = l, ri = s->rp[c];
    for (int hop = 0;; ++hop) {
      mark(flag, dist - s->p.d_look);
      if (dist >= s->p.d_look) break; /* free */
      int nxt;
      if (!is_internal(s, cur)) {
        int en = route_at(s, c, ri + 1);
        if (en < 0) break; /* destination edge: open end */
        nxt = choose_succ(s, cur, en, route_at(s, c, ri + 2));
        int stop = 0;
        if (nxt < 0) {
          stop = 1;
        } else {
          int sg = or_signal_state(s, cur, s->t);
          if (sg == SIG_RED) stop = 1;
          else if (sg == SIG_YELLOW) {
            double m = dist - v * v / (2.0 * s->p.b);
            mark(flag, m);
            if (m >= 0.0) stop = 1;
          }
        }
        if (stop) {
          r.kind = K_OBST; r.gap = dist; r.vl = 0.0; r.end_obstacle = (hop == 0);
          break;
        }
      } else {
        nxt = s->net.succ_lane[s->net.succ_off[cur]];
        ri += 1;
      }
      if (s->lane_closed[nxt]) {   /* R14 */
        r.kind = K_OBST; r.gap = dist; r.vl = 0.0; r.end_obstacle = (hop == 0);
        break;
      }
      if (hop + 1 >= HOP_CAP) {
        r.kind = K_OBST; r.gap = dist; r.vl = 0.0; r.end_obstacle = (hop == 0);
        break;
      }
      if (s->seg_cnt[nxt] > 0) {
        int j = s->order[s->seg_start[nxt]];
        r.kind = K_VEH; r.gap = (dist + s->x[j]) - L; r.vl = s->v[j]; r.lead_id = j;
        break;
      }
      dist += (double)s->net.lane_len[nxt];
      cur = nxt;
    }
  }
  /* R3: merge projection for vehicles on a feeder of a merge */
  if (is_internal(s, l)) {
    int tgt = s->net.succ_lane[s->net.succ_off[l]];
    if (s->pred_off[tgt + 1] - s->pred_off[tgt] > 1) {
      double dc = (double)s->net.lane_len[l] - x;
      for (int q = s->pred_off[tgt]; q < s->pred_off[tgt + 1]; ++q) {
        int f = s->pred_ids[q];
        if (f == l) continue;
        int cnt = s->seg_cnt[f];
        const int *o = s->order + s->seg_start[f];
        double lf = (double)s->net.lane_len[f];
        /* first j (ascending x) with d_j < dc or (d_j == dc and id_j < c) */
        int found = -1;
        for (int jj = 0; jj < cnt; ++jj) {
          int j = o[jj];
          double dj = lf - s->x[j];
          mark(flag, dc - dj);
          if (dj < dc || (dj == dc && j < c)) { found = j; break; }
        }
        if (found >= 0) {
          double dj = lf - s->x[found];
          double g = (dc - dj) - L;
          if (r.kind != K_FREE) mark(flag, g - r.gap);
          if (r.kind == K_FREE || g < r.gap) {
            r.kind = K_VEH; r.gap = g; r.vl = s->v[found]; r.lead_id = found;
            r.end_obstacle = 0;
          }
        }
      }
    }
  }
  return r;
}

/* obstacle rule at the end of an edge lane l (same edge as the vehicle), evaluated for a
   vehicle at (x, v) whose next route edge is en: returns 1 if the lane end is a stopped
   obstacle for it */
static int end_blocks(const or_sim *s, int l, int en, double x, double v, int *flag) {
  if (en < 0) return 0;
  if (!connects(s, l, en)) return 1;
  int sg = or_signal_state(s, l, s->t);
  if (sg == SIG_RED) return 1;
  if (sg == SIG_YELLOW) {
    double m = ((double)s->net.lane_len[l] - x) - v * v / (2.0 * s->p.b);
    mark(flag, m);
    return m >= 0.0;
  }
  return 0;
}

typedef struct {
  int dir, cand;
  int tau_lead, tau_foll, old_foll;
  double incentive;
  int tau_kind;
  double tau_gap, tau_vl;
  double a_new;
  int safe, mandatory, step_dir; /* every safety test passed; mandatory change; direction allowed */
  double gF, vF, aF_new;         /* new follower (tau_foll >= 0): gap, speed, acceleration behind */
} lc_t;


/* R4 */
static lc_t lane_change(const or_sim *s, int c, const leader_t *own, double a_c, int *flag) {
  const or_params *p = &s->p;
  const double L = p->veh_len;
  lc_t r;
  memset(&r, 0, sizeof(r));
  r.tau_lead = r.tau_foll = r.old_foll = -1;
  int l = s->lane[c];
  if (is_internal(s, l)) return r;
  double x = s->x[c], v = s->v[c], v0 = s->v0[c];
  double len = (double)s->net.lane_len[l];
  int en = route_at(s, c, s->rp[c] + 1);
  int step_dir = (s->t % 2 == 0) ? +1 : -1;
  int tau = step_dir > 0 ? s->net.lane_left[l] : s->net.lane_right[l];
  if (tau < 0) return r;
  if (s->lane_closed[tau]) return r;   /* R14 */
  int mandatory = !connects(s, l, en);
  r.mandatory = mandatory;
  r.step_dir = step_dir;
  if (mandatory) {
    /* nearest connecting lane on the same edge */
    int e = s->net.lane_edge[l];
    int l0 = s->net.edge_lane0[e], k = s->net.edge_nlanes[e];
    int idx = s->net.lane_index[l], best = -1, bestd = 1 << 30;
    for (int q = 0; q < k; ++q)
      if (connects(s, l0 + q, en) && abs(q - idx) < bestd) { bestd = abs(q - idx); best = q; }
    if (best < 0) return r;
    int want = best > idx ? +1 : -1;
    if (want != step_dir) return r;
  }
  mark(flag, x - p->x_lc_min);
  if (x < p->x_lc_min) return r;
  if (!mandatory) {
    if (!connects(s, tau, en)) return r;
    mark(flag, (len - x) - p->x_lc_end);
    if (len - x < p->x_lc_end) return r;
    uint64_t h = or_splitmix64(p->seed ^ ((uint64_t)(uint32_t)s->t << 32) ^ (uint64_t)(uint32_t)c);
    uint64_t thr = (uint64_t)floor(p->p_lc * 16777216.0);
    if ((h >> 40) >= thr) return r;
  }
  r.cand = 1;
  /* target-lane neighbours */
  int j = seg_upper(s, tau, x);
  int cnt = s->seg_cnt[tau];
  const int *o = s->order + s->seg_start[tau];
  int Lt = j < cnt ? o[j] : -1;
  int Ft = j > 0 ? o[j - 1] : -1;
  r.tau_lead = Lt;
  r.tau_foll = Ft;
  if (Lt >= 0) {
    r.tau_kind = K_VEH; r.tau_gap = (s->x[Lt] - x) - L; r.tau_vl = s->v[Lt];
  } else if (end_blocks(s, tau, en, x, v, flag)) {
    r.tau_kind = K_OBST; r.tau_gap = len - x; r.tau_vl = 0.0;
  } else {
    r.tau_kind = K_FREE;
  }
  if (r.tau_kind == K_VEH) {
    mark(flag, r.tau_gap);
    if (r.tau_gap <= 0.0) return r;
  }
  double aF_new = 0.0, gF = 0.0;
  if (Ft >= 0) {
    gF = (x - s->x[Ft]) - L;
    double guard = s->v[Ft] * p->dt + 0.5 * p->a * p->dt * p->dt;
    mark(flag, gF - guard);
    if (gF < guard) return r;
    aF_new = idm(s, s->v[Ft], v0_on(s, Ft, tau), 1, gF, v);
    mark(flag, aF_new + p->bsafe);
    if (aF_new < -p->bsafe) return r;
    r.gF = gF;
    r.vF = s->v[Ft];
    r.aF_new = aF_new;
  }
  r.safe = 1;
  r.a_new = idm(s, v, fmin(v0, s->lane_vmax[tau]), r.tau_kind != K_FREE, r.tau_gap, r.tau_vl);
  if (!mandatory) {
    double delta = r.a_new - a_c;
    if (Ft >= 0) {
      double aF_old;
      if (Lt >= 0) {
        aF_old = idm(s, s->v[Ft], v0_on(s, Ft, tau), 1, (s->x[Lt] - s->x[Ft]) - L, s->v[Lt]);
      } else if (end_blocks(s, tau, en, s->x[Ft], s->v[Ft], flag)) {
        aF_old = idm(s, s->v[Ft], v0_on(s, Ft, tau), 1, len - s->x[Ft], 0.0);
      } else {
        aF_old = idm(s, s->v[Ft], v0_on(s, Ft, tau), 0, 0.0, 0.0);
      }
      delta += p->p * (aF_new - aF_old);
    }
    int k = s->pos[c] - s->seg_start[l];
    if (k > 0) {
      int O = s->order[s->seg_start[l] + k - 1];
      r.old_foll = O;
      double gO = (x - s->x[O]) - L;
      double aO_old = idm(s, s->v[O], v0_on(s, O, l), 1, gO, v);
      double aO_new;
      if (own->kind != K_FREE)
        aO_new = idm(s, s->v[O], v0_on(s, O, l), 1, own->gap + (x - s->x[O]), own->vl);
      else
        aO_new = idm(s, s->v[O], v0_on(s, O, l), 0, 0.0, 0.0);
      delta += p->p * (aO_new - aO_old);
    }
    r.incentive = delta;
    const double th_c = trip_threshold(p, c);
    mark(flag, delta - th_c);
    if (!(delta > th_c)) return r;
  }
  r.dir = step_dir;
  return r;
}

/* ------------------------------------------------------------------------------------ */
/* R19: learned lane change                                                              */
/* ------------------------------------------------------------------------------------ */

/* BF16 (8 significant bits, 8-bit exponent) nearest to x, ties to even */
double or_bf16(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  int e;
  const double m = frexp(x, &e);              /* x = m 2^e, 0.5 <= |m| < 1 */
  if (e < -125) return nearbyint(ldexp(x, 133)) * ldexp(1.0, -133);   /* BF16 subnormals */
  return ldexp(nearbyint(ldexp(m, 8)), e - 8);
}

/* the BF16 value next to r (itself BF16, nonzero) away from zero (up = 1) or toward it */
static double bf16_next(double r, int up) {
  const double a = fabs(r);
  int e;
  frexp(a, &e);                               /* a = 2^(e-1) ... 2^e */
  const double ulp = ldexp(1.0, e - 1 - 7);
  const double n = up ? a + ulp : (a == ldexp(1.0, e - 1) ? a - ulp / 2 : a - ulp);
  return r < 0 ? -n : n;
}

/* v (FP64, rounded here to r) lies within delta of a BF16 rounding boundary: *alt is the
   value the other side of that boundary rounds to */
static int near_boundary(double v, double r, double delta, double *alt) {
  if (fabs(v) < 1e-30 || r == 0.0) return 0;
  const double out = bf16_next(r, 1), in = bf16_next(r, 0);
  if (fabs(v - 0.5 * (r + out)) <= delta) { *alt = out; return 1; }
  if (fabs(v - 0.5 * (r + in)) <= delta) { *alt = in; return 1; }
  return 0;
}

static void mlp_hidden1(const struct or_mlp *m, const double xb[16], double a1[64], double s1[64]) {
  for (int j = 0; j < 64; ++j) {
    double acc = 0.0, mag = 0.0;
    for (int k = 0; k < 16; ++k) {
      acc += m->w1[j][k] * xb[k];
      mag += fabs(m->w1[j][k] * xb[k]);
    }
    a1[j] = acc + m->b1[j];
    s1[j] = mag + fabs(m->b1[j]);
  }
}

static void mlp_hidden2(const struct or_mlp *m, const double h1[64], double a2[64], double s2[64]) {
  for (int j = 0; j < 64; ++j) {
    double acc = 0.0, mag = 0.0;
    for (int k = 0; k < 64; ++k) {
      acc += m->w2[j][k] * h1[k];
      mag += fabs(m->w2[j][k] * h1[k]);
    }
    a2[j] = acc + m->b2[j];
    s2[j] = mag + fabs(m->b2[j]);
  }
}

static void mlp_logits(const struct or_mlp *m, const double h2[64], double z[3]) {
  for (int q = 0; q < 3; ++q) {
    double acc = 0.0;
    for (int k = 0; k < 64; ++k) acc += m->w3[q][k] * h2[k];
    z[q] = acc + m->b3[q];
  }
}

/* softmax margin top1 - top2 and the argmax class (the lower class on a tie) */
static double mlp_margin(const double z[3], int *cls) {
  const double mx = fmax(z[0], fmax(z[1], z[2]));
  double pr[3], sum = 0.0;
  for (int q = 0; q < 3; ++q) sum += (pr[q] = exp(z[q] - mx));
  for (int q = 0; q < 3; ++q) pr[q] /= sum;
  int c = 0;
  for (int q = 1; q < 3; ++q)
    if (pr[q] > pr[c]) c = q;
  double sec = -1.0;
  for (int q = 0; q < 3; ++q)
    if (q != c && pr[q] > sec) sec = pr[q];
  *cls = c;
  return pr[c] - sec;
}

static int class_dir(int cls) { return cls == 1 ? +1 : (cls == 2 ? -1 : 0); }

/* decision (direction) from the network's class and margin, else the rule's */
static int learned_dir(const struct or_mlp *m, int cls, double mg, int rule_dir, int step_dir) {
  if (mg < m->margin) return rule_dir;
  const int d = class_dir(cls);
  return (d != 0 && d != step_dir) ? 0 : d;
}

/* the network from BF16 inputs xb, from hidden layer 1 (h1 given) or from hidden layer 2
   (h2 given): margin and class */
static double mlp_from(const struct or_mlp *m, const double *xb, const double *h1g, const double *h2g,
                       double z[3], int *cls) {
  double a1[64], s1[64], h1[64], a2[64], s2[64], h2[64];
  if (!h2g) {
    if (!h1g) {
      mlp_hidden1(m, xb, a1, s1);
      for (int j = 0; j < 64; ++j) h1[j] = or_bf16(fmax(a1[j], 0.0));
      h1g = h1;
    }
    mlp_hidden2(m, h1g, a2, s2);
    for (int j = 0; j < 64; ++j) h2[j] = or_bf16(fmax(a2[j], 0.0));
    h2g = h2;
  }
  mlp_logits(m, h2g, z);
  return mlp_margin(z, cls);
}

/* the 16 inputs of R19 for candidate c */
static void lc_inputs(const or_sim *s, int c, const leader_t *own, double a_c, const lc_t *lc, double f[16]) {
  const or_params *p = &s->p;
  const double L = p->veh_len;
  const int l = s->lane[c];
  const double x = s->x[c], v = s->v[c];
  const int k = s->pos[c] - s->seg_start[l];
  const int O = k > 0 ? s->order[s->seg_start[l] + k - 1] : -1;   /* old follower */
  f[0] = v / 20.0;
  f[1] = (double)s->v0[c] / 20.0;
  f[2] = own->kind != K_FREE ? fmin(own->gap, 200.0) / 100.0 : 2.0;
  f[3] = own->kind == K_VEH ? (v - own->vl) / 10.0 : (own->kind == K_OBST ? v / 10.0 : 0.0);
  f[4] = a_c / p->a;
  f[5] = (double)lc->step_dir;
  f[6] = lc->tau_kind != K_FREE ? fmin(lc->tau_gap, 200.0) / 100.0 : 2.0;
  f[7] = lc->tau_kind == K_VEH ? (v - lc->tau_vl) / 10.0 : (lc->tau_kind == K_OBST ? v / 10.0 : 0.0);
  f[8] = lc->tau_foll >= 0 ? fmin(lc->gF, 200.0) / 100.0 : 2.0;
  f[9] = lc->tau_foll >= 0 ? lc->vF / 20.0 : 0.0;
  f[10] = lc->tau_foll >= 0 ? lc->aF_new / p->a : 0.0;
  f[11] = lc->a_new / p->a;
  f[12] = O >= 0 ? s->v[O] / 20.0 : 0.0;
  f[13] = fmin((double)s->net.lane_len[l] - x, 200.0) / 100.0;
  f[14] = own->kind == K_VEH ? own->vl / 20.0 : (own->kind == K_OBST ? 0.0 : 1.0);
  f[15] = O >= 0 ? fmin((x - s->x[O]) - L, 200.0) / 100.0 : 2.0;
}

/* absolute part of the input error bound (see R19) */
static double input_delta(int k) {
  switch (k) {
    case 2: case 6: case 8: case 13: case 15: return 1e-5;   /* gaps, distance to the end */
    case 4: case 10: case 11: return 5e-5;                   /* accelerations */
    default: return 0.0;
  }
}

typedef struct {
  double f[16], z[3], margin;
  int cls, near, dir;
} learned_t;

/* R19 decision of candidate c (rule decision lc->dir) with its flag */
static learned_t learned_decision(const or_sim *s, int c, const leader_t *own, double a_c, const lc_t *lc,
                                  int *flag) {
  const struct or_mlp *m = s->mlp;
  learned_t r;
  lc_inputs(s, c, own, a_c, lc, r.f);
  double xb[16], a1[64], s1[64], h1[64], a2[64], s2[64], h2[64];
  for (int k = 0; k < 16; ++k) xb[k] = or_bf16(r.f[k]);
  mlp_hidden1(m, xb, a1, s1);
  for (int j = 0; j < 64; ++j) h1[j] = or_bf16(fmax(a1[j], 0.0));
  mlp_hidden2(m, h1, a2, s2);
  for (int j = 0; j < 64; ++j) h2[j] = or_bf16(fmax(a2[j], 0.0));
  mlp_logits(m, h2, r.z);
  r.margin = mlp_margin(r.z, &r.cls);
  r.dir = learned_dir(m, r.cls, r.margin, lc->dir, lc->step_dir);
  /* every value near a rounding boundary, rounded the other way */
  const double u = ldexp(1.0, -22);
  double sens = 0.0, alt, z2[3];
  int changes = 0, c2;
  r.near = 0;
  for (int k = 0; k < 16; ++k) {
    if (!near_boundary(r.f[k], xb[k], u * fabs(r.f[k]) + input_delta(k), &alt)) continue;
    double xa[16];
    memcpy(xa, xb, sizeof(xa));
    xa[k] = alt;
    const double mg = mlp_from(m, xa, NULL, NULL, z2, &c2);
    sens += fabs(mg - r.margin);
    changes |= learned_dir(m, c2, mg, lc->dir, lc->step_dir) != r.dir;
    r.near++;
  }
  for (int j = 0; j < 64; ++j) {
    const double hv = fmax(a1[j], 0.0);
    if (!near_boundary(hv, h1[j], 17.0 * u * s1[j], &alt)) continue;
    double ha[64];
    memcpy(ha, h1, sizeof(ha));
    ha[j] = alt;
    const double mg = mlp_from(m, NULL, ha, NULL, z2, &c2);
    sens += fabs(mg - r.margin);
    changes |= learned_dir(m, c2, mg, lc->dir, lc->step_dir) != r.dir;
    r.near++;
  }
  for (int j = 0; j < 64; ++j) {
    const double hv = fmax(a2[j], 0.0);
    if (!near_boundary(hv, h2[j], 65.0 * u * s2[j], &alt)) continue;
    double ha[64];
    memcpy(ha, h2, sizeof(ha));
    ha[j] = alt;
    const double mg = mlp_from(m, NULL, NULL, ha, z2, &c2);
    sens += fabs(mg - r.margin);
    changes |= learned_dir(m, c2, mg, lc->dir, lc->step_dir) != r.dir;
    r.near++;
  }
  if (changes || fabs(r.margin - m->margin) < FLAG_EPS + sens) *flag = 1;
  return r;
}

void or_set_threads(or_sim *s, int threads) { s->threads = threads > 1 ? threads : 1; }

int or_set_lc_model(or_sim *s, const float *theta, double margin) {
  if (!theta) {
    free(s->mlp);
    s->mlp = NULL;
    return 0;
  }
  if (!(margin >= 0.0 && margin <= 1.0)) return -1;
  if (!s->mlp) s->mlp = (struct or_mlp *)calloc(1, sizeof(struct or_mlp));
  struct or_mlp *m = s->mlp;
  const float *q = theta;   /* W1[64][16], b1[64], W2[64][64], b2[64], W3[3][64], b3[3] */
  for (int j = 0; j < 64; ++j)
    for (int k = 0; k < 16; ++k) m->w1[j][k] = or_bf16((double)*q++);
  for (int j = 0; j < 64; ++j) m->b1[j] = (double)*q++;
  for (int j = 0; j < 64; ++j)
    for (int k = 0; k < 64; ++k) m->w2[j][k] = or_bf16((double)*q++);
  for (int j = 0; j < 64; ++j) m->b2[j] = (double)*q++;
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 64; ++k) m->w3[j][k] = or_bf16((double)*q++);
  for (int j = 0; j < 3; ++j) m->b3[j] = (double)*q++;
  m->margin = margin;
  return 0;
}

int or_step(or_sim *s, or_debug *dbg) {
  const or_params *p = &s->p;
  const double L = p->veh_len;
  int err = 0;
  prepare(s);
  if (p->signal_mode == 1) mp_advance(s);   /* R13: controllers at step t */
  /* R10 metrics on the snapshot */
  int w = s->t / p->window;
  if (w < p->n_windows) {
    for (int k = 0; k < s->n_act; ++k) {
      int c = s->order[k];
      s->vsum[(size_t)w * s->net.n_lanes + s->lane[c]] += s->v[c];
      s->vcnt[(size_t)w * s->net.n_lanes + s->lane[c]] += 1;
    }
  }
  if (dbg) {
    for (int i = 0; i < s->n; ++i) { dbg->active_before[i] = 0; dbg->inserted[i] = 0; dbg->flag[i] = 0; }
  }
  /* update phase: every vehicle reads only the snapshot and writes only its own outputs,
     so the vehicles may be updated in any order or at once (or_set_threads) */
#pragma omp parallel for schedule(dynamic, 256) reduction(min : err) num_threads(s->threads) if (s->threads > 1)
  for (int k = 0; k < s->n_act; ++k) {
    int c = s->order[k];
    int flag = 0;
    int l = s->lane[c];
    double x = s->x[c], v = s->v[c];
    double len = (double)s->net.lane_len[l];
    leader_t own = own_leader(s, c, &flag);
    double a_c = idm(s, v, v0_on(s, c, s->lane[c]), own.kind != K_FREE, own.gap, own.vl);
    lc_t lc = lane_change(s, c, &own, a_c, &flag);
    int learned = 0;
    learned_t ln;
    if (s->mlp && lc.cand && lc.safe && !lc.mandatory) {   /* R19 */
      ln = learned_decision(s, c, &own, a_c, &lc, &flag);
      lc.dir = ln.dir;
      learned = 1;
    }
    double a_use = lc.dir ? fmin(a_c, lc.a_new) : a_c;
    /* R6 */
    double vraw = v + a_use * p->dt;
    double vn, d;
    if (vraw > 0.0) {
      vn = fmin(vraw, p->v_max);
      d = 0.5 * (v + vn) * p->dt;
    } else {
      vn = 0.0;
      d = v > 0.0 ? (v * v) / (-2.0 * a_use) : 0.0;
    }
    double gmin = INFINITY;
    if (own.kind != K_FREE) gmin = own.gap;
    if (lc.dir) {
      if (lc.tau_kind != K_FREE) gmin = fmin(gmin, lc.tau_gap);
      gmin = fmin(gmin, len - x);
    }
    double dmax = fmax(0.0, gmin);
    if (d > dmax) {
      d = dmax;
      vn = fmin(vn, d / p->dt);
    }
    double xn = x + d;
    if (own.end_obstacle || lc.dir) xn = fmin(xn, len);
    int nl = lc.dir ? (lc.dir > 0 ? s->net.lane_left[l] : s->net.lane_right[l]) : l;
    int nrp = s->rp[c];
    int nst = ST_ACTIVE;
    /* R7 */
    if (!lc.dir) {
      mark(&flag, xn - len);
      if (xn > len) {
        if (!is_internal(s, l) && route_at(s, c, s->rp[c] + 1) < 0) {
          nst = ST_DONE;
        } else {
          xn -= len;
          if (!is_internal(s, l)) {
            nl = choose_succ(s, l, route_at(s, c, s->rp[c] + 1), route_at(s, c, s->rp[c] + 2));
          } else {
            nl = s->net.succ_lane[s->net.succ_off[l]];
            nrp += 1;
          }
          if (nl < 0 || xn > (double)s->net.lane_len[nl]) { err = -3; nl = l; }
        }
      }
    }
    s->n_lane[c] = nl;
    s->n_x[c] = xn;
    s->n_v[c] = vn;
    s->n_rp[c] = nrp;
    s->n_status[c] = nst;
    s->n_flag[c] = flag;
    if (dbg) {
      dbg->active_before[c] = 1;
      dbg->lead_kind[c] = own.kind;
      dbg->lead_id[c] = own.lead_id;
      dbg->s_own[c] = own.gap;
      dbg->vl_own[c] = own.vl;
      dbg->a_own[c] = a_c;
      dbg->lc_dir[c] = lc.dir;
      dbg->lc_cand[c] = lc.cand;
      dbg->tau_lead[c] = lc.tau_lead;
      dbg->tau_foll[c] = lc.tau_foll;
      dbg->old_foll[c] = lc.old_foll;
      dbg->incentive[c] = lc.incentive;
      dbg->a_use[c] = a_use;
      dbg->flag[c] = flag;
      if (dbg->lc_learn) {
        dbg->lc_learn[c] = learned;
        if (learned) {
          dbg->lc_margin[c] = ln.margin;
          dbg->lc_near[c] = ln.near;
          for (int q = 0; q < 3; ++q) dbg->lc_logit[3 * c + q] = ln.z[q];
          for (int q = 0; q < 16; ++q) dbg->lc_feat[16 * c + q] = ln.f[q];
        }
      }
    }
  }
  /* per-lane minimum rear of the vehicles entering the lane this step (R8), and whether a
     flagged vehicle enters it */
  double *arr_min = (double *)malloc(sizeof(double) * (size_t)s->net.n_lanes);
  for (int l = 0; l < s->net.n_lanes; ++l) arr_min[l] = INFINITY;
  int *arr_flag = (int *)calloc((size_t)s->net.n_lanes, sizeof(int));
  for (int k = 0; k < s->n_act; ++k) {
    const int c = s->order[k], nl = s->n_lane[c];
    if (s->n_status[c] == ST_ACTIVE && nl != s->lane[c]) {
      arr_min[nl] = fmin(arr_min[nl], s->n_x[c] - L);
      if (s->n_flag[c]) arr_flag[nl] = 1;
    }
  }
  /* R8 departures, decided on the snapshot (before the update is applied) */
  int n_ins = 0;
  int *ins = (int *)malloc(sizeof(int) * (size_t)(s->net.n_lanes + 1));
  for (int l = 0; l < s->net.n_lanes; ++l) {
    int qe = s->q_off[l + 1];
    while (s->q_head[l] < qe && s->status[s->q_ids[s->q_head[l]]] != ST_WAIT) s->q_head[l]++;
    if (s->q_head[l] >= qe) continue;
    int h = s->q_ids[s->q_head[l]];
    if (s->t_dep[h] > s->t) continue;
    if (s->lane_closed[l]) continue;   /* R14: the queue waits */
    int fl = 0;
    int room = 1;
    if (s->seg_cnt[l] > 0) {
      int tail = s->order[s->seg_start[l]];
      double m = (s->x[tail] - L) - (L + p->s0);
      mark(&fl, m);
      if (m < 0.0) room = 0;
    }
    if (arr_min[l] < INFINITY) {
      double m = arr_min[l] - (L + p->s0);
      mark(&fl, m);
      if (m < 0.0) room = 0;
    }
    if (arr_flag[l]) fl = 1;
    if (dbg && fl) dbg->flag[h] = 1;
    if (room) {
      ins[n_ins++] = h;
      s->q_head[l]++;
    }
  }
  /* apply the update synchronously */
  for (int k = 0; k < s->n_act; ++k) {
    int c = s->order[k];
    if (s->n_status[c] == ST_DONE) {
      s->status[c] = ST_DONE;
      s->t_arr[c] = s->t + 1;
      s->counters[1] += 1;
      s->counters[2] += (int64_t)(s->t + 1 - s->t_dep[c]);
    } else {
      s->lane[c] = s->n_lane[c];
      s->x[c] = s->n_x[c];
      s->v[c] = s->n_v[c];
      s->rp[c] = s->n_rp[c];
    }
  }
  for (int q = 0; q < n_ins; ++q) {
    int h = ins[q];
    s->status[h] = ST_ACTIVE;
    s->lane[h] = s->dep_lane[h];
    s->x[h] = L;
    s->v[h] = 0.0;
    s->rp[h] = 0;
    s->counters[0] += 1;
    if (dbg) dbg->inserted[h] = 1;
  }
  free(ins);
  free(arr_min);
  free(arr_flag);
  if (err) s->counters[3] += 1;
  s->t += 1;
  return err;
}

int or_run(or_sim *s, int n_steps) {
  int err = 0;
  for (int k = 0; k < n_steps; ++k) {
    int e = or_step(s, NULL);
    if (e && !err) err = e;
  }
  return err;
}

/* ------------------------------------------------------------------------------------ */
/* construction and state access                                                         */
/* ------------------------------------------------------------------------------------ */

int or_departure_lane(const or_sim *s, int trip) {
  int e0 = route_at(s, trip, 0);
  int e1 = route_at(s, trip, 1);
  int l0 = s->net.edge_lane0[e0], k = s->net.edge_nlanes[e0];
  if (e1 < 0) return l0;
  for (int q = 0; q < k; ++q)
    if (connects(s, l0 + q, e1)) return l0 + q;
  return -1;
}

static const or_sim *g_q_sim;
static int cmp_dep(const void *pa, const void *pb) {
  const or_sim *s = g_q_sim;
  int a = *(const int *)pa, b = *(const int *)pb;
  if (s->dep_lane[a] != s->dep_lane[b]) return s->dep_lane[a] < s->dep_lane[b] ? -1 : 1;
  if (s->t_dep[a] != s->t_dep[b]) return s->t_dep[a] < s->t_dep[b] ? -1 : 1;
  return a < b ? -1 : (a > b);
}

or_sim *or_create(const or_net *net, const or_params *p, int n_trips, const int *t_dep,
                  const float *v0, const int64_t *route_off, const int *route_edges,
                  const int *lane0, const float *x0, const float *vinit) {
  or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
  s->net = *net;
  s->p = *p;
  s->n = n_trips;
  s->t_dep = t_dep;
  s->v0 = v0;
  s->route_off = route_off;
  s->route_edges = route_edges;
  size_t n = (size_t)n_trips, L = (size_t)net->n_lanes;
  s->status = (int *)calloc(n, sizeof(int));
  s->lane = (int *)calloc(n, sizeof(int));
  s->rp = (int *)calloc(n, sizeof(int));
  s->t_arr = (int *)malloc(n * sizeof(int));
  s->x = (double *)calloc(n, sizeof(double));
  s->v = (double *)calloc(n, sizeof(double));
  s->dep_lane = (int *)malloc(n * sizeof(int));
  s->order = (int *)malloc((n + 1) * sizeof(int));
  s->pos = (int *)malloc((n + 1) * sizeof(int));
  s->seg_start = (int *)calloc(L, sizeof(int));
  s->seg_cnt = (int *)calloc(L, sizeof(int));
  s->n_lane = (int *)malloc((n + 1) * sizeof(int));
  s->n_rp = (int *)malloc((n + 1) * sizeof(int));
  s->n_status = (int *)malloc((n + 1) * sizeof(int));
  s->n_flag = (int *)malloc((n + 1) * sizeof(int));
  s->threads = 1;
  s->n_x = (double *)malloc((n + 1) * sizeof(double));
  s->n_v = (double *)malloc((n + 1) * sizeof(double));
  s->vsum = (double *)calloc((size_t)p->n_windows * L, sizeof(double));
  s->vcnt = (int64_t *)calloc((size_t)p->n_windows * L, sizeof(int64_t));
  {
    const int C = net->n_ctrl;
    s->mp_g = (int *)calloc((size_t)C + 1, sizeof(int));
    s->mp_pend = (int *)calloc((size_t)C + 1, sizeof(int));
    s->mp_yend = (int *)calloc((size_t)C + 1, sizeof(int));
    s->mp_poff = (int *)calloc((size_t)C + 1, sizeof(int));
    for (int c = 0; c < C; ++c) s->mp_poff[c + 1] = s->mp_poff[c] + net->ctrl_nphase[c];
    s->mp_pres = (int64_t *)calloc((size_t)s->mp_poff[C] + 1, sizeof(int64_t));
  }
  s->link_off = (unsigned char *)calloc((size_t)net->succ_off[L] + 1, 1);
  s->lane_vmax = (double *)malloc(sizeof(double) * (size_t)L);
  s->lane_closed = (int *)calloc((size_t)L, sizeof(int));
  for (int l = 0; l < L; ++l) s->lane_vmax[l] = INFINITY;
  for (size_t i = 0; i < n; ++i) {
    s->t_arr[i] = -1;
    if (lane0 && lane0[i] >= 0) {
      s->status[i] = ST_ACTIVE;
      s->lane[i] = lane0[i];
      s->x[i] = x0[i];
      s->v[i] = vinit[i];
    }
    s->dep_lane[i] = or_departure_lane(s, (int)i);
  }
  /* departure FIFOs */
  int *ids = (int *)malloc((n + 1) * sizeof(int));
  for (size_t i = 0; i < n; ++i) ids[i] = (int)i;
  g_q_sim = s;
  qsort(ids, n, sizeof(int), cmp_dep);
  s->q_off = (int *)calloc(L + 1, sizeof(int));
  s->q_head = (int *)calloc(L, sizeof(int));
  for (size_t i = 0; i < n; ++i)
    if (s->dep_lane[i] >= 0) s->q_off[s->dep_lane[i] + 1]++;
  for (size_t l = 0; l < L; ++l) s->q_off[l + 1] += s->q_off[l];
  s->q_ids = ids; /* sorted by (dep_lane, t_dep, id); lanes with dep_lane < 0 sort first */
  int skip = 0;
  for (size_t i = 0; i < n; ++i)
    if (s->dep_lane[i] < 0) skip++;
  for (size_t l = 0; l <= L; ++l) s->q_off[l] += skip;
  for (size_t l = 0; l < L; ++l) s->q_head[l] = s->q_off[l];
  /* feeders of each lane */
  s->pred_off = (int *)calloc(L + 1, sizeof(int));
  for (size_t l = 0; l < L; ++l)
    if (net->lane_edge[l] < 0) s->pred_off[net->succ_lane[net->succ_off[l]] + 1]++;
  for (size_t l = 0; l < L; ++l) s->pred_off[l + 1] += s->pred_off[l];
  s->pred_ids = (int *)malloc(sizeof(int) * (size_t)(s->pred_off[L] + 1));
  int *fill = (int *)calloc(L, sizeof(int));
  for (size_t l = 0; l < L; ++l)
    if (net->lane_edge[l] < 0) {
      int tg = net->succ_lane[net->succ_off[l]];
      s->pred_ids[s->pred_off[tg] + fill[tg]++] = (int)l;
    }
  free(fill);
  mp_reset(s);
  return s;
}

void or_destroy(or_sim *s) {
  if (!s) return;
  free(s->mp_g); free(s->mp_pend); free(s->mp_yend); free(s->mp_pres); free(s->mp_poff);
  free(s->lane_vmax); free(s->lane_closed); free(s->link_off);
  free(s->status); free(s->lane); free(s->rp); free(s->t_arr); free(s->x); free(s->v);
  free(s->dep_lane); free(s->order); free(s->pos); free(s->seg_start); free(s->seg_cnt);
  free(s->n_lane); free(s->n_rp); free(s->n_status); free(s->n_flag); free(s->n_x); free(s->n_v);
  free(s->vsum); free(s->vcnt); free(s->q_off); free(s->q_head); free(s->q_ids);
  free(s->pred_off); free(s->pred_ids); free(s->mlp);
  free(s);
}

void or_get_state(const or_sim *s, int *status, int *lane, double *x, double *v, int *rp,
                  int *t_arr, int *t) {
  size_t n = (size_t)s->n;
  if (status) memcpy(status, s->status, n * sizeof(int));
  if (lane) memcpy(lane, s->lane, n * sizeof(int));
  if (x) memcpy(x, s->x, n * sizeof(double));
  if (v) memcpy(v, s->v, n * sizeof(double));
  if (rp) memcpy(rp, s->rp, n * sizeof(int));
  if (t_arr) memcpy(t_arr, s->t_arr, n * sizeof(int));
  if (t) *t = s->t;
}

void or_set_state(or_sim *s, const int *status, const int *lane, const double *x,
                  const double *v, const int *rp, const int *t_arr, int t) {
  size_t n = (size_t)s->n;
  memcpy(s->status, status, n * sizeof(int));
  memcpy(s->lane, lane, n * sizeof(int));
  memcpy(s->x, x, n * sizeof(double));
  memcpy(s->v, v, n * sizeof(double));
  memcpy(s->rp, rp, n * sizeof(int));
  if (t_arr) memcpy(s->t_arr, t_arr, n * sizeof(int));
  s->t = t;
  for (int l = 0; l < s->net.n_lanes; ++l) s->q_head[l] = s->q_off[l];
  mp_reset(s);
}

void or_set_lane_limits(or_sim *s, int n, const int *lanes, const float *vmax, const int *closed) {
  for (int k = 0; k < n; ++k) {
    const int l = lanes[k];
    if (l < 0 || l >= s->net.n_lanes) continue;
    if (vmax) s->lane_vmax[l] = (vmax[k] > 0.0f && isfinite(vmax[k])) ? (double)vmax[k] : INFINITY;
    if (closed) s->lane_closed[l] = closed[k] != 0;
  }
}

int or_set_links(or_sim *s, int n, const int *lanes, const unsigned *open_mask) {
  for (int k = 0; k < n; ++k) {   /* validate first: nothing changes on a bad entry */
    const int l = lanes[k];
    if (l < 0 || l >= s->net.n_lanes || is_internal(s, l)) return -1;
    if (s->net.succ_off[l + 1] - s->net.succ_off[l] > 32) return -1;
  }
  for (int k = 0; k < n; ++k) {
    const int l = lanes[k];
    for (int j = s->net.succ_off[l]; j < s->net.succ_off[l + 1]; ++j)
      s->link_off[j] = !((open_mask[k] >> (j - s->net.succ_off[l])) & 1u);
  }
  return 0;
}

void or_get_ctrl_state(or_sim *s, int *out) {
  if (s->p.signal_mode == 1) {
    prepare(s);
    mp_advance(s);
  }
  for (int c = 0; c < s->net.n_ctrl; ++c) {
    out[3 * c] = s->mp_g[c];
    out[3 * c + 1] = s->mp_pend[c];
    out[3 * c + 2] = s->mp_yend[c];
  }
}

void or_set_ctrl_state(or_sim *s, const int *in) {
  for (int c = 0; c < s->net.n_ctrl; ++c) {
    s->mp_g[c] = in[3 * c];
    s->mp_pend[c] = in[3 * c + 1];
    s->mp_yend[c] = in[3 * c + 2];
  }
}

void or_get_metrics(const or_sim *s, double *vsum, int64_t *vcnt, int64_t *counters) {
  size_t m = (size_t)s->p.n_windows * (size_t)s->net.n_lanes;
  if (vsum) memcpy(vsum, s->vsum, m * sizeof(double));
  if (vcnt) memcpy(vcnt, s->vcnt, m * sizeof(int64_t));
  if (counters) memcpy(counters, s->counters, sizeof(s->counters));
}

void or_neighbors(or_sim *s, int *out) {
  prepare(s);
  for (int i = 0; i < 6 * s->n; ++i) out[i] = -1;
  for (int k = 0; k < s->n_act; ++k) {
    int c = s->order[k];
    int l = s->lane[c];
    int kk = s->pos[c] - s->seg_start[l];
    const int *o = s->order + s->seg_start[l];
    if (kk + 1 < s->seg_cnt[l]) out[6 * c + 0] = o[kk + 1];
    if (kk > 0) out[6 * c + 1] = o[kk - 1];
    int side[2] = {s->net.lane_left[l], s->net.lane_right[l]};
    for (int q = 0; q < 2; ++q) {
      int tau = side[q];
      if (tau < 0) continue;
      int j = seg_upper(s, tau, s->x[c]);
      const int *ot = s->order + s->seg_start[tau];
      if (j < s->seg_cnt[tau]) out[6 * c + 2 + 2 * q] = ot[j];
      if (j > 0) out[6 * c + 3 + 2 * q] = ot[j - 1];
    }
  }
}
