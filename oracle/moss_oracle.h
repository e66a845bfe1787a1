/*
 * moss_oracle.h -- FP64 CPU oracle of the per-time-step vehicle update (TEST INFRASTRUCTURE).
 *
 * This is the slow, plain reference that the CUDA path is checked against.  Only tests/,
 * __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm may load it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * The step follows Sec. III-A of the paper: a prepare phase that indexes vehicles by lane
 * and position from a read-only snapshot, then an update phase in which every vehicle
 * senses its environment, computes IDM car following (Treiber 2000) and a randomized
 * MOBIL lane-change decision (Kesting 2007), and advances by Newton's equations of motion
 * (dt = 1 s by default, Sec. III-A / IV-A).  Every rule the paper leaves open is fixed by
 * the readings listed in the header comment of moss_oracle.c.
 */
#ifndef MOSS_ORACLE_H
#define MOSS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n_lanes, n_edges, n_ctrl;
  const float *lane_len;
  const int *lane_edge, *lane_index, *lane_left, *lane_right;
  const int *succ_off, *succ_lane, *succ_edge;
  const int *lane_ctrl, *lane_group;
  const int *ctrl_offset, *ctrl_green, *ctrl_yellow, *ctrl_nphase;
  const int *edge_nlanes, *edge_lane0;
} or_net;

typedef struct {
  double dt, veh_len, a, b, T, s0;
  double p, th, bsafe, p_lc, a_min, v_max, d_look, x_lc_min, x_lc_end;
  int window, n_windows;
  uint64_t seed;
  double th_jitter;   /* R12: half-width of each trip's incentive-threshold offset (0: off) */
  int signal_mode;    /* 0: fixed-time plans (R9); 1: max pressure (R13) */
  int mp_interval;    /* R13: steps between phase decisions */
} or_params;

/* per-vehicle record of one step (indexed by trip id; valid where active_before == 1) */
typedef struct {
  int *active_before;
  int *lead_kind;    /* 0 free, 1 vehicle, 2 stopped obstacle */
  int *lead_id;      /* trip id of the leader, -1 if none/obstacle */
  double *s_own, *vl_own, *a_own;
  int *lc_dir;       /* -1 right, 0 none, +1 left */
  int *lc_cand;      /* 1 if a target lane was evaluated */
  int *tau_lead, *tau_foll, *old_foll;  /* ids, -1 none */
  double *incentive;
  double *a_use;
  int *flag;         /* 1 if any decision margin was within eps of its threshold */
  int *inserted;     /* trip ids inserted this step get 1 */
  /* R19 learned lane change (all NULL, or all set): lc_learn 1 where the network decided;
     there its softmax margin, logits [3 per trip], inputs before rounding [16 per trip]
     and the number of its values near a BF16 rounding boundary */
  int *lc_learn;
  double *lc_margin, *lc_logit, *lc_feat;
  int *lc_near;
} or_debug;

typedef struct or_sim or_sim;

or_sim *or_create(const or_net *net, const or_params *p, int n_trips, const int *t_dep,
                  const float *v0, const int64_t *route_off, const int *route_edges,
                  const int *lane0, const float *x0, const float *vinit);
void or_destroy(or_sim *s);
/* threads of the update phase (OpenMP; default 1).  Every vehicle's update reads only the
   snapshot and writes only its own outputs, so results do not depend on the count. */
void or_set_threads(or_sim *s, int threads);
/* one step; dbg may be NULL.  Returns 0, or a negative error code. */
int or_step(or_sim *s, or_debug *dbg);
int or_run(or_sim *s, int n_steps);
/* status: 0 waiting, 1 active, 2 arrived; rp is the route index of the current edge
   (approach edge on junction-internal lanes) */
void or_get_state(const or_sim *s, int *status, int *lane, double *x, double *v, int *rp,
                  int *t_arr, int *t);
void or_set_state(or_sim *s, const int *status, const int *lane, const double *x,
                  const double *v, const int *rp, const int *t_arr, int t);
/* per-window per-lane speed sums and counts [n_windows][n_lanes] */
void or_get_metrics(const or_sim *s, double *vsum, int64_t *vcnt, int64_t *counters);
int or_signal_state(const or_sim *s, int lane, int t); /* 0 green, 1 yellow, 2 red */
/* R13 controller state, 3 ints per controller: green phase, pending phase (-1 none), step
   at which the pending phase turns green.  or_create / or_set_state reset it to {0, -1, 0}.
   The getter first advances the controllers to the current step t (on the snapshot at t;
   advancing twice to the same step changes nothing), so it reports the state step t uses. */
void or_get_ctrl_state(or_sim *s, int *out);
/* R14 lane modifications, in effect from the next step: for lanes[k], a speed limit vmax[k]
   (m/s; <= 0 or non-finite: none) and closed[k] (0 / 1).  Either array may be NULL. */
void or_set_lane_limits(or_sim *s, int n, const int *lanes, const float *vmax, const int *closed);
void or_set_ctrl_state(or_sim *s, const int *in);
/* R17 dynamic lanes, in effect from the next step: for edge lane lanes[k], bit j of
   open_mask[k] opens (1) or closes (0) its j-th lane link (successor entry, CSR order).
   Returns -1 (nothing changed) for an internal or out-of-range lane or more than 32 links. */
int or_set_links(or_sim *s, int n, const int *lanes, const unsigned *open_mask);
uint64_t or_splitmix64(uint64_t state);
/* R19: the learned lane-change network (theta: 5443 floats, W1[64][16], b1[64], W2[64][64],
   b2[64], W3[3][64], b3[3], out x in) and its margin in [0, 1]; theta NULL: the rule alone.
   Returns -1 for a margin outside [0, 1]. */
int or_set_lc_model(or_sim *s, const float *theta, double margin);
/* BF16 value nearest to x (round to nearest, ties to even) */
double or_bf16(double x);
/* neighbour search on the current snapshot (for the brute-force check): for each trip id:
   own-lane leader, own-lane follower, left-lane leader/follower, right-lane leader/follower
   (ids or -1) -> out[6*n_trips] */
void or_neighbors(or_sim *s, int *out);
int or_departure_lane(const or_sim *s, int trip);

#ifdef __cplusplus
}
#endif
#endif
