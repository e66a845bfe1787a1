/*
 * moss103.h -- C ABI of the B300 (sm_103a) per-time-step vehicle update of a lane-level
 * microscopic traffic simulator (arxiv 2405.12520, MOSS, Sec. III-A).
 *
 * One simulation step t -> t+1 has the paper's two phases (Sec. III-A): a prepare phase
 * that indexes vehicles by lane and position from a read-only snapshot, and an update phase
 * in which every vehicle senses its neighbours, computes IDM car following and a randomized
 * MOBIL lane-change decision, and advances by Newton's equations of motion.  The simulator
 * takes a lane-level road network and trip demand as input and produces per-vehicle
 * position and speed every step and per-lane mean speeds (Sec. III-A, last paragraph).
 *
 * Conventions for every entry point:
 *  - return value: MS_OK (0) or a negative MS_ERR_* code; ms_last_error() then holds a
 *    one-line message.  A failed call leaves the simulation unchanged unless noted.
 *  - host arrays passed in are read during the call only and copied; the library owns all
 *    device memory it allocates (cudaMalloc at load time, freed by ms_destroy).
 *  - lane ids: the lanes of edge e are edge_lane0[e] + idx (idx 0 rightmost); junction-
 *    internal lanes have lane_edge -1.  Positions x are the front bumper along the lane from
 *    its start, metres; speeds m/s; FP32.
 *  - not thread-safe per ms_sim; distinct ms_sim objects are independent.
 */
#ifndef MOSS103_H
#define MOSS103_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MS_OK 0
#define MS_ERR_ARG (-1)      /* invalid argument or input data (message says which) */
#define MS_ERR_ROUTE (-2)    /* a route has consecutive edges without a lane link */
#define MS_ERR_CAPACITY (-3) /* more vehicles than the simulation was sized for */
#define MS_ERR_CUDA (-4)     /* a CUDA runtime call failed */
#define MS_ERR_DEVICE (-5)   /* a device-side check set an error bit (see ms_metrics.err) */
#define MS_ERR_STATE (-6)    /* call out of order (e.g. step before load) */

/* device error bits (ms_metrics.err) */
#define MS_DEV_HOP 1u        /* a vehicle crossed more than one lane end in a step */
#define MS_DEV_SCAN 2u       /* reserved (the lane scan no longer waits on other blocks) */
#define MS_DEV_ORDER 4u      /* debug check: output not sorted by (lane, x) or gap < 0 */
#define MS_DEV_BUCKET 8u     /* a moved vehicle did not find its merge record */
#define MS_DEV_TIMEOUT 16u   /* a kernel's wait for its own shared-memory copies ran out (the
                                kernel stopped; the step's results are not valid) */

/* Model parameters.  Values the paper fixes: dt (1 s, Sec. III-A, IV-A); the model families
   (IDM, randomized MOBIL, Sec. III-A).  All other values are parameters of those models or
   readings of what the paper leaves open. */
typedef struct ms_params {
  float dt;        /* s, step length */
  float veh_len;   /* m, vehicle length L (all vehicles) */
  float idm_a;     /* m/s^2, IDM maximum acceleration */
  float idm_b;     /* m/s^2, IDM comfortable deceleration */
  float idm_T;     /* s, IDM time headway */
  float idm_s0;    /* m, IDM jam distance */
  float mobil_p;   /* MOBIL politeness */
  float mobil_th;  /* m/s^2, MOBIL threshold */
  float mobil_bsafe; /* m/s^2, MOBIL safe braking */
  float p_lc;      /* probability that a discretionary lane change is considered, [0,1] */
  float a_min;     /* m/s^2, emergency deceleration bound (negative) */
  float v_max;     /* m/s, speed cap; every lane must be longer than v_max*dt */
  float d_look;    /* m, look-ahead horizon for the leader search */
  float x_lc_min;  /* m, no lane change with x below this */
  float x_lc_end;  /* m, no discretionary lane change within this distance of the lane end */
  int window;      /* steps per metric window (per-lane mean speed) */
  int n_windows;   /* metric windows kept on the device (steps beyond are not recorded) */
  uint64_t seed;   /* seed of the counter-based lane-change gate */
  int debug;       /* 1: record per-vehicle sensing and decisions of each step (tests) */
  int block;       /* threads per block of the vehicle kernels, multiple of 32 (0: 256) */
  int id_base;     /* added to trip ids in the lane-change gate hash (0; a stand-alone run of
                      one scenario of a batch sets it to the scenario's first trip id) */
  float mobil_th_jitter; /* m/s^2, >= 0: randomized-MOBIL variant -- trip i's incentive
                      threshold is mobil_th + mobil_th_jitter * (2u - 1), with u the top 24
                      bits of SplitMix64(seed ^ 0x9E3779B97F4A7C15 ^ (i + id_base)) / 2^24,
                      fixed for the trip (driver heterogeneity; Sec. III-A "randomized
                      improvement" leaves the form open); 0 = off */
  int signal_mode;  /* 0: fixed-time plans (ctrl_offset/green/yellow, Sec. IV-E "FP");
                       1: max pressure (the paper's MP baseline, Sec. IV-E; Varaiya 2013 with
                       unit saturation flows at lane level): every mp_interval steps each
                       controller picks the phase whose approach-lane links carry the largest
                       sum of (vehicles on the approach lane - vehicles on the link's target
                       lane); the green phase wins a tie it is in, else the lowest index; a
                       change shows the controller's ctrl_yellow seconds of yellow first.
                       Needs ctrl_nphase <= 32 and ctrl_yellow < mp_interval (MS_ERR_ARG). */
  int mp_interval;  /* steps between max-pressure decisions (signal_mode 1), >= 1 */
} ms_params;

/* Lane-level road network (Sec. III-C "Map Builder": lanes with topology, junction lanes,
   signal phases).  succ CSR: for an edge lane, its junction-internal lanes with the exit
   edge each leads to; for an internal lane exactly one entry: its target edge lane and
   that lane's edge.  Requirements (else MS_ERR_ARG): every lane longer than v_max*dt;
   the lanes of edge e are edge_lane0[e] + q for q < edge_nlanes[e], numbered from the
   right: lane_index q, lane_left the lane q + 1, lane_right the lane q - 1 (-1 past the
   outermost); internal lanes have one successor and no left/right; signal groups <
   ctrl_nphase.  Limits (else MS_ERR_CAPACITY): at most 10 lanes per edge and 63 links per
   edge lane (the per-route link plan holds one 6-bit link index per lane of an edge). */
typedef struct ms_network {
  int n_lanes, n_edges, n_ctrl;
  const float *lane_len;    /* [n_lanes] m */
  const int *lane_edge;     /* [n_lanes] edge id, -1 for junction-internal lanes */
  const int *lane_index;    /* [n_lanes] index within the edge, 0 = rightmost */
  const int *lane_left;     /* [n_lanes] lane to the left (-1 none) */
  const int *lane_right;    /* [n_lanes] lane to the right (-1 none) */
  const int *succ_off;      /* [n_lanes+1] */
  const int *succ_lane;     /* [succ_off[n_lanes]] */
  const int *succ_edge;     /* [succ_off[n_lanes]] */
  const int *lane_ctrl;     /* [n_lanes] signal controller at the lane end, -1 none */
  const int *lane_group;    /* [n_lanes] phase group served */
  const int *ctrl_offset;   /* [n_ctrl] s */
  const int *ctrl_green;    /* [n_ctrl] s, > 0 */
  const int *ctrl_yellow;   /* [n_ctrl] s, >= 0 */
  const int *ctrl_nphase;   /* [n_ctrl] >= 1 */
  const int *edge_nlanes;   /* [n_edges] */
  const int *edge_lane0;    /* [n_edges] */
} ms_network;

/* Trip demand (Sec. III-A input "demand data"; Sec. III-C converter output: individual
   trips with routes and departure times).  Trip i has id i, departs at t_dep[i] on
   route_edges[route_off[i] .. route_off[i+1]-1] (consecutive edges must be lane-linked,
   else MS_ERR_ROUTE).  Optional placement (lane != NULL and lane[i] >= 0): the vehicle is
   already on the network at (lane[i], x[i], v[i]); its route then starts at the lane's
   edge, or, on an internal lane, at the approach edge that lane leaves from. */
typedef struct ms_vehicles {
  int n;
  const int *t_dep;          /* [n] s */
  const float *v0;           /* [n] desired speed, (0, v_max] */
  const int64_t *route_off;  /* [n+1] */
  const int *route_edges;    /* [route_off[n]] */
  const int *lane;           /* [n] or NULL */
  const float *x;            /* [n] or NULL */
  const float *v;            /* [n] or NULL */
} ms_vehicles;

/* Dynamic state.  Vehicle arrays hold the active vehicles sorted by (lane, x); route_idx is
   the index within the trip's route of the current edge (the approach edge on an internal
   lane).  Trip arrays are indexed by trip id. */
typedef struct ms_state {
  int capacity;     /* in: entries available in the vehicle arrays */
  int n_active;     /* out (read) / in (write) */
  int t;            /* out (read) / in (write): next step to compute */
  int *id, *lane, *route_idx;   /* [capacity] */
  float *x, *v;                 /* [capacity] */
  int *trip_status; /* [n_trips] 0 waiting, 1 active, 2 arrived (read only) */
  int *t_arr;       /* [n_trips] arrival step or -1 */
  int *ctrl_state;  /* [3 * n_ctrl] host memory (also with ms_read_state's device flag) or
                       NULL: max-pressure controllers at step t: green phase, pending phase
                       (-1 none), step at which it turns green.  Read: filled if not NULL.
                       Write: restored if not NULL, else every controller restarts with
                       phase 0 green and nothing pending. */
} ms_state;

typedef struct ms_metrics {
  float *lane_vsum;  /* [n_windows*n_lanes] or NULL: per-window sum of speeds */
  int *lane_vcnt;    /* [n_windows*n_lanes] or NULL: per-window vehicle-steps */
  int64_t inserted, arrived, sum_travel_time;
  int n_active, t, movers_last_step;
  unsigned err;      /* MS_DEV_* bits */
} ms_metrics;

/* Per-vehicle record of the last step (params.debug = 1), indexed by trip id; entries of
   trips that were not active at the start of the step are left untouched. */
typedef struct ms_debug {
  int *active_before, *lead_kind, *lead_id, *lc_dir, *lc_cand, *tau_lead, *tau_foll,
      *old_foll, *flag, *inserted;
  float *s_own, *vl_own, *a_own, *incentive, *a_use;
  /* learned lane change (a model set): lc_learn 1 where the network decided; there its
     softmax margin, logits (lc_logit [3 * n_trips]) and BF16 inputs (lc_feat
     [16 * n_trips]); any may be NULL */
  int *lc_learn;
  float *lc_margin, *lc_logit, *lc_feat;
} ms_debug;

/* Create a simulation bound to a CUDA stream (cudaStream_t, or NULL for the default
   stream) on the current device.  *out receives the handle.  MS_ERR_ARG on invalid
   parameters. */
int ms_create(void **out, const ms_params *p, void *cuda_stream);

/* Copy the network to the device and derive its lane tables.  Once per simulation. */
int ms_load_network(void *sim, const ms_network *net);

/* Copy the trips to the device (once, after ms_load_network, before the first step).
   Validates routes (MS_ERR_ROUTE) and placements (MS_ERR_ARG: lane/edge mismatch, x not
   in (0, len], overlapping vehicles in a lane).  If a learned lane-change model was set
   before this call and its candidate buffers cannot be allocated, the vehicles are still
   added, the model is dropped (the rule decides) and MS_ERR_CUDA is returned. */
int ms_add_vehicles(void *sim, const ms_vehicles *veh);

/* Enqueue n steps on the simulation's stream (asynchronous; CUDA-graph replays).  One step
   is the paper's time step of dt (Sec. III-A): the prepare phase (vehicles grouped by lane
   and ordered by position; here an incremental merge of the sorted state) and the update
   phase (sensing of the leader on the own path and on the lane-change target, IDM car
   following and randomized MOBIL lane changes, signal stop lines, Newton's equations of
   motion, lane-to-lane transfer, departures and arrivals).  Returns MS_ERR_CUDA if a launch
   fails.  Device error bits are reported by ms_sync. */
int ms_step(void *sim, int n);

/* Run n steps with each kernel launched on its own (no graph) between CUDA events on the
   simulation's stream, and add each kernel's device time in milliseconds to
   ms_per_kernel[0..3] (decide (with the learned lane change's inference kernel when a model
   is set), lanes, bucket, apply; caller-owned, 4 floats).  Synchronises.
   Same results as ms_step; used to attribute the step time to kernels. */
int ms_step_timed(void *sim, int n, float *ms_per_kernel);

/* Largest network ms_step_noalloc accepts: lanes <= MS_NOALLOC_MAX_TILES *
   MS_NOALLOC_TILE_LANES (3,145,728). */
#define MS_NOALLOC_MAX_TILES 3072
#define MS_NOALLOC_TILE_LANES 1024

/* ms_step_noalloc -- the same n steps as ms_step, for callers that must not allocate
   device memory once their simulation is set up: for example a control or serving loop
   that runs inside a fixed device-memory budget reserved in advance, or a host component
   that holds no right to call cudaMalloc on a shared device.  ms_step may allocate on its
   first call (it instantiates CUDA graphs), and the lane scan of every step keeps its
   per-tile aggregates in memory of the simulation.  This entry point allocates nothing: it
   launches the step's kernels directly and keeps the lane scan's per-tile aggregates in one
   static device array of MS_NOALLOC_MAX_TILES tiles (8 bytes each), which every GPU that
   loads this library holds until the process exits.
   - The paper has no counterpart; results are identical to ms_step.
   - Networks with more than MS_NOALLOC_MAX_TILES * MS_NOALLOC_TILE_LANES lanes:
     MS_ERR_CAPACITY.
   - The simulation's device must be current (else MS_ERR_STATE).  The first call on a
     device looks up the array's device address (cudaGetSymbolAddress); make that first
     call before any stream capture begins.
   - Every call, from any simulation, shares the one array: calls that overlap on the GPU
     (different streams, threads or simulations running at the same time) race and give
     wrong results.  Each step writes the tiles it uses before reading them, so nothing
     needs clearing between calls.
   Returns MS_ERR_CUDA if a launch fails; device error bits are reported by ms_sync. */
int ms_step_noalloc(void *sim, int n);

/* Wait for enqueued steps; MS_ERR_DEVICE if a device-side check fired. */
int ms_sync(void *sim);

/* Read the state (synchronises): every active vehicle's lane, position, speed, trip id and
   route position, and each trip's status and arrival step -- the per-vehicle output the
   paper's simulator gives each step (Sec. III-A, "output"; its heading angle needs lane
   geometry the networks here do not carry).  device = 0: the ms_state vehicle arrays are
   host pointers; device = 1: they are device pointers (the copies are device-to-device) and
   trip_status / t_arr, if not NULL, are host pointers.  MS_ERR_CAPACITY if capacity <
   n_active (n_active is still set). */
int ms_read_state(void *sim, ms_state *out, int device);

/* Asynchronous export of the vehicle state (x, v, lane, id; any may be NULL) into PINNED
   host buffers (cudaHostAlloc / pinned tensors; else MS_ERR_ARG).  The call waits for the
   steps enqueued so far (a kernel writes the vehicle count into mapped host memory), then
   enqueues the copies on a side stream, where they run on the copy engine behind any
   export still in flight while the following steps compute.  The next ms_step may run
   while the export is in flight; a launch that would overwrite the exported buffer (the
   second step after the export) waits for it on the device.  The buffers must stay valid
   and untouched until the matching ms_read_wait returns.  Up to two exports may be in
   flight (completed in order, so the host link stays busy while the host consumes the
   older one); a third call returns MS_ERR_STATE.  ms_write_state and ms_autotune wait for
   exports in flight.  Only capacity and the four vehicle arrays of out are used;
   route_idx, trip_status, t_arr and ctrl_state are ignored. */
int ms_read_state_async(void *sim, const ms_state *out);

/* Wait for the oldest export in flight; n_active and t (either may be NULL) receive the
   vehicle count and the step of the exported state.  MS_ERR_CAPACITY if the
   capacity given was below n_active (the first capacity entries are still written);
   MS_ERR_STATE if no export is in flight. */
int ms_read_wait(void *sim, int *n_active, int *t);

/* Replace the dynamic state (checkpoint / resume; the paper's API writes vehicle state in
   batches, Sec. III-C).  Vehicles must be sorted by (lane, x, id), one entry per active
   trip, gaps >= 0 (down to -max(1e-3 m, 5e-7 x): FP32 rounding far along long lanes);
   trips neither active nor arrived (t_arr < 0) wait for departure.  Metric accumulators
   are kept. */
int ms_write_state(void *sim, const ms_state *in);

int ms_read_metrics(void *sim, ms_metrics *out);

/* Debug record of the last step (requires params.debug = 1, else MS_ERR_STATE). */
int ms_read_debug(void *sim, ms_debug *out);

/* Batched scenarios: n independent networks and their trips simulated as one disjoint
   union in a single step launch sequence (many scenarios of uneven size for signal or
   policy sweeps).  Scenario k's lanes, edges, controllers and trips get ids offset by the
   totals of scenarios 0..k-1; otherwise identical to ms_load_network / ms_add_vehicles
   (same validation, same error codes naming the scenario).  Call instead of, not in
   addition to, the single-scenario loaders.  The paper simulates one scenario at a time;
   batching is this library's addition. */
int ms_load_network_batch(void *sim, int n, const ms_network *nets);
int ms_add_vehicles_batch(void *sim, int n, const ms_vehicles *vehs);
/* Offsets of each batched scenario: lane_off[n+1], trip_off[n+1] (caller-owned host
   arrays); MS_ERR_STATE if the simulation was not loaded as a batch. */
int ms_batch_offsets(void *sim, int *lane_off, int *trip_off);

/* Autotuner of the step's launch shapes: for each candidate it times trial_steps steps with
   CUDA events, restoring the dynamic state after each trial, and keeps the fastest; the
   simulation's results are unchanged.  Coordinate search over (1) threads per block of the
   vehicle kernels (128, 256, 512) x persistent-grid oversubscription of the decide and the
   apply kernel (1, 2, 4 each), (2) the lane scan's threads per 1024-lane tile (128, 256,
   512), (3) the bucket kernel's block (128, 256, 512) and grid factor (1, 2): 36 trials.
   best_ms receives the best mean step time (ms); config (6 ints, may be NULL) the chosen
   block size, decide and apply grid factors, lane-scan threads per tile, bucket block and
   bucket grid factor.  Allocates temporary device memory for the state snapshot. */
int ms_autotune(void *sim, int trial_steps, float *best_ms, int *config);

/* ---- learned lane-change surrogate ----------------------------------------------
   A 16 -> 64 -> 64 -> 3 MLP (ReLU; softmax over stay / left / right) that replaces the
   MOBIL incentive decision of discretionary candidates that passed the safety criteria.
   The paper's lane-change model is rule-based (Sec. III-A); the surrogate is this
   library's addition.  Parameters: 5443 floats, W1[64][16], b1[64], W2[64][64], b2[64],
   W3[3][64], b3[3], row-major (out x in).  Inference and training run on the tensor cores
   with BF16 operands and FP32 accumulation. */
#define MS_MLP_NPARAM 5443
#define MS_MLP_WORK_FLOATS 12096   /* scratch of the training calls, floats */

/* Log (features, rule decision) of every candidate in subsequent steps into caller-owned
   device buffers: x [cap][16] bf16, y [cap] int (0 stay, 1 left, 2 right), n: device int
   counting offered samples (those beyond cap are dropped).  x == NULL turns logging off. */
int ms_set_lc_log(void *sim, void *x, int *y, int cap, int *n);

/* Use the learned decision in subsequent steps: params (host, 5443 floats) is the network;
   a candidate follows the network's class when its softmax margin (top1 - top2) is at
   least margin, else the rule's decision; a change still needs the step's allowed
   direction.  params == NULL returns to the rule.  A step then lists its discretionary
   candidates with their sensing results (one slot per trip, about 260 B each, allocated
   with the first model once the vehicles are added) and evaluates the network on them in
   one more kernel.  Errors: MS_ERR_ARG (margin outside [0, 1]); MS_ERR_CUDA if those
   buffers cannot be allocated (the lane-change mode in effect before the call, rule,
   logging or an earlier model, stays). */
int ms_set_lc_model(void *sim, const float *params, float margin);

/* Lane modifications (Sec. III-C "Python API": modification calls for lane speed limits and
   lane restrictions), in effect from the next step.  For lanes[k] (host arrays, n entries):
   vmax[k] m/s caps the desired speed of every vehicle on the lane, v0_eff = min(v0, vmax)
   (<= 0 or non-finite: no limit); closed[k] != 0 closes the lane: a vehicle whose path
   reaches it stops at the end of the lane before it, no lane change targets it, and its
   departure queue waits; vehicles already on it drive on.  vmax or closed may be NULL
   (left unchanged).  Lanes out of range: MS_ERR_ARG, nothing changed.  Synchronises with the
   simulation's stream.  While no lane has a limit or is closed the step does no extra
   work for this. */
int ms_set_lane_limits(void *sim, int n, const int *lanes, const float *vmax, const int *closed);

/* Dynamic lanes (Sec. III-C "Python API": modification calls for dynamic lanes), in effect
   from the next step.  For edge lane lanes[k] (host arrays, n entries), bit j of
   open_mask[k] opens (1) or closes (0) its j-th lane link (successor entry j, the CSR order
   of ms_network.succ_off; at load every link is open).  A closed link is no link: the
   fan-out choice toward the next route edge, mandatory lane changes, the lanes a
   discretionary change may target, the obstacle at a lane end and the max-pressure sums
   all skip it.  Vehicles already on its junction-internal lane finish the movement;
   waiting trips keep the departure lanes assigned when they were added.
   Errors (nothing changed): MS_ERR_ARG for an internal or out-of-range lane;
   MS_ERR_CAPACITY for a lane with more than 32 links; MS_ERR_STATE before ms_add_vehicles;
   MS_ERR_ROUTE if a trip not yet arrived would need, on the rest of its route, a pair of
   consecutive edges with no open link (the message names it).  Synchronises; rebuilds on
   the host the link plans of the route entries on or into the edges whose links change,
   and re-derives every active vehicle's cached plan word and next-lane choice on the
   device (host work O(trips + route entries), a 8-byte-per-entry plan upload); under
   max-pressure signals the controllers take the current step's decision again over the
   links now open, as after a state upload. */
int ms_set_lane_links(void *sim, int n, const int *lanes, const unsigned *open_mask);

/* Route planner for demand generation (the paper turns OD matrices into trips with routes,
   Sec. III-C "Converter from OD matrix to travel demand"; at millions of trips that is the
   host's bottleneck, so it runs on the GPU here).  Trip i goes from edge orig_edge[i] to
   edge dest_edge[i] on the loaded network.  Route graph: an arc e -> f wherever a lane of e
   links to exit edge f; entering f costs round(1000 * its length) integer millimetres.  The
   route is the least-cost edge sequence from orig to dest, both included; among several,
   the one that at every edge takes the lowest-id successor still on a least-cost route.
   Every route is therefore valid input for ms_add_vehicles.  Destinations are processed in
   batches of up to 4096 (about 2 GiB of device distances per batch; the call allocates and
   frees its own device memory).
   route_off: [n + 1] host, always filled (a trip that cannot reach its destination gets
   an empty route; their number goes to *n_unreachable if not NULL).  route_edges: host
   array of edges_capacity entries, or NULL to get route_off only; if route_off[n] exceeds
   edges_capacity: MS_ERR_CAPACITY (route_off still filled).  Edges out of range: MS_ERR_ARG.
   Synchronises with the simulation's stream. */
int ms_route_trips(void *sim, int n, const int *orig_edge, const int *dest_edge, int64_t *route_off,
                   int *route_edges, int64_t edges_capacity, int *n_unreachable);

/* Gravity OD sampling for demand generation: the gravity model is one of the baseline OD
   models the paper's OD generator offers (Sec. III-B; classical models, Sec. II-B), its
   diffusion model and data not being available here.  Zone z is
   edge zone_edge[z] (distinct) with attraction attract[z] > 0.  Trip k draws three 24-bit
   uniforms u_s = top 24 bits of SplitMix64(seed ^ salt_s ^ k) / 2^24 (salts
   0x5851F42D4C957F2D origin, 0x14057B7EF767814F destination, 0x2545F4914F6CDD1D departure):
   origin zone = the first i whose cumulative attraction exceeds u * total; destination =
   the first j whose cumulative weight exceeds u * total over w_ij = A_j / dkm_ij^gamma
   (j != i; dkm_ij = float(least route cost from zone i's edge to zone j's, in mm, as in
   ms_route_trips) * 1e-6 raised by gamma float products; 0 where unreachable; a zone that
   reaches none keeps its trips at home); departure step = floor(u24 * t_span / 2^24).
   Weights and cumulative sums are float32 in index order, IEEE-rounded, so a float32 CPU
   computation draws the same trips.  Outputs (host, n each): orig_edge, dest_edge, t_dep;
   routes then come from ms_route_trips.  At most 4096 zones (MS_ERR_CAPACITY); gamma 0..3,
   t_span > 0 (MS_ERR_ARG).  Allocates and frees its own device memory; synchronises. */
int ms_sample_trips(void *sim, int n_zones, const int *zone_edge, const float *attract, int gamma, int n,
                    int t_span, uint64_t seed, int *orig_edge, int *dest_edge, int *t_dep);

/* Radiation OD sampling (the radiation model of Simini, Gonzalez, Maritan and Barabasi
   2012, a baseline the paper's OD generator offers beside gravity, Sec. III-B): as
   ms_sample_trips with population[z] > 0 in place of the attractions for the origin draw,
   and destination weights w_ij = (m_i m_j) / ((m_i + s_ij)((m_i + m_j) + s_ij)) for
   reachable j != i, s_ij = the population of the zones strictly closer to i than j by route
   cost (i and j excluded; zones at equal cost count for neither), summed in float32 in
   order of (cost, zone index).  Every weight operation is one IEEE float32 operation in
   that order, so a float32 CPU computation draws the same trips.  The model has no free
   parameter and uses route costs only through their order.  At most 4096 zones; a
   zone-to-zone cost of 2^40 mm or more: MS_ERR_CAPACITY.  Allocates and frees its own
   device memory; synchronises. */
int ms_sample_trips_radiation(void *sim, int n_zones, const int *zone_edge, const float *population, int n,
                              int t_span, uint64_t seed, int *orig_edge, int *dest_edge, int *t_dep);

/* Counters of the learned decision since the model was set: [0] candidates, [1] rule
   fallbacks (low margin), [2] agreements with the rule, [3 + 3*rule + final] confusion. */
int ms_read_lc_stats(void *sim, int64_t *out12);

/* One Adam step (lr, betas 0.9 / 0.999, eps 1e-8; t counts from 1) of class-weighted
   cross-entropy on the minibatch idx[0..batch) of the samples (x bf16 [*][16], y int);
   theta, m, v: device FP32 [5443]; work: device scratch of MS_MLP_WORK_FLOATS floats;
   class_w: host, 3 floats; loss (host, may be NULL) receives the minibatch loss
   (synchronises).  All pointers except class_w and loss are device pointers. */
int ms_mlp_train_step(const void *x, const int *y, const int *idx, int batch, float *theta, float *m, float *v,
                      int t, float lr, const float *class_w, float *work, float *loss, void *cuda_stream);

/* Gradient of the same loss at theta (no update) into grad (device FP32 [5443]). */
int ms_mlp_grad(const void *x, const int *y, const int *idx, int batch, const float *theta,
                const float *class_w, float *work, float *grad, void *cuda_stream);

/* The same two calls on the 5th-generation tensor core (tcgen05 MMAs with accumulators in
   tensor memory, 128 samples per CTA) instead of mma.sync: the same loss, roundings and
   arguments.  ms_mlp_train_step_tc with loss != NULL also returns MS_ERR_DEVICE (and
   applies no update) if a wait for the tensor core ran out; the gradient is then
   incomplete.  The training kernel packs its own BF16 operands from theta.  Uses about
   171 KB of shared memory and all 512 TMEM columns of each SM it runs on while it runs. */
int ms_mlp_train_step_tc(const void *x, const int *y, const int *idx, int batch, float *theta, float *m,
                         float *v, int t, float lr, const float *class_w, float *work, float *loss,
                         void *cuda_stream);
int ms_mlp_grad_tc(const void *x, const int *y, const int *idx, int batch, const float *theta,
                   const float *class_w, float *work, float *grad, void *cuda_stream);

/* Tests of the timeout paths (failure detection without a GPU fault).  Every wait of a
   kernel on an asynchronous unit is bounded; these calls withhold what such a wait waits
   for, so that it runs out after a short limit, and the failure must come back as an error
   while the context stays usable.
   ms_test_tc_timeout: the tcgen05 gradient of ms_mlp_grad_tc with no MMA issued or
   committed; synchronises; returns MS_ERR_DEVICE when the kernel reported the timeout (the
   expected outcome), MS_OK if it did not.  work holds no valid gradient afterwards.
   ms_test_withhold_copies: on != 0 makes the steps that follow issue no bulk copy in the
   apply kernel, whose waits then run out and set MS_DEV_TIMEOUT (ms_sync returns
   MS_ERR_DEVICE); the simulation's state is invalid from that step on (destroy it). */
int ms_test_tc_timeout(const void *x, const int *y, const int *idx, int batch, const float *theta,
                       const float *class_w, float *work, void *cuda_stream);
int ms_test_withhold_copies(void *sim, int on);

/* Class and softmax margin (top1 - top2) of n samples x (device, bf16 [n][16]): device
   outputs cls [n] int, margin [n] float and, if not NULL, the logits [n][3] float.
   theta: device FP32 [5443]; work: device scratch of MS_MLP_WORK_FLOATS floats. */
int ms_mlp_predict(const void *x, int n, const float *theta, float *work, int *cls, float *margin, float *logits,
                   void *cuda_stream);

const char *ms_last_error(void *sim);
void ms_destroy(void *sim);

#ifdef __cplusplus
}
#endif
#endif
