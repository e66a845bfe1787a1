// moss103.cu -- host side of the C ABI declared in include/moss103.h.
//
// Owns the device memory of one simulation, validates and converts the network and the
// trips into the device layout (sorted structure-of-arrays vehicle state, 32-byte lane
// records, CSR successor / feeder tables, per-route link plans, per-lane departure FIFOs),
// and replays the step's kernels of step_kernels.cuh (decide, two lane-scan passes, bucket,
// apply; max-pressure signals when enabled) as captured CUDA graphs with programmatic
// dependent launch.  Also the route planner and OD sampler of route_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "moss103.h"
#include "route_kernels.cuh"
#include "step_kernels.cuh"

using namespace moss;

namespace {

constexpr int GRAPH_STEPS = 16;

// launch shape of the vehicle kernels (chosen by ms_autotune; defaults from occupancy)
struct LaunchCfg {
  int blk_decide = 256, grid_decide = 1;
  int blk_apply = 256, grid_apply = 1;
  int blk_bucket = 256, grid_bucket = 1;
  int grid_learn = 1;   // k_learn (LEARN_THREADS per block), learned lane change only
  int f_decide = 1, f_apply = 1, f_bucket = 1;   // grid = factor x resident blocks x SMs
  int lane_threads = LANE_THREADS;   // lane scan: threads per tile of LANE_TILE lanes
};

// the lane scan's passes for a tile shape (threads per tile: 128, 256 or 512)
typedef void (*LanesKernel)(StepArgs);
LanesKernel lanes_kernel(int pass, int th) {
  if (th == 128) return pass ? k_lanes_t<1, 128> : k_lanes_t<0, 128>;
  if (th == 512) return pass ? k_lanes_t<1, 512> : k_lanes_t<0, 512>;
  return pass ? k_lanes_t<1, 256> : k_lanes_t<0, 256>;
}

struct Sim {
  ms_params prm{};
  DevParams P{};
  cudaStream_t stream = nullptr;   // caller's stream
  cudaStream_t cap = nullptr;      // private capture stream
  // asynchronous state exports (ms_read_state_async): side stream, up to MS_EXPORTS in
  // flight, completed in order (slot (ex_head + i) % MS_EXPORTS is the i-th oldest)
  static constexpr int MS_EXPORTS = 2;
  cudaStream_t xs = nullptr;
  cudaEvent_t ev_ready = nullptr, ev_export[MS_EXPORTS] = {};
  int *h_meta = nullptr;           // [MS_EXPORTS][2] {n_active, t} written by k_export
  long long export_t[MS_EXPORTS] = {};   // step whose state each slot exports
  int export_cap[MS_EXPORTS] = {};
  int ex_head = 0, ex_count = 0;
  long long t_host = 0;            // step the next launch computes (host count)
  int device = 0, n_sm = 0;
  std::string err;
  bool net_loaded = false, veh_loaded = false;
  // network (host copies needed by validation and state I/O)
  int n_lanes = 0, n_edges = 0, n_ctrl = 0;
  std::vector<float> lane_len;
  std::vector<unsigned char> link_off;   // per successor entry: 1 = closed (dynamic lanes)
  std::vector<int> lane_edge, lane_left, lane_right, succ_off, succ_lane, succ_edge, edge_nlanes,
      edge_lane0;
  // trips
  int n_trips = 0;
  std::vector<int> h_route0, h_routes, h_tdep, h_qoff, h_qtrip;
  std::vector<unsigned long long> h_plan;   // link plan per routes[] entry
  std::vector<float> h_v0;
  // device
  LaneInfo *d_li = nullptr;
  int2 *d_succ = nullptr;
  unsigned char *d_link_off = nullptr;        // per successor entry: 1 = closed (dynamic lanes)
  int *d_pred = nullptr;
  int4 *d_ctrl4 = nullptr;
  std::vector<int4> h_ctrl4;
  int *d_sig[2]{};   // signal table per step parity (see sig_pack)
  int4 *d_mp = nullptr;                             // max-pressure controller state
  int *d_ctrl_loff = nullptr, *d_ctrl_lanes = nullptr;   // approach lanes per controller
  float *d_lane_vmax = nullptr;           // lane speed limits (+inf: none)
  unsigned char *d_lane_closed = nullptr;
  std::vector<float> h_lane_vmax;
  std::vector<unsigned char> h_lane_closed;
  // route graph of the route planner (built on first use)
  int *d_rg_off = nullptr, *d_rg_dst = nullptr;
  long long *d_rg_cost = nullptr;
  int *d_routes = nullptr;
  unsigned long long *d_plan = nullptr;
  Soa A[2]{};
  int4 *d_dyn[2]{};
  DevCtrl *d_ctrl = nullptr;
  unsigned *d_leave = nullptr;
  int *d_arr_cnt = nullptr, *d_amin = nullptr, *d_arr_start = nullptr;
  int4 *d_bucket = nullptr;
  float *d_res_x = nullptr, *d_res_v = nullptr;
  int *d_res_code = nullptr, *d_res_nl = nullptr, *d_arr_fill = nullptr;
  int *d_cand = nullptr;   // learned lane change: the step's listed candidates and their
  Upd *d_rec_u = nullptr;  // sensing results (one slot per trip; allocated once a model and
  VCtx *d_rec_c = nullptr; // the vehicles are both set)
  int2 *d_res_pos = nullptr;
  unsigned long long *d_tile_agg = nullptr;
  int *d_qoff = nullptr, *d_qtrip = nullptr;
  int2 *d_qhd = nullptr;
  int4 *d_qent = nullptr, *d_qent2 = nullptr;
  int *d_tdep = nullptr, *d_route0 = nullptr, *d_tarr = nullptr;
  unsigned long long *d_vsum = nullptr;   // per window x lane: sum of speeds, 2^-24 m/s units
  int *d_vcnt = nullptr;
  DebugOut dbg{};
  int n_tiles = 0;
  LaunchCfg cfg{};
  // batches of independent scenarios: offsets of each scenario's lanes and trips
  std::vector<int> batch_lane_off, batch_trip_off;
  cudaGraphExec_t g_many = nullptr, g_one = nullptr;
  // learned lane change
  int lc_mode = MODE_PLAIN;
  LcAux lc{};
  MlpDev *d_model = nullptr;
  unsigned long long *d_lcstats = nullptr;
  float *d_theta = nullptr;
  std::vector<void *> allocs;
};

int fail(Sim *s, int code, const std::string &msg) {
  if (s) s->err = msg;
  return code;
}

#define CK(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(s, MS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
int dalloc(Sim *s, T **p, size_t n) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) return fail(s, MS_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  s->allocs.push_back(q);
  *p = static_cast<T *>(q);
  return MS_OK;
}

#define DALLOC(ptr, n)                       \
  do {                                       \
    int r_ = dalloc(s, &(ptr), (size_t)(n)); \
    if (r_) return r_;                       \
  } while (0)

StepArgs make_args(Sim *s) {
  StepArgs a{};
  a.li = s->d_li;
  a.succ = s->d_succ;
  a.link_off = s->d_link_off;
  a.pred = s->d_pred;
  a.ctrl4 = s->d_ctrl4;
  a.sig[0] = s->d_sig[0];
  a.sig[1] = s->d_sig[1];
  a.n_ctrl = s->n_ctrl;
  a.mp = s->d_mp;
  a.ctrl_loff = s->d_ctrl_loff;
  a.ctrl_lanes = s->d_ctrl_lanes;
  a.lane_vmax = s->d_lane_vmax;
  a.lane_closed = s->d_lane_closed;
  a.routes = s->d_routes;
  a.plan = s->d_plan;
  a.A[0] = s->A[0];
  a.A[1] = s->A[1];
  a.dyn[0] = s->d_dyn[0];
  a.dyn[1] = s->d_dyn[1];
  a.ctrl = s->d_ctrl;
  a.leave = s->d_leave;
  a.arr_cnt = s->d_arr_cnt;
  a.amin = s->d_amin;
  a.arr_start = s->d_arr_start;
  a.bucket = s->d_bucket;
  a.res_x = s->d_res_x;
  a.res_v = s->d_res_v;
  a.res_code = s->d_res_code;
  a.res_code_nl = s->d_res_nl;
  a.res_pos = s->d_res_pos;
  a.arr_fill = s->d_arr_fill;
  a.tile_agg = s->d_tile_agg;
  a.q_off = s->d_qoff;
  a.q_trip = s->d_qtrip;
  a.q_hd = s->d_qhd;
  a.q_ent = s->d_qent;
  a.q_ent2 = s->d_qent2;
  a.trip_tdep = s->d_tdep;
  a.t_arr = s->d_tarr;
  a.vsum = s->d_vsum;
  a.vcnt = s->d_vcnt;
  a.dbg = s->dbg;
  a.lc = s->lc;
  a.P = s->P;
  return a;
}

// the k_decide instance for the simulation's lane-change mode and debug setting
typedef void (*DecideKernel)(StepArgs);
template <bool MODS>
DecideKernel decide_kernel_m(int mode, bool dbg) {
  if (mode == MODE_LEARN) return dbg ? k_decide_t<MODE_LEARN, true, MODS> : k_decide_t<MODE_LEARN, false, MODS>;
  if (mode == MODE_LOG) return dbg ? k_decide_t<MODE_LOG, true, MODS> : k_decide_t<MODE_LOG, false, MODS>;
  return dbg ? k_decide_t<MODE_PLAIN, true, MODS> : k_decide_t<MODE_PLAIN, false, MODS>;
}
DecideKernel decide_kernel(int mode, bool dbg, bool mods) {
  return mods ? decide_kernel_m<true>(mode, dbg) : decide_kernel_m<false>(mode, dbg);
}
DecideKernel learn_kernel(bool dbg) { return dbg ? k_learn<true> : k_learn<false>; }

// a step kernel launch with programmatic stream serialization: it may start while the
// previous kernel in the stream drains (the kernel waits in pdl_enter before reading)
template <typename... Args>
cudaError_t launch_pdl(void (*k)(Args...), int grid, int block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// one step = five launches (six with the learned lane change; + max-pressure controllers,
// + the debug order check); ev (5 events) brackets the step's parts: decide (with k_learn),
// the two lane-scan passes together, bucket, apply
cudaError_t launch_step(const Sim *s, const StepArgs &a, cudaStream_t st, cudaEvent_t *ev) {
  const LaunchCfg &c = s->cfg;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  if (ev) cudaEventRecord(ev[0], st);
  ok(launch_pdl(decide_kernel(s->lc_mode, s->prm.debug != 0, a.P.lane_mods != 0), c.grid_decide, c.blk_decide, 0,
                st, a));
  if (s->lc_mode == MODE_LEARN) {
    // an ordinary launch: launched early (programmatic), its waiting blocks took the SMs
    // the decide kernel's last blocks were freeing and the pair took 18 us longer
    learn_kernel(s->prm.debug != 0)<<<c.grid_learn, LEARN_THREADS, learn_smem(LEARN_THREADS), st>>>(a);
    ok(cudaGetLastError());
  }
  if (ev) cudaEventRecord(ev[1], st);
  ok(launch_pdl(lanes_kernel(0, c.lane_threads), s->n_tiles, c.lane_threads, 0, st, a));   // tile aggregates
  ok(launch_pdl(lanes_kernel(1, c.lane_threads), s->n_tiles, c.lane_threads, 0, st, a));   // counts, starts, ...
  if (ev) cudaEventRecord(ev[2], st);
  ok(launch_pdl(k_bucket, c.grid_bucket, c.blk_bucket, 0, st, a));
  if (ev) cudaEventRecord(ev[3], st);
  ok(launch_pdl(k_apply, c.grid_apply, c.blk_apply, app_smem(c.blk_apply), st, a));
  if (s->P.signal_mode == 1 && s->n_ctrl > 0)   // controllers of the next step
    ok(launch_pdl(k_signals, (s->n_ctrl + 7) / 8, 256, 0, st, a));
  if (ev) cudaEventRecord(ev[4], st);
  if (s->prm.debug) ok(launch_pdl(k_check, c.grid_bucket, c.blk_bucket, 0, st, a));
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t enqueue_step(Sim *s, cudaStream_t st) { return launch_step(s, make_args(s), st, nullptr); }

// persistent grids: blocks = factor * (resident blocks per SM) * SMs, capped by the work;
// the decide kernel's residency is that of the instance the current lane-change mode runs
// (the learned and logging instances hold more registers and shared memory)
int shape_grids(Sim *s, LaunchCfg &c, int f_decide, int f_apply, int f_bucket) {
  const int N = s->n_trips;
  int od = 0, oa = 0, ob = 0;
  c.f_decide = f_decide;
  c.f_apply = f_apply;
  c.f_bucket = f_bucket;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&od, decide_kernel(s->lc_mode, s->prm.debug != 0, false),
                                                   c.blk_decide, 0));
  // k_learn: one block per SM, each warp looping over 16-candidate chunks (1,184 warps;
  // about 16k candidates a step on the 1M-vehicle grid use 1,030 of them)
  c.grid_learn = s->n_sm;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oa, k_apply, c.blk_apply, app_smem(c.blk_apply)));
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, k_bucket, c.blk_bucket, 0));
  auto g = [&](int blk, int occ, int f) {
    return std::max(1, std::min((N + blk - 1) / blk, f * std::max(1, occ) * s->n_sm));
  };
  c.grid_decide = g(c.blk_decide, od, f_decide);
  c.grid_apply = g(c.blk_apply, oa, f_apply);
  c.grid_bucket = g(c.blk_bucket, ob, f_bucket);
  return MS_OK;
}

// learned lane change: the candidate list and records, one slot per trip (a vehicle is
// listed at most once a step), allocated once a model and the vehicles are both set
int alloc_cand(Sim *s) {
  const int N = s->n_trips;
  DALLOC(s->d_cand, N);
  DALLOC(s->d_rec_u, N);
  DALLOC(s->d_rec_c, N);
  return MS_OK;
}
int ensure_cand(Sim *s) {
  if ((s->d_cand && s->d_rec_u && s->d_rec_c) || !s->veh_loaded || s->lc_mode != MODE_LEARN) return MS_OK;
  if (int r = alloc_cand(s)) {   // no room: the rule keeps deciding
    s->lc_mode = MODE_PLAIN;
    s->lc.model = nullptr;
    return r;
  }
  s->lc.cand = s->d_cand;
  s->lc.rec_u = s->d_rec_u;
  s->lc.rec_c = s->d_rec_c;
  s->lc.cand_cap = s->n_trips;
  return MS_OK;
}

void drop_graphs(Sim *s) {
  if (s->g_many) cudaGraphExecDestroy(s->g_many);
  if (s->g_one) cudaGraphExecDestroy(s->g_one);
  s->g_many = s->g_one = nullptr;
}

int build_graphs(Sim *s) {
  if (s->g_many) return MS_OK;
  for (int which = 0; which < 2; ++which) {
    int steps = which == 0 ? GRAPH_STEPS : 1;
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = enqueue_step(s, s->cap);
    cudaError_t e2 = cudaStreamEndCapture(s->cap, &g);
    if (e != cudaSuccess) return fail(s, MS_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    if (e2 != cudaSuccess) return fail(s, MS_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e2));
    cudaGraphExec_t ex;
    CK(cudaGraphInstantiate(&ex, g, 0));
    CK(cudaGraphDestroy(g));
    (which == 0 ? s->g_many : s->g_one) = ex;
  }
  return MS_OK;
}

// The fan-out rule: among edge lane l's links toward edge en, the first whose target lane
// links to en2 (any link if en2 < 0), else the first; returns its index among l's successor
// entries, -1 if l has no link toward en.
bool lane_links_to(const Sim *s, int l, int e);
int host_choose_entry(const Sim *s, int l, int en, int en2) {
  int first = -1;
  for (int k = s->succ_off[l]; k < s->succ_off[l + 1]; ++k) {
    if (s->succ_edge[k] != en || s->link_off[k]) continue;   // closed links are no links
    const int j = k - s->succ_off[l];
    if (first < 0) first = j;
    if (en2 < 0) return j;
    if (lane_links_to(s, s->succ_lane[s->succ_off[s->succ_lane[k]]], en2)) return j;
  }
  return first;
}

// Link plan word of routes[] entry r (layout in step_kernels.cuh): the fan-out choice of
// every lane of edge routes[r] toward routes[r + 1], by lane position.
constexpr unsigned long long PLAN_ALL_NONE = (1ull << (PLAN_BITS * PLAN_LANES)) - 1;
unsigned long long plan_word(const Sim *s, size_t r) {
  const int *R = s->h_routes.data();
  const int e = R[r];
  if (e < 0 || R[r + 1] < 0) return PLAN_ALL_NONE | PLAN_END;
  const int en = R[r + 1], en2 = R[r + 2];
  unsigned long long w = PLAN_ALL_NONE;
  for (int q = 0; q < s->edge_nlanes[e]; ++q) {
    const int k = host_choose_entry(s, s->edge_lane0[e] + q, en, en2);
    if (k >= 0) w &= ~((unsigned long long)(PLAN_NONE ^ (unsigned)k) << (PLAN_BITS * q));
  }
  return w;
}

void build_plans(Sim *s) {
  const size_t n = s->h_routes.size();
  s->h_plan.assign(n, 0);
  const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  const size_t chunk = (n + nt - 1) / nt;
  std::vector<std::thread> th;
  for (unsigned k = 0; k < nt; ++k)
    th.emplace_back([s, k, chunk, n] {
      for (size_t r = k * chunk; r < std::min(n, (k + 1) * chunk); ++r) s->h_plan[r] = plan_word(s, r);
    });
  for (auto &x : th) x.join();
}

// lane entered at the end of edge lane l (plan word w, l's successor entries)
int plan_lane(const Sim *s, unsigned long long w, int l) {
  if (w & PLAN_END) return NL_END;
  const unsigned k = plan_nib(w, l - s->edge_lane0[s->lane_edge[l]]);
  return k == PLAN_NONE ? NL_NONE : s->succ_lane[s->succ_off[l] + k];
}

// the cached next-lane choice of a vehicle on `lane` at route entry rp (on an internal lane:
// the choice at the end of its target lane, from the plan of the target's edge)
int host_next_choice(const Sim *s, int lane, int rp) {
  if (s->lane_edge[lane] >= 0) return plan_lane(s, s->h_plan[rp], lane);
  return plan_lane(s, s->h_plan[rp + 1], s->succ_lane[s->succ_off[lane]]);
}

bool lane_links_to(const Sim *s, int l, int e) {
  for (int k = s->succ_off[l]; k < s->succ_off[l + 1]; ++k)
    if (s->succ_edge[k] == e && !s->link_off[k]) return true;
  return false;
}

// queue heads and the departure step of each head trip
int upload_queues(Sim *s, const std::vector<int> &qhead) {
  std::vector<int> due(s->n_lanes);   // a closed lane's head is parked (never due)
  for (int l = 0; l < s->n_lanes; ++l)
    due[l] = qhead[l] < s->h_qoff[l + 1] && !s->h_lane_closed[l] ? s->h_tdep[s->h_qtrip[qhead[l]]] : 0x7fffffff;
  std::vector<int2> hd(s->n_lanes);
  for (int l = 0; l < s->n_lanes; ++l) hd[l] = make_int2(qhead[l], due[l]);
  CK(cudaMemcpy(s->d_qhd, hd.data(), sizeof(int2) * s->n_lanes, cudaMemcpyHostToDevice));
  return MS_OK;
}

// What a departure writes is known beforehand: the trip, its route start, second edge and
// next-lane choice on the departure lane, its v0, and when the lane's next trip is due (the
// choice and the plan word depend on the lane links, so a link change rebuilds them).
int upload_queue_entries(Sim *s) {
  std::vector<int4> qe(s->h_qtrip.size(), make_int4(0, 0, 0, 0));
  std::vector<int4> qe2(s->h_qtrip.size(), make_int4(0, 0, 0x7fffffff, 0));
  for (int l = 0; l < s->n_lanes; ++l)
    for (int j = s->h_qoff[l]; j < s->h_qoff[l + 1]; ++j) {
      const int trip = s->h_qtrip[j], r0 = s->h_route0[trip];
      float v0 = s->h_v0[trip];
      int v0b;
      std::memcpy(&v0b, &v0, 4);
      qe[j] = make_int4(trip, r0, host_next_choice(s, l, r0), v0b);
      const unsigned long long w = s->h_plan[r0];
      qe2[j] = make_int4((int)(unsigned)(w & 0xffffffffu), (int)(unsigned)(w >> 32),
                         j + 1 < s->h_qoff[l + 1] ? s->h_tdep[s->h_qtrip[j + 1]] : 0x7fffffff, 0);
    }
  CK(cudaMemcpy(s->d_qent, qe.data(), sizeof(int4) * qe.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_qent2, qe2.data(), sizeof(int4) * qe2.size(), cudaMemcpyHostToDevice));
  return MS_OK;
}

int upload_state(Sim *s, const std::vector<int> &ids, const std::vector<int> &lanes,
                 const std::vector<float> &xs, const std::vector<float> &vs,
                 const std::vector<int> &route_idx, int t, const int *ctrl_state) {
  // vehicles must be sorted by (lane, x, id); builds the SoA of parity t & 1
  const int n = (int)ids.size();
  if (n > s->n_trips) return fail(s, MS_ERR_CAPACITY, "more active vehicles than trips");
  std::vector<float> v0(n);
  std::vector<int> rp(n), nlc(n);
  std::vector<unsigned long long> pl(n);
  std::vector<int> cnt(s->n_lanes, 0);
  std::vector<char> seen(s->n_trips, 0);
  for (int i = 0; i < n; ++i) {
    int id = ids[i], l = lanes[i];
    if (id < 0 || id >= s->n_trips || seen[id]) return fail(s, MS_ERR_ARG, "vehicle id invalid or repeated");
    seen[id] = 1;
    if (l < 0 || l >= s->n_lanes) return fail(s, MS_ERR_ARG, "vehicle lane out of range");
    if (!(xs[i] > 0.f) || !(xs[i] <= s->lane_len[l])) return fail(s, MS_ERR_ARG, "vehicle x not in (0, len]");
    if (!(vs[i] >= 0.f) || vs[i] > s->P.v_max) return fail(s, MS_ERR_ARG, "vehicle speed outside [0, v_max]");
    if (i > 0) {
      int pl = lanes[i - 1];
      if (pl > l || (pl == l && xs[i - 1] > xs[i]))
        return fail(s, MS_ERR_ARG, "vehicles not sorted by (lane, x)");
      // gap-0 stops round by a few FP32 ulps of x (about 2e-3 m at 18 km)
      if (pl == l && (xs[i] - s->P.L) - xs[i - 1] < -std::max(1e-3f, 5e-7f * xs[i]))
        return fail(s, MS_ERR_ARG, "overlapping vehicles (gap < 0) on a lane");
    }
    int r0 = s->h_route0[id];
    int rlen = 0;
    while (s->h_routes[r0 + rlen] >= 0) ++rlen;
    int ri = route_idx[i];
    if (ri < 0 || ri >= rlen) return fail(s, MS_ERR_ARG, "route index out of range");
    int e = s->h_routes[r0 + ri];
    if (s->lane_edge[l] >= 0) {
      if (s->lane_edge[l] != e) return fail(s, MS_ERR_ARG, "vehicle lane is not on its route edge");
    } else {
      int en = ri + 1 < rlen ? s->h_routes[r0 + ri + 1] : -1;
      int tg = s->succ_lane[s->succ_off[l]];
      bool ok = en >= 0 && s->lane_edge[tg] == en;
      if (ok) {
        ok = false;   // the internal lane must leave from a lane of edge e
        for (int q = 0; q < s->edge_nlanes[e] && !ok; ++q) {
          int al = s->edge_lane0[e] + q;
          for (int k = s->succ_off[al]; k < s->succ_off[al + 1]; ++k)
            if (s->succ_lane[k] == l) ok = true;
        }
      }
      if (!ok) return fail(s, MS_ERR_ARG, "vehicle on an internal lane that its route does not use");
    }
    v0[i] = s->h_v0[id];
    rp[i] = r0 + ri;
    pl[i] = s->h_plan[r0 + ri];
    nlc[i] = host_next_choice(s, l, r0 + ri);
    cnt[l]++;
  }
  std::vector<int4> dyn(s->n_lanes);
  int acc = 0;
  for (int l = 0; l < s->n_lanes; ++l) {
    dyn[l] = make_int4(acc, cnt[l], 0, 0);
    if (cnt[l]) {   // tail fields: the rearmost vehicle of the lane
      float tx = xs[acc], tv = vs[acc];
      std::memcpy(&dyn[l].z, &tx, 4);
      std::memcpy(&dyn[l].w, &tv, 4);
    }
    acc += cnt[l];
  }
  const int p = t & 1;
  cudaStream_t st = s->stream;
  Soa &B = s->A[p];
  if (n) {
    CK(cudaMemcpyAsync(B.x, xs.data(), n * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.v, vs.data(), n * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.v0, v0.data(), n * sizeof(float), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.lane, lanes.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.rp, rp.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.pl, pl.data(), n * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.nl, nlc.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B.id, ids.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  CK(cudaMemcpyAsync(s->d_dyn[p], dyn.data(), s->n_lanes * sizeof(int4), cudaMemcpyHostToDevice, st));
  if (s->prm.signal_mode == 0) {   // signal table of step t (later steps': k_lanes)
    std::vector<int> sig(s->h_ctrl4.size(), 0);
    for (int c = 0; c < s->n_ctrl; ++c) sig[c] = sig_pack(s->h_ctrl4[c], t);
    CK(cudaMemcpyAsync(s->d_sig[p], sig.data(), sig.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  DevCtrl c{};
  CK(cudaMemcpyAsync(&c, s->d_ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  c.t = t;
  s->t_host = t;
  c.t_apply = t;
  c.n_active[p] = n;
  c.n_movers = 0;
  CK(cudaMemcpyAsync(s->d_ctrl, &c, sizeof(DevCtrl), cudaMemcpyHostToDevice, st));
  if (s->prm.signal_mode == 1 && s->n_ctrl > 0) {
    // max-pressure controllers: restored, or restarted with phase 0 green; then advanced to
    // step t on the uploaded state (a no-op for a state already at t), which writes the
    // signal table of step t
    std::vector<int4> mp(s->n_ctrl, make_int4(0, -1, 0, 0));
    if (ctrl_state)
      for (int k = 0; k < s->n_ctrl; ++k) {
        mp[k] = make_int4(ctrl_state[3 * k], ctrl_state[3 * k + 1], ctrl_state[3 * k + 2], 0);
        if (mp[k].x < 0 || mp[k].x >= s->h_ctrl4[k].w || mp[k].y < -1 || mp[k].y >= s->h_ctrl4[k].w)
          return fail(s, MS_ERR_ARG, "ctrl_state phase out of range");
      }
    CK(cudaMemcpyAsync(s->d_mp, mp.data(), mp.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    k_signals<<<(s->n_ctrl + 7) / 8, 256, 0, st>>>(make_args(s));
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(st));
  return MS_OK;
}

}  // namespace

// Cached choices of the vehicles of the current state under rebuilt link plans: the plan
// word of the current route entry and the next-lane choice (for a vehicle on an internal
// lane, the choice at the end of its target lane, from the next entry's plan).
__global__ void k_refresh_choices(StepArgs a, Soa S, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int rp = S.rp[i];
    const LaneInfo li = a.li[S.lane[i]];
    const unsigned long long pl = a.plan[rp];
    S.pl[i] = pl;
    S.nl[i] = li.edge >= 0 ? plan_next(a, pl, li.idx, li.succ) : plan_next(a, a.plan[rp + 1], li.idx, li.left);
  }
}

// run f(k0, k1) over [0, n) in chunks on the host's threads
template <class F>
static void host_parallel(size_t n, F f) {
  const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  const size_t chunk = (n + nt - 1) / nt;
  std::vector<std::thread> th;
  for (unsigned k = 0; k < nt; ++k)
    th.emplace_back([=] { f(std::min(n, k * chunk), std::min(n, (k + 1) * chunk)); });
  for (auto &x : th) x.join();
}

extern "C" {

int ms_create(void **out, const ms_params *p, void *cuda_stream) {
  if (!out || !p) return MS_ERR_ARG;
  *out = nullptr;
  Sim *s = new Sim();
  s->prm = *p;
  if (s->prm.block == 0) s->prm.block = 256;
  auto bad = [&](const char *m) {
    std::fprintf(stderr, "ms_create: %s\n", m);
    delete s;
    return MS_ERR_ARG;
  };
  if (!(p->dt > 0) || !(p->veh_len > 0) || !(p->idm_a > 0) || !(p->idm_b > 0) || !(p->idm_T >= 0) ||
      !(p->idm_s0 >= 0))
    return bad("dt, veh_len, idm_a, idm_b must be > 0; idm_T, idm_s0 >= 0");
  if (!(p->p_lc >= 0 && p->p_lc <= 1)) return bad("p_lc must be in [0, 1]");
  if (!(p->mobil_th_jitter >= 0)) return bad("mobil_th_jitter must be >= 0");
  if (p->signal_mode != 0 && p->signal_mode != 1) return bad("signal_mode must be 0 or 1");
  if (p->signal_mode == 1 && p->mp_interval < 1) return bad("mp_interval must be >= 1");
  if (!(p->a_min < 0) || !(p->v_max > 0) || !(p->d_look > 0)) return bad("a_min < 0, v_max > 0, d_look > 0 required");
  if (p->window <= 0 || p->n_windows < 0) return bad("window > 0 and n_windows >= 0 required");
  if (s->prm.block % 32 || s->prm.block < 32 || s->prm.block > 512) return bad("block must be a multiple of 32 in [32, 512]");
  DevParams &P = s->P;
  P.dt = p->dt; P.L = p->veh_len; P.a = p->idm_a; P.b = p->idm_b; P.T = p->idm_T; P.s0 = p->idm_s0;
  P.p = p->mobil_p; P.th = p->mobil_th; P.bsafe = p->mobil_bsafe; P.a_min = p->a_min;
  P.v_max = p->v_max; P.d_look = p->d_look; P.x_lc_min = p->x_lc_min; P.x_lc_end = p->x_lc_end;
  P.inv2sqrtab = (float)(1.0 / (2.0 * std::sqrt((double)p->idm_a * (double)p->idm_b)));
  P.inv2b = (float)(1.0 / (2.0 * (double)p->idm_b));
  P.lc_thresh = (uint32_t)std::floor((double)p->p_lc * 16777216.0);
  P.seed = p->seed;
  P.window = p->window;
  P.n_windows = p->n_windows;
  P.debug = p->debug;
  P.id_base = p->id_base;
  P.th_jitter = p->mobil_th_jitter;
  P.signal_mode = p->signal_mode;
  P.mp_interval = p->mp_interval;
  s->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, s->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->xs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_ready, cudaEventDisableTiming);
  for (int k = 0; k < Sim::MS_EXPORTS; ++k)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_export[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->h_meta, 2 * Sim::MS_EXPORTS * sizeof(int), cudaHostAllocMapped);
  if (e != cudaSuccess) {
    std::fprintf(stderr, "ms_create: %s\n", cudaGetErrorString(e));
    delete s;
    return MS_ERR_CUDA;
  }
  *out = s;
  return MS_OK;
}

int ms_load_network(void *sim, const ms_network *net) {
  Sim *s = (Sim *)sim;
  if (!s || !net) return MS_ERR_ARG;
  if (s->net_loaded) return fail(s, MS_ERR_STATE, "network already loaded");
  const int L = net->n_lanes, E = net->n_edges, C = net->n_ctrl;
  if (L <= 0 || E <= 0 || C < 0) return fail(s, MS_ERR_ARG, "n_lanes, n_edges must be > 0");
  // a lane id travels in the low CODE_LANE_BITS bits of a vehicle's result code
  if (L > CODE_LANE_MASK) return fail(s, MS_ERR_CAPACITY, "more lanes than a result code can name");
  if (!net->lane_len || !net->lane_edge || !net->lane_index || !net->lane_left || !net->lane_right ||
      !net->succ_off || !net->succ_lane || !net->succ_edge || !net->lane_ctrl || !net->lane_group ||
      !net->edge_nlanes || !net->edge_lane0 || (C > 0 && (!net->ctrl_offset || !net->ctrl_green ||
                                                          !net->ctrl_yellow || !net->ctrl_nphase)))
    return fail(s, MS_ERR_ARG, "network array missing");
  s->n_lanes = L; s->n_edges = E; s->n_ctrl = C;
  s->lane_len.assign(net->lane_len, net->lane_len + L);
  s->lane_edge.assign(net->lane_edge, net->lane_edge + L);
  s->lane_left.assign(net->lane_left, net->lane_left + L);
  s->lane_right.assign(net->lane_right, net->lane_right + L);
  s->succ_off.assign(net->succ_off, net->succ_off + L + 1);
  s->edge_nlanes.assign(net->edge_nlanes, net->edge_nlanes + E);
  s->edge_lane0.assign(net->edge_lane0, net->edge_lane0 + E);
  const int S = s->succ_off[L];
  if (s->succ_off[0] != 0 || S < 0) return fail(s, MS_ERR_ARG, "succ_off must start at 0");
  for (int l = 0; l < L; ++l)
    if (s->succ_off[l + 1] < s->succ_off[l]) return fail(s, MS_ERR_ARG, "succ_off not monotone");
  s->succ_lane.assign(net->succ_lane, net->succ_lane + S);
  s->succ_edge.assign(net->succ_edge, net->succ_edge + S);
  s->link_off.assign(std::max(1, S), 0);   // every lane link open
  const float min_len = s->P.v_max * s->P.dt;
  std::vector<LaneInfo> li(L);
  std::vector<int> npred(L, 0);
  for (int l = 0; l < L; ++l) {
    const int e = s->lane_edge[l];
    const int ns = s->succ_off[l + 1] - s->succ_off[l];
    if (!(s->lane_len[l] > min_len))
      return fail(s, MS_ERR_ARG, "lane " + std::to_string(l) + " not longer than v_max*dt");
    if (e >= E) return fail(s, MS_ERR_ARG, "lane_edge out of range");
    for (int k = s->succ_off[l]; k < s->succ_off[l + 1]; ++k) {
      int sl = s->succ_lane[k], se = s->succ_edge[k];
      if (sl < 0 || sl >= L || se < 0 || se >= E) return fail(s, MS_ERR_ARG, "successor out of range");
      if (e >= 0 && s->lane_edge[sl] >= 0) return fail(s, MS_ERR_ARG, "edge lane successors must be internal lanes");
      if (e < 0 && (s->lane_edge[sl] != se)) return fail(s, MS_ERR_ARG, "internal lane target / edge mismatch");
    }
    if (e < 0) {
      if (ns != 1) return fail(s, MS_ERR_ARG, "internal lane must have exactly one successor");
      if (s->lane_left[l] >= 0 || s->lane_right[l] >= 0) return fail(s, MS_ERR_ARG, "internal lane with neighbours");
      npred[s->succ_lane[s->succ_off[l]]]++;
    } else {
      if (ns > (int)PLAN_NONE) return fail(s, MS_ERR_CAPACITY, "an edge lane has more than 63 lane links");
      int lf = s->lane_left[l], rt = s->lane_right[l];
      if (lf >= L || rt >= L) return fail(s, MS_ERR_ARG, "left/right out of range");
      if (lf >= 0 && (s->lane_edge[lf] != e || s->lane_right[lf] != l)) return fail(s, MS_ERR_ARG, "left/right inconsistent");
      if (rt >= 0 && (s->lane_edge[rt] != e || s->lane_left[rt] != l)) return fail(s, MS_ERR_ARG, "left/right inconsistent");
      if (s->lane_len[l] != s->lane_len[s->edge_lane0[e]]) return fail(s, MS_ERR_ARG, "lanes of an edge differ in length");
    }
    int c = net->lane_ctrl[l];
    if (c >= C || (c >= 0 && (net->lane_group[l] < 0 || net->lane_group[l] >= net->ctrl_nphase[c] ||
                              net->lane_group[l] > 255)))
      return fail(s, MS_ERR_ARG, "lane_ctrl / lane_group invalid");
    li[l].len = s->lane_len[l];
    li[l].edge = e;
    if (e >= 0) {
      li[l].left = s->lane_left[l];
      li[l].right = s->lane_right[l];
    } else {   // internal lane: its target lane's successor range
      const int tg = s->succ_lane[s->succ_off[l]];
      li[l].left = s->succ_off[tg];
      li[l].right = s->succ_off[tg + 1] - s->succ_off[tg];
    }
    li[l].succ = e < 0 ? s->succ_lane[s->succ_off[l]] : s->succ_off[l];
    li[l].ctrl = c;
    li[l].n_succ = (unsigned char)(e < 0 ? 1 : ns);
    li[l].group = (unsigned char)(c >= 0 ? net->lane_group[l] : 0);
  }
  // an edge's lanes are lanes edge_lane0 .. edge_lane0 + nlanes - 1, numbered from the right:
  // index q = l - edge_lane0, left neighbour q + 1, right neighbour q - 1
  for (int e = 0; e < E; ++e) {
    const int l0 = s->edge_lane0[e], ne = s->edge_nlanes[e];
    if (ne <= 0 || l0 < 0 || l0 + ne > L) return fail(s, MS_ERR_ARG, "edge lanes out of range");
    if (ne > PLAN_LANES) return fail(s, MS_ERR_CAPACITY, "an edge has more than 10 lanes");
    for (int q = 0; q < ne; ++q) {
      const int l = l0 + q;
      if (s->lane_edge[l] != e || net->lane_index[l] != q || s->lane_left[l] != (q + 1 < ne ? l + 1 : -1) ||
          s->lane_right[l] != (q > 0 ? l - 1 : -1))
        return fail(s, MS_ERR_ARG, "lanes of edge " + std::to_string(e) +
                                       " must be edge_lane0 + q with lane_index q, left q + 1, right q - 1");
    }
  }
  for (int l = 0; l < L; ++l) {
    const int e = s->lane_edge[l];
    if (e >= 0 && (l < s->edge_lane0[e] || l >= s->edge_lane0[e] + s->edge_nlanes[e]))
      return fail(s, MS_ERR_ARG, "lane " + std::to_string(l) + " lies outside its edge's lane range");
  }
  // plan position: an edge lane's index across its edge; an internal lane's target's index
  for (int l = 0; l < L; ++l) {
    const int e = s->lane_edge[l];
    const int q = e >= 0 ? l - s->edge_lane0[e] : s->succ_lane[s->succ_off[l]] - s->edge_lane0[s->lane_edge[s->succ_lane[s->succ_off[l]]]];
    li[l].idx = (unsigned char)q;
  }
  std::vector<int> pred_off(L + 1, 0);
  for (int l = 0; l < L; ++l) {
    if (npred[l] > 255) return fail(s, MS_ERR_ARG, "more than 255 feeders");
    pred_off[l + 1] = pred_off[l] + npred[l];
    li[l].pred = pred_off[l];
    li[l].n_pred = (unsigned char)npred[l];
  }
  std::vector<int> pred(std::max(1, pred_off[L])), fill(L, 0);
  for (int l = 0; l < L; ++l)
    if (s->lane_edge[l] < 0) {
      int tg = s->succ_lane[s->succ_off[l]];
      pred[pred_off[tg] + fill[tg]++] = l;
    }
  std::vector<int2> succ(std::max(1, S));
  for (int k = 0; k < S; ++k) succ[k] = make_int2(s->succ_lane[k], s->succ_edge[k]);
  std::vector<int4> c4(std::max(1, C));
  for (int c = 0; c < C; ++c) {
    if (net->ctrl_green[c] <= 0 || net->ctrl_yellow[c] < 0 || net->ctrl_nphase[c] <= 0)
      return fail(s, MS_ERR_ARG, "controller timing invalid");
    c4[c] = make_int4(net->ctrl_offset[c], net->ctrl_green[c], net->ctrl_yellow[c], net->ctrl_nphase[c]);
  }
  s->P.n_lanes = L;
  DALLOC(s->d_li, L);
  DALLOC(s->d_succ, succ.size());
  DALLOC(s->d_link_off, s->link_off.size());
  DALLOC(s->d_pred, pred.size());
  DALLOC(s->d_ctrl4, c4.size());
  DALLOC(s->d_sig[0], c4.size());
  DALLOC(s->d_sig[1], c4.size());
  s->h_ctrl4 = c4;
  {   // approach edge lanes of each controller, for the max-pressure controllers
    std::vector<int> off(c4.size() + 1, 0), lanes;
    for (int l = 0; l < L; ++l)
      if (net->lane_ctrl[l] >= 0 && s->lane_edge[l] >= 0) off[net->lane_ctrl[l] + 1]++;
    for (size_t c = 0; c < c4.size(); ++c) off[c + 1] += off[c];
    lanes.assign(std::max(1, off[c4.size()]), 0);
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (int l = 0; l < L; ++l)
      if (net->lane_ctrl[l] >= 0 && s->lane_edge[l] >= 0) lanes[fill[net->lane_ctrl[l]]++] = l;
    if (s->prm.signal_mode == 1)
      for (int c = 0; c < C; ++c) {
        if (c4[c].w > 32) return fail(s, MS_ERR_ARG, "max-pressure control takes at most 32 phases per controller");
        if (c4[c].z >= s->prm.mp_interval) return fail(s, MS_ERR_ARG, "ctrl_yellow must be below mp_interval");
      }
    DALLOC(s->d_mp, c4.size());
    std::vector<int4> mp0(c4.size(), make_int4(0, -1, 0, 0));
    CK(cudaMemcpy(s->d_mp, mp0.data(), mp0.size() * sizeof(int4), cudaMemcpyHostToDevice));
    DALLOC(s->d_ctrl_loff, off.size());
    DALLOC(s->d_ctrl_lanes, lanes.size());
    CK(cudaMemcpy(s->d_ctrl_loff, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(s->d_ctrl_lanes, lanes.data(), lanes.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  CK(cudaMemcpy(s->d_li, li.data(), L * sizeof(LaneInfo), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_succ, succ.data(), succ.size() * sizeof(int2), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_link_off, s->link_off.data(), s->link_off.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_pred, pred.data(), pred.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_ctrl4, c4.data(), c4.size() * sizeof(int4), cudaMemcpyHostToDevice));
  s->n_tiles = (L + LANE_TILE - 1) / LANE_TILE;
  s->h_lane_vmax.assign(L, INFINITY);
  s->h_lane_closed.assign(L, 0);
  DALLOC(s->d_lane_vmax, L);
  DALLOC(s->d_lane_closed, L);
  CK(cudaMemcpy(s->d_lane_vmax, s->h_lane_vmax.data(), L * sizeof(float), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_lane_closed, s->h_lane_closed.data(), L, cudaMemcpyHostToDevice));
  s->net_loaded = true;
  return MS_OK;
}

int ms_add_vehicles(void *sim, const ms_vehicles *veh) {
  Sim *s = (Sim *)sim;
  if (!s || !veh) return MS_ERR_ARG;
  if (!s->net_loaded) return fail(s, MS_ERR_STATE, "load the network first");
  if (s->veh_loaded) return fail(s, MS_ERR_STATE, "vehicles already added");
  const int n = veh->n;
  if (n <= 0 || !veh->t_dep || !veh->v0 || !veh->route_off || !veh->route_edges)
    return fail(s, MS_ERR_ARG, "vehicle arrays missing or n <= 0");
  s->n_trips = n;
  s->h_route0.resize(n);
  s->h_tdep.assign(veh->t_dep, veh->t_dep + n);
  s->h_v0.assign(veh->v0, veh->v0 + n);
  s->h_routes.clear();
  s->h_routes.reserve((size_t)veh->route_off[n] + n);
  for (int i = 0; i < n; ++i) {
    int64_t a = veh->route_off[i], b = veh->route_off[i + 1];
    if (b <= a) return fail(s, MS_ERR_ARG, "empty route for trip " + std::to_string(i));
    if (!(s->h_v0[i] > 0.f) || s->h_v0[i] > s->P.v_max) return fail(s, MS_ERR_ARG, "v0 outside (0, v_max]");
    s->h_route0[i] = (int)s->h_routes.size();
    for (int64_t k = a; k < b; ++k) {
      int e = veh->route_edges[k];
      if (e < 0 || e >= s->n_edges) return fail(s, MS_ERR_ARG, "route edge out of range");
      if (k > a) {
        int pe = veh->route_edges[k - 1];
        bool ok = false;
        for (int q = 0; q < s->edge_nlanes[pe] && !ok; ++q) ok = lane_links_to(s, s->edge_lane0[pe] + q, e);
        if (!ok)
          return fail(s, MS_ERR_ROUTE, "trip " + std::to_string(i) + ": edges " + std::to_string(pe) + " -> " +
                                           std::to_string(e) + " have no lane link");
      }
      s->h_routes.push_back(e);
    }
    s->h_routes.push_back(-1);
    if (s->h_routes.size() > (size_t)0x7fff0000) return fail(s, MS_ERR_CAPACITY, "routes too long");
  }
  build_plans(s);
  // placed vehicles, sorted by (lane, x, id)
  std::vector<int> placed;
  if (veh->lane) {
    if (!veh->x || !veh->v) return fail(s, MS_ERR_ARG, "placement needs x and v");
    for (int i = 0; i < n; ++i) {
      int l = veh->lane[i];
      if (l >= s->n_lanes) return fail(s, MS_ERR_ARG, "placement lane out of range");
      if (l >= 0) placed.push_back(i);
    }
    std::sort(placed.begin(), placed.end(), [&](int a, int b) {
      if (veh->lane[a] != veh->lane[b]) return veh->lane[a] < veh->lane[b];
      if (veh->x[a] != veh->x[b]) return veh->x[a] < veh->x[b];
      return a < b;
    });
  }
  // departure FIFOs of unplaced trips: lowest-index lane of the first edge that links to the
  // second edge, ordered by (t_dep, id)
  std::vector<int> dep_lane(n, -1);
  std::vector<char> is_placed(n, 0);
  for (int i : placed) is_placed[i] = 1;
  std::vector<int> qcnt(s->n_lanes, 0);
  for (int i = 0; i < n; ++i) {
    if (is_placed[i]) continue;
    int r0 = s->h_route0[i];
    int e0 = s->h_routes[r0], e1 = s->h_routes[r0 + 1];
    int dl = -1;
    for (int q = 0; q < s->edge_nlanes[e0] && dl < 0; ++q) {
      int l = s->edge_lane0[e0] + q;
      if (e1 < 0 || lane_links_to(s, l, e1)) dl = l;
    }
    dep_lane[i] = dl;
    qcnt[dl]++;
  }
  s->h_qoff.assign(s->n_lanes + 1, 0);
  for (int l = 0; l < s->n_lanes; ++l) s->h_qoff[l + 1] = s->h_qoff[l] + qcnt[l];
  s->P.fifo = s->h_qoff[s->n_lanes] > 0 ? 1 : 0;
  s->h_qtrip.assign(std::max(1, s->h_qoff[s->n_lanes]), 0);
  {
    std::vector<int> ord;
    for (int i = 0; i < n; ++i)
      if (!is_placed[i]) ord.push_back(i);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) {
      if (dep_lane[a] != dep_lane[b]) return dep_lane[a] < dep_lane[b];
      if (s->h_tdep[a] != s->h_tdep[b]) return s->h_tdep[a] < s->h_tdep[b];
      return a < b;
    });
    for (size_t k = 0; k < ord.size(); ++k) s->h_qtrip[k] = ord[k];
  }
  // device allocations sized for every trip at once; the vehicle arrays to a multiple of four
  // entries (the apply kernel copies whole 16-byte words of them into shared memory)
  const int N = n;
  const int NS = (N + 3) & ~3;
  for (int b = 0; b < 2; ++b) {
    DALLOC(s->A[b].x, NS); DALLOC(s->A[b].v, NS); DALLOC(s->A[b].v0, NS);
    DALLOC(s->A[b].lane, NS); DALLOC(s->A[b].rp, NS); DALLOC(s->A[b].pl, NS); DALLOC(s->A[b].nl, NS);
    DALLOC(s->A[b].id, NS);
    DALLOC(s->d_dyn[b], s->n_lanes);
  }
  DALLOC(s->d_ctrl, 1);
  // k_decide writes one word per warp of every block iteration below n: up to (N + block) / 32
  const int leave_words = (N + 1024) / 32 + 2;
  DALLOC(s->d_leave, leave_words);
  DALLOC(s->d_arr_cnt, s->n_lanes);
  DALLOC(s->d_amin, s->n_lanes);
  DALLOC(s->d_arr_start, s->n_lanes + 1);
  DALLOC(s->d_bucket, N);
  DALLOC(s->d_res_x, NS);
  DALLOC(s->d_res_v, NS);
  DALLOC(s->d_res_code, N + 4);   // k_bucket reads it four codes at a time
  DALLOC(s->d_res_nl, N);
  DALLOC(s->d_res_pos, N);
  DALLOC(s->d_arr_fill, s->n_lanes);
  DALLOC(s->d_tile_agg, s->n_tiles);
  DALLOC(s->d_qoff, s->n_lanes + 1);
  DALLOC(s->d_qtrip, s->h_qtrip.size());
  DALLOC(s->d_qent, s->h_qtrip.size());
  DALLOC(s->d_qent2, s->h_qtrip.size());
  DALLOC(s->d_plan, s->h_plan.size());
  DALLOC(s->d_qhd, s->n_lanes);
  DALLOC(s->d_tdep, N);
  DALLOC(s->d_route0, N);
  DALLOC(s->d_tarr, N);
  DALLOC(s->d_routes, s->h_routes.size());
  if (s->prm.n_windows > 0) {
    DALLOC(s->d_vsum, (size_t)s->prm.n_windows * s->n_lanes);
    DALLOC(s->d_vcnt, (size_t)s->prm.n_windows * s->n_lanes);
    CK(cudaMemset(s->d_vsum, 0, sizeof(unsigned long long) * s->prm.n_windows * s->n_lanes));
    CK(cudaMemset(s->d_vcnt, 0, sizeof(int) * s->prm.n_windows * s->n_lanes));
  }
  if (s->prm.debug) {
    DebugOut &d = s->dbg;
    DALLOC(d.id, N); DALLOC(d.lead_kind, N); DALLOC(d.lead_id, N); DALLOC(d.lc_dir, N);
    DALLOC(d.lc_cand, N); DALLOC(d.tau_lead, N); DALLOC(d.tau_foll, N); DALLOC(d.old_foll, N);
    DALLOC(d.flag, N); DALLOC(d.s_own, N); DALLOC(d.vl_own, N); DALLOC(d.a_own, N);
    DALLOC(d.incentive, N); DALLOC(d.a_use, N); DALLOC(d.trip_ins, N); DALLOC(d.trip_flag, N);
    DALLOC(d.arr_flag, s->n_lanes);
    DALLOC(d.lc_learn, N); DALLOC(d.lc_margin, N); DALLOC(d.lc_logit, (size_t)3 * N);
    DALLOC(d.lc_feat, (size_t)MLP_IN * N);
    CK(cudaMemset(d.trip_ins, 0, sizeof(int) * N));
    CK(cudaMemset(d.trip_flag, 0, sizeof(int) * N));
    CK(cudaMemset(d.arr_flag, 0, sizeof(int) * s->n_lanes));
  }
  CK(cudaMemset(s->d_ctrl, 0, sizeof(DevCtrl)));
  CK(cudaMemset(s->d_arr_cnt, 0, sizeof(int) * s->n_lanes));
  CK(cudaMemset(s->d_arr_fill, 0, sizeof(int) * s->n_lanes));
  {
    std::vector<int> amin(s->n_lanes, AMIN_NONE);
    CK(cudaMemcpy(s->d_amin, amin.data(), sizeof(int) * s->n_lanes, cudaMemcpyHostToDevice));
  }
  CK(cudaMemset(s->d_leave, 0, sizeof(unsigned) * leave_words));
  std::vector<int> tarr(n, -1);
  CK(cudaMemcpy(s->d_tarr, tarr.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_qoff, s->h_qoff.data(), sizeof(int) * (s->n_lanes + 1), cudaMemcpyHostToDevice));
  {
    int rq = upload_queues(s, std::vector<int>(s->h_qoff.begin(), s->h_qoff.end() - 1));
    if (rq) return rq;
  }
  CK(cudaMemcpy(s->d_qtrip, s->h_qtrip.data(), sizeof(int) * s->h_qtrip.size(), cudaMemcpyHostToDevice));
  {
    int rq = upload_queue_entries(s);
    if (rq) return rq;
  }
  CK(cudaMemcpy(s->d_tdep, s->h_tdep.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_route0, s->h_route0.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_routes, s->h_routes.data(), sizeof(int) * s->h_routes.size(), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_plan, s->h_plan.data(), sizeof(unsigned long long) * s->h_plan.size(), cudaMemcpyHostToDevice));
  // launch shapes: persistent grids sized by occupancy
  s->cfg.blk_decide = s->cfg.blk_apply = s->prm.block;
  s->cfg.blk_bucket = 256;
  {
    int r0 = shape_grids(s, s->cfg, 1, 1, 1);
    if (r0) return r0;
  }
  s->veh_loaded = true;
  // a model set before the vehicles needs its candidate buffers now; without room for them
  // the model is dropped, the rule decides, and the call still adds the vehicles (the error
  // is returned once they are in place)
  const int r_cand = ensure_cand(s);
  const std::string cand_msg = r_cand ? s->err : std::string();
  if (r_cand) {
    int r0 = shape_grids(s, s->cfg, 1, 1, 1);   // the rule's decide instance
    if (r0) {
      s->veh_loaded = false;
      return r0;
    }
  }
  // initial state
  std::vector<int> ids, lanes, ridx;
  std::vector<float> xs, vs;
  for (int i : placed) {
    ids.push_back(i);
    lanes.push_back(veh->lane[i]);
    xs.push_back(veh->x[i]);
    vs.push_back(veh->v[i]);
    ridx.push_back(0);
  }
  int r = upload_state(s, ids, lanes, xs, vs, ridx, 0, nullptr);
  if (r) {
    s->veh_loaded = false;
    return r;
  }
  if (r_cand)
    return fail(s, r_cand, "vehicles added, but the learned lane-change model was dropped (" + cand_msg +
                               "): the rule decides");
  return MS_OK;
}

// The state at step e sits in buffer e & 1: advancing step e reads it and writes buffer
// (e + 1) & 1, advancing step e + 1 overwrites it.  An export of the state at step e may
// overlap the advance of step e; a launch that includes step e + 1 first waits for it.
static int export_guard(Sim *s, long long n_steps) {
  for (int i = 0; i < s->ex_count; ++i) {
    const int k = (s->ex_head + i) % Sim::MS_EXPORTS;
    if (s->t_host + n_steps > s->export_t[k] + 1) CK(cudaStreamWaitEvent(s->stream, s->ev_export[k], 0));
  }
  return MS_OK;
}

// entry points that overwrite the state buffers from the host wait for an export in flight
static int export_drain(Sim *s) {
  if (s->ex_count > 0) CK(cudaStreamSynchronize(s->xs));
  return MS_OK;
}

int ms_step(void *sim, int n) {
  Sim *s = (Sim *)sim;
  if (!s) return MS_ERR_ARG;
  if (!s->veh_loaded) return fail(s, MS_ERR_STATE, "add vehicles before stepping");
  if (n < 0) return fail(s, MS_ERR_ARG, "n < 0");
  int r = build_graphs(s);
  if (r) return r;
  r = export_guard(s, n);
  if (r) return r;
  s->t_host += n;
  while (n >= GRAPH_STEPS) {
    CK(cudaGraphLaunch(s->g_many, s->stream));
    n -= GRAPH_STEPS;
  }
  while (n-- > 0) CK(cudaGraphLaunch(s->g_one, s->stream));
  return MS_OK;
}

int ms_step_timed(void *sim, int n, float *ms_per_kernel) {
  Sim *s = (Sim *)sim;
  if (!s || !ms_per_kernel) return MS_ERR_ARG;
  if (!s->veh_loaded) return fail(s, MS_ERR_STATE, "add vehicles before stepping");
  {
    int r = export_guard(s, n);
    if (r) return r;
    s->t_host += n;
  }
  cudaEvent_t ev[5];
  for (auto &e : ev) CK(cudaEventCreate(&e));
  cudaStream_t st = s->stream;
  StepArgs a = make_args(s);
  for (int k = 0; k < n; ++k) {
    CK(launch_step(s, a, st, ev));
    CK(cudaEventSynchronize(ev[4]));
    for (int q = 0; q < 4; ++q) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[q], ev[q + 1]));
      ms_per_kernel[q] += ms;
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  return MS_OK;
}

// Lane-scan tile aggregates for ms_step_noalloc (8 bytes per tile, MS_NOALLOC_MAX_TILES
// tiles).  One copy per device for the whole process; shared by every call (see moss103.h).
static_assert(LANE_TILE == MS_NOALLOC_TILE_LANES, "scan tile size and the header disagree");
static __device__ __align__(256) unsigned long long g_noalloc_scan[MS_NOALLOC_MAX_TILES];
static unsigned long long *g_noalloc_addr[256];   // device address per device ordinal

int ms_step_noalloc(void *sim, int n) {
  Sim *s = (Sim *)sim;
  if (!s) return MS_ERR_ARG;
  if (!s->veh_loaded) return fail(s, MS_ERR_STATE, "add vehicles before stepping");
  if (n < 0) return fail(s, MS_ERR_ARG, "n < 0");
  // every refusal comes before anything changes: the host step count (which picks the
  // buffer an export copies) moves only once the steps are really enqueued
  if (s->n_tiles > MS_NOALLOC_MAX_TILES)
    return fail(s, MS_ERR_CAPACITY, "network has " + std::to_string(s->n_lanes) + " lanes; ms_step_noalloc takes at most " +
                                        std::to_string(MS_NOALLOC_MAX_TILES * LANE_TILE));
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != s->device || dev < 0 || dev >= 256) return fail(s, MS_ERR_STATE, "make the simulation's device current");
  if (!g_noalloc_addr[dev]) {
    // host code sees g_noalloc_scan only as a host-side stand-in: resolve the device address
    unsigned long long *ptr = nullptr;
    CK(cudaGetSymbolAddress((void **)&ptr, g_noalloc_scan));
    g_noalloc_addr[dev] = ptr;
  }
  unsigned long long *base = g_noalloc_addr[dev];
  {
    int r = export_guard(s, n);
    if (r) return r;
    s->t_host += n;
  }
  StepArgs a = make_args(s);
  a.tile_agg = base;   // every step's first lane pass writes each tile before any is read
  cudaStream_t st = s->stream;
  for (int k = 0; k < n; ++k) CK(launch_step(s, a, st, nullptr));
  return MS_OK;
}

int ms_sync(void *sim) {
  Sim *s = (Sim *)sim;
  if (!s) return MS_ERR_ARG;
  CK(cudaStreamSynchronize(s->stream));
  if (!s->veh_loaded) return MS_OK;
  unsigned err = 0;
  CK(cudaMemcpy(&err, &s->d_ctrl->err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (err) return fail(s, MS_ERR_DEVICE, "device error bits " + std::to_string(err));
  return MS_OK;
}

int ms_read_state(void *sim, ms_state *out, int device) {
  Sim *s = (Sim *)sim;
  if (!s || !out) return MS_ERR_ARG;
  if (!s->veh_loaded) return fail(s, MS_ERR_STATE, "no vehicles");
  CK(cudaStreamSynchronize(s->stream));
  DevCtrl c;
  CK(cudaMemcpy(&c, s->d_ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost));
  const int p = c.t & 1, n = c.n_active[p];
  out->t = c.t;
  out->n_active = n;
  if (out->capacity < n) return fail(s, MS_ERR_CAPACITY, "state capacity too small");
  const Soa &B = s->A[p];
  // host scratch only for the fields derived on the host (route index, trip status)
  const bool host_ridx = !device && out->route_idx;
  const bool need_ids = host_ridx || out->trip_status;
  std::vector<int> ids(need_ids ? n : 0), rp(host_ridx ? n : 0);
  if (n) {
    cudaMemcpyKind k = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (out->x) CK(cudaMemcpyAsync(out->x, B.x, n * sizeof(float), k, s->stream));
    if (out->v) CK(cudaMemcpyAsync(out->v, B.v, n * sizeof(float), k, s->stream));
    if (out->lane) CK(cudaMemcpyAsync(out->lane, B.lane, n * sizeof(int), k, s->stream));
    if (out->id) CK(cudaMemcpyAsync(out->id, B.id, n * sizeof(int), k, s->stream));
    if (device && out->route_idx) {
      k_route_idx<<<std::min(1024, (n + 255) / 256), 256, 0, s->stream>>>(B.rp, B.id, s->d_route0,
                                                                           out->route_idx, nullptr, n);
      CK(cudaGetLastError());
    }
    if (need_ids) CK(cudaMemcpyAsync(ids.data(), B.id, n * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    if (host_ridx) CK(cudaMemcpyAsync(rp.data(), B.rp, n * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  }
  std::vector<int> tarr(out->t_arr || out->trip_status ? s->n_trips : 0);
  if (out->t_arr || out->trip_status)
    CK(cudaMemcpyAsync(tarr.data(), s->d_tarr, s->n_trips * sizeof(int), cudaMemcpyDeviceToHost, s->stream));
  std::vector<int4> mp(out->ctrl_state ? s->n_ctrl : 0);
  if (!mp.empty())
    CK(cudaMemcpyAsync(mp.data(), s->d_mp, mp.size() * sizeof(int4), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  for (size_t k = 0; k < mp.size(); ++k) {   // host memory in either mode
    out->ctrl_state[3 * k] = mp[k].x;
    out->ctrl_state[3 * k + 1] = mp[k].y;
    out->ctrl_state[3 * k + 2] = mp[k].z;
  }
  if (host_ridx)
    for (int i = 0; i < n; ++i) out->route_idx[i] = rp[i] - s->h_route0[ids[i]];
  if (out->t_arr) std::memcpy(out->t_arr, tarr.data(), s->n_trips * sizeof(int));
  if (out->trip_status) {
    for (int i = 0; i < s->n_trips; ++i) out->trip_status[i] = tarr[i] >= 0 ? 2 : 0;
    for (int i = 0; i < n; ++i) out->trip_status[ids[i]] = 1;
  }
  return MS_OK;
}

int ms_read_state_async(void *sim, const ms_state *out) {
  Sim *s = (Sim *)sim;
  if (!s || !out || out->capacity < 0) return MS_ERR_ARG;
  if (!s->veh_loaded) return fail(s, MS_ERR_STATE, "no vehicles");
  void *ptrs[4] = {out->x, out->v, out->lane, out->id};
  for (void *q : ptrs) {
    if (!q) continue;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, q) != cudaSuccess || at.type != cudaMemoryTypeHost) {
      cudaGetLastError();
      return fail(s, MS_ERR_ARG, "ms_read_state_async needs pinned host buffers (cudaHostAlloc / pinned tensors)");
    }
  }
  if (s->ex_count == Sim::MS_EXPORTS)
    return fail(s, MS_ERR_STATE, "exports in flight at the limit: call ms_read_wait first");
  const int k = (s->ex_head + s->ex_count) % Sim::MS_EXPORTS;
  // the steps enqueued so far are waited for (not the exports in flight); the copies then
  // run on the copy engine, queued behind any export in flight, while the next steps compute
  int *meta = s->h_meta + 2 * k;
  k_export_meta<<<1, 1, 0, s->stream>>>(s->d_ctrl, (int)s->t_host, meta);
  CK(cudaGetLastError());
  CK(cudaEventRecord(s->ev_ready, s->stream));
  CK(cudaEventSynchronize(s->ev_ready));
  const int p = (int)(s->t_host & 1);
  const size_t m = (size_t)std::min(meta[0], out->capacity);
  const Soa &S = s->A[p];
  if (m > 0) {
    if (out->x) CK(cudaMemcpyAsync(out->x, S.x, m * sizeof(float), cudaMemcpyDeviceToHost, s->xs));
    if (out->v) CK(cudaMemcpyAsync(out->v, S.v, m * sizeof(float), cudaMemcpyDeviceToHost, s->xs));
    if (out->lane) CK(cudaMemcpyAsync(out->lane, S.lane, m * sizeof(int), cudaMemcpyDeviceToHost, s->xs));
    if (out->id) CK(cudaMemcpyAsync(out->id, S.id, m * sizeof(int), cudaMemcpyDeviceToHost, s->xs));
  }
  CK(cudaEventRecord(s->ev_export[k], s->xs));
  s->export_t[k] = s->t_host;
  s->export_cap[k] = out->capacity;
  ++s->ex_count;
  return MS_OK;
}

int ms_read_wait(void *sim, int *n_active, int *t) {
  Sim *s = (Sim *)sim;
  if (!s) return MS_ERR_ARG;
  if (s->ex_count == 0) return fail(s, MS_ERR_STATE, "no export in flight");
  const int k = s->ex_head;
  CK(cudaEventSynchronize(s->ev_export[k]));
  s->ex_head = (k + 1) % Sim::MS_EXPORTS;
  --s->ex_count;
  const int n = s->h_meta[2 * k];
  if (n_active) *n_active = n;
  if (t) *t = s->h_meta[2 * k + 1];
  if (n > s->export_cap[k]) return fail(s, MS_ERR_CAPACITY, "state capacity too small");
  return MS_OK;
}

int ms_write_state(void *sim, const ms_state *in) {
  Sim *s = (Sim *)sim;
  if (!s || !in) return MS_ERR_ARG;
  if (!s->veh_loaded) return fail(s, MS_ERR_STATE, "add vehicles first");
  const int n = in->n_active;
  if (n < 0 || in->t < 0 || (n > 0 && (!in->id || !in->lane || !in->x || !in->v || !in->route_idx)) || !in->t_arr)
    return fail(s, MS_ERR_ARG, "state arrays missing");
  CK(cudaStreamSynchronize(s->stream));
  if (int r0 = export_drain(s)) return r0;
  std::vector<int> ids(in->id, in->id + n), lanes(in->lane, in->lane + n), ridx(in->route_idx, in->route_idx + n);
  std::vector<float> xs(in->x, in->x + n), vs(in->v, in->v + n);
  for (int i = 1; i < n; ++i)
    if (lanes[i - 1] == lanes[i] && xs[i - 1] == xs[i] && ids[i - 1] > ids[i])
      return fail(s, MS_ERR_ARG, "vehicles not sorted by (lane, x, id)");
  std::vector<char> active(s->n_trips, 0);
  for (int i = 0; i < n; ++i)
    if (ids[i] >= 0 && ids[i] < s->n_trips) active[ids[i]] = 1;
  for (int i = 0; i < s->n_trips; ++i)
    if (active[i] && in->t_arr[i] >= 0) return fail(s, MS_ERR_ARG, "trip both active and arrived");
  int r = upload_state(s, ids, lanes, xs, vs, ridx, in->t, in->ctrl_state);
  if (r) return r;
  // queue heads: first waiting trip of each FIFO
  std::vector<int> qhead(s->n_lanes);
  for (int l = 0; l < s->n_lanes; ++l) {
    int q = s->h_qoff[l];
    while (q < s->h_qoff[l + 1] && (active[s->h_qtrip[q]] || in->t_arr[s->h_qtrip[q]] >= 0)) ++q;
    qhead[l] = q;
  }
  {
    int rq = upload_queues(s, qhead);
    if (rq) return rq;
  }
  CK(cudaMemcpy(s->d_tarr, in->t_arr, sizeof(int) * s->n_trips, cudaMemcpyHostToDevice));
  return MS_OK;
}

int ms_read_metrics(void *sim, ms_metrics *out) {
  Sim *s = (Sim *)sim;
  if (!s || !out) return MS_ERR_ARG;
  if (!s->veh_loaded) return fail(s, MS_ERR_STATE, "no vehicles");
  CK(cudaStreamSynchronize(s->stream));
  DevCtrl c;
  CK(cudaMemcpy(&c, s->d_ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost));
  size_t m = (size_t)s->prm.n_windows * s->n_lanes;
  if (out->lane_vsum && m) {   // exact integer sums in units of 2^-24 m/s
    std::vector<unsigned long long> q(m);
    CK(cudaMemcpy(q.data(), s->d_vsum, m * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < m; ++k) out->lane_vsum[k] = (float)std::ldexp((double)q[k], -24);
  }
  if (out->lane_vcnt && m) CK(cudaMemcpy(out->lane_vcnt, s->d_vcnt, m * sizeof(int), cudaMemcpyDeviceToHost));
  out->inserted = (int64_t)c.inserted;
  out->arrived = (int64_t)c.arrived;
  out->sum_travel_time = (int64_t)c.sum_tt;
  out->n_active = c.n_active[c.t & 1];
  out->t = c.t;
  out->movers_last_step = c.movers_last;
  out->err = c.err;
  return MS_OK;
}

int ms_read_debug(void *sim, ms_debug *out) {
  Sim *s = (Sim *)sim;
  if (!s || !out) return MS_ERR_ARG;
  if (!s->prm.debug || !s->veh_loaded) return fail(s, MS_ERR_STATE, "debug recording is off");
  CK(cudaStreamSynchronize(s->stream));
  DevCtrl c;
  CK(cudaMemcpy(&c, s->d_ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost));
  if (c.t == 0) return fail(s, MS_ERR_STATE, "no step taken");
  const int n = c.n_active[(c.t - 1) & 1];
  const DebugOut &d = s->dbg;
  std::vector<int> id(n), ik(n);
  std::vector<float> fk(n);
  if (n) CK(cudaMemcpy(id.data(), d.id, n * sizeof(int), cudaMemcpyDeviceToHost));
  auto scat_i = [&](int *dst, const int *src) -> int {
    if (!dst || !n) return MS_OK;
    CK(cudaMemcpy(ik.data(), src, n * sizeof(int), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) dst[id[i]] = ik[i];
    return MS_OK;
  };
  auto scat_f = [&](float *dst, const float *src) -> int {
    if (!dst || !n) return MS_OK;
    CK(cudaMemcpy(fk.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i) dst[id[i]] = fk[i];
    return MS_OK;
  };
  int r = 0;
  if (out->active_before) for (int i = 0; i < n; ++i) out->active_before[id[i]] = 1;
  if ((r = scat_i(out->lead_kind, d.lead_kind)) || (r = scat_i(out->lead_id, d.lead_id)) ||
      (r = scat_i(out->lc_dir, d.lc_dir)) || (r = scat_i(out->lc_cand, d.lc_cand)) ||
      (r = scat_i(out->tau_lead, d.tau_lead)) || (r = scat_i(out->tau_foll, d.tau_foll)) ||
      (r = scat_i(out->old_foll, d.old_foll)) || (r = scat_i(out->flag, d.flag)) ||
      (r = scat_f(out->s_own, d.s_own)) || (r = scat_f(out->vl_own, d.vl_own)) ||
      (r = scat_f(out->a_own, d.a_own)) || (r = scat_f(out->incentive, d.incentive)) ||
      (r = scat_f(out->a_use, d.a_use)) || (r = scat_i(out->lc_learn, d.lc_learn)) ||
      (r = scat_f(out->lc_margin, d.lc_margin)))
    return r;
  // per-vehicle vectors of the learned decision: logits (3) and inputs (16)
  auto scat_v = [&](float *dst, const float *src, int w) -> int {
    if (!dst || !n) return MS_OK;
    std::vector<float> buf((size_t)w * n);
    CK(cudaMemcpy(buf.data(), src, buf.size() * sizeof(float), cudaMemcpyDeviceToHost));
    for (int i = 0; i < n; ++i)
      for (int q = 0; q < w; ++q) dst[(size_t)id[i] * w + q] = buf[(size_t)i * w + q];
    return MS_OK;
  };
  if ((r = scat_v(out->lc_logit, d.lc_logit, 3)) || (r = scat_v(out->lc_feat, d.lc_feat, MLP_IN))) return r;
  std::vector<int> stamp(s->n_trips);
  if (out->inserted) {
    CK(cudaMemcpy(stamp.data(), d.trip_ins, s->n_trips * sizeof(int), cudaMemcpyDeviceToHost));
    for (int i = 0; i < s->n_trips; ++i) out->inserted[i] = stamp[i] == c.t ? 1 : 0;
  }
  if (out->flag) {
    CK(cudaMemcpy(stamp.data(), d.trip_flag, s->n_trips * sizeof(int), cudaMemcpyDeviceToHost));
    for (int i = 0; i < s->n_trips; ++i)
      if (stamp[i] == c.t) out->flag[i] = 1;
  }
  return MS_OK;
}

// ---------------------------------------------------------------------------------
// batches of independent scenarios
// ---------------------------------------------------------------------------------

int ms_load_network_batch(void *sim, int n, const ms_network *nets) {
  Sim *s = (Sim *)sim;
  if (!s || !nets || n <= 0) return MS_ERR_ARG;
  if (s->net_loaded) return fail(s, MS_ERR_STATE, "network already loaded");
  long long L64 = 0, E64 = 0, C64 = 0, S64 = 0;
  for (int k = 0; k < n; ++k) {
    const ms_network &q = nets[k];
    if (q.n_lanes <= 0 || q.n_edges <= 0 || q.n_ctrl < 0 || !q.succ_off)
      return fail(s, MS_ERR_ARG, "scenario " + std::to_string(k) + ": empty or missing network");
    L64 += q.n_lanes;
    E64 += q.n_edges;
    C64 += q.n_ctrl;
    S64 += q.succ_off[q.n_lanes];
  }
  if (L64 > CODE_LANE_MASK || E64 > INT_MAX || C64 > INT_MAX || S64 > INT_MAX)
    return fail(s, MS_ERR_CAPACITY, "the union of the scenarios has too many lanes, edges or links");
  const int L = (int)L64, E = (int)E64, C = (int)C64, S = (int)S64;
  std::vector<float> len(L);
  std::vector<int> edge(L), idx(L), left(L), right(L), soff(L + 1), sl(std::max(1, S)), se(std::max(1, S)),
      lctrl(L), lgrp(L), coff(std::max(1, C)), cg(std::max(1, C)), cy(std::max(1, C)), cp(std::max(1, C)),
      enl(E), el0(E);
  s->batch_lane_off.assign(1, 0);
  int lo = 0, eo = 0, co = 0, so = 0;
  auto shift = [](int v, int o) { return v >= 0 ? v + o : v; };
  for (int k = 0; k < n; ++k) {
    const ms_network &q = nets[k];
    for (int l = 0; l < q.n_lanes; ++l) {
      len[lo + l] = q.lane_len[l];
      edge[lo + l] = shift(q.lane_edge[l], eo);
      idx[lo + l] = q.lane_index[l];
      left[lo + l] = shift(q.lane_left[l], lo);
      right[lo + l] = shift(q.lane_right[l], lo);
      soff[lo + l] = q.succ_off[l] + so;
      lctrl[lo + l] = shift(q.lane_ctrl[l], co);
      lgrp[lo + l] = q.lane_group[l];
    }
    const int qs = q.succ_off[q.n_lanes];
    for (int j = 0; j < qs; ++j) {
      sl[so + j] = q.succ_lane[j] + lo;
      se[so + j] = q.succ_edge[j] + eo;
    }
    for (int c = 0; c < q.n_ctrl; ++c) {
      coff[co + c] = q.ctrl_offset[c];
      cg[co + c] = q.ctrl_green[c];
      cy[co + c] = q.ctrl_yellow[c];
      cp[co + c] = q.ctrl_nphase[c];
    }
    for (int e = 0; e < q.n_edges; ++e) {
      enl[eo + e] = q.edge_nlanes[e];
      el0[eo + e] = q.edge_lane0[e] + lo;
    }
    lo += q.n_lanes;
    eo += q.n_edges;
    co += q.n_ctrl;
    so += qs;
    s->batch_lane_off.push_back(lo);
  }
  soff[L] = so;
  ms_network u{L, E, C, len.data(), edge.data(), idx.data(), left.data(), right.data(), soff.data(), sl.data(),
               se.data(), lctrl.data(), lgrp.data(), coff.data(), cg.data(), cy.data(), cp.data(), enl.data(),
               el0.data()};
  int r = ms_load_network(sim, &u);
  if (r) s->batch_lane_off.clear();
  return r;
}

int ms_add_vehicles_batch(void *sim, int n, const ms_vehicles *vehs) {
  Sim *s = (Sim *)sim;
  if (!s || !vehs || n <= 0) return MS_ERR_ARG;
  if ((int)s->batch_lane_off.size() != n + 1) return fail(s, MS_ERR_STATE, "load the batch's networks first (same n)");
  // edge offsets of the scenarios, from the union's edge -> lane table
  std::vector<int> edge_off(n + 1, 0);
  {
    int k = 0;
    for (int e = 0; e < s->n_edges; ++e) {
      while (k < n && s->edge_lane0[e] >= s->batch_lane_off[k + 1]) edge_off[++k] = e;
    }
    for (int q = k + 1; q <= n; ++q) edge_off[q] = s->n_edges;
  }
  int T = 0;
  int64_t R = 0;
  bool any_place = false;
  for (int k = 0; k < n; ++k) {
    if (vehs[k].n < 0 || (vehs[k].n > 0 && (!vehs[k].route_off || !vehs[k].route_edges || !vehs[k].t_dep || !vehs[k].v0)))
      return fail(s, MS_ERR_ARG, "scenario " + std::to_string(k) + ": vehicle arrays missing");
    T += vehs[k].n;
    if (vehs[k].n) R += vehs[k].route_off[vehs[k].n];
    any_place |= vehs[k].lane != nullptr;
  }
  std::vector<int> tdep(T), rte((size_t)std::max<int64_t>(1, R)), lane(T, -1);
  std::vector<float> v0(T), x(T, 0.f), v(T, 0.f);
  std::vector<int64_t> roff(T + 1, 0);
  s->batch_trip_off.assign(1, 0);
  int to = 0;
  int64_t ro = 0;
  for (int k = 0; k < n; ++k) {
    const ms_vehicles &q = vehs[k];
    const int lo = s->batch_lane_off[k], eo = edge_off[k];
    const int ne = edge_off[k + 1] - eo;
    for (int i = 0; i < q.n; ++i) {
      tdep[to + i] = q.t_dep[i];
      v0[to + i] = q.v0[i];
      roff[to + i] = ro + q.route_off[i];
      if (q.lane && q.lane[i] >= 0) {
        lane[to + i] = q.lane[i] + lo;
        x[to + i] = q.x[i];
        v[to + i] = q.v[i];
      }
    }
    const int64_t qr = q.n ? q.route_off[q.n] : 0;
    for (int64_t j = 0; j < qr; ++j) {
      const int e = q.route_edges[j];
      if (e < 0 || e >= ne) return fail(s, MS_ERR_ARG, "scenario " + std::to_string(k) + ": route edge out of range");
      rte[ro + j] = e + eo;
    }
    to += q.n;
    ro += qr;
    s->batch_trip_off.push_back(to);
  }
  roff[T] = ro;
  ms_vehicles u{T, tdep.data(), v0.data(), roff.data(), rte.data(), any_place ? lane.data() : nullptr,
                any_place ? x.data() : nullptr, any_place ? v.data() : nullptr};
  int r = ms_add_vehicles(sim, &u);
  if (r) s->batch_trip_off.clear();
  return r;
}

int ms_batch_offsets(void *sim, int *lane_off, int *trip_off) {
  Sim *s = (Sim *)sim;
  if (!s) return MS_ERR_ARG;
  if (s->batch_lane_off.empty()) return fail(s, MS_ERR_STATE, "not a batch");
  if (lane_off) std::copy(s->batch_lane_off.begin(), s->batch_lane_off.end(), lane_off);
  if (trip_off) std::copy(s->batch_trip_off.begin(), s->batch_trip_off.end(), trip_off);
  return MS_OK;
}

// ---------------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------------

namespace {
// device-to-device snapshot of everything a step reads or writes
struct Snapshot {
  std::vector<std::pair<void *, size_t>> regions;
  std::vector<void *> copies;
};

int snap_take(Sim *s, Snapshot &sn) {
  const size_t N = s->n_trips, L = s->n_lanes, W = (size_t)s->prm.n_windows * L;
  auto add = [&](void *p, size_t bytes) { if (p && bytes) sn.regions.push_back({p, bytes}); };
  for (int b = 0; b < 2; ++b) {
    add(s->A[b].x, N * 4); add(s->A[b].v, N * 4); add(s->A[b].v0, N * 4); add(s->A[b].lane, N * 4);
    add(s->A[b].rp, N * 4); add(s->A[b].pl, N * 8); add(s->A[b].nl, N * 4); add(s->A[b].id, N * 4);
    add(s->d_dyn[b], L * sizeof(int4));
  }
  add(s->d_ctrl, sizeof(DevCtrl));
  add(s->d_qhd, L * 8);
  add(s->d_sig[0], s->h_ctrl4.size() * 4);
  add(s->d_mp, s->h_ctrl4.size() * 16);
  add(s->d_sig[1], s->h_ctrl4.size() * 4);
  add(s->d_tarr, N * 4);
  add(s->d_vsum, W * 8);
  add(s->d_vcnt, W * 4);
  for (auto &r : sn.regions) {
    void *c = nullptr;
    cudaError_t e = cudaMalloc(&c, r.second);
    if (e != cudaSuccess) return fail(s, MS_ERR_CUDA, std::string("autotune snapshot: ") + cudaGetErrorString(e));
    sn.copies.push_back(c);
    CK(cudaMemcpyAsync(c, r.first, r.second, cudaMemcpyDeviceToDevice, s->stream));
  }
  return MS_OK;
}

int snap_restore(Sim *s, Snapshot &sn) {
  for (size_t k = 0; k < sn.regions.size(); ++k)
    CK(cudaMemcpyAsync(sn.regions[k].first, sn.copies[k], sn.regions[k].second, cudaMemcpyDeviceToDevice, s->stream));
  return MS_OK;
}

void snap_free(Snapshot &sn) {
  for (void *c : sn.copies) cudaFree(c);
  sn.copies.clear();
}
}  // namespace

int ms_autotune(void *sim, int trial_steps, float *best_ms, int *config) {
  Sim *s = (Sim *)sim;
  if (!s || trial_steps <= 0) return MS_ERR_ARG;
  if (!s->veh_loaded) return fail(s, MS_ERR_STATE, "add vehicles first");
  CK(cudaStreamSynchronize(s->stream));
  if (int r0 = export_drain(s)) return r0;
  Snapshot sn;
  int r = snap_take(s, sn);
  if (r) { snap_free(sn); return r; }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  StepArgs a = make_args(s);
  LaunchCfg best = s->cfg;
  float best_t = 3.4e38f;
  // one candidate: a warm-up step of its shape, then trial_steps timed steps; the state is
  // restored afterwards, so the simulation's results do not depend on the search
  auto trial = [&](const LaunchCfg &c) -> int {
    s->cfg = c;
    CK(launch_step(s, a, s->stream, nullptr));
    CK(cudaEventRecord(e0, s->stream));
    for (int k = 0; k < trial_steps; ++k) CK(launch_step(s, a, s->stream, nullptr));
    CK(cudaEventRecord(e1, s->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    ms /= trial_steps;
    if (int rr = snap_restore(s, sn)) return rr;
    if (ms < best_t) {
      best_t = ms;
      best = c;
    }
    return MS_OK;
  };
  // coordinate search: (threads per block of the vehicle kernels, grid factors of decide and
  // apply), then the lane scan's tile shape, then k_bucket's block and grid factor
  const int blocks[] = {128, 256, 512};
  const int factors[] = {1, 2, 4};
  for (int blk : blocks)
    for (int fd : factors)
      for (int fa : factors) {
        LaunchCfg c = s->cfg;
        c.blk_decide = c.blk_apply = blk;
        c.blk_bucket = 256;
        c.lane_threads = LANE_THREADS;
        if ((r = shape_grids(s, c, fd, fa, 1)) || (r = trial(c))) { snap_free(sn); return r; }
      }
  const LaunchCfg stage1 = best;
  for (int th : {128, 512}) {
    LaunchCfg c = stage1;
    c.lane_threads = th;
    if ((r = trial(c))) { snap_free(sn); return r; }
  }
  const LaunchCfg stage2 = best;
  for (int bb : blocks)
    for (int fb : {1, 2}) {
      if (bb == stage2.blk_bucket && fb == stage2.f_bucket) continue;
      LaunchCfg c = stage2;
      c.blk_bucket = bb;
      if ((r = shape_grids(s, c, c.f_decide, c.f_apply, fb)) || (r = trial(c))) { snap_free(sn); return r; }
    }
  CK(cudaStreamSynchronize(s->stream));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  snap_free(sn);
  s->cfg = best;
  drop_graphs(s);   // rebuilt with the chosen shapes on the next ms_step
  if (best_ms) *best_ms = best_t;
  if (config) {
    const int out[6] = {best.blk_decide, best.f_decide, best.f_apply, best.lane_threads, best.blk_bucket,
                        best.f_bucket};
    std::copy(out, out + 6, config);
  }
  return MS_OK;
}

// ---------------------------------------------------------------------------------
// learned lane change
// ---------------------------------------------------------------------------------

int ms_set_lc_log(void *sim, void *x, int *y, int cap, int *n) {
  Sim *s = (Sim *)sim;
  if (!s) return MS_ERR_ARG;
  if (x && (!y || !n || cap <= 0)) return fail(s, MS_ERR_ARG, "log needs x, y, n and cap > 0");
  s->lc.log_x = (__nv_bfloat16 *)x;
  s->lc.log_y = y;
  s->lc.log_cap = cap;
  s->lc.log_n = n;
  s->lc_mode = x ? MODE_LOG : (s->d_model && s->lc.model ? MODE_LEARN : MODE_PLAIN);
  drop_graphs(s);
  if (s->veh_loaded) return shape_grids(s, s->cfg, s->cfg.f_decide, s->cfg.f_apply, s->cfg.f_bucket);
  return MS_OK;
}

// ---- route planner (demand generation) ------------------------------------------------

int build_route_graph(Sim *s) {
  if (s->d_rg_off) return MS_OK;
  const int E = s->n_edges;
  std::vector<int> off(E + 1, 0), dst;
  std::vector<long long> cost(E);
  for (int e = 0; e < E; ++e) {
    std::vector<int> outs;
    for (int q = 0; q < s->edge_nlanes[e]; ++q) {
      const int l = s->edge_lane0[e] + q;
      for (int k = s->succ_off[l]; k < s->succ_off[l + 1]; ++k) outs.push_back(s->succ_edge[k]);
    }
    std::sort(outs.begin(), outs.end());
    outs.erase(std::unique(outs.begin(), outs.end()), outs.end());
    dst.insert(dst.end(), outs.begin(), outs.end());
    off[e + 1] = (int)dst.size();
    cost[e] = std::llrint((double)s->lane_len[s->edge_lane0[e]] * 1000.0);   // mm, ties to even
  }
  if (dst.empty()) dst.push_back(0);
  DALLOC(s->d_rg_off, off.size());
  DALLOC(s->d_rg_dst, dst.size());
  DALLOC(s->d_rg_cost, cost.size());
  CK(cudaMemcpy(s->d_rg_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_rg_dst, dst.data(), dst.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_rg_cost, cost.data(), cost.size() * sizeof(long long), cudaMemcpyHostToDevice));
  return MS_OK;
}

// least route costs toward nb destination edges (device array dd), in columns of d[E * B]:
// pull sweeps until a round of 16 changes nothing (at most E sweeps, Bellman-Ford)
cudaError_t route_distances(Sim *s, const RouteGraph &g, const int *dd, int nb, int B, long long *d, int *flag,
                            bool &converged) {
  cudaStream_t st = s->stream;
  const long long EB = (long long)g.E * B;
  const int blocks = (int)((EB + 255) / 256);
  k_route_init<<<blocks, 256, 0, st>>>(d, g.E, B, dd, nb);
  cudaError_t e = cudaGetLastError();
  converged = false;
  for (int sweeps = 0; e == cudaSuccess && sweeps <= g.E + 16; sweeps += 16) {
    int h = 0;
    e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    for (int k = 0; k < 16 && e == cudaSuccess; ++k) {
      k_route_relax<<<blocks, 256, 0, st>>>(d, g, B, flag);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && !h) {
      converged = true;
      break;
    }
  }
  return e;
}

int ms_route_trips(void *sim, int n, const int *orig_edge, const int *dest_edge, int64_t *route_off,
                   int *route_edges, int64_t edges_capacity, int *n_unreachable) {
  Sim *s = (Sim *)sim;
  if (!s || n < 0 || (n > 0 && (!orig_edge || !dest_edge)) || !route_off) return MS_ERR_ARG;
  if (!s->net_loaded) return fail(s, MS_ERR_STATE, "load the network first");
  const int E = s->n_edges;
  for (int i = 0; i < n; ++i)
    if (orig_edge[i] < 0 || orig_edge[i] >= E || dest_edge[i] < 0 || dest_edge[i] >= E)
      return fail(s, MS_ERR_ARG, "trip edge out of range");
  {
    int r = build_route_graph(s);
    if (r) return r;
  }
  const RouteGraph g{s->d_rg_off, s->d_rg_dst, s->d_rg_cost, E};
  cudaStream_t st = s->stream;
  // trips grouped by destination; destinations in batches of B columns (multiple of 32)
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dest_edge[a] < dest_edge[b]; });
  std::vector<int> dests;
  for (int k = 0; k < n; ++k)
    if (k == 0 || dest_edge[order[k]] != dest_edge[order[k - 1]]) dests.push_back(dest_edge[order[k]]);
  const size_t budget = size_t(2) << 30;   // bytes of distances per batch
  const int bmax = (int)std::max<size_t>(32, std::min<size_t>(4096, budget / (8 * (size_t)E)) / 32 * 32);
  const int B = std::min(bmax, std::max(32, ((int)dests.size() + 31) / 32 * 32));
  long long *d = nullptr;
  int *dd = nullptr, *flag = nullptr, *dlen = nullptr, *dout = nullptr;
  int4 *dtr = nullptr;
  long long *doff = nullptr;
  auto release = [&]() {
    cudaFree(d); cudaFree(dd); cudaFree(flag); cudaFree(dlen); cudaFree(dout); cudaFree(dtr); cudaFree(doff);
  };
#define RCK(x)                                                                                   \
  do {                                                                                           \
    cudaError_t e_ = (x);                                                                        \
    if (e_ != cudaSuccess) {                                                                     \
      release();                                                                                 \
      return fail(s, MS_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e_));                \
    }                                                                                            \
  } while (0)
  RCK(cudaMalloc(&d, sizeof(long long) * (size_t)B * E));
  RCK(cudaMalloc(&dd, sizeof(int) * B));
  RCK(cudaMalloc(&flag, sizeof(int) * 2));
  RCK(cudaMalloc(&dlen, sizeof(int) * std::max(1, n)));
  RCK(cudaMalloc(&dtr, sizeof(int4) * std::max(1, n)));
  RCK(cudaMalloc(&doff, sizeof(long long) * (std::max(1, n) + 1)));
  std::vector<int> len(n, 0);
  std::vector<std::vector<int>> batch_edges;   // routes of each batch, in batch trip order
  std::vector<std::pair<int, long long>> where(n, {-1, 0});   // trip -> (batch, offset)
  int herr = 0;
  size_t k0 = 0;   // first trip (in `order`) of the batch
  for (size_t b0 = 0; b0 < dests.size(); b0 += B) {
    const int nb = (int)std::min<size_t>(B, dests.size() - b0);
    RCK(cudaMemcpyAsync(dd, dests.data() + b0, sizeof(int) * nb, cudaMemcpyHostToDevice, st));
    bool conv = false;
    RCK(route_distances(s, g, dd, nb, B, d, flag, conv));
    if (!conv) {
      release();
      return fail(s, MS_ERR_CUDA, "route distances did not converge");
    }
    // this batch's trips
    std::vector<int4> tr;
    size_t k1 = k0;
    while (k1 < (size_t)n && dest_edge[order[k1]] <= dests[b0 + nb - 1]) {
      const int i = order[k1];
      const int col = (int)(std::lower_bound(dests.begin() + b0, dests.begin() + b0 + nb, dest_edge[i]) -
                            (dests.begin() + b0));
      tr.push_back(make_int4(i, orig_edge[i], dest_edge[i], col));
      ++k1;
    }
    k0 = k1;
    const int nt = (int)tr.size();
    if (nt == 0) continue;
    RCK(cudaMemcpyAsync(dtr, tr.data(), sizeof(int4) * nt, cudaMemcpyHostToDevice, st));
    RCK(cudaMemsetAsync(flag + 1, 0, sizeof(int), st));
    k_route_walk<<<(nt + 255) / 256, 256, 0, st>>>(d, g, B, dtr, nt, nullptr, dlen, nullptr, E, flag + 1);
    std::vector<int> bl(nt);
    RCK(cudaMemcpyAsync(bl.data(), dlen, sizeof(int) * nt, cudaMemcpyDeviceToHost, st));
    RCK(cudaStreamSynchronize(st));
    std::vector<long long> bo(nt + 1, 0);
    for (int j = 0; j < nt; ++j) bo[j + 1] = bo[j] + bl[j];
    batch_edges.emplace_back(std::max<long long>(1, bo[nt]));
    RCK(cudaFree(dout));
    dout = nullptr;
    RCK(cudaMalloc(&dout, sizeof(int) * std::max<long long>(1, bo[nt])));
    RCK(cudaMemcpyAsync(doff, bo.data(), sizeof(long long) * (nt + 1), cudaMemcpyHostToDevice, st));
    k_route_walk<<<(nt + 255) / 256, 256, 0, st>>>(d, g, B, dtr, nt, doff, dlen, dout, E, flag + 1);
    RCK(cudaGetLastError());
    RCK(cudaMemcpyAsync(batch_edges.back().data(), dout, sizeof(int) * bo[nt], cudaMemcpyDeviceToHost, st));
    int e2 = 0;
    RCK(cudaMemcpyAsync(&e2, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    RCK(cudaStreamSynchronize(st));
    herr |= e2;
    for (int j = 0; j < nt; ++j) {
      len[tr[j].x] = bl[j];
      where[tr[j].x] = {(int)batch_edges.size() - 1, bo[j]};
    }
  }
  release();
#undef RCK
  if (herr) return fail(s, MS_ERR_CUDA, "route walk left a least-cost route (device check)");
  int bad = 0;
  route_off[0] = 0;
  for (int i = 0; i < n; ++i) {
    route_off[i + 1] = route_off[i] + len[i];
    bad += len[i] == 0;
  }
  if (n_unreachable) *n_unreachable = bad;
  if (!route_edges) return MS_OK;
  if (route_off[n] > edges_capacity)
    return fail(s, MS_ERR_CAPACITY, "route_edges needs " + std::to_string(route_off[n]) + " entries");
  for (int i = 0; i < n; ++i)
    if (len[i])
      std::memcpy(route_edges + route_off[i], batch_edges[where[i].first].data() + where[i].second,
                  sizeof(int) * len[i]);
  return MS_OK;
}

// OD sampling shared by the gravity (gamma 0..3) and radiation (gamma < 0) models
static int sample_trips(Sim *s, int n_zones, const int *zone_edge, const float *attract, int gamma, int n,
                        int t_span, uint64_t seed, int *orig_edge, int *dest_edge, int *t_dep) {
  if (!s || n_zones <= 0 || !zone_edge || !attract || n < 0 || (n > 0 && (!orig_edge || !dest_edge || !t_dep)))
    return MS_ERR_ARG;
  if (!s->net_loaded) return fail(s, MS_ERR_STATE, "load the network first");
  if (n_zones > 4096) return fail(s, MS_ERR_CAPACITY, "at most 4096 zones");
  if (gamma > 3 || t_span <= 0) return fail(s, MS_ERR_ARG, "gamma must be in 0..3 and t_span > 0");
  {
    std::vector<int> z(zone_edge, zone_edge + n_zones);
    std::sort(z.begin(), z.end());
    if (z.front() < 0 || z.back() >= s->n_edges) return fail(s, MS_ERR_ARG, "zone edge out of range");
    if (std::adjacent_find(z.begin(), z.end()) != z.end()) return fail(s, MS_ERR_ARG, "zone edges must differ");
    for (int k = 0; k < n_zones; ++k)
      if (!(attract[k] > 0.f) || !std::isfinite(attract[k])) return fail(s, MS_ERR_ARG, "attractions must be > 0");
  }
  {
    int r = build_route_graph(s);
    if (r) return r;
  }
  const RouteGraph g{s->d_rg_off, s->d_rg_dst, s->d_rg_cost, s->n_edges};
  cudaStream_t st = s->stream;
  const int B = (n_zones + 31) / 32 * 32;
  long long *d = nullptr;
  int *dz = nullptr, *flag = nullptr, *dout = nullptr;
  float *da = nullptr, *cdf_d = nullptr, *cdf_o = nullptr;
  auto release = [&]() {
    cudaFree(d); cudaFree(dz); cudaFree(flag); cudaFree(dout); cudaFree(da); cudaFree(cdf_d); cudaFree(cdf_o);
  };
#define RCK(x)                                                                                   \
  do {                                                                                           \
    cudaError_t e_ = (x);                                                                        \
    if (e_ != cudaSuccess) {                                                                     \
      release();                                                                                 \
      return fail(s, MS_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e_));                \
    }                                                                                            \
  } while (0)
  RCK(cudaMalloc(&d, sizeof(long long) * (size_t)B * s->n_edges));
  RCK(cudaMalloc(&dz, sizeof(int) * n_zones));
  RCK(cudaMalloc(&flag, sizeof(int)));
  RCK(cudaMalloc(&da, sizeof(float) * n_zones));
  RCK(cudaMalloc(&cdf_d, sizeof(float) * (size_t)n_zones * n_zones));
  RCK(cudaMalloc(&cdf_o, sizeof(float) * n_zones));
  RCK(cudaMalloc(&dout, sizeof(int) * 3 * (size_t)std::max(1, n)));
  RCK(cudaMemcpyAsync(dz, zone_edge, sizeof(int) * n_zones, cudaMemcpyHostToDevice, st));
  RCK(cudaMemcpyAsync(da, attract, sizeof(float) * n_zones, cudaMemcpyHostToDevice, st));
  bool conv = false;
  RCK(route_distances(s, g, dz, n_zones, B, d, flag, conv));
  if (!conv) {
    release();
    return fail(s, MS_ERR_CUDA, "route distances did not converge");
  }
  if (gamma >= 0) {
    k_od_cdf<<<(n_zones + 127) / 128, 128, 0, st>>>(d, B, dz, da, n_zones, gamma, cdf_d, cdf_o);
    RCK(cudaGetLastError());
  } else {
    int P = 1;
    while (P < n_zones) P <<= 1;
    const size_t smem = 8 * (size_t)P + 8 * (size_t)n_zones;
    static bool attr = false;
    if (!attr) {
      RCK(cudaFuncSetAttribute(k_od_radiation_cdf, cudaFuncAttributeMaxDynamicSharedMemorySize, 8 * 4096 + 8 * 4096));
      attr = true;
    }
    RCK(cudaMemsetAsync(flag, 0, sizeof(int), st));
    k_od_radiation_cdf<<<n_zones, OD_RAD_THREADS, smem, st>>>(d, B, dz, da, n_zones, P, cdf_d, cdf_o, flag);
    RCK(cudaGetLastError());
    int far = 0;
    RCK(cudaMemcpyAsync(&far, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    RCK(cudaStreamSynchronize(st));
    if (far) {
      release();
      return fail(s, MS_ERR_CAPACITY, "a zone-to-zone route cost of 2^40 mm or more");
    }
  }
  if (n > 0) {
    k_od_sample<<<(n + 255) / 256, 256, 0, st>>>(cdf_d, cdf_o, dz, n_zones, n, t_span, seed, dout, dout + n,
                                                 dout + 2 * (size_t)n);
    RCK(cudaGetLastError());
    RCK(cudaMemcpyAsync(orig_edge, dout, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    RCK(cudaMemcpyAsync(dest_edge, dout + n, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    RCK(cudaMemcpyAsync(t_dep, dout + 2 * (size_t)n, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  }
  RCK(cudaStreamSynchronize(st));
  release();
#undef RCK
  return MS_OK;
}

int ms_sample_trips(void *sim, int n_zones, const int *zone_edge, const float *attract, int gamma, int n,
                    int t_span, uint64_t seed, int *orig_edge, int *dest_edge, int *t_dep) {
  Sim *s = (Sim *)sim;
  if (s && gamma < 0) return fail(s, MS_ERR_ARG, "gamma must be in 0..3 and t_span > 0");
  return sample_trips(s, n_zones, zone_edge, attract, gamma, n, t_span, seed, orig_edge, dest_edge, t_dep);
}

int ms_sample_trips_radiation(void *sim, int n_zones, const int *zone_edge, const float *population, int n,
                              int t_span, uint64_t seed, int *orig_edge, int *dest_edge, int *t_dep) {
  return sample_trips((Sim *)sim, n_zones, zone_edge, population, -1, n, t_span, seed, orig_edge, dest_edge,
                      t_dep);
}

int ms_set_lane_limits(void *sim, int n, const int *lanes, const float *vmax, const int *closed) {
  Sim *s = (Sim *)sim;
  if (!s || n < 0 || (n > 0 && !lanes)) return MS_ERR_ARG;
  if (!s->net_loaded) return fail(s, MS_ERR_STATE, "load the network first");
  for (int k = 0; k < n; ++k)
    if (lanes[k] < 0 || lanes[k] >= s->n_lanes) return fail(s, MS_ERR_ARG, "lane out of range");
  std::vector<int> flip;   // lanes whose closure changes
  for (int k = 0; k < n; ++k) {
    const int l = lanes[k];
    if (vmax) s->h_lane_vmax[l] = (vmax[k] > 0.f && std::isfinite(vmax[k])) ? vmax[k] : INFINITY;
    if (closed && s->h_lane_closed[l] != (closed[k] != 0)) {
      s->h_lane_closed[l] = closed[k] != 0;
      flip.push_back(l);
    }
  }
  if (!flip.empty() && s->veh_loaded) {
    // a closed lane's departure queue waits: its head is parked at INT_MAX (never due) and
    // gets its trip's departure step back when the lane reopens
    std::vector<int2> hd(s->n_lanes);
    CK(cudaStreamSynchronize(s->stream));
    CK(cudaMemcpy(hd.data(), s->d_qhd, sizeof(int2) * s->n_lanes, cudaMemcpyDeviceToHost));
    for (int l : flip)
      hd[l].y = s->h_lane_closed[l] || hd[l].x >= s->h_qoff[l + 1] ? 0x7fffffff : s->h_tdep[s->h_qtrip[hd[l].x]];
    CK(cudaMemcpy(s->d_qhd, hd.data(), sizeof(int2) * s->n_lanes, cudaMemcpyHostToDevice));
  }
  int mods = 0;
  for (int l = 0; l < s->n_lanes && !mods; ++l) mods = std::isfinite(s->h_lane_vmax[l]) || s->h_lane_closed[l];
  CK(cudaMemcpyAsync(s->d_lane_vmax, s->h_lane_vmax.data(), s->n_lanes * sizeof(float), cudaMemcpyHostToDevice,
                     s->stream));
  CK(cudaMemcpyAsync(s->d_lane_closed, s->h_lane_closed.data(), s->n_lanes, cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (mods != s->P.lane_mods) {   // the flag is baked into the captured step graphs
    s->P.lane_mods = mods;
    drop_graphs(s);
  }
  return MS_OK;
}

// an edge lane of edge e has an open link toward edge f (under the link states off)
static bool edge_links_to(const Sim *s, const std::vector<unsigned char> &off, int e, int f) {
  for (int q = 0; q < s->edge_nlanes[e]; ++q) {
    const int l = s->edge_lane0[e] + q;
    for (int k = s->succ_off[l]; k < s->succ_off[l + 1]; ++k)
      if (s->succ_edge[k] == f && !off[k]) return true;
  }
  return false;
}

int ms_set_lane_links(void *sim, int n, const int *lanes, const unsigned *open_mask) {
  Sim *s = (Sim *)sim;
  if (!s || n < 0 || (n > 0 && (!lanes || !open_mask))) return MS_ERR_ARG;
  if (!s->veh_loaded) return fail(s, MS_ERR_STATE, "add vehicles first");
  std::vector<unsigned char> off = s->link_off;
  for (int k = 0; k < n; ++k) {
    const int l = lanes[k];
    if (l < 0 || l >= s->n_lanes || s->lane_edge[l] < 0) return fail(s, MS_ERR_ARG, "not an edge lane");
    const int deg = s->succ_off[l + 1] - s->succ_off[l];
    if (deg > 32) return fail(s, MS_ERR_CAPACITY, "an edge lane with more than 32 links");
    for (int j = 0; j < deg; ++j) off[s->succ_off[l] + j] = !((open_mask[k] >> j) & 1u);
  }
  // edges whose lanes' links change: only route pairs leaving them can lose connectivity,
  // and only plan entries of them or leading into them (the fan-out tie looks at the
  // next edge's lanes) change
  std::vector<char> touched(s->n_edges, 0);
  bool any = false;
  for (int l = 0; l < s->n_lanes; ++l)
    if (s->lane_edge[l] >= 0)
      for (int k = s->succ_off[l]; k < s->succ_off[l + 1]; ++k)
        if (off[k] != s->link_off[k]) touched[s->lane_edge[l]] = any = true;
  if (!any) return MS_OK;
  // where each trip stands: arrived (t_arr >= 0), active (its current route entry), waiting
  CK(cudaStreamSynchronize(s->stream));
  if (int r0 = export_drain(s)) return r0;
  DevCtrl c;
  CK(cudaMemcpy(&c, s->d_ctrl, sizeof(DevCtrl), cudaMemcpyDeviceToHost));
  const int p = c.t & 1, na = c.n_active[p], N = s->n_trips;
  std::vector<int> rp(na), lane(na), id(na), tarr(N);
  const Soa &A = s->A[p];
  if (na) {
    CK(cudaMemcpy(rp.data(), A.rp, sizeof(int) * na, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(lane.data(), A.lane, sizeof(int) * na, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(id.data(), A.id, sizeof(int) * na, cudaMemcpyDeviceToHost));
  }
  CK(cudaMemcpy(tarr.data(), s->d_tarr, sizeof(int) * N, cudaMemcpyDeviceToHost));
  std::vector<long long> from(N);   // first routes[] index whose pair must stay connected
  for (int trip = 0; trip < N; ++trip) from[trip] = tarr[trip] >= 0 ? -1 : s->h_route0[trip];
  for (int i = 0; i < na; ++i) from[id[i]] = rp[i] + (s->lane_edge[lane[i]] < 0 ? 1 : 0);
  std::atomic<int> broken{-1};
  const int *R = s->h_routes.data();
  host_parallel((size_t)N, [&](size_t t0, size_t t1) {
    for (size_t trip = t0; trip < t1 && broken.load() < 0; ++trip) {
      if (from[trip] < 0) continue;
      for (long long k = from[trip]; R[k] >= 0 && R[k + 1] >= 0; ++k)
        if (touched[R[k]] && !edge_links_to(s, off, R[k], R[k + 1])) {
          broken.store((int)trip);
          break;
        }
    }
  });
  if (broken.load() >= 0) {
    const int trip = broken.load();
    long long k = from[trip];
    while (!(touched[R[k]] && !edge_links_to(s, off, R[k], R[k + 1]))) ++k;
    return fail(s, MS_ERR_ROUTE, "trip " + std::to_string(trip) + " would need edge " + std::to_string(R[k]) +
                                     " -> " + std::to_string(R[k + 1]) + " with no open lane link");
  }
  s->link_off = off;
  CK(cudaMemcpy(s->d_link_off, s->link_off.data(), s->link_off.size(), cudaMemcpyHostToDevice));
  const size_t nr = s->h_routes.size();
  host_parallel(nr, [&](size_t r0, size_t r1) {
    for (size_t r = r0; r < r1; ++r)
      if (R[r] >= 0 && (touched[R[r]] || (r + 1 < nr && R[r + 1] >= 0 && touched[R[r + 1]])))
        s->h_plan[r] = plan_word(s, r);
  });
  CK(cudaMemcpy(s->d_plan, s->h_plan.data(), sizeof(unsigned long long) * nr, cudaMemcpyHostToDevice));
  if (int r = upload_queue_entries(s)) return r;
  if (na) {
    k_refresh_choices<<<std::max(1, std::min(4 * s->n_sm, (na + 255) / 256)), 256, 0, s->stream>>>(make_args(s), A, na);
    CK(cudaGetLastError());
  }
  if (s->prm.signal_mode == 1 && s->n_ctrl > 0) {
    // the max-pressure decision of the current step is taken again over the links now open
    // (advancing the controllers to the step they are at again, as a state upload does)
    k_signals<<<(s->n_ctrl + 7) / 8, 256, 0, s->stream>>>(make_args(s));
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(s->stream));
  return MS_OK;
}

int ms_set_lc_model(void *sim, const float *params, float margin) {
  Sim *s = (Sim *)sim;
  if (!s) return MS_ERR_ARG;
  drop_graphs(s);
  if (!params) {
    s->lc.model = nullptr;
    s->lc_mode = s->lc.log_x ? MODE_LOG : MODE_PLAIN;
    if (s->veh_loaded) return shape_grids(s, s->cfg, s->cfg.f_decide, s->cfg.f_apply, s->cfg.f_bucket);
    return MS_OK;
  }
  if (!(margin >= 0.f && margin <= 1.f)) return fail(s, MS_ERR_ARG, "margin must be in [0, 1]");
  if (!s->d_model) {
    DALLOC(s->d_model, 1);
    DALLOC(s->d_lcstats, LC_STATS);
    DALLOC(s->d_theta, MLP_NPARAM);
    static bool attr = false;
    if (!attr) {
      for (int d = 0; d < 2; ++d)
        CK(cudaFuncSetAttribute(learn_kernel(d != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                learn_smem(LEARN_THREADS)));
      attr = true;
    }
  }
  // the candidate buffers first: without room for them nothing changes (the mode in effect,
  // a logging mode included, stays)
  const int prev_mode = s->lc_mode;
  const LcAux prev_lc = s->lc;
  s->lc_mode = MODE_LEARN;
  if (int r = ensure_cand(s)) {
    const std::string msg = s->err;
    s->lc_mode = prev_mode;
    s->lc = prev_lc;
    if (s->veh_loaded) shape_grids(s, s->cfg, s->cfg.f_decide, s->cfg.f_apply, s->cfg.f_bucket);
    return fail(s, r, msg + " (the previous lane-change mode stays)");
  }
  CK(cudaMemcpyAsync(s->d_theta, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, s->stream));
  k_mlp_pack<<<8, 256, 0, s->stream>>>(s->d_theta, s->d_model);
  CK(cudaGetLastError());
  CK(cudaMemsetAsync(s->d_lcstats, 0, sizeof(unsigned long long) * LC_STATS, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->lc.model = s->d_model;
  s->lc.margin = margin;
  s->lc.stats = s->d_lcstats;
  s->lc.log_x = nullptr;
  if (s->veh_loaded) return shape_grids(s, s->cfg, s->cfg.f_decide, s->cfg.f_apply, s->cfg.f_bucket);
  return MS_OK;
}

int ms_read_lc_stats(void *sim, int64_t *out12) {
  Sim *s = (Sim *)sim;
  if (!s || !out12) return MS_ERR_ARG;
  if (!s->d_lcstats) return fail(s, MS_ERR_STATE, "no model set");
  CK(cudaStreamSynchronize(s->stream));
  unsigned long long h[LC_STATS];
  CK(cudaMemcpy(h, s->d_lcstats, sizeof(h), cudaMemcpyDeviceToHost));
  for (int k = 0; k < LC_STATS; ++k) out12[k] = (int64_t)h[k];
  return MS_OK;
}

namespace {
// one gradient accumulation over the minibatch into work (gradient, then {weight sum, loss
// sum, error bits}); tc: the tcgen05 kernel (128 samples per CTA, packing its own operands
// from theta) instead of mma.sync (operands packed by k_mlp_pack)
int mlp_run(const void *x, const int *y, const int *idx, int batch, const float *theta, const float *class_w,
            float *work, cudaStream_t st, bool tc, bool withhold = false) {
  Sim *s = nullptr;
  static_assert(MLP_NPARAM == MS_MLP_NPARAM, "parameter count");
  static_assert(MLP_NPARAM + 4 + (int)(sizeof(MlpDev) / 4) <= MS_MLP_WORK_FLOATS, "work size");
  if (!x || !y || !idx || batch <= 0 || !theta || !class_w || !work) return MS_ERR_ARG;
  float *grad = work, *stats = work + MLP_NPARAM;
  MlpDev *model = reinterpret_cast<MlpDev *>(work + MLP_NPARAM + 4);
  static bool attr = false;
  if (!attr) {
    CK(cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, TR_SMEM));
    CK(cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    attr = true;
  }
  if (!tc) k_mlp_pack<<<8, 256, 0, st>>>(theta, model);
  CK(cudaMemsetAsync(work, 0, sizeof(float) * (MLP_NPARAM + 4), st));
  TrainArgs a{};
  a.X = (const __nv_bfloat16 *)x;
  a.y = y;
  a.idx = idx;
  a.batch = batch;
  a.model = model;
  a.cw[0] = class_w[0];
  a.cw[1] = class_w[1];
  a.cw[2] = class_w[2];
  a.grad = grad;
  a.stats = stats;
  a.err = reinterpret_cast<unsigned *>(stats + 2);
  a.theta = theta;
  a.withhold = withhold ? 1 : 0;
  if (tc)
    k_mlp_train_tc<<<(batch + TC_ROWS - 1) / TC_ROWS, TC_ROWS, TC_SMEM, st>>>(a);
  else
    k_mlp_train<<<(batch + TR_ROWS - 1) / TR_ROWS, TR_ROWS * 2, TR_SMEM, st>>>(a);
  CK(cudaGetLastError());
  return MS_OK;
}

int mlp_train_step(const void *x, const int *y, const int *idx, int batch, float *theta, float *m, float *v, int t,
                   float lr, const float *class_w, float *work, float *loss, void *cuda_stream, bool tc) {
  Sim *s = nullptr;
  if (!m || !v || t < 1) return MS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int r = mlp_run(x, y, idx, batch, theta, class_w, work, st, tc);
  if (r) return r;
  if (loss) {
    float h[3];
    CK(cudaMemcpyAsync(h, work + MLP_NPARAM, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    unsigned e;
    std::memcpy(&e, &h[2], sizeof(e));
    if (e) return MS_ERR_DEVICE;   // a tensor-core wait ran out: the gradient is incomplete
    *loss = h[0] > 0.f ? h[1] / h[0] : 0.f;
  }
  k_mlp_adam<<<8, 256, 0, st>>>(theta, m, v, work, work + MLP_NPARAM, t, lr, 0.9f, 0.999f, 1e-8f);
  CK(cudaGetLastError());
  return MS_OK;
}

int mlp_grad(const void *x, const int *y, const int *idx, int batch, const float *theta, const float *class_w,
             float *work, float *grad, void *cuda_stream, bool tc) {
  Sim *s = nullptr;
  if (!grad) return MS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int r = mlp_run(x, y, idx, batch, theta, class_w, work, st, tc);
  if (r) return r;
  k_mlp_scale<<<8, 256, 0, st>>>(work, work + MLP_NPARAM, grad);
  CK(cudaGetLastError());
  return MS_OK;
}
}  // namespace

int ms_mlp_train_step(const void *x, const int *y, const int *idx, int batch, float *theta, float *m, float *v,
                      int t, float lr, const float *class_w, float *work, float *loss, void *cuda_stream) {
  return mlp_train_step(x, y, idx, batch, theta, m, v, t, lr, class_w, work, loss, cuda_stream, false);
}

int ms_mlp_grad(const void *x, const int *y, const int *idx, int batch, const float *theta, const float *class_w,
                float *work, float *grad, void *cuda_stream) {
  return mlp_grad(x, y, idx, batch, theta, class_w, work, grad, cuda_stream, false);
}

int ms_mlp_train_step_tc(const void *x, const int *y, const int *idx, int batch, float *theta, float *m, float *v,
                         int t, float lr, const float *class_w, float *work, float *loss, void *cuda_stream) {
  return mlp_train_step(x, y, idx, batch, theta, m, v, t, lr, class_w, work, loss, cuda_stream, true);
}

int ms_mlp_grad_tc(const void *x, const int *y, const int *idx, int batch, const float *theta, const float *class_w,
                   float *work, float *grad, void *cuda_stream) {
  return mlp_grad(x, y, idx, batch, theta, class_w, work, grad, cuda_stream, true);
}

int ms_test_tc_timeout(const void *x, const int *y, const int *idx, int batch, const float *theta,
                       const float *class_w, float *work, void *cuda_stream) {
  Sim *s = nullptr;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int r = mlp_run(x, y, idx, batch, theta, class_w, work, st, true, true);
  if (r) return r;
  unsigned e = 0;
  CK(cudaMemcpyAsync(&e, work + MLP_NPARAM + 2, sizeof(e), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return e ? MS_ERR_DEVICE : MS_OK;
}

int ms_test_withhold_copies(void *sim, int on) {
  Sim *s = (Sim *)sim;
  if (!s) return MS_ERR_ARG;
  CK(cudaStreamSynchronize(s->stream));
  s->P.test_withhold = on ? 1 : 0;
  drop_graphs(s);   // the flag is baked into the captured step graphs
  return MS_OK;
}

int ms_mlp_predict(const void *x, int n, const float *theta, float *work, int *cls, float *margin, float *logits,
                   void *cuda_stream) {
  Sim *s = nullptr;
  if (!x || n <= 0 || !theta || !work || !cls || !margin) return MS_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  MlpDev *model = reinterpret_cast<MlpDev *>(work + MLP_NPARAM + 4);
  k_mlp_pack<<<8, 256, 0, st>>>(theta, model);
  k_mlp_predict<<<std::min(4096, (n + 63) / 64), 128, 0, st>>>((const __nv_bfloat16 *)x, n, model, cls, margin,
                                                                logits);
  CK(cudaGetLastError());
  return MS_OK;
}

const char *ms_last_error(void *sim) {
  Sim *s = (Sim *)sim;
  return s ? s->err.c_str() : "null simulation";
}

void ms_destroy(void *sim) {
  Sim *s = (Sim *)sim;
  if (!s) return;
  if (s->veh_loaded || s->net_loaded) cudaStreamSynchronize(s->stream);
  if (s->xs) cudaStreamSynchronize(s->xs);
  drop_graphs(s);
  for (void *p : s->allocs) cudaFree(p);
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->xs) cudaStreamDestroy(s->xs);
  if (s->ev_ready) cudaEventDestroy(s->ev_ready);
  for (cudaEvent_t ev : s->ev_export)
    if (ev) cudaEventDestroy(ev);
  if (s->h_meta) cudaFreeHost(s->h_meta);
  delete s;
}

}  // extern "C"
