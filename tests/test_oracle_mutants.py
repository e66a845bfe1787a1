"""Planted mistakes in the oracle: its pins must catch the mistakes they exist for.

Each case copies oracle/ into a scratch directory, plants one plausible mistake in the copy
(a dropped term, a wrong sign, a transposed index or operand, a reversed comparison, an
off-by-one), and runs the pins named for that mistake (from the four pin files below)
against that copy in a child process: one of them must fail.  A control copy with nothing
planted must pass every pin of the four files, and the child must be shown to import the
copy, not this tree's oracle.  CPU only: the copies are plain C and
numpy, built with gcc in the scratch directory.

Mistakes that change nothing the pins can reach are not listed: the clamp of a position to
the lane end when the own lane ends in an obstacle is a no-op in FP64 (x + (len - x) is
exact for FP32 positions; it exists for rounding on the device); the id order of two
vehicles at the same position on one lane applies only to states with a negative gap, which
the state checks refuse; a merge feeder that does not skip its own lane in the projection
finds its own leader again, at the same gap; and a mistake that sends a vehicle to a lane
that does not exist ends the child process instead of failing a pin."""
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["tests/test_oracle_pins.py", "tests/test_learned_oracle.py", "tests/test_mlp_oracle.py",
             "tests/test_routing_oracle.py"]

# (name, file under oracle/, exact text (occurs once), replacement, pins that must fail)
MUTANTS = [
    # R2: own-path leader across lane ends
    ("lookahead_gap_one_lane_too_long", "moss_oracle.c",
     "r.kind = K_VEH; r.gap = (dist + s->x[j]) - L; r.vl = s->v[j]; r.lead_id = j;\n        break;",
     "r.kind = K_VEH; r.gap = (dist + s->x[j] + (double)s->net.lane_len[nxt]) - L; r.vl = s->v[j];"
     " r.lead_id = j;\n        break;",
     ["test_step_leaders_and_target_neighbours_match_brute_force"]),
    ("lookahead_gap_drops_the_distance", "moss_oracle.c",
     "r.kind = K_VEH; r.gap = (dist + s->x[j]) - L; r.vl = s->v[j]; r.lead_id = j;\n        break;",
     "r.kind = K_VEH; r.gap = (s->x[j]) - L; r.vl = s->v[j]; r.lead_id = j;\n        break;",
     ["test_step_leaders_and_target_neighbours_match_brute_force"]),
    ("own_leader_gap_keeps_the_length", "moss_oracle.c",
     "r.kind = K_VEH; r.gap = (s->x[j] - x) - L;",
     "r.kind = K_VEH; r.gap = (s->x[j] - x);",
     ["test_idm_ring_equilibrium_is_fixed_point"]),
    # R1: IDM
    ("idm_interaction_sign", "moss_oracle.c",
     "v * p->T + v * dv / (2.0 * sqrt(p->a * p->b))",
     "v * p->T - v * dv / (2.0 * sqrt(p->a * p->b))",
     ["test_stop_at_long_red_reaches_standstill_gap"]),
    ("idm_interaction_not_squared", "moss_oracle.c",
     "a = p->a * (freeterm - q * q);", "a = p->a * (freeterm - q);",
     ["test_idm_ring_equilibrium_is_fixed_point"]),
    ("idm_free_road_exponent_two", "moss_oracle.c",
     "double freeterm = 1.0 - r2 * r2;", "double freeterm = 1.0 - r2;",
     ["test_idm_ring_equilibrium_is_fixed_point"]),
    ("idm_drops_the_jam_distance", "moss_oracle.c",
     "double ss = p->s0 + fmax(", "double ss = fmax(",
     ["test_idm_ring_equilibrium_is_fixed_point"]),
    ("lookahead_reads_the_next_lanes_signal", "moss_oracle.c",
     "int sg = or_signal_state(s, cur, s->t);\n          if (sg == SIG_RED) stop = 1;",
     "int sg = or_signal_state(s, nxt, s->t);\n          if (sg == SIG_RED) stop = 1;",
     ["test_stop_at_long_red_reaches_standstill_gap", "test_yellow_stop_rule"]),
    ("lookahead_horizon_doubled", "moss_oracle.c",
     "if (dist >= s->p.d_look) break; /* free */", "if (dist >= 2.0 * s->p.d_look) break; /* free */",
     ["test_step_leaders_and_target_neighbours_match_brute_force"]),
    ("lookahead_internal_lane_keeps_the_route_cursor", "moss_oracle.c",
     "nxt = s->net.succ_lane[s->net.succ_off[cur]];\n        ri += 1;",
     "nxt = s->net.succ_lane[s->net.succ_off[cur]];",
     ["test_step_leaders_and_target_neighbours_match_brute_force"]),
    ("fan_out_ignores_the_edge_after_next", "moss_oracle.c",
     "    if (connects(s, tg, en2)) return il;\n", "    return il;\n",
     ["test_step_leaders_and_target_neighbours_match_brute_force"]),
    ("lookahead_lane_cap_one_short", "moss_oracle.c",
     "if (hop + 1 >= HOP_CAP) {", "if (hop + 2 >= HOP_CAP) {",
     ["test_lookahead_ends_at_the_twelfth_lane"]),
    ("merge_gap_keeps_the_length", "moss_oracle.c",
     "double g = (dc - dj) - L;", "double g = (dc - dj);",
     ["test_merge_projection_leader"]),
    ("merge_takes_the_farther_leader", "moss_oracle.c",
     "if (r.kind == K_FREE || g < r.gap) {", "if (r.kind == K_FREE || g > r.gap) {",
     ["test_step_leaders_and_target_neighbours_match_brute_force"]),
    ("idm_without_the_a_min_clamp", "moss_oracle.c",
     "return fmax(a, p->a_min);", "return a;",
     ["test_motion_stop_within_the_step_and_gap_clamp"]),
    ("fan_out_without_its_fallback", "moss_oracle.c",
     "  return first;\n}", "  return -1;\n}",
     ["test_fan_out_falls_back_to_the_first_open_link"]),
    ("idm_gap_floored_at_one_metre", "moss_oracle.c",
     "double q = ss / fmax(gap, 0.01);", "double q = ss / fmax(gap, 1.0);",
     ["test_idm_below_one_metre_of_gap"]),
    # R9: fixed-time signals
    ("signal_offset_sign", "moss_oracle.c",
     "int tau = ((t + s->net.ctrl_offset[c]) % cyc + cyc) % cyc;",
     "int tau = ((t - s->net.ctrl_offset[c]) % cyc + cyc) % cyc;",
     ["test_signal_offsets_shift_the_table"]),
    ("signal_green_one_second_long", "moss_oracle.c",
     "return (tau % (g + y)) < g ? SIG_GREEN : SIG_YELLOW;",
     "return (tau % (g + y)) <= g ? SIG_GREEN : SIG_YELLOW;",
     ["test_signal_table_closed_form"]),
    ("signal_phase_by_the_green_time_alone", "moss_oracle.c",
     "int k = tau / (g + y);", "int k = tau / g;",
     ["test_signal_table_closed_form"]),
    # R5: stop lines (yellow: stop when the vehicle can)
    ("yellow_rule_reversed", "moss_oracle.c",
     "            mark(flag, m);\n            if (m >= 0.0) stop = 1;",
     "            mark(flag, m);\n            if (m < 0.0) stop = 1;",
     ["test_yellow_stop_rule"]),
    # R4: randomized MOBIL
    ("mobil_own_incentive_sign", "moss_oracle.c",
     "double delta = r.a_new - a_c;", "double delta = a_c - r.a_new;",
     ["test_mobil_incentive_is_free_gain_with_empty_target"]),
    ("mobil_new_follower_term_sign", "moss_oracle.c",
     "delta += p->p * (aF_new - aF_old);", "delta += p->p * (aF_old - aF_new);",
     ["test_mobil_politeness_terms_closed_form"]),
    ("mobil_drops_the_old_follower_term", "moss_oracle.c",
     "delta += p->p * (aO_new - aO_old);", "delta += 0.0 * (aO_new - aO_old);",
     ["test_mobil_politeness_terms_closed_form"]),
    ("mobil_safety_threshold_sign", "moss_oracle.c",
     "if (aF_new < -p->bsafe) return r;", "if (aF_new < p->bsafe) return r;",
     ["test_mobil_safety_criteria"]),
    ("mobil_conflict_guard_drops_the_acceleration_term", "moss_oracle.c",
     "double guard = s->v[Ft] * p->dt + 0.5 * p->a * p->dt * p->dt;", "double guard = s->v[Ft] * p->dt;",
     ["test_mobil_safety_criteria"]),
    ("mobil_new_follower_old_gap_keeps_the_length", "moss_oracle.c",
     "(s->x[Lt] - s->x[Ft]) - L, s->v[Lt]);", "(s->x[Lt] - s->x[Ft]), s->v[Lt]);",
     ["test_mobil_politeness_with_a_target_leader"]),
    ("mobil_old_follower_new_gap_loses_a_length", "moss_oracle.c",
     "own->gap + (x - s->x[O]), own->vl);", "own->gap + (x - s->x[O]) - L, own->vl);",
     ["test_mobil_politeness_terms_closed_form"]),
    ("mandatory_direction_reversed", "moss_oracle.c",
     "int want = best > idx ? +1 : -1;", "int want = best > idx ? -1 : +1;",
     ["test_mandatory_change_toward_connecting_lane"]),
    ("lane_end_zone_measured_from_the_start", "moss_oracle.c",
     "if (len - x < p->x_lc_end) return r;", "if (x < p->x_lc_end) return r;",
     ["test_mobil_zones_and_gate"]),
    ("threshold_jitter_one_sided", "moss_oracle.c",
     "return p->th + p->th_jitter * (2.0 * u - 1.0);", "return p->th + p->th_jitter * u;",
     ["test_mobil_threshold_jitter_is_uniform_over_trips"]),
    ("mandatory_tie_goes_to_the_upper_lane", "moss_oracle.c",
     "abs(q - idx) < bestd) { bestd", "abs(q - idx) <= bestd) { bestd",
     ["test_mandatory_change_tie_goes_to_the_lower_lane"]),
    ("target_lane_end_never_blocks", "moss_oracle.c",
     "} else if (end_blocks(s, tau, en, x, v, flag)) {", "} else if (0) {",
     ["test_target_lane_end_at_red_is_an_obstacle"]),
    ("target_lane_end_yellow_rule_reversed", "moss_oracle.c",
     "    return m >= 0.0;\n", "    return m < 0.0;\n",
     ["test_target_lane_end_at_yellow_and_the_followers_old_gap"]),
    ("follower_gap_to_the_target_lane_end_loses_a_length", "moss_oracle.c",
     "aF_old = idm(s, s->v[Ft], v0_on(s, Ft, tau), 1, len - s->x[Ft], 0.0);",
     "aF_old = idm(s, s->v[Ft], v0_on(s, Ft, tau), 1, len - s->x[Ft] - L, 0.0);",
     ["test_target_lane_end_at_yellow_and_the_followers_old_gap"]),
    ("connects_ignores_closed_links", "moss_oracle.c",
     "    if (s->net.succ_edge[k] == en && !s->link_off[k]) return 1;", "    if (s->net.succ_edge[k] == en) return 1;",
     ["test_closed_links_force_the_mandatory_change"]),
    ("target_lane_end_stopping_distance_doubled", "moss_oracle.c",
     "    double m = ((double)s->net.lane_len[l] - x) - v * v / (2.0 * s->p.b);",
     "    double m = ((double)s->net.lane_len[l] - x) - v * v / (1.0 * s->p.b);",
     ["test_target_lane_end_at_yellow_takes_the_stopping_distance"]),
    ("conflict_guard_divides_by_dt", "moss_oracle.c",
     "    double guard = s->v[Ft] * p->dt + 0.5 * p->a * p->dt * p->dt;",
     "    double guard = s->v[Ft] / p->dt + 0.5 * p->a * p->dt * p->dt;",
     ["test_motion_and_the_conflict_guard_scale_with_dt"]),
    ("target_lane_speed_limit_ignored", "moss_oracle.c",
     "r.a_new = idm(s, v, fmin(v0, s->lane_vmax[tau]),", "r.a_new = idm(s, v, v0,",
     ["test_mobil_uses_the_target_lanes_limit"]),
    ("level_target_vehicle_taken_as_the_leader", "moss_oracle.c",
     "    if (s->x[o[mid]] > x) hi = mid; else lo = mid + 1;", "    if (s->x[o[mid]] >= x) hi = mid; else lo = mid + 1;",
     ["test_level_vehicle_in_the_target_lane_is_the_follower"]),
    ("lane_start_zone_ten_metres_too_long", "moss_oracle.c",
     "  if (x < p->x_lc_min) return r;", "  if (x <= p->x_lc_min + 10.0) return r;",
     ["test_mobil_zones_and_gate"]),
    ("discretionary_target_need_not_serve_the_route", "moss_oracle.c",
     "    if (!connects(s, tau, en)) return r;\n", "",
     ["test_discretionary_change_only_toward_a_lane_serving_the_route"]),
    ("old_follower_present_acceleration_under_the_target_limit", "moss_oracle.c",
     "      double aO_old = idm(s, s->v[O], v0_on(s, O, l), 1, gO, v);",
     "      double aO_old = idm(s, s->v[O], v0_on(s, O, tau), 1, gO, v);",
     ["test_old_follower_drives_under_its_own_lanes_limit"]),
    ("old_follower_prospective_acceleration_under_the_target_limit", "moss_oracle.c",
     "        aO_new = idm(s, s->v[O], v0_on(s, O, l), 1, own->gap + (x - s->x[O]), own->vl);",
     "        aO_new = idm(s, s->v[O], v0_on(s, O, tau), 1, own->gap + (x - s->x[O]), own->vl);",
     ["test_old_follower_drives_under_its_own_lanes_limit"]),
    ("lookahead_hop_adds_the_lane_left_behind", "moss_oracle.c",
     "      dist += (double)s->net.lane_len[nxt];", "      dist += (double)s->net.lane_len[cur];",
     ["test_lookahead_ends_at_the_twelfth_lane"]),
    ("new_follower_under_its_present_lanes_limit", "moss_oracle.c",
     "aF_new = idm(s, s->v[Ft], v0_on(s, Ft, tau), 1, gF, v);", "aF_new = idm(s, s->v[Ft], v0_on(s, Ft, l), 1, gF, v);",
     ["test_new_follower_drives_under_the_target_lanes_limit"]),
    ("target_leader_and_follower_transposed", "moss_oracle.c",
     "int Lt = j < cnt ? o[j] : -1;\n  int Ft = j > 0 ? o[j - 1] : -1;",
     "int Lt = j > 0 ? o[j - 1] : -1;\n  int Ft = j < cnt ? o[j] : -1;",
     ["test_step_leaders_and_target_neighbours_match_brute_force"]),
    ("step_direction_parity_reversed", "moss_oracle.c",
     "int step_dir = (s->t % 2 == 0) ? +1 : -1;", "int step_dir = (s->t % 2 == 0) ? -1 : +1;",
     ["test_mobil_direction_alternates_with_step_parity"]),
    ("random_gate_reversed", "moss_oracle.c",
     "if ((h >> 40) >= thr) return r;", "if ((h >> 40) < thr) return r;",
     ["test_mobil_zones_and_gate"]),
    ("random_gate_the_same_at_every_step", "moss_oracle.c",
     "    uint64_t h = or_splitmix64(p->seed ^ ((uint64_t)(uint32_t)s->t << 32) ^ (uint64_t)(uint32_t)c);",
     "    uint64_t h = or_splitmix64(p->seed ^ (uint64_t)(uint32_t)c);",
     ["test_random_gate_is_a_fresh_draw_per_trip_and_step"]),
    ("random_gate_the_same_for_every_trip", "moss_oracle.c",
     "    uint64_t h = or_splitmix64(p->seed ^ ((uint64_t)(uint32_t)s->t << 32) ^ (uint64_t)(uint32_t)c);",
     "    uint64_t h = or_splitmix64(p->seed ^ ((uint64_t)(uint32_t)s->t << 32));",
     ["test_random_gate_is_a_fresh_draw_per_trip_and_step"]),
    # R6, R7: motion and transfer
    ("advance_by_the_end_speed", "moss_oracle.c",
     "d = 0.5 * (v + vn) * p->dt;", "d = vn * p->dt;",
     ["test_free_road_accelerates_to_v0"]),
    ("transfer_drops_the_overshoot", "moss_oracle.c",
     "          xn -= len;\n", "          xn = 0.0;\n",
     ["test_free_road_accelerates_to_v0"]),
    ("stop_within_the_step_does_not_move", "moss_oracle.c",
     "d = v > 0.0 ? (v * v) / (-2.0 * a_use) : 0.0;", "d = 0.0;",
     ["test_motion_stop_within_the_step_and_gap_clamp"]),
    ("gap_clamp_keeps_the_speed", "moss_oracle.c",
     "      d = dmax;\n      vn = fmin(vn, d / p->dt);", "      d = dmax;",
     ["test_motion_stop_within_the_step_and_gap_clamp"]),
    ("no_speed_cap", "moss_oracle.c",
     "vn = fmin(vraw, p->v_max);", "vn = vraw;",
     ["test_speed_is_capped_at_v_max"]),
    ("changer_moves_with_the_prospective_acceleration", "moss_oracle.c",
     "double a_use = lc.dir ? fmin(a_c, lc.a_new) : a_c;", "double a_use = lc.dir ? lc.a_new : a_c;",
     ["test_mobil_incentive_is_free_gain_with_empty_target"]),
    ("changer_not_held_at_its_lane_end", "moss_oracle.c",
     "      gmin = fmin(gmin, len - x);\n", "",
     ["test_changer_stops_at_its_lane_end"]),
    ("junction_transfer_keeps_the_route_cursor", "moss_oracle.c",
     "            nrp += 1;\n", "",
     ["test_small_grid_run_invariants"]),
    ("speed_update_divides_by_dt", "moss_oracle.c",
     "    double vraw = v + a_use * p->dt;", "    double vraw = v + a_use / p->dt;",
     ["test_motion_and_the_conflict_guard_scale_with_dt"]),
    ("advance_divides_by_dt", "moss_oracle.c",
     "      d = 0.5 * (v + vn) * p->dt;", "      d = 0.5 * (v + vn) / p->dt;",
     ["test_motion_and_the_conflict_guard_scale_with_dt"]),
    ("gap_clamp_speed_multiplies_by_dt", "moss_oracle.c",
     "      vn = fmin(vn, d / p->dt);", "      vn = fmin(vn, d * p->dt);",
     ["test_motion_and_the_conflict_guard_scale_with_dt"]),
    ("retires_one_edge_early", "moss_oracle.c",
     "if (!is_internal(s, l) && route_at(s, c, s->rp[c] + 1) < 0) {",
     "if (!is_internal(s, l) && route_at(s, c, s->rp[c] + 2) < 0) {",
     ["test_closed_lane_is_never_entered_until_reopened"]),
    ("arrival_clock_off_by_one", "moss_oracle.c",
     "      s->t_arr[c] = s->t + 1;\n      s->counters[1] += 1;", "      s->t_arr[c] = s->t;\n      s->counters[1] += 1;",
     ["test_travel_time_is_the_arrival_clock_minus_the_departure"]),
    ("edge_lane_transfer_advances_the_route_cursor", "moss_oracle.c",
     "            nl = choose_succ(s, l, route_at(s, c, s->rp[c] + 1), route_at(s, c, s->rp[c] + 2));\n",
     "            nl = choose_succ(s, l, route_at(s, c, s->rp[c] + 1), route_at(s, c, s->rp[c] + 2));\n            nrp += 1;\n",
     ["test_small_grid_run_invariants"]),
    ("travel_time_off_by_one", "moss_oracle.c",
     "s->counters[2] += (int64_t)(s->t + 1 - s->t_dep[c]);", "s->counters[2] += (int64_t)(s->t - s->t_dep[c]);",
     ["test_travel_time_is_the_arrival_clock_minus_the_departure"]),
    # R10: lane metrics
    ("metrics_window_off_by_one", "moss_oracle.c",
     "int w = s->t / p->window;", "int w = (s->t + 1) / p->window;",
     ["test_metrics_window_sums"]),
    # R8: departures
    ("departure_room_ignores_the_tail_length", "moss_oracle.c",
     "double m = (s->x[tail] - L) - (L + p->s0);", "double m = s->x[tail] - (L + p->s0);",
     ["test_departures_fifo_and_room"]),
    ("departs_a_step_early", "moss_oracle.c",
     "if (s->t_dep[h] > s->t) continue;", "if (s->t_dep[h] > s->t + 1) continue;",
     ["test_departure_waits_for_its_time"]),
    ("inserted_front_at_the_lane_start", "moss_oracle.c",
     "    s->x[h] = L;\n    s->v[h] = 0.0;", "    s->x[h] = 0.0;\n    s->v[h] = 0.0;",
     ["test_departure_waits_for_its_time"]),
    ("departure_lane_ignores_the_links", "moss_oracle.c",
     "    if (connects(s, l0 + q, e1)) return l0 + q;\n  return -1;", "    if (1) return l0 + q;\n  return -1;",
     ["test_departures_enter_the_first_lane_linked_to_the_next_edge"]),
    ("departure_queue_latest_first", "moss_oracle.c",
     "  if (s->t_dep[a] != s->t_dep[b]) return s->t_dep[a] < s->t_dep[b] ? -1 : 1;",
     "  if (s->t_dep[a] != s->t_dep[b]) return s->t_dep[a] > s->t_dep[b] ? -1 : 1;",
     ["test_departure_queue_is_first_in_first_out_by_departure_time"]),
    ("departure_queue_tie_by_the_higher_id", "moss_oracle.c",
     "  if (s->t_dep[a] != s->t_dep[b]) return s->t_dep[a] < s->t_dep[b] ? -1 : 1;\n  return a < b ? -1 : (a > b);",
     "  if (s->t_dep[a] != s->t_dep[b]) return s->t_dep[a] < s->t_dep[b] ? -1 : 1;\n  return a > b ? -1 : (a < b);",
     ["test_departures_fifo_and_room"]),
    ("arrival_rear_without_the_length", "moss_oracle.c",
     "arr_min[nl] = fmin(arr_min[nl], s->n_x[c] - L);", "arr_min[nl] = fmin(arr_min[nl], s->n_x[c]);",
     ["test_small_grid_run_invariants"]),
    ("departure_room_ignores_s0_behind_arrivals", "moss_oracle.c",
     "double m = arr_min[l] - (L + p->s0);", "double m = arr_min[l] - L;",
     ["test_departure_room_counts_the_arrivals_of_the_step"]),
    ("departures_enter_a_closed_lane", "moss_oracle.c",
     "    if (s->lane_closed[l]) continue;   /* R14: the queue waits */\n", "",
     ["test_departures_wait_on_a_closed_lane"]),
    ("state_write_keeps_the_queue_heads", "moss_oracle.c",
     "  for (int l = 0; l < s->net.n_lanes; ++l) s->q_head[l] = s->q_off[l];\n  mp_reset(s);",
     "  for (int l = 0; l >= s->net.n_lanes; ++l) s->q_head[l] = s->q_off[l];\n  mp_reset(s);",
     ["test_rewinding_a_run_resumes_it_exactly"]),
    ("lane_link_changes_unchecked", "moss_oracle.c",
     "  for (int k = 0; k < n; ++k) {   /* validate first: nothing changes on a bad entry */",
     "  for (int k = 0; k >= n; ++k) {   /* validate first: nothing changes on a bad entry */",
     ["test_lane_link_changes_are_checked"]),
    # R3: merge projection
    ("merge_projection_order_reversed", "moss_oracle.c",
     "if (dj < dc || (dj == dc && j < c)) { found = j; break; }",
     "if (dj > dc || (dj == dc && j < c)) { found = j; break; }",
     ["test_merge_projection_leader"]),
    ("merge_tie_break_reversed", "moss_oracle.c",
     "if (dj < dc || (dj == dc && j < c)) { found = j; break; }",
     "if (dj < dc || (dj == dc && j > c)) { found = j; break; }",
     ["test_merge_projection_leader"]),
    # R13: max pressure
    ("max_pressure_sign", "moss_oracle.c",
     "sum += s->seg_cnt[l] - s->seg_cnt[m];", "sum += s->seg_cnt[m] - s->seg_cnt[l];",
     ["test_max_pressure_switches_to_the_loaded_phase"]),
    ("max_pressure_tie_leaves_the_green_phase", "moss_oracle.c",
     "if (pr[s->mp_g[c]] == pr[best]) best = s->mp_g[c];", "",
     ["test_max_pressure_holds_the_green_phase_on_ties"]),
    ("max_pressure_counts_closed_links", "moss_oracle.c",
     "if (s->link_off[k]) continue;   /* R17 */\n        const int il", "const int il",
     ["test_max_pressure_skips_closed_links"]),
    ("max_pressure_counts_the_junction_lane", "moss_oracle.c",
     "const int m = s->net.succ_lane[s->net.succ_off[il]];", "const int m = il;",
     ["test_max_pressure_run_matches_brute_force_and_never_runs_red"]),
    ("max_pressure_yellow_one_step_short", "moss_oracle.c",
     "s->mp_yend[c] = t + s->net.ctrl_yellow[c];", "s->mp_yend[c] = t + s->net.ctrl_yellow[c] - 1;",
     ["test_max_pressure_run_matches_brute_force_and_never_runs_red"]),
    ("max_pressure_tie_goes_to_the_higher_phase", "moss_oracle.c",
     "if (pr[ph] > pr[best]) best = ph;", "if (pr[ph] >= pr[best]) best = ph;",
     ["test_max_pressure_tie_between_two_other_phases_goes_to_the_lower"]),
    ("max_pressure_yellow_ends_a_step_late", "moss_oracle.c",
     "if (s->mp_pend[c] >= 0 && t >= s->mp_yend[c]) {", "if (s->mp_pend[c] >= 0 && t > s->mp_yend[c]) {",
     ["test_max_pressure_run_matches_brute_force_and_never_runs_red"]),
    ("max_pressure_decides_while_a_switch_is_pending", "moss_oracle.c",
     "if (!decide || s->mp_pend[c] >= 0) continue;", "if (!decide) continue;",
     ["test_max_pressure_run_matches_brute_force_and_never_runs_red"]),
    ("max_pressure_decision_steps_shifted", "moss_oracle.c",
     "const int decide = (t % s->p.mp_interval) == 0;", "const int decide = ((t + 1) % s->p.mp_interval) == 0;",
     ["test_max_pressure_run_matches_brute_force_and_never_runs_red"]),
    ("max_pressure_switch_without_yellow", "moss_oracle.c",
     "return s->mp_pend[c] >= 0 ? SIG_YELLOW : SIG_GREEN;", "return SIG_GREEN;",
     ["test_max_pressure_switches_to_the_loaded_phase"]),
    ("step_leaves_the_controllers_to_the_state_read", "moss_oracle.c",
     "  if (p->signal_mode == 1) mp_advance(s);   /* R13: controllers at step t */",
     "  if (p->signal_mode != 1) mp_advance(s);   /* R13: controllers at step t */",
     ["test_max_pressure_steps_advance_the_controllers_themselves"]),
    # R14: lane limits and closures
    ("speed_limit_ignored", "moss_oracle.c",
     "return fmin((double)s->v0[c], s->lane_vmax[l]);", "return (double)s->v0[c];",
     ["test_lane_speed_limit_caps_the_desired_speed"]),
    ("closed_target_lane_entered", "moss_oracle.c",
     "if (s->lane_closed[tau]) return r;   /* R14 */", "",
     ["test_mobil_uses_the_target_lanes_limit"]),
    # R19: BF16 rounding of the learned decision
    ("bf16_rounds_to_seven_bits", "moss_oracle.c",
     "return ldexp(nearbyint(ldexp(m, 8)), e - 8);", "return ldexp(nearbyint(ldexp(m, 7)), e - 7);",
     ["test_bf16_rounding_follows_the_format"]),
    ("learned_margin_test_reversed", "moss_oracle.c",
     "if (mg < m->margin) return rule_dir;", "if (mg > m->margin) return rule_dir;",
     ["test_full_fallback_network_is_the_rule_over_a_run"]),
    ("learned_classes_left_and_right_swapped", "moss_oracle.c",
     "static int class_dir(int cls) { return cls == 1 ? +1 : (cls == 2 ? -1 : 0); }",
     "static int class_dir(int cls) { return cls == 1 ? -1 : (cls == 2 ? +1 : 0); }",
     ["test_probe_network_decides_by_one_physical_quantity"]),
    ("learned_margin_is_the_top_probability", "moss_oracle.c",
     "return pr[c] - sec;", "return pr[c];",
     ["test_learned_logits_match_the_numpy_bf16_forward"]),
    ("learned_disallowed_direction_falls_back_to_the_rule", "moss_oracle.c",
     "return (d != 0 && d != step_dir) ? 0 : d;", "return (d != 0 && d != step_dir) ? rule_dir : d;",
     ["test_always_right_network_changes_only_on_right_steps"]),
    ("learned_inputs_8_and_9_swapped", "moss_oracle.c",
     "f[8] = lc->tau_foll >= 0 ? fmin(lc->gF, 200.0) / 100.0 : 2.0;\n  f[9] = lc->tau_foll >= 0 ? lc->vF / 20.0 : 0.0;",
     "f[9] = lc->tau_foll >= 0 ? fmin(lc->gF, 200.0) / 100.0 : 2.0;\n  f[8] = lc->tau_foll >= 0 ? lc->vF / 20.0 : 0.0;",
     ["test_learned_inputs_follow_from_the_state"]),
    ("learned_input_12_reads_the_own_speed", "moss_oracle.c",
     "f[12] = O >= 0 ? s->v[O] / 20.0 : 0.0;", "f[12] = O >= 0 ? v / 20.0 : 0.0;",
     ["test_learned_inputs_follow_from_the_state"]),
    ("learned_hidden_layer_drops_its_bias", "moss_oracle.c",
     "a1[j] = acc + m->b1[j];", "a1[j] = acc;",
     ["test_learned_logits_match_the_numpy_bf16_forward"]),
    ("in_step_flag_rule_tests_the_rounded_hidden_value", "moss_oracle.c",
     "if (!near_boundary(hv, h1[j], 17.0 * u * s1[j], &alt)) continue;",
     "if (!near_boundary(h1[j], h1[j], 17.0 * u * s1[j], &alt)) continue;",
     ["test_in_step_flag_rule_counts_a_hidden_value_on_a_rounding_midpoint"]),
    ("learned_class_tie_goes_to_the_higher_index", "moss_oracle.c",
     "    if (pr[q] > pr[c]) c = q;", "    if (pr[q] >= pr[c]) c = q;",
     ["test_tied_classes_go_to_the_lower_index"]),
    ("network_decides_mandatory_changes", "moss_oracle.c",
     "if (s->mlp && lc.cand && lc.safe && !lc.mandatory) {", "if (s->mlp && lc.cand && lc.safe) {",
     ["test_mandatory_changes_bypass_the_network"]),
    ("learned_acceleration_input_unscaled", "moss_oracle.c",
     "  f[4] = a_c / p->a;", "  f[4] = a_c;",
     ["test_learned_inputs_follow_from_the_state"]),
    ("flag_rule_upper_neighbour_below", "moss_oracle.c",
     "  const double n = up ? a + ulp : (a == ldexp(1.0, e - 1) ? a - ulp / 2 : a - ulp);",
     "  const double n = up ? a - ulp : (a == ldexp(1.0, e - 1) ? a - ulp / 2 : a - ulp);",
     ["test_in_step_flag_rule_counts_a_hidden_value_on_a_rounding_midpoint"]),
    ("flag_rule_misses_the_power_of_two_below", "moss_oracle.c",
     "  const double n = up ? a + ulp : (a == ldexp(1.0, e - 1) ? a - ulp / 2 : a - ulp);",
     "  const double n = up ? a + ulp : (a == ldexp(1.0, e + 1) ? a - ulp / 2 : a - ulp);",
     ["test_in_step_flag_rule_counts_a_hidden_value_on_a_rounding_midpoint"]),
    ("flag_rule_half_step_below_a_power_of_two_upward", "moss_oracle.c",
     "  const double n = up ? a + ulp : (a == ldexp(1.0, e - 1) ? a - ulp / 2 : a - ulp);",
     "  const double n = up ? a + ulp : (a == ldexp(1.0, e - 1) ? a + ulp / 2 : a - ulp);",
     ["test_in_step_flag_rule_counts_a_hidden_value_on_a_rounding_midpoint"]),
    ("flag_rule_upper_midpoint_misplaced", "moss_oracle.c",
     "  if (fabs(v - 0.5 * (r + out)) <= delta) { *alt = out; return 1; }",
     "  if (fabs(v - 0.5 * (r - out)) <= delta) { *alt = out; return 1; }",
     ["test_in_step_flag_rule_counts_a_hidden_value_on_a_rounding_midpoint"]),
    ("flag_rule_re_evaluation_skips_hidden_layer_1", "moss_oracle.c",
     "      for (int j = 0; j < 64; ++j) h1[j] = or_bf16(fmax(a1[j], 0.0));\n",
     "      for (int j = 0; j >= 64; ++j) h1[j] = or_bf16(fmax(a1[j], 0.0));\n",
     ["test_in_step_flag_rule_counts_a_hidden_value_on_a_rounding_midpoint"]),
    ("flag_rule_skips_the_inputs", "moss_oracle.c",
     "  for (int k = 0; k < 16; ++k) {\n    if (!near_boundary(", "  for (int k = 0; k >= 16; ++k) {\n    if (!near_boundary(",
     ["test_in_step_flag_rule_counts_a_hidden_value_on_a_rounding_midpoint"]),
    ("flag_rule_lower_neighbour_above", "moss_oracle.c",
     "  const double n = up ? a + ulp : (a == ldexp(1.0, e - 1) ? a - ulp / 2 : a - ulp);",
     "  const double n = up ? a + ulp : (a == ldexp(1.0, e - 1) ? a - ulp / 2 : a + ulp);",
     ["test_in_step_flag_rule_counts_a_hidden_value_on_a_rounding_midpoint"]),
    ("learned_input_10_only_without_a_follower", "moss_oracle.c",
     "  f[10] = lc->tau_foll >= 0 ? lc->aF_new / p->a : 0.0;", "  f[10] = lc->tau_foll < 0 ? lc->aF_new / p->a : 0.0;",
     ["test_learned_inputs_follow_from_the_state"]),
    ("learned_input_11_unscaled_the_other_way", "moss_oracle.c",
     "  f[11] = lc->a_new / p->a;", "  f[11] = lc->a_new * p->a;",
     ["test_learned_inputs_follow_from_the_state"]),
    # the network's gradient and optimiser (numpy)
    ("mlp_gradient_wrong_relu_mask", "mlp.py",
     "da1 = dh1 * (a1 > 0)\n    g[\"W1\"]", "da1 = dh1 * (a1 >= -1.0)\n    g[\"W1\"]",
     ["test_gradient_matches_central_differences"]),
    ("mlp_bias_gradient_before_the_mask", "mlp.py",
     "g[\"b2\"] = da2.sum(0)\n    dh1 = da2 @ prm", "g[\"b2\"] = dh2.sum(0)\n    dh1 = da2 @ prm",
     ["test_gradient_matches_central_differences"]),
    ("loss_weights_not_normalised", "mlp.py",
     "dz *= (w / W)[:, None]", "dz *= w[:, None]",
     ["test_gradient_matches_central_differences"]),
    ("bf16_gradient_keeps_the_hidden_gradient_unrounded", "mlp.py",
     "da2 = bf16((db @ W3) * (h2 > 0))", "da2 = (db @ W3) * (h2 > 0)",
     ["test_bf16_gradient_rounds_the_hidden_gradient"]),
    ("margin_is_top_minus_lowest", "mlp.py",
     "return s[:, -1] - s[:, -2], p.argmax(1)", "return s[:, -1] - s[:, 0], p.argmax(1)",
     ["test_learned_logits_match_the_numpy_bf16_forward"]),
    ("network_inputs_not_rounded", "mlp.py",
     "    Xb = bf16(X)\n    u = 2.0 ** -22\n    near", "    Xb = X\n    u = 2.0 ** -22\n    near",
     ["test_bf16_forward_rounds_where_the_kernel_rounds"]),
    ("flag_rule_tests_the_rounded_hidden_value", "mlp.py",
     "n1, alt1 = _near_alt(np.maximum(a1, 0.0), h1,", "n1, alt1 = _near_alt(h1, h1,",
     ["test_flag_rule_rounds_a_boundary_value_the_other_way"]),
    ("flag_rule_always_rounds_up", "mlp.py",
     "alt = np.sign(r) * np.where(n_up, up, dn)", "alt = np.sign(r) * up",
     ["test_flag_rule_rounds_a_boundary_value_the_other_way"]),
    ("flag_rule_logit_bound_ignores_the_changes", "mlp.py",
     "        np.add.at(zb, s, np.abs(z2 - z[s]))\n", "        pass\n",
     ["test_flag_rule_rounds_a_boundary_value_the_other_way"]),
    ("flag_rule_accumulation_bound_of_the_wrong_layer", "mlp.py",
     "    zb = 65 * u * (np.abs(h2) @ np.abs(W3).T + np.abs(b3))\n    m, c = margin_class(z)",
     "    zb = 17 * u * (np.abs(h2) @ np.abs(W3).T + np.abs(b3))\n    m, c = margin_class(z)",
     ["test_flag_rule_rounds_a_boundary_value_the_other_way"]),
    ("flag_rule_upper_side_misplaced", "mlp.py",
     "    n_up = (a > 0) & (np.abs(av - (a + up) / 2) <= delta)", "    n_up = (a > 0) & (np.abs(av - (a - up) / 2) <= delta)",
     ["test_flag_rule_in_every_rounding_position"]),
    ("flag_rule_power_of_two_step_not_halved", "mlp.py",
     "    ulp_in = np.where(a == np.ldexp(1.0, e - 1), ulp / 2, ulp)\n    up, dn",
     "    ulp_in = np.where(a == np.ldexp(1.0, e + 1), ulp / 2, ulp)\n    up, dn",
     ["test_flag_rule_in_every_rounding_position"]),
    ("flag_rule_logit_bound_subtracts_the_bias", "mlp.py",
     "    zb = 65 * u * (np.abs(h2) @ np.abs(W3).T + np.abs(b3))", "    zb = 65 * u * (np.abs(h2) @ np.abs(W3).T - np.abs(b3))",
     ["test_flag_rule_in_every_rounding_position"]),
    ("flag_rule_input_path_subtracts_the_hidden_bias", "mlp.py",
     "            _, h2a = tail(bf16(np.maximum(xa @ W1.T + b1, 0.0)))", "            _, h2a = tail(bf16(np.maximum(xa @ W1.T - b1, 0.0)))",
     ["test_flag_rule_on_an_input_tie_and_the_prediction_margin"]),
    ("prediction_margin_top_plus_second", "mlp.py",
     "    return p.argmax(1), s[:, -1] - s[:, -2]", "    return p.argmax(1), s[:, -1] + s[:, -2]",
     ["test_flag_rule_on_an_input_tie_and_the_prediction_margin"]),
    ("adam_without_second_moment_correction", "mlp.py",
     "vh = v / (1 - b2 ** t)", "vh = v",
     ["test_adam_first_step_is_lr_times_sign"]),
    # R16, R18: demand generation (numpy)
    ("gravity_decay_one_power_short", "routing.py",
     "            for _ in range(gamma):\n                p = np.float32(p * dkm)\n            W[i, j]",
     "            for _ in range(gamma - 1):\n                p = np.float32(p * dkm)\n            W[i, j]",
     ["test_gravity_decays_with_route_distance"]),
    ("gravity_origins_uniform", "routing.py",
     "cdf_o = np.cumsum(A, dtype=np.float32)\n    W = np.zeros",
     "cdf_o = np.cumsum(np.ones_like(A), dtype=np.float32)\n    W = np.zeros",
     ["test_gravity_origins_and_destinations_follow_the_weights"]),
    ("route_takes_the_last_least_cost_successor", "routing.py",
     "                    nxt = f\n                    break", "                    nxt = f",
     ["test_routes_are_the_lexicographically_smallest_least_cost_paths"]),
    ("uniform_draws_one_bit_short", "routing.py",
     "return splitmix64((seed ^ salt ^ k) % 2 ** 64) >> 40", "return splitmix64((seed ^ salt ^ k) % 2 ** 64) >> 41",
     ["test_gravity_origins_and_destinations_follow_the_weights"]),
    ("route_cost_of_the_edge_left", "routing.py",
     "csr_matrix((c[dst].astype(np.float64), (dst, src))", "csr_matrix((c[src].astype(np.float64), (dst, src))",
     ["test_routes_are_the_lexicographically_smallest_least_cost_paths"]),
    ("gravity_includes_the_origin_zone", "routing.py",
     "if j == i or not np.isfinite(cost[i, j]):", "if not np.isfinite(cost[i, j]):",
     ["test_gravity_origins_and_destinations_follow_the_weights"]),
    ("radiation_departure_times_modulo_the_span", "routing.py",
     "        td[k] = (_u24(splitmix64, seed, SALT_TIME, k) * int(t_span)) >> 24\n    return o, de, td\n\n\n# ----",
     "        td[k] = _u24(splitmix64, seed, SALT_TIME, k) % int(t_span)\n    return o, de, td\n\n\n# ----",
     ["test_departure_times_scale_with_the_span"]),
    ("radiation_origins_not_by_population", "routing.py",
     "    W = (radiation_weights if m.shape[0] <= 256 else radiation_weights_vec)(cost, m)\n    cdf_o = np.cumsum(m, dtype=np.float32)\n"
     "    cdf_d = np.cumsum(W, axis=1, dtype=np.float32)\n    o = np.zeros(n, np.int32)\n    de = np.zeros(n, np.int32)\n"
     "    td = np.zeros(n, np.int32)\n    for k in range(n):\n        uo = np.float32(_u24(splitmix64, seed, SALT_ORIGIN, k)) * np.float32(2.0 ** -24)\n        i = _first_above(cdf_o, np.float32(uo * cdf_o[-1]))\n        ud",
     "    W = (radiation_weights if m.shape[0] <= 256 else radiation_weights_vec)(cost, m)\n    cdf_o = np.cumsum(m, dtype=np.float32)\n"
     "    cdf_d = np.cumsum(W, axis=1, dtype=np.float32)\n    o = np.zeros(n, np.int32)\n    de = np.zeros(n, np.int32)\n"
     "    td = np.zeros(n, np.int32)\n    for k in range(n):\n        uo = np.float32(_u24(splitmix64, seed, SALT_ORIGIN, k)) * np.float32(2.0 ** -24)\n        i = _first_above(cdf_o, np.float32(uo / cdf_o[-1]))\n        ud",
     ["test_radiation_sampling_follows_the_weights_and_is_scale_free"]),
    ("radiation_drops_the_destination_population", "routing.py",
     "den = np.float32(np.float32(m[i] + s[j]) * np.float32(np.float32(m[i] + m[j]) + s[j]))\n"
     "            W[i, j] = np.float32(num / den)\n    return W\n\n\ndef radiation_weights_vec",
     "den = np.float32(np.float32(m[i] + s[j]) * np.float32(np.float32(m[i]) + s[j]))\n"
     "            W[i, j] = np.float32(num / den)\n    return W\n\n\ndef radiation_weights_vec",
     ["test_radiation_weights_closed_form_on_a_line"]),
]

_FAILED = re.compile(r"^FAILED \S+::(\w+)")


def _copy_oracle(dst):
    """oracle/'s sources (no built library, no caches) under dst/oracle."""
    src = os.path.join(ROOT, "oracle")
    os.makedirs(os.path.join(dst, "oracle"))
    for f in os.listdir(src):
        if f.endswith((".py", ".c", ".h")):
            shutil.copy(os.path.join(src, f), os.path.join(dst, "oracle", f))


def _plant(dst, fname, old, new):
    path = os.path.join(dst, "oracle", fname)
    text = open(path).read()
    assert text.count(old) == 1, f"{fname}: the text to change must occur exactly once: {old!r}"
    with open(path, "w") as f:
        f.write(text.replace(old, new))


def _child_env():
    # the child runs in the scratch directory, which python -m puts first on sys.path, so
    # `import oracle` finds the copy; this tree comes after it for the package and tests
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT
    env["OMP_NUM_THREADS"] = "1"
    env.pop("PYTEST_ADDOPTS", None)
    return env


def _pin_ids(names):
    """pytest node ids of the named pins (every parametrization of each)."""
    ids = []
    for f in PIN_FILES:
        defined = set(re.findall(r"^def (test_\w+)", open(os.path.join(ROOT, f)).read(), re.M))
        ids += [f"{os.path.join(ROOT, f)}::{n}" for n in sorted(defined & set(names))]
    assert len(ids) == len(set(names)), f"pins not found: {sorted(set(names))}"
    return ids


def _run_pins(job):
    """Run pins against the oracle copy in dst: the named ones, or all four pin files when
    none are named; (exit code, failed test names, tail)."""
    dst, names = job
    args = [sys.executable, "-m", "pytest", "-q", "-rf", "-p", "no:cacheprovider", "--rootdir", ROOT,
            "-c", os.path.join(ROOT, "pytest.ini"), "-m", "not gpu"]
    args += _pin_ids(names) if names else [os.path.join(ROOT, f) for f in PIN_FILES]
    r = subprocess.run(args, cwd=dst, env=_child_env(), capture_output=True, text=True, timeout=900)
    failed = sorted({m.group(1) for m in map(_FAILED.match, r.stdout.splitlines()) if m})
    return r.returncode, failed, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """The control copy against every pin, and every planted mistake against the pins named
    for it, run concurrently (one child each)."""
    jobs = {}
    ctl = str(tmp_path_factory.mktemp("control"))
    _copy_oracle(ctl)
    jobs["control"] = (ctl, None)
    for name, fname, old, new, catchers in MUTANTS:
        d = str(tmp_path_factory.mktemp(name))
        _copy_oracle(d)
        _plant(d, fname, old, new)
        jobs[name] = (d, catchers)
    # the child imports the copy, not this tree's oracle
    r = subprocess.run([sys.executable, "-c", "import oracle; print(oracle.__file__)"], cwd=ctl,
                       env=_child_env(), capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and os.path.realpath(r.stdout.strip()).startswith(os.path.realpath(ctl)), r
    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        res = dict(zip(jobs, ex.map(_run_pins, jobs.values())))
    return res


def test_control_copy_passes_every_pin(outcomes):
    code, failed, tail = outcomes["control"]
    assert code == 0 and not failed, tail


@pytest.mark.parametrize("name, fname, old, new, catchers", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(outcomes, name, fname, old, new, catchers):
    code, failed, tail = outcomes[name]
    # exit code 1: the named pins ran and some failed (not a crash, a collection error or a
    # timeout), and one of those that failed is named for this mistake
    assert code == 1, f"{name}: pins exit code {code}\n{tail}"
    assert set(catchers) & set(failed), f"{name}: caught only by {failed}, not by {catchers}\n{tail}"
