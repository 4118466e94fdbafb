"""Mutation tests of the oracle's pins (no GPU).

Each mutant plants one plausible mistake -- a dropped term, a wrong sign, a
wrong index or operand -- in a temporary copy of ``oracle/sta_oracle.c``,
compiles it with gcc and runs the pin suite (test_oracle_pins.py) against it
in a child process.  The pins must fail on every mutant: a mutant that
passes marks a formula the pins do not fix."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "sta_oracle.c")

# (name, text to replace, replacement, which occurrence (0-based))
MUTANTS = [
    # O1 NLDM interpolation and its partials
    ("lut_corner_swap", "t * (1 - u) * v10 + (1 - t) * u * v01", "t * (1 - u) * v01 + (1 - t) * u * v10", 0),
    ("lut_ds_no_width", "u * (v11 - v01)) / (x1 - x0);", "u * (v11 - v01));", 0),
    ("lut_dl_weight", "out3[2] = ((1 - t) * (v01 - v00)", "out3[2] = ((1 - u) * (v01 - v00)", 0),
    ("lut_t_offset", "double t = (s - x0) / (x1 - x0);", "double t = (s - x1) / (x1 - x0);", 0),
    # O3 Elmore and second moment
    ("elmore_local_cap", "D[i] = D[parent[i]] + R[i] * cdown[i];", "D[i] = D[parent[i]] + R[i] * C[i];", 0),
    ("elmore_beta_factor", "var[i] = 2.0 * beta[i] - D[i] * D[i];", "var[i] = beta[i] - D[i] * D[i];", 0),
    ("elmore_moment_cap", "M[i] = C[i] * D[i];", "M[i] = cdown[i] * D[i];", 0),
    ("net_no_pin_cap", "C[node] += 1e3 * pin_cap_of", "C[node] += 0.0 * pin_cap_of", 0),
    ("star_no_root_half", "C[0] += 0.5 * f * d->c_per_um * L;", "C[0] += 0.0;", 0),
    ("star_manhattan_index", "double L = fabs(xd - xs) + fabs(yd - ys);", "double L = fabs(xd - xs) + fabs(yd - xs);", 0),
    ("rc_corner_scale", "double f = d->rc_scale ? d->rc_scale[corner] : 1.0;", "double f = 1.0;", 0),
    # O2 forward propagation
    ("wire_slew_no_var", "sqrt(sd * sd + Vn[p])", "sqrt(sd * sd)", 0),
    ("wire_at_no_delay", "at[IX(p, k, j)] = a + Dn[p];", "at[IX(p, k, j)] = a;", 0),
    ("neg_unate_as_pos", "case S_NEG: rf_in[0] = 1 - rf_out;", "case S_NEG: rf_in[0] = rf_out;", 0),
    ("non_unate_one_edge", "case S_NON: rf_in[0] = 0; rf_in[1] = 1; return 2;", "case S_NON: rf_in[0] = 0; rf_in[1] = 1; return 1;", 0),
    ("fwd_delay_table_rf", "sc * lut(d, t, s, rfo ? TB_DF : TB_DR, si, l, 0, 0);", "sc * lut(d, t, s, rfo ? TB_DR : TB_DF, si, l, 0, 0);", 0),
    ("fwd_slew_merge_late", "slew[IX(p, k, JJ(el, rfo))] = merge(cs, n, el, d->gamma_ns);", "slew[IX(p, k, JJ(el, rfo))] = merge(cs, n, 1, d->gamma_ns);", 0),
    ("merge_min_max_swap", "m = late ? fmax(m, x[i]) : fmin(m, x[i]);", "m = late ? fmin(m, x[i]) : fmax(m, x[i]);", 0),
    ("lse_early_sign", "return late ? m + gamma * log(s) : m - gamma * log(s);", "return m + gamma * log(s);", 0),
    ("fwd_lut_corner", "double sc = d->lut_scale ? d->lut_scale[kc] : 1.0;", "double sc = d->lut_scale ? d->lut_scale[0] : 1.0;", 0),
    ("pi_arrival_zero", "double a = (r == R_PI) ? d->pi_at_ns : 0.0;", "double a = 0.0;", 0),
    ("clock_slew_is_pi_slew", "d->pi_slew_ns : d->clk_slew_ns", "d->pi_slew_ns : d->pi_slew_ns", 0),
    # O4 required times, slack, WNS/TNS
    ("setup_sign", "rl[0] = rl[1] = d->period_ns - d->setup_ns;", "rl[0] = rl[1] = d->period_ns + d->setup_ns;", 0),
    ("hold_zero", "re[0] = re[1] = d->hold_ns;", "re[0] = re[1] = 0.0;", 0),
    ("rat_net_no_delay", "rat[IX(s, ks, JJ(1, rf))] - Dn[s]);", "rat[IX(s, ks, JJ(1, rf))]);", 0),
    ("rat_early_net_min", "re[rf] = fmax(re[rf], rat[IX(s, ks, JJ(0, rf))] - Dn[s]);", "re[rf] = fmin(re[rf], rat[IX(s, ks, JJ(0, rf))] - Dn[s]);", 0),
    ("rat_cell_early_slew", "slew[IX(p, k, JJ(1, ri))], load[z], 0, 0);", "slew[IX(p, k, JJ(0, ri))], load[z], 0, 0);", 0),
    ("rat_cell_rf_index", "rat[IX(z, k, JJ(1, rfo))] - dl);", "rat[IX(z, k, JJ(1, ri))] - dl);", 0),
    ("bwd_lut_corner", "double sc = d->lut_scale ? d->lut_scale[kc] : 1.0;", "double sc = d->lut_scale ? d->lut_scale[0] : 1.0;", 1),
    ("hold_slack_sign", "slack[IX(p, k, JJ(0, rf))] = at[IX(p, k, JJ(0, rf))] - rat[IX(p, k, JJ(0, rf))];",
     "slack[IX(p, k, JJ(0, rf))] = rat[IX(p, k, JJ(0, rf))] - at[IX(p, k, JJ(0, rf))];", 0),
    ("tns_sign", "if (ss < 0) { tns_s += ss;", "if (ss < 0) { tns_s -= ss;", 0),
    ("wns_max", "wns_s = fmin(wns_s, ss);", "wns_s = fmax(wns_s, ss);", 0),
    ("endpoint_best_edge", "double ss = fmin(slack[IX(p, k, JJ(1, 0))], slack[IX(p, k, JJ(1, 1))]);",
     "double ss = fmax(slack[IX(p, k, JJ(1, 0))], slack[IX(p, k, JJ(1, 1))]);", 0),
    ("cycle_not_detected", "if (mark[q] == 1) {", "if (mark[q] == 3) {", 0),
    # O7 Arnoldi reduced-order net model
    ("arn_tree_solve_path", "for (int32_t i = 1; i < n; ++i) x[i] = x[parent[i]] + R[i] * x[i];",
     "for (int32_t i = 1; i < n; ++i) x[i] = R[i] * x[i];", 0),
    ("arn_start_vector", "for (int32_t i = 1; i < n; ++i) V[i] = 1.0 / sqrt((double)m);",
     "for (int32_t i = 1; i < n; ++i) V[i] = (double)i / m;", 0),
    ("arn_gram_schmidt_sign", "for (int32_t i = 1; i < n; ++i) x[i] -= dot * V[p * n + i];",
     "for (int32_t i = 1; i < n; ++i) x[i] += dot * V[p * n + i];", 0),
    ("arn_edge_conductance", "g += dp * dr / R[i];", "g += dp * dr * R[i];", 0),
    ("arn_cap_weight", "cc += C[i] * V[p * n + i] * V[r * n + i];", "cc += V[p * n + i] * V[r * n + i];", 0),
    ("arn_root_conductance", "if (parent[i] == 0) s += V[p * n + i] / R[i];", "if (parent[i] == 0) s += V[p * n + i] * R[i];", 0),
    ("arn_cholesky_diag", "L[i * qq + i] = sqrt(s);", "L[i * qq + i] = s;", 0),
    ("arn_modal_inverse", "yinf[k] = s / lam[k];", "yinf[k] = s * lam[k];", 0),
    ("arn_half_threshold", "if (v >= 0.5 * vinf) hi = mid;", "if (v >= 0.4 * vinf) hi = mid;", 0),
    ("arn_model_switch", "if (d->net_model == 1 && (d->rc_ptr || steiner)) {", "if (d->net_model == 2 && d->rc_ptr) {", 0),
    # O8 timing exceptions
    ("exc_seed_not_masked", "if (src_on && !src_on[p])", "if (src_on && src_on[p] > 1)", 0),
    ("exc_first_group_wins", "if (!tag_of[p]) tag_of[p] = (int8_t)base[g];", "tag_of[p] = (int8_t)base[g];", 0),
    ("exc_false_still_checked", "late = INFINITY;   /* false path: no check */", "late = late;", 0),
    ("exc_multicycle_edge", "late = r == R_D ? M * T - d->setup_ns : M * T;", "late = r == R_D ? M * T : M * T;", 0),
    ("exc_to_list_ignored", "if (grp >= 0 && (applies_all || in_to[p])) {", "if (grp >= 0) {", 0),
    ("exc_tag_max_not_min", "ssm = fmin(ssm, ss);", "ssm = fmax(ssm, ss);", 0),
    # O6 smoothed objective and its adjoint
    ("tns_softplus_sign", "tns += -g * softplus(-seed[p] / g);", "tns += -g * softplus(seed[p] / g);", 0),
    ("seed_sigmoid_sign", "w_tns * sigmoid(-s / g)", "w_tns * sigmoid(s / g)", 0),
    ("adj_wire_slew_ratio", "asl[2 * drv + rf] += asl[2 * p + rf] * sd / sp;", "asl[2 * drv + rf] += asl[2 * p + rf] * sp / sd;", 0),
    ("adj_var_half", "aV[p] += asl[2 * p + rf] / (2.0 * sp);", "aV[p] += asl[2 * p + rf] / sp;", 0),
    ("adj_load_no_slew_term", "aload[p] += Aa * wa * sc * ddl[i] + As * ws * sc * sdl[i];", "aload[p] += Aa * wa * sc * ddl[i];", 0),
    ("adj_at_weight", "aat[2 * a + rf] += Aa * wa;", "aat[2 * a + rf] += Aa;", 0),
    ("adj_dDdL_half", "double dDdL = r * (cc * L + cp);", "double dDdL = r * (0.5 * cc * L + cp);", 0),
    ("adj_var_term", "aV[s] * 1e-12 * 2.0 * Draw * dDdL", "aV[s] * 1e-12 * Draw * dDdL", 0),
    ("adj_sink_sign", "if (cs >= 0) { grad_xy[2 * cs] -= dJdL * sx;", "if (cs >= 0) { grad_xy[2 * cs] += dJdL * sx;", 0),
    ("adj_y_uses_x", "double sx = (xd > xs) - (xd < xs), sy = (yd > ys) - (yd < ys);",
     "double sx = (xd > xs) - (xd < xs), sy = sx;", 0),
    # O8 -through stages
    ("thru_inflow_ignored", "const int inflow = adv && t >= 1 && ((adv[p] >> (t - 1)) & 1u);", "const int inflow = 0;", 0),
    ("thru_stay_always", "const int stay = !adv || !((adv[p] >> t) & 1u);", "const int stay = 1;", 0),
    ("thru_bwd_same_state", "const int32_t ks = adv && ((adv[s] >> t) & 1u) ? k + 1 : k;",
     "const int32_t ks = k;", 0),
    ("thru_action_first_stage", "if (t == base[g] + nthru[g]) grp = g;", "if (t == base[g]) grp = g;", 0),
    ("thru_adv_next_tag", "adv[p] |= 1u << (base[g] + j);", "adv[p] |= 1u << (base[g] + nthru[g]);", 0),
    # O9 Steiner tree RC from positions
    ("steiner_nm_truncates", "return (int64_t)lrintf(p);", "return (int64_t)p;", 0),
    ("steiner_median_is_middle_arg", "if ((a <= b && b <= c) || (c <= b && b <= a)) return b;", "return b;", 0),
    ("steiner_gain_drops_w", " - mdist(mx, my, x[w], y[w]);", ";", 0),
    ("steiner_new_node_drops_w", "ADJ(s, bw) = ADJ(bw, s) = 1;", "ADJ(s, bw) = ADJ(bw, s) = 0;", 0),
    ("steiner_bfs_old_parent", "parent[nodes] = newid[a];", "parent[nodes] = a;", 0),
    ("steiner_no_merge_same_point", "if (x[b] == x[a] && y[b] == y[a]) {", "if (0) {", 0),
    ("steiner_ry_uses_rx", "R[i] = f * (rx * lx + ry * ly);", "R[i] = f * (rx * lx + rx * ly);", 0),
    ("steiner_no_parent_half_cap", "C[par[i]] += 0.5 * cw;", "C[par[i]] += 0.0 * cw;", 0),
    ("steiner_no_scale", "double cw = f * (cx * lx + cy * ly);", "double cw = (cx * lx + cy * ly);", 0),
    ("exc_maxdelay_no_setup", "late = r == R_D ? V - d->setup_ns : V;", "late = V;", 0),
    ("exc_mindelay_no_hold", "early = r == R_D ? V + d->hold_ns : V;", "early = V;", 0),
    ("exc_maxdelay_as_multicycle", "late = r == R_D ? V - d->setup_ns : V;", "late = r == R_D ? V * T - d->setup_ns : V * T;", 0),
    # O6 on Steiner trees: the RC-tree adjoint and the tree-held-fixed chain to positions
    ("rcadj_no_var_D", "db[i] = Dbar[i] - 2.0 * D[i] * Vbar[i] + mb[i] * C[i];", "db[i] = Dbar[i] + mb[i] * C[i];", 0),
    ("rcadj_beta_factor", "bb[i] = 2.0 * Vbar[i];", "bb[i] = Vbar[i];", 0),
    ("rcadj_no_load", "cb[i] = (i ? db[i] * R[i] + cb[parent[i]] : Lbar);", "cb[i] = (i ? db[i] * R[i] + cb[parent[i]] : 0.0);", 0),
    ("rcadj_moment_down_order", "mb[i] = (i ? bb[i] * R[i] : 0.0) + (i ? mb[parent[i]] : 0.0);", "mb[i] = (i ? bb[i] * R[i] : 0.0);", 0),
    ("stgrad_no_parent_cap", "0.5 * cx * (Cb[i] + Cb[p])", "0.5 * cx * Cb[i]", 0),
    ("stgrad_y_uses_rx", "f * (ry * Rb[i] + 0.5 * cy", "f * (rx * Rb[i] + 0.5 * cy", 0),
    ("stgrad_parent_sign", "if (cq >= 0) grad_xy[2 * cq + ax] -= gl[ax] * sg;", "if (cq >= 0) grad_xy[2 * cq + ax] += gl[ax] * sg;", 0),
    ("stgrad_sink_var_scale", "Vb[pnode[k]] += 1e-12 * aV[s];", "Vb[pnode[k]] += 1e-6 * aV[s];", 0),
    # O6 smoothed merges with several candidates (a single candidate is unchanged by each)
    ("lse_half_gamma", "return late ? m + gamma * log(s) : m - gamma * log(s);",
     "return late ? m + 0.5 * gamma * log(s) : m - 0.5 * gamma * log(s);", 0),
    ("lse_max_only", "for (int i = 0; i < n; ++i) s += exp((late ? (x[i] - m) : (m - x[i])) / gamma);",
     "for (int i = 0; i < n; ++i) s += (x[i] == m);", 0),
    ("lse_flipped_offsets", "s += exp((late ? (x[i] - m) : (m - x[i])) / gamma);",
     "s += exp((late ? (m - x[i]) : (x[i] - m)) / gamma);", 0),
]

# Mutants of the Python side of the oracle (oracle/__init__.py): the path
# reports with a per-endpoint limit
PY_SRC = os.path.join(ROOT, "oracle", "__init__.py")
PY_MUTANTS = [
    # the arc delay at the early slew instead of the late one: invisible when delays do not depend on slew
    ("nworst_early_slew", "slew[a, 2 + rfi], load[p])[0]", "slew[a, rfi], load[p])[0]", 0),
    ("nworst_input_load", "slew[a, 2 + rfi], load[p])[0]", "slew[a, 2 + rfi], load[a])[0]", 0),
    ("nworst_endpoint_edge", "heapq.heappush(heap, (float(sl[2 + rf]), seq, rf, ()))",
     "heapq.heappush(heap, (float(sl[2]), seq, rf, ()))", 0),
]


def _mutate(text: str, old: str, new: str, nth: int) -> str:
    pos = -1
    for _ in range(nth + 1):
        pos = text.find(old, pos + 1)
        assert pos >= 0, "mutation site not found: %r (occurrence %d)" % (old, nth)
    return text[:pos] + new + text[pos + len(old):]


def test_mutation_sites_exist():
    for src, muts in ((SRC, MUTANTS), (PY_SRC, PY_MUTANTS)):
        text = open(src).read()
        names = [m[0] for m in muts]
        assert len(set(names)) == len(names)
        for _, old, new, nth in muts:
            assert _mutate(text, old, new, nth) != text


@pytest.mark.parametrize("name,old,new,nth", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_reject_mutant(name, old, new, nth, tmp_path):
    src = tmp_path / "sta_oracle.c"
    src.write_text(_mutate(open(SRC).read(), old, new, nth))
    env = dict(os.environ, ORACLE_MUTANT_SRC=str(src))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "tests._oracle_mutant"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert "liboracle_mutant" not in r.stderr or r.returncode != 4, r.stderr[-2000:]
    assert r.returncode == 1, "mutant %s survived the pins (exit %d):\n%s" % (name, r.returncode,
                                                                            r.stdout[-1500:])


@pytest.mark.parametrize("name,old,new,nth", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_reject_python_mutant(name, old, new, nth, tmp_path):
    src = tmp_path / "oracle_mutant.py"
    src.write_text(_mutate(open(PY_SRC).read(), old, new, nth))
    env = dict(os.environ, ORACLE_MUTANT_PY=str(src))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "tests._oracle_mutant"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 1, "mutant %s survived the pins (exit %d):\n%s" % (name, r.returncode,
                                                                            r.stdout[-1500:])
