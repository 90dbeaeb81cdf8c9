"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one of them (CPU only; the real oracle is never modified)."""
import pytest

import oracle
import pins

MUTANTS = {
    "feq_quadratic_coeff": ("4.5 * cu * cu", "4.0 * cu * cu"),
    "feq_uu_sign": ("- 1.5 * uu", "+ 1.5 * uu"),
    "weight_d3q15_diag": ("1.0 / 72.0", "1.0 / 64.0"),
    "d3q19_direction_order": ("{1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},",
                              "{1, 0, -1}, {-1, 0, -1}, {1, 0, 1}, {-1, 0, 1},"),
    "bounce_back_same_dir": ("fout[(int64_t)L.opp[i] * n + x] = fs;",
                             "fout[(int64_t)i * n + x] = fs;"),
    "relaxation_tau_times": ("(g[i] - feq[i]) / tau", "(g[i] - feq[i]) * tau"),
    "collision_sign": ("g[i] - (g[i] - feq[i]) / tau", "g[i] + (g[i] - feq[i]) / tau"),
    "iolet_time_plus_one": ("double feq_k[19];\n                double rk = iolet_rho(k, t, rho_mean",
                            "double feq_k[19];\n                double rk = iolet_rho(k, t + 1, rho_mean"),
    "adj_iolet_time": ("double rk = iolet_rho(k, t, rho_mean, amp, period, phase);\n                double feq_k[19], d[3];",
                       "double rk = iolet_rho(k, t + 1, rho_mean, amp, period, phase);\n                double feq_k[19], d[3];"),
    "iolet_wrong_direction": ("= feq_k[L.opp[i]];", "= feq_k[i];"),
    "wss_factor": ("double coef = -(1.0 - 1.0 / (2.0 * tau));\n        double tr[3];",
                   "double coef = -(1.0 - 1.0 / tau);\n        double tr[3];"),
    "objective_wss_factor": ("double coef = -(1.0 - 1.0 / (2.0 * tau));\n        double tr[3], tn",
                             "double coef = -(1.0 - 1.0 / tau);\n        double tr[3], tn"),
    "velocity_not_divided": ("u[a] = j[a] / r;", "u[a] = j[a];"),
    "no_periodic_wrap": ("if (periodic && periodic[a] > 0) y[a] =", "if (0) y[a] ="),
    "iolet_id_off_by_one": ("(k >= 0 ? 2 + k : 1)", "(k >= 0 ? 1 + k : 1)"),
    "adj_relaxation_sign": ("(1.0 - om) * ls[(int64_t)j * n + x]", "(1.0 + om) * ls[(int64_t)j * n + x]"),
    "adj_dfeq_du_coeff": ("9.0 * cu * L->e[i][a]", "4.5 * cu * L->e[i][a]"),
    "adj_drho_k_scale": ("lo * feq_k[oi] / rk, dmean", "lo * feq_k[oi], dmean"),
    "adj_phase_cos": ("dphase[k] += d * amp[k] * cos(arg);", "dphase[k] += d * amp[k] * sin(arg);"),
    "adj_tau_power": ("(g[i] - feq[i]) / (tau * tau);", "(g[i] - feq[i]) / tau;"),
    "adj_wall_lambda": ("const double lo = lam_next[o];\n                if (qw == 0.5)",
                        "const double lo = lam_next[(int64_t)i * n + x];\n                if (qw == 0.5)"),
    "adj_velocity_term": ("double dj = (L.e[j][c] - u[c]) / rho;", "double dj = L.e[j][c] / rho;"),
    "ladd_factor": ("fs - 6.0 * L.w[i] * rho * cub;", "fs - 3.0 * L.w[i] * rho * cub;"),
    "ladd_sign": ("fs - 6.0 * L.w[i] * rho * cub;", "fs + 6.0 * L.w[i] * rho * cub;"),
    "ladd_weight_ignored": ("double wx = weight ? weight[x] : 1.0;\n                double cub", "double wx = 1.0;\n                double cub"),
    "ladd_normal_index": ("wx * U * io_normal[3 * k + a];", "wx * U * io_normal[a];"),
    "render_dt_dropped": ("double a = e[3] * l;", "double a = e[3];"),
    "render_no_transmittance": ("C[c] += (1.0 - A) * a * e[c];", "C[c] += a * e[c];"),
    "render_lut_index_scale": ("0.0, 1.0) * 255.0;", "0.0, 1.0) * 254.0;"),
    "render_tf_offset_sign": ("clampd((v - tf_offset) * tf_scale", "clampd((v + tf_offset) * tf_scale"),
    "render_trilinear_x": ("double c00 = V(i0, j0, k0) * (1 - fx) + V(i1, j0, k0) * fx;",
                           "double c00 = V(i0, j0, k0) * fx + V(i1, j0, k0) * (1 - fx);"),
    "render_trilinear_z": ("return c0 * (1 - fz) + c1 * fz;", "return c0 * fz + c1 * (1 - fz);"),
    "render_right_flipped": ("for (int a = 0; a < 3; ++a) r[a] /= rn;", "for (int a = 0; a < 3; ++a) r[a] /= -rn;"),
    "render_up_flipped": ("u[1] = r[2] * f[0] - r[0] * f[2];", "u[1] = r[0] * f[2] - r[2] * f[0];"),
    "render_full_fov": ("tan(0.5 * fov_y)", "tan(fov_y)"),
    "render_pixel_corner": ("((px + 0.5) / W * 2.0 - 1.0)", "((px + 0.0) / W * 2.0 - 1.0)"),
    "render_aspect_inverted": ("* th * aspect;", "* th / aspect;"),
    "render_sample_at_start": ("double t = t0 + 0.5 * l;", "double t = t0;"),
    "render_last_segment_full": ("double l = tf - t0 < dt ? tf - t0 : dt;", "double l = dt;"),
    "render_behind_eye": ("if (tn < 0.0) tn = 0.0;", "if (tn < -1e300) tn = 0.0;"),
    "render_no_early_stop": ("if (t0 >= tf || A >= a_stop) break;", "if (t0 >= tf || A >= 1.0) break;"),
    "render_no_alpha_clamp": ("if (a > 1.0) a = 1.0;", "if (a > 9.0) a = 1.0;"),
    "bfl_weights_swapped": ("val = 2.0 * qw * fs + (1.0 - 2.0 * qw) * post_collision(",
                            "val = (1.0 - 2.0 * qw) * fs + 2.0 * qw * post_collision("),
    "bfl_upstream_population": ("post_collision(&L, f, n, nbr[ob], i, tau)",
                                "post_collision(&L, f, n, nbr[ob], L.opp[i], tau)"),
    "bfl_high_own_population": ("(1.0 - 1.0 / (2.0 * qw)) * fsa[L.opp[i]]", "(1.0 - 1.0 / (2.0 * qw)) * fsa[i]"),
    "bfl_high_factor": ("fs / (2.0 * qw) +", "fs / qw +"),
    "bfl_collision_tau": ("return h[i] - (h[i] - he[i]) / tau;", "return h[i] - (h[i] - he[i]) * tau;"),
    "mass_direction_dropped": ("for (int i = 0; i < q; ++i) m += f[(int64_t)i * n + x];",
                               "for (int i = 1; i < q; ++i) m += f[(int64_t)i * n + x];"),
    "mass_last_site_dropped": ("for (int64_t x = 0; x < n; ++x)\n        for (int i = 0; i < q; ++i) m +=",
                               "for (int64_t x = 0; x < n - 1; ++x)\n        for (int i = 0; i < q; ++i) m +="),
    "mass_plane_stride": ("m += f[(int64_t)i * n + x];", "m += f[(int64_t)i * q + x];"),
    "adj_bfl_upstream_weight": ("ls[(int64_t)i * n + nbr[o]] += (1.0 - 2.0 * qw) * lo;",
                                "ls[(int64_t)i * n + nbr[o]] += 2.0 * qw * lo;"),
    "adj_bfl_own_weight": ("ls[(int64_t)i * n + x] += 2.0 * qw * lo;", "ls[(int64_t)i * n + x] += lo;"),
    "adj_bfl_high_second_term": ("ls[o] += (1.0 - 1.0 / (2.0 * qw)) * lo;", "ls[o] += 0.0 * lo;"),
    "adj_velocity_rho_sign": ("gv[x] += -6.0 * L.w[i] * wx * U * cn * lo;", "gv[x] += 6.0 * L.w[i] * wx * U * cn * lo;"),
    "adj_velocity_param_rho": ("-6.0 * L.w[i] * rho * wx * cn * lo, dmean", "-6.0 * L.w[i] * wx * cn * lo, dmean"),
    "adj_velocity_term_dropped": ("om * s + h + gv[x];", "om * s + h;"),
    "adj_wss_M": ("lam[(int64_t)j * n + x] += scale * m[x] * coef * (M[j] - s);",
                  "lam[(int64_t)j * n + x] += scale * m[x] * coef * (M[j] + s);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = oracle.source()
    assert src.count(old) == 1, "mutation anchor must be unique: %r" % old
    o = oracle.variant(src.replace(old, new), str(tmp_path))
    caught = []
    for pin_name, fn in pins.ALL_FAST:
        try:
            fn(o)
        except (AssertionError, ValueError, FloatingPointError) as exc:
            caught.append(pin_name)
            break
    assert caught, "no pin caught the planted mistake %s" % name
