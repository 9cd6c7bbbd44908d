"""Planted mistakes in the oracle fail its pins.

Each case below copies the oracle's C source, makes one plausible mistake in the copy (a dropped
term, a flipped sign or comparison, a transposed index, an off-by-one), builds the copy with the
oracle's own gcc command and runs tests/test_oracle_pins.py against that library in a child
process.  The pins pass on an unmodified copy and must fail on every mutant, as test failures
(pytest exit status 1), not as a crash.  The oracle's own source and library are never touched.
"""
import concurrent.futures as cf
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "kb_oracle.c")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (name, [(text in the source, replacement, occurrences)]); every occurrence is replaced, and the
# count must match so that an edit of the source cannot silently disarm a mutant.
MUTANTS = [
    # erfinv and the sigma_G coefficient (Section 3.1, Eqs. 2-5)
    ("erfinv_bisects_the_wrong_way",
     [("if (erf(mid) < y) lo = mid;", "if (erf(mid) > y) lo = mid;", 1)]),
    ("coeff_drops_sqrt2",
     [("1.0 / (sqrt(2.0) * (kbo_erfinv", "1.0 / (1.0 * (kbo_erfinv", 1)]),
    ("coeff_quartiles_swapped",
     [("(kbo_erfinv(2.0 * q_hi - 1.0) - kbo_erfinv(2.0 * q_lo - 1.0))",
       "(kbo_erfinv(2.0 * q_lo - 1.0) - kbo_erfinv(2.0 * q_hi - 1.0))", 1)]),
    # percentiles (linear interpolation between order statistics)
    ("percentile_lower_order_statistic",
     [("return s[lo] + (h - (double)lo) * (s[hi] - s[lo]);", "return s[lo];", 1)]),
    ("percentile_rank_n_not_n_minus_1",
     [("double h = (double)(n - 1) * q;", "double h = (double)n * q;", 1)]),
    # the clip (Section 3.1)
    ("clip_exclusive_bounds",
     [("a[i] >= lower && a[i] <= upper", "a[i] > lower && a[i] < upper", 1)]),
    ("clip_centre_is_lower_quartile",
     [("double x_mid = kbo_percentile_sorted(s, n, q_mid);",
       "double x_mid = kbo_percentile_sorted(s, n, q_lo);", 1)]),
    ("clip_upper_side_only",
     [("double lower = x_mid - n_sigma * sigma_g,", "double lower = -INFINITY,", 1)]),
    ("clip_lower_side_only",
     [("upper = x_mid + n_sigma * sigma_g;", "upper = INFINITY;", 1)]),
    ("clip_half_width_one_sigma",
     [("double lower = x_mid - n_sigma * sigma_g, upper = x_mid + n_sigma * sigma_g;",
       "double lower = x_mid - sigma_g, upper = x_mid + sigma_g;", 1)]),
    ("clip_width_fixed_at_two",
     [("double lower = x_mid - n_sigma * sigma_g, upper = x_mid + n_sigma * sigma_g;",
       "double lower = x_mid - 2.0 * sigma_g, upper = x_mid + 2.0 * sigma_g;", 1)]),
    ("clip_centre_fixed_at_the_median",
     [("double x_mid = kbo_percentile_sorted(s, n, q_mid);",
       "double x_mid = kbo_percentile_sorted(s, n, 0.5);", 1)]),
    ("clip_quartiles_fixed",
     [("double sigma_g = kbo_sigma_g_coeff(q_lo, q_hi) * (x_hi - x_lo);",
       "double sigma_g = kbo_sigma_g_coeff(0.25, 0.75) * (x_hi - x_lo);", 1)]),
    # the clip-bound margin of reading R6 (test infrastructure of the parity comparison)
    ("clip_margin_upper_bound_only",
     [("double d = fmin(fabs(a[i] - lower), fabs(a[i] - upper));",
       "double d = fabs(a[i] - upper);", 1)]),
    ("clip_margin_scale_sigma_only",
     [("double scale = fmax(fmax(sg, fabs(med)), 1e-30);", "double scale = fmax(sg, 1e-30);", 1)]),
    # track rounding
    ("track_round_half_even", [("return (int32_t)floorf(e);", "return (int32_t)rintf(d);", 1)]),
    ("track_truncates", [("return (int32_t)floorf(e);", "return (int32_t)e;", 1)]),
    ("track_time_reversed", [("float dt = (float)(t - t0);", "float dt = (float)(t0 - t);", 1)]),
    ("track_time_not_from_the_first_epoch",
     [("offx[(size_t)j * T + t] = track_offset(vx[j], times[t], times[0]);",
       "offx[(size_t)j * T + t] = track_offset(vx[j], times[t], 0.0);", 1),
      ("offy[(size_t)j * T + t] = track_offset(vy[j], times[t], times[0]);",
       "offy[(size_t)j * T + t] = track_offset(vy[j], times[t], 0.0);", 1)]),
    ("track_time_difference_in_float32",
     [("float dt = (float)(t - t0);", "float dt = (float)t - (float)t0;", 1)]),
    ("track_y_uses_vx",
     [("offy[(size_t)j * T + t] = track_offset(vy[j]", "offy[(size_t)j * T + t] = track_offset(vx[j]",
       1)]),
    # psi / phi (Section 3)
    ("psi_unweighted", [("s_psi += w * (double)img[i] * p;", "s_psi += (double)img[i] * p;", 2)]),
    ("phi_psf_not_squared", [("s_phi += w * p * p;", "s_phi += w * p;", 2)]),
    ("weight_inverse_sigma",
     [("double w = 1.0 / (double)var[i];", "double w = 1.0 / sqrt((double)var[i]);", 2)]),
    ("weight_of_the_centre_pixel",
     [("double w = 1.0 / (double)var[i];", "double w = 1.0 / (double)var[o];", 2)]),
    ("psf_convolved_not_correlated",
     [("P[(uy + r) * k + (ux + r)]", "P[(r - uy) * k + (r - ux)]", 2)]),
    ("psf_transposed", [("P[(uy + r) * k + (ux + r)]", "P[(ux + r) * k + (uy + r)]", 2)]),
    ("masked_neighbours_used",
     [("            if (pixel_masked(img, var, mask, i)) continue;\n            double w",
       "            double w", 1),
      ("        if (pixel_masked(img, var, mask, i)) continue;\n        double w",
       "        double w", 1)]),
    ("sampled_psi_phi_use_masked_neighbours",
     [("        if (pixel_masked(img, var, mask, i)) continue;\n        double w",
       "        double w", 1)]),
    ("masked_centre_not_zeroed",
     [("if (pixel_masked(img, var, mask, o)) { psi[o] = 0.0; phi[o] = 0.0; continue; }", "", 1),
      ("if (pixel_masked(img, var, mask, o)) { psi[s] = 0.0; phi[s] = 0.0; continue; }", "", 1)]),
    # one trajectory: gather, clip, clipped sums (Section 3, 3.1)
    ("lh_without_sqrt", [("res->lh = s_psi / sqrt(s_phi);", "res->lh = s_psi / s_phi;", 1)]),
    ("flux_with_sqrt", [("res->flux = s_psi / s_phi;", "res->flux = s_psi / sqrt(s_phi);", 1)]),
    ("clip_quantity_swapped",
     [("buf_a[n] = clip_on ? p / sqrt(f) : p / f;", "buf_a[n] = clip_on ? p / f : p / sqrt(f);", 1)]),
    ("sums_ignore_the_clip", [("if (!buf_keep[i]) continue;", "", 1)]),
    ("zero_phi_epoch_valid", [("if (!(f > 0.0) || !isfinite(p)", "if (!(f >= 0.0) || !isfinite(p)", 1)]),
    ("min_obs_strict", [("if (n < min_obs || n == 0) return;", "if (n <= min_obs || n == 0) return;", 1)]),
    ("x_wraps_into_the_next_row",
     [("int x = x0 + ox[t], y = y0 + oy[t];\n    if (x < 0 || x >= W || y < 0 || y >= H) continue;",
       "int x = x0 + ox[t], y = y0 + oy[t];\n    if (y < 0 || y >= H) continue;", 1)]),
    ("nkept_counts_valid_epochs", [("res->nkept = nk;", "res->nkept = n;", 1)]),
    ("nvalid_counts_kept_epochs", [("res->nkept = nk;", "res->nkept = nk; res->nvalid = nk;", 1)]),
    ("kept_mask_bit_off_by_one",
     [("res->mask[buf_t[i] >> 5] |= 1u << (buf_t[i] & 31);",
       "res->mask[buf_t[i] >> 5] |= 1u << ((buf_t[i] + 1) & 31);", 1)]),
    # threshold and per-pixel top-K (Section 3.2)
    ("threshold_exclusive", [("!(r.lh >= lh_min)", "!(r.lh > lh_min)", 1)]),
    ("top_k_ascending", [("(lh[s] > r.lh ||", "(lh[s] < r.lh ||", 1)]),
    ("ties_to_the_higher_index", [("(lh[s] == r.lh && ix[s] < j)", "(lh[s] == r.lh && ix[s] > j)", 1)]),
    ("top_k_shift_drops_a_slot", [("for (int m = K - 1; m > s; --m) {", "for (int m = K - 1; m > s + 1; --m) {", 1)]),
    ("window_axes_swapped", [("int x0 = x_lo + p % ww, y0 = y_lo + p / ww;",
                              "int x0 = x_lo + p / ww, y0 = y_lo + p % ww;", 1)]),
    # coadded stamps (Section 3.3)
    ("stamp_mean_over_all_epochs", [("out_mean[o] = s / m;", "out_mean[o] = s / T;", 1)]),
    ("stamp_even_median_upper",
     [("0.5 * (vals[m / 2 - 1] + vals[m / 2])", "vals[m / 2]", 1)]),
    ("stamp_ignores_the_kept_mask", [("if (keep_mask && !((keep_mask", "if (0 && keep_mask && !((keep_mask", 1)]),
    ("stamp_uses_masked_pixels",
     [("if (pixel_masked(img, var, mask, i)) continue;\n            vals[m++]", "vals[m++]", 1)]),
    ("stamp_empty_pixel_zero_not_nan",
     [("if (m == 0) { out_mean[o] = NAN; out_median[o] = NAN; continue; }",
       "if (m == 0) { out_mean[o] = 0.0; out_median[o] = 0.0; continue; }", 1)]),
    ("stamp_kept_mask_bit_off_by_one",
     [("(keep_mask[(size_t)c * mw + (t >> 5)] >> (t & 31)) & 1u",
       "(keep_mask[(size_t)c * mw + (t >> 5)] >> ((t + 1) & 31)) & 1u", 1)]),
    ("stamp_flipped", [("int x = x0[c] + ox[t] + sx, y = y0[c] + oy[t] + sy;",
                        "int x = x0[c] + ox[t] - sx, y = y0[c] + oy[t] - sy;", 1)]),
    # sub-pixel evaluation, its gradient and the VJP
    ("bilinear_weights_transposed",
     [("double top = v00 + ax * (v01 - v00), bot = v10 + ax * (v11 - v10);",
       "double top = v00 + ay * (v01 - v00), bot = v10 + ay * (v11 - v10);", 1),
      ("return top + ay * (bot - top);", "return top + ax * (bot - top);", 1)]),
    ("bilinear_dx_rows_swapped",
     [("*dx = (1.0 - ay) * (v01 - v00) + ay * (v11 - v10);",
       "*dx = ay * (v01 - v00) + (1.0 - ay) * (v11 - v10);", 1)]),
    ("gradient_drops_dt",
     [("dPs[2] += gpx * dt; dPs[3] += gpy * dt;", "dPs[2] += gpx; dPs[3] += gpy;", 2)]),
    ("subpixel_time_not_from_the_first_epoch",
     [("double dt = times[t] - times[0];", "double dt = times[t];", 3)]),
    ("vjp_taps_at_transposed_offsets",
     [("int xx = ix + (k & 1), yy = iy + (k >> 1);", "int xx = ix + (k >> 1), yy = iy + (k & 1);", 1)]),
    ("gradient_phi_term_sign",
     [("double dL_dPh = -0.5 * Ps / (Ph * sqrt(Ph));", "double dL_dPh = 0.5 * Ps / (Ph * sqrt(Ph));", 1)]),
    ("vjp_drops_the_alpha_phi_term",
     [("double cPh = -0.5 * gL * Ps / (Ph * sqrt(Ph)) - gA * Ps / (Ph * Ph);",
       "double cPh = -0.5 * gL * Ps / (Ph * sqrt(Ph));", 1)]),
    ("vjp_alpha_psi_term_squared",
     [("double cPs = gL / sqrt(Ph) + gA / Ph;", "double cPs = gL / sqrt(Ph) + gA / (Ph * Ph);", 1)]),
    ("vjp_params_overwritten_not_accumulated",
     [("grad_params[i] += cPs * dPs[i] + cPh * dPh[i];", "grad_params[i] = cPs * dPs[i] + cPh * dPh[i];",
       1)]),
    ("vjp_image_taps_overwritten_not_accumulated",
     [("if (grad_psi) grad_psi[i] += cPs * w;", "if (grad_psi) grad_psi[i] = cPs * w;", 1)]),
    ("vjp_tap_weights_transposed",
     [("double w = ((k & 1) ? ax : 1.0 - ax) * ((k >> 1) ? ay : 1.0 - ay);",
       "double w = ((k & 1) ? ay : 1.0 - ay) * ((k >> 1) ? ax : 1.0 - ax);", 1)]),
    # Adam refinement
    ("adam_without_bias_correction",
     [("double mh = m[i] / (1.0 - b1k), vh = v[i] / (1.0 - b2k);", "double mh = m[i], vh = v[i];", 1)]),
    ("adam_second_moment_decay_uses_beta1", [("b2k *= b2;", "b2k *= b1;", 1)]),
    ("adam_descends", [("params[i] += lr * mh / (sqrt(vh) + eps);", "params[i] -= lr * mh / (sqrt(vh) + eps);", 1)]),
    ("adam_rates_swapped", [("double lr = i < 2 ? lr_pos : lr_vel;", "double lr = i < 2 ? lr_vel : lr_pos;", 1)]),
    ("adam_second_moment_unsquared",
     [("v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];", "v[i] = b2 * v[i] + (1.0 - b2) * fabs(g[i]);", 1)]),
    # stamp moments and the filter (Section 3.3)
    ("moments_axes_swapped", [("double dx = col - r, dy = row - r;", "double dx = row - r, dy = col - r;", 1)]),
    ("moments_without_the_minimum", [("double w = v - lo;", "double w = v;", 1)]),
    ("filter_limits_of_xx_yy_swapped", [("out[4] < lim[3] && out[5] < lim[4]", "out[4] < lim[4] && out[5] < lim[3]", 1)]),
    ("filter_xy_without_abs", [("fabs(out[3]) < lim[2]", "out[3] < lim[2]", 1)]),
    ("filter_x_without_abs", [("fabs(out[1]) < lim[0]", "out[1] < lim[0]", 1)]),
    ("filter_y_without_abs", [("fabs(out[2]) < lim[1]", "out[2] < lim[1]", 1)]),
    ("filter_yy_not_strict", [("out[5] < lim[4]", "out[5] <= lim[4]", 1)]),
    # clustering
    ("cluster_against_any_earlier", [("if (keep[j] && kbo_dup(", "if (kbo_dup(", 1)]),
    ("cluster_start_only", [("return dx1 * dx1 + dy1 * dy1 <= r2;", "return 1;", 1)]),
    ("cluster_end_only", [("if (dx0 * dx0 + dy0 * dy0 > r2) return 0;", "", 1)]),
    ("cluster_ignores_valid", [("if (valid && !valid[i]) continue;", "", 1)]),
    ("cluster_keeps_placeholders",
     [("if (x0[i] < 0 || x0[i] >= (1 << 20) || y0[i] < 0 || y0[i] >= (1 << 20)) continue;", "", 1)]),
    ("cluster_radius_not_squared", [("double r2 = r * r;", "double r2 = r;", 1)]),
    ("cluster_end_y_uses_vx",
     [("(double)vy[i] * dt", "(double)vx[i] * dt", 1), ("(double)vy[j] * dt", "(double)vx[j] * dt", 1)]),
    ("cluster_last_representative", [("for (int j = 0; j < i && found < 0; ++j)", "for (int j = 0; j < i; ++j)", 1)]),
]

_CHILD = r"""
import sys
sys.path.insert(0, sys.argv[1])
import oracle.build
oracle.build.build = lambda force=False: sys.argv[2]
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", sys.argv[3]]))
"""


def _mutate(text, edits):
    for old, new, count in edits:
        found = text.count(old)
        assert found == count, f"{old!r}: {found} occurrences, expected {count}"
        text = text.replace(old, new)
    return text


def _run(name, text, tmp):
    from oracle import build as oracle_build
    src = os.path.join(tmp, f"{name}.c")
    lib = os.path.join(tmp, f"lib_{name}.so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(oracle_build.command(src, lib), check=True, capture_output=True)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", _CHILD, ROOT, lib, PINS], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    failed = re.findall(r"FAILED \S+::(\w+(?:\[[^\]]*\])?)", r.stdout)
    return r.returncode, failed, r.stdout[-2000:] + r.stderr[-2000:]


def test_pins_fail_on_every_planted_mistake(tmp_path):
    with open(SRC) as f:
        text = f.read()
    mutated = {name: _mutate(text, edits) for name, edits in MUTANTS}
    assert len(mutated) == len(MUTANTS), "mutant names must be unique"
    jobs = [("unmodified", text)] + list(mutated.items())
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = dict(zip([n for n, _ in jobs],
                           ex.map(lambda job: _run(job[0], job[1], str(tmp_path)), jobs)))
    rc, _, log = results.pop("unmodified")
    assert rc == 0, "the pins must pass on an unmodified copy of the oracle:\n" + log
    survivors = [n for n, (rc, _, _) in results.items() if rc == 0]
    crashed = {n: rc for n, (rc, _, _) in results.items() if rc not in (0, 1)}
    assert not survivors, f"mutants the pins do not catch: {survivors}"
    assert not crashed, f"mutants that crash instead of failing a pin: {crashed}"
