"""Planted mistakes in the oracle must trip at least one pin.

Each case copies rvh_oracle.c, applies one plausible slip (a dropped term, a
wrong sign or index, a transposed operand, an off-by-one in the draw, the
wrong tie-break), compiles the copy on the CPU and runs the pins of
oracle_pins.py against it.  A mutant that passes every pin would mean the
pins cannot tell that slip from the real method.
"""
import os
import subprocess

import pytest

import oracle
from tests import oracle_pins

MUTANTS = {
    "line_median_nan_first": ("return isnan(x) - isnan(y);", "return isnan(y) - isnan(x);"),
    "line_extreme_keeps_nan": ("vmin = fmin(vmin, w[q]);", "vmin = vmin < w[q] ? vmin : w[q];"),
    "first_cluster_ignored": ("oracle_draw(p->seed, p->first_cluster + ci, h, n, k, qs)",
                              "oracle_draw(p->seed, ci, h, n, k, qs)"),
    "fragile_margin_dropped": ("double amp = 1e-14 * (1.0 + 1.0 / fabs(hyp_det[h]));", "double amp = 0.0;"),
    "fragile_margin_too_wide": ("double amp = 1e-14 * (1.0 + 1.0 / fabs(hyp_det[h]));",
                                "double amp = 1e-8 * (1.0 + 1.0 / fabs(hyp_det[h]));"),
    "fragile_det_margin_dropped": ("int frag = min_det_margin < 1e-13;", "int frag = 0;"),
    "det2_sign": ("return fma(x, w, -(y * z));", "return fma(x, w, (y * z));"),
    "det3_cofactor_sign": ("fma(-m0[1], k1, m0[0] * k0)", "fma(m0[1], k1, m0[0] * k0)"),
    "det3_minor_index": ("double k1 = det2(m1[0], m1[2], m2[0], m2[2]);",
                         "double k1 = det2(m1[0], m1[2], m2[0], m2[1]);"),
    "residual_transposed": ("return w - fma(v[0], a[0], v[1] * a[1]);",
                            "return w - fma(v[0], a[1], v[1] * a[0]);"),
    "residual_dropped_z": ("return w - fma(v[0], a[0], fma(v[1], a[1], v[2] * a[2]));",
                           "return w - fma(v[0], a[0], v[1] * a[1]);"),
    "rows_swapped": ("double c = cos(t), s = sin(t);", "double c = sin(t), s = cos(t);"),
    "elev_row": ("a[3 * q + 2] = se;", "a[3 * q + 2] = ce;"),
    "philox_no_key_bump": ("k0 += weyl0;", "k0 += 0u;"),
    "philox_swapped_words": ("uint32_t y1 = lo1;", "uint32_t y1 = lo0;"),
    "draw_skip_off_by_one": ("if (q1 >= q0) q1 += 1u;", "if (q1 > q0) q1 += 1u;"),
    "draw3_skip_order": ("if (q2 >= lo) q2 += 1u;\n    if (q2 >= hi) q2 += 1u;",
                         "if (q2 >= hi) q2 += 1u;\n    if (q2 >= lo) q2 += 1u;"),
    "tiebreak_last": ("        if (count > best_count) {\n          best_count = count;\n          best = h;\n        }\n"
                      "      } while (0);",
                      "        if (count >= best_count) {\n          best_count = count;\n          best = h;\n        }\n"
                      "      } while (0);"),
    "line_threshold_reports_median": ("      if (threshold) threshold[oi] = thresh;",
                                      "      if (threshold) threshold[oi] = med;"),
    "line_tiebreak_last": ("          if (count > best_count) {\n            best_count = count;",
                           "          if (count >= best_count) {\n            best_count = count;"),
    "refine_wrong_product": ("G[r][c] = fma(aq[r], aq[c], G[r][c]);",
                             "G[r][c] = fma(aq[r], aq[r], G[r][c]);"),
    "refine_dropped_rhs": ("g[r] = fma(aq[r], w[q], g[r]);", "g[r] = aq[r] * w[q];"),
    "heading_swapped": ("heading[oi] = atan2(vout[1], vout[0]);",
                        "heading[oi] = atan2(vout[0], vout[1]);"),
    "cond_test_inverted": ("*ok = fabs(det) >= eps;\n    if (*ok) {\n      v[0]",
                           "*ok = fabs(det) >= 0.5 * eps + 0.5;\n    if (*ok) {\n      v[0]"),
    "fallback_limit_dropped": ("if (n_in >= k && fabs(detG) > limit) {",
                               "if (fabs(detG) > 0.0) {"),
    "lo_mask_not_updated": ("for (int32_t q = 0; q < n; ++q) mask[o + q] = m2[q];", ""),
    "lo_winner_velocity": ("double r = residual(k, aq, w[q], vout);", "double r = residual(k, aq, w[q], vb);"),
    "lo_dropped_rhs": ("g2[rr] = fma(aq[rr], w[q], g2[rr]);", "g2[rr] = fma(aq[rr], aq[rr], g2[rr]);"),
    "lo_count_not_updated": ("n_in = n2;", ""),
    "adaptive_eps_not_powered": ("double ek = k == 2 ? eps * eps : (eps * eps) * eps;", "double ek = eps;"),
    "adaptive_power_off_by_block": ("adaptive_stop(best_count, n, k, trials, p->confidence))",
                                    "adaptive_stop(best_count, n, k, trials - p->trial_block + 1, p->confidence))"),
    "adaptive_every_trial": ("trials % p->trial_block == 0 && trials < H", "trials < H"),
    "adaptive_pow_skips_bit": ("if (n & 1) r = r * b;", "if (n & 2) r = r * b;"),
    "line_intercept_sign": ("double distn = (-m) * x + 1.0 * y + (-c);", "double distn = (-m) * x + 1.0 * y + c;"),
    "line_distd_no_one": ("double distd = sqrt(m * m + 1.0);", "double distd = sqrt(m * m + 1e-300);"),
    "line_mad_not_abs": ("for (int32_t q = 0; q < n; ++q) tmp[q] = fabs(yn[q] - med);",
                         "for (int32_t q = 0; q < n; ++q) tmp[q] = yn[q] - med;"),
    "line_norm_swapped_range": ("double rv = vmax > vmin ? 1.0 / (vmax - vmin) : 0.0;",
                                "double rv = tmax > tmin ? 1.0 / (tmax - tmin) : 0.0;"),
    "line_slope_inverted": ("double m = (yn[qs[1]] - yn[qs[0]]) / dx;", "double m = dx / (yn[qs[1]] - yn[qs[0]]);"),
    "dbscan_strict_eps": ("if (feat_dist2(&feat[p * dim], &feat[q * dim], dim) <= eps2) ++count;",
                          "if (feat_dist2(&feat[p * dim], &feat[q * dim], dim) < eps2 * 0.999) ++count;"),
    "dbscan_self_not_counted": ("is_core[p] = count >= min_pts;", "is_core[p] = count > min_pts;"),
    "dbscan_border_any_point": ("if (is_core[q] && feat_dist2(&feat[p * dim], &feat[q * dim], dim) <= eps2) {",
                                "if (labels[q] >= 0 && feat_dist2(&feat[p * dim], &feat[q * dim], dim) <= eps2) {"),
    "dbscan_dist_dropped_dim": ("for (int32_t k = 0; k < dim; ++k) {\n    double d = a[k] - b[k];",
                                "for (int32_t k = 1; k < dim; ++k) {\n    double d = a[k] - b[k];"),
    "dbscan_grow_through_border": ("        if (!is_core[q] || labels[q] != -1) continue;\n        if (feat_dist2(&feat[u * dim]",
                                   "        if (labels[q] != -1) continue;\n        if (feat_dist2(&feat[u * dim]"),
}


def _build_mutant(tmp_path, name):
    src = open(oracle.SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not unique in the oracle source"
    mutated = tmp_path / f"{name}.c"
    mutated.write_text(src.replace(old, new))
    hdr = tmp_path / "rvh_oracle.h"
    if not hdr.exists():
        hdr.write_text(open(os.path.join(oracle.HERE, "rvh_oracle.h")).read())
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-w",
                    "-o", str(so), str(mutated), "-lm"], check=True)
    return oracle.load(str(so))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    L = _build_mutant(tmp_path, name)
    failed = []
    for check in oracle_pins.ALL_CHECKS:
        try:
            check(L)
        except (AssertionError, ValueError, FloatingPointError, IndexError, KeyError):
            failed.append(check.__name__)
    assert failed, f"mutant {name} passed every pin"
