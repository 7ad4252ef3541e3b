"""Mutation check of the oracle pins: each plausible mistake below is planted in
a temporary copy of the oracle (on the CPU only) and the pin suite must fail on
it. A mutant that survives means a part of the oracle is not pinned."""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "swap_dxdy": ("    dx = L[ys, xs + 1] - L[ys, xs - 1]\n    dy = L[ys + 1, xs] - L[ys - 1, xs]",
                  "    dy = L[ys, xs + 1] - L[ys, xs - 1]\n    dx = L[ys + 1, xs] - L[ys - 1, xs]"),
    "drop_dxy": ("    H = np.array([[dxx, dxy, dxs], [dxy, dyy, dys], [dxs, dys, dss]])",
                 "    H = np.array([[dxx, 0.0, dxs], [0.0, dyy, dys], [dxs, dys, dss]])"),
    "rotation_sign": ("    rx = (ct * ox + st * oy) / wbin\n    ry = (-st * ox + ct * oy) / wbin",
                      "    rx = (ct * ox - st * oy) / wbin\n    ry = (st * ox + ct * oy) / wbin"),
    "uv_transposed": ("                np.add.at(hist, (vv[inb], uu[inb], oo[inb])",
                      "                np.add.at(hist, (uu[inb], vv[inb], oo[inb])"),
    "relative_angle_sign": ("    phi = np.arctan2(dy, dx) - th", "    phi = th - np.arctan2(dy, dx)"),
    "offset_sign": ("        delta = cramer_solve(H, -g)", "        delta = cramer_solve(H, g)"),
    "contrast_no_half": ("    contrast = D[s, y, x] + 0.5 * float(g @ delta)",
                         "    contrast = D[s, y, x] + float(g @ delta)"),
    "kappa_linear": ("    return [math.sqrt(s[i] ** 2 - s[i - 1] ** 2) for i in range(1, len(s))]",
                     "    return [s[i] - s[i - 1] for i in range(1, len(s))]"),
    "edge_ratio_dropped": ("    lhs, rhs = tr * tr * r, (r + 1) ** 2 * det",
                           "    lhs, rhs = tr * tr, (r + 1) ** 2 * det"),
    "two_smoothing_passes": (
        "    return 0.25 * np.roll(hist, 1) + 0.5 * hist + 0.25 * np.roll(hist, -1)",
        "    h = 0.25 * np.roll(hist, 1) + 0.5 * hist + 0.25 * np.roll(hist, -1)\n"
        "    return 0.25 * np.roll(h, 1) + 0.5 * h + 0.25 * np.roll(h, -1)"),
    "parabola_sign": ("            kf = k + 0.5 * (hm - hp) / (hm - 2.0 * hk + hp)",
                      "            kf = k - 0.5 * (hm - hp) / (hm - 2.0 * hk + hp)"),
    "descriptor_window_sigma": (
        "    wt = mag * np.exp(-(rx * rx + ry * ry) / (2.0 * (0.5 * d) ** 2))",
        "    wt = mag * np.exp(-(rx * rx + ry * ry) / (2.0 * (0.5 * d)))"),
    "decimate_odd_phase": ("    return img[0:2 * (h // 2):2, 0:2 * (w // 2):2].copy()",
                           "    return img[1:2 * (h // 2):2, 1:2 * (w // 2):2].copy()"),
    "upsample_no_average": ("        out[1::2] = 0.5 * (a + nxt)", "        out[1::2] = a"),
    "border_off_by_one": (
        "        if s < 1 or s > S or x < b or x >= w - b or y < b or y >= h - b:",
        "        if s < 1 or s > S or x < b or x > w - b or y < b or y > h - b:"),
    "orientation_window_sigma": ("    wt = np.exp(-(i * i + j * j) / (2.0 * sw * sw))",
                                 "    wt = np.exp(-(i * i + j * j) / (2.0 * sw))"),
    "clip_missing": ("    vec = np.minimum(vec / nrm, p.desc_clip)", "    vec = vec / nrm"),
    "extremum_not_strict": ("        is_max = c > nmax\n        is_min = c < nmin",
                            "        is_max = c >= nmax\n        is_min = c <= nmin"),
    "nearest_bin_floor": (
        "    bins = np.floor(n * th / (2 * math.pi) + 0.5).astype(np.int64) % n",
        "    bins = np.floor(n * th / (2 * math.pi)).astype(np.int64) % n"),
    "taps_not_normalised": ("    return r, w / w.sum()", "    return r, w / (math.sqrt(2 * math.pi) * sigma)"),
    "dsp_grid_no_half": ("    c = (np.arange(G) + 0.5) * d / G - 0.5 * d",
                         "    c = np.arange(G) * d / G - 0.5 * d"),
    "dsp_rotation_sign": ("    x = xk + wbin * (ct * rx - st * ry)\n    y = yk + wbin * (st * rx + ct * ry)",
                          "    x = xk + wbin * (ct * rx + st * ry)\n    y = yk + wbin * (-st * rx + ct * ry)"),
    "dsp_scale_ignored": ("    wbin = p.desc_scale * sigma_oct * scale",
                          "    wbin = p.desc_scale * sigma_oct"),
    "dsp_weight_in_pixels": (
        "    wt = mag * np.exp(-(rx * rx + ry * ry) / (2.0 * (0.5 * d) ** 2))\n    return _trilinear_histogram(rx",
        "    wt = mag * np.exp(-wbin * wbin * (rx * rx + ry * ry) / (2.0 * (0.5 * d) ** 2))\n"
        "    return _trilinear_histogram(rx"),
    "dsp_dy_from_x": ("    dy = bilinear(L, x, y + 1) - bilinear(L, x, y - 1)",
                      "    dy = bilinear(L, x + 1, y + 1) - bilinear(L, x - 1, y - 1)"),
    "magnify_limit_exclusive": ("(p.upsample_max_px <= 0 or h * w <= p.upsample_max_px)",
                                "(p.upsample_max_px <= 0 or h * w < p.upsample_max_px)"),
    "decimate_wrong_level": ("g0 = decimate(octaves[o - 1][p.n_scales])",
                             "g0 = decimate(octaves[o - 1][p.n_scales + 1])"),
    "smoothing_flat": ("    return 0.25 * np.roll(hist, 1) + 0.5 * hist + 0.25 * np.roll(hist, -1)",
                       "    return (np.roll(hist, 1) + hist + np.roll(hist, -1)) / 3.0"),
    "descriptor_bin_width": ("    wbin = p.desc_scale * sigma_oct\n", "    wbin = 2.0 * sigma_oct\n"),
    "contrast_test_signed": ("    if abs(contrast) < p.contrast_thr:", "    if contrast < p.contrast_thr:"),
    "peak_ratio_ignored": ("    thr = p.ori_peak_ratio * hmax", "    thr = hmax"),
    "orientation_mag_squared": ("    mag = np.sqrt(dx * dx + dy * dy)\n    th = np.arctan2(dy, dx)",
                                "    mag = dx * dx + dy * dy\n    th = np.arctan2(dy, dx)"),
    "refine_threshold_loose": ("        if m < 0.5:", "        if m < 0.6:"),
    "blur_border_symmetric": ('    return np.pad(a, pad, mode="reflect")  # numpy',
                              '    return np.pad(a, pad, mode="symmetric")  # numpy'),
    "descriptor_first_norm_l1": ("    nrm = math.sqrt(float(vec @ vec))\n    if nrm == 0:",
                                 "    nrm = float(np.sum(np.abs(vec)))\n    if nrm == 0:"),
    "octave_min_side_strict": ("    while min(h, w) >= p.min_octave_side:",
                               "    while min(h, w) > p.min_octave_side:"),
    "descriptor_orientation_no_wrap": ("                oo = (o0 + do) % nb",
                                       "                oo = np.minimum(o0 + do, nb - 1)"),
    "orientation_radius_ceil": ("    R = _round_pos(p.ori_radius_factor * sw)",
                                "    R = int(math.ceil(p.ori_radius_factor * sw))"),
    "orientation_peak_not_strict": ("        is_lmax = hk > hm and hk > hp",
                                    "        is_lmax = hk >= hm and hk >= hp"),
    "descriptor_offsets_from_pixel": ("    ox = xs - xk\n    oy = ys - yk\n    rx = (ct * ox + st * oy) / wbin",
                                      "    ox = xs - xi\n    oy = ys - yi\n    rx = (ct * ox + st * oy) / wbin"),
    "descriptor_radius_no_sqrt2": ("    R = _round_pos(wbin * math.sqrt(2.0) * (d + 1) * 0.5)",
                                   "    R = _round_pos(wbin * (d + 1) * 0.5)"),
    "upsample_wraps": ("        nxt = np.concatenate([a[1:], a[-1:]], axis=0)",
                       "        nxt = np.concatenate([a[1:], a[:1]], axis=0)"),
    "taps_radius_round": ("    r = int(math.ceil(4.0 * sigma))", "    r = int(round(4.0 * sigma))"),
    "extrema_same_layer_only": ("        for ds in (-1, 0, 1):\n            for dy in (-1, 0, 1):",
                                "        for ds in (0,):\n            for dy in (-1, 0, 1):"),
    "extrema_layers_off_by_one": ("    for s in range(1, S + 1):\n        c = D[s, b:h - b, b:w - b]",
                                  "    for s in range(1, S):\n        c = D[s, b:h - b, b:w - b]"),
    "pregate_ignored": ("        gate = np.abs(c) > thr", "        gate = np.abs(c) >= 0"),
    "output_no_half_when_upsampled": ("    scale_up = 0.5 if p.upsample else 1.0",
                                      "    scale_up = 1.0"),
    "output_octave_scale_missing": ("        f = (2.0 ** o) * scale_up", "        f = scale_up"),
    "dsp_stencil_bound_inclusive": ("    ok = (x >= 1) & (x < w - 2) & (y >= 1) & (y < h - 2)\n    x, y, rx, ry = x[ok], y[ok], rx[ok], ry[ok]",
                                    "    ok = (x >= 1) & (x <= w - 2) & (y >= 1) & (y <= h - 2)\n    x, y, rx, ry = x[ok], y[ok], rx[ok], ry[ok]"),
    "dsp_stencil_lower_strict": ("    ok = (x >= 1) & (x < w - 2) & (y >= 1) & (y < h - 2)\n    x, y, rx, ry = x[ok], y[ok], rx[ok], ry[ok]",
                                 "    ok = (x > 1) & (x < w - 2) & (y > 1) & (y < h - 2)\n    x, y, rx, ry = x[ok], y[ok], rx[ok], ry[ok]"),
    "dsp_scales_four": ("    dsp_scales: tuple = (0.5, 2 ** -0.5, 1.0, 2 ** 0.5, 2.0)",
                        "    dsp_scales: tuple = (2 ** -0.5, 1.0, 2 ** 0.5, 2.0)"),
    "dog_reversed": ("    return octave[1:] - octave[:-1]", "    return octave[:-1] - octave[1:]"),
    "refine_round_half_even": ("    return int(math.floor(abs(v) + 0.5)) * (1 if v >= 0 else -1)",
                               "    return int(round(v))"),
    "refine_four_iterations": ("    for _ in range(p.max_refine_iter):",
                               "    for _ in range(p.max_refine_iter - 1):"),
    "edge_ratio_equality_kept": ("    if det <= 0 or lhs >= rhs:", "    if det <= 0 or lhs > rhs:"),
    "peak_ratio_strict": ("        above = hk >= thr", "        above = hk > thr"),
    "margin_skips_convergence": ("        margin = min(margin, abs(0.5 - m) / 0.5)\n", "\n"),
    "orientation_edge_columns_dropped": (
        "    ys, xs, i, j = ys[ok], xs[ok], i[ok], j[ok]",
        "    ok = ok & (xs >= 2) & (xs <= w - 3) & (ys >= 2) & (ys <= h - 3)\n"
        "    ys, xs, i, j = ys[ok], xs[ok], i[ok], j[ok]"),
    "descriptor_edge_pixels_dropped": (
        "    ys, xs = ys[ok], xs[ok]\n    ox = xs - xk",
        "    ok = ok & (xs >= 2) & (xs <= w - 3) & (ys >= 2) & (ys <= h - 3)\n"
        "    ys, xs = ys[ok], xs[ok]\n    ox = xs - xk"),
    "descriptor_on_next_level": ("            desc[t] = descriptor(pyr[o][r.s], xk, yk",
                                 "            desc[t] = descriptor(pyr[o][r.s + 1], xk, yk"),
    "orientation_on_next_level": ("            L = G[r.s]\n", "            L = G[r.s + 1]\n"),
    "extremum_margin_absolute": ("        m_ext.append(gap / np.abs(cv))", "        m_ext.append(gap)"),
    "gate_margin_absolute": ("        m_gate.append((np.abs(cv) - thr) / np.maximum(np.abs(cv), thr))",
                             "        m_gate.append(np.abs(cv) - thr)"),
    "margin_skips_contrast": (
        "    margin = min(margin, abs(abs(contrast) - p.contrast_thr) / max(abs(contrast), p.contrast_thr))\n",
        "\n"),
    "margin_skips_edge": ("        margin = min(margin, abs(rhs - lhs) / denom)\n", "        pass\n"),
    "margin_skips_peak_ratio": ("            margin = min(margin, abs(hk - thr) / hmax)\n", "            pass\n"),
    "margin_skips_rounding": ("            margin = min(margin, abs(a - edge) / edge)\n", "            pass\n"),
    "response_signed": ("                   abs(contrast), margin)", "                   contrast, margin)"),
    "keypoint_margin_skips_candidate": (
        "            m0 = min(float(mg[ci]), float(me[ci]), r.margin)", "            m0 = r.margin"),
    "fp16_storage_ignored": ("        return level.astype(np.float16).astype(np.float64)",
                             "        return level"),
    "fp16_storage_truncates": ("        return level.astype(np.float16).astype(np.float64)",
                               "        return np.trunc(level * 2048.0) / 2048.0"),
    "fp16_storage_octave0_too": ("    if p.fp16_pyramid and o > 0:", "    if p.fp16_pyramid and o >= 0:"),
    "fp16_storage_after_the_chain": ("            levels.append(store_level(blur(levels[-1], k), o, p))",
                                     "            levels.append(blur(levels[-1], k))"),
    "diagonal_votes_downward": ("    bins = np.where(diag, (n * (2 * q + 1) + 4) // 8 % n, bins)",
                                "    bins = np.where(diag, (n * (2 * q + 1) + 3) // 8 % n, bins)"),
    "diagonal_quadrants_swapped": ("    q = np.where(dy > 0, np.where(dx > 0, 0, 1), np.where(dx < 0, 2, 3))",
                                   "    q = np.where(dy > 0, np.where(dx > 0, 1, 0), np.where(dx < 0, 2, 3))"),
    "vote_margin_counts_diagonals": ("    votes = (wt * mag > 0) & ~diag\n", "    votes = wt * mag > 0\n"),
    "keypoint_margin_skips_votes": (
        "                m1 = min(m1, orientation_vote_margin(L, r.x, r.y, sigma_oct, p))\n", "\n"),
    "vote_margin_from_bin_centre": ("    t = n * th[votes] / (2 * math.pi) + 0.5   # bin",
                                    "    t = n * th[votes] / (2 * math.pi)   # bin"),
    "vote_margin_in_radians": ("    t = n * th[votes] / (2 * math.pi) + 0.5   # bin",
                               "    t = th[votes] + 0.5   # bin"),
    "vote_margin_one_sided": ("    return float(np.minimum(f, 1.0 - f).min())",
                              "    return float(f.min())"),
    "vote_margin_counts_zero_weight": ("    votes = (wt * mag > 0) & ~diag\n", "    votes = (wt * mag >= 0) & ~diag\n"),
    "keypoint_margin_skips_orientation": (
        "                rows.append((o, r, sigma_oct, a, min(m0, m1)))",
        "                rows.append((o, r, sigma_oct, a, m0))"),
    "reported_layer_off_by_one": ("        layer[t] = r.s\n", "        layer[t] = r.s - 1\n"),
    "cap_not_applied": (
        "    keep = cap_topk(resp, p.max_kpts) if p.max_kpts > 0 else np.arange(len(rows))",
        "    keep = np.arange(len(rows))"),
    "cap_keeps_smallest": ("    resp = np.array([row[1].response for row in rows])",
                           "    resp = -np.array([row[1].response for row in rows])"),
    "upright_angle_nonzero": ("                angles, m1 = [0.0], math.inf",
                              "                angles, m1 = [90.0], math.inf"),
    "rootsift_no_l1": ("        vec = np.sqrt(vec / l1) if l1 > 0 else vec",
                       "        vec = np.sqrt(vec) if l1 > 0 else vec"),
}


# Mistakes planted in the MAGSAC++ oracle, caught by its own pin file.
MAGSAC_MUTANTS = {
    "magsac_loss_no_truncation_shift": (
        "        + 0.5 * rc * rc * (_upper_gamma(a, x) - _upper_gamma(a, k * k / 2.0)))",
        "        + 0.5 * rc * rc * _upper_gamma(a, x))"),
    "magsac_loss_lower_gamma_order": ("sigma_max * sigma_max * _lower_gamma(a + 1.0, x)",
                                      "sigma_max * sigma_max * _lower_gamma(a, x)"),
    "magsac_no_denormalise": ("    H = np.linalg.inv(Tb) @ Hn @ Ta", "    H = Hn"),
    "magsac_dlt_row": ("[-x, -y, -1.0, 0.0, 0.0, 0.0, u * x, u * y, u]",
                       "[-x, -y, -1.0, 0.0, 0.0, 0.0, u * x, v * y, u]"),
    "magsac_residual_wrong_image": ("np.sqrt((px - xb[:, 0]) ** 2 + (py - xb[:, 1]) ** 2)",
                                    "np.sqrt((px - xa[:, 0]) ** 2 + (py - xa[:, 1]) ** 2)"),
    "magsac_inlier_threshold_sigma": ("inl = residuals(H, xa, xb) <= chi_quantile() * sigma_max",
                                      "inl = residuals(H, xa, xb) <= sigma_max"),
    "magsac_best_is_worst": ("    best = int(np.argmin(scores))",
                             "    best = int(np.argmax(np.where(np.isfinite(scores), scores, -np.inf)))"),
    "magsac_two_dof": ("DOF = 4 ", "DOF = 2 "),
    "magsac_normaliser_unit_distance": ("    s = math.sqrt(2.0) / d if d > 0 else 1.0",
                                        "    s = 1.0 / d if d > 0 else 1.0"),
    "magsac_normaliser_no_centroid": (
        "    return np.array([[s, 0.0, -s * c[0]], [0.0, s, -s * c[1]], [0.0, 0.0, 1.0]])",
        "    return np.array([[s, 0.0, 0.0], [0.0, s, 0.0], [0.0, 0.0, 1.0]])"),
    "magsac_collinear_first_image_only": ("    if _collinear(pa) or _collinear(pb):",
                                          "    if _collinear(pa):"),
    "magsac_normalised_h33_unchecked": ("    if abs(v[8]) < 1e-9:", "    if False:"),
    "magsac_h22_unchecked": ("    if abs(H[2, 2]) < 1e-12 * np.abs(H).max():", "    if False:"),
    "magsac_weight_sigma_scale": (
        "    x = t * t / (2.0 * sigma_max * sigma_max)",
        "    x = t * t / (sigma_max * sigma_max)"),
}

# Mistakes planted in the matcher oracle, caught by its own pin file.
MATCHER_MUTANTS = {
    "matcher_no_mutual_check": ("keep = ib[j] == i and da1[i] < ratio * da2[i]",
                                "keep = da1[i] < ratio * da2[i]"),
    "matcher_ratio_one_side": ("and da1[i] < ratio * da2[i] and db1[j] < ratio * db2[j]",
                               "and da1[i] < ratio * da2[i]"),
    "matcher_ratio_default_07": ("def match(desc_a: np.ndarray, desc_b: np.ndarray, ratio: float = 0.8,",
                                 "def match(desc_a: np.ndarray, desc_b: np.ndarray, ratio: float = 0.7,"),
    "matcher_robust_without_gap": (
        "                             and sa1[i] - sa2[i] > 2 * eps and sb1[j] - sb2[j] > 2 * eps)",
        "                             )"),
    "matcher_robust_one_side": ("                             and _ratio_robust(sb1[j], sb2[j], ratio, eps)\n",
                                "\n"),
    "matcher_single_member_sets": ("    if na < 2 or nb < 2:", "    if na < 1 or nb < 1:"),
    "matcher_ties_to_last": ("    j1 = np.argmax(S, axis=1)                      # first occurrence = smallest index",
                             "    j1 = S.shape[1] - 1 - np.argmax(S[:, ::-1], axis=1)"),
}

# Mistakes planted in the parity comparator, caught by its own test file.
COMPARE_MUTANTS = {
    "compare_position_tolerance": ("POS_TOL = 0.01", "POS_TOL = 0.05"),
    "compare_angle_without_wrap": (
        "    return np.abs((np.asarray(a) - np.asarray(b) + 180.0) % 360.0 - 180.0)",
        "    return np.abs(np.asarray(a) - np.asarray(b))"),
    "compare_no_margin_excuse": ("    eligible = oracle_res.margin >= margin_eps",
                                 "    eligible = oracle_res.margin >= 0"),
    "compare_position_x_only": (
        "        dpos = np.maximum(np.abs(gx[cand] - ox[i]), np.abs(gy[cand] - oy[i]))",
        "        dpos = np.abs(gx[cand] - ox[i])"),
    "compare_scale_absolute": ("        ds = np.abs(gsig[near] - osig[i]) / osig[i]",
                               "        ds = np.abs(gsig[near] - osig[i]) / 10.0"),
    "compare_ignores_layer": ("        cand = buckets.get((int(ooct[i]), int(olay[i])))",
                              "        cand = np.concatenate(list(buckets.values()))"),
    "compare_desc_not_max": ("                desc_max = max(desc_max, dd)",
                             "                desc_max = dd"),
    "compare_excused_count": ("        return self.n_oracle - self.n_eligible",
                              "        return self.n_oracle - self.n_found"),
    "compare_hit_needs_scale": (
        "        gpu_hit[near] = True\n",
        "        gpu_hit[near[(np.abs(gsig[near] - osig[i]) / osig[i] < SIGMA_RTOL)]] = True\n"),
    "compare_counts_excused": ("        if not eligible[i]:\n            continue\n", "\n"),
    "compare_pair_not_closest_angle": ("            j = ok[np.argmin(angle_diff(gang[ok], oang[i]))]",
                                       "            j = ok[-1]"),
    "compare_worst_is_last": (
        '            worst["pos"] = max(worst["pos"], float(max(abs(gx[j] - ox[i]), abs(gy[j] - oy[i]))))',
        '            worst["pos"] = float(max(abs(gx[j] - ox[i]), abs(gy[j] - oy[i])))'),
    "compare_pairs_uncounted": ("                pairs += 1", "                pairs += 0"),
    "compare_scale_ignored_for_angle": ("    pos_tol, sig_tol, ang_tol = POS_TOL * tol_scale, SIGMA_RTOL * tol_scale, ANGLE_TOL * tol_scale",
                                        "    pos_tol, sig_tol, ang_tol = POS_TOL * tol_scale, SIGMA_RTOL * tol_scale, ANGLE_TOL"),
    "compare_fp16_scale_four": ("FP16_TOL_SCALE = 5.0", "FP16_TOL_SCALE = 4.0"),
}

CASES = ([(n, "sift_oracle.py", "test_oracle_pins.py") for n in sorted(MUTANTS)]
         + [(n, "magsac.py", "test_magsac_oracle.py") for n in sorted(MAGSAC_MUTANTS)]
         + [(n, "matcher.py", "test_matcher_oracle.py") for n in sorted(MATCHER_MUTANTS)]
         + [(n, "compare.py", "test_compare.py") for n in sorted(COMPARE_MUTANTS)])
_TABLE = {"sift_oracle.py": MUTANTS, "magsac.py": MAGSAC_MUTANTS, "matcher.py": MATCHER_MUTANTS,
          "compare.py": COMPARE_MUTANTS}


def _run_mutant(name, target, pins, work):
    """Plant one mutant in a copy of the oracle under `work` and run its pin file;
    returns (exit code, tail of the output)."""
    before, after = _TABLE[target][name]
    src = open(os.path.join(ROOT, "oracle", target)).read()
    if before not in src:
        return None, "mutation anchor missing: " + name
    for d in ("oracle", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), os.path.join(work, d),
                        ignore=shutil.ignore_patterns("__pycache__"))
    os.mkdir(os.path.join(work, "tests"))
    for f in ("conftest.py", pins):
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(work, "tests", f))
    with open(os.path.join(work, "oracle", target), "w") as fh:
        fh.write(src.replace(before, after))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests/" + pins, "-q", "-x",
                        "-p", "no:cacheprovider"], cwd=work, capture_output=True, text=True,
                       env=env)
    return r.returncode, r.stdout[-2000:]


@pytest.fixture(scope="module")
def mutant_results(tmp_path_factory):
    """All mutants run at once, one pin-suite process per core."""
    base = tmp_path_factory.mktemp("mutants")
    workers = max(1, min(8, os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        futs = {c[0]: ex.submit(_run_mutant, *c, str(base / c[0])) for c in CASES}
        return {k: f.result() for k, f in futs.items()}


@pytest.mark.parametrize("name,target,pins", CASES, ids=[c[0] for c in CASES])
def test_pins_catch_mutant(name, target, pins, mutant_results):
    code, out = mutant_results[name]
    assert code is not None, out
    assert code != 0, f"mutant {name} survived the pins:\n{out}"
