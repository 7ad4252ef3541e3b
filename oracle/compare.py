"""Keypoint-set comparison between the CUDA extractor and the FP64 oracle
(test infrastructure only).

Outputs are compared as sets, never by index: FP32 rounding may flip a
decision that sits within a hair of its threshold, which changes counts and
therefore indices. The oracle records, for every keypoint, the smallest
relative distance of any of its discrete decisions from the threshold (the
pre-gate, the extremum test, the refinement steps, contrast, edge, the
orientation peaks and the nearest-bin votes of the orientation histogram);
oracle keypoints closer than `margin_eps` (1e-4) to a threshold are excused,
and the number excused is reported.

Tolerances (GPU FP32 vs oracle FP64): position within 0.01 px (input-image
pixels), scale within 1e-3 relative, orientation within 0.5 degrees, and
descriptor L2 difference at most 1e-3 on matched keypoints. Every quantity
is compared directly: the comparison never evaluates the oracle on a value
the GPU produced.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

POS_TOL = 0.01
SIGMA_RTOL = 1e-3
ANGLE_TOL = 0.5
DESC_TOL = 1e-3
MARGIN_EPS = 1e-4
# fp16 storage mode (levels above octave 0 stored as binary16): a stored level
# value can differ from the oracle's by one binary16 ulp of [0, 1) values,
# 2^-11 (the GPU rounds its FP32 result, the oracle its FP64 one), where the
# FP32 mode's pyramid differs by at most 1e-4. Everything downstream is a
# Lipschitz function of the level values, so the FP32 mode's position, scale,
# angle and descriptor tolerances are scaled by the ratio of the two pyramid
# bounds, 2^-11 / 1e-4 = 4.9, rounded up to 5.
FP16_TOL_SCALE = 5.0


def angle_diff(a, b):
    return np.abs((np.asarray(a) - np.asarray(b) + 180.0) % 360.0 - 180.0)


@dataclass
class Match:
    n_oracle: int
    n_eligible: int        # oracle keypoints not near a threshold
    n_found: int           # eligible oracle keypoints matched by a GPU keypoint
    n_gpu: int
    n_gpu_unmatched: int   # GPU keypoints with no oracle keypoint at the same place
    desc_max_l2: float     # largest descriptor L2 difference over the matched pairs
    desc_pairs: int
    worst: dict

    @property
    def found_frac(self):
        return self.n_found / max(self.n_eligible, 1)

    @property
    def n_excused(self):
        """Oracle keypoints within margin_eps of a decision threshold."""
        return self.n_oracle - self.n_eligible


def match(oracle_res, gpu: dict, margin_eps: float = MARGIN_EPS, tol_scale: float = 1.0) -> Match:
    """oracle_res: oracle Result; gpu: dict of numpy arrays (x, y, sigma, angle,
    octave, layer, desc); tol_scale multiplies the position, scale and angle
    tolerances (FP16_TOL_SCALE for the fp16 storage mode)."""
    pos_tol, sig_tol, ang_tol = POS_TOL * tol_scale, SIGMA_RTOL * tol_scale, ANGLE_TOL * tol_scale
    ox, oy, osig, oang = oracle_res.x, oracle_res.y, oracle_res.sigma, oracle_res.angle
    ooct, olay = oracle_res.octave, oracle_res.layer
    gx, gy, gsig, gang = (np.asarray(gpu[k], dtype=np.float64) for k in ("x", "y", "sigma", "angle"))
    goct, glay = np.asarray(gpu["octave"]), np.asarray(gpu["layer"])
    gdesc = np.asarray(gpu["desc"], dtype=np.float64)
    eligible = oracle_res.margin >= margin_eps
    n_found = 0
    desc_max = 0.0
    pairs = 0
    worst = {"pos": 0.0, "sigma": 0.0, "angle": 0.0}
    # Bucket GPU keypoints by (octave, layer) for the neighbour search.
    buckets = {}
    for i in range(len(gx)):
        buckets.setdefault((int(goct[i]), int(glay[i])), []).append(i)
    buckets = {k: np.array(v) for k, v in buckets.items()}
    gpu_hit = np.zeros(len(gx), bool)
    for i in range(len(ox)):
        cand = buckets.get((int(ooct[i]), int(olay[i])))
        if cand is None:
            continue
        dpos = np.maximum(np.abs(gx[cand] - ox[i]), np.abs(gy[cand] - oy[i]))
        near = cand[dpos < pos_tol]
        if len(near) == 0:
            continue
        gpu_hit[near] = True
        ds = np.abs(gsig[near] - osig[i]) / osig[i]
        da = angle_diff(gang[near], oang[i])
        ok = near[(ds < sig_tol) & (da < ang_tol)]
        if not eligible[i]:
            continue
        if len(ok):
            n_found += 1
            j = ok[np.argmin(angle_diff(gang[ok], oang[i]))]
            worst["pos"] = max(worst["pos"], float(max(abs(gx[j] - ox[i]), abs(gy[j] - oy[i]))))
            worst["sigma"] = max(worst["sigma"], float(abs(gsig[j] - osig[i]) / osig[i]))
            worst["angle"] = max(worst["angle"], float(angle_diff(gang[j], oang[i])))
            if len(oracle_res.desc) and len(gdesc):
                dd = float(np.linalg.norm(gdesc[j] - oracle_res.desc[i]))
                desc_max = max(desc_max, dd)
                pairs += 1
    return Match(len(ox), int(eligible.sum()), n_found, len(gx), int((~gpu_hit).sum()),
                 desc_max, pairs, worst)
