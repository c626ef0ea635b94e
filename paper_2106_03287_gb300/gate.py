"""Pose-distribution error between two runs (the "at fixed pose error" gate).

Two registration runs that should agree are compared by their particles'
mean pose and spread: the largest translation difference (mm) and the
largest angle difference (degrees) of the means, and the same for the
standard deviations (square roots of the covariance diagonals).  The gate is
1 mm and 0.05 degrees on both.

No arithmetic of the method lives here: this only compares two results.
"""
from __future__ import annotations

import hashlib
import math

import numpy as np

GATE_MM, GATE_DEG = 1.0, 0.05


def pose_errors(mean_a, cov_a, mean_b, cov_b) -> dict:
    """Largest |difference| of the means and of the standard deviations, split
    into translation (mm) and rotation (degrees)."""
    ma, mb = np.asarray(mean_a, np.float64), np.asarray(mean_b, np.float64)
    sa = np.sqrt(np.clip(np.diag(np.asarray(cov_a, np.float64).reshape(6, 6)), 0, None))
    sb = np.sqrt(np.clip(np.diag(np.asarray(cov_b, np.float64).reshape(6, 6)), 0, None))
    dm, ds = np.abs(ma - mb), np.abs(sa - sb)
    return {"dmean_mm": 1e3 * float(dm[:3].max()), "dmean_deg": math.degrees(float(dm[3:].max())),
            "dsd_mm": 1e3 * float(ds[:3].max()), "dsd_deg": math.degrees(float(ds[3:].max()))}


def within(err: dict, mm: float = GATE_MM, deg: float = GATE_DEG) -> bool:
    return (err["dmean_mm"] <= mm and err["dsd_mm"] <= mm and err["dmean_deg"] <= deg and err["dsd_deg"] <= deg)


def worst(errs) -> dict:
    """Component-wise maximum of several pose_errors results."""
    errs = list(errs)
    return {k: max(e[k] for e in errs) for k in errs[0]} if errs else {}


def inputs_hash(d) -> str:
    """Short hash of a problem's float32 inputs (reference, source, particles),
    to tell whether two machines generated the same clouds."""
    h = hashlib.sha256()
    for k in ("ref", "src", "particles"):
        h.update(np.ascontiguousarray(d[k], np.float32).tobytes())
    return h.hexdigest()[:16]
