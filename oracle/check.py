"""Acceptance metrics against the FP64 oracle (test infrastructure).

Eq. 5 (Section 6) defines the per-input criterion
    e_rel = ||Y_hat - Y||_F / ||X||_F,
with X the input of the call, an absolute check for all-zero inputs and no
denominator floor.  Readings used here:

* e_rel is evaluated per array (the paper checks one input at a time).  For
  the orthonormal transform ||X||_F = ||Y||_F (Parseval), so the criterion is
  also output-relative.  For the unnormalized transform, whose output is
  4hw-scaled, the denominator is ||Y_ref||_F.
* Maximum absolute error is bounded relative to max(max|X|, max|Y_ref|) of
  the same array: FP32 rounding of a large DC coefficient alone can exceed a
  bound taken on max|X| only (at 256x256 the DC of a constant input is 256x
  the input amplitude).
* The bars are the accepted-path tolerances: e_rel <= 1e-6 and
  max_abs <= 4e-6 * scale.  The paper's own bar (2e-5) is looser.
"""
from __future__ import annotations

import numpy as np

ERR_REL_TOL = 1e-6
MAX_ABS_TOL = 4e-6


def _flat(a: np.ndarray, h: int, w: int) -> np.ndarray:
    return np.asarray(a, dtype=np.float64).reshape(-1, h * w)


def metrics(y_hat, y_ref, x, output_relative: bool = False) -> dict:
    """Per-array error statistics of ``y_hat`` against the oracle ``y_ref``.

    ``x`` is the input of the call (for a round trip, y_ref is x itself).
    ``output_relative`` selects ||Y_ref||_F as the denominator (unnormalized
    transforms).  Returns a dict with per-array ``e_rel`` and ``max_abs_ratio``
    plus their maxima and a flag for non-zero output on all-zero input.
    """
    y_hat = np.asarray(y_hat)
    h, w = y_hat.shape[-2:]
    yh = _flat(y_hat, h, w)
    yr = _flat(y_ref, h, w)
    xx = _flat(x, h, w)
    diff = yh - yr
    num = np.sqrt(np.sum(diff * diff, axis=1))
    den = np.sqrt(np.sum((yr if output_relative else xx) ** 2, axis=1))
    zero = den == 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        e_rel = np.where(zero, np.where(num == 0.0, 0.0, np.inf), num / np.where(zero, 1.0, den))
    scale = np.maximum(np.max(np.abs(xx), axis=1), np.max(np.abs(yr), axis=1))
    maxabs = np.max(np.abs(diff), axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        ratio = np.where(scale == 0.0, np.where(maxabs == 0.0, 0.0, np.inf),
                         maxabs / np.where(scale == 0.0, 1.0, scale))
    lit_scale = np.max(np.abs(xx), axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        lit_ratio = np.where(lit_scale == 0.0, np.where(maxabs == 0.0, 0.0, np.inf),
                             maxabs / np.where(lit_scale == 0.0, 1.0, lit_scale))
    nonfinite = ~np.all(np.isfinite(yh), axis=1)
    return {
        "e_rel": e_rel,
        "e_rel_max": float(np.max(e_rel)) if e_rel.size else 0.0,
        "e_rel_aggregate": float(np.sqrt(np.sum(num ** 2)) / max(np.sqrt(np.sum(den ** 2)), 1e-300))
        if e_rel.size else 0.0,
        "max_abs_ratio": ratio,
        "max_abs_ratio_max": float(np.max(ratio)) if ratio.size else 0.0,
        "max_abs_ratio_literal_max": float(np.max(lit_ratio)) if lit_ratio.size else 0.0,
        "zero_input_violations": int(np.sum(zero & (num != 0.0))),
        "nonfinite": int(np.sum(nonfinite)),
    }


def accept(m: dict, rel_tol: float = ERR_REL_TOL, abs_tol: float = MAX_ABS_TOL) -> bool:
    """True when every array meets both bars and nothing is non-finite."""
    return (m["nonfinite"] == 0 and m["zero_input_violations"] == 0
            and m["e_rel_max"] <= rel_tol and m["max_abs_ratio_max"] <= abs_tol)


def boundary_metrics(y_hat, y_ref, x, rel_tol: float = ERR_REL_TOL) -> dict:
    """Boundary diagnostics (Section 6: extreme amplitudes and subnormals).

    Per array: ``representable`` -- every exact output below FLT_MAX in
    magnitude; ``passed`` -- the output is finite where representable and its
    error stays within rel_tol * ||X||_F plus twice the error of rounding the
    exact result to float32 (no float32 output can do better than that
    rounding, which for subnormal results is far above 1e-6 relative).
    """
    y_hat = np.asarray(y_hat, dtype=np.float64)
    h, w = y_hat.shape[-2:]
    yh = y_hat.reshape(-1, h * w)
    yr = np.asarray(y_ref, dtype=np.float64).reshape(-1, h * w)
    xx = np.asarray(x, dtype=np.float64).reshape(-1, h * w)
    fmax = float(np.finfo(np.float32).max)
    representable = np.max(np.abs(yr), axis=1) < fmax
    with np.errstate(over="ignore", invalid="ignore"):
        floor = np.sqrt(np.sum((yr.astype(np.float32).astype(np.float64) - yr) ** 2, axis=1))
        err = np.sqrt(np.sum((yh - yr) ** 2, axis=1))
    finite = np.all(np.isfinite(yh), axis=1)
    bound = rel_tol * np.sqrt(np.sum(xx * xx, axis=1)) + 2.0 * floor
    passed = representable & finite & (err <= bound)
    return {"representable": representable, "passed": passed, "err": err, "bound": bound,
            "checks": int(len(yh)), "n_representable": int(np.sum(representable)),
            "n_failed": int(np.sum(representable & ~passed))}
