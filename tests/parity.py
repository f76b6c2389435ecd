"""Comparison helpers for CUDA-vs-oracle parity tests.

Tolerances (FP32 GPU against the FP64 oracle):
* power and loss: per element |gpu - ref| <= 1e-4 |ref| + 1e-4 * 1e-6 * max|ref|
  (relative 1e-4, with a floor for receivers in deep shadow whose power is
  many orders below the scene's brightest receiver).  At large alpha some
  receivers' power is ill-conditioned in FP32: the smoothing's slope (alpha/6
  per unit of distance for the hard sigmoid) turns the ~1e-7 rounding of a
  distance into more than 1e-4 of a nearly blocked path's power.  A test may
  then pass ``sens`` (``fp32_sensitivity``: how far the oracle's own FP64
  result moves when every input coordinate moves by two FP32 roundings) and
  ``min_strict``: at least that fraction of elements must meet the plain
  bound, and every element must meet max(plain bound, 2 * sens);
* gradients: norm-wise ||gpu - ref|| <= 1e-3 ||ref||, and per element
  |gpu - ref| <= 1e-3 |ref| + 1e-3 * 1e-3 * max|ref|.
"""
from __future__ import annotations

import numpy as np

POWER_RTOL = 1e-4
POWER_FLOOR = 1e-6
GRAD_RTOL = 1e-3
GRAD_FLOOR = 1e-3


SENS_REL = 2 * 2.0 ** -24    # perturbation size: 2 FP32 unit roundings, relative
SENS_DRAWS = 4
SENS_FACTOR = 2.0


def fp32_sensitivity(power_fn, walls, tx, rx, seed=0):
    """max over a few draws of |P(x + dx) - P(x)|, each input coordinate x perturbed
    by dx uniform in [-SENS_REL, SENS_REL] * max(|x|, 1) (FP64 oracle ``power_fn``)."""
    rng = np.random.default_rng(seed)
    walls = np.asarray(walls, np.float64)
    tx = np.asarray(tx, np.float64)
    rx = np.asarray(rx, np.float64)
    base = power_fn(walls, tx, rx)
    out = np.zeros_like(base)

    def jitter(a):
        return a + rng.uniform(-SENS_REL, SENS_REL, a.shape) * np.maximum(np.abs(a), 1.0)

    for _ in range(SENS_DRAWS):
        out = np.maximum(out, np.abs(power_fn(jitter(walls), jitter(tx), jitter(rx)) - base))
    return out


def power_errors(gpu, ref, sens=None):
    """(err, plain tolerance, widened tolerance) per element."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.abs(ref).max() if ref.size else 0.0
    plain = POWER_RTOL * np.abs(ref) + POWER_RTOL * POWER_FLOOR * scale
    wide = plain if sens is None else np.maximum(plain, SENS_FACTOR * np.asarray(sens, np.float64))
    return np.abs(gpu - ref), plain, wide


def strict_fraction(gpu, ref):
    err, plain, _ = power_errors(gpu, ref)
    return float(np.mean(err <= plain)) if err.size else 1.0


def assert_power_close(gpu, ref, what="power", sens=None, min_strict=1.0):
    err, plain, tol = power_errors(gpu, ref, sens)
    frac = float(np.mean(err <= plain)) if err.size else 1.0
    if frac < min_strict:
        raise AssertionError(f"{what}: only {frac:.3f} of elements within the plain 1e-4 bound "
                             f"(need {min_strict})")
    bad = np.nonzero(~(err <= tol))[0]
    if bad.size:
        i = bad[np.argmax(err[bad] / np.maximum(tol[bad], 1e-300))]
        raise AssertionError(
            f"{what}: {bad.size}/{err.size} elements out of tolerance; worst index {i}: "
            f"gpu {np.asarray(gpu)[i]!r} ref {np.asarray(ref)[i]!r} err {err[i]:.3e} tol {tol[i]:.3e}")


def assert_grad_close(gpu, ref, what="gradient"):
    gpu = np.asarray(gpu, np.float64).ravel()
    ref = np.asarray(ref, np.float64).ravel()
    nref = np.linalg.norm(ref)
    nerr = np.linalg.norm(gpu - ref)
    if not nerr <= GRAD_RTOL * nref:
        raise AssertionError(f"{what}: norm-wise error {nerr:.3e} > {GRAD_RTOL} * {nref:.3e}")
    scale = np.abs(ref).max() if ref.size else 0.0
    tol = GRAD_RTOL * np.abs(ref) + GRAD_RTOL * GRAD_FLOOR * scale
    err = np.abs(gpu - ref)
    bad = np.nonzero(~(err <= tol))[0]
    if bad.size:
        i = bad[np.argmax(err[bad] / np.maximum(tol[bad], 1e-300))]
        raise AssertionError(f"{what}: {bad.size}/{err.size} elements out of tolerance; worst "
                             f"index {i}: gpu {gpu[i]!r} ref {ref[i]!r}")
