"""The parity gate the GPU tests share: the CUDA path against the FP64 oracle.

A pixel is held to max |GPU - oracle| <= TOL (1e-3 on the 0..255 scale) when
the oracle's conditioning number kappa (oracle.gp_bf(..., return_kappa=True))
predicts that FP32 arithmetic resolves it: KAPPA_ULP units of roundoff per
term, times kappa, stay below 8e-4.  kappa has three parts: every product that
enters P and Q carries a relative error (the recursive filter's taps at the
scale of their modal terms), and the centred intensity itself is rounded
(the first-order change of the result, over random-sign probes and the
all-pixel ones), and the result itself is rounded when the centre is added
back.  The records below keep, per result, the largest |err| / kappa in units
of roundoff.  kappa is an upper bound: outside (R / sigma_r)^2 of a few
hundred the pixels it excludes also agree to about 1e-4.  Each test's floor on
the gated fraction is what the oracle's kappa gives on that input (computed on
the CPU), rounded down.

Every other pixel is checked as well: it must be finite (the oracle is finite
everywhere: where Q <= 0 both sides keep the pixel's own value), and, for an
even order with the window sum (all weights positive), lie inside the
minimum and maximum of the input over its window.  Each call records the
gated fraction, the largest gated error, and the count and largest error of
the pixels outside the gate; the records go to the JSON file named by the
environment variable BFGP_PARITY_REPORT at the end of the session.
"""
from __future__ import annotations

import numpy as np

TOL = 1e-3
KAPPA_ULP = 6
KAPPA_GATE = 8e-4 * 2.0 ** 24 / KAPPA_ULP
EPS32 = 2.0 ** -24

REPORT = []


def gpu_centre(bf, ws_ptr, plane=0, stream=0) -> float:
    """The centre the FP32 arithmetic used for `plane` (the FP32 value of the
    FP64 mean the statistics pass formed), to hand the oracle the same t_c."""
    tc, _ = bf.bf_gp_get_plane_stats(ws_ptr, plane, stream)
    return float(np.float32(tc))


def window_bounds(f, w):
    """Minimum and maximum of f over the (2w+1)^2 window of every pixel, the
    window clipped at the image edge."""
    from scipy.ndimage import maximum_filter, minimum_filter
    f = np.asarray(f, np.float64)
    return minimum_filter(f, size=2 * w + 1, mode="nearest"), maximum_filter(f, size=2 * w + 1, mode="nearest")


def gate(gpu, ref, kappa=None, *, min_gated=1.0, f=None, window=None, label=""):
    """Assert the parity bar on one result; return (and record) its figures.

    gpu, ref: the GPU result and the oracle's (same shape).  kappa: the
    oracle's conditioning number (None: every pixel is gated).  min_gated:
    the smallest gated fraction expected (a property of the oracle's kappa on
    this input).  f, window: the input and the window half-width, for the
    local min/max bound (even order with the window sum only)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape
    assert np.isfinite(ref).all(), "the oracle is finite everywhere"
    assert np.isfinite(gpu).all(), f"{label}: {int((~np.isfinite(gpu)).sum())} non-finite GPU values"
    gated = np.ones(ref.shape, bool) if kappa is None else (kappa <= KAPPA_GATE)
    err = np.abs(gpu - ref)
    ex = ~gated
    rec = {"label": label, "pixels": int(ref.size), "gated_frac": float(gated.mean()),
           "max_err_gated": float(err[gated].max()) if gated.any() else 0.0,
           "excluded": int(ex.sum()), "max_err_excluded": float(err[ex].max()) if ex.any() else 0.0}
    if kappa is not None:
        k = np.isfinite(kappa) & (kappa > 0)
        rec["max_err_per_kappa_ulp"] = float((err[k] / (kappa[k] * EPS32)).max()) if k.any() else 0.0
    if window is not None:
        lo, hi = window_bounds(f, window)
        out = (gpu < lo - TOL) | (gpu > hi + TOL)
        rec["outside_window_bounds"] = int(out.sum())
    REPORT.append(rec)
    print(f"parity {label}: " + ", ".join(f"{k}={v:.4g}" if isinstance(v, float) else f"{k}={v}"
                                          for k, v in rec.items() if k != "label"))
    assert rec["gated_frac"] >= min_gated, f"{label}: only {rec['gated_frac']:.5f} of the pixels are resolvable"
    assert rec["max_err_gated"] <= TOL, f"{label}: max err {rec['max_err_gated']:.3e} on a resolvable pixel"
    if window is not None:
        assert rec["outside_window_bounds"] == 0, f"{label}: {rec['outside_window_bounds']} pixels leave their window's range"
    return rec


def kept_value_pixels(gpu, f, kappa):
    """Where the oracle's Q <= 0 (kappa = inf) both sides keep the pixel's own
    value: assert the GPU did, and return how many such pixels there are."""
    q0 = ~np.isfinite(kappa)
    assert np.array_equal(np.asarray(gpu, np.float64)[q0], np.asarray(f, np.float64)[q0])
    return int(q0.sum())
