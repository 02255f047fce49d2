"""FP64 CPU oracle for the Gauss-polynomial bilateral filter.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline legs of ``bench.py`` import this package.  It shares no code
with the CUDA library (``paper_1505_00077_gb300``) and never imports it.

The arithmetic lives in ``bf_oracle.c`` (plain C, double precision, OpenMP over
independent lines); this module builds it with gcc and wraps it with ctypes.

Functions (each cites the passage of Chaudhury's paper it follows):

* :func:`direct_bf`  -- O1, Eq. (1)-(2) evaluated by brute force on the window
  [-w, w]^2 (Sec. 1), in-image neighbours only.
* :func:`gp_bf`      -- O2, Algorithm 1 (GPF) / Eqs. (7)-(11) with the centring
  of Sec. 2, spatial operator FIR (Eq. (8)) or Deriche's recursive Gaussian.
* :func:`line_filter`, :func:`deriche_response`, :func:`deriche_coefs` -- the
  1-D spatial operators and the recursive filter's impulse response.
* :func:`gp_adjoint` -- O3, the reverse-mode derivative of O2 (w.r.t. f and sigma_r).
* :func:`gp_kernel` -- Eq. (5), the Gauss-polynomial range kernel.
* :func:`gp_tangent`, :func:`kappa_input` -- the first-order change of O2 under
  relative perturbations of the centred intensity (forward-mode derivative of
  Eqs. (7)-(11)), and the part of the conditioning number kappa it gives.
* :func:`window` -- W = ceil(3 sigma_s) (Sec. 1).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbf_oracle.so")

FIR = 1
IIR = 2

_lib = None


def build(force: bool = False) -> str:
    """Compile bf_oracle.c into oracle/_build/libbf_oracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    dp = ctypes.POINTER(ctypes.c_double)
    i, d = ctypes.c_int, ctypes.c_double
    lib.bfo_direct.argtypes = [dp, i, i, d, d, i, i, i, i, i, dp]
    lib.bfo_direct.restype = None
    ip = ctypes.POINTER(ctypes.c_int)
    lib.bfo_gp.argtypes = [dp, i, i, d, d, i, ip, d, i, i, i, i, i, i, dp, dp, dp]
    lib.bfo_gp_tangent.argtypes = [dp, dp, i, i, d, d, i, ip, d, i, i, i, i, i, i, dp, i, dp, dp, dp, dp, dp]
    lib.bfo_gp_tangent.restype = i
    lib.bfo_gp_probe_sign.argtypes = [ctypes.c_ulonglong, ctypes.c_long, i]
    lib.bfo_gp_probe_sign.restype = d
    lib.bfo_gp.restype = i
    lib.bfo_line_filter.argtypes = [dp, i, i, d, i, i, dp]
    lib.bfo_line_filter.restype = None
    lib.bfo_deriche_response.argtypes = [d, i, dp]
    lib.bfo_deriche_response.restype = None
    lib.bfo_deriche_coefs.argtypes = [d, dp]
    lib.bfo_deriche_coefs.restype = None
    lib.bfo_max_threads.argtypes = []
    lib.bfo_max_threads.restype = i
    lib.bfo_set_threads.argtypes = [i]
    lib.bfo_set_threads.restype = None
    lib.bfo_mean.argtypes = [dp, ctypes.c_long]
    lib.bfo_mean.restype = d
    lib.bfo_gp_adjoint.argtypes = [dp, i, i, d, d, i, d, i, i, dp, dp, dp]
    lib.bfo_gp_adjoint.restype = i
    lib.bfo_gp_kernel.argtypes = [d, d, d, i]
    lib.bfo_gp_kernel.restype = d
    lib.bfo_direct_joint.argtypes = [dp, dp, i, i, d, d, i, i, i, i, i, dp]
    lib.bfo_direct_joint.restype = None
    lib.bfo_gp_joint.argtypes = [dp, dp, i, i, d, d, i, d, i, i, i, i, i, i, dp, dp, dp]
    lib.bfo_gp_joint.restype = i
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _orders(N):
    """(increasing orders as a C int array, count, whether N was a single order)."""
    single = np.isscalar(N)
    ns = [int(N)] if single else [int(n) for n in N]
    if not ns or any(n < 0 for n in ns) or any(b <= a for a, b in zip(ns, ns[1:])):
        raise ValueError(f"orders must be increasing and >= 0: {N}")
    arr = (ctypes.c_int * len(ns))(*ns)
    return arr, len(ns), single


def window(sigma_s: float) -> int:
    """Half-width of the square window: W = ceil(3 sigma_s) (Sec. 1, 'W = 3 sigma_s')."""
    return int(math.ceil(3.0 * sigma_s - 1e-12))


BOX = 10  # BOX + P: P passes of a box of half-width r (window half-width P r)


IIR_ERR = 3  # line_filter only: the recursive filter's tap error scale sum_m |A_m| |p_m|^d


def _spatial(spatial, sigma_s, w, box):
    """(operator code, window half-width) for 'fir', 'iir', 'iir_err' (line_filter only) or 'box'
    (box = (r, passes))."""
    if spatial == "iir_err":
        return IIR_ERR, 0
    if spatial == "box":
        r, passes = (int(v) for v in box)
        if not (r >= 1 and 1 <= passes <= 3):
            raise ValueError(f"bad box {box}")
        return BOX + passes, passes * r
    return (FIR if spatial == "fir" else IIR), (window(sigma_s) if w is None else int(w))


def max_threads() -> int:
    return int(_load().bfo_max_threads())


def set_threads(n: int) -> None:
    _load().bfo_set_threads(int(n))


def _crop(crop, H, W):
    if crop is None:
        return 0, H, 0, W
    r0, r1, c0, c1 = (int(v) for v in crop)
    if not (0 <= r0 < r1 <= H and 0 <= c0 < c1 <= W):
        raise ValueError(f"bad crop {crop} for {H}x{W}")
    return r0, r1, c0, c1


def direct_bf(f, sigma_s, sigma_r, w=None, crop=None):
    """O1: Eq. (1) by direct summation over the window (in-image neighbours)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    H, W = f.shape
    w = window(sigma_s) if w is None else int(w)
    r0, r1, c0, c1 = _crop(crop, H, W)
    out = np.empty((r1 - r0, c1 - c0), np.float64)
    _load().bfo_direct(_ptr(f), H, W, float(sigma_s), float(sigma_r), w, r0, r1, c0, c1, _ptr(out))
    return out


def mean(f) -> float:
    f = np.ascontiguousarray(f, dtype=np.float64)
    return float(_load().bfo_mean(_ptr(f), f.size))


# Probes of the input's part of kappa: four with independent random signs at every pixel
# (delta, eta, xi = +-1), then one each with the same sign everywhere (delta = 1; eta = 1; xi = 1).
_RANDOM_PROBES = [(0.0, 1.0, 0.0, 1.0, 0.0, 1.0, float(seed)) for seed in (11, 12, 13, 14)]
_SYSTEMATIC_PROBES = [(1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0), (0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 0.0),
                      (0.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0)]


def gp_tangent(f, sigma_s, sigma_r, N, spatial="fir", t_c=None, w=None, crop=None, box=None, g=None,
               delta=None, eta=None, xi=None, lam=None, probes=None):
    """First-order change of gp_bf (g given: of gp_bf_joint with guide g) on the
    crop under relative perturbations, per pixel, of the centred intensity
    (delta: in the exponential and the power of Eq. (7) and in G_n = H^n),
    of the argument of the exponential of Eq. (7) alone (eta), and of the
    centred data (xi, joint filter only).  Either explicit [H, W] patterns
    (None = zero), or probes = [(d0, d1, e0, e1, x0, x1, seed), ...] drawn
    with signs s = probe_sign(seed, y W + x, k): delta = d0 + d1 s(k = 0),
    eta = e0 + e1 s(k = 1), xi = x0 + x1 s(k = 2).  lam: per-pixel factor on
    the exponential's argument (None = 1), the point the derivative is taken at.
    N: an order or a list of increasing orders (one pass).  Returns [crop]
    (explicit patterns) or [len(probes), crop], with an order axis after the
    probe axis when N is a list."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    H, W = f.shape
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
    sp, w = _spatial(spatial, sigma_s, w, box)
    r0, r1, c0, c1 = _crop(crop, H, W)

    def arr(a):
        if a is None:
            return None
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), (H, W)))
        return a

    pats = [arr(delta), arr(eta), arr(xi)]
    lam_a = arr(lam)
    explicit = any(a is not None for a in pats)
    if explicit == (probes is not None):
        raise ValueError("give either explicit patterns or probes")
    npr = 1 if explicit else len(probes)
    spec = None if explicit else np.ascontiguousarray(np.array(probes, np.float64).reshape(npr, 7))
    ns, nN, single = _orders(N)
    out = np.empty((npr, nN, r1 - r0, c1 - c0), np.float64)
    tc = float("nan") if t_c is None else float(t_c)
    P = lambda a: _ptr(a) if a is not None else None
    rc = _load().bfo_gp_tangent(_ptr(f), P(gg), H, W, float(sigma_s), float(sigma_r), nN, ns, tc, sp, w,
                                r0, r1, c0, c1, P(lam_a), npr, P(spec), P(pats[0]), P(pats[1]), P(pats[2]),
                                _ptr(out))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    if single:
        out = out[:, 0]
    return out[0] if explicit else out


def probe_sign(seed, pixel, k):
    """The sign gp_tangent draws at pixel index y W + x for component k (0 delta, 1 eta, 2 xi)."""
    return float(_load().bfo_gp_probe_sign(int(seed), int(pixel), int(k)))


def kappa_input(f, sigma_s, sigma_r, N, spatial="fir", t_c=None, w=None, crop=None, box=None, g=None):
    """The input's part of kappa: how far relative errors eps in the centred
    intensity at every pixel (and in the argument of the exponential of
    Eq. (7), and in the centred data for the joint filter) move the result,
    per eps: the root mean square over four probes with independent random
    signs at every pixel (the size of a sum of independent roundings) plus the
    changes under the same sign everywhere (a rounding shared by every pixel,
    such as that of the scale).  N: an order or a list of increasing orders."""
    probes = _RANDOM_PROBES + _SYSTEMATIC_PROBES[:2] + (_SYSTEMATIC_PROBES[2:] if g is not None else [])
    d = gp_tangent(f, sigma_s, sigma_r, N, spatial, t_c=t_c, w=w, crop=crop, box=box, g=g, probes=probes)
    nr = len(_RANDOM_PROBES)
    return np.sqrt(np.mean(d[:nr] ** 2, axis=0)) + np.abs(d[nr:]).sum(axis=0)


def gp_bf(f, sigma_s, sigma_r, N, spatial="fir", t_c=None, w=None, crop=None, return_kappa=False, box=None,
          lam=None):
    """O2: Algorithm 1 (GPF) in FP64.

    spatial: 'fir' (window sum of Eq. (8), zero extension), 'iir' (Deriche's
    recursive Gaussian, causal + anticausal) or 'box' with box = (r, passes):
    the window sum with the passes-fold iterated box of half-width r in place
    of the Gaussian (the paper's constant-time alternative).  t_c: centre (None = image mean,
    the algorithm's first step).  crop: (r0, r1, c0, c1) output region; the
    operator still reads every sample it needs from the full image.  lam:
    per-pixel factor on the argument of the exponential of Eq. (7) (None = 1).
    return_kappa: also return kappa, how far relative errors eps in the
    arithmetic move the result (error about kappa * eps; inf where Q <= 0):
    the terms' part sigma_r (sum|p_n| + |P/Q| sum|q_n|) / |Q| (a relative
    error in every product entering Eqs. (9)-(10)) plus kappa_input (the
    rounding of the centred intensity itself) plus |y| (the rounding of the
    result itself when the centre is added back).  return_kappa="parts" returns
    (y, kappa, terms' part, input's part).  Where Q <= 0, Eq. (11) is undefined
    and the pixel keeps its own value (kappa = inf there).  N: an order, or a
    list of increasing orders computed in one pass (results stacked on a first
    axis): the terms of order N are a prefix of Algorithm 1's loop.
    """
    f = np.ascontiguousarray(f, dtype=np.float64)
    H, W = f.shape
    sp, w = _spatial(spatial, sigma_s, w, box)
    r0, r1, c0, c1 = _crop(crop, H, W)
    ns, nN, single = _orders(N)
    out = np.empty((nN, r1 - r0, c1 - c0), np.float64)
    kap = np.empty_like(out) if return_kappa else None
    tc = float("nan") if t_c is None else float(t_c)
    lam_a = None if lam is None else np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float64), (H, W)))
    rc = _load().bfo_gp(_ptr(f), H, W, float(sigma_s), float(sigma_r), nN, ns, tc, sp, w,
                        r0, r1, c0, c1, _ptr(lam_a) if lam_a is not None else None, _ptr(out),
                        _ptr(kap) if kap is not None else None)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    if single:
        out = out[0]
        kap = kap[0] if kap is not None else None
    if not return_kappa:
        return out
    ku = kappa_input(f, sigma_s, sigma_r, N, spatial, t_c=t_c, w=w, crop=crop, box=box)
    # the last operation, adding the centre back (Eq. (6)), rounds the result itself: eps |y|
    total = np.where(np.isfinite(kap), kap + ku + np.abs(out), np.inf)
    return (out, total, kap, ku) if return_kappa == "parts" else (out, total)


def direct_bf_joint(f, g, sigma_s, sigma_r, w=None, crop=None):
    """Joint (cross) bilateral filter by direct summation: Eq. (1) with the range
    kernel on the guide g and the data f."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    assert f.shape == g.shape
    H, W = f.shape
    w = window(sigma_s) if w is None else int(w)
    r0, r1, c0, c1 = _crop(crop, H, W)
    out = np.empty((r1 - r0, c1 - c0), np.float64)
    _load().bfo_direct_joint(_ptr(f), _ptr(g), H, W, float(sigma_s), float(sigma_r), w, r0, r1, c0, c1, _ptr(out))
    return out


def gp_bf_joint(f, g, sigma_s, sigma_r, N, spatial="fir", t_c=None, w=None, crop=None, return_kappa=False,
                box=None, lam=None):
    """Joint (cross) bilateral filter by the Gauss-polynomial decomposition in
    FP64: Algorithm 1 with the range kernel on the centred guide g (t_c = None:
    the guide's mean), 2 (N + 1) filterings (F_n and F_n (f - t_c)).  Arguments
    as gp_bf; kappa without the sigma_r factor, its input's part also counting
    a relative error in the centred data."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    assert f.shape == g.shape
    H, W = f.shape
    sp, w = _spatial(spatial, sigma_s, w, box)
    r0, r1, c0, c1 = _crop(crop, H, W)
    out = np.empty((r1 - r0, c1 - c0), np.float64)
    kap = np.empty_like(out) if return_kappa else None
    tc = float("nan") if t_c is None else float(t_c)
    lam_a = None if lam is None else np.ascontiguousarray(np.broadcast_to(np.asarray(lam, np.float64), (H, W)))
    rc = _load().bfo_gp_joint(_ptr(f), _ptr(g), H, W, float(sigma_s), float(sigma_r), int(N), tc, sp, w,
                              r0, r1, c0, c1, _ptr(lam_a) if lam_a is not None else None, _ptr(out),
                              _ptr(kap) if kap is not None else None)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    if not return_kappa:
        return out
    ku = kappa_input(f, sigma_s, sigma_r, N, spatial, t_c=t_c, w=w, crop=crop, box=box, g=g)
    # the last operation, adding the centre back (Eq. (6)), rounds the result itself: eps |y|
    total = np.where(np.isfinite(kap), kap + ku + np.abs(out), np.inf)
    return (out, total, kap, ku) if return_kappa == "parts" else (out, total)


def gp_adjoint(f, sigma_s, sigma_r, N, ybar, spatial="fir", t_c=None, w=None, box=None):
    """O3: reverse-mode derivative of gp_bf (Algorithm 1) on the full image.

    Returns (dL/df, dL/dsigma_r) for L = sum(ybar * gp_bf(f, ...)).  t_c=None is
    the mean centre of the algorithm's first step (its derivative included);
    a given t_c is held fixed.
    """
    f = np.ascontiguousarray(f, dtype=np.float64)
    H, W = f.shape
    yb = np.ascontiguousarray(ybar, dtype=np.float64)
    assert yb.shape == f.shape
    sp, w = _spatial(spatial, sigma_s, w, box)
    fb = np.empty_like(f)
    srb = np.zeros(1)
    tc = float("nan") if t_c is None else float(t_c)
    rc = _load().bfo_gp_adjoint(_ptr(f), H, W, float(sigma_s), float(sigma_r), int(N), tc,
                                sp, w, _ptr(yb), _ptr(fb), _ptr(srb))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return fb, float(srb[0])


def line_filter(x, sigma_s, spatial="fir", w=None, box=None):
    """The 1-D spatial operator applied to each row of x (zero extension)."""
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    count, n = x.shape
    sp, w = _spatial(spatial, sigma_s, w, box)
    y = np.empty_like(x)
    _load().bfo_line_filter(_ptr(x), count, n, float(sigma_s), sp, w, _ptr(y))
    return y


def deriche_response(sigma_s, n):
    """h(d), d = 0..n-1, of the recursive Gaussian at scale sigma_s."""
    h = np.empty(int(n), np.float64)
    _load().bfo_deriche_response(float(sigma_s), int(n), _ptr(h))
    return h


def gp_kernel(t, tau, sigma_r, N):
    """Eq. (5): degree-N Gauss-polynomial approximation of g_{sigma_r}(t - tau)."""
    lib = _load()
    t = np.asarray(t, np.float64)
    flat = [lib.bfo_gp_kernel(float(v), float(tau), float(sigma_r), int(N)) for v in t.ravel()]
    return np.array(flat, np.float64).reshape(t.shape)


def deriche_coefs(sigma_s):
    """(poles[2], residues[2]) as complex numpy arrays."""
    o = np.empty(8, np.float64)
    _load().bfo_deriche_coefs(float(sigma_s), _ptr(o))
    return o[0:4:2] + 1j * o[1:4:2], o[4:8:2] + 1j * o[5:8:2]
