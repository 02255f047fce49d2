"""Pins for the FP64 oracle (CPU only, no GPU).

Every test checks the oracle against something other than its own code:
brute force on tiny images, closed forms, library routines (scipy), exact
invariants stated or implied by the paper, the Taylor-remainder bound of
Eq. (4), and the numbers the paper prints (tests/golden/paper_values.json).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.ndimage import correlate1d

import oracle
import synthetic

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))

# Deriche's published 4th-order constants, restated here in his real (cos/sin)
# form so the oracle's complex-pole form is checked against an independent
# evaluation.
_DERICHE = dict(a0=1.680, a1=3.735, b0=1.783, b1=1.723, c0=-0.6803, c1=-0.2598, w0=0.6318, w1=1.997)


def deriche_real(d, sigma):
    k = _DERICHE
    x = np.abs(np.asarray(d, np.float64)) / sigma
    return ((k["a0"] * np.cos(k["w0"] * x) + k["a1"] * np.sin(k["w0"] * x)) * np.exp(-k["b0"] * x)
            + (k["c0"] * np.cos(k["w1"] * x) + k["c1"] * np.sin(k["w1"] * x)) * np.exp(-k["b1"] * x))


def brute_bf(f, spatial_weight, sigma_r, w):
    """Literal Eq. (1): four nested loops, in-image neighbours only."""
    H, W = f.shape
    out = np.empty((H, W))
    for y in range(H):
        for x in range(W):
            num = den = 0.0
            for dy in range(-w, w + 1):
                for dx in range(-w, w + 1):
                    yy, xx = y - dy, x - dx
                    if 0 <= yy < H and 0 <= xx < W:
                        t = float(f[yy, xx])
                        rng = 1.0 if math.isinf(sigma_r) else math.exp(-(t - f[y, x]) ** 2 / (2 * sigma_r ** 2))
                        g = spatial_weight(dx, dy) * rng
                        num += g * t
                        den += g
            out[y, x] = num / den
    return out


def small_image(H, W, seed, n_rect=6, noise=10.0, ramp=0.0):
    return synthetic.make_image(H, W, n_rect, noise, ramp, seed).astype(np.float64)


def gauss_filter_scipy(a, sigma_s, w):
    taps = np.exp(-np.arange(-w, w + 1) ** 2 / (2.0 * sigma_s ** 2))
    return correlate1d(correlate1d(a, taps, axis=1, mode="constant"), taps, axis=0, mode="constant")


# ------------------------------------------------------------------ O1 direct


@pytest.mark.parametrize("ss,sr", [(1.0, 20.0), (1.5, 40.0), (2.0, 10.0)])
def test_direct_matches_brute_force(ss, sr):
    f = small_image(11, 9, 11, n_rect=4)
    w = oracle.window(ss)
    ref = brute_bf(f, lambda dx, dy: math.exp(-(dx * dx + dy * dy) / (2 * ss * ss)), sr, w)
    np.testing.assert_allclose(oracle.direct_bf(f, ss, sr), ref, rtol=0, atol=1e-11)


def test_direct_crop_is_slice():
    f = small_image(30, 26, 12)
    full = oracle.direct_bf(f, 2.0, 25.0)
    np.testing.assert_array_equal(oracle.direct_bf(f, 2.0, 25.0, crop=(5, 17, 3, 20)), full[5:17, 3:20])


def test_direct_shift_equivariance_prop_2_1():
    """Proposition (Eq. (6)): f_BF(i) = h_BF(i) + t_c for h = f - t_c."""
    f = small_image(24, 20, 13)
    tc = 97.25
    np.testing.assert_allclose(oracle.direct_bf(f - tc, 2.0, 30.0) + tc, oracle.direct_bf(f, 2.0, 30.0),
                               rtol=0, atol=1e-10)


def test_window_rule():
    """W = 3 sigma_s (Sec. 1), rounded up for non-integer sigma_s."""
    assert oracle.window(3.0) == 9
    assert oracle.window(10.0) == 30
    assert oracle.window(1.2) == 4


# --------------------------------------------------------- spatial operators


@pytest.mark.parametrize("sigma", [1.5, 3.0, 10.0, 25.0])
def test_deriche_impulse_response(sigma):
    d = np.arange(0, int(6 * sigma) + 1)
    h = oracle.deriche_response(sigma, len(d))
    # complex-pole form equals Deriche's real form
    np.testing.assert_allclose(h, deriche_real(d, sigma), rtol=0, atol=1e-12)
    # the published fit approximates exp(-d^2 / 2 sigma^2) to about 5e-4 of the peak
    assert np.abs(h - np.exp(-d ** 2 / (2.0 * sigma ** 2))).max() < 6e-4


@pytest.mark.parametrize("sigma,n", [(2.0, 17), (5.0, 40), (12.0, 64)])
def test_iir_line_operator_is_symmetric_toeplitz(sigma, n):
    """Causal + anticausal recursions with zero state = the matrix h(|i - j|)."""
    M = oracle.line_filter(np.eye(n), sigma, "iir")  # row l = S e_l
    i = np.arange(n)
    ref = deriche_real(i[:, None] - i[None, :], sigma)
    np.testing.assert_allclose(M, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("sigma,n", [(2.0, 40), (7.5, 90)])
def test_iir_error_scale_is_the_modal_magnitude(sigma, n):
    """The recursive filter's tap error scale used by kappa, M(d) = sum_m |A_m| |p_m|^d
    (the magnitudes of the modal terms that h(d) is formed from), filtered by its
    recursions, equals the explicit convolution with M; M >= |h| everywhere, and far
    above it where the terms cancel (around the kernel's negative lobe)."""
    p, A = oracle.deriche_coefs(sigma)
    d = np.arange(n)
    M = sum(abs(A[m]) * abs(p[m]) ** d for m in range(2))
    x = np.random.default_rng(8).normal(size=(3, n))
    y = oracle.line_filter(x, sigma, "iir_err")
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    np.testing.assert_allclose(y, x @ M[np.abs(i - j)].T, rtol=1e-12, atol=1e-12)
    h = np.abs(oracle.deriche_response(sigma, n))
    assert np.all(M >= h) and np.max(M[1:] / h[1:]) > 5


@pytest.mark.parametrize("sigma", [1.0, 3.0, 4.5])
def test_fir_line_matches_scipy(sigma):
    x = np.random.default_rng(5).normal(size=(3, 50))
    w = oracle.window(sigma)
    taps = np.exp(-np.arange(-w, w + 1) ** 2 / (2.0 * sigma ** 2))
    np.testing.assert_allclose(oracle.line_filter(x, sigma, "fir"), correlate1d(x, taps, axis=1, mode="constant"),
                               rtol=0, atol=1e-12)


# ----------------------------------------------------------------- O2 GPF


@pytest.mark.parametrize("sr,N", [(30.0, 60), (50.0, 40)])
def test_gp_fir_converges_to_direct(sr, N):
    """With enough terms the Taylor series of Eq. (4) is exact, so Algorithm 1
    with the window sum of Eq. (8) reproduces Eq. (1)."""
    f = small_image(40, 36, 21, n_rect=8)
    np.testing.assert_allclose(oracle.gp_bf(f, 2.0, sr, N, "fir"), oracle.direct_bf(f, 2.0, sr), rtol=0, atol=1e-9)


def test_gp_iir_converges_to_brute_force_with_recursive_kernel():
    """Algorithm 1 with the recursive Gaussian = Eq. (1) with the spatial kernel
    h(|dx|) h(|dy|) over the whole image (brute force, Deriche's real form)."""
    f = small_image(12, 10, 22, n_rect=4)
    sigma = 2.5
    ref = brute_bf(f, lambda dx, dy: float(deriche_real(dx, sigma) * deriche_real(dy, sigma)), 40.0, 12)
    np.testing.assert_allclose(oracle.gp_bf(f, sigma, 40.0, 50, "iir"), ref, rtol=0, atol=1e-9)


def test_gp_equals_explicit_eqs_7_to_11():
    """Algorithm 1's recursive powers and factorials equal Eqs. (7)-(11) written
    out with explicit powers, factorials and scipy's separable filter."""
    f = small_image(32, 28, 23, n_rect=6)
    ss, sr, N = 2.0, 30.0, 12
    w = oracle.window(ss)
    tc = f.mean()
    h = f - tc
    G = lambda n: (h / sr) ** n                                  # Eq. (7)
    F = lambda n: np.exp(-h ** 2 / (2 * sr ** 2)) * G(n)          # Eq. (7)
    Fb = [gauss_filter_scipy(F(n), ss, w) for n in range(N + 2)]  # Eq. (8)
    P = sr * sum(G(n) * Fb[n + 1] / math.factorial(n) for n in range(N + 1))  # Eq. (9)
    Q = sum(G(n) * Fb[n] / math.factorial(n) for n in range(N + 1))           # Eq. (10)
    ref = P / Q + tc                                              # Eq. (11) + Eq. (6)
    np.testing.assert_allclose(oracle.gp_bf(f, ss, sr, N, "fir"), ref, rtol=0, atol=1e-10)


def _remainder_bound(f, ss, sr, N, w, tc):
    """Per-pixel bound on |GPF - Eq. (1)| from the Lagrange remainder of Eq. (4):
    |exp(x) - T_N(x)| <= |x|^{N+1} / (N+1)! * exp(max(x, 0))."""
    H, W = f.shape
    h = f - tc
    bound = np.empty((H, W))
    for y in range(H):
        for x in range(W):
            y0, y1 = max(0, y - w), min(H, y + w + 1)
            x0, x1 = max(0, x - w), min(W, x + w + 1)
            t = h[y0:y1, x0:x1]
            tau = h[y, x]
            dy = np.arange(y0, y1)[:, None] - y
            dx = np.arange(x0, x1)[None, :] - x
            gs = np.exp(-(dx ** 2 + dy ** 2) / (2 * ss ** 2))
            xx = tau * t / sr ** 2
            e = np.exp(-(tau ** 2 + t ** 2) / (2 * sr ** 2)) * np.abs(xx) ** (N + 1) / math.factorial(N + 1) \
                * np.exp(np.maximum(xx, 0))
            g = np.exp(-(t - tau) ** 2 / (2 * sr ** 2))
            D = (gs * g).sum()
            Nn = (gs * g * t).sum()
            eD = (gs * e).sum()
            eN = (gs * e * np.abs(t)).sum()
            bound[y, x] = (eN + abs(Nn / D) * eD) / (D - eD) if D > eD else np.inf
    return bound


@pytest.mark.parametrize("sr,N", [(50.0, 6), (50.0, 10), (35.0, 14), (30.0, 20)])
def test_gp_error_within_taylor_remainder_bound(sr, N):
    f = small_image(20, 18, 24, n_rect=5)
    ss, w = 2.0, oracle.window(2.0)
    tc = f.mean()
    err = np.abs(oracle.gp_bf(f, ss, sr, N, "fir") - oracle.direct_bf(f, ss, sr))
    bound = _remainder_bound(f, ss, sr, N, w, tc)
    assert np.all(err <= bound * (1 + 1e-9) + 1e-10)
    assert err.max() > 0  # the truncation is visible at these orders


def test_constant_image_is_unchanged():
    c = 77.25
    f = np.full((32, 32), c)
    for sp in ("fir", "iir"):
        assert np.all(oracle.gp_bf(f, 3.0, 30.0, 20, sp) == c)
    np.testing.assert_allclose(oracle.direct_bf(f, 3.0, 30.0), c, rtol=0, atol=1e-12)


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_sigma_r_infinite_is_normalised_gaussian(sp):
    """sigma_r -> inf: the range kernel is 1 and Eq. (1) is the normalised spatial filter."""
    f = small_image(26, 22, 25)
    ss = 2.0
    w = oracle.window(ss)
    if sp == "fir":
        ref = gauss_filter_scipy(f, ss, w) / gauss_filter_scipy(np.ones_like(f), ss, w)
        np.testing.assert_allclose(oracle.direct_bf(f, ss, math.inf), ref, rtol=0, atol=1e-10)
    else:
        Srow = lambda a: oracle.line_filter(a, ss, "iir")
        S = lambda a: Srow(Srow(a).T).T
        ref = S(f) / S(np.ones_like(f))
    np.testing.assert_allclose(oracle.gp_bf(f, ss, math.inf, 20, sp), ref, rtol=0, atol=1e-10)
    # finite but huge sigma_r approaches the limit at rate O((R / sigma_r)^2 R)
    np.testing.assert_allclose(oracle.gp_bf(f, ss, 1e6, 20, sp), ref, rtol=0, atol=1e-5)


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_negation_symmetry(sp):
    f = small_image(30, 24, 26)
    np.testing.assert_allclose(oracle.gp_bf(-f, 3.0, 30.0, 20, sp), -oracle.gp_bf(f, 3.0, 30.0, 20, sp),
                               rtol=0, atol=1e-11)


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_affine_equivariance(sp):
    """GP with sigma_r scaled by a on a f + b equals a GP(f) + b."""
    f = small_image(30, 24, 27)
    a, b = 2.0, 10.0
    np.testing.assert_allclose(oracle.gp_bf(a * f + b, 3.0, a * 30.0, 20, sp), a * oracle.gp_bf(f, 3.0, 30.0, 20, sp) + b,
                               rtol=0, atol=1e-9)


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_transpose_equivariance(sp):
    f = small_image(30, 22, 28)
    np.testing.assert_allclose(oracle.gp_bf(f.T.copy(), 2.5, 25.0, 20, sp), oracle.gp_bf(f, 2.5, 25.0, 20, sp).T,
                               rtol=0, atol=1e-9)


@pytest.mark.parametrize("sr", [15.0, 30.0, 60.0])
def test_even_order_stays_within_local_min_max(sr):
    """Even N: the truncated exponential is positive, so every weight is positive
    and the output is a convex combination of the window's intensities."""
    f = small_image(40, 40, 29, n_rect=8)
    ss = 2.0
    w = oracle.window(ss)
    y = oracle.gp_bf(f, ss, sr, 20, "fir")
    from scipy.ndimage import maximum_filter, minimum_filter
    lo = minimum_filter(f, size=2 * w + 1, mode="nearest")
    hi = maximum_filter(f, size=2 * w + 1, mode="nearest")
    assert np.all(y >= lo - 1e-9) and np.all(y <= hi + 1e-9)


@pytest.mark.parametrize("sr", [30.0, 50.0])
def test_error_decreases_with_even_order(sr):
    f = synthetic.make_image(48, 48, 8, 10.0, 0.0, synthetic.seed_for(1, 77)).astype(np.float64)
    ref = oracle.direct_bf(f, 3.0, sr)
    mse = [np.mean((oracle.gp_bf(f, 3.0, sr, N, "fir") - ref) ** 2) for N in range(4, 42, 2)]
    assert all(b <= a for a, b in zip(mse, mse[1:])), mse


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_crop_equals_full_slice(sp):
    f = small_image(48, 40, 30)
    full = oracle.gp_bf(f, 3.0, 25.0, 20, sp)
    tc = f.mean()
    part = oracle.gp_bf(f, 3.0, 25.0, 20, sp, t_c=tc, crop=(9, 31, 4, 27))
    np.testing.assert_allclose(part, full[9:31, 4:27], rtol=0, atol=1e-10)


def test_odd_order_can_give_non_positive_denominator():
    """Odd N: the truncated exponential has a real root, so Q <= 0 can happen; Eq. (11)
    is undefined there and the pixel keeps its own value (the reading for that case).
    Even N with the window sum never has Q <= 0."""
    f = np.zeros((16, 16))
    f[:, 8] = 255.0  # a thin bright line: its pixels see mostly negative weights
    y, k = oracle.gp_bf(f, 3.0, 20.0, 5, "fir", return_kappa=True)
    assert np.all(y[:, 8] == 255.0) and np.all(np.isinf(k[:, 8]))
    others = np.delete(y, 8, axis=1)
    assert np.all(np.isfinite(np.delete(k, 8, axis=1))) and np.all(others < 255.0)
    _, k6 = oracle.gp_bf(f, 3.0, 20.0, 6, "fir", return_kappa=True)
    assert np.all(np.isfinite(k6))


def test_adjoint_where_the_denominator_is_not_positive():
    """O3 with pixels whose Q <= 0 (odd N): they pass dL/dy to their own input,
    against central differences of O2 (which keeps their value there)."""
    f = np.zeros((9, 10))
    f[:, 5] = 255.0
    f += synthetic.make_image(9, 10, 2, 4.0, 0.0, synthetic.seed_for(9, 47)).astype(np.float64) * 0.05
    _, k = oracle.gp_bf(f, 1.5, 20.0, 5, "fir", return_kappa=True)
    assert np.isinf(k).sum() >= 5  # some pixels take the Q <= 0 branch
    yb = np.random.default_rng(7).normal(size=f.shape)
    g, gs = oracle.gp_adjoint(f, 1.5, 20.0, 5, yb, "fir")
    L = lambda ff, sr=20.0: float((yb * oracle.gp_bf(ff, 1.5, sr, 5, "fir")).sum())
    eps = 1e-5
    fd = np.empty_like(f)
    for idx in np.ndindex(f.shape):
        e = np.zeros_like(f)
        e[idx] = eps
        fd[idx] = (L(f + e) - L(f - e)) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-6 * max(1.0, np.abs(fd).max()))
    fds = (L(f, 20.0 + 1e-4) - L(f, 20.0 - 1e-4)) / 2e-4
    assert abs(gs - fds) <= 1e-6 * max(1.0, abs(fds))


# ------------------------------------------------------- Eq. (5) and Fig. 1-3


def test_fig1_scale_factor():
    g = GOLDEN["fig1_scale_factor"]
    tau, sr = g["tau"], g["sigma_r"]
    # at t = 0 the Gauss-polynomial is exactly the scale factor exp(-tau^2 / 2 sigma_r^2)
    v = float(oracle.gp_kernel(np.array([0.0]), tau, sr, 20)[0])
    assert float(f"{v:.{g['printed_digits']}g}") == g["printed"]
    # and the decomposition of Eq. (3) is exact once the series has converged
    t = np.linspace(0.0, 255.0, 256)
    np.testing.assert_allclose(oracle.gp_kernel(t, tau, sr, 90), np.exp(-(t - tau) ** 2 / (2 * sr ** 2)),
                               rtol=0, atol=1e-12)


def test_tau_zero_needs_no_approximation():
    """Sec. 2: for tau = 0 the exponential factor is 1, so any degree is exact."""
    t = np.linspace(-255.0, 255.0, 101)
    for N in (0, 1, 5, 20):
        np.testing.assert_allclose(oracle.gp_kernel(t, 0.0, 30.0, N), np.exp(-t ** 2 / 1800.0), rtol=1e-15, atol=0)


def test_centring_reduces_kernel_error():
    """Sec. 2 / Fig. 3: degree 20 at sigma_r 30.  Over [0, 255] with tau in
    {0, 10, 50, 120} (Fig. 3(a)) the worst error is far larger than over the
    centred interval [-127.5, 127.5] with tau in {-100, -50, 0, 10, 50, 100}
    (Fig. 3(b)); centring shrinks max |tau| (e.g. 255 -> 155 at t_c = 100)."""
    g = GOLDEN["centring_example"]
    L, U, tc = g["L"], g["U"], g["t_c"]
    assert max(abs(L - tc), abs(U - tc)) == g["max_abs_tau_after"]
    assert max(abs(L), abs(U)) == g["max_abs_tau_before"]

    def worst(t, taus):
        return max(np.abs(oracle.gp_kernel(t, tau, 30.0, 20) - np.exp(-(t - tau) ** 2 / 1800.0)).max() for tau in taus)

    raw = worst(np.linspace(0.0, 255.0, 256), (0.0, 10.0, 50.0, 120.0))
    centred = worst(np.linspace(-127.5, 127.5, 256), (-100.0, -50.0, 0.0, 10.0, 50.0, 100.0))
    assert centred < 0.5 * raw
    # and for a fixed centre, the worst error shrinks as max |tau| shrinks
    assert worst(np.linspace(-tc, U - tc, 256), (-tc, U - tc)) < worst(np.linspace(L, U, 256), (L, U))


def test_error_grows_with_abs_tau():
    """Sec. 2 / Fig. 3(a): for fixed degree the error grows with |tau|."""
    t = np.linspace(0.0, 255.0, 256)
    errs = [np.abs(oracle.gp_kernel(t, tau, 30.0, 20) - np.exp(-(t - tau) ** 2 / 1800.0)).max() for tau in (0, 10, 50, 120)]
    assert errs[0] < 1e-15 and errs[1] < errs[2] < errs[3]


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_kappa_lower_bound_and_equality(sp):
    """The terms' part of kappa is >= 2 |y - t_c| by the triangle inequality; with
    non-negative terms (f >= t_c = 0 and the positive window weights) it is equal.
    The total adds the input's part, which is non-negative, and |y| (the final
    rounding)."""
    f = small_image(30, 26, 31)
    y, k, kt, ku = oracle.gp_bf(f, 2.0, 30.0, 20, sp, return_kappa="parts")
    tc = f.mean()
    assert np.all(kt >= 2 * np.abs(y - tc) * (1 - 1e-12))
    assert np.all(ku >= 0) and np.array_equal(k, kt + ku + np.abs(y))
    if sp == "fir":
        y0, _, k0, _ = oracle.gp_bf(f, 2.0, 30.0, 20, sp, t_c=0.0, return_kappa="parts")
        np.testing.assert_allclose(k0, 2 * np.abs(y0), rtol=1e-12)


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_several_orders_in_one_pass(sp):
    """The terms of order N are a prefix of Algorithm 1's loop: a list of orders in
    one pass gives, bit for bit, what each order gives alone (result, kappa, tangent)."""
    f = small_image(40, 33, 48, n_rect=6)
    Ns = [0, 3, 4, 10, 20]
    ys, ks = oracle.gp_bf(f, 2.0, 25.0, Ns, sp, return_kappa=True)
    for q, n in enumerate(Ns):
        y, k = oracle.gp_bf(f, 2.0, 25.0, n, sp, return_kappa=True)
        assert np.array_equal(y, ys[q]) and np.allclose(k, ks[q], rtol=1e-12, atol=0)


# ------------------------------------------- first-order sensitivity to the input's rounding


def _pm1(shape, seed):
    return np.random.default_rng(seed).choice([-1.0, 1.0], size=shape)


@pytest.mark.parametrize("sp,ss,sr", [("fir", 1.5, 25.0), ("fir", 2.0, 10.0), ("iir", 2.0, 25.0), ("iir", 3.0, 10.0),
                                      ("fir", 1.5, math.inf), ("iir", 2.0, math.inf)])
def test_tangent_matches_central_differences(sp, ss, sr):
    """gp_tangent is the derivative of Eqs. (7)-(11): against central differences of
    O2 under h -> h (1 + e delta) (the centred intensity, given centre) and under a
    per-pixel factor 1 + e eta on the exponential's argument."""
    f = small_image(14, 11, 44, n_rect=5)
    tc = float(f.mean())
    d, e = _pm1(f.shape, 1), _pm1(f.shape, 2)
    t = oracle.gp_tangent(f, ss, sr, 12, sp, t_c=tc, delta=d, eta=e)
    eps = 1e-6
    yp = oracle.gp_bf(tc + (f - tc) * (1 + eps * d), ss, sr, 12, sp, t_c=tc, lam=1 + eps * e)
    ym = oracle.gp_bf(tc + (f - tc) * (1 - eps * d), ss, sr, 12, sp, t_c=tc, lam=1 - eps * e)
    fd = (yp - ym) / (2 * eps)
    np.testing.assert_allclose(t, fd, rtol=0, atol=1e-9 * max(1.0, np.abs(fd).max()) + 1e-7)
    # each part alone (a dropped term in either would show here)
    td = oracle.gp_tangent(f, ss, sr, 12, sp, t_c=tc, delta=d)
    te = oracle.gp_tangent(f, ss, sr, 12, sp, t_c=tc, eta=e)
    np.testing.assert_allclose(td + te, t, rtol=1e-12, atol=1e-12)
    fde = (oracle.gp_bf(f, ss, sr, 12, sp, t_c=tc, lam=1 + eps * e)
           - oracle.gp_bf(f, ss, sr, 12, sp, t_c=tc, lam=1 - eps * e)) / (2 * eps)
    np.testing.assert_allclose(te, fde, rtol=0, atol=1e-9 * max(1.0, np.abs(fde).max()) + 1e-7)


@pytest.mark.parametrize("sp,ss", [("fir", 1.5), ("iir", 2.5)])
def test_joint_tangent_matches_central_differences(sp, ss):
    """The joint filter's tangent: guide intensity (delta), exponential's argument (eta)
    and data (xi), against central differences of its O2."""
    f = small_image(14, 11, 45, n_rect=5)
    g = small_image(14, 11, 46, n_rect=4)
    tc = float(g.mean())
    d, e, x = _pm1(f.shape, 3), _pm1(f.shape, 4), _pm1(f.shape, 5)
    t = oracle.gp_tangent(f, ss, 25.0, 12, sp, t_c=tc, g=g, delta=d, eta=e, xi=x)
    eps = 1e-6
    yp = oracle.gp_bf_joint(tc + (f - tc) * (1 + eps * x), tc + (g - tc) * (1 + eps * d), ss, 25.0, 12, sp, t_c=tc,
                            lam=1 + eps * e)
    ym = oracle.gp_bf_joint(tc + (f - tc) * (1 - eps * x), tc + (g - tc) * (1 - eps * d), ss, 25.0, 12, sp, t_c=tc,
                            lam=1 - eps * e)
    fd = (yp - ym) / (2 * eps)
    np.testing.assert_allclose(t, fd, rtol=0, atol=1e-9 * max(1.0, np.abs(fd).max()) + 1e-7)


def test_probe_signs_are_balanced_and_independent():
    """The drawn probe signs: +-1, mean near 0, no correlation between the three
    components or between seeds (Rademacher probes)."""
    n = 200000
    s = np.array([[oracle.probe_sign(seed, j, k) for j in range(0, n, 97)] for seed in (11, 12) for k in (0, 1, 2)])
    assert set(np.unique(s)) == {-1.0, 1.0}
    assert np.all(np.abs(s.mean(axis=1)) < 0.03)
    c = np.corrcoef(s)
    assert np.all(np.abs(c[~np.eye(len(c), dtype=bool)]) < 0.05)


@pytest.mark.parametrize("sp,ss,sr", [("fir", 2.0, 30.0), ("iir", 3.0, 10.0)])
def test_kappa_input_predicts_the_change_under_rounding(sp, ss, sr):
    """kappa_input * eps is the size of the change of O2 when every pixel's centred
    intensity and exponential argument carry an independent relative error of up to
    eps (as rounding gives): over 6 such random perturbations the change stays below
    3 kappa_input eps everywhere, and reaches a fair share of it (the prediction is not
    vacuous).  And a perturbation by the same factor everywhere moves O2 by at most
    kappa_input eps."""
    f = synthetic.make_image(40, 36, 8, 10.0, 30.0, synthetic.seed_for(9, 46)).astype(np.float64)
    tc = float(f.mean())
    y = oracle.gp_bf(f, ss, sr, 20, sp, t_c=tc)
    ku = oracle.kappa_input(f, ss, sr, 20, sp, t_c=tc)
    eps = 1e-7
    rng = np.random.default_rng(6)
    ratios = []
    for _ in range(6):
        d, e = rng.uniform(-1, 1, size=(2,) + f.shape)
        dy = oracle.gp_bf(tc + (f - tc) * (1 + eps * d), ss, sr, 20, sp, t_c=tc, lam=1 + eps * e) - y
        ratios.append(np.abs(dy) / (ku * eps))
    r = np.max(ratios, axis=0)
    assert r.max() <= 3.0, r.max()
    assert np.median(r) >= 0.1, np.median(r)
    dy = oracle.gp_bf(tc + (f - tc) * (1 + eps), ss, sr, 20, sp, t_c=tc) - y
    assert np.all(np.abs(dy) <= ku * eps * (1 + 1e-3) + 1e-12)


# --------------------------------------------------------------- O3 adjoint

@pytest.mark.parametrize("sp,ss", [("fir", 1.5), ("iir", 2.0)])
def test_spatial_operator_is_self_adjoint(sp, ss):
    """<S x, z> = <x, S z>: the backward pass filters the adjoint channels with S itself."""
    rng = np.random.default_rng(3)
    x, z = rng.normal(size=(2, 5, 41))
    Sx, Sz = oracle.line_filter(x, ss, sp), oracle.line_filter(z, ss, sp)
    np.testing.assert_allclose((Sx * z).sum(axis=1), (x * Sz).sum(axis=1), rtol=1e-12, atol=0)


@pytest.mark.parametrize("sp,ss", [("fir", 1.5), ("iir", 2.0)])
@pytest.mark.parametrize("tc", [None, 110.0])
def test_adjoint_matches_central_differences_every_pixel(sp, ss, tc):
    """O3 against central differences of O2 in FP64, pixel by pixel on a tiny image,
    for the mean centre (its derivative included) and a fixed centre."""
    f = small_image(9, 8, 41, n_rect=3)
    yb = np.random.default_rng(4).normal(size=f.shape)
    g, gs = oracle.gp_adjoint(f, ss, 25.0, 10, yb, sp, t_c=tc)
    L = lambda ff, sr=25.0: float((yb * oracle.gp_bf(ff, ss, sr, 10, sp, t_c=tc)).sum())
    eps = 1e-4
    fd = np.empty_like(f)
    for idx in np.ndindex(f.shape):
        e = np.zeros_like(f)
        e[idx] = eps
        fd[idx] = (L(f + e) - L(f - e)) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=0, atol=1e-7 * max(1.0, np.abs(fd).max()))
    fds = (L(f, 25.0 + 1e-4) - L(f, 25.0 - 1e-4)) / 2e-4
    assert abs(gs - fds) <= 1e-7 * max(1.0, abs(fds))


@pytest.mark.parametrize("sp,ss", [("fir", 3.0), ("iir", 5.0)])
def test_adjoint_directional_derivatives(sp, ss):
    """Random directions on a 48 x 40 image: <grad, v> = d/dt L(f + t v)."""
    f = small_image(48, 40, 42, n_rect=8)
    rng = np.random.default_rng(5)
    yb = rng.normal(size=f.shape)
    g, _ = oracle.gp_adjoint(f, ss, 25.0, 20, yb, sp)
    L = lambda ff: float((yb * oracle.gp_bf(ff, ss, 25.0, 20, sp)).sum())
    for _ in range(6):
        v = rng.normal(size=f.shape)
        fd = (L(f + 1e-4 * v) - L(f - 1e-4 * v)) / 2e-4
        assert abs((g * v).sum() - fd) <= 1e-6 * max(1.0, abs(fd))


# ------------------------------------------------ joint (cross) bilateral


def brute_joint(f, g, gs, sr, w):
    """Eq. (1) with the range kernel on the guide g, written out (4 loops)."""
    H, W = f.shape
    out = np.empty_like(f)
    for y in range(H):
        for x in range(W):
            num = den = 0.0
            for dy in range(-w, w + 1):
                for dx in range(-w, w + 1):
                    yy, xx = y - dy, x - dx
                    if 0 <= yy < H and 0 <= xx < W:
                        wgt = gs(dx, dy) * math.exp(-(g[yy, xx] - g[y, x]) ** 2 / (2 * sr * sr))
                        num += wgt * f[yy, xx]
                        den += wgt
            out[y, x] = num / den
    return out


def test_joint_direct_matches_brute_force():
    f = small_image(11, 9, 21, n_rect=4)
    g = small_image(11, 9, 22, n_rect=3)
    w = oracle.window(1.5)
    ref = brute_joint(f, g, lambda dx, dy: math.exp(-(dx * dx + dy * dy) / (2 * 1.5 * 1.5)), 30.0, w)
    np.testing.assert_allclose(oracle.direct_bf_joint(f, g, 1.5, 30.0), ref, rtol=0, atol=1e-11)


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_joint_with_guide_equal_to_data_is_the_bilateral_filter(sp):
    """g = f: the joint filter is the bilateral filter, directly and by Algorithm 1
    (the pinned single-image oracles)."""
    f = small_image(40, 36, 23)
    np.testing.assert_allclose(oracle.direct_bf_joint(f, f, 2.0, 30.0), oracle.direct_bf(f, 2.0, 30.0),
                               rtol=0, atol=1e-11)
    np.testing.assert_allclose(oracle.gp_bf_joint(f, f, 2.0, 30.0, 16, sp), oracle.gp_bf(f, 2.0, 30.0, 16, sp),
                               rtol=0, atol=1e-9)


@pytest.mark.parametrize("sr,N", [(30.0, 80), (50.0, 50)])
def test_joint_gp_converges_to_direct(sr, N):
    """Eq. (4)'s remainder at x = s^2 = (R / sigma_r)^2 (30 and 11 for this guide)
    is negligible at these orders: the decomposition reproduces Eq. (1)."""
    f = small_image(36, 30, 24, ramp=40.0)
    g = small_image(36, 30, 25)
    np.testing.assert_allclose(oracle.gp_bf_joint(f, g, 2.0, sr, N, "fir"), oracle.direct_bf_joint(f, g, 2.0, sr),
                               rtol=0, atol=1e-8)


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_joint_constant_guide_is_normalised_gaussian(sp):
    """A constant guide makes every range weight 1: the result is S(f) / S(1)
    (scipy's separable filter for the window sum)."""
    f = small_image(30, 34, 26)
    g = np.full_like(f, 91.0)
    out = oracle.gp_bf_joint(f, g, 2.0, 25.0, 10, sp)
    if sp == "fir":
        ref = gauss_filter_scipy(f, 2.0, 6) / gauss_filter_scipy(np.ones_like(f), 2.0, 6)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-10)
    np.testing.assert_allclose(out, oracle.gp_bf_joint(f, g, 2.0, float("inf"), 10, sp), rtol=0, atol=1e-10)


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_joint_is_linear_in_the_data(sp):
    """For a fixed guide the filter is linear in f (weights depend on g only)."""
    g = small_image(32, 28, 27)
    f1, f2 = small_image(32, 28, 28), small_image(32, 28, 29, ramp=30.0)
    a, b = 0.75, -1.5
    lhs = oracle.gp_bf_joint(a * f1 + b * f2, g, 2.5, 35.0, 14, sp)
    rhs = a * oracle.gp_bf_joint(f1, g, 2.5, 35.0, 14, sp) + b * oracle.gp_bf_joint(f2, g, 2.5, 35.0, 14, sp)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-9)


@pytest.mark.parametrize("sp", ["fir", "iir"])
def test_joint_guide_affine_equivariance(sp):
    """Scaling the guide by a and sigma_r by a, and shifting the guide, leaves the
    weights and hence the result unchanged (Eq. (3) depends on (t - tau) / sigma_r)."""
    f = small_image(30, 30, 30)
    g = small_image(30, 30, 31)
    np.testing.assert_allclose(oracle.gp_bf_joint(f, 2.0 * g + 17.0, 2.0, 60.0, 16, sp),
                               oracle.gp_bf_joint(f, g, 2.0, 30.0, 16, sp), rtol=0, atol=1e-9)


# ------------------------------------------------------------ box variant


@pytest.mark.parametrize("r,passes", [(1, 1), (4, 1), (2, 2), (3, 3), (4, 3)])
def test_box_line_operator_is_iterated_flat_kernel(r, passes):
    """The box variant's line operator: the passes-fold convolution of 2r + 1
    ones (numpy), applied with zero extension (scipy correlate1d)."""
    k = np.ones(2 * r + 1)
    for _ in range(passes - 1):
        k = np.convolve(k, np.ones(2 * r + 1))
    x = np.random.default_rng(5).normal(size=(3, 57))
    ref = correlate1d(x, k, axis=1, mode="constant")
    np.testing.assert_allclose(oracle.line_filter(x, 1.0, "box", box=(r, passes)), ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("r,passes", [(2, 1), (1, 3)])
def test_box_gp_converges_to_brute_force_with_box_weights(r, passes):
    """Algorithm 1 with S = the iterated box reproduces Eq. (1) with those spatial
    weights (brute force) once N is large."""
    f = small_image(12, 11, 32, n_rect=4)
    k = np.ones(2 * r + 1)
    for _ in range(passes - 1):
        k = np.convolve(k, np.ones(2 * r + 1))
    w = passes * r
    ref = brute_bf(f, lambda dx, dy: float(k[w + dx] * k[w + dy]), 40.0, w)
    np.testing.assert_allclose(oracle.gp_bf(f, 1.0, 40.0, 60, "box", box=(r, passes)), ref, rtol=0, atol=1e-9)


def test_box_sigma_r_infinite_is_normalised_box():
    f = small_image(30, 28, 33)
    k = np.convolve(np.ones(5), np.ones(5))
    ref = correlate1d(correlate1d(f - oracle.mean(f), k, axis=1, mode="constant"), k, axis=0, mode="constant")
    one = correlate1d(correlate1d(np.ones_like(f), k, axis=1, mode="constant"), k, axis=0, mode="constant")
    np.testing.assert_allclose(oracle.gp_bf(f, 1.0, float("inf"), 8, "box", box=(2, 2)), ref / one + oracle.mean(f),
                               rtol=0, atol=1e-10)
