"""GPU parity of the hand-written adjoint (bf_gp_backward) against the FP64
reverse-mode oracle O3 (oracle.gp_adjoint), which is itself pinned to central
differences of Algorithm 1.  Bar: max |dL/df_gpu - dL/df_oracle| <= 1e-3 of
max |dL/df_oracle|, and the same for dL/dsigma_r."""
import math

import numpy as np
import pytest

import oracle
import parity
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = 1e-3


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00077_gb300 as m
    m.build()
    return m


def gpu_fwd_bwd(bf, imgs, gys, ss, sr, N, spatial, t_c=None):
    """imgs, gys: [planes, H, W] float32.  Returns (y, grad_f, grad_sigma_r per plane, status)."""
    x = torch.from_numpy(np.ascontiguousarray(imgs, np.float32)).cuda()
    gy = torch.from_numpy(np.ascontiguousarray(gys, np.float32)).cuda()
    planes, H, W = x.shape
    o = bf.make_opts(N, spatial, t_c)
    need = bf.bf_gp_workspace_size(planes, H, W, ss, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    saved = torch.empty((planes, 4, H, W), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward_train(x.data_ptr(), y.data_ptr(), saved.data_ptr(), planes, H, W, W, ss, sr, o, ws.data_ptr(),
                           need, s)
    gx = torch.empty_like(x)
    gsr = torch.empty(planes, dtype=torch.float32, device="cuda")
    bf.bf_gp_backward(x.data_ptr(), gy.data_ptr(), saved.data_ptr(), gx.data_ptr(), gsr.data_ptr(), planes, H, W, W,
                      ss, sr, o, ws.data_ptr(), need, s)
    bits = bf.bf_gp_get_device_status(ws.data_ptr(), s)
    return y.cpu().numpy(), gx.cpu().numpy().astype(np.float64), gsr.cpu().numpy().astype(np.float64), bits


def check_grad(g_gpu, g_ref, what):
    scale = np.abs(g_ref).max()
    err = np.abs(g_gpu - g_ref).max()
    assert np.isfinite(g_gpu).all(), f"{what}: non-finite"
    assert err <= RTOL * scale, f"{what}: max err {err:.3e} vs scale {scale:.3e}"


@pytest.mark.parametrize("spatial,ss", [("fir", 2.0), ("fir", 3.5), ("iir", 3.0), ("iir", 9.0)])
@pytest.mark.parametrize("shape", [(37, 53), (130, 96), (600, 45)])
@pytest.mark.parametrize("t_c", [None, 120.0])
def test_backward_matches_oracle_adjoint(bf, spatial, ss, shape, t_c):
    H, W = shape
    img = synthetic.make_image(H, W, 8, 10.0, 0.0, synthetic.seed_for(5, H * 3 + W))
    gy = np.random.default_rng(H + W).normal(size=(H, W)).astype(np.float32)
    y, gx, gsr, bits = gpu_fwd_bwd(bf, img[None], gy[None], ss, 25.0, 20, spatial, t_c)
    assert bits == 0
    ref_g, ref_s = oracle.gp_adjoint(img.astype(np.float64), ss, 25.0, 20, gy.astype(np.float64), spatial, t_c=t_c)
    check_grad(gx[0], ref_g, "dL/df")
    assert abs(gsr[0] - ref_s) <= RTOL * max(abs(ref_s), 1e-6 * np.abs(ref_g).max() * H * W), (gsr[0], ref_s)


@pytest.mark.parametrize("H", [3000, 6000])
def test_backward_tall_columns(bf, H):
    """Columns of more than 4096 rows: the adjoint column pass in 16-CTA
    clusters (and one of up to 8 CTAs for comparison)."""
    W = 24
    img = synthetic.make_image(H, W, 8, 10.0, 0.0, synthetic.seed_for(5, 7000 + H))
    gy = np.random.default_rng(H).normal(size=(H, W)).astype(np.float32)
    y, gx, gsr, bits = gpu_fwd_bwd(bf, img[None], gy[None], 9.0, 40.0, 12, "iir")
    assert bits == 0
    ref_g, ref_s = oracle.gp_adjoint(img.astype(np.float64), 9.0, 40.0, 12, gy.astype(np.float64), "iir")
    check_grad(gx[0], ref_g, "dL/df")
    assert abs(gsr[0] - ref_s) <= RTOL * max(abs(ref_s), 1e-6 * np.abs(ref_g).max() * H * W), (gsr[0], ref_s)


def test_batch512_forward_backward(bf):
    """16 x 1 x 512^2, sigma_s 5, sigma_r 25, N 20 (recursive filter): every plane's
    forward against O2, and the adjoint of four of them against O3."""
    x = synthetic.batch512(16)[:, 0]
    rng = np.random.default_rng(55)
    gy = rng.normal(size=x.shape).astype(np.float32)
    y, gx, gsr, bits = gpu_fwd_bwd(bf, x, gy, 5.0, 25.0, 20, "iir")
    assert bits == 0
    for i in (0, 5, 10, 15):
        f = x[i].astype(np.float64)
        assert np.abs(y[i] - oracle.gp_bf(f, 5.0, 25.0, 20, "iir")).max() <= 1e-3
        ref_g, ref_s = oracle.gp_adjoint(f, 5.0, 25.0, 20, gy[i].astype(np.float64), "iir")
        check_grad(gx[i], ref_g, f"plane {i} dL/df")
        assert abs(gsr[i] - ref_s) <= RTOL * abs(ref_s)


def test_forward_train_equals_forward(bf):
    img = synthetic.make_image(200, 170, 8, 10.0, 0.0, 77)
    x = torch.from_numpy(img).cuda()
    y_plain = bf.bilateral_gp(x, 6.0, 30.0, 20, "iir")
    y, _, _, _ = gpu_fwd_bwd(bf, img[None], np.zeros_like(img)[None], 6.0, 30.0, 20, "iir")
    assert np.array_equal(y[0], y_plain.cpu().numpy())


def test_constant_plane_gradient(bf):
    """A constant image is filtered (not copied) when training; its derivative
    matches the oracle's."""
    img = np.full((40, 50), 90.5, np.float32)
    gy = np.random.default_rng(9).normal(size=img.shape).astype(np.float32)
    y, gx, gsr, _ = gpu_fwd_bwd(bf, img[None], gy[None], 2.0, 30.0, 20, "fir")
    assert np.all(y == 90.5)
    ref_g, _ = oracle.gp_adjoint(img.astype(np.float64), 2.0, 30.0, 20, gy.astype(np.float64), "fir")
    check_grad(gx[0], ref_g, "dL/df")


def test_sigma_r_infinite_has_no_sigma_r_gradient(bf):
    img = synthetic.make_image(64, 64, 6, 10.0, 0.0, 3)
    gy = np.ones_like(img)
    _, gx, gsr, _ = gpu_fwd_bwd(bf, img[None], gy[None], 2.0, math.inf, 20, "fir")
    assert gsr[0] == 0.0 and np.isfinite(gx).all()


def test_autograd_function(bf):
    img = synthetic.make_image(96, 80, 6, 10.0, 0.0, 12)
    x = torch.from_numpy(img).cuda().requires_grad_(True)
    sr = torch.tensor(25.0, device="cuda", requires_grad=True)
    y = bf.bilateral_gp_autograd(x, 4.0, sr, 20, "iir")
    w = torch.from_numpy(np.random.default_rng(2).normal(size=img.shape).astype(np.float32)).cuda()
    (y * w).sum().backward()
    ref_g, ref_s = oracle.gp_adjoint(img.astype(np.float64), 4.0, 25.0, 20, w.cpu().numpy().astype(np.float64), "iir")
    check_grad(x.grad.cpu().numpy().astype(np.float64), ref_g, "autograd dL/df")
    assert abs(float(sr.grad) - ref_s) <= RTOL * abs(ref_s)


def test_backward_where_the_denominator_is_not_positive(bf):
    """Odd N: the pixels whose Q <= 0 keep their value in the forward pass and pass
    dL/dy straight to their own input in the backward pass, as in O3."""
    img = np.zeros((40, 36), np.float32)
    img[:, 17] = 255.0
    img += synthetic.make_image(40, 36, 3, 3.0, 0.0, synthetic.seed_for(5, 7100)) * 0.05
    gy = np.random.default_rng(13).normal(size=img.shape).astype(np.float32)
    for spatial, ss in (("fir", 2.0), ("iir", 2.5)):
        y, gx, gsr, bits = gpu_fwd_bwd(bf, img[None], gy[None], ss, 20.0, 5, spatial)
        assert bits == 0  # the backward call's own status (the forward's flag is reset by it)
        _, kap = oracle.gp_bf(img.astype(np.float64), ss, 20.0, 5, spatial, return_kappa=True)
        assert parity.kept_value_pixels(y[0], img, kap) > 0
        ref_g, ref_s = oracle.gp_adjoint(img.astype(np.float64), ss, 20.0, 5, gy.astype(np.float64), spatial)
        check_grad(gx[0], ref_g, f"{spatial} dL/df")
        assert abs(gsr[0] - ref_s) <= RTOL * max(abs(ref_s), 1e-6 * np.abs(ref_g).max() * img.size), (gsr[0], ref_s)


# ------------------------------------------- finite differences at the 16 x 512^2 workload's settings

FD_STEP = 1e-2          # central differences of the FP64 forward (O2)
FD_SS, FD_SR, FD_N = 5.0, 25.0, 20
CROP = 32
HALO = 30               # 6 sigma_s: the recursive kernel is below 1e-4 of its peak there


def _fd_subproblem():
    """The 32 x 32 crop of image 0 (centre rows/columns 240..271) with a 30-pixel halo,
    as a standalone image, and the centre t_c of the full image (FP32 value), held fixed."""
    full = synthetic.batch512(1)[0, 0].astype(np.float64)
    r0 = c0 = 240 - HALO
    sub = full[r0:r0 + CROP + 2 * HALO, c0:c0 + CROP + 2 * HALO].copy()
    tc = float(np.float32(full.mean()))
    return sub, tc


def _fd_gradients(f, ybar, tc, pixels):
    """Central differences (step 1e-2) of L = sum(ybar * O2(f)) for every pixel in `pixels`,
    and for sigma_r; t_c is held at tc (None: the image mean, its derivative included)."""
    L = lambda ff, sr=FD_SR: float((ybar * oracle.gp_bf(ff, FD_SS, sr, FD_N, "iir", t_c=tc)).sum())
    g = np.zeros_like(f)
    for idx in pixels:
        e = np.zeros_like(f)
        e[idx] = FD_STEP
        g[idx] = (L(f + e) - L(f - e)) / (2 * FD_STEP)
    gs = (L(f, FD_SR + FD_STEP) - L(f, FD_SR - FD_STEP)) / (2 * FD_STEP)
    return g, gs, L


def test_finite_differences_on_a_32x32_crop(bf):
    """Every pixel of the 32 x 32 crop (2048 forward evaluations, t_c fixed) and 16
    random directions supported on the crop: central differences of O2 against O3 and
    against the GPU's bf_gp_backward on the same sub-problem (centre given)."""
    f, tc = _fd_subproblem()
    rng = np.random.default_rng(16)
    ybar = rng.normal(size=f.shape)
    crop = [(r, c) for r in range(HALO, HALO + CROP) for c in range(HALO, HALO + CROP)]
    fd, fds, L = _fd_gradients(f, ybar, tc, crop)
    o3, o3s = oracle.gp_adjoint(f, FD_SS, FD_SR, FD_N, ybar, "iir", t_c=tc)
    _, gx, gsr, bits = gpu_fwd_bwd(bf, f.astype(np.float32)[None], ybar.astype(np.float32)[None], FD_SS, FD_SR, FD_N,
                                   "iir", t_c=tc)
    assert bits == 0
    sl = np.s_[HALO:HALO + CROP, HALO:HALO + CROP]
    scale = np.abs(fd[sl]).max()
    # FP64 O3 against FP64 differences (truncation error of the 1e-2 step only)
    assert np.abs(o3[sl] - fd[sl]).max() <= 1e-5 * scale
    assert abs(o3s - fds) <= 1e-5 * abs(fds)
    # the GPU adjoint (FP32) against both
    assert np.abs(gx[0][sl] - fd[sl]).max() <= RTOL * scale
    assert np.abs(gx[0] - o3).max() <= RTOL * np.abs(o3).max()
    assert abs(gsr[0] - fds) <= RTOL * abs(fds)
    # directional derivatives along 16 random directions supported on the crop
    for _ in range(16):
        v = np.zeros_like(f)
        v[sl] = rng.normal(size=(CROP, CROP))
        dd = (L(f + FD_STEP * v) - L(f - FD_STEP * v)) / (2 * FD_STEP)
        assert abs((o3 * v).sum() - dd) <= 1e-5 * max(1.0, abs(dd))
        assert abs((gx[0] * v).sum() - dd) <= RTOL * np.abs(gx[0][sl] * v[sl]).sum()


def test_finite_differences_standalone_32x32_with_mean_centre(bf):
    """A standalone 32 x 32 image (the crop of image 0) with the mean centre of
    Algorithm 1's first step: the centring term of the derivative, every pixel, by
    central differences (step 1e-2) against O3 and the GPU."""
    f, _ = _fd_subproblem()
    f = f[HALO:HALO + CROP, HALO:HALO + CROP].copy()
    ybar = np.random.default_rng(17).normal(size=f.shape)
    fd, fds, _ = _fd_gradients(f, ybar, None, list(np.ndindex(f.shape)))
    o3, o3s = oracle.gp_adjoint(f, FD_SS, FD_SR, FD_N, ybar, "iir")
    _, gx, gsr, bits = gpu_fwd_bwd(bf, f.astype(np.float32)[None], ybar.astype(np.float32)[None], FD_SS, FD_SR, FD_N,
                                   "iir")
    assert bits == 0
    scale = np.abs(fd).max()
    assert np.abs(o3 - fd).max() <= 1e-5 * scale and abs(o3s - fds) <= 1e-5 * abs(fds)
    assert np.abs(gx[0] - fd).max() <= RTOL * scale
    assert abs(gsr[0] - fds) <= RTOL * abs(fds)
