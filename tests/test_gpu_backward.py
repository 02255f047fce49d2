"""GPU parity of the hand-written adjoint (bf_gp_backward) against the FP64
reverse-mode oracle O3 (oracle.gp_adjoint), which is itself pinned to central
differences of Algorithm 1.  Bar: max |dL/df_gpu - dL/df_oracle| <= 1e-3 of
max |dL/df_oracle|, and the same for dL/dsigma_r."""
import math

import numpy as np
import pytest

import oracle
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
