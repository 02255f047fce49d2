"""GPU parity of the joint (cross) bilateral filter (bf_gp_forward_joint): range
weights from a guide, data from a second image, 2 (N + 1) filterings, against
the FP64 oracle of the same decomposition (pinned in test_oracle_pins.py)."""
import numpy as np
import pytest

import oracle
import parity
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = parity.TOL


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00077_gb300 as m
    m.build()
    return m


def run_joint(bf, f, g, ss, sr, N, spatial):
    ft = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).cuda()
    gt = torch.from_numpy(np.ascontiguousarray(g, dtype=np.float32)).cuda()
    H, W = ft.shape[-2], ft.shape[-1]
    planes = max(1, ft.numel() // (H * W))
    o = bf.make_opts(N, spatial)
    need = bf.bf_gp_joint_workspace_size(planes, H, W, ss, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.full_like(ft, float("nan"))
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward_joint(ft.data_ptr(), gt.data_ptr(), y.data_ptr(), planes, H, W, W, ss, sr, o, ws.data_ptr(), need, s)
    bits = bf.bf_gp_get_device_status(ws.data_ptr(), s)
    tcs = [parity.gpu_centre(bf, ws.data_ptr(), c, s) for c in range(planes)]
    return y.cpu().numpy().astype(np.float64), bits, tcs


@pytest.mark.parametrize("shape,ss,sr,N,spatial", [
    ((96, 112), 2.0, 30.0, 20, "fir"), ((200, 333), 3.0, 40.0, 16, "fir"), ((1, 77), 1.0, 50.0, 10, "fir"),
    ((300, 260), 6.0, 30.0, 20, "iir"), ((1030, 64), 12.0, 45.0, 14, "iir"), ((64, 700), 9.0, 60.0, 31, "iir"),
])
def test_joint_matches_oracle(bf, shape, ss, sr, N, spatial):
    H, W = shape
    f = synthetic.make_image(H, W, 6, 10.0, 30.0, synthetic.seed_for(10, H * 7 + W))
    g = synthetic.make_image(H, W, 5, 8.0, 0.0, synthetic.seed_for(10, H * 11 + W))
    out, bits, tcs = run_joint(bf, f, g, ss, sr, N, spatial)
    assert (bits & ~bf.BF_DEV_NONPOS_Q) == 0
    ref, kap = oracle.gp_bf_joint(f.astype(np.float64), g.astype(np.float64), ss, sr, N, spatial, t_c=tcs[0],
                                  return_kappa=True)
    even_fir = spatial == "fir" and N % 2 == 0
    parity.gate(out, ref, kap, min_gated=0.99, f=f if even_fir else None, window=oracle.window(ss) if even_fir else None,
                label=f"joint {shape} {spatial} ss={ss:g} sr={sr:g} N={N}")
    assert parity.kept_value_pixels(out, f, kap) == 0 or bits & bf.BF_DEV_NONPOS_Q


def test_joint_with_guide_equal_to_data_is_the_single_image_filter(bf):
    img = synthetic.make_image(150, 170, 6, 10.0, 20.0, synthetic.seed_for(10, 9))
    out, bits, _ = run_joint(bf, img, img, 5.0, 30.0, 20, "iir")
    assert bits == 0
    x = torch.from_numpy(img).cuda()
    single = bf.bilateral_gp(x, 5.0, 30.0, 20, "iir").cpu().numpy().astype(np.float64)
    assert np.abs(out - single).max() <= 2e-3


def test_joint_constant_guide_and_nonfinite_guide(bf):
    f = synthetic.make_image(80, 90, 6, 10.0, 0.0, synthetic.seed_for(10, 10))
    g = np.full_like(f, 42.0)
    out, bits, tcs = run_joint(bf, f, g, 3.0, 30.0, 12, "fir")
    assert bits == 0
    ref = oracle.gp_bf_joint(f.astype(np.float64), g.astype(np.float64), 3.0, 30.0, 12, "fir", t_c=tcs[0])
    parity.gate(out, ref, label="joint constant guide")
    g2 = synthetic.make_image(80, 90, 6, 10.0, 0.0, synthetic.seed_for(10, 11))
    g2[5, 5] = np.inf
    out2, bits2, _ = run_joint(bf, f, g2, 3.0, 30.0, 12, "fir")
    assert bits2 & bf.BF_DEV_NONFINITE_IN
    assert np.array_equal(out2, f.astype(np.float64))


def test_joint_batch_of_planes_and_convenience_call(bf):
    f = synthetic.make_image(70, 66, 6, 10.0, 10.0, synthetic.seed_for(10, 12), planes=3)
    g = synthetic.make_image(70, 66, 4, 10.0, 0.0, synthetic.seed_for(10, 13), planes=3)
    y = bf.bilateral_gp_joint(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), 4.0, 35.0, 18, "iir")
    y = y.cpu().numpy().astype(np.float64)
    _, _, tcs = run_joint(bf, f, g, 4.0, 35.0, 18, "iir")
    for c in range(3):
        ref, kap = oracle.gp_bf_joint(f[c].astype(np.float64), g[c].astype(np.float64), 4.0, 35.0, 18, "iir",
                                      t_c=tcs[c], return_kappa=True)
        parity.gate(y[c], ref, kap, min_gated=0.99, label=f"joint plane {c}")


def test_joint_order_limit(bf):
    o = bf.make_opts(32, "iir")
    with pytest.raises(bf.BFError):
        bf.bf_gp_joint_workspace_size(1, 64, 64, 3.0, o)
