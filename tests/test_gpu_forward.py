"""GPU parity of the forward filter against the FP64 oracle (Algorithm 1).

Every case runs the CUDA path through the C ABI (bf_gp_forward) and compares
element by element with oracle.gp_bf on the same seeded image, with the same
spatial operator and the centre the GPU used.  Bar (tests/parity.py): max
|GPU - oracle| <= 1e-3 on the 0..255 scale on every pixel the FP32 arithmetic
resolves; every other pixel finite and, for an even order with the window
sum, inside its window's range; where Q <= 0 both keep the pixel's value.
"""
import math

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


def run_gpu(bf, img, ss, sr, N, spatial, status=False, **kw):
    """GPU result (FP64 copy), and with status=True also (status bits, counters, centre used)."""
    x = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()
    H, W = x.shape[-2], x.shape[-1]
    planes = max(1, x.numel() // (H * W))
    o = bf.make_opts(N, spatial, kw.get("t_c"), kw.get("fir_halfwidth", 0))
    need = bf.bf_gp_workspace_size(planes, H, W, ss, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = bf.bilateral_gp(x, ss, sr, N, spatial, ws=ws, **kw)
    s = torch.cuda.current_stream().cuda_stream
    bits = bf.bf_gp_get_device_status(ws.data_ptr(), s)
    out = y.cpu().numpy().astype(np.float64)
    if not status:
        return out
    return out, bits, bf.bf_gp_get_device_counters(ws.data_ptr(), s), parity.gpu_centre(bf, ws.data_ptr(), 0, s)


def compare(bf, img, ss, sr, N, spatial, min_gated=1.0, label="", **kw):
    """GPU vs oracle (with kappa) on the whole image, at the GPU's centre."""
    out, bits, counters, tc = run_gpu(bf, img, ss, sr, N, spatial, status=True, **kw)
    f64 = np.asarray(img, np.float64)
    ref, kap = oracle.gp_bf(f64, ss, sr, N, spatial, t_c=kw.get("t_c", tc), return_kappa=True)
    even_fir = spatial == "fir" and N % 2 == 0
    rec = parity.gate(out, ref, kap, min_gated=min_gated, f=f64 if even_fir else None,
                      window=oracle.window(ss) if even_fir else None, label=label or f"{f64.shape} {spatial} "
                      f"ss={ss:g} sr={sr:g} N={N}")
    n_q0 = parity.kept_value_pixels(out, f64, kap)
    assert counters[0] == n_q0 and bool(bits & bf.BF_DEV_NONPOS_Q) == (n_q0 > 0)
    assert (bits & ~bf.BF_DEV_NONPOS_Q) == 0
    return rec


# ---------------------------------------------------------------- 256^2 rectangles, sigma_s 3, sigma_r 30

@pytest.mark.parametrize("N", [20, 34, 38])
def test_rects256_fir(bf, N):
    """The paper's setting (N = 20), the order the kernel-error rule gives for sigma_r 30
    over this image's range (N = 38, bf_gp_order_for_tol at 1e-3), and one between."""
    compare(bf, synthetic.rects256_image(), 3.0, 30.0, N, "fir")


def test_rects256_order_from_the_error_rule_is_38(bf):
    img = synthetic.rects256_image().astype(np.float64)
    R = float(np.max(np.abs(img - img.mean())))
    assert bf.bf_gp_order_for_tol(30.0, R, 1e-3) == 38


def test_rects256_iir(bf):
    compare(bf, synthetic.rects256_image(), 3.0, 30.0, 20, "iir", min_gated=0.999)


# ---------------------------------------------------------------- ragged shapes

SHAPES = [(1, 1), (1, 7), (5, 1), (2, 3), (17, 33), (31, 64), (65, 129), (300, 260), (517, 37), (1030, 75),
          (37, 1500), (1600, 200)]


@pytest.mark.parametrize("spatial,ss", [("fir", 1.5), ("fir", 4.0), ("iir", 2.5), ("iir", 9.0)])
@pytest.mark.parametrize("shape", SHAPES)
def test_ragged_shapes(bf, shape, spatial, ss):
    H, W = shape
    img = synthetic.make_image(H, W, 6, 10.0, 0.0, synthetic.seed_for(9, H * 7 + W))
    # floors: the oracle's own resolvable fraction on these inputs (>= 0.91; >= 0.6 below 10 pixels)
    compare(bf, img, ss, 30.0, 12, spatial, min_gated=0.5 if H * W < 10 else 0.9)


@pytest.mark.parametrize("H", [511, 512, 513, 1024, 2047, 2049, 3000, 4096, 4097, 6000, 8192])
def test_iir_column_cluster_sizes(bf, H):
    """Columns spanning 1..16 CTAs of the clustered column pass (more than 8:
    the non-portable cluster size)."""
    img = synthetic.make_image(H, 24, 8, 10.0, 30.0, synthetic.seed_for(9, H))
    compare(bf, img, 7.0, 40.0, 10, "iir", min_gated=0.8)  # the oracle's fraction here: >= 0.84


@pytest.mark.parametrize("engine", [0, 1])
@pytest.mark.parametrize("H", [4600, 8192])
def test_iir_tall_columns_engines_and_training(bf, H, engine):
    """Columns of more than 4096 rows on both CUDA-core column engines, and the
    forward that saves the sums for the backward pass (its column pass holds
    the most shared memory per CTA)."""
    W = 40
    img = synthetic.make_image(H, W, 8, 10.0, 30.0, synthetic.seed_for(9, H + engine))
    o = bf.make_opts(10, "iir", engine=engine)
    x = torch.from_numpy(img).cuda()
    need = bf.bf_gp_workspace_size(1, H, W, 9.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    y = torch.full_like(x, float("nan"))
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, 9.0, 40.0, o, ws.data_ptr(), need, s)
    assert bf.bf_gp_get_device_status(ws.data_ptr(), s) == 0
    tc = parity.gpu_centre(bf, ws.data_ptr(), 0, s)
    ref, kap = oracle.gp_bf(img.astype(np.float64), 9.0, 40.0, 10, "iir", t_c=tc, return_kappa=True)
    parity.gate(y.cpu().numpy(), ref, kap, min_gated=0.9, label=f"tall {H} engine {engine}")  # oracle: >= 0.92
    saved = torch.empty((1, 4, H, W), dtype=torch.float32, device="cuda")
    y2 = torch.full_like(x, float("nan"))
    bf.bf_gp_forward_train(x.data_ptr(), y2.data_ptr(), saved.data_ptr(), 1, H, W, W, 9.0, 40.0, o, ws.data_ptr(),
                           need, s)
    parity.gate(y2.cpu().numpy(), ref, kap, min_gated=0.9, label=f"tall {H} engine {engine} training")


@pytest.mark.parametrize("W", [511, 512, 513, 1024, 4095, 4096, 4097, 8192])
def test_iir_long_rows(bf, W):
    img = synthetic.make_image(12, W, 8, 10.0, 30.0, synthetic.seed_for(9, W))
    compare(bf, img, 11.0, 40.0, 10, "iir", min_gated=0.75)  # the oracle's fraction here: >= 0.79


# ---------------------------------------------------------------- 1024^2 rectangles + ramp: the full sweep

# sigma_s in {2, 5, 10, 20} x sigma_r in {10, 30, 50} x every even order 4..20, on the full
# 1024^2 image: the recursive filter for every sigma_s, the window sum also for sigma_s = 2.
# The oracle computes every order of one (sigma_s, sigma_r, operator) in one pass.
SWEEP_ORDERS = list(range(4, 21, 2))
SWEEP = [(ss, sr, "iir") for ss in (2.0, 5.0, 10.0, 20.0) for sr in (10.0, 30.0, 50.0)] + \
        [(2.0, sr, "fir") for sr in (10.0, 30.0, 50.0)]
# the smallest resolvable fraction kappa gives on this image (sigma_r = 10: (R / sigma_r)^2 = 234)
SWEEP_MIN_GATED = {10.0: 0.92, 30.0: 0.996, 50.0: 0.999}
_sweep_cache = {}


def _sweep_oracle(img, ss, sr, spatial, tc):
    key = (ss, sr, spatial, tc)
    if key not in _sweep_cache:
        _sweep_cache.clear()
        _sweep_cache[key] = oracle.gp_bf(img.astype(np.float64), ss, sr, SWEEP_ORDERS, spatial, t_c=tc,
                                         return_kappa=True)
    return _sweep_cache[key]


@pytest.mark.parametrize("N", SWEEP_ORDERS)
@pytest.mark.parametrize("ss,sr,spatial", SWEEP)
def test_rects_ramp1024_sweep(bf, ss, sr, spatial, N):
    img = synthetic.rects_ramp1024_image()
    out, bits, counters, tc = run_gpu(bf, img, ss, sr, N, spatial, status=True)
    refs, kaps = _sweep_oracle(img, ss, sr, spatial, tc)
    q = SWEEP_ORDERS.index(N)
    f64 = img.astype(np.float64)
    fir = spatial == "fir"
    parity.gate(out, refs[q], kaps[q], min_gated=SWEEP_MIN_GATED[sr], f=f64 if fir else None,
                window=oracle.window(ss) if fir else None, label=f"1024^2 {spatial} ss={ss:g} sr={sr:g} N={N}")
    n_q0 = parity.kept_value_pixels(out, f64, kaps[q])
    assert counters[0] == n_q0 and bool(bits & bf.BF_DEV_NONPOS_Q) == (n_q0 > 0)
    assert (bits & ~bf.BF_DEV_NONPOS_Q) == 0


def test_large_s2_stays_in_fp32_range(bf):
    """(R / sigma_r)^2 = 234 on the 1024^2 image (R = 153, sigma_r = 10): exp(-s^2 u^2 / 2)
    would underflow FP32 at |u| = 1 without the common power-of-two channel scale."""
    compare(bf, synthetic.rects_ramp1024_image(), 2.0, 10.0, 20, "fir", min_gated=0.999)


def test_range_flag_beyond_fp32(bf):
    img = np.zeros((64, 64), np.float32)
    img[:, 32:] = 255.0
    _, bits, _, _ = run_gpu(bf, img, 3.0, 3.0, 20, "fir", status=True)  # s^2 = (127.5 / 3)^2 = 1806
    assert bits & bf.BF_DEV_RANGE
    # two planes beyond the range, one inside it: the counter counts planes
    x = torch.from_numpy(np.stack([img, img, np.full_like(img, 7.0)])).cuda()
    o = bf.make_opts(20, "fir")
    need = bf.bf_gp_workspace_size(3, 64, 64, 3.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 3, 64, 64, 64, 3.0, 3.0, o, ws.data_ptr(), need, s)
    assert bf.bf_gp_get_device_counters(ws.data_ptr(), s)[2] == 2


# ---------------------------------------------------------------- 4096^2 rectangles, sigma_s 10, sigma_r 20

def test_rects4096_crop(bf):
    """4096^2, sigma_s 10, sigma_r 20, N 20, recursive filter: a 512^2 crop of the
    GPU output against the oracle run on full lines of the full image, and a
    border crop (the zero extension at the image edge)."""
    img = synthetic.rects4096_image()
    f64 = img.astype(np.float64)
    gpu, bits, _, tc = run_gpu(bf, img, 10.0, 20.0, 20, "iir", status=True)
    assert bits == 0
    for r0, r1, c0, c1 in ((1792, 2304, 2304, 2816), (4096 - 64, 4096, 0, 64)):
        ref, kap = oracle.gp_bf(f64, 10.0, 20.0, 20, "iir", t_c=tc, crop=(r0, r1, c0, c1), return_kappa=True)
        parity.gate(gpu[r0:r1, c0:c1], ref, kap, min_gated=0.99, label=f"4096^2 crop {r0}:{r1},{c0}:{c1}")


# ---------------------------------------------------------------- special cases

def test_constant_image_exact(bf):
    img = np.full((70, 90), 123.5, np.float32)
    for sp in ("fir", "iir"):
        assert np.all(run_gpu(bf, img, 3.0, 30.0, 20, sp) == 123.5)


def test_sigma_r_infinite(bf):
    img = synthetic.make_image(96, 80, 6, 10.0, 0.0, synthetic.seed_for(9, 1))
    for sp, ss in (("fir", 2.0), ("iir", 6.0)):
        compare(bf, img, ss, math.inf, 20, sp)


def test_given_centre(bf):
    img = synthetic.make_image(64, 64, 6, 10.0, 0.0, synthetic.seed_for(9, 2))
    compare(bf, img, 2.0, 30.0, 20, "fir", t_c=127.5)


def test_multi_plane_independent_centres(bf):
    imgs = np.stack([synthetic.make_image(50, 70, 5, 10.0, 0.0, synthetic.seed_for(9, 10 + i)) for i in range(3)])
    imgs[1] *= 0.3
    x = torch.from_numpy(imgs).cuda()
    o = bf.make_opts(20, "fir")
    need = bf.bf_gp_workspace_size(3, 50, 70, 2.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 3, 50, 70, 70, 2.0, 25.0, o, ws.data_ptr(), need, s)
    gpu = y.cpu().numpy()
    for i in range(3):
        tc = parity.gpu_centre(bf, ws.data_ptr(), i, s)
        assert abs(tc - imgs[i].astype(np.float64).mean()) < 1e-3  # each plane its own mean
        ref, kap = oracle.gp_bf(imgs[i].astype(np.float64), 2.0, 25.0, 20, "fir", t_c=tc, return_kappa=True)
        parity.gate(gpu[i], ref, kap, f=imgs[i], window=oracle.window(2.0), label=f"plane {i}")


def test_pitched_input(bf):
    img = synthetic.make_image(40, 50, 5, 10.0, 0.0, synthetic.seed_for(9, 3))
    big = np.zeros((40, 53), np.float32)
    big[:, :50] = img
    x = torch.from_numpy(big).cuda()
    y = torch.full_like(x, -7.0)
    o = bf.make_opts(20, "fir")
    need = bf.bf_gp_workspace_size(1, 40, 50, 2.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, 40, 50, 53, 2.0, 30.0, o, ws.data_ptr(), need, s)
    tc = parity.gpu_centre(bf, ws.data_ptr(), 0, s)
    out = y.cpu().numpy()
    ref, kap = oracle.gp_bf(img.astype(np.float64), 2.0, 30.0, 20, "fir", t_c=tc, return_kappa=True)
    parity.gate(out[:, :50], ref, kap, f=img, window=oracle.window(2.0), label="pitched")
    assert np.all(out[:, 50:] == -7.0)  # padding untouched


def test_device_stats_readback(bf):
    img = synthetic.make_image(123, 77, 5, 10.0, 0.0, synthetic.seed_for(9, 4))
    x = torch.from_numpy(img).cuda()
    o = bf.make_opts(20, "fir")
    need = bf.bf_gp_workspace_size(1, 123, 77, 2.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, 123, 77, 77, 2.0, 30.0, o, ws.data_ptr(), need, s)
    tc, R = bf.bf_gp_get_plane_stats(ws.data_ptr(), 0, s)
    f64 = img.astype(np.float64)
    assert abs(tc - f64.mean()) <= 1e-9 * 255
    assert R == max(f64.max() - tc, tc - f64.min())
    assert bf.bf_gp_get_device_status(ws.data_ptr(), s) == 0


@pytest.mark.parametrize("spatial,two_pass", [("fir", False), ("fir", True), ("iir", False)])
def test_odd_order_flags_and_counts_nonpositive_denominator(bf, spatial, two_pass):
    """Odd N: pixels with Q <= 0 keep their own value (Eq. (11) is undefined
    there), the flag is raised and the counter holds exactly the number of
    such pixels (fused FIR kernel, FIR column pass, recursive column pass)."""
    img = np.zeros((16, 16), np.float32)
    img[:, 8] = 255.0
    x = torch.from_numpy(img).cuda()
    o = bf.make_opts(5, spatial, fir_two_pass=two_pass)
    need = bf.bf_gp_workspace_size(1, 16, 16, 3.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.full_like(x, float("nan"))
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, 16, 16, 16, 3.0, 20.0, o, ws.data_ptr(), need, s)
    bits = bf.bf_gp_get_device_status(ws.data_ptr(), s)
    counters = bf.bf_gp_get_device_counters(ws.data_ptr(), s)
    out = y.cpu().numpy()
    assert np.isfinite(out).all()
    assert counters[0] > 0 and bits & bf.BF_DEV_NONPOS_Q and counters[1:] == [0, 0, 0]
    assert np.all(out[:, 8] == 255.0)  # the line's pixels (Q <= 0) keep their value
    tc = parity.gpu_centre(bf, ws.data_ptr(), 0, s)
    ref, kap = oracle.gp_bf(img.astype(np.float64), 3.0, 20.0, 5, spatial, t_c=tc, return_kappa=True)
    assert parity.kept_value_pixels(out, img, kap) == counters[0]
    parity.gate(out, ref, kap, min_gated=0.5, label=f"odd N {spatial} two_pass={two_pass}")


def test_tcgen05_wait_gives_up_cleanly(bf):
    """The tcgen05 column pass told to issue no tensor-core product and to give up
    each wait for one after 2000 polls: nothing is in flight when it gives up, so it
    frees its tensor memory and returns; the call reports BF_DEV_TIMEOUT with one
    count per CTA, writes the plane as copied, and the context stays usable."""
    H, W, ss = 1030, 64, 6.0
    img = synthetic.make_image(H, W, 8, 10.0, 0.0, synthetic.seed_for(9, 9100))
    x = torch.from_numpy(img).cuda()
    s = torch.cuda.current_stream().cuda_stream
    o = bf.make_opts(20, "iir", engine=3, tc5_wait_test=2000)
    need = bf.bf_gp_workspace_size(1, H, W, ss, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.full_like(x, float("nan"))
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, 30.0, o, ws.data_ptr(), need, s)
    bits = bf.bf_gp_get_device_status(ws.data_ptr(), s)
    counters = bf.bf_gp_get_device_counters(ws.data_ptr(), s)
    assert bits & bf.BF_DEV_TIMEOUT and (bits & ~bf.BF_DEV_TIMEOUT) == 0
    ctas = (W // 8) * ((H + 511) // 512)
    assert counters == [0, 0, 0, ctas]
    assert np.array_equal(y.cpu().numpy(), img)
    # the same context, the normal engine-3 call: no timeout, the oracle's result
    compare(bf, img, ss, 30.0, 20, "iir", min_gated=0.95, label="engine 3 after a timed-out call")
    o3 = bf.make_opts(20, "iir", engine=3)
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, 30.0, o3, ws.data_ptr(), need, s)
    assert bf.bf_gp_get_device_status(ws.data_ptr(), s) == 0


def test_nonfinite_input_is_passed_through_and_flagged(bf):
    img = synthetic.make_image(20, 20, 3, 10.0, 0.0, 5)
    img[3, 4] = np.nan
    x = torch.from_numpy(img).cuda()
    o = bf.make_opts(20, "fir")
    need = bf.bf_gp_workspace_size(1, 20, 20, 3.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, 20, 20, 20, 3.0, 30.0, o, ws.data_ptr(), need, s)
    assert bf.bf_gp_get_device_status(ws.data_ptr(), s) & bf.BF_DEV_NONFINITE_IN
    assert bf.bf_gp_get_device_counters(ws.data_ptr(), s) == [0, 1, 0, 0]
    out = y.cpu().numpy()
    assert np.array_equal(out, img, equal_nan=True)
    # the next call on the same workspace starts from zero counts
    x.copy_(torch.from_numpy(synthetic.make_image(20, 20, 3, 10.0, 0.0, 5)))
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, 20, 20, 20, 3.0, 30.0, o, ws.data_ptr(), need, s)
    assert bf.bf_gp_get_device_status(ws.data_ptr(), s) == 0
    assert bf.bf_gp_get_device_counters(ws.data_ptr(), s) == [0, 0, 0, 0]


@pytest.mark.parametrize("inp", ["pinned", "pageable"])
@pytest.mark.parametrize("out", ["pinned", "pinned_view", "pageable"])
@pytest.mark.parametrize("spatial", ["iir", "fir"])
def test_host_entry_point_matches_device_entry_point(bf, inp, out, spatial):
    """Host buffers give the device path's bytes. A mapped pinned input is
    read by the statistics pass itself; a mapped pinned result buffer is
    written by the last pass directly; a view inside a larger pinned buffer
    takes the same route; pageable memory takes the staged copies."""
    H, W = 200, 180
    img = synthetic.make_image(H, W, 8, 10.0, 0.0, synthetic.seed_for(9, 6))
    ss = 6.0 if spatial == "iir" else 3.0
    o = bf.make_opts(20, spatial)
    need = bf.bf_gp_host_workspace_size(1, H, W, ss, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    fh = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32))
    if inp == "pinned":
        fh = fh.pin_memory()
    if out == "pinned":
        yh = torch.empty_like(fh).pin_memory()
        keep = yh
    elif out == "pinned_view":
        keep = torch.full((H * W + 96,), -7.0, dtype=torch.float32).pin_memory()
        yh = keep[32:32 + H * W].view(H, W)
    else:
        keep = np.full((H, W), -7.0, dtype=np.float32)
        yh = torch.from_numpy(keep)
    bf.bf_gp_forward_host(fh.data_ptr(), yh.data_ptr(), 1, H, W, ss, 30.0, o, ws.data_ptr(), need,
                          torch.cuda.current_stream().cuda_stream)
    dev = run_gpu(bf, img, ss, 30.0, 20, spatial)
    assert np.array_equal(yh.numpy().astype(np.float64), dev)
    if out == "pinned_view":
        # nothing outside the view is written
        assert torch.all(keep[:32] == -7.0) and torch.all(keep[32 + H * W:] == -7.0)


def test_host_entry_point_nonfinite_input(bf):
    """A NaN in a mapped pinned input reaches the device copy the statistics
    pass writes: the plane is flagged and passed through unchanged."""
    H, W = 64, 72
    img = synthetic.make_image(H, W, 8, 10.0, 0.0, synthetic.seed_for(9, 8)).astype(np.float32)
    img[5, 7] = np.nan
    o = bf.make_opts(20, "iir")
    need = bf.bf_gp_host_workspace_size(1, H, W, 4.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    fh = torch.from_numpy(img).pin_memory()
    yh = torch.empty_like(fh).pin_memory()
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward_host(fh.data_ptr(), yh.data_ptr(), 1, H, W, 4.0, 30.0, o, ws.data_ptr(), need, s)
    assert bf.bf_gp_get_device_status(ws.data_ptr(), s) & bf.BF_DEV_NONFINITE_IN
    assert np.array_equal(yh.numpy(), img, equal_nan=True)


def test_repeat_calls_are_deterministic(bf):
    img = synthetic.make_image(300, 300, 8, 10.0, 0.0, synthetic.seed_for(9, 7))
    a = run_gpu(bf, img, 8.0, 30.0, 20, "iir")
    b = run_gpu(bf, img, 8.0, 30.0, 20, "iir")
    assert np.array_equal(a, b)


@pytest.mark.parametrize("engine", [0, 1, 2, 3])
@pytest.mark.parametrize("shape,ss", [((300, 260), 6.0), ((1030, 600), 12.0), ((2049, 75), 20.0)])
def test_engines_agree_with_oracle(bf, engine, shape, ss):
    """Recursive filter on tensor cores (rows and/or columns) and on CUDA cores."""
    H, W = shape
    img = synthetic.make_image(H, W, 8, 10.0, 20.0, synthetic.seed_for(9, 5000 + H + W))
    x = torch.from_numpy(img).cuda()
    o = bf.make_opts(20, "iir", engine=engine)
    need = bf.bf_gp_workspace_size(1, H, W, ss, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, 30.0, o, ws.data_ptr(), need, s)
    assert bf.bf_gp_get_device_status(ws.data_ptr(), s) == 0
    tc = parity.gpu_centre(bf, ws.data_ptr(), 0, s)
    ref, kap = oracle.gp_bf(img.astype(np.float64), ss, 30.0, 20, "iir", t_c=tc, return_kappa=True)
    parity.gate(y.cpu().numpy(), ref, kap, min_gated=0.9, label=f"engine {engine} {shape} ss={ss:g}")


# ---------------------------------------------------------------- fused FIR forward

def _forward(bf, img, ss, sr, N, two_pass, centre=False, fir_tile=0):
    x = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).cuda()
    H, W = x.shape
    o = bf.make_opts(N, "fir", fir_two_pass=two_pass, fir_tile=fir_tile)
    need = bf.bf_gp_workspace_size(1, H, W, ss, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.full_like(x, float("nan"))
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, o, ws.data_ptr(), need, s)
    out = (y.cpu().numpy().astype(np.float64), bf.bf_gp_get_device_status(ws.data_ptr(), s))
    return out + (parity.gpu_centre(bf, ws.data_ptr(), 0, s),) if centre else out


@pytest.mark.parametrize("shape,ss", [((1, 1), 1.0), ((7, 300), 0.4), ((33, 65), 2.0), ((256, 256), 3.0),
                                      ((100, 1030), 3.7), ((300, 47), 4.0)])
def test_fir_fused_matches_two_pass_and_oracle(bf, shape, ss):
    """One fused kernel per 32 x 32 tile (channels, both filters and the combine in
    shared memory) against the two-pass form and the oracle: tiles straddling
    every image edge, windows from W = 2 to 12."""
    H, W = shape
    img = synthetic.make_image(H, W, 6, 10.0, 20.0, synthetic.seed_for(9, 7000 + H + W))
    fused, b1, tc = _forward(bf, img, ss, 30.0, 20, False, centre=True)
    two, b2 = _forward(bf, img, ss, 30.0, 20, True)
    assert b1 == 0 and b2 == 0
    assert np.abs(fused - two).max() <= 2e-4
    ref, kap = oracle.gp_bf(img.astype(np.float64), ss, 30.0, 20, "fir", t_c=tc, return_kappa=True)
    parity.gate(fused, ref, kap, min_gated=0.999, f=img, window=oracle.window(ss), label=f"fused {shape} ss={ss:g}")
    parity.gate(two, ref, kap, min_gated=0.999, f=img, window=oracle.window(ss), label=f"two-pass {shape} ss={ss:g}")


@pytest.mark.parametrize("shape,ss", [((1, 1), 1.0), ((7, 300), 0.4), ((33, 65), 2.0), ((70, 45), 4.0),
                                      ((100, 1030), 3.7), ((129, 47), 3.2)])
def test_fir_fused_tile_heights(bf, shape, ss):
    """The fused kernel with 16- and 64-row output tiles (the autotuner's other
    tile shapes) gives the 32-row result bit for bit: every output is the same
    window sums of the same channel values; only which CTA forms it changes.
    Windows up to W = 12 make the 64-row tile's halo 88 rows (two row-filter
    items per thread)."""
    H, W = shape
    img = synthetic.make_image(H, W, 6, 10.0, 20.0, synthetic.seed_for(9, 7100 + H + W))
    base, b0, tc = _forward(bf, img, ss, 30.0, 20, False, centre=True)
    assert b0 == 0
    for th in (16, 64):
        out, b = _forward(bf, img, ss, 30.0, 20, False, fir_tile=th)
        assert b == 0
        assert np.array_equal(out, base), th
    ref, kap = oracle.gp_bf(img.astype(np.float64), ss, 30.0, 20, "fir", t_c=tc, return_kappa=True)
    parity.gate(out, ref, kap, min_gated=0.999, f=img, window=oracle.window(ss), label=f"fused 64-row tiles {shape} ss={ss:g}")


def test_fir_fused_copy_planes(bf):
    """Constant plane -> itself; non-finite input -> passed through and flagged."""
    img = np.full((40, 50), 77.25, np.float32)
    out, bits = _forward(bf, img, 2.0, 30.0, 20, False)
    assert bits == 0 and np.array_equal(out, img.astype(np.float64))
    img2 = synthetic.make_image(40, 50, 4, 10.0, 0.0, synthetic.seed_for(9, 7100))
    img2[3, 4] = np.nan
    out2, bits2 = _forward(bf, img2, 2.0, 30.0, 20, False)
    assert bits2 & bf.BF_DEV_NONFINITE_IN
    assert np.array_equal(np.isnan(out2), np.isnan(img2)) and np.array_equal(out2[~np.isnan(out2)], img2[~np.isnan(img2)].astype(np.float64))


# ---------------------------------------------------------------- box variant

@pytest.mark.parametrize("shape,r,passes", [((96, 100), 1, 1), ((130, 70), 12, 1), ((64, 256), 3, 2), ((257, 33), 6, 2),
                                            ((200, 190), 2, 3), ((45, 300), 4, 3)])
def test_box_variant_matches_oracle(bf, shape, r, passes):
    """S = passes-fold iterated box of half-width r by running sums in the fused
    tile kernel, against Algorithm 1 with that operator (oracle, explicit taps)."""
    H, W = shape
    img = synthetic.make_image(H, W, 6, 10.0, 15.0, synthetic.seed_for(9, 8000 + 7 * r + passes))
    x = torch.from_numpy(img).cuda()
    o = bf.make_opts(20, "box", fir_halfwidth=r, box_passes=passes)
    need = bf.bf_gp_workspace_size(1, H, W, 1.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.full_like(x, float("nan"))
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, 1.0, 30.0, o, ws.data_ptr(), need, s)
    assert bf.bf_gp_get_device_status(ws.data_ptr(), s) == 0
    tc = parity.gpu_centre(bf, ws.data_ptr(), 0, s)
    ref, kap = oracle.gp_bf(img.astype(np.float64), 1.0, 30.0, 20, "box", box=(r, passes), t_c=tc,
                            return_kappa=True)
    parity.gate(y.cpu().numpy(), ref, kap, min_gated=0.999, f=img, window=r * passes,
                label=f"box {shape} r={r} passes={passes}")


def test_box_variant_radius_from_sigma_and_limits(bf):
    """Without a radius the box is matched to sigma_s (passes ((2r+1)^2 - 1) / 12
    closest to sigma_s^2); wider windows than 12 and the two-pass form are refused."""
    img = synthetic.make_image(120, 140, 6, 10.0, 0.0, synthetic.seed_for(9, 8100))
    x = torch.from_numpy(img).cuda()
    o0 = bf.make_opts(20, "box")
    need0 = bf.bf_gp_workspace_size(1, 120, 140, 3.0, o0)
    ws0 = torch.empty(need0, dtype=torch.uint8, device="cuda")
    y = bf.bilateral_gp(x, 3.0, 30.0, 20, "box", ws=ws0).cpu().numpy().astype(np.float64)
    tc = parity.gpu_centre(bf, ws0.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
    r = int(round((np.sqrt(12 * 9.0 / 3 + 1) - 1) / 2))
    ref, kap = oracle.gp_bf(img.astype(np.float64), 3.0, 30.0, 20, "box", box=(r, 3), t_c=tc, return_kappa=True)
    parity.gate(y, ref, kap, min_gated=0.999, f=img, window=3 * r, label="box radius from sigma")
    with pytest.raises(bf.BFError):
        bf.bf_gp_workspace_size(1, 64, 64, 1.0, bf.make_opts(20, "box", fir_halfwidth=5, box_passes=3))
    o = bf.make_opts(20, "box", fir_halfwidth=2, box_passes=2, fir_two_pass=True)
    need = bf.bf_gp_workspace_size(1, 120, 140, 1.0, o)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    with pytest.raises(bf.BFError):
        bf.bf_gp_forward(x.data_ptr(), torch.empty_like(x).data_ptr(), 1, 120, 140, 140, 1.0, 30.0, o, ws.data_ptr(),
                         need, torch.cuda.current_stream().cuda_stream)
