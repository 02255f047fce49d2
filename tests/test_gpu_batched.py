"""GPU parity of the batched path (bf_gp_batched): uneven plane sizes, per-plane
sigma_s / sigma_r / order, captured into a CUDA graph and replayed.  Sampled
planes are checked against the FP64 oracle (recursive filter) and every plane
against the single-image path."""
import math

import numpy as np
import pytest

import oracle
import parity
import synthetic

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1505_00077_gb300 as m
    m.build()
    return m


def make_batch(n_images, lo, hi, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_images):
        H, W = int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))
        ss = float(math.exp(rng.uniform(0.0, math.log(16.0))))
        sr = float(math.exp(rng.uniform(math.log(10.0), math.log(60.0))))
        img = synthetic.make_image(H, W, max(1, 16 * H * W // 65536), 10.0, 0.0, seed * 100 + i, planes=3)
        out.append((img, ss, sr))
    return out


def test_batched_graph_matches_single_and_oracle(bf):
    batch = make_batch(10, 33, 700, 4)
    planes = []
    for img, ss, sr in batch:
        for c in range(3):
            x = torch.from_numpy(np.ascontiguousarray(img[c])).cuda()
            planes.append((x, torch.full_like(x, float("nan")), ss, sr, 20 if c != 1 else 12))
    bfilt = bf.BatchedFilter(planes)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bfilt.run()  # warm up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    for x, y, *_ in planes:
        y.fill_(float("nan"))
    with torch.cuda.graph(g):
        bfilt.run()
    g.replay()
    torch.cuda.synchronize()
    assert (bfilt.status() & ~bf.BF_DEV_NONPOS_Q) == 0
    outs = [y.cpu().numpy() for _, y, *_ in planes]
    assert all(np.isfinite(o).all() for o in outs)  # Q <= 0 pixels keep their value
    singles = []
    for i, (x, y, ss, sr, order) in enumerate(planes):
        # the batch runs each plane through the single-image launches: the same result bit for bit
        o = bf.make_opts(order, "iir")
        need = bf.bf_gp_workspace_size(1, x.shape[0], x.shape[1], ss, o)
        wsb = torch.empty(need, dtype=torch.uint8, device="cuda")
        single = torch.empty_like(x)
        st = torch.cuda.current_stream().cuda_stream
        bf.bf_gp_forward(x.data_ptr(), single.data_ptr(), 1, x.shape[0], x.shape[1], x.shape[1], ss, sr, o,
                         wsb.data_ptr(), need, st)
        torch.cuda.synchronize()
        assert np.array_equal(outs[i], single.cpu().numpy()), i
        singles.append((bf.bf_gp_get_device_counters(wsb.data_ptr(), st)[0], parity.gpu_centre(bf, wsb.data_ptr(), 0, st)))
    # the batch's counters are the sums over its planes
    n_q0 = sum(c for c, _ in singles)
    assert bfilt.counters() == [n_q0, 0, 0, 0]
    assert ((bfilt.status() & bf.BF_DEV_NONPOS_Q) != 0) == (n_q0 > 0)
    for i in (0, 4, 7, 11, 14, 19, 22, 29):  # 8 sampled planes
        x, y, ss, sr, order = planes[i]
        f = x.cpu().numpy()
        ref, kap = oracle.gp_bf(f.astype(np.float64), ss, sr, order, "iir", t_c=singles[i][1], return_kappa=True)
        # sigma_r is drawn down to 10: some pixels are unresolvable, some have Q <= 0
        parity.gate(outs[i], ref, kap, min_gated=0.98, label=f"batched plane {i} ss={ss:.3g} sr={sr:.3g} N={order}")
        assert parity.kept_value_pixels(outs[i], f, kap) == singles[i][0]
    # replaying again gives the same result
    before = [y.clone() for _, y, *_ in planes]
    g.replay()
    torch.cuda.synchronize()
    for b0, (_, y, *_) in zip(before, planes):
        assert torch.equal(b0, y)


def test_batched_rejects_bad_plans(bf):
    x = torch.zeros((16, 16), device="cuda")
    with pytest.raises(bf.BFError):
        bf.bf_gp_batched_plan_create([(x.data_ptr(), x.data_ptr(), 16, 16, 8, 2.0, 30.0, 20)])  # pitch < W
    with pytest.raises(bf.BFError):
        bf.bf_gp_batched_plan_create([(x.data_ptr(), x.data_ptr(), 9000, 16, 16, 2.0, 30.0, 20)])  # H > 8192
    with pytest.raises(bf.BFError):
        bf.bf_gp_batched_plan_create([(x.data_ptr(), x.data_ptr(), 16, 9000, 9000, 2.0, 30.0, 20)])  # W > 8192


def test_adaptive_order_per_plane(bf):
    """tol given: each plane's order is the smallest even N whose kernel error on
    [-R, R] is <= tol, with R = max |f - mean f| measured on the device, capped
    at 62 and at the FP32 range limit; no plane raises BF_DEV_RANGE, every
    plane matches the FP64 oracle run with its own order, and a plane that
    gets more than N = 20 is closer to Eq. (1) than N = 20."""
    specs = [(300, 280, 3.0, 70.0), (256, 512, 2.0, 45.0), (640, 200, 8.0, 30.0), (200, 200, 4.0, 20.0),
             (129, 333, 1.5, 100.0), (512, 96, 6.0, 15.0)]
    planes, imgs = [], []
    for i, (H, W, ss, sr) in enumerate(specs):
        img = synthetic.make_image(H, W, 8, 10.0, 0.0, synthetic.seed_for(4, 500 + i))
        imgs.append(img)
        x = torch.from_numpy(img).cuda()
        planes.append((x, torch.empty_like(x), ss, sr))
    tol = 1e-3
    bfilt = bf.BatchedFilter(planes, tol=tol)
    f64 = [im.astype(np.float64) for im in imgs]
    expect = []
    for im, (H, W, ss, sr) in zip(f64, specs):
        R = float(np.max(np.abs(im - oracle.mean(im))))
        n = bf.bf_gp_order_for_tol(sr, R, tol)
        n = 62 if n < 0 else min(n, 62)
        expect.append(max(0, min(n, bf.bf_gp_order_fp32_limit(ss, sr, R))))
    assert bfilt.orders == expect
    assert len(set(expect)) >= 4 and max(expect) > 20  # uneven channel counts in one batch
    bfilt.run()
    torch.cuda.synchronize()
    assert (bfilt.status() & ~bf.BF_DEV_NONPOS_Q) == 0
    for i, ((x, y, ss, sr), im, N) in enumerate(zip(planes, f64, bfilt.orders)):
        tc = float(np.float32(oracle.mean(im)))
        ref, kap = oracle.gp_bf(im, ss, sr, N, "iir", t_c=tc, return_kappa=True)
        # floor: the oracle's own fraction on these planes (>= 0.96)
        parity.gate(y.cpu().numpy(), ref, kap, min_gated=0.95, label=f"adaptive plane {i} N={N}")
    i = int(np.argmax(expect))
    ref20 = oracle.gp_bf(f64[i], specs[i][2], specs[i][3], 20, "iir")
    exact = oracle.direct_bf(f64[i], specs[i][2], specs[i][3])
    out = planes[i][1].cpu().numpy().astype(np.float64)
    assert np.mean((out - exact) ** 2) < np.mean((ref20 - exact) ** 2)


def _persistent_shape(planes):
    """Cluster size of the persistent launch and each plane's column items."""
    def p2(v):
        return 1 << max(0, (v - 1).bit_length())
    pcl = p2(max((x.shape[0] + 511) // 512 for x, *_ in planes))
    items = []
    for x, *_ in planes:
        G = p2((x.shape[0] + 511) // 512)
        strips = (x.shape[1] + 7) // 8
        per = pcl // G
        items.append((strips + per - 1) // per)
    return pcl, items


def _forked_outputs(bfilt, planes):
    for _, y, *_ in planes:
        y.fill_(float("nan"))
    bfilt.run()
    torch.cuda.synchronize()
    return [y.clone() for _, y, *_ in planes], bfilt.status(), bfilt.counters()


@pytest.mark.parametrize("n_images,lo,hi,seed", [(10, 33, 700, 4), (6, 256, 2048, 8)])
def test_persistent_matches_forked_path(bf, n_images, lo, hi, seed):
    """One persistent launch over the whole batch (work items taken from a
    counter, per-plane readiness counters) gives every plane the forked
    path's result bit for bit, the same status and counters, also when
    captured into a graph and replayed.  The second batch has sides up to
    2048: column strips of 1, 2 and 4 CTAs share clusters of 4."""
    batch = make_batch(n_images, lo, hi, seed)
    planes = []
    for img, ss, sr in batch:
        for c in range(3):
            x = torch.from_numpy(np.ascontiguousarray(img[c])).cuda()
            planes.append((x, torch.empty_like(x), ss, sr, 20 if c != 1 else 12))
    bfilt = bf.BatchedFilter(planes)
    ref, st_ref, cnt_ref = _forked_outputs(bfilt, planes)
    for _, y, *_ in planes:
        y.fill_(float("nan"))
    bfilt.run_persistent()
    torch.cuda.synchronize()
    assert bfilt.status() == st_ref
    assert bfilt.counters() == cnt_ref
    for i, (r, (_, y, *_)) in enumerate(zip(ref, planes)):
        assert torch.equal(r, y), i
    # captured and replayed
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            bfilt.run_persistent()
    torch.cuda.current_stream().wait_stream(s)
    for rep in range(2):
        for _, y, *_ in planes:
            y.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert bfilt.status() == st_ref
        for i, (r, (_, y, *_)) in enumerate(zip(ref, planes)):
            assert torch.equal(r, y), (rep, i)


def test_persistent_wait_gives_up_on_a_starved_counter(bf):
    """The host makes one plane's column items wait for a row group that does
    not exist: each of them gives up after its budget, raises BF_DEV_TIMEOUT
    and counts one wait in counter 3; the launch ends, the plane's output is
    left as it was, every other plane is still filtered, and the next launch
    with the normal budget is clean."""
    batch = make_batch(5, 64, 1200, 12)
    planes = []
    for img, ss, sr in batch:
        for c in range(3):
            x = torch.from_numpy(np.ascontiguousarray(img[c])).cuda()
            planes.append((x, torch.empty_like(x), ss, sr, 16))
    bfilt = bf.BatchedFilter(planes)
    ref, st_ref, cnt_ref = _forked_outputs(bfilt, planes)
    _, items = _persistent_shape(planes)
    starved = 4
    bf.bf_gp_batched_plan_set_wait(bfilt.plan, 1 << 20, starved)  # about half a millisecond per wait
    for _, y, *_ in planes:
        y.fill_(-7.0)
    bfilt.run_persistent()
    torch.cuda.synchronize()
    assert bfilt.status() & bf.BF_DEV_TIMEOUT
    assert bfilt.counters()[3] == items[starved]
    for i, (r, (_, y, *_)) in enumerate(zip(ref, planes)):
        if i == starved:
            assert bool((y == -7.0).all())
        else:
            assert torch.equal(r, y), i
    bf.bf_gp_batched_plan_set_wait(bfilt.plan, 1 << 32, -1)
    bfilt.run_persistent()
    torch.cuda.synchronize()
    assert bfilt.status() == st_ref and bfilt.counters() == cnt_ref
    for r, (_, y, *_) in zip(ref, planes):
        assert torch.equal(r, y)
    with pytest.raises(bf.BFError):
        bf.bf_gp_batched_plan_set_wait(bfilt.plan, 0, -1)
    with pytest.raises(bf.BFError):
        bf.bf_gp_batched_plan_set_wait(bfilt.plan, 100, len(planes))


def test_persistent_rejects_rows_longer_than_4096(bf):
    x = torch.zeros((64, 5000), device="cuda")
    bfilt = bf.BatchedFilter([(x, torch.empty_like(x), 3.0, 30.0, 8)])
    with pytest.raises(bf.BFError):
        bfilt.run_persistent()


def test_persistent_edge_planes(bf):
    """Edge planes through the persistent launch: a constant plane (copied), a
    plane holding a NaN (copied, BF_DEV_NONFINITE_IN), 1 x 1, single rows and
    columns, a column 3 CTAs tall run by a group of 4. Bit for bit the forked
    path's output, status word and counters."""
    rng = np.random.default_rng(31)
    shapes = [(40, 70), (33, 33), (1, 1), (1, 7), (5, 1), (700, 3), (1300, 20), (257, 513)]
    planes = []
    for i, (H, W) in enumerate(shapes):
        img = synthetic.make_image(H, W, 4, 10.0, 0.0, synthetic.seed_for(13, i))
        if i == 0:
            img[:] = 77.0
        if i == 1:
            img[5, 7] = np.nan
        x = torch.from_numpy(np.ascontiguousarray(img)).cuda()
        planes.append((x, torch.empty_like(x), float(rng.uniform(1, 12)), float(rng.uniform(15, 60)), 18))
    bfilt = bf.BatchedFilter(planes)
    ref, st_ref, cnt_ref = _forked_outputs(bfilt, planes)
    assert st_ref & bf.BF_DEV_NONFINITE_IN and cnt_ref[1] == 1
    for _, y, *_ in planes:
        y.fill_(-3.0)
    bfilt.run_persistent()
    torch.cuda.synchronize()
    assert bfilt.status() == st_ref and bfilt.counters() == cnt_ref
    for i, (r, (x, y, *_)) in enumerate(zip(ref, planes)):
        assert torch.equal(torch.nan_to_num(r, nan=-1.0), torch.nan_to_num(y, nan=-1.0)), i
    assert torch.equal(planes[0][1], planes[0][0])  # the constant plane comes back unchanged


def test_full_size_uneven_batch(bf):
    """The batched workload at full size (64 images with sides in 256..2048, 3
    planes each, 290 Mpx, N = 20), in the launch configurations the bench
    times: the forked graph path and the persistent launch give every plane
    the same result bit for bit, and three sampled planes (the smallest, a
    middle one and the largest) pass the parity gate against the FP64
    oracle on the whole plane."""
    specs = synthetic.uneven_batch_specs()
    planes, imgs = [], []
    for spec in specs:
        img = synthetic.uneven_batch_image(spec)
        for c in range(3):
            a = np.ascontiguousarray(img[c])
            x = torch.from_numpy(a).cuda()
            planes.append((x, torch.empty_like(x), spec[3], spec[4], 20))
            imgs.append((spec, c))
    assert len(planes) == 192
    bfilt = bf.BatchedFilter(planes)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        bfilt.run()
        with torch.cuda.graph(g, stream=s):
            bfilt.run()
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    torch.cuda.synchronize()
    st, cnt = bfilt.status(), bfilt.counters()
    assert (st & ~bf.BF_DEV_NONPOS_Q) == 0
    forked = [y.clone() for _, y, *_ in planes]
    for _, y, *_ in planes:
        y.fill_(float("nan"))
    bfilt.run_persistent()
    torch.cuda.synchronize()
    assert bfilt.status() == st and bfilt.counters() == cnt
    for i, (r, (_, y, *_)) in enumerate(zip(forked, planes)):
        assert torch.equal(r, y), i
    sizes = [x.numel() for x, *_ in planes]
    order = np.argsort(sizes, kind="stable")  # planes 48, 39 and 68
    for i in (int(order[0]), int(order[len(order) // 2]), int(order[-1])):
        x, y, ss, sr, N = planes[i]
        f = x.cpu().numpy().astype(np.float64)
        tc = float(np.float32(oracle.mean(f)))
        ref, kap = oracle.gp_bf(f, ss, sr, N, "iir", t_c=tc, return_kappa=True)
        gpu = y.cpu().numpy()
        # floor: the oracle's own resolvable fractions on these planes, 0.996, 0.975 (sigma_r 10.9) and 0.998
        parity.gate(gpu, ref, kap, min_gated=0.97, label=f"full batch plane {i} {x.shape[0]}x{x.shape[1]} ss={ss:.3g} sr={sr:.3g}")
        parity.kept_value_pixels(gpu, f, kap)
