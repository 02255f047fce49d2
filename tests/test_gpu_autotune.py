"""GPU checks of the autotuner (bf_gp_autotune, bf_gp_batched_plan_tune): it
times every candidate, keeps the fastest per shape class, and the filter it
picks still agrees with the FP64 oracle; batched planes with tuned engines
give the single-image path's bytes."""
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


def _gated_max_err(gpu, ref, kap):
    return parity.gate(gpu, ref, kap, min_gated=0.99, label="autotuned")["max_err_gated"]


def _setup(bf, H, W, ss, spatial):
    img = synthetic.make_image(H, W, 8, 10.0, 20.0, synthetic.seed_for(11, H * 7 + W))
    x = torch.from_numpy(img).cuda()
    y = torch.empty_like(x)
    o = bf.make_opts(20, spatial)
    need = max(bf.bf_gp_workspace_size(1, H, W, ss, bf.make_opts(20, spatial, engine=e, fir_two_pass=t))
               for e in range(4) for t in (False, True))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    return img, x, y, o, ws, need


def test_autotune_recursive_times_every_engine_and_stores_the_fastest(bf):
    H, W, ss, sr = 300, 260, 6.0, 30.0
    img, x, y, o, ws, need = _setup(bf, H, W, ss, "iir")
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_autotune_clear()
    o, ms = bf.bf_gp_autotune(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, o, ws.data_ptr(), need, s, reps=3)
    assert all(t > 0 for t in ms), ms  # engines 0..3, each with 256- and 512-thread row-pass CTAs
    best = int(np.argmin(ms))
    assert o.engine == best // 2 and o.row_threads == (256, 512)[best % 2]
    # the stored choice: nothing timed, same engine and row-pass CTA
    o2 = bf.make_opts(20, "iir", engine=0)
    o2, ms2 = bf.bf_gp_autotune(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, o2, ws.data_ptr(), need, s)
    assert ms2 == [-1.0] * 8 and o2.engine == o.engine and o2.row_threads == o.row_threads
    # the tuned filter still agrees with the oracle
    y.fill_(float("nan"))
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, o, ws.data_ptr(), need, s)
    assert bf.bf_gp_get_device_status(ws.data_ptr(), s) == 0
    ref, kap = oracle.gp_bf(img.astype(np.float64), ss, sr, 20, "iir", t_c=parity.gpu_centre(bf, ws.data_ptr(), 0, s),
                            return_kappa=True)
    assert _gated_max_err(y.cpu().numpy().astype(np.float64), ref, kap) <= TOL
    # forgetting the choice times again
    bf.bf_gp_autotune_clear()
    _, ms3 = bf.bf_gp_autotune(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, bf.make_opts(20, "iir"),
                               ws.data_ptr(), need, s, reps=1)
    assert all(t > 0 for t in ms3)


def test_autotune_fir_chooses_between_fused_and_two_pass(bf):
    H, W, ss, sr = 256, 256, 3.0, 30.0
    img, x, y, o, ws, need = _setup(bf, H, W, ss, "fir")
    s = torch.cuda.current_stream().cuda_stream
    bf.bf_gp_autotune_clear()
    o, ms = bf.bf_gp_autotune(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, o, ws.data_ptr(), need, s, reps=3)
    # fused (32-row tiles); two-pass with 256 / 512 row threads; fused with 16- / 64-row tiles
    assert all(t > 0 for t in ms[:5]) and ms[5:] == [-1.0] * 3
    best = int(np.argmin(ms[:5]))
    assert o.fir_two_pass == (best in (1, 2)) and o.row_threads == (0, 256, 512, 0, 0)[best]
    assert o.fir_tile == (32, 0, 0, 16, 64)[best]
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, o, ws.data_ptr(), need, s)
    ref, kap = oracle.gp_bf(img.astype(np.float64), ss, sr, 20, "fir", t_c=parity.gpu_centre(bf, ws.data_ptr(), 0, s),
                            return_kappa=True)
    assert _gated_max_err(y.cpu().numpy().astype(np.float64), ref, kap) <= TOL


def test_autotune_rejects_a_workspace_too_small_for_every_candidate(bf):
    H, W, ss = 64, 64, 4.0
    img, x, y, o, ws, need = _setup(bf, H, W, ss, "iir")
    bf.bf_gp_autotune_clear()
    with pytest.raises(bf.BFError) as e:
        bf.bf_gp_autotune(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, 30.0, o, ws.data_ptr(), 256,
                          torch.cuda.current_stream().cuda_stream)
    assert e.value.status == bf.BF_ERR_UNSUPPORTED


def test_batched_plan_tune_gives_the_single_image_bytes_per_plane(bf):
    shapes = [(256, 256, 3.0, 20.0), (1030, 300, 9.0, 40.0), (300, 1030, 2.0, 25.0), (700, 900, 12.0, 30.0)]
    planes = []
    for i, (H, W, ss, sr) in enumerate(shapes):
        img = synthetic.make_image(H, W, 16, 10.0, 0.0, synthetic.seed_for(12, i))
        x = torch.from_numpy(img).cuda()
        planes.append((x, torch.full_like(x, float("nan")), ss, sr, 20))
    bf.bf_gp_autotune_clear()
    bfilt = bf.BatchedFilter(planes, autotune=True)
    assert all(e in (0, 1, 2, 3) for e in bfilt.engines)
    for x, y, *_ in planes:
        y.fill_(float("nan"))
    bfilt.run()
    torch.cuda.synchronize()
    for (x, y, ss, sr, order), eng in zip(planes, bfilt.engines):
        H, W = x.shape
        o = bf.make_opts(order, "iir", engine=eng)
        need = bf.bf_gp_workspace_size(1, H, W, ss, o)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        y1 = torch.empty_like(x)
        bf.bf_gp_forward(x.data_ptr(), y1.data_ptr(), 1, H, W, W, ss, sr, o, ws.data_ptr(), need,
                         torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert torch.equal(y, y1)


@pytest.mark.parametrize("spatial,engine,ss", [("iir", 0, 6.0), ("iir", 1, 6.0), ("iir", 2, 6.0), ("fir", 0, 2.0)])
def test_row_threads_change_nothing_but_the_launch(bf, spatial, engine, ss):
    """The row pass's CTA size (one knob the autotuner turns) regroups rows into CTAs;
    every row is filtered the same way, so the result is the same bit for bit."""
    H, W = 301, 700
    img = synthetic.make_image(H, W, 8, 10.0, 20.0, synthetic.seed_for(11, 77))
    x = torch.from_numpy(img).cuda()
    s = torch.cuda.current_stream().cuda_stream
    outs = []
    for rt in (0, 256, 512):
        o = bf.make_opts(20, spatial, engine=engine, fir_two_pass=True, row_threads=rt)
        need = bf.bf_gp_workspace_size(1, H, W, ss, o)
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        y = torch.full_like(x, float("nan"))
        bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, 30.0, o, ws.data_ptr(), need, s)
        outs.append(y.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    with pytest.raises(bf.BFError):
        bf.bf_gp_workspace_size(1, H, W, ss, bf.make_opts(20, spatial, row_threads=384))
