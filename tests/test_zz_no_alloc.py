"""The no-allocation forward entry point, bf_gp_forward_noalloc.

For callers that cannot allocate device memory or hand the library a
workspace (plug-in hosts that only pass input and output buffers, code that
runs while a stream is captured, latency-bound loops that cannot afford the
device synchronisation cudaMalloc/cudaFree may cause): the entry point uses a
static scratch array inside the library instead.  These tests call it
through the C ABI twice in a row and compare each result with bf_gp_forward
(the workspace entry point) on the same input, bit for bit (the same
launches; only where the scratch lives differs); they also check that a
request larger than the scratch is refused before anything runs.  Collected last so a failure here comes after
every other test has run.
"""
import numpy as np
import pytest

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


def _with_workspace(bf, x, H, W, ss, sr, opts, stream):
    need = bf.bf_gp_workspace_size(1, H, W, ss, opts)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    bf.bf_gp_forward(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, opts, ws.data_ptr(), need, stream)
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("H,W,ss,sr,N,spatial", [
    (256, 256, 3.0, 30.0, 20, "fir"),   # the 256x256 workload
    (300, 260, 6.0, 25.0, 20, "iir"),   # ragged, recursive filter
    (512, 512, 10.0, 20.0, 20, "iir"),  # near the scratch limit (23 MB of 32 MB)
])
def test_noalloc_matches_workspace_entry_point_twice(bf, H, W, ss, sr, N, spatial):
    img = synthetic.make_image(H, W, 12, 10.0, 0.0, synthetic.seed_for(7, H + W))
    x = torch.from_numpy(img).cuda()
    opts = bf.make_opts(N, spatial)
    assert bf.bf_gp_workspace_size(1, H, W, ss, opts) <= bf.BF_GP_NOALLOC_SCRATCH_BYTES
    stream = torch.cuda.current_stream().cuda_stream
    ref = _with_workspace(bf, x, H, W, ss, sr, opts, stream)
    for _ in range(2):  # two calls in a row share the same scratch
        y = torch.full_like(x, float("nan"))
        bf.bf_gp_forward_noalloc(x.data_ptr(), y.data_ptr(), 1, H, W, W, ss, sr, opts, stream)
        torch.cuda.synchronize()
        out = y.cpu().numpy()
        # the same launches on the same input as the workspace entry point: only where the
        # scratch lives differs, so the result is the same bit for bit
        assert np.array_equal(out, ref)


def test_noalloc_rejects_requests_beyond_the_scratch(bf):
    x = torch.zeros((1024, 1024), dtype=torch.float32, device="cuda")
    y = torch.full_like(x, 3.0)
    opts = bf.make_opts(20, "iir")
    assert bf.bf_gp_workspace_size(1, 1024, 1024, 10.0, opts) > bf.BF_GP_NOALLOC_SCRATCH_BYTES
    with pytest.raises(bf.BFError) as e:
        bf.bf_gp_forward_noalloc(x.data_ptr(), y.data_ptr(), 1, 1024, 1024, 1024, 10.0, 20.0, opts,
                                 torch.cuda.current_stream().cuda_stream)
    assert e.value.status == bf.BF_ERR_WORKSPACE
    assert "scratch" in bf.last_cuda_error()
    torch.cuda.synchronize()
    assert bool((y == 3.0).all())  # nothing ran
