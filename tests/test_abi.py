"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h; host-side argument checks reject bad input without touching a GPU."""
import ctypes
import glob
import os
import re

import pytest

import paper_1505_00077_gb300 as bfgp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ \*]*?\b(bf_[A-Za-z0-9_]+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = bfgp.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "bf_gp_forward" in names and len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_declarations():
    assert set(declared_functions()) <= set(bfgp.exported_symbols())


def test_status_strings():
    assert bfgp.status_string(bfgp.BF_OK) == "BF_OK"
    assert bfgp.status_string(bfgp.BF_ERR_WORKSPACE) == "BF_ERR_WORKSPACE"


def test_workspace_size_formula():
    o = bfgp.make_opts(20, "iir")
    n = bfgp.bf_gp_workspace_size(1, 4096, 4096, 10.0, o)
    # K = 22 channel planes of FP32 dominate
    assert 22 * 4096 * 4096 * 4 <= n < 22 * 4096 * 4096 * 4 + (1 << 20)
    assert bfgp.bf_gp_workspace_size(3, 100, 30, 2.0, bfgp.make_opts(4, "fir")) >= 3 * 6 * 100 * 32 * 4


@pytest.mark.parametrize("args", [
    (0, 16, 16, 3.0), (1, 0, 16, 3.0), (1, 16, 0, 3.0), (1, 16, 16, 0.0), (1, 16, 16, float("nan")),
])
def test_workspace_size_rejects_bad_sizes(args):
    with pytest.raises(bfgp.BFError) as e:
        bfgp.bf_gp_workspace_size(*args, bfgp.make_opts())
    assert e.value.status == bfgp.BF_ERR_INVALID_ARG


def test_bad_options_rejected():
    for o in (bfgp.make_opts(order=-1), bfgp.make_opts(order=63), bfgp.make_opts(spatial=7)):
        with pytest.raises(bfgp.BFError):
            bfgp.bf_gp_workspace_size(1, 32, 32, 2.0, o)
    o = bfgp.make_opts()
    o.reserved[1] = 1
    with pytest.raises(bfgp.BFError):
        bfgp.bf_gp_workspace_size(1, 32, 32, 2.0, o)
    for t in (8, 48, 128, -1):  # fused FIR tile heights are 16, 32 and 64 rows
        with pytest.raises(bfgp.BFError):
            bfgp.bf_gp_workspace_size(1, 32, 32, 2.0, bfgp.make_opts(20, "fir", fir_tile=t))
    for t in (0, 16, 32, 64):
        assert bfgp.bf_gp_workspace_size(1, 32, 32, 2.0, bfgp.make_opts(20, "fir", fir_tile=t)) > 0


def test_unsupported_sizes_reported():
    # FIR window wider than the kernels' 12 taps, rows longer than 8192, IIR columns longer than 8192
    # (CUDA-core column pass) or 4096 (tensor-core column passes)
    with pytest.raises(bfgp.BFError) as e:
        bfgp.bf_gp_workspace_size(1, 64, 64, 5.0, bfgp.make_opts(20, "fir"))
    assert e.value.status == bfgp.BF_ERR_UNSUPPORTED
    with pytest.raises(bfgp.BFError):
        bfgp.bf_gp_workspace_size(1, 16, 8193, 5.0, bfgp.make_opts(20, "iir"))
    for engine, hmax in ((0, 8192), (1, 8192), (2, 4096), (3, 4096)):
        o = bfgp.make_opts(20, "iir", engine=engine)
        with pytest.raises(bfgp.BFError) as e:
            bfgp.bf_gp_workspace_size(1, hmax + 1, 16, 5.0, o)
        assert e.value.status == bfgp.BF_ERR_UNSUPPORTED
        assert bfgp.bf_gp_workspace_size(1, hmax, 16, 5.0, o) > 0
    assert bfgp.bf_gp_workspace_size(1, 4096, 8192, 5.0, bfgp.make_opts(20, "iir")) > 0


def test_forward_rejects_bad_pointers_before_any_cuda_call():
    o = bfgp.make_opts()
    with pytest.raises(bfgp.BFError) as e:
        bfgp.bf_gp_forward(0, 0, 1, 16, 16, 16, 3.0, 30.0, o, 0, 0)
    assert e.value.status == bfgp.BF_ERR_INVALID_ARG
    # pitch < W
    with pytest.raises(bfgp.BFError) as e:
        bfgp.bf_gp_forward(256, 1 << 20, 1, 16, 16, 8, 3.0, 30.0, o, 1 << 24, 1 << 20)
    assert e.value.status == bfgp.BF_ERR_INVALID_ARG
    # sigma_r <= 0
    with pytest.raises(bfgp.BFError) as e:
        bfgp.bf_gp_forward(256, 1 << 20, 1, 16, 16, 16, 3.0, 0.0, o, 1 << 24, 1 << 20)
    assert e.value.status == bfgp.BF_ERR_INVALID_ARG
    # workspace too small / misaligned
    with pytest.raises(bfgp.BFError) as e:
        bfgp.bf_gp_forward(256, 1 << 20, 1, 16, 16, 16, 3.0, 30.0, o, 1 << 24, 64)
    assert e.value.status == bfgp.BF_ERR_WORKSPACE
    with pytest.raises(bfgp.BFError) as e:
        bfgp.bf_gp_forward(256, 1 << 20, 1, 16, 16, 16, 3.0, 30.0, o, (1 << 24) + 8, 1 << 30)
    assert e.value.status == bfgp.BF_ERR_WORKSPACE
    # input or output not 4-byte aligned
    for f_ptr, y_ptr in ((258, 1 << 20), (256, (1 << 20) + 2)):
        with pytest.raises(bfgp.BFError) as e:
            bfgp.bf_gp_forward(f_ptr, y_ptr, 1, 16, 16, 16, 3.0, 30.0, o, 1 << 24, 1 << 30)
        assert e.value.status == bfgp.BF_ERR_INVALID_ARG
    # overlapping input and output
    with pytest.raises(bfgp.BFError) as e:
        bfgp.bf_gp_forward(1 << 20, (1 << 20) + 64, 1, 16, 16, 16, 3.0, 30.0, o, 1 << 24, 1 << 30)
    assert e.value.status == bfgp.BF_ERR_INVALID_ARG


def test_autotuner_rejects_bad_pointers_before_any_cuda_call():
    o = bfgp.make_opts()
    for args in ((0, 256), (256, 0)):
        with pytest.raises(bfgp.BFError) as e:
            bfgp.bf_gp_autotune(args[0], args[1], 1, 16, 16, 16, 3.0, 30.0, o, 1 << 20, 1 << 20)
        assert e.value.status == bfgp.BF_ERR_INVALID_ARG
    with pytest.raises(bfgp.BFError) as e:
        bfgp.bf_gp_batched_plan_tune(0, 1 << 20, 1 << 20)
    assert e.value.status == bfgp.BF_ERR_INVALID_ARG
    bfgp.bf_gp_autotune_clear()  # no device needed


def test_order_rule():
    """Smallest even N whose Gauss-polynomial kernel error is <= eps on [-R, R]."""
    assert bfgp.bf_gp_order_for_tol(30.0, 127.5, 1e-3) == 34
    assert bfgp.bf_gp_order_for_tol(50.0, 127.5, 1e-3) == 16
    assert bfgp.bf_gp_order_for_tol(1e9, 127.5, 1e-3) == 0
    assert bfgp.bf_gp_order_for_tol(5.0, 127.5, 1e-3) == -1


def test_fp32_order_limit():
    """The host copy of the range test: wide range kernels carry any order,
    the limit falls as (R / sigma_r)^2 grows, and none is possible where
    exp(-s^2 / 2) leaves FP32 altogether."""
    import paper_1505_00077_gb300 as bf
    assert bf.bf_gp_order_fp32_limit(3.0, 100.0, 127.5) == 62
    lims = [bf.bf_gp_order_fp32_limit(3.0, sr, 127.5) for sr in (60.0, 30.0, 20.0, 15.0, 12.0, 10.0)]
    assert all(a >= b for a, b in zip(lims, lims[1:]))
    assert lims[0] == 62 and lims[-1] < 62
    assert bf.bf_gp_order_fp32_limit(3.0, 0.1, 127.5) == -1
    assert bf.bf_gp_order_fp32_limit(3.0, -1.0, 127.5) == -1
