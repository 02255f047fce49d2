"""GB300 (sm_103a) Gauss-polynomial bilateral filter -- Python binding.

A thin ctypes layer over the C ABI in include/bf_gp.h (libbfgp.so, built
in-tree by :func:`paper_1505_00077_gb300.build.build`).  Functions named
``bf_gp_*`` take the same arguments as the C entry points (device pointers
as integers, a stream handle as an integer); :func:`bilateral_gp` is the
tensor-level convenience wrapper that allocates the output and a cached
workspace with PyTorch and calls :func:`bf_gp_forward` on the current stream.
Every step of the filter runs in the library's CUDA kernels; there is no CPU
path.

Method: Chaudhury, "Fast and Accurate Bilateral Filtering using
Gauss-Polynomial Decomposition" (Algorithm 1, Eqs. (7)-(11)).
"""
from __future__ import annotations

import ctypes
import math
import os

from .build import LIB, build  # noqa: F401

BF_OK = 0
BF_ERR_INVALID_ARG = 1
BF_ERR_WORKSPACE = 2
BF_ERR_CUDA = 3
BF_ERR_UNSUPPORTED = 4
BF_ERR_TIMEOUT = 5

BF_DEV_NONPOS_Q = 0x1
BF_DEV_NONFINITE_IN = 0x2
BF_DEV_RANGE = 0x4
BF_DEV_TIMEOUT = 0x8

BF_SPATIAL_AUTO = 0
BF_SPATIAL_FIR = 1
BF_SPATIAL_IIR = 2
BF_SPATIAL_BOX = 3
_SPATIAL = {"auto": BF_SPATIAL_AUTO, "fir": BF_SPATIAL_FIR, "iir": BF_SPATIAL_IIR, "box": BF_SPATIAL_BOX}

BF_CENTRE_MEAN = 0
BF_CENTRE_GIVEN = 1


class BFError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}"
                         + (f" ({last_cuda_error()})" if status == BF_ERR_CUDA else ""))


class bf_gp_opts(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("spatial", ctypes.c_int), ("centre", ctypes.c_int),
                ("fir_halfwidth", ctypes.c_int), ("t_c", ctypes.c_double), ("engine", ctypes.c_int),
                ("fir_two_pass", ctypes.c_int), ("box_passes", ctypes.c_int), ("tc5_wait_test", ctypes.c_int),
                ("row_threads", ctypes.c_int), ("fir_tile", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class bf_gp_plane(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p), ("y", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("pitch", ctypes.c_int), ("sigma_s", ctypes.c_float), ("sigma_r", ctypes.c_float),
                ("order", ctypes.c_int)]


_lib = None


def _load():
    """Load libbfgp.so; fail loudly if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError(f"CUDA library not built ({LIB}); run paper_1505_00077_gb300.build.build()")
    lib = ctypes.CDLL(LIB)
    c_int, c_float, c_double, c_size_t, c_void_p = ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p
    P = ctypes.POINTER
    sig = {
        "bf_gp_default_opts": (None, [P(bf_gp_opts)]),
        "bf_status_string": (ctypes.c_char_p, [c_int]),
        "bf_gp_last_cuda_error": (ctypes.c_char_p, []),
        "bf_gp_version": (c_int, []),
        "bf_gp_workspace_size": (c_int, [c_int, c_int, c_int, c_float, P(bf_gp_opts), P(c_size_t)]),
        "bf_gp_forward": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float, c_float, P(bf_gp_opts),
                                  c_void_p, c_size_t, c_void_p]),
        "bf_gp_phase_stats": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_float, c_float, P(bf_gp_opts),
                                      c_void_p, c_size_t, c_void_p]),
        "bf_gp_phase_rows": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_float, c_float, P(bf_gp_opts),
                                     c_void_p, c_size_t, c_void_p]),
        "bf_gp_phase_cols": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float, c_float,
                                     P(bf_gp_opts), c_void_p, c_size_t, c_void_p]),
        "bf_gp_forward_train": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float, c_float,
                                        P(bf_gp_opts), c_void_p, c_size_t, c_void_p]),
        "bf_gp_backward": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int,
                                   c_float, c_float, P(bf_gp_opts), c_void_p, c_size_t, c_void_p]),
        "bf_gp_batched_plan_create": (c_int, [P(bf_gp_plane), c_int, P(bf_gp_opts), P(c_void_p)]),
        "bf_gp_batched_plan_workspace": (c_int, [c_void_p, P(c_size_t)]),
        "bf_gp_batched_plan_upload": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p]),
        "bf_gp_batched": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p]),
        "bf_gp_batched_plan_destroy": (None, [c_void_p]),
        "bf_gp_batched_plan_stats_workspace": (c_int, [c_void_p, P(c_size_t)]),
        "bf_gp_batched_plane_stats": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p, P(c_double), P(c_double)]),
        "bf_gp_forward_noalloc": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float, c_float,
                                          P(bf_gp_opts), c_void_p]),
        "bf_gp_host_workspace_size": (c_int, [c_int, c_int, c_int, c_float, P(bf_gp_opts), P(c_size_t)]),
        "bf_gp_forward_host": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_float, c_float, P(bf_gp_opts),
                                       c_void_p, c_size_t, c_void_p]),
        "bf_gp_get_device_status": (c_int, [c_void_p, c_void_p, P(ctypes.c_uint32)]),
        "bf_gp_get_plane_stats": (c_int, [c_void_p, c_int, c_void_p, P(c_double), P(c_double)]),
        "bf_gp_get_device_counters": (c_int, [c_void_p, c_void_p, P(ctypes.c_ulonglong)]),
        "bf_gp_order_for_tol": (c_int, [c_double, c_double, c_double]),
        "bf_gp_order_fp32_limit": (c_int, [c_double, c_double, c_double]),
        "bf_gp_joint_workspace_size": (c_int, [c_int, c_int, c_int, c_float, P(bf_gp_opts), P(c_size_t)]),
        "bf_gp_forward_joint": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float, c_float,
                                        P(bf_gp_opts), c_void_p, c_size_t, c_void_p]),
        "bf_gp_autotune": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_int, c_float, c_float, P(bf_gp_opts),
                                   c_void_p, c_size_t, c_void_p, c_int, P(c_float)]),
        "bf_gp_autotune_clear": (None, []),
        "bf_gp_batched_plan_tune": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p, c_int]),
        "bf_gp_batched_plan_engines": (c_int, [c_void_p, P(c_int)]),
        "bf_gp_batched_persistent": (c_int, [c_void_p, c_void_p, c_size_t, c_void_p]),
        "bf_gp_batched_plan_set_wait": (c_int, [c_void_p, ctypes.c_longlong, c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the binding expects the library to export."""
    return ["bf_gp_default_opts", "bf_status_string", "bf_gp_last_cuda_error", "bf_gp_version",
            "bf_gp_workspace_size", "bf_gp_forward", "bf_gp_phase_stats", "bf_gp_phase_rows", "bf_gp_phase_cols",
            "bf_gp_forward_train", "bf_gp_backward", "bf_gp_batched_plan_create", "bf_gp_batched_plan_workspace",
            "bf_gp_batched_plan_upload", "bf_gp_batched", "bf_gp_batched_plan_destroy",
            "bf_gp_batched_plan_stats_workspace", "bf_gp_batched_plane_stats", "bf_gp_forward_noalloc",
            "bf_gp_host_workspace_size", "bf_gp_forward_host",
            "bf_gp_get_device_status", "bf_gp_get_device_counters", "bf_gp_get_plane_stats", "bf_gp_order_for_tol", "bf_gp_order_fp32_limit",
            "bf_gp_joint_workspace_size", "bf_gp_forward_joint", "bf_gp_autotune", "bf_gp_autotune_clear",
            "bf_gp_batched_plan_tune", "bf_gp_batched_plan_engines", "bf_gp_batched_persistent",
            "bf_gp_batched_plan_set_wait"]


def status_string(status: int) -> str:
    return _load().bf_status_string(int(status)).decode()


def last_cuda_error() -> str:
    return _load().bf_gp_last_cuda_error().decode()


ENGINE_AUTO = 0        # tensor-core row pass, CUDA-core column pass
ENGINE_CUDA_CORE = 1
ENGINE_TENSOR = 2
ENGINE_TCGEN05 = 3     # half-chunk products on tcgen05 where a pass has such a kernel


def make_opts(order: int = 20, spatial="auto", t_c=None, fir_halfwidth: int = 0, engine: int = ENGINE_AUTO,
              fir_two_pass: bool = False, box_passes: int = 0, tc5_wait_test: int = 0,
              row_threads: int = 0, fir_tile: int = 0) -> bf_gp_opts:
    """spatial 'box': box_passes passes (0 = 3) of a flat kernel of half-width
    fir_halfwidth (0 = matched to sigma_s).  tc5_wait_test: see bf_gp_opts
    (testing the tcgen05 column pass's bounded wait only)."""
    o = bf_gp_opts()
    _load().bf_gp_default_opts(ctypes.byref(o))
    o.order = int(order)
    o.engine = int(engine)
    o.fir_two_pass = int(bool(fir_two_pass))
    o.box_passes = int(box_passes)
    o.tc5_wait_test = int(tc5_wait_test)
    o.row_threads = int(row_threads)
    o.fir_tile = int(fir_tile)
    o.spatial = _SPATIAL[spatial] if isinstance(spatial, str) else int(spatial)
    o.fir_halfwidth = int(fir_halfwidth)
    if t_c is not None:
        o.centre = BF_CENTRE_GIVEN
        o.t_c = float(t_c)
    return o


def _check(st: int, what: str):
    if st != BF_OK:
        raise BFError(st, what)


# ------------------------------------------------------- C-ABI mirrors


def bf_gp_workspace_size(planes, H, W, sigma_s, opts=None) -> int:
    n = ctypes.c_size_t(0)
    _check(_load().bf_gp_workspace_size(int(planes), int(H), int(W), float(sigma_s),
                                        ctypes.byref(opts) if opts is not None else None, ctypes.byref(n)),
           "bf_gp_workspace_size")
    return int(n.value)


def bf_gp_forward(f_ptr, y_ptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws_ptr, ws_bytes, stream=0) -> None:
    _check(_load().bf_gp_forward(ctypes.c_void_p(int(f_ptr)), ctypes.c_void_p(int(y_ptr)), int(planes), int(H),
                                 int(W), int(pitch), float(sigma_s), float(sigma_r),
                                 ctypes.byref(opts) if opts is not None else None,
                                 ctypes.c_void_p(int(ws_ptr)), int(ws_bytes), ctypes.c_void_p(int(stream))),
           "bf_gp_forward")


def _vp(v):
    return ctypes.c_void_p(int(v))


def _op(opts):
    return ctypes.byref(opts) if opts is not None else None


def bf_gp_phase_stats(f_ptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws_ptr, ws_bytes, stream=0) -> None:
    _check(_load().bf_gp_phase_stats(_vp(f_ptr), int(planes), int(H), int(W), int(pitch), float(sigma_s),
                                     float(sigma_r), _op(opts), _vp(ws_ptr), int(ws_bytes), _vp(stream)),
           "bf_gp_phase_stats")


def bf_gp_phase_rows(f_ptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws_ptr, ws_bytes, stream=0) -> None:
    _check(_load().bf_gp_phase_rows(_vp(f_ptr), int(planes), int(H), int(W), int(pitch), float(sigma_s),
                                    float(sigma_r), _op(opts), _vp(ws_ptr), int(ws_bytes), _vp(stream)),
           "bf_gp_phase_rows")


def bf_gp_phase_cols(f_ptr, y_ptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws_ptr, ws_bytes, stream=0) -> None:
    _check(_load().bf_gp_phase_cols(_vp(f_ptr), _vp(y_ptr), int(planes), int(H), int(W), int(pitch),
                                    float(sigma_s), float(sigma_r), _op(opts), _vp(ws_ptr), int(ws_bytes),
                                    _vp(stream)), "bf_gp_phase_cols")


def bf_gp_forward_train(f_ptr, y_ptr, saved_ptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws_ptr, ws_bytes,
                        stream=0) -> None:
    _check(_load().bf_gp_forward_train(_vp(f_ptr), _vp(y_ptr), _vp(saved_ptr), int(planes), int(H), int(W),
                                       int(pitch), float(sigma_s), float(sigma_r), _op(opts), _vp(ws_ptr),
                                       int(ws_bytes), _vp(stream)), "bf_gp_forward_train")


def bf_gp_backward(f_ptr, gy_ptr, saved_ptr, gf_ptr, gsr_ptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws_ptr,
                   ws_bytes, stream=0) -> None:
    _check(_load().bf_gp_backward(_vp(f_ptr), _vp(gy_ptr), _vp(saved_ptr), _vp(gf_ptr), _vp(gsr_ptr or 0),
                                  int(planes), int(H), int(W), int(pitch), float(sigma_s), float(sigma_r),
                                  _op(opts), _vp(ws_ptr), int(ws_bytes), _vp(stream)), "bf_gp_backward")


def bf_gp_batched_plan_create(planes, opts=None) -> int:
    """planes: list of (f_ptr, y_ptr, H, W, pitch, sigma_s, sigma_r, order).  Returns the plan handle."""
    arr = (bf_gp_plane * len(planes))()
    for i, (f, y, H, W, pitch, ss, sr, order) in enumerate(planes):
        arr[i] = bf_gp_plane(f, y, H, W, pitch, ss, sr, order)
    h = ctypes.c_void_p(0)
    _check(_load().bf_gp_batched_plan_create(arr, len(planes), _op(opts), ctypes.byref(h)), "bf_gp_batched_plan_create")
    return int(h.value)


def bf_gp_batched_plan_workspace(plan) -> int:
    n = ctypes.c_size_t(0)
    _check(_load().bf_gp_batched_plan_workspace(_vp(plan), ctypes.byref(n)), "bf_gp_batched_plan_workspace")
    return int(n.value)


def bf_gp_batched_plan_upload(plan, ws_ptr, ws_bytes, stream=0) -> None:
    _check(_load().bf_gp_batched_plan_upload(_vp(plan), _vp(ws_ptr), int(ws_bytes), _vp(stream)),
           "bf_gp_batched_plan_upload")


def bf_gp_batched(plan, ws_ptr, ws_bytes, stream=0) -> None:
    _check(_load().bf_gp_batched(_vp(plan), _vp(ws_ptr), int(ws_bytes), _vp(stream)), "bf_gp_batched")


def bf_gp_batched_persistent(plan, ws_ptr, ws_bytes, stream=0) -> None:
    """The whole batched forward as one persistent launch (see include/bf_gp.h)."""
    _check(_load().bf_gp_batched_persistent(_vp(plan), _vp(ws_ptr), int(ws_bytes), _vp(stream)),
           "bf_gp_batched_persistent")


def bf_gp_batched_plan_set_wait(plan, wait_cycles, starve_plane=-1) -> None:
    _check(_load().bf_gp_batched_plan_set_wait(_vp(plan), int(wait_cycles), int(starve_plane)),
           "bf_gp_batched_plan_set_wait")


BF_GP_TUNE_CANDIDATES = 8


def bf_gp_autotune(f_ptr, y_ptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws_ptr, ws_bytes, stream=0, reps=0):
    """Fastest engine (recursive filter) or FIR form, and row-pass CTA size, for
    this shape class, written into opts (a bf_gp_opts, modified in place and returned) with each
    candidate's mean time in ms (-1: not timed, e.g. a stored choice).  Times
    on the given buffers (y is overwritten) and synchronises; see include/bf_gp.h."""
    ms = (ctypes.c_float * BF_GP_TUNE_CANDIDATES)()
    _check(_load().bf_gp_autotune(_vp(f_ptr), _vp(y_ptr), int(planes), int(H), int(W), int(pitch), float(sigma_s),
                                  float(sigma_r), ctypes.byref(opts), _vp(ws_ptr), int(ws_bytes), _vp(stream),
                                  int(reps), ms),
           "bf_gp_autotune")
    return opts, [float(v) for v in ms]


def bf_gp_autotune_clear() -> None:
    _load().bf_gp_autotune_clear()


def bf_gp_batched_plan_tune(plan, ws_ptr, ws_bytes, stream=0, reps=0) -> None:
    _check(_load().bf_gp_batched_plan_tune(_vp(plan), _vp(ws_ptr), int(ws_bytes), _vp(stream), int(reps)),
           "bf_gp_batched_plan_tune")


def bf_gp_batched_plan_engines(plan, n):
    e = (ctypes.c_int * n)()
    _check(_load().bf_gp_batched_plan_engines(_vp(plan), e), "bf_gp_batched_plan_engines")
    return [int(v) for v in e]


def bf_gp_batched_plan_stats_workspace(plan) -> int:
    n = ctypes.c_size_t(0)
    _check(_load().bf_gp_batched_plan_stats_workspace(_vp(plan), ctypes.byref(n)), "bf_gp_batched_plan_stats_workspace")
    return int(n.value)


def bf_gp_batched_plane_stats(plan, n, ws_ptr, ws_bytes, stream=0):
    """(t_c, R) per plane of the plan, from its statistics pass (synchronises)."""
    tc = (ctypes.c_double * n)()
    R = (ctypes.c_double * n)()
    _check(_load().bf_gp_batched_plane_stats(_vp(plan), _vp(ws_ptr), int(ws_bytes), _vp(stream), tc, R),
           "bf_gp_batched_plane_stats")
    return list(tc), list(R)


def bf_gp_batched_plan_destroy(plan) -> None:
    _load().bf_gp_batched_plan_destroy(_vp(plan))


MAX_ORDER = 62  # K = N + 2 <= 64 channels


class BatchedFilter:
    """Owns a batched plan and its workspace for a fixed list of (input, output,
    sigma_s, sigma_r, order) planes (float32 CUDA tensors [H, W]).  run()
    enqueues every plane's forward on the plan's streams, forked from and
    joined back into the current stream; it is safe to capture in a CUDA graph.

    With tol, each plane gets its own order: the smallest even N whose
    Gauss-polynomial kernel error on [-R, R] is at most tol
    (bf_gp_order_for_tol), with R = max |f - t_c| measured on the device by
    the plan's statistics pass, capped at max_order and at the largest order
    whose terms FP32 can hold (bf_gp_order_fp32_limit).  The chosen orders are
    in self.orders.

    With autotune, each plane runs with the engine the autotuner measures
    fastest for its shape (bf_gp_batched_plan_tune; the outputs are written
    while it times).  The engines are in self.engines."""

    def __init__(self, planes, order_default=20, t_c=None, tol=None, max_order=MAX_ORDER, autotune=False):
        import torch
        self._keep = []
        spec = []
        for item in planes:
            x, y, ss, sr = item[:4]
            order = item[4] if len(item) > 4 else order_default
            assert x.is_cuda and x.dtype == torch.float32 and x.dim() == 2 and x.is_contiguous()
            assert y.shape == x.shape and y.is_contiguous()
            self._keep.append((x, y))
            spec.append((x.data_ptr(), y.data_ptr(), x.shape[0], x.shape[1], x.shape[1], float(ss), float(sr), int(order)))
        opts = make_opts(order_default, "iir", t_c)
        if tol is not None:
            spec = self._adaptive_orders(spec, opts, float(tol), int(max_order))
        self.orders = [p[7] for p in spec]
        self.plan = bf_gp_batched_plan_create(spec, opts)
        self.ws_bytes = bf_gp_batched_plan_workspace(self.plan)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device="cuda")
        bf_gp_batched_plan_upload(self.plan, self.ws.data_ptr(), self.ws_bytes,
                                  torch.cuda.current_stream().cuda_stream)
        if autotune:
            bf_gp_batched_plan_tune(self.plan, self.ws.data_ptr(), self.ws_bytes,
                                    torch.cuda.current_stream().cuda_stream)
        self.engines = bf_gp_batched_plan_engines(self.plan, len(spec))

    @staticmethod
    def _adaptive_orders(spec, opts, tol, max_order):
        import torch
        probe = bf_gp_batched_plan_create([p[:7] + (0,) for p in spec], opts)
        try:
            need = bf_gp_batched_plan_stats_workspace(probe)
            ws = torch.empty(need, dtype=torch.uint8, device="cuda")
            _, R = bf_gp_batched_plane_stats(probe, len(spec), ws.data_ptr(), need,
                                             torch.cuda.current_stream().cuda_stream)
        finally:
            bf_gp_batched_plan_destroy(probe)
        out = []
        for p, r in zip(spec, R):
            n = bf_gp_order_for_tol(p[6], r, tol)
            n = max_order if n < 0 else min(n, max_order)
            lim = bf_gp_order_fp32_limit(p[5], p[6], r)
            out.append(p[:7] + (max(0, min(n, lim)),))
        return out

    def run(self, stream=None):
        import torch
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        bf_gp_batched(self.plan, self.ws.data_ptr(), self.ws_bytes, s)

    def run_persistent(self, stream=None):
        """The same forward (engine 0) as one persistent launch."""
        import torch
        s = torch.cuda.current_stream().cuda_stream if stream is None else stream
        bf_gp_batched_persistent(self.plan, self.ws.data_ptr(), self.ws_bytes, s)

    def status(self):
        import torch
        return bf_gp_get_device_status(self.ws.data_ptr(), torch.cuda.current_stream().cuda_stream)

    def counters(self):
        """The device counters of the last run, summed over the planes."""
        import torch
        return bf_gp_get_device_counters(self.ws.data_ptr(), torch.cuda.current_stream().cuda_stream)

    def __del__(self):
        try:
            if getattr(self, "plan", None):
                bf_gp_batched_plan_destroy(self.plan)
                self.plan = None
        except Exception:
            pass


BF_GP_NOALLOC_SCRATCH_BYTES = 32 << 20


def bf_gp_forward_noalloc(f_ptr, y_ptr, planes, H, W, pitch, sigma_s, sigma_r, opts, stream=0) -> None:
    """bf_gp_forward without a workspace: uses the library's own static device
    scratch (at most BF_GP_NOALLOC_SCRATCH_BYTES); see include/bf_gp.h."""
    _check(_load().bf_gp_forward_noalloc(_vp(f_ptr), _vp(y_ptr), int(planes), int(H), int(W), int(pitch),
                                         float(sigma_s), float(sigma_r), _op(opts), _vp(stream)),
           "bf_gp_forward_noalloc")


def bf_gp_host_workspace_size(planes, H, W, sigma_s, opts=None) -> int:
    n = ctypes.c_size_t(0)
    _check(_load().bf_gp_host_workspace_size(int(planes), int(H), int(W), float(sigma_s),
                                             ctypes.byref(opts) if opts is not None else None, ctypes.byref(n)),
           "bf_gp_host_workspace_size")
    return int(n.value)


def bf_gp_forward_host(f_host_ptr, y_host_ptr, planes, H, W, sigma_s, sigma_r, opts, ws_ptr, ws_bytes,
                       stream=0) -> None:
    _check(_load().bf_gp_forward_host(ctypes.c_void_p(int(f_host_ptr)), ctypes.c_void_p(int(y_host_ptr)),
                                      int(planes), int(H), int(W), float(sigma_s), float(sigma_r),
                                      ctypes.byref(opts) if opts is not None else None,
                                      ctypes.c_void_p(int(ws_ptr)), int(ws_bytes), ctypes.c_void_p(int(stream))),
           "bf_gp_forward_host")


BF_GP_NCOUNTERS = 4


def bf_gp_get_device_counters(ws_ptr, stream=0):
    """[pixels with Q <= 0, non-finite input values, planes beyond the FP32
    range, bounded waits that gave up] of the last call that used ws."""
    c = (ctypes.c_ulonglong * BF_GP_NCOUNTERS)()
    _check(_load().bf_gp_get_device_counters(_vp(ws_ptr), _vp(stream), c), "bf_gp_get_device_counters")
    return [int(v) for v in c]


def bf_gp_get_device_status(ws_ptr, stream=0) -> int:
    b = ctypes.c_uint32(0)
    _check(_load().bf_gp_get_device_status(ctypes.c_void_p(int(ws_ptr)), ctypes.c_void_p(int(stream)), ctypes.byref(b)),
           "bf_gp_get_device_status")
    return int(b.value)


def bf_gp_get_plane_stats(ws_ptr, plane, stream=0):
    tc, R = ctypes.c_double(0), ctypes.c_double(0)
    _check(_load().bf_gp_get_plane_stats(ctypes.c_void_p(int(ws_ptr)), int(plane), ctypes.c_void_p(int(stream)),
                                         ctypes.byref(tc), ctypes.byref(R)), "bf_gp_get_plane_stats")
    return tc.value, R.value


def bf_gp_order_for_tol(sigma_r, R, eps) -> int:
    return int(_load().bf_gp_order_for_tol(float(sigma_r), float(R), float(eps)))


def bf_gp_order_fp32_limit(sigma_s, sigma_r, R) -> int:
    return int(_load().bf_gp_order_fp32_limit(float(sigma_s), float(sigma_r), float(R)))


def bf_gp_version() -> int:
    return int(_load().bf_gp_version())


# ------------------------------------------------------- tensor wrapper

_ws_cache = {}


def workspace(nbytes: int, device=None):
    """A cached uint8 CUDA tensor of at least nbytes (256-byte aligned by the caching allocator)."""
    import torch
    dev = torch.device("cuda") if device is None else torch.device(device)
    key = (dev.type, dev.index if dev.index is not None else torch.cuda.current_device())
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=dev)
        _ws_cache[key] = buf
    return buf


def bilateral_gp(x, sigma_s: float, sigma_r: float, order: int = 20, spatial="auto", t_c=None,
                 fir_halfwidth: int = 0, out=None, ws=None, autotune=False):
    """Filter a float32 CUDA tensor [..., H, W] (leading dims are independent planes).

    Every plane gets its own centre (the plane mean unless t_c is given) and
    scale.  Runs asynchronously on torch's current stream.  With autotune, the
    engine (or FIR form) is the autotuner's choice for this shape class: the
    first call for a class times the candidates (and waits for them), later
    calls reuse the choice.
    """
    import torch
    if not (x.is_cuda and x.dtype == torch.float32):
        raise TypeError("bilateral_gp needs a float32 CUDA tensor")
    if x.dim() < 2:
        raise ValueError("need at least [H, W]")
    xc = x.contiguous()
    H, W = xc.shape[-2], xc.shape[-1]
    planes = max(1, xc.numel() // (H * W))
    opts = make_opts(order, spatial, t_c, fir_halfwidth)
    need = bf_gp_workspace_size(planes, H, W, sigma_s, opts)
    buf = ws if ws is not None else workspace(need, xc.device)
    if buf.numel() < need:
        raise ValueError(f"workspace too small: {buf.numel()} < {need}")
    y = torch.empty_like(xc) if out is None else out
    stream = torch.cuda.current_stream(xc.device).cuda_stream
    if autotune:
        bf_gp_autotune(xc.data_ptr(), y.data_ptr(), planes, H, W, W, sigma_s, sigma_r, opts, buf.data_ptr(),
                       buf.numel(), stream)
    bf_gp_forward(xc.data_ptr(), y.data_ptr(), planes, H, W, W, sigma_s, sigma_r, opts, buf.data_ptr(),
                  buf.numel(), stream)
    return y


def bf_gp_joint_workspace_size(planes, H, W, sigma_s, opts=None) -> int:
    n = ctypes.c_size_t(0)
    _check(_load().bf_gp_joint_workspace_size(int(planes), int(H), int(W), float(sigma_s), _op(opts),
                                              ctypes.byref(n)), "bf_gp_joint_workspace_size")
    return int(n.value)


def bf_gp_forward_joint(f_ptr, g_ptr, y_ptr, planes, H, W, pitch, sigma_s, sigma_r, opts, ws_ptr, ws_bytes,
                        stream=0) -> None:
    _check(_load().bf_gp_forward_joint(_vp(f_ptr), _vp(g_ptr), _vp(y_ptr), int(planes), int(H), int(W), int(pitch),
                                       float(sigma_s), float(sigma_r), _op(opts), _vp(ws_ptr), int(ws_bytes),
                                       _vp(stream)), "bf_gp_forward_joint")


def bilateral_gp_joint(f, g, sigma_s: float, sigma_r: float, order: int = 20, spatial="auto", t_c=None,
                       out=None, ws=None):
    """Joint (cross) bilateral filter of the float32 CUDA tensor f with range
    weights from the guide g (same shape [..., H, W]); see bf_gp_forward_joint."""
    import torch
    if not (f.is_cuda and g.is_cuda and f.dtype == torch.float32 and g.dtype == torch.float32):
        raise TypeError("bilateral_gp_joint needs float32 CUDA tensors")
    if f.shape != g.shape or f.dim() < 2:
        raise ValueError("f and g need the same shape [..., H, W]")
    fc, gc = f.contiguous(), g.contiguous()
    H, W = fc.shape[-2], fc.shape[-1]
    planes = max(1, fc.numel() // (H * W))
    opts = make_opts(order, spatial, t_c)
    need = bf_gp_joint_workspace_size(planes, H, W, sigma_s, opts)
    buf = ws if ws is not None else workspace(need, fc.device)
    if buf.numel() < need:
        raise ValueError(f"workspace too small: {buf.numel()} < {need}")
    y = torch.empty_like(fc) if out is None else out
    stream = torch.cuda.current_stream(fc.device).cuda_stream
    bf_gp_forward_joint(fc.data_ptr(), gc.data_ptr(), y.data_ptr(), planes, H, W, W, sigma_s, sigma_r, opts,
                        buf.data_ptr(), buf.numel(), stream)
    return y


# ------------------------------------------------------- autograd

def _autograd_function():
    import torch

    class BilateralGPFunction(torch.autograd.Function):
        """y = bilateral_gp(x, sigma_s, sigma_r, order) with the hand-written
        adjoint (bf_gp_backward) as its backward: gradients w.r.t. the image
        and sigma_r (summed over planes when sigma_r is shared)."""

        @staticmethod
        def forward(ctx, x, sigma_r, sigma_s, order, spatial, t_c):
            xc = x.contiguous()
            H, W = xc.shape[-2], xc.shape[-1]
            planes = max(1, xc.numel() // (H * W))
            sr = float(sigma_r)
            opts = make_opts(order, spatial, t_c)
            need = bf_gp_workspace_size(planes, H, W, sigma_s, opts)
            ws = workspace(need, xc.device)
            y = torch.empty_like(xc)
            saved = torch.empty((planes, 4, H, W), dtype=torch.float32, device=xc.device)
            stream = torch.cuda.current_stream(xc.device).cuda_stream
            bf_gp_forward_train(xc.data_ptr(), y.data_ptr(), saved.data_ptr(), planes, H, W, W, sigma_s, sr, opts,
                                ws.data_ptr(), ws.numel(), stream)
            ctx.save_for_backward(xc, saved)
            ctx.cfg = (planes, H, W, float(sigma_s), sr, int(order), spatial, t_c)
            return y

        @staticmethod
        def backward(ctx, gy):
            xc, saved = ctx.saved_tensors
            planes, H, W, ss, sr, order, spatial, t_c = ctx.cfg
            opts = make_opts(order, spatial, t_c)
            need = bf_gp_workspace_size(planes, H, W, ss, opts)
            ws = workspace(need, xc.device)
            gyc = gy.contiguous()
            gx = torch.empty_like(xc)
            gsr = torch.empty(planes, dtype=torch.float32, device=xc.device)
            stream = torch.cuda.current_stream(xc.device).cuda_stream
            bf_gp_backward(xc.data_ptr(), gyc.data_ptr(), saved.data_ptr(), gx.data_ptr(), gsr.data_ptr(), planes, H,
                           W, W, ss, sr, opts, ws.data_ptr(), ws.numel(), stream)
            gsig = gsr.sum() if ctx.needs_input_grad[1] else None
            return gx, gsig, None, None, None, None

    return BilateralGPFunction


_fn = None


def bilateral_gp_autograd(x, sigma_s: float, sigma_r, order: int = 20, spatial="auto", t_c=None):
    """Differentiable filter: gradients flow to x and (if it is a tensor) sigma_r."""
    global _fn
    if _fn is None:
        _fn = _autograd_function()
    return _fn.apply(x, sigma_r, sigma_s, order, spatial, t_c)
