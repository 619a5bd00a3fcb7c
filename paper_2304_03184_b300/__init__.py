"""Python binding of libinvr.so, the sm_103a hot path of Instant-NVR's deformed hash-grid
radiance field (warp -> hash encoding -> MLPs -> volume rendering, forward and backward).

Argument marshalling only: every step runs in the library's CUDA kernels.  Tensors are
torch CUDA tensors (device memory and streams); the calls are enqueued on the current
torch stream.  There is no CPU fallback: if libinvr.so is missing the first call raises.

The C names (invr_*) are exported as module functions taking ctypes arguments; the
classes Context, Field, Graph, View and the functions render_rays / train_step /
forward_train / backward / ray_samples / warp_points / encode_points / mlp_points /
query_points wrap them for torch tensors.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libinvr.so")

INVR_FP32, INVR_MLP_FP16, INVR_MLP_BF16 = 0, 1, 2
_STATUS = {0: "INVR_OK", -1: "INVR_E_ARG", -2: "INVR_E_OOM", -3: "INVR_E_CUDA", -4: "INVR_E_TIMEOUT",
           -5: "INVR_E_NONFINITE", -6: "INVR_E_STATE"}


# ----------------------------------------------------------------------- C structs
class invr_field_desc(C.Structure):
    _fields_ = [("L", C.c_int), ("log2_T", C.c_int), ("F", C.c_int), ("N_min", C.c_int),
                ("growth", C.c_double), ("mlp_in", C.c_int), ("mlp_hidden", C.c_int),
                ("geo_out", C.c_int), ("col_hidden", C.c_int), ("prec", C.c_int)]


class invr_graph_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("K", C.c_int), ("radius", C.c_float), ("n_frames", C.c_int)]


class invr_field_view(C.Structure):
    _fields_ = [("field", C.c_void_p), ("graph", C.c_void_p), ("frame", C.c_int),
                ("rigid_dq", C.POINTER(C.c_float)), ("occupancy_dev", C.c_void_p),
                ("deform", C.c_void_p), ("pose_dev", C.c_void_p)]


class invr_deform_desc(C.Structure):
    _fields_ = [("L", C.c_int), ("log2_T", C.c_int), ("F", C.c_int), ("N_min", C.c_int), ("growth", C.c_double),
                ("pose_dim", C.c_int), ("hidden", C.c_int), ("n_hidden", C.c_int), ("prec", C.c_int)]


class invr_render_args(C.Structure):
    _fields_ = [("n_rays", C.c_int64), ("o_dev", C.c_void_p), ("d_dev", C.c_void_p),
                ("n_samples", C.c_int), ("t_eps", C.c_float), ("n_views", C.c_int),
                ("views", C.POINTER(invr_field_view)), ("rgba_dev", C.c_void_p), ("depth_dev", C.c_void_p)]


class invr_train_args(C.Structure):
    _fields_ = [("n_batches", C.c_int), ("batches", C.POINTER(invr_render_args)),
                ("targets_dev", C.c_void_p), ("huber_delta", C.c_float), ("lr", C.c_float),
                ("beta1", C.c_float), ("beta2", C.c_float), ("adam_eps", C.c_float),
                ("loss_dev", C.c_void_p), ("loss", C.c_int), ("masks_dev", C.c_void_p),
                ("depths_dev", C.c_void_p), ("depth_weight", C.c_float)]


_VP, _I64, _I, _F = C.c_void_p, C.c_int64, C.c_int, C.c_float
_SIGNATURES = {
    "invr_ctx_create": [C.POINTER(C.c_void_p), _I],
    "invr_ctx_destroy": [_VP],
    "invr_ctx_reserve": [_VP, _I64, _I],
    "invr_ctx_sync": [_VP, _VP],
    "invr_last_error_detail": [_VP, C.c_char_p, C.c_size_t],
    "invr_field_create": [_VP, C.POINTER(invr_field_desc), C.POINTER(C.c_void_p)],
    "invr_field_destroy": [_VP],
    "invr_field_set_params": [_VP, _VP, _VP, _VP],
    "invr_field_get_params": [_VP, _VP, _VP, _VP, _VP, C.POINTER(C.c_int64), _VP],
    "invr_field_get_grads": [_VP, _VP, _VP, _VP],
    "invr_field_zero_grads": [_VP, _VP],
    "invr_graph_create": [_VP, C.POINTER(invr_graph_desc), _VP, C.POINTER(C.c_void_p)],
    "invr_graph_set_pose": [_VP, _I, _VP, _VP, _VP],
    "invr_graph_destroy": [_VP],
    "invr_render_rays": [_VP, C.POINTER(invr_render_args), _VP],
    "invr_train_step": [_VP, C.POINTER(invr_train_args), _VP],
    "invr_field_forward_train": [_VP, C.POINTER(invr_train_args), _VP],
    "invr_field_backward": [_VP, C.POINTER(invr_train_args), _F, _VP],
    "invr_field_adam": [_VP, _F, _F, _F, _F, _VP],
    "invr_ray_samples": [_VP, _I64, _VP, _VP, _I, _VP, _VP, _VP, _VP, _VP],
    "invr_warp_points": [_VP, C.POINTER(invr_field_view), _I64, _VP, _VP, _VP, _VP],
    "invr_encode_points": [_VP, _VP, _I64, _VP, _VP, _VP, _VP],
    "invr_mlp_points": [_VP, _VP, _I64, _VP, _VP, _VP],
    "invr_query_points": [_VP, C.POINTER(invr_field_view), _I64, _VP, _VP, _VP],
    "invr_ctx_enable_timing": [_VP, _I],
    "invr_ctx_timing": [_VP, C.POINTER(C.c_char_p), C.POINTER(C.c_double), C.POINTER(C.c_int64), _I],
    "invr_query_points_noalloc": [_VP, C.POINTER(invr_field_view), _I64, _VP, _VP, _VP],
    "invr_render_rays_joint": [_VP, C.POINTER(invr_render_args), _VP],
    "invr_deform_create": [_VP, C.POINTER(invr_deform_desc), C.POINTER(C.c_void_p)],
    "invr_deform_destroy": [_VP],
    "invr_deform_set_params": [_VP, _VP, _VP, _VP],
    "invr_deform_get_params": [_VP, _VP, _VP, _VP],
    "invr_deform_get_grads": [_VP, _VP, _VP, _VP],
    "invr_deform_zero_grads": [_VP, _VP],
    "invr_occupancy_update": [_VP, C.POINTER(invr_field_view), C.c_float, C.c_float, _VP, _VP, _VP],
    "invr_graph_enable_lut": [_VP, C.c_int, _VP],
    "invr_graph_disable_lut": [_VP],
    "invr_graph_get_lut": [_VP, C.c_int, _VP, _VP, _VP],
    "invr_probe_l2_read": [_VP, _VP, _I64, C.c_int, _VP, _VP],
    "invr_probe_l2_atomic": [_VP, _VP, _I64, C.c_int, _I64, _VP],
    "invr_probe_l2_gather": [_VP, _VP, _I64, C.c_int, _I64, _VP, _VP],
    "invr_ctx_autotune": [_VP, C.POINTER(invr_train_args), _VP],
    "invr_ctx_get_tune": [_VP, C.POINTER(C.c_int)],
    "invr_ctx_set_tune": [_VP, C.POINTER(C.c_int)],
    "invr_field_copy_params": [_VP, _VP, _VP],
    "invr_ctx_set_wait_limit": [_VP, C.c_uint32],
}

_lib_handle = None


def lib() -> C.CDLL:
    """Load libinvr.so (built by paper_2304_03184_b300/build.py); raise if it is missing."""
    global _lib_handle
    if _lib_handle is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python paper_2304_03184_b300/build.py`")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int
        L.invr_status_string.argtypes = [C.c_int]
        L.invr_status_string.restype = C.c_char_p
        L.invr_field_weight_count.argtypes = [C.POINTER(invr_field_desc)]
        L.invr_field_weight_count.restype = C.c_int64
        _lib_handle = L
    return _lib_handle


def exported_symbols() -> List[str]:
    return sorted(list(_SIGNATURES) + ["invr_status_string", "invr_field_weight_count"])


class InvrError(RuntimeError):
    pass


def _check(status: int, ctx_handle=None):
    if status != 0:
        detail = ""
        if ctx_handle:
            buf = C.create_string_buffer(512)
            lib().invr_last_error_detail(ctx_handle, buf, 512)
            detail = buf.value.decode(errors="replace")
        raise InvrError(f"{_STATUS.get(status, status)} ({lib().invr_status_string(status).decode()}): {detail}")


def _torch():
    import torch
    return torch


def _stream():
    return _torch().cuda.current_stream().cuda_stream


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    torch = _torch()
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    return t.data_ptr()


# ----------------------------------------------------------------------- handles
class Context:
    def __init__(self, device: int = 0):
        h = C.c_void_p()
        _check(lib().invr_ctx_create(C.byref(h), device))
        self.h, self.device = h, device

    def reserve(self, max_rays: int, max_samples: int):
        _check(lib().invr_ctx_reserve(self.h, max_rays, max_samples), self.h)

    def sync(self):
        _check(lib().invr_ctx_sync(self.h, _stream()), self.h)

    def autotune(self, tb: "TrainBatches"):
        """Pick the launch shapes for this workload (times forward + backward candidates)."""
        _check(lib().invr_ctx_autotune(self.h, C.byref(tb.args), _stream()), self.h)
        return self.tune()

    def set_wait_limit(self, polls: int):
        """Polls per bounded device wait (0: every wait gives up at once; default 2^22)."""
        _check(lib().invr_ctx_set_wait_limit(self.h, polls), self.h)

    TUNE_KEYS = ("warp_ctas_per_sm", "encode_ctas_per_sm", "encode_bwd_ctas_per_sm", "agg_res", "fused", "chunk")

    def tune(self):
        out = (C.c_int * len(self.TUNE_KEYS))()
        _check(lib().invr_ctx_get_tune(self.h, out), self.h)
        return dict(zip(self.TUNE_KEYS, list(out)))

    def set_tune(self, tune: dict):
        """Set the launch shapes (a dict as returned by tune() / autotune())."""
        arr = (C.c_int * len(self.TUNE_KEYS))(*[int(tune[k]) for k in self.TUNE_KEYS])
        _check(lib().invr_ctx_set_tune(self.h, arr), self.h)

    def enable_timing(self, on: bool = True):
        _check(lib().invr_ctx_enable_timing(self.h, 1 if on else 0), self.h)

    def timing(self):
        """{kernel name: (total ms, launches)} since enable_timing (synchronises)."""
        n = 64
        names = (C.c_char_p * n)()
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        k = lib().invr_ctx_timing(self.h, names, ms, cnt, n)
        if k < 0:
            _check(k, self.h)
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(k)}

    def close(self):
        if self.h:
            lib().invr_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def field_desc(L, log2_T, F=2, N_min=16, growth=1.5, hidden=64, geo_out=16, col_hidden=64, prec=INVR_FP32):
    return invr_field_desc(L, log2_T, F, N_min, float(growth), L * F, hidden, geo_out, col_hidden, prec)


class Field:
    """Hash tables + MLP weights + gradients + Adam state of one canonical field."""

    def __init__(self, ctx: Context, desc: invr_field_desc):
        h = C.c_void_p()
        _check(lib().invr_field_create(ctx.h, C.byref(desc), C.byref(h)), ctx.h)
        self.ctx, self.desc, self.h = ctx, desc, h
        self.n_tables = desc.L * (1 << desc.log2_T) * desc.F
        self.n_weights = lib().invr_field_weight_count(C.byref(desc))

    @classmethod
    def from_synth(cls, ctx: Context, fp, prec: int = INVR_FP32):
        d = fp.desc
        f = cls(ctx, field_desc(d.L, d.log2_T, d.F, d.N_min, d.growth, d.hidden, d.geo_out, d.col_hidden, prec))
        torch = _torch()
        f.set_params(torch.from_numpy(fp.tables).cuda(), torch.from_numpy(fp.weights).cuda())
        return f

    def set_params(self, tables=None, weights=None):
        _check(lib().invr_field_set_params(self.h, _ptr(tables), _ptr(weights), _stream()), self.ctx.h)

    def get_params(self):
        torch = _torch()
        t = torch.empty(self.n_tables, device="cuda")
        w = torch.empty(self.n_weights, device="cuda")
        m = torch.empty(self.n_tables + self.n_weights, device="cuda")
        v = torch.empty_like(m)
        step = C.c_int64()
        _check(lib().invr_field_get_params(self.h, _ptr(t), _ptr(w), _ptr(m), _ptr(v), C.byref(step), _stream()),
               self.ctx.h)
        return t, w, m, v, step.value

    def get_grads(self):
        torch = _torch()
        gt = torch.empty(self.n_tables, device="cuda")
        gw = torch.empty(self.n_weights, device="cuda")
        _check(lib().invr_field_get_grads(self.h, _ptr(gt), _ptr(gw), _stream()), self.ctx.h)
        return gt, gw

    def copy_params_from(self, src: "Field"):
        """Snapshot src's tables and weights into this field (enqueued on the current stream)."""
        _check(lib().invr_field_copy_params(self.h, src.h, _stream()), self.ctx.h)

    def zero_grads(self):
        _check(lib().invr_field_zero_grads(self.h, _stream()), self.ctx.h)

    def adam(self, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15):
        _check(lib().invr_field_adam(self.h, lr, beta1, beta2, eps, _stream()), self.ctx.h)

    def close(self):
        if self.h:
            lib().invr_field_destroy(self.h)
            self.h = None


class Graph:
    """Deformation-graph nodes with per-frame poses (and their nearest-node grids)."""

    def __init__(self, ctx: Context, n_nodes: int, K: int, radius: float = 0.1, n_frames: int = 1, x_canon=None):
        h = C.c_void_p()
        desc = invr_graph_desc(n_nodes, K, radius, n_frames)
        _check(lib().invr_graph_create(ctx.h, C.byref(desc), _ptr(x_canon), C.byref(h)), ctx.h)
        self.ctx, self.desc, self.h = ctx, desc, h

    def set_pose(self, frame: int, dq, x_live):
        _check(lib().invr_graph_set_pose(self.h, frame, _ptr(dq), _ptr(x_live), _stream()), self.ctx.h)

    def enable_lut(self, resolution: int = 512):
        """Look-up-table neighbour search (invr_graph_enable_lut)."""
        _check(lib().invr_graph_enable_lut(self.h, resolution, _stream()), self.ctx.h)
        self.lut_res = resolution

    def disable_lut(self):
        _check(lib().invr_graph_disable_lut(self.h), self.ctx.h)
        self.lut_res = 0

    def get_lut(self, frame: int = 0):
        """Device copies of the canonical KNN field ([G^3][K] node ids, int16 holding uint16)
        and of the frame's live index field ([G^3], int32 holding uint32; -1 = none)."""
        torch = _torch()
        G = self.lut_res
        canon = torch.empty((G ** 3, self.desc.K), dtype=torch.int16, device="cuda")
        live = torch.empty(G ** 3, dtype=torch.int32, device="cuda")
        _check(lib().invr_graph_get_lut(self.h, frame, _ptr(canon), _ptr(live), _stream()), self.ctx.h)
        return canon, live

    def close(self):
        if self.h:
            lib().invr_graph_destroy(self.h)
            self.h = None


class Deform:
    """A pose-conditioned deformation net (invr_deform): its hash tables, weights, gradients
    and Adam state on the device."""

    def __init__(self, ctx: Context, L=16, log2_T=19, F=2, N_min=16, growth=1.38, pose_dim=72, hidden=128,
                 n_hidden=4, prec: int = INVR_FP32):
        h = C.c_void_p()
        desc = invr_deform_desc(L, log2_T, F, N_min, growth, pose_dim, hidden, n_hidden, prec)
        _check(lib().invr_deform_create(ctx.h, C.byref(desc), C.byref(h)), ctx.h)
        self.ctx, self.desc, self.h = ctx, desc, h
        self.n_tab = L * (1 << log2_T) * F
        self.n_w = hidden * (L * F + pose_dim) + (n_hidden - 1) * hidden * hidden + 3 * hidden

    @classmethod
    def from_synth(cls, ctx: Context, dp, prec: int = INVR_FP32):
        torch = _torch()
        d = dp.desc
        net = cls(ctx, d.L, d.log2_T, d.F, d.N_min, d.growth, d.pose_dim, d.hidden, d.n_hidden, prec)
        net.set_params(torch.from_numpy(dp.tables.reshape(-1)).cuda(), torch.from_numpy(dp.weights).cuda())
        return net

    def set_params(self, tables, weights):
        _check(lib().invr_deform_set_params(self.h, _ptr(tables), _ptr(weights), _stream()), self.ctx.h)

    def get_params(self):
        torch = _torch()
        t = torch.empty(self.n_tab, device="cuda")
        w = torch.empty(self.n_w, device="cuda")
        _check(lib().invr_deform_get_params(self.h, _ptr(t), _ptr(w), _stream()), self.ctx.h)
        return t, w

    def get_grads(self):
        torch = _torch()
        t = torch.empty(self.n_tab, device="cuda")
        w = torch.empty(self.n_w, device="cuda")
        _check(lib().invr_deform_get_grads(self.h, _ptr(t), _ptr(w), _stream()), self.ctx.h)
        return t, w

    def zero_grads(self):
        _check(lib().invr_deform_zero_grads(self.h, _stream()), self.ctx.h)

    def close(self):
        if self.h:
            lib().invr_deform_destroy(self.h)
            self.h = None


class View:
    """A field seen in one frame: through `graph` at `frame`, or through rigid_dq; the human
    view may carry a deformation net and the frame's pose (a CUDA float32 tensor)."""

    def __init__(self, field: Field, graph: Optional[Graph] = None, frame: int = 0, rigid_dq=None, occupancy=None,
                 deform: Optional[Deform] = None, pose=None):
        self.field, self.graph, self.frame, self.occupancy = field, graph, frame, occupancy
        self.deform, self.pose = deform, pose
        self._dq = None
        if rigid_dq is not None:
            import numpy as np
            self._dq = (C.c_float * 8)(*[float(x) for x in np.asarray(rigid_dq).reshape(-1)])

    def c(self) -> invr_field_view:
        return invr_field_view(self.field.h, self.graph.h if self.graph else None, self.frame,
                               C.cast(self._dq, C.POINTER(C.c_float)) if self._dq is not None else None,
                               _ptr(self.occupancy), self.deform.h if self.deform else None, _ptr(self.pose))


def _views_array(views: Sequence[View]):
    arr = (invr_field_view * len(views))(*[v.c() for v in views])
    return arr


# ----------------------------------------------------------------------- calls
def render_rays(ctx: Context, o, d, n_samples: int, t_eps: float, views: Sequence[View], joint: bool = False):
    """Render R rays (o, d: [3][R] CUDA float32) through 1 or 2 views -> (rgba [4][R], depth [R]).
    Two views are composed by depth (the nearer image over the farther) or, with joint=True,
    composited together per sample (invr_render_rays_joint)."""
    torch = _torch()
    R = o.shape[1]
    rgba = torch.empty((4, R), device=o.device)
    depth = torch.empty(R, device=o.device)
    arr = _views_array(views)
    args = invr_render_args(R, _ptr(o), _ptr(d), n_samples, t_eps, len(views), arr, _ptr(rgba), _ptr(depth))
    fn = lib().invr_render_rays_joint if joint else lib().invr_render_rays
    _check(fn(ctx.h, C.byref(args), _stream()), ctx.h)
    return rgba, depth


OCC_RES = 128


def occupancy_update(ctx: Context, view: View, density, bits, decay: float = 0.95, threshold: float = 0.01):
    """invr_occupancy_update: density [128^3] float32 (updated in place) and bits [65536]
    int32 / uint32 words (written) on the device."""
    cv = view.c()
    _check(lib().invr_occupancy_update(ctx.h, C.byref(cv), decay, threshold, _ptr(density), _ptr(bits), _stream()),
           ctx.h)
    return density, bits


INVR_LOSS_HUBER, INVR_LOSS_PAPER = 0, 1
LOSSES = {"huber": INVR_LOSS_HUBER, "paper": INVR_LOSS_PAPER}


class TrainBatches:
    """Key-frame ray batches of one training call: each batch = (o, d, view, target) or,
    for the paper's losses, (o, d, view, target, mask, depth) with mask [R] (or None for
    M = 1) and sensor depth [R].  loss = "huber" or "paper" (see invr_loss)."""

    def __init__(self, batches, n_samples: int, t_eps: float = 1e-4, huber_delta: float = 0.1, lr: float = 1e-2,
                 beta1: float = 0.9, beta2: float = 0.99, adam_eps: float = 1e-15, keep_outputs: bool = False,
                 loss: str = "huber", depth_weight: float = 1.0):
        torch = _torch()
        self.batches = [tuple(b) for b in batches]
        # each batch's [3][R_b] target block, back to back
        self.targets = torch.cat([b[3].reshape(-1) for b in self.batches]).contiguous()
        self.loss = torch.zeros(1, device=self.targets.device)
        self.masks = self.depths = None
        kind = LOSSES[loss]
        if kind == INVR_LOSS_PAPER:
            if any(len(b) < 6 or b[5] is None for b in self.batches):
                raise ValueError("the paper's depth loss needs every batch's sensor depth")
            self.depths = torch.cat([b[5].reshape(-1) for b in self.batches]).contiguous()
            if any(b[4] is not None for b in self.batches):
                self.masks = torch.cat([b[4].reshape(-1) if b[4] is not None else
                                        torch.ones(b[0].shape[1], device=b[0].device) for b in self.batches])
        self._views = [_views_array([b[2]]) for b in self.batches]
        self.outputs = []
        rargs = []
        for (o, d, view, *_), va in zip(self.batches, self._views):
            R = o.shape[1]
            rgba = torch.empty((4, R), device=o.device) if keep_outputs else None
            depth = torch.empty(R, device=o.device) if keep_outputs else None
            self.outputs.append((rgba, depth))
            rargs.append(invr_render_args(R, _ptr(o), _ptr(d), n_samples, t_eps, 1, va, _ptr(rgba), _ptr(depth)))
        self._rargs = (invr_render_args * len(rargs))(*rargs)
        self.args = invr_train_args(len(rargs), self._rargs, _ptr(self.targets), huber_delta, lr, beta1, beta2,
                                    adam_eps, _ptr(self.loss), kind, _ptr(self.masks), _ptr(self.depths),
                                    depth_weight)
        self.ctx = None


class TrainGraph:
    """A training step captured once into a CUDA graph and replayed: every batch of the step
    (key frames x fields) goes through one launch per stage, and the whole step is one graph
    launch.  The context must have been sized with Context.reserve first."""

    def __init__(self, ctx: Context, tb: TrainBatches, warmup: int = 2):
        torch = _torch()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(warmup):
                train_step(ctx, tb)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            train_step(ctx, tb)
        self.ctx, self.tb = ctx, tb

    def replay(self):
        self.graph.replay()
        return self.tb.loss


def train_step(ctx: Context, tb: TrainBatches):
    """Forward + Huber loss + backward + Adam on every field of the batches; returns loss tensor."""
    _check(lib().invr_train_step(ctx.h, C.byref(tb.args), _stream()), ctx.h)
    return tb.loss


def forward_train(ctx: Context, tb: TrainBatches):
    _check(lib().invr_field_forward_train(ctx.h, C.byref(tb.args), _stream()), ctx.h)
    return tb.loss


def backward(ctx: Context, tb: TrainBatches, grad_scale: float = 1.0):
    _check(lib().invr_field_backward(ctx.h, C.byref(tb.args), grad_scale, _stream()), ctx.h)


def ray_samples(ctx: Context, o, d, n_samples: int, occupancy=None):
    torch = _torch()
    R = o.shape[1]
    count = torch.zeros(R, dtype=torch.int32, device=o.device)
    t = torch.zeros((R, n_samples), device=o.device)
    p = torch.zeros((3, R, n_samples), device=o.device)
    _check(lib().invr_ray_samples(ctx.h, R, _ptr(o), _ptr(d), n_samples, _ptr(occupancy), _ptr(count), _ptr(t),
                                  _ptr(p), _stream()), ctx.h)
    return count, t, p


def warp_points(ctx: Context, view: View, p, with_ids: bool = False):
    torch = _torch()
    n = p.shape[1]
    vc = torch.empty((3, n), device=p.device)
    ids = None
    if with_ids and view.graph is not None:
        ids = torch.full((view.graph.desc.K, n), -1, dtype=torch.int32, device=p.device)
    cv = view.c()
    _check(lib().invr_warp_points(ctx.h, C.byref(cv), n, _ptr(p), _ptr(vc), _ptr(ids), _stream()), ctx.h)
    return (vc, ids) if with_ids else vc


def encode_points(ctx: Context, field: Field, x, with_index: bool = False):
    torch = _torch()
    n = x.shape[1]
    feat = torch.empty((field.desc.mlp_in, n), device=x.device)
    idx = torch.empty((field.desc.L * 8, n), dtype=torch.int32, device=x.device) if with_index else None
    _check(lib().invr_encode_points(ctx.h, field.h, n, _ptr(x), _ptr(feat), _ptr(idx), _stream()), ctx.h)
    return (feat, idx) if with_index else feat


def mlp_points(ctx: Context, field: Field, feat):
    torch = _torch()
    n = feat.shape[1]
    out = torch.empty((4, n), device=feat.device)
    _check(lib().invr_mlp_points(ctx.h, field.h, n, _ptr(feat), _ptr(out), _stream()), ctx.h)
    return out


def query_points(ctx: Context, view: View, p):
    torch = _torch()
    n = p.shape[1]
    out = torch.empty((4, n), device=p.device)
    cv = view.c()
    _check(lib().invr_query_points(ctx.h, C.byref(cv), n, _ptr(p), _ptr(out), _stream()), ctx.h)
    return out


NOALLOC_MAX_POINTS = 65536


def query_points_noalloc(ctx: Context, view: View, p, out=None):
    """invr_query_points_noalloc: query without any device allocation inside the library
    (scratch in a fixed 9.2 MB device array, at most NOALLOC_MAX_POINTS points per call; calls
    share that array, so calls that overlap on the GPU must be serialised by the caller)."""
    torch = _torch()
    n = p.shape[1]
    if out is None:
        out = torch.empty((4, n), device=p.device)
    cv = view.c()
    _check(lib().invr_query_points_noalloc(ctx.h, C.byref(cv), n, _ptr(p), _ptr(out), _stream()), ctx.h)
    return out


def _autograd():
    torch = _torch()

    class FieldRenderLoss(torch.autograd.Function):
        """Huber render loss of one field's batches as a function of (tables, weights).

        forward copies the tensors into the field and runs invr_field_forward_train;
        backward runs invr_field_backward (recomputing MLP activations per sample and
        scatter-adding hash-table gradients) and returns the gradients."""

        @staticmethod
        def forward(actx, tables, weights, ctx: Context, field: Field, tb: TrainBatches):
            field.set_params(tables, weights)
            loss = forward_train(ctx, tb).clone()
            actx.saved = (ctx, field, tb)
            return loss

        @staticmethod
        def backward(actx, g):
            ctx, field, tb = actx.saved
            field.zero_grads()
            backward(ctx, tb, float(g.reshape(-1)[0].item()))
            gt, gw = field.get_grads()
            return gt, gw, None, None, None

    return FieldRenderLoss


def field_render_loss(tables, weights, ctx: Context, field: Field, tb: TrainBatches):
    """Differentiable Huber render loss (torch.autograd) of one field's training batches."""
    return _autograd().apply(tables, weights, ctx, field, tb)


def probe_l2_read(ctx: Context, buf, passes: int, sink):
    """invr_probe_l2_read: `passes` 16-byte coalesced reads of every float of `buf` (a CUDA
    float32 tensor meant to stay resident in L2); the caller times it with events."""
    _check(lib().invr_probe_l2_read(ctx.h, _ptr(buf), buf.numel(), passes, _ptr(sink), _stream()), ctx.h)


def probe_l2_atomic(ctx: Context, table, width: int, n_ops: int):
    """invr_probe_l2_atomic: n_ops float4 (width 4) or float2 (width 2) atomic adds at
    pseudo-random entries of `table` (a CUDA float32 tensor)."""
    _check(lib().invr_probe_l2_atomic(ctx.h, _ptr(table), table.numel(), width, n_ops, _stream()), ctx.h)


def probe_l2_gather(ctx: Context, table, width: int, n_ops: int, sink):
    """invr_probe_l2_gather: n_ops 32-byte (width 8), float4 (width 4) or float2 (width 2) loads
    at pseudo-random entries of `table` (a CUDA float32 tensor)."""
    _check(lib().invr_probe_l2_gather(ctx.h, _ptr(table), table.numel(), width, n_ops, _ptr(sink), _stream()), ctx.h)
