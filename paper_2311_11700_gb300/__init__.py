"""Python binding of libgsr.so, the sm_103a differentiable RGB-D Gaussian
splatting renderer of GS-SLAM (arXiv 2311.11700).

The binding only marshals arguments: every step of the renderer runs in the
CUDA kernels behind the C ABI declared in include/gsr.h.  PyTorch provides
device memory (tensors), the current stream and autograd.  There is no CPU
fallback: if libgsr.so is missing or fails to load, the first call raises.

Functions with the C ABI's names take the same arguments as the C functions,
with tensors in place of device pointers:

    gs_render_forward(ctx, scenes, views, workspace, max_pairs, out)
    gs_loss_l1(ctx, views, rendered, target_rgb, target_depth, w_c, w_d, loss, dL_dout)
    gs_render_backward(ctx, scenes, views, workspace, max_pairs, dL_dout, grads, dL_dtwist, pose_mode)
    gs_pose_grad(ctx, scenes, views, workspace, max_pairs, dL_dout, dL_dtwist, pose_mode)
    gs_workspace_query / gs_workspace_layout / gs_workspace_status

`Renderer` wraps a context with workspace management (capacity growth), and
`RenderRGBD` is the torch.autograd.Function of the forward/backward pair.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsr.so")

MAX_VIEWS = 32
MAX_SCENES = 32

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_TIMEOUT, GS_ERR_CUDA, GS_ERR_UNSUPPORTED, GS_ERR_STATE = range(7)
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_TIMEOUT", 4: "GS_ERR_CUDA",
                5: "GS_ERR_UNSUPPORTED", 6: "GS_ERR_STATE"}

PARAM_KEYS = ("mean", "log_scale", "quat", "opacity_logit", "sh")


class GsrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


# ----------------------------------------------------------------------------
# ctypes mirror of include/gsr.h
# ----------------------------------------------------------------------------
_fp = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p


class gs_scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mean", _vp), ("log_scale", _vp), ("quat", _vp), ("opacity_logit", _vp), ("sh", _vp),
                ("mask", _vp)]


class gs_grads(ctypes.Structure):
    _fields_ = [("mean", _vp), ("log_scale", _vp), ("quat", _vp), ("opacity_logit", _vp), ("sh", _vp),
                ("vs_grad_norm", _vp), ("vs_count", _vp)]


class gs_densify_params(ctypes.Structure):
    _fields_ = [("grad_thr", ctypes.c_float), ("scale_thr", ctypes.c_float), ("split_scale", ctypes.c_float),
                ("reserved", ctypes.c_int32)]


class gs_view(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("scene", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("z_near", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("T_cw", ctypes.c_float * 12), ("T_cw_dev", _vp),
                ("pixel_mask", _vp)]


class gs_images(ctypes.Structure):
    _fields_ = [("color", _vp), ("depth", _vp), ("acc", _vp)]


class gs_layout(ctypes.Structure):
    _fields_ = [("rec", ctypes.c_int64), ("rect", ctypes.c_int64), ("ntiles", ctypes.c_int64),
                ("dkey", ctypes.c_int64), ("ranges", ctypes.c_int64), ("pair_val", ctypes.c_int64),
                ("header", ctypes.c_int64), ("n_splats", ctypes.c_int64), ("n_tiles", ctypes.c_int64),
                ("splat_off", ctypes.c_int64 * MAX_VIEWS), ("tile_off", ctypes.c_int64 * MAX_VIEWS),
                ("order", ctypes.c_int64)]


class gs_expand_params(ctypes.Structure):
    _fields_ = [("tau_T", ctypes.c_float), ("tau_D", ctypes.c_float), ("eta", ctypes.c_float),
                ("gamma", ctypes.c_float), ("init_opacity", ctypes.c_float), ("density", ctypes.c_float),
                ("prune_opacity", ctypes.c_float), ("flags", ctypes.c_int32)]


class gs_scene_out(ctypes.Structure):
    _fields_ = [("mean", _vp), ("log_scale", _vp), ("quat", _vp), ("opacity_logit", _vp), ("sh", _vp)]


GS_EXPAND_ADD, GS_EXPAND_DELETE, GS_EXPAND_PRUNE, GS_EXPAND_CHECKERBOARD = 1, 2, 4, 8

STAGES = ("setup", "project", "emit", "tile_sort", "composite_fwd", "loss", "composite_bwd", "project_bwd",
          "composite_step", "tile_scan", "sort_short", "sort_long")


class gs_tune_result(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int), ("tile_h", ctypes.c_int), ("strip_fwd", ctypes.c_int),
                ("strip_bwd", ctypes.c_int), ("binning", ctypes.c_int), ("ms_fwd", ctypes.c_float),
                ("ms_bwd", ctypes.c_float), ("timed", ctypes.c_int)]


class gs_timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 16), ("launches", ctypes.c_int64 * 16), ("calls", ctypes.c_int64)]


# exported entry points and their argument types
ABI = {
    "gs_ctx_create": ([ctypes.POINTER(_vp), ctypes.c_int], ctypes.c_int),
    "gs_ctx_destroy": ([_vp], None),
    "gs_last_error": ([_vp], ctypes.c_char_p),
    "gs_ctx_set_tiling": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "gs_ctx_set_strip": ([_vp, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "gs_ctx_set_binning": ([_vp, ctypes.c_int], ctypes.c_int),
    "gs_ctx_set_grad_mode": ([_vp, ctypes.c_int], ctypes.c_int),
    "gs_ctx_set_compact": ([_vp, ctypes.c_int], ctypes.c_int),
    "gs_autotune_workspace_query": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int64,
                                     ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "gs_autotune": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int64, _vp, _vp,
                     _vp, ctypes.c_int, ctypes.c_int, _vp, _vp], ctypes.c_int),
    "gs_autotune_step_l1": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int64,
                             _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp, ctypes.c_int,
                             ctypes.c_int, ctypes.c_int, _vp, _vp], ctypes.c_int),
    "gs_autotune_save": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "gs_densify_workspace_query": ([_vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "gs_outlier_mask_workspace_query": ([_vp, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "gs_outlier_mask": ([_vp, _vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, _vp,
                         _vp, ctypes.c_size_t, _vp], ctypes.c_int),
    "gs_densify": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp, ctypes.c_size_t, _vp],
                   ctypes.c_int),
    "gs_autotune_load": ([_vp, ctypes.c_char_p], ctypes.c_int),
    "gs_workspace_query": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int64,
                            ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "gs_workspace_layout": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int64, _vp], ctypes.c_int),
    "gs_render_forward": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int64,
                           _vp, _vp], ctypes.c_int),
    "gs_loss_l1": ([_vp, _vp, ctypes.c_int, _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp],
                   ctypes.c_int),
    "gs_render_backward": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int64,
                            _vp, _vp, _vp, ctypes.c_int, _vp], ctypes.c_int),
    "gs_pose_grad": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int64, _vp,
                      _vp, ctypes.c_int, _vp], ctypes.c_int),
    "gs_workspace_status": ([_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "gs_ctx_set_timing": ([_vp, ctypes.c_int], ctypes.c_int),
    "gs_ctx_read_timing": ([_vp, _vp, ctypes.c_int], ctypes.c_int),
    "gs_workspace_counters": ([_vp, _vp, _vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "gs_render_forward_l1": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int64,
                              _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp], ctypes.c_int),
    "gs_render_step_l1": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int64,
                           _vp, _vp, _vp, ctypes.c_float, ctypes.c_float, _vp, _vp, _vp, ctypes.c_int, _vp],
                          ctypes.c_int),
    "gs_pose_adam": ([_vp, ctypes.c_int, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_float), ctypes.c_float,
                      ctypes.c_float, ctypes.c_float, _vp], ctypes.c_int),
    "gs_select_reliable": ([_vp, _vp, _vp, _vp, ctypes.c_float, _vp, _vp], ctypes.c_int),
    "gs_select_opacity": ([_vp, _vp, ctypes.c_float, _vp, _vp, _vp], ctypes.c_int),
    "gs_expand_workspace_query": ([_vp, ctypes.c_int64, _vp, ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "gs_expand": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp, ctypes.c_size_t, _vp],
                  ctypes.c_int),
    "gs_render_forward_static": ([_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int64, _vp, _vp],
                                 ctypes.c_int),
    "gs_render_forward_static_status": ([_vp, _vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "gs_ctx_set_spin_limit": ([_vp, ctypes.c_uint32], ctypes.c_int),
    "gs_ctx_set_persistent": ([_vp, ctypes.c_int], ctypes.c_int),
    "gs_pose_apply": ([_vp, ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
    "gs_twist_chain": ([_vp, ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
}

_lib = None


def lib():
    """The loaded libgsr.so (raises if it is not built: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is not built; run paper_2311_11700_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in ABI.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# ----------------------------------------------------------------------------
# scenes and views
# ----------------------------------------------------------------------------
class Scene:
    """One Gaussian parameter set on the GPU: float32 planes mean [3,N],
    log_scale [3,N], quat [4,N], opacity_logit [N], sh [3K,N]; mask uint8 [N]."""

    def __init__(self, mean, log_scale, quat, opacity_logit, sh, sh_degree, mask=None):
        self.mean, self.log_scale, self.quat = mean, log_scale, quat
        self.opacity_logit, self.sh, self.sh_degree, self.mask = opacity_logit, sh, int(sh_degree), mask
        n = mean.shape[1]
        K = (self.sh_degree + 1) ** 2
        for name, t, shape in (("mean", mean, (3, n)), ("log_scale", log_scale, (3, n)), ("quat", quat, (4, n)),
                               ("opacity_logit", opacity_logit, (n,)), ("sh", sh, (3 * K, n))):
            if tuple(t.shape) != shape or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"scene.{name}: need a contiguous float32 CUDA tensor of shape {shape}")
        if mask is not None and (mask.dtype != torch.uint8 or tuple(mask.shape) != (n,)):
            raise ValueError("scene.mask: need uint8 [N]")

    @property
    def n(self):
        return self.mean.shape[1]

    def params(self):
        return [getattr(self, k) for k in PARAM_KEYS]

    @staticmethod
    def from_numpy(d, device="cuda", mask=None):
        t = {k: torch.as_tensor(np.ascontiguousarray(d[k]), dtype=torch.float32, device=device)
             for k in PARAM_KEYS}
        m = None if mask is None else torch.as_tensor(np.asarray(mask, np.uint8), device=device)
        return Scene(t["mean"], t["log_scale"], t["quat"], t["opacity_logit"], t["sh"], d["sh_degree"], m)

    def with_params(self, params, mask="keep"):
        return Scene(*params, self.sh_degree, self.mask if mask == "keep" else mask)

    def c_struct(self):
        return gs_scene(self.n, self.sh_degree, 0, _ptr(self.mean), _ptr(self.log_scale), _ptr(self.quat),
                        _ptr(self.opacity_logit), _ptr(self.sh), _ptr(self.mask))


def view_struct(v):
    """A gs_view from a dict (width, height, fx, fy, cx, cy, z_near, bg, T_cw, scene?,
    T_cw_dev? (CUDA float32 tensor [12]), pixel_mask? (CUDA uint8 [H, W]))."""
    s = gs_view()
    s.width, s.height = int(v["width"]), int(v["height"])
    s.scene = int(v.get("scene", 0))
    s.fx, s.fy, s.cx, s.cy = float(v["fx"]), float(v["fy"]), float(v["cx"]), float(v["cy"])
    s.z_near = float(v.get("z_near", 0.2))
    bg = np.asarray(v.get("bg", (0, 0, 0)), np.float32)
    for k in range(3):
        s.bg[k] = float(bg[k])
    T = np.asarray(v["T_cw"], np.float32).reshape(12)
    for k in range(12):
        s.T_cw[k] = float(T[k])
    td = v.get("T_cw_dev")
    s.T_cw_dev = None if td is None else td.data_ptr()
    pm = v.get("pixel_mask")
    s.pixel_mask = None if pm is None else pm.data_ptr()
    return s


def _arrays(scenes, views):
    sc = (gs_scene * len(scenes))(*[s.c_struct() for s in scenes])
    vw = (gs_view * len(views))(*[view_struct(v) for v in views])
    return sc, vw


def pixel_offsets(views):
    offs, o = [], 0
    for v in views:
        offs.append(o)
        o += int(v["width"]) * int(v["height"])
    return offs, o


def _images(color, depth, acc):
    return gs_images(_ptr(color), _ptr(depth), _ptr(acc))


def _check(ctx, status):
    if status != GS_OK:
        msg = lib().gs_last_error(ctx.handle) if ctx is not None else b""
        raise GsrError(status, (msg or b"").decode(errors="replace"))


# ----------------------------------------------------------------------------
# context and the C-ABI-named functions
# ----------------------------------------------------------------------------
class Context:
    def __init__(self, device: int = 0, tile=(16, 16)):
        h = ctypes.c_void_p()
        st = lib().gs_ctx_create(ctypes.byref(h), int(device))
        if st != GS_OK:
            raise GsrError(st, f"gs_ctx_create(device={device}) failed")
        self.handle = h
        self.device = device
        self.tile = tuple(tile)
        self.strip = (2, 2)
        self.binning = 0
        self.grad_mode = 0
        self.compact = 1
        self.persistent = 0
        if tuple(tile) != (16, 16):
            _check(self, lib().gs_ctx_set_tiling(self.handle, int(tile[0]), int(tile[1])))

    def set_tiling(self, tw, th):
        _check(self, lib().gs_ctx_set_tiling(self.handle, int(tw), int(th)))
        self.tile = (tw, th)

    def set_strip(self, strip_fwd, strip_bwd=None):
        strip_bwd = strip_fwd if strip_bwd is None else strip_bwd
        _check(self, lib().gs_ctx_set_strip(self.handle, int(strip_fwd), int(strip_bwd)))
        self.strip = (int(strip_fwd), int(strip_bwd))

    def autotune_save(self, path):
        _check(self, lib().gs_autotune_save(self.handle, str(path).encode()))

    def autotune_load(self, path):
        _check(self, lib().gs_autotune_load(self.handle, str(path).encode()))

    def set_grad_mode(self, mode):
        """0: the backward adds (+=) to the gradient buffers; 1: it writes them (=)."""
        _check(self, lib().gs_ctx_set_grad_mode(self.handle, int(mode)))
        self.grad_mode = int(mode)

    def set_persistent(self, mode):
        """Launch form of the fused step's compositing kernel: 0 one CTA per tile, 1
        persistent (warps take tiles from a ticket)."""
        _check(self, lib().gs_ctx_set_persistent(self.handle, int(mode)))
        self.persistent = int(mode)

    def set_spin_limit(self, window_reads):
        """Bound of the device-side look-back waits (window reads; 0: give up at once)."""
        _check(self, lib().gs_ctx_set_spin_limit(self.handle, int(window_reads)))

    def set_binning(self, mode):
        """0: per-tile counting sort + segment sorts (default); 1: global LSD radix sort."""
        _check(self, lib().gs_ctx_set_binning(self.handle, int(mode)))
        self.binning = int(mode)

    def set_compact(self, mode):
        """Compositing form: 0 warp strips; 1 (default) compacted pixels when every view
        of a call has a pixel mask; 2 compacted pixels always."""
        _check(self, lib().gs_ctx_set_compact(self.handle, int(mode)))
        self.compact = int(mode)

    def close(self):
        if self.handle:
            lib().gs_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_workspace_query(ctx, scenes, views, max_pairs):
    sc, vw = _arrays(scenes, views)
    n = ctypes.c_size_t()
    _check(ctx, lib().gs_workspace_query(ctx.handle, sc, len(scenes), vw, len(views), int(max_pairs),
                                         ctypes.byref(n)))
    return int(n.value)


def gs_workspace_layout(ctx, scenes, views, max_pairs):
    sc, vw = _arrays(scenes, views)
    lay = gs_layout()
    _check(ctx, lib().gs_workspace_layout(ctx.handle, sc, len(scenes), vw, len(views), int(max_pairs),
                                          ctypes.byref(lay)))
    return lay


def gs_render_forward(ctx, scenes, views, workspace, max_pairs, out, stream=None):
    """out = (color [3*P], depth [P], acc [P]) packed float32 CUDA tensors (None = not written)."""
    sc, vw = _arrays(scenes, views)
    img = _images(*out)
    _check(ctx, lib().gs_render_forward(ctx.handle, sc, len(scenes), vw, len(views), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), int(max_pairs),
                                        ctypes.byref(img), _stream_handle(stream)))


def gs_render_forward_l1(ctx, scenes, views, workspace, max_pairs, out, target_rgb, target_depth, w_c, w_d, loss,
                         dL_dout, stream=None):
    """Forward render with the L1 loss and its adjoint fused into the compositing epilogue."""
    sc, vw = _arrays(scenes, views)
    img = _images(*out)
    d = _images(*dL_dout)
    _check(ctx, lib().gs_render_forward_l1(ctx.handle, sc, len(scenes), vw, len(views), _ptr(workspace),
                                           workspace.numel() * workspace.element_size(), int(max_pairs),
                                           ctypes.byref(img), _ptr(target_rgb), _ptr(target_depth), float(w_c),
                                           float(w_d), _ptr(loss), ctypes.byref(d), _stream_handle(stream)))


def gs_render_forward_static(ctx, scenes, views, max_pairs, out, stream=None):
    """gs_render_forward without a workspace: the library's static 32 MiB device
    scratch is used instead (for callers that cannot allocate device memory when
    they render).  Calls share that scratch: do not overlap them on the GPU."""
    sc, vw = _arrays(scenes, views)
    img = _images(*out)
    _check(ctx, lib().gs_render_forward_static(ctx.handle, sc, len(scenes), vw, len(views), int(max_pairs),
                                               ctypes.byref(img), _stream_handle(stream)))


def gs_render_forward_static_status(ctx, stream=None):
    """(status, pairs_needed) of the last gs_render_forward_static on the context's
    device; synchronises the stream."""
    n = ctypes.c_int64()
    st = lib().gs_render_forward_static_status(ctx.handle, _stream_handle(stream), ctypes.byref(n))
    return st, int(n.value)


def gs_loss_l1(ctx, views, rendered, target_rgb, target_depth, w_c, w_d, loss, dL_dout, stream=None):
    vw = (gs_view * len(views))(*[view_struct(v) for v in views])
    r = _images(*rendered)
    d = _images(*dL_dout)
    _check(ctx, lib().gs_loss_l1(ctx.handle, vw, len(views), ctypes.byref(r), _ptr(target_rgb),
                                 _ptr(target_depth), float(w_c), float(w_d), _ptr(loss), ctypes.byref(d),
                                 _stream_handle(stream)))


def _grads_array(grads):
    if grads is None:
        return None
    arr = (gs_grads * len(grads))()
    for i, g in enumerate(grads):
        if g is not None:
            arr[i] = gs_grads(*[_ptr(g.get(k)) for k in PARAM_KEYS], _ptr(g.get("vs_grad_norm")),
                              _ptr(g.get("vs_count")))
    return arr


def gs_render_backward(ctx, scenes, views, workspace, max_pairs, dL_dout, grads, dL_dtwist=None, pose_mode=0,
                       stream=None):
    """grads: per scene a dict of float32 CUDA tensors shaped like the parameters
    (accumulated +=); dL_dtwist: float32 [V, 6] (accumulated) or None."""
    sc, vw = _arrays(scenes, views)
    d = _images(*dL_dout)
    ga = _grads_array(grads)
    _check(ctx, lib().gs_render_backward(ctx.handle, sc, len(scenes), vw, len(views), _ptr(workspace),
                                         workspace.numel() * workspace.element_size(), int(max_pairs),
                                         ctypes.byref(d), ga, _ptr(dL_dtwist), int(pose_mode),
                                         _stream_handle(stream)))


def gs_render_step_l1(ctx, scenes, views, workspace, max_pairs, out, target_rgb, target_depth, w_c, w_d, loss,
                      grads=None, dL_dtwist=None, pose_mode=0, stream=None):
    """Forward, fused L1 loss and backward in one call (one compositing kernel).
    out = (color, depth, acc) or None; grads as in gs_render_backward, or None for
    the pose gradient alone (then dL_dtwist is required)."""
    sc, vw = _arrays(scenes, views)
    img = _images(*(out if out is not None else (None, None, None)))
    ga = _grads_array(grads)
    _check(ctx, lib().gs_render_step_l1(ctx.handle, sc, len(scenes), vw, len(views), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(), int(max_pairs),
                                        ctypes.byref(img), _ptr(target_rgb), _ptr(target_depth), float(w_c),
                                        float(w_d), _ptr(loss), ga, _ptr(dL_dtwist), int(pose_mode),
                                        _stream_handle(stream)))


def gs_pose_grad(ctx, scenes, views, workspace, max_pairs, dL_dout, dL_dtwist, pose_mode=0, stream=None):
    sc, vw = _arrays(scenes, views)
    d = _images(*dL_dout)
    _check(ctx, lib().gs_pose_grad(ctx.handle, sc, len(scenes), vw, len(views), _ptr(workspace),
                                   workspace.numel() * workspace.element_size(), int(max_pairs), ctypes.byref(d),
                                   _ptr(dL_dtwist), int(pose_mode), _stream_handle(stream)))


def gs_autotune_workspace_query(ctx, scenes, views, max_pairs):
    sc, vw = _arrays(scenes, views)
    b = ctypes.c_size_t()
    _check(ctx, lib().gs_autotune_workspace_query(ctx.handle, sc, len(scenes), vw, len(views), int(max_pairs),
                                                  ctypes.byref(b)))
    return int(b.value)


def gs_autotune(ctx, scenes, views, workspace, max_pairs, out, dL_dout, grads, reps=3, force=False, stream=None):
    """Times the configurations of the search space on this batch and applies the
    fastest (see gs_autotune in gsr.h); returns the chosen configuration as a dict."""
    sc, vw = _arrays(scenes, views)
    o, d = _images(*out), _images(*dL_dout)
    ga = _grads_array(grads)
    r = gs_tune_result()
    _check(ctx, lib().gs_autotune(ctx.handle, sc, len(scenes), vw, len(views), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(), int(max_pairs), ctypes.byref(o),
                                  ctypes.byref(d), ga, int(reps), int(bool(force)), ctypes.byref(r),
                                  _stream_handle(stream)))
    ctx.tile = (r.tile_w, r.tile_h)
    ctx.strip = (r.strip_fwd, r.strip_bwd)
    ctx.binning = r.binning
    return {"tile": (r.tile_w, r.tile_h), "strip": (r.strip_fwd, r.strip_bwd), "binning": r.binning,
            "ms_fwd": r.ms_fwd, "ms_bwd": r.ms_bwd, "timed": r.timed}


def gs_autotune_step_l1(ctx, scenes, views, workspace, max_pairs, out, target_rgb, target_depth, w_c, w_d, loss,
                        grads=None, dL_dtwist=None, pose_mode=0, reps=3, force=False, stream=None):
    """Times the configurations of the search space with the fused step itself
    (gs_render_step_l1's arguments) and applies the fastest (see
    gs_autotune_step_l1 in gsr.h); returns the chosen configuration as a dict
    (ms_fwd: the step's time)."""
    sc, vw = _arrays(scenes, views)
    img = _images(*(out if out is not None else (None, None, None)))
    ga = _grads_array(grads)
    r = gs_tune_result()
    _check(ctx, lib().gs_autotune_step_l1(ctx.handle, sc, len(scenes), vw, len(views), _ptr(workspace),
                                          workspace.numel() * workspace.element_size(), int(max_pairs),
                                          ctypes.byref(img), _ptr(target_rgb), _ptr(target_depth), float(w_c),
                                          float(w_d), _ptr(loss), ga, _ptr(dL_dtwist), int(pose_mode), int(reps),
                                          int(bool(force)), ctypes.byref(r), _stream_handle(stream)))
    ctx.tile = (r.tile_w, r.tile_h)
    ctx.strip = (r.strip_fwd, r.strip_bwd)
    ctx.binning = r.binning
    return {"tile": (r.tile_w, r.tile_h), "strip": (r.strip_fwd, r.strip_bwd), "binning": r.binning,
            "ms_fwd": r.ms_fwd, "ms_bwd": r.ms_bwd, "timed": r.timed}


def gs_workspace_status(ctx, workspace, stream=None):
    """(status, pairs_needed); synchronises the stream."""
    n = ctypes.c_int64()
    st = lib().gs_workspace_status(ctx.handle, _ptr(workspace), _stream_handle(stream), ctypes.byref(n))
    return st, int(n.value)


def gs_pose_adam(ctx, T_cw_dev, dL_dtwist, state, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step on every view's device-resident pose (T_cw_dev [V, 12])."""
    lr6 = (ctypes.c_float * 6)(*[float(x) for x in lr])
    _check(ctx, lib().gs_pose_adam(ctx.handle, int(T_cw_dev.shape[0]), _ptr(T_cw_dev), _ptr(dL_dtwist), _ptr(state),
                                   lr6, float(beta1), float(beta2), float(eps), _stream_handle(stream)))


def gs_pose_apply(ctx, twist, T_in, T_out, stream=None):
    """T_out[v] = exp(twist[v]^) T_in[v] (twist [V, 6], poses [V, 12], CUDA float32)."""
    _check(ctx, lib().gs_pose_apply(ctx.handle, int(twist.shape[0]), _ptr(twist), _ptr(T_in), _ptr(T_out),
                                    _stream_handle(stream)))


def gs_twist_chain(ctx, twist, dL_deps, dL_dtwist, stream=None):
    """dL_dtwist[v] = J(twist[v])^T dL_deps[v] (the SE(3) left Jacobian; [V, 6] CUDA float32)."""
    _check(ctx, lib().gs_twist_chain(ctx.handle, int(twist.shape[0]), _ptr(twist), _ptr(dL_deps), _ptr(dL_dtwist),
                                     _stream_handle(stream)))


def gs_select_reliable(ctx, scene, view, obs_depth, eps, mask_out, stream=None):
    sc = scene.c_struct()
    vw = view_struct(view)
    _check(ctx, lib().gs_select_reliable(ctx.handle, ctypes.byref(sc), ctypes.byref(vw), _ptr(obs_depth),
                                         float(eps), _ptr(mask_out), _stream_handle(stream)))


def gs_select_opacity(ctx, scene, thr, keep, mask_out, stream=None):
    sc = scene.c_struct()
    _check(ctx, lib().gs_select_opacity(ctx.handle, ctypes.byref(sc), float(thr), _ptr(keep), _ptr(mask_out),
                                        _stream_handle(stream)))


def gs_densify(ctx, scene, vs_grad_norm, vs_count, noise, out, capacity, count, grad_thr=0.002, scale_thr=0.02,
               split_scale=1.6, workspace=None, stream=None):
    """Clone / split density control (see gs_densify in gsr.h) into `out` (dict of
    planes with `capacity` columns); count: int64 CUDA tensor [4] receives (kept,
    cloned, split, needed)."""
    sc = scene.c_struct()
    if workspace is None:
        b = ctypes.c_size_t()
        _check(ctx, lib().gs_densify_workspace_query(ctx.handle, int(scene.n), ctypes.byref(b)))
        workspace = alloc_workspace(int(b.value), scene.mean.device)
    prm = gs_densify_params(float(grad_thr), float(scale_thr), float(split_scale), 0)
    o = gs_scene_out(*[_ptr(out[k]) for k in PARAM_KEYS])
    _check(ctx, lib().gs_densify(ctx.handle, ctypes.byref(sc), _ptr(vs_grad_norm), _ptr(vs_count), _ptr(noise),
                                 ctypes.byref(prm), ctypes.byref(o), int(capacity), _ptr(count), _ptr(workspace),
                                 workspace.numel(), _stream_handle(stream)))


def gs_outlier_mask(ctx, views, rendered, target_rgb, target_depth, w_c, w_d, factor, mask_out, workspace=None,
                    stream=None):
    """Tracking-loss outlier rejection (see gs_outlier_mask in gsr.h): mask_out (uint8
    [P]) = the pixels of each view's pixel_mask whose loss is at most factor x the
    view's median loss.  rendered = (color, depth)."""
    vw = (gs_view * len(views))(*[view_struct(v) for v in views])
    if workspace is None:
        b = ctypes.c_size_t()
        _check(ctx, lib().gs_outlier_mask_workspace_query(ctx.handle, vw, len(views), ctypes.byref(b)))
        workspace = alloc_workspace(int(b.value), mask_out.device)
    img = _images(rendered[0], rendered[1], None)
    _check(ctx, lib().gs_outlier_mask(ctx.handle, vw, len(views), ctypes.byref(img), _ptr(target_rgb),
                                      _ptr(target_depth), float(w_c), float(w_d), float(factor), _ptr(mask_out),
                                      _ptr(workspace), workspace.numel(), _stream_handle(stream)))


def gs_expand_workspace_query(ctx, n, view):
    vw = view_struct(view)
    b = ctypes.c_size_t()
    _check(ctx, lib().gs_expand_workspace_query(ctx.handle, int(n), ctypes.byref(vw), ctypes.byref(b)))
    return int(b.value)


def gs_expand(ctx, scene, view, rendered_acc, rendered_depth, obs_rgb, obs_depth, params, out, capacity, count,
              workspace, stream=None):
    """Adaptive expansion (Sec. 3.2) into `out` (dict of planes with `capacity` columns);
    count: int64 CUDA tensor [4] = (kept, added, written, total)."""
    sc = scene.c_struct()
    vw = view_struct(view)
    prm = gs_expand_params(float(params.get("tau_T", 0.5)), float(params.get("tau_D", 0.1)),
                           float(params.get("eta", 0.01)), float(params.get("gamma", 0.1)),
                           float(params.get("init_opacity", 0.1)), float(params.get("density", 1.0)),
                           float(params.get("prune_opacity", 0.005)),
                           int(params.get("flags", GS_EXPAND_ADD | GS_EXPAND_DELETE | GS_EXPAND_PRUNE)))
    o = gs_scene_out(*[_ptr(out[k]) for k in PARAM_KEYS])
    _check(ctx, lib().gs_expand(ctx.handle, ctypes.byref(sc), ctypes.byref(vw), _ptr(rendered_acc),
                                _ptr(rendered_depth), _ptr(obs_rgb), _ptr(obs_depth), ctypes.byref(prm),
                                ctypes.byref(o), int(capacity), _ptr(count), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream_handle(stream)))


def gs_ctx_set_timing(ctx, on):
    """on: 0 (or False) off; 1 (or True) stage events and the compositing work
    counters; 2 stage events only, with the kernels of the untimed path."""
    _check(ctx, lib().gs_ctx_set_timing(ctx.handle, int(on)))


def gs_ctx_read_timing(ctx, reset=True):
    """{stage: (ms, launches)} accumulated since the last reset, plus 'calls'."""
    t = gs_timing()
    _check(ctx, lib().gs_ctx_read_timing(ctx.handle, ctypes.byref(t), int(reset)))
    out = {name: (t.ms[i], int(t.launches[i])) for i, name in enumerate(STAGES)}
    out["calls"] = int(t.calls)
    return out


def gs_workspace_counters(ctx, workspace, stream=None):
    """(visible splats, pairs, blended pairs fwd, blended pairs bwd, bwd warp-Gaussian
    iterations visited, with a blend, reduced, tile segments longer than 512)."""
    arr = (ctypes.c_int64 * 8)()
    _check(ctx, lib().gs_workspace_counters(ctx.handle, _ptr(workspace), _stream_handle(stream), arr))
    return tuple(int(x) for x in arr)


# ----------------------------------------------------------------------------
# convenience: workspace management and autograd
# ----------------------------------------------------------------------------
def alloc_workspace(nbytes, device="cuda"):
    # 256-byte alignment: the caching allocator returns 512-byte aligned blocks
    t = torch.empty(int(nbytes), dtype=torch.uint8, device=device)
    assert t.data_ptr() % 256 == 0
    return t


class Renderer:
    """A context plus a pair capacity that grows when a forward overflows it."""

    def __init__(self, device=0, tile=(16, 16), pairs_per_splat=8.0):
        self.ctx = Context(device, tile)
        self.device = torch.device("cuda", device)
        self.pairs_per_splat = pairs_per_splat
        self.max_pairs = None

    def _capacity(self, scenes, views):
        if self.max_pairs is None:
            n = sum(scenes[int(v.get("scene", 0))].n for v in views)
            self.max_pairs = int(max(4096, self.pairs_per_splat * n))
        return self.max_pairs

    def new_workspace(self, scenes, views):
        mp = self._capacity(scenes, views)
        return alloc_workspace(gs_workspace_query(self.ctx, scenes, views, mp), self.device), mp

    def forward(self, scenes, views, workspace=None, check=True, want=("color", "depth", "acc")):
        """Render; returns (color [3P], depth [P], acc [P], workspace, max_pairs).  With
        check=True the stream is synchronised once to detect a pair-list overflow,
        which is fixed by growing the capacity and rendering again."""
        _, P = pixel_offsets(views)
        dev = self.device
        color = torch.empty(3 * P, device=dev) if "color" in want else None
        depth = torch.empty(P, device=dev) if "depth" in want else None
        acc = torch.empty(P, device=dev) if "acc" in want else None
        for _ in range(4):
            mp = self._capacity(scenes, views)
            need = gs_workspace_query(self.ctx, scenes, views, mp)
            if workspace is None or workspace.numel() < need:
                workspace = alloc_workspace(need, dev)
            gs_render_forward(self.ctx, scenes, views, workspace, mp, (color, depth, acc))
            if not check:
                break
            st, needed = gs_workspace_status(self.ctx, workspace)
            if st == GS_ERR_CAPACITY and needed >= mp:
                self.max_pairs = int(needed * 1.25) + 4096
                continue
            _check(self.ctx, st)
            break
        else:
            raise GsrError(GS_ERR_CAPACITY, f"pair list still over capacity after growing it to {mp}")
        return color, depth, acc, workspace, mp


    def autotune(self, scenes, views, reps=3, force=False, pairs_headroom=4.0, step=None):
        """Pick the fastest tile / binning / strip configuration for this batch by
        timing it; the choice is cached in the context by batch shape.  step=None
        times separate forward and backward calls (gs_autotune).  step = dict(
        target_rgb, target_depth, w_c=1.0, w_d=0.5, out=False, grads=True,
        twist=True) times the fused L1 step as the caller will run it
        (gs_autotune_step_l1): images written or not, parameter gradients or the
        pose gradient alone, the twist gradient or not.  The pair capacity is
        raised to pairs_headroom x what the current tiling needs, so that the
        finer tilings (more pairs) can be timed too."""
        _, P = pixel_offsets(views)
        dev = self.device
        *_, ws, mp = self.forward(scenes, views)
        _, needed = gs_workspace_status(self.ctx, ws)
        self.max_pairs = max(mp, int(needed * pairs_headroom) + 4096)
        nbytes = gs_autotune_workspace_query(self.ctx, scenes, views, self.max_pairs)
        ws = alloc_workspace(nbytes, dev)
        out = (torch.empty(3 * P, device=dev), torch.empty(P, device=dev), torch.empty(P, device=dev))
        grads = [{k: torch.zeros_like(getattr(s, k)) for k in PARAM_KEYS} for s in scenes]
        if step is None:
            dL = (torch.ones(3 * P, device=dev), torch.ones(P, device=dev), None)
            return gs_autotune(self.ctx, scenes, views, ws, self.max_pairs, out, dL, grads, reps, force)
        loss = torch.zeros(len(views), device=dev)
        twist = torch.zeros(len(views), 6, device=dev) if step.get("twist", True) else None
        return gs_autotune_step_l1(self.ctx, scenes, views, ws, self.max_pairs, out if step.get("out") else None,
                                   step["target_rgb"], step["target_depth"], step.get("w_c", 1.0),
                                   step.get("w_d", 0.5), loss, grads if step.get("grads", True) else None, twist,
                                   0, reps, force)


class RenderRGBD(torch.autograd.Function):
    """Differentiable render of one or more views.

    forward(renderer, scenes, views, twist, pose_mode, *params) -> (color, depth, acc)
    params = the five parameter tensors of every scene, in order; twist = [V, 6]
    (rho, phi): view v renders at the pose exp(twist[v]^) T_v (gs_pose_apply), T_v its
    T_cw_dev or T_cw.  The twist's gradient is the left-perturbation pose gradient at
    that pose chained through the exponential (gs_twist_chain); at twist = 0 it is the
    pose gradient itself."""

    @staticmethod
    def forward(ctx, renderer, scenes, views, twist, pose_mode, *params):
        dev = renderer.device
        scenes = [s.with_params(params[5 * i:5 * i + 5]) for i, s in enumerate(scenes)]
        T_in = torch.stack([v["T_cw_dev"].reshape(12) if v.get("T_cw_dev") is not None else
                            torch.as_tensor(np.asarray(v["T_cw"], np.float32).reshape(12), device=dev)
                            for v in views])
        tw = twist.detach().to(dev, torch.float32).contiguous()
        T = torch.empty_like(T_in)
        gs_pose_apply(renderer.ctx, tw, T_in, T)
        views = [dict(v, T_cw_dev=T[i]) for i, v in enumerate(views)]
        color, depth, acc, ws, mp = renderer.forward(scenes, views)
        ctx.renderer, ctx.scenes, ctx.views, ctx.ws, ctx.mp = renderer, scenes, views, ws, mp
        ctx.T, ctx.tw = T, tw  # the device poses the views point at stay alive for the backward
        ctx.pose_mode = pose_mode
        ctx.n_params = len(params)
        return color, depth, acc

    @staticmethod
    def backward(ctx, gC, gD, gA):
        grads = [{k: torch.zeros_like(getattr(s, k)) for k in PARAM_KEYS} for s in ctx.scenes]
        dtw = torch.zeros(len(ctx.views), 6, device=ctx.renderer.device)
        f = lambda t: None if t is None else t.contiguous()  # noqa: E731
        gs_render_backward(ctx.renderer.ctx, ctx.scenes, ctx.views, ctx.ws, ctx.mp, (f(gC), f(gD), f(gA)), grads,
                           dtw, ctx.pose_mode)
        gs_twist_chain(ctx.renderer.ctx, ctx.tw, dtw, dtw)
        flat = [g[k] for g in grads for k in PARAM_KEYS]
        return (None, None, None, dtw, None, *flat)


def render_rgbd(renderer, scenes, views, twist=None, pose_mode=0):
    if twist is None:
        twist = torch.zeros(len(views), 6, device=renderer.device, requires_grad=True)
    params = [p for s in scenes for p in s.params()]
    return RenderRGBD.apply(renderer, scenes, views, twist, pose_mode, *params)
