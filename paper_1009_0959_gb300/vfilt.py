"""Python binding of the C ABI in include/vfilt.h (argument marshalling only).

Every filter step runs in the CUDA library libvfilt.so; this module only
turns torch tensors into pointers, sizes and the current CUDA stream.  There
is no fallback: if the library has not been built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libvfilt.so")

CRITERIA = {"vmf": 0, "bvdf": 1, "amnfe": 2, "amnfg": 3, "evmf": 4, "evbdf": 5}
APPROX = {"exact": 0, "poly": 1, "rational": 2, "rational_fit": 3}
PRECISION = {"fp32": 0, "fp16x2": 1, "bf16x2": 2}
FUNCTIONS = {"acos_lo": 0, "acos_hi": 1, "exp": 2, "ent": 3, "half_angle": 4}
STATUS = {0: "VF_OK", 1: "VF_ERR_ARG", 2: "VF_ERR_ALIAS", 3: "VF_ERR_UNSUPPORTED",
          4: "VF_ERR_CUDA", 5: "VF_ERR_TIMEOUT", 6: "VF_ERR_OOM"}

STAT_PIXELS, STAT_NEAR_TIES, STAT_SWITCHED = 0, 1, 2


class VFError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status
        self.name = STATUS.get(status, str(status))


class Params(ctypes.Structure):
    """vf_params."""
    _fields_ = [("window", ctypes.c_int), ("criterion", ctypes.c_int),
                ("approx", ctypes.c_int), ("degree", ctypes.c_int),
                ("precision", ctypes.c_int), ("kappa", ctypes.c_float),
                ("exp_cutoff", ctypes.c_float), ("ent_cutoff", ctypes.c_float)]


class ImageDesc(ctypes.Structure):
    """vf_image_desc."""
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
                ("height", ctypes.c_int), ("width", ctypes.c_int), ("channels", ctypes.c_int),
                ("in_pitch", ctypes.c_size_t), ("out_pitch", ctypes.c_size_t),
                ("params", Params)]


_lock = threading.Lock()
_lib = None
_tls = threading.local()


def lib():
    """The loaded libvfilt.so (raises if it is missing: no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libvfilt.so is not built (%s); run "
                                   "paper_1009_0959_gb300.build.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            P, I, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
            L.vf_create.argtypes = [ctypes.POINTER(P)]
            L.vf_create.restype = I
            L.vf_destroy.argtypes = [P]
            L.vf_destroy.restype = None
            L.vf_status_string.argtypes = [I]
            L.vf_status_string.restype = ctypes.c_char_p
            L.vf_last_error.argtypes = [P]
            L.vf_last_error.restype = ctypes.c_char_p
            L.vf_set_option.argtypes = [P, I, I]
            L.vf_set_option.restype = I
            L.vf_default_params.argtypes = [ctypes.POINTER(Params)]
            L.vf_default_params.restype = None
            L.vf_get_approximant.argtypes = [P, I, I, I, ctypes.c_double, ctypes.c_double, P,
                                             ctypes.POINTER(I), P, ctypes.POINTER(I),
                                             ctypes.POINTER(ctypes.c_double)]
            L.vf_get_approximant.restype = I
            L.vf_set_coefficients.argtypes = [P, I, I, I, P, I, P, I, ctypes.c_double,
                                              ctypes.c_double]
            L.vf_set_coefficients.restype = I
            L.vf_row_quantum.argtypes = [P, ctypes.POINTER(Params), ctypes.POINTER(I)]
            L.vf_row_quantum.restype = I
            L.vf_band_plan.argtypes = [I, I, I, I, I] + [ctypes.POINTER(I)] * 4
            L.vf_band_plan.restype = I
            L.vf_filter.argtypes = [P, P, P, I, I, I, S, S, ctypes.POINTER(Params), P, P]
            L.vf_filter.restype = I
            L.vf_filter_host.argtypes = [P, P, P, I, I, I, S, S, ctypes.POINTER(Params), P]
            L.vf_filter_host.restype = I
            L.vf_filter_host_async.argtypes = [P, P, P, I, I, I, S, S, ctypes.POINTER(Params), P]
            L.vf_filter_host_async.restype = I
            L.vf_host_sync.argtypes = [P]
            L.vf_host_sync.restype = I
            L.vf_batch_create.argtypes = [P, P, I, ctypes.POINTER(P)]
            L.vf_batch_create.restype = I
            L.vf_batch_launch.argtypes = [P, P]
            L.vf_batch_launch.restype = I
            L.vf_batch_graph_launch.argtypes = [P, P]
            L.vf_batch_graph_launch.restype = I
            L.vf_batch_autotune.argtypes = [P, P, ctypes.POINTER(I), ctypes.POINTER(I),
                                            ctypes.POINTER(ctypes.c_float)]
            L.vf_batch_autotune.restype = I
            L.vf_batch_configure.argtypes = [P, I, I]
            L.vf_batch_configure.restype = I
            L.vf_batch_set_pixels_per_thread.argtypes = [P, I]
            L.vf_batch_set_pixels_per_thread.restype = I
            L.vf_batch_get_config.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I),
                                              ctypes.POINTER(I)]
            L.vf_batch_get_config.restype = I
            L.vf_batch_set_mode.argtypes = [P, I]
            L.vf_batch_set_mode.restype = I
            L.vf_batch_get_mode.argtypes = [P, ctypes.POINTER(I)]
            L.vf_batch_get_mode.restype = I
            L.vf_batch_destroy.argtypes = [P]
            L.vf_batch_destroy.restype = None
            L.vf_batch_run_static.argtypes = [P, P, I, P]
            L.vf_batch_run_static.restype = I
            L.vf_gate_create.argtypes = [P, ctypes.c_ulonglong, ctypes.POINTER(P)]
            L.vf_gate_create.restype = I
            L.vf_gate_set_params.argtypes = [P, P, I]
            L.vf_gate_set_params.restype = I
            L.vf_gate_get_params.argtypes = [P, P, I]
            L.vf_gate_get_params.restype = I
            L.vf_gate_gradient.argtypes = [P, P, P, I, I, I, I, S, P, P, P, P]
            L.vf_gate_gradient.restype = I
            L.vf_gate_train_step.argtypes = [P, P, P, I, I, I, I, S, ctypes.c_float, P, P]
            L.vf_gate_train_step.restype = I
            L.vf_gate_infer.argtypes = [P, P, I, I, I, S, ctypes.c_float, P, S, P, P]
            L.vf_gate_infer.restype = I
            L.vf_filter_gated.argtypes = [P, P, P, I, I, I, S, S, P, S, ctypes.POINTER(Params), P,
                                          P]
            L.vf_filter_gated.restype = I
            L.vf_gate_save.argtypes = [P, ctypes.c_char_p]
            L.vf_gate_save.restype = I
            L.vf_gate_load.argtypes = [P, ctypes.c_char_p]
            L.vf_gate_load.restype = I
            L.vf_gate_step_count.argtypes = [P]
            L.vf_gate_step_count.restype = ctypes.c_ulonglong
            L.vf_gate_check.argtypes = [P]
            L.vf_gate_check.restype = I
            L.vf_gate_destroy.argtypes = [P]
            L.vf_gate_destroy.restype = None
            L.vf_debug_fail_alloc.argtypes = [I]
            L.vf_debug_fail_alloc.restype = I
            _lib = L
        return _lib


def context():
    """A per-thread library context (vf_ctx)."""
    ctx = getattr(_tls, "ctx", None)
    if ctx is None:
        ctx = ctypes.c_void_p()
        st = lib().vf_create(ctypes.byref(ctx))
        if st != 0:
            raise VFError(st, "vf_create failed")
        _tls.ctx = ctx
    return ctx


OPTIONS = {"pair_reuse": 0, "tile_rows": 1, "gate_tensor_cores": 2, "overlap_launch": 3,
           "gated_sparse": 4}


def set_option(name: str, value: int):
    """vf_set_option on this thread's context."""
    ctx = context()
    _check(lib().vf_set_option(ctx, OPTIONS[name], int(value)), ctx)


def _check(st: int, ctx):
    if st != 0:
        raise VFError(st, lib().vf_last_error(ctx).decode())


def make_params(window=3, criterion="vmf", approx="exact", degree=4, precision="fp32",
                kappa=0.33, exp_cutoff=10.0, ent_cutoff=-1.0) -> Params:
    p = Params()
    lib().vf_default_params(ctypes.byref(p))
    p.window = int(window)
    p.criterion = CRITERIA[criterion] if isinstance(criterion, str) else int(criterion)
    p.approx = APPROX[approx] if isinstance(approx, str) else int(approx)
    p.degree = int(degree)
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.kappa, p.exp_cutoff, p.ent_cutoff = float(kappa), float(exp_cutoff), float(ent_cutoff)
    return p


def _image_args(t):
    if t.dim() != 3 or t.shape[2] not in (3, 4):
        raise ValueError("expected an H x W x C (C = 3 or 4) uint8 tensor")
    if str(t.dtype) != "torch.uint8" or not t.is_cuda:
        raise ValueError("expected a CUDA uint8 tensor")
    if t.stride(2) != 1 or t.stride(1) != t.shape[2]:
        raise ValueError("pixels must be interleaved and rows dense (pitch = stride(0))")
    return t.data_ptr(), int(t.shape[0]), int(t.shape[1]), int(t.shape[2]), int(t.stride(0))


def filter(inp, out=None, *, stream=None, stats=None, **params):
    """d_out = F(W(d_in)) for an H x W x C uint8 CUDA tensor (vf_filter).

    params: window, criterion, approx, degree, precision, kappa, exp_cutoff,
    ent_cutoff.  `stream` is a torch.cuda.Stream (default: the current one);
    `stats` an optional int64 CUDA tensor of 3 counters accumulated in place.
    """
    import torch
    if out is None:
        out = torch.empty_like(inp)
    ip, h, w, c, ipitch = _image_args(inp)
    op, h2, w2, c2, opitch = _image_args(out)
    if (h, w, c) != (h2, w2, c2):
        raise ValueError("input and output shapes differ")
    p = make_params(**params)
    s = stream if stream is not None else torch.cuda.current_stream(inp.device)
    sp = None
    if stats is not None:
        if stats.dtype != torch.int64 or not stats.is_cuda or stats.numel() < 3:
            raise ValueError("stats must be a CUDA int64 tensor of 3 counters")
        sp = stats.data_ptr()
    ctx = context()
    _check(lib().vf_filter(ctx, ip, op, h, w, c, ipitch, opitch, ctypes.byref(p),
                           ctypes.c_void_p(s.cuda_stream), sp), ctx)
    return out


def filter_host(inp, out=None, *, stream=None, **params):
    """vf_filter_host on H x W x C uint8 CPU tensors (pinned or pageable):
    the copies to and from the device and the filter all run in the library.
    Returns `out` when the call has completed."""
    import torch
    if inp.is_cuda or inp.dim() != 3 or inp.dtype != torch.uint8:
        raise ValueError("expected an H x W x C uint8 CPU tensor")
    if out is None:
        out = torch.empty_like(inp)
    if inp.stride(2) != 1 or inp.stride(1) != inp.shape[2] or out.stride(1) != out.shape[2]:
        raise ValueError("pixels must be interleaved and rows dense")
    p = make_params(**params)
    s = stream if stream is not None else torch.cuda.current_stream()
    ctx = context()
    _check(lib().vf_filter_host(ctx, inp.data_ptr(), out.data_ptr(), int(inp.shape[0]),
                                int(inp.shape[1]), int(inp.shape[2]), int(inp.stride(0)),
                                int(out.stride(0)), ctypes.byref(p),
                                ctypes.c_void_p(s.cuda_stream)), ctx)
    return out


def filter_host_async(inp, out, *, stream=None, **params):
    """vf_filter_host_async on H x W x C uint8 CPU tensors (pinned for the
    copies to overlap): enqueues the copies and the filter and returns; call
    host_sync() before reading `out` or changing `inp`."""
    import torch
    if inp.is_cuda or inp.dim() != 3 or inp.dtype != torch.uint8:
        raise ValueError("expected an H x W x C uint8 CPU tensor")
    if inp.stride(2) != 1 or inp.stride(1) != inp.shape[2] or out.stride(1) != out.shape[2]:
        raise ValueError("pixels must be interleaved and rows dense")
    p = make_params(**params)
    s = stream if stream is not None else torch.cuda.current_stream()
    ctx = context()
    _check(lib().vf_filter_host_async(ctx, inp.data_ptr(), out.data_ptr(), int(inp.shape[0]),
                                      int(inp.shape[1]), int(inp.shape[2]), int(inp.stride(0)),
                                      int(out.stride(0)), ctypes.byref(p),
                                      ctypes.c_void_p(s.cuda_stream)), ctx)
    return out


def host_sync():
    """vf_host_sync: wait for every filter_host_async call of this thread's
    context."""
    ctx = context()
    _check(lib().vf_host_sync(ctx), ctx)


class Batch:
    """vf_batch: many (input, output, params) images in one persistent launch.

    images: list of (inp, out, params_dict) with H x W x C uint8 CUDA tensors.
    The tensors must stay alive as long as the batch is used."""

    def __init__(self, images):
        descs = (ImageDesc * len(images))()
        self._keep = []
        for i, (inp, out, params) in enumerate(images):
            ip, h, w, c, ipitch = _image_args(inp)
            op, h2, w2, c2, opitch = _image_args(out)
            if (h, w, c) != (h2, w2, c2):
                raise ValueError("input and output shapes differ")
            d = descs[i]
            d.d_in, d.d_out, d.height, d.width, d.channels = ip, op, h, w, c
            d.in_pitch, d.out_pitch = ipitch, opitch
            d.params = make_params(**params)
            self._keep += [inp, out]
        self.ctx = context()
        self.handle = ctypes.c_void_p()
        _check(lib().vf_batch_create(self.ctx, descs, len(images), ctypes.byref(self.handle)),
               self.ctx)

    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    def launch(self, stream=None):
        _check(lib().vf_batch_launch(self.handle, self._stream(stream)), self.ctx)

    def graph_launch(self, stream=None):
        _check(lib().vf_batch_graph_launch(self.handle, self._stream(stream)), self.ctx)

    def autotune(self, stream=None):
        ty, ctas, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _check(lib().vf_batch_autotune(self.handle, self._stream(stream), ctypes.byref(ty),
                                       ctypes.byref(ctas), ctypes.byref(ms)), self.ctx)
        cfg = self.config()
        cfg["ms"] = ms.value
        return cfg

    def configure(self, tile_rows=4, ctas_per_sm=0, pixels_per_thread=None):
        if pixels_per_thread is not None:
            _check(lib().vf_batch_set_pixels_per_thread(self.handle, int(pixels_per_thread)),
                   self.ctx)
        _check(lib().vf_batch_configure(self.handle, int(tile_rows), int(ctas_per_sm)), self.ctx)

    MODES = {"one_kernel": 0, "class_kernels": 1}

    def set_mode(self, mode):
        """vf_batch_set_mode: "one_kernel" (one persistent kernel for every
        class) or "class_kernels" (one persistent kernel per class, run
        concurrently)."""
        _check(lib().vf_batch_set_mode(self.handle, self.MODES[mode]), self.ctx)

    def config(self):
        """mode, tile_rows, ctas_per_sm (0: occupancy maximum) and
        pixels_per_thread (the last three apply to the one-kernel form)."""
        ty, ctas, ppt, mode = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().vf_batch_get_config(self.handle, ctypes.byref(ty), ctypes.byref(ctas),
                                         ctypes.byref(ppt)), self.ctx)
        _check(lib().vf_batch_get_mode(self.handle, ctypes.byref(mode)), self.ctx)
        names = {v: k for k, v in self.MODES.items()}
        return {"mode": names[mode.value], "tile_rows": ty.value, "ctas_per_sm": ctas.value,
                "pixels_per_thread": ppt.value}

    def close(self):
        if self.handle:
            lib().vf_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


GATE_NPARAM = 2913


class Gate:
    """vf_gate: the learned impulse detector (training, inference, checkpoints)."""

    def __init__(self, seed: int = 0):
        self.ctx = context()
        self.handle = ctypes.c_void_p()
        _check(lib().vf_gate_create(self.ctx, int(seed), ctypes.byref(self.handle)), self.ctx)

    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    @staticmethod
    def _batch(imgs):
        """imgs: B x H x W x C uint8 CUDA tensor (dense)."""
        if imgs.dim() != 4 or not imgs.is_cuda or not imgs.is_contiguous():
            raise ValueError("expected a dense B x H x W x C uint8 CUDA tensor")
        B, H, W, C = imgs.shape
        return imgs.data_ptr(), int(B), int(H), int(W), int(C), int(W * C)

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().vf_gate_set_params(self.handle, a.ctypes.data, a.size), self.ctx)

    def get_params(self):
        import numpy as np
        a = np.zeros(GATE_NPARAM, dtype=np.float32)
        _check(lib().vf_gate_get_params(self.handle, a.ctypes.data, a.size), self.ctx)
        return a

    def gradient(self, imgs, targets, stream=None):
        """(grad, loss, prob) tensors of the mean BCE on a batch (device)."""
        import torch
        p, B, H, W, C, pitch = self._batch(imgs)
        grad = torch.zeros(GATE_NPARAM, dtype=torch.float32, device=imgs.device)
        loss = torch.zeros(1, dtype=torch.float32, device=imgs.device)
        prob = torch.zeros((B, H, W), dtype=torch.float32, device=imgs.device)
        _check(lib().vf_gate_gradient(self.handle, p, targets.data_ptr(), B, H, W, C, pitch,
                                      grad.data_ptr(), loss.data_ptr(), prob.data_ptr(),
                                      self._stream(stream)), self.ctx)
        return grad, loss, prob

    def train_step(self, imgs, targets, lr, loss=None, stream=None):
        p, B, H, W, C, pitch = self._batch(imgs)
        _check(lib().vf_gate_train_step(self.handle, p, targets.data_ptr(), B, H, W, C, pitch,
                                        float(lr), loss.data_ptr() if loss is not None else None,
                                        self._stream(stream)), self.ctx)

    def infer(self, img, threshold=0.5, flags=None, prob=None, stream=None):
        """Fused inference on one H x W x C image: flags (uint8) and/or prob."""
        import torch
        ip, h, w, c, pitch = _image_args(img)
        if flags is None and prob is None:
            flags = torch.empty((h, w), dtype=torch.uint8, device=img.device)
        _check(lib().vf_gate_infer(self.handle, ip, h, w, c, pitch, float(threshold),
                                   flags.data_ptr() if flags is not None else None,
                                   flags.stride(0) if flags is not None else 0,
                                   prob.data_ptr() if prob is not None else None,
                                   self._stream(stream)), self.ctx)
        return flags if prob is None else (flags, prob)

    def save(self, path):
        _check(lib().vf_gate_save(self.handle, str(path).encode()), self.ctx)

    def load(self, path):
        _check(lib().vf_gate_load(self.handle, str(path).encode()), self.ctx)

    def check(self):
        """vf_gate_check: raises VFError (VF_ERR_TIMEOUT) if a tensor-core wait
        of an inference since the last check gave up."""
        _check(lib().vf_gate_check(self.handle), self.ctx)

    @property
    def step(self):
        return lib().vf_gate_step_count(self.handle)

    def close(self):
        if self.handle:
            lib().vf_gate_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def filter_gated(inp, flags, out=None, *, stream=None, stats=None, **params):
    """vf_filter_gated: the window filter on flagged pixels, a copy elsewhere."""
    import torch
    if out is None:
        out = torch.empty_like(inp)
    ip, h, w, c, ipitch = _image_args(inp)
    op, _, _, _, opitch = _image_args(out)
    if flags.dtype != torch.uint8 or tuple(flags.shape) != (h, w) or flags.stride(1) != 1:
        raise ValueError("flags must be an H x W uint8 tensor with unit column stride")
    p = make_params(**params)
    s = stream if stream is not None else torch.cuda.current_stream(inp.device)
    ctx = context()
    _check(lib().vf_filter_gated(ctx, ip, op, h, w, c, ipitch, opitch, flags.data_ptr(),
                                 flags.stride(0), ctypes.byref(p), ctypes.c_void_p(s.cuda_stream),
                                 stats.data_ptr() if stats is not None else None), ctx)
    return out


STATIC_MAX_IMAGES = 256


def batch_run_static(images, stream=None) -> int:
    """vf_batch_run_static: the batched filter without any device allocation
    by the library (its scratch is a fixed array inside the library).  For
    callers that may not allocate GPU memory on their filtering path.
    images: list of (inp, out, params_dict) as for Batch.  Returns the status
    code (0 = VF_OK); no error text is recorded for this call."""
    import torch
    descs = (ImageDesc * max(len(images), 1))()
    for i, (inp, out, params) in enumerate(images):
        ip, h, w, c, ipitch = _image_args(inp)
        op, h2, w2, c2, opitch = _image_args(out)
        if (h, w, c) != (h2, w2, c2):
            raise ValueError("input and output shapes differ")
        d = descs[i]
        d.d_in, d.d_out, d.height, d.width, d.channels = ip, op, h, w, c
        d.in_pitch, d.out_pitch = ipitch, opitch
        d.params = make_params(**params)
    s = stream if stream is not None else torch.cuda.current_stream()
    return lib().vf_batch_run_static(context(), descs, len(images), ctypes.c_void_p(s.cuda_stream))


def filter_ptr(d_in: int, d_out: int, height: int, width: int, channels: int, in_pitch: int,
               out_pitch: int, stream_handle: int = 0, stats_ptr=None, **params):
    """vf_filter on raw device pointers (for tests of the ABI itself)."""
    p = make_params(**params)
    ctx = context()
    return lib().vf_filter(ctx, d_in, d_out, height, width, channels, in_pitch, out_pitch,
                           ctypes.byref(p), ctypes.c_void_p(stream_handle), stats_ptr)


def get_approximant(fn: str, approx: str = "poly", degree: int = 4, lo: float = 0.0,
                    hi: float = 1.0):
    """(num, den, eps) of the approximant the library evaluates (host)."""
    num = (ctypes.c_double * 8)()
    den = (ctypes.c_double * 8)()
    nl, dl = ctypes.c_int(), ctypes.c_int()
    eps = ctypes.c_double()
    ctx = context()
    _check(lib().vf_get_approximant(ctx, FUNCTIONS[fn], APPROX[approx], int(degree), float(lo),
                                    float(hi), num, ctypes.byref(nl), den, ctypes.byref(dl),
                                    ctypes.byref(eps)), ctx)
    return list(num[: nl.value]), list(den[: dl.value]), eps.value


def set_coefficients(fn: str, approx: str, degree: int, num=None, den=None, lo: float = 0.0,
                     hi: float = 1.0):
    """vf_set_coefficients: the caller's own approximant of `fn` (increasing
    powers) for every later call of this thread's context; num=None restores
    the library's fit."""
    ctx = context()
    if num is None:
        st = lib().vf_set_coefficients(ctx, FUNCTIONS[fn], APPROX[approx], int(degree), None, 0,
                                       None, 0, float(lo), float(hi))
    else:
        n = (ctypes.c_double * len(num))(*num)
        d = (ctypes.c_double * len(den))(*den) if den else None
        st = lib().vf_set_coefficients(ctx, FUNCTIONS[fn], APPROX[approx], int(degree), n,
                                       len(num), d, len(den) if den else 0, float(lo), float(hi))
    _check(st, ctx)


def row_quantum(**params) -> int:
    """vf_row_quantum: output rows per tile of the kernel vf_filter runs for
    these parameters (this thread's context options)."""
    p = make_params(**params)
    q = ctypes.c_int()
    ctx = context()
    _check(lib().vf_row_quantum(ctx, ctypes.byref(p), ctypes.byref(q)), ctx)
    return q.value


def band_plan(height: int, window: int, quantum: int, bands: int, band: int):
    """vf_band_plan: (in_row0, in_rows, out_row0, out_rows) of one row band."""
    v = [ctypes.c_int() for _ in range(4)]
    st = lib().vf_band_plan(int(height), int(window), int(quantum), int(bands), int(band),
                            *[ctypes.byref(x) for x in v])
    if st != 0:
        raise VFError(st, "vf_band_plan: bad arguments")
    return tuple(x.value for x in v)


def filter_band(host_img, band: int, bands: int, out=None, stream=None, **params):
    """One row band of a host image (H x W x C uint8 tensor, pinned or not):
    copies the band's input rows (with the halo) into device memory of the
    current GPU, filters them there with vf_filter and copies the band's
    output rows back into the rows [out_row0, out_row0 + out_rows) of the host
    tensor `out` (allocated when None).  Returns (out, out_row0, out_rows).
    Several processes, one per GPU, each filter their own band of an image
    in shared host memory; no data moves between the GPUs."""
    import torch
    H = host_img.shape[0]
    q = row_quantum(**params)
    a, n, r0, m = band_plan(H, params.get("window", 3), q, bands, band)
    if out is None:
        out = torch.empty_like(host_img)
    s = stream if stream is not None else torch.cuda.current_stream()
    with torch.cuda.stream(s):
        d_in = host_img[a:a + n].to("cuda", non_blocking=True)
        d_out = filter(d_in, stream=s, **params)
        out[r0:r0 + m].copy_(d_out[r0 - a:r0 - a + m], non_blocking=False)
    return out, r0, m


def debug_fail_alloc(after: int) -> int:
    """vf_debug_fail_alloc: fail the library's allocation after the next
    `after` ones (< 0 disarms); returns the previous setting."""
    return lib().vf_debug_fail_alloc(int(after))


def status_string(code: int) -> str:
    return lib().vf_status_string(int(code)).decode()
