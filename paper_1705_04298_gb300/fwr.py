"""Python binding of the C ABI in include/fwr.h (ctypes).

Argument marshalling only: every step of the reconstruction runs in the CUDA
library. PyTorch supplies device memory and streams; tensors are passed as raw
pointers with `tensor.data_ptr()` and the current stream's handle. If the
library has not been built this module raises on first use: there is no CPU
fallback.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfwr.so")

LSQ = 0
WIENER = 1
PERIODIC_BEFORE_EACH_FFT = 0
PERIODIC_FINAL_ONLY = 1
PERIODIC_NONE = 2
OPT_PERIODIC = 1
OPT_TRANSFORM = 2
OPT_G_MODEL = 3
OPT_PIXEL = 4
G_AVERAGED = 0
G_FRIED = 1
OPT_EXTENSION = 5
OPT_SHAPE = 6
OPT_CTAS = 7
OPT_L2_PERSIST = 8
EXT_ZERO = 0
EXT_HUDGIN = 1
TRANSFORM_FFT = 0
TRANSFORM_DFT_BF16X3 = 1
TRANSFORM_DFT_BF16X6 = 2
STATIC_SCRATCH_GRIDS = 16
NET_OPT_CONV = 1
NET_CONV_AUTO = 0
NET_CONV_SIMT = 1

STATUS = {0: "FWR_OK", 1: "FWR_ERR_ARG", 2: "FWR_ERR_UNSUPPORTED", 3: "FWR_ERR_CUDA",
          4: "FWR_ERR_NONFINITE", 5: "FWR_ERR_TIMEOUT"}

# Every symbol include/fwr.h declares, with its ctypes signature.
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
SIGNATURES = {
    "fwr_plan_create": (_I, [ctypes.POINTER(_P), _I, _D, _P, _I, _D, _D, _D]),
    "fwr_plan_create_grid": (_I, [ctypes.POINTER(_P), _I, _I, _P, _I, _D, _D, _D]),
    "fwr_plan_destroy": (None, [_P]),
    "fwr_plan_grid": (_I, [_P]),
    "fwr_plan_valid_count": (_I, [_P]),
    "fwr_plan_set_option": (_I, [_P, _I, _D]),
    "fwr_reconstruct": (_I, [_P, _P, _I, _I, _P, _P]),
    "fwr_reconstruct_ex": (_I, [_P, _P, _P, _I, _I, _P, _P, _P]),
    "fwr_reconstruct_f64": (_I, [_P, _P, _P, _I, _I, _P, _P, _P]),
    "fwr_reconstruct_host": (_I, [_P, _P, _I, _I, _P, _P]),
    "fwr_reconstruct_static": (_I, [_P, _P, _I, _I, _P, _I, _P]),
    "fwr_plan_reserve": (_I, [_P, _I]),
    "fwr_plan_autotune": (_I, [_P, _P, _I, _I, _P, _P, ctypes.c_char_p]),
    "fwr_plan_shape": (_I, [_P]),
    "fwr_plan_ctas": (_I, [_P]),
    "fwr_plan_l2_persist": (_I, [_P]),
    "fwr_l2_persist_reset": (_I, [_I]),
    "fwr_batch_shape": (_I, [_P]),
    "fwr_batch_set_shape": (_I, [_P, _I]),
    "fwr_fft2": (_I, [_I, _P, _P, _I, _I, _P]),
    "fwr_dft2_bf16x3": (_I, [_I, _P, _P, _I, _I, _P]),
    "fwr_batch_create": (_I, [ctypes.POINTER(_P), _P, _I, _P, _I, _I]),
    "fwr_batch_run": (_I, [_P, _P, _P, _P]),
    "fwr_batch_schedule": (_I, [_P, _I, _D]),
    "fwr_batch_autotune": (_I, [_P, _P, _P, _P, ctypes.c_char_p]),
    "fwr_batch_ctas": (_I, [_P]),
    "fwr_batch_cost_ratio": (_D, [_P]),
    "fwr_batch_destroy": (None, [_P]),
    "fwr_schedule_lpt": (_I, [_P, _I, _I, _P, _P]),
    "fwr_reconstruct_ragged": (_I, [_P, _I, _P, _P, _I, _I, _P, _P]),
    "fwr_ragged_release": (None, []),
    "fwr_net_create": (_I, [ctypes.POINTER(_P), _I, _I, _P, _I]),
    "fwr_net_destroy": (None, [_P]),
    "fwr_net_param_count": (_I, [_P]),
    "fwr_net_get_weights": (_I, [_P, _P, _I]),
    "fwr_net_set_weights": (_I, [_P, _P, _I]),
    "fwr_net_forward": (_I, [_P, _P, _P, _I, _P, _P]),
    "fwr_net_gradients": (_I, [_P, _P, _P, _P, _I, _P, _P, _P]),
    "fwr_net_train_step": (_I, [_P, _P, _P, _P, _I, ctypes.c_float, _P, _P]),
    "fwr_net_set_option": (_I, [_P, _I, _I]),
    "fwr_net_tc_layers": (_I, [_P]),
    "fwr_linws_create": (_I, [ctypes.POINTER(_P), _P, _I, _P, _P, _I]),
    "fwr_linws_destroy": (None, [_P]),
    "fwr_linws_valid_count": (_I, [_P]),
    "fwr_linws_forward": (_I, [_P, _P, _I, _P, _P]),
    "fwr_linws_reconstruct": (_I, [_P, _P, _P, _I, _I, _P, _P]),
    "fwr_linws_status": (_I, [_P]),
    "fwr_gemm_bf16_tc": (_I, [_P, _P, _I, _I, _I, _P, _P]),
    "fwr_gemm_bf16_tc_limit": (_I, [_P, _P, _I, _I, _I, _P, ctypes.c_longlong, _P]),
    "fwr_get_status": (_I, [_P]),
    "fwr_fp32_fma_peak": (_I, [_P, _P, _P]),
    "fwr_status_string": (ctypes.c_char_p, [_I]),
    "fwr_last_error": (ctypes.c_char_p, []),
}

_lib = None


class FwrError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = "%s failed: %s" % (where, STATUS.get(code, code))
        if code == 3 and _lib is not None:
            msg += " (%s)" % _lib.fwr_last_error().decode()
        super().__init__(msg)


def load(path=LIB_PATH):
    """Load libfwr.so and bind every declared symbol (raises if missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libfwr.so is not built (%s); run __graft_entry__.build() "
                           "or python -m paper_1705_04298_gb300.build_lib" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(code, where):
    if code != 0:
        raise FwrError(code, where)


# Argument marshalling is on every call's path (a call on an idle GPU waits
# for it), so it is kept lean: pointers and streams go to ctypes as plain
# integers (the argtypes convert them) and the checks are attribute compares.

def _ptr(t):
    return None if t is None else t.data_ptr()


def _stream(stream, device=None):
    """The raw handle of `stream`, or of the current stream of `device` (the
    current device when None)."""
    import torch
    if stream is not None:
        return stream.cuda_stream
    raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
    if raw is not None:  # the current stream without building a Stream object
        return raw(torch.cuda.current_device() if device is None else device)
    return torch.cuda.current_stream(device).cuda_stream


def _need(t, dtype, shape, name):
    if t is None:
        return
    try:
        ok = t.dtype == dtype and t.shape == shape and t.is_cuda and t.is_contiguous()
    except (AttributeError, TypeError):
        ok = False
    if not ok:
        if getattr(t, "dtype", None) != dtype or tuple(getattr(t, "shape", ())) != tuple(shape):
            raise ValueError("%s must be a %s tensor of shape %s" % (name, dtype, tuple(shape)))
        raise ValueError("%s must be a contiguous CUDA tensor" % name)


class Plan:
    """A reconstruction plan (fwr_plan_create): pupil, grid, filters.

    mask: (n, n) array-like of bool; r0 and L0 in lenslet pitches. grid: the
    grid size N itself (fwr_plan_create_grid: any even N in [16, 64] or a
    power of two up to 256) instead of the next power of two >= pad_factor n.
    """

    def __init__(self, mask, pad_factor=2.0, filter=LSQ, noise_var=0.0, r0=1.0, L0=100.0,
                 periodic=PERIODIC_BEFORE_EACH_FFT, grid=None):
        lib = load()
        m = np.ascontiguousarray(np.asarray(mask).astype(np.uint8))
        if m.ndim != 2 or m.shape[0] != m.shape[1]:
            raise ValueError("mask must be square")
        self.n = m.shape[0]
        self._lib = lib
        h = ctypes.c_void_p()
        if grid is None:
            _check(lib.fwr_plan_create(ctypes.byref(h), self.n, float(pad_factor),
                                       m.ctypes.data_as(ctypes.c_void_p), int(filter),
                                       float(noise_var), float(r0), float(L0)), "fwr_plan_create")
        else:
            _check(lib.fwr_plan_create_grid(ctypes.byref(h), self.n, int(grid),
                                            m.ctypes.data_as(ctypes.c_void_p), int(filter),
                                            float(noise_var), float(r0), float(L0)), "fwr_plan_create_grid")
        self._h = h
        self.N = lib.fwr_plan_grid(h)
        self.valid_count = lib.fwr_plan_valid_count(h)
        self.set_periodic(periodic)

    def set_periodic(self, mode):
        _check(self._lib.fwr_plan_set_option(self._h, OPT_PERIODIC, float(mode)), "fwr_plan_set_option")
        self.periodic = mode

    def set_model(self, g_model=G_AVERAGED, pixel=0.0):
        """Measurement model of the filter tables: G_AVERAGED or G_FRIED and
        d_px / d in [0, 0.5]; rebuilds the tables (synchronises the device)."""
        _check(self._lib.fwr_plan_set_option(self._h, OPT_G_MODEL, float(g_model)), "fwr_plan_set_option")
        _check(self._lib.fwr_plan_set_option(self._h, OPT_PIXEL, float(pixel)), "fwr_plan_set_option")

    def set_extension(self, mode):
        """EXT_ZERO (default) or EXT_HUDGIN: the slopes outside the pupil
        before the first iteration when no warm start is given."""
        _check(self._lib.fwr_plan_set_option(self._h, OPT_EXTENSION, float(mode)), "fwr_plan_set_option")

    def set_shape(self, shape):
        """Launch shape (FWR_OPT_SHAPE, 0..2; bitwise the same result)."""
        _check(self._lib.fwr_plan_set_option(self._h, OPT_SHAPE, float(shape)), "fwr_plan_set_option")

    def set_l2_persist(self, on):
        """FWR_OPT_L2_PERSIST: keep the slab kernel's working memory persisting in
        L2 (256^2 / 512^2 plans; raises the process's persisting-L2 set-aside)."""
        _check(self._lib.fwr_plan_set_option(self._h, OPT_L2_PERSIST, float(bool(on))), "fwr_plan_set_option")

    def set_ctas(self, ctas):
        """Persistent CTAs of a launch (FWR_OPT_CTAS; 0 = every SM)."""
        _check(self._lib.fwr_plan_set_option(self._h, OPT_CTAS, float(ctas)), "fwr_plan_set_option")

    @property
    def shape(self):
        return self._lib.fwr_plan_shape(self._h)

    @property
    def ctas(self):
        return self._lib.fwr_plan_ctas(self._h)

    @property
    def l2_persist(self):
        return self._lib.fwr_plan_l2_persist(self._h)

    def autotune(self, slopes, iters, phase, cache_path=None, stream=None):
        """Time the launch shapes on these frames and keep the fastest
        (fwr_plan_autotune); returns (shape, ctas)."""
        import torch
        F = slopes.shape[0]
        _need(slopes, torch.float32, (F, 2, self.n, self.n), "slopes")
        _need(phase, torch.float32, (F, self.N, self.N), "phase")
        path = None if cache_path is None else str(cache_path).encode()
        _check(self._lib.fwr_plan_autotune(self._h, _ptr(slopes), F, int(iters), _ptr(phase), _stream(stream), path),
               "fwr_plan_autotune")
        return self.shape, self.ctas

    def set_transform(self, mode):
        """TRANSFORM_FFT (default) or TRANSFORM_DFT_BF16X3 (tensor-core split-BF16
        DFT: per-frame products for N = 32/64, batched tcgen05 GEMMs for N =
        128/256, whose workspace this call allocates)."""
        _check(self._lib.fwr_plan_set_option(self._h, OPT_TRANSFORM, float(mode)), "fwr_plan_set_option")
        self.transform = mode

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fwr_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reconstruct(self, slopes, iters, phase=None, ext_init=None, ext_out=None, stream=None):
        """FP32 path (fwr_reconstruct_ex). slopes: (F, 2, n, n) float32 CUDA.
        Returns the phase tensor (F, N, N) (allocated when not given)."""
        import torch
        F = slopes.shape[0]
        n, N = self.n, self.N
        _need(slopes, torch.float32, (F, 2, n, n), "slopes")
        if phase is None:
            phase = torch.empty((F, N, N), dtype=torch.float32, device=slopes.device)
        _need(phase, torch.float32, (F, N, N), "phase")
        _need(ext_init, torch.float32, (F, 2, N, N), "ext_init")
        _need(ext_out, torch.float32, (F, 2, N, N), "ext_out")
        _check(self._lib.fwr_reconstruct_ex(self._h, _ptr(slopes), _ptr(ext_init), F, int(iters),
                                            _ptr(phase), _ptr(ext_out), _stream(stream, slopes.device.index)),
               "fwr_reconstruct_ex")
        return phase

    def reconstruct_f64(self, slopes, iters, phase=None, ext_init=None, ext_out=None, stream=None):
        """FP64 path (fwr_reconstruct_f64), N <= 64."""
        import torch
        F = slopes.shape[0]
        n, N = self.n, self.N
        _need(slopes, torch.float64, (F, 2, n, n), "slopes")
        if phase is None:
            phase = torch.empty((F, N, N), dtype=torch.float64, device=slopes.device)
        _need(phase, torch.float64, (F, N, N), "phase")
        _need(ext_init, torch.float64, (F, 2, N, N), "ext_init")
        _need(ext_out, torch.float64, (F, 2, N, N), "ext_out")
        _check(self._lib.fwr_reconstruct_f64(self._h, _ptr(slopes), _ptr(ext_init), F, int(iters),
                                             _ptr(phase), _ptr(ext_out), _stream(stream)),
               "fwr_reconstruct_f64")
        return phase

    def reconstruct_static(self, slopes, iters, phase=None, ctas=STATIC_SCRATCH_GRIDS, stream=None):
        """256x256 grids without any device allocation (fwr_reconstruct_static):
        the working memory is the library's own static array, shared by every
        call on the device, so calls must not overlap on the GPU."""
        import torch
        F = slopes.shape[0]
        n, N = self.n, self.N
        _need(slopes, torch.float32, (F, 2, n, n), "slopes")
        if phase is None:
            phase = torch.empty((F, N, N), dtype=torch.float32, device=slopes.device)
        _need(phase, torch.float32, (F, N, N), "phase")
        _check(self._lib.fwr_reconstruct_static(self._h, _ptr(slopes), F, int(iters), _ptr(phase), int(ctas),
                                                _stream(stream)), "fwr_reconstruct_static")
        return phase

    def reserve(self, n_frames):
        _check(self._lib.fwr_plan_reserve(self._h, int(n_frames)), "fwr_plan_reserve")

    def reconstruct_host(self, slopes_host, iters, phase_host, stream=None):
        """End-to-end call on host tensors (pinned for asynchronous copies):
        slopes_host (F, 2, n, n) float32 CPU, phase_host (F, N, N) float32 CPU.
        Ordered on `stream`: the copies of later and earlier chunks overlap the
        reconstruction of the current one on the plan's copy streams."""
        import torch
        F = slopes_host.shape[0]
        for t, shp, name in ((slopes_host, (F, 2, self.n, self.n), "slopes_host"),
                             (phase_host, (F, self.N, self.N), "phase_host")):
            if t.dtype != torch.float32 or tuple(t.shape) != shp or t.is_cuda or not t.is_contiguous():
                raise ValueError("%s must be a contiguous float32 CPU tensor of shape %s" % (name, shp))
        _check(self._lib.fwr_reconstruct_host(self._h, _ptr(slopes_host), F, int(iters),
                                              _ptr(phase_host), _stream(stream)),
               "fwr_reconstruct_host")
        return phase_host

    def status(self):
        """Read and clear the sticky device status (synchronises)."""
        return STATUS.get(self._lib.fwr_get_status(self._h))


def reconstruct_ragged(plans, frame_plan, slopes_ptrs, phase_ptrs, iters, stream=None):
    """One-call ragged reconstruction (fwr_reconstruct_ragged): frame f through
    plans[frame_plan[f]], one launch. frame_plan: int32 CUDA tensor (n_frames);
    slopes_ptrs / phase_ptrs: int64 CUDA tensors of per-frame device pointers
    (Batch.pointer_table). The schedule is built on the first call for these
    arguments and kept until ragged_release()."""
    import torch
    lib = load()
    if not (isinstance(frame_plan, torch.Tensor) and frame_plan.is_cuda and frame_plan.dtype == torch.int32
            and frame_plan.is_contiguous() and frame_plan.dim() == 1):
        raise ValueError("frame_plan must be a contiguous 1-D int32 CUDA tensor")
    F = frame_plan.shape[0]
    for t, name in ((slopes_ptrs, "slopes_ptrs"), (phase_ptrs, "phase_ptrs")):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.int64 and tuple(t.shape) == (F,)):
            raise ValueError("%s must be an int64 CUDA tensor of %d pointers" % (name, F))
    arr = (ctypes.c_void_p * len(plans))(*[p._h.value for p in plans])
    _check(lib.fwr_reconstruct_ragged(ctypes.cast(arr, ctypes.c_void_p), len(plans), _ptr(frame_plan),
                                      _ptr(slopes_ptrs), F, int(iters), _ptr(phase_ptrs), _stream(stream)),
           "fwr_reconstruct_ragged")


def ragged_release():
    """Free the schedules kept by reconstruct_ragged (fwr_ragged_release)."""
    load().fwr_ragged_release()


class Batch:
    """A ragged batch (fwr_batch_*): frames of several plans, one launch.

    plans: list of Plan; frame_plan: sequence of plan indices, one per frame.
    """

    def __init__(self, plans, frame_plan, iters):
        lib = load()
        self._lib = lib
        self.plans = list(plans)  # the plans must outlive the batch
        fp = np.ascontiguousarray(np.asarray(frame_plan, dtype=np.int32))
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib.fwr_batch_create(ctypes.byref(h), ctypes.cast(arr, ctypes.c_void_p), len(self.plans),
                                    fp.ctypes.data_as(ctypes.c_void_p), len(fp), int(iters)), "fwr_batch_create")
        self._h = h
        self.frame_plan = fp
        self.iters = int(iters)

    @staticmethod
    def pointer_table(tensors, device="cuda"):
        """Device array of the tensors' data pointers (int64)."""
        import torch
        return torch.tensor([t.data_ptr() for t in tensors], dtype=torch.int64, device=device)

    def run(self, slopes_ptrs, phase_ptrs, stream=None):
        """slopes_ptrs / phase_ptrs: int64 CUDA tensors of per-frame device pointers."""
        _check(self._lib.fwr_batch_run(self._h, _ptr(slopes_ptrs), _ptr(phase_ptrs), _stream(stream)),
               "fwr_batch_run")

    def schedule(self, ctas, cost_ratio):
        _check(self._lib.fwr_batch_schedule(self._h, int(ctas), float(cost_ratio)), "fwr_batch_schedule")

    def autotune(self, slopes_ptrs, phase_ptrs, cache_path=None, stream=None):
        path = None if cache_path is None else str(cache_path).encode()
        _check(self._lib.fwr_batch_autotune(self._h, _ptr(slopes_ptrs), _ptr(phase_ptrs), _stream(stream), path),
               "fwr_batch_autotune")
        return self.ctas, self.cost_ratio

    @property
    def ctas(self):
        return self._lib.fwr_batch_ctas(self._h)

    @property
    def shape(self):
        return self._lib.fwr_batch_shape(self._h)

    def set_shape(self, shape):
        _check(self._lib.fwr_batch_set_shape(self._h, int(shape)), "fwr_batch_set_shape")

    @property
    def cost_ratio(self):
        return self._lib.fwr_batch_cost_ratio(self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fwr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """The warm-start U-Net (fwr_net_*): width w, largest batch, optional
    initial weights (flat FP32 vector, layer by layer, W[cout][dy][dx][cin]
    then bias)."""

    def __init__(self, width, max_batch, weights=None):
        lib = load()
        self._lib = lib
        h = ctypes.c_void_p()
        if weights is None:
            _check(lib.fwr_net_create(ctypes.byref(h), int(width), int(max_batch), None, 0), "fwr_net_create")
        else:
            w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
            _check(lib.fwr_net_create(ctypes.byref(h), int(width), int(max_batch),
                                      w.ctypes.data_as(ctypes.c_void_p), len(w)), "fwr_net_create")
        self._h = h
        self.width = int(width)
        self.max_batch = int(max_batch)
        self.param_count = lib.fwr_net_param_count(h)

    def weights(self):
        w = np.empty(self.param_count, dtype=np.float32)
        _check(self._lib.fwr_net_get_weights(self._h, w.ctypes.data_as(ctypes.c_void_p), len(w)),
               "fwr_net_get_weights")
        return w

    def set_weights(self, weights):
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.float32))
        _check(self._lib.fwr_net_set_weights(self._h, w.ctypes.data_as(ctypes.c_void_p), len(w)),
               "fwr_net_set_weights")

    def forward(self, plan, slopes, ext_init=None, stream=None):
        """slopes (F, 2, n, n) float32 CUDA -> warm start (F, 2, 128, 128)."""
        import torch
        F = slopes.shape[0]
        _need(slopes, torch.float32, (F, 2, plan.n, plan.n), "slopes")
        if ext_init is None:
            ext_init = torch.empty((F, 2, plan.N, plan.N), dtype=torch.float32, device=slopes.device)
        _need(ext_init, torch.float32, (F, 2, plan.N, plan.N), "ext_init")
        _check(self._lib.fwr_net_forward(self._h, plan._h, _ptr(slopes), F, _ptr(ext_init), _stream(stream)),
               "fwr_net_forward")
        return ext_init

    def gradients(self, plan, slopes, target_ext, stream=None):
        """(loss, gradient as a flat float32 array) at the current weights."""
        import torch
        F = slopes.shape[0]
        _need(slopes, torch.float32, (F, 2, plan.n, plan.n), "slopes")
        _need(target_ext, torch.float32, (F, 2, plan.N, plan.N), "target_ext")
        g = np.empty(self.param_count, dtype=np.float32)
        loss = ctypes.c_float()
        _check(self._lib.fwr_net_gradients(self._h, plan._h, _ptr(slopes), _ptr(target_ext), F,
                                           g.ctypes.data_as(ctypes.c_void_p), ctypes.byref(loss), _stream(stream)),
               "fwr_net_gradients")
        return float(loss.value), g

    def train_step(self, plan, slopes, target_ext, lr, stream=None):
        import torch
        F = slopes.shape[0]
        _need(slopes, torch.float32, (F, 2, plan.n, plan.n), "slopes")
        _need(target_ext, torch.float32, (F, 2, plan.N, plan.N), "target_ext")
        loss = ctypes.c_float()
        _check(self._lib.fwr_net_train_step(self._h, plan._h, _ptr(slopes), _ptr(target_ext), F, float(lr),
                                            ctypes.byref(loss), _stream(stream)), "fwr_net_train_step")
        return float(loss.value)

    def set_conv(self, mode):
        """NET_CONV_AUTO (tensor-core forward where the layer allows it) or
        NET_CONV_SIMT."""
        _check(self._lib.fwr_net_set_option(self._h, NET_OPT_CONV, int(mode)), "fwr_net_set_option")

    @property
    def tc_layers(self):
        return self._lib.fwr_net_tc_layers(self._h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fwr_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def schedule_lpt(costs, ctas):
    """Host-only LPT schedule (fwr_schedule_lpt): returns (cta_off, order)."""
    lib = load()
    c = np.ascontiguousarray(np.asarray(costs, dtype=np.float64))
    off = np.zeros(int(ctas) + 1, dtype=np.int32)
    order = np.zeros(max(1, len(c)), dtype=np.int32)
    _check(lib.fwr_schedule_lpt(c.ctypes.data_as(ctypes.c_void_p), len(c), int(ctas),
                                off.ctypes.data_as(ctypes.c_void_p), order.ctypes.data_as(ctypes.c_void_p)),
           "fwr_schedule_lpt")
    return off, order[:len(c)]


class LinearWarmStart:
    """Rank-r linear warm start (fwr_linws_*): ext_init = (X A) V^T on the
    tcgen05 tensor cores, X the measured slopes of the plan's valid cells
    (x slopes, then y slopes, row-major cell order). A: (2 n_valid, r), V:
    (2 N^2, r), float arrays, r a multiple of 128."""

    def __init__(self, plan, A, V, max_batch):
        lib = load()
        self._lib = lib
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float32))
        V = np.ascontiguousarray(np.asarray(V, dtype=np.float32))
        if A.ndim != 2 or V.ndim != 2 or A.shape[1] != V.shape[1]:
            raise ValueError("A (2 n_valid, r) and V (2 N^2, r) must share r")
        if A.shape[0] != 2 * plan.valid_count or V.shape[0] != 2 * plan.N * plan.N:
            raise ValueError("A must have 2 n_valid rows and V 2 N^2 rows")
        h = ctypes.c_void_p()
        _check(lib.fwr_linws_create(ctypes.byref(h), plan._h, int(A.shape[1]), A.ctypes.data_as(_P),
                                    V.ctypes.data_as(_P), int(max_batch)), "fwr_linws_create")
        self._h = h
        self.plan = plan
        self.rank = int(A.shape[1])
        self.max_batch = int(max_batch)

    def forward(self, slopes, ext_init=None, stream=None):
        """slopes (F, 2, n, n) float32 CUDA -> ext_init (F, 2, N, N) float32."""
        import torch
        F = slopes.shape[0]
        _need(slopes, torch.float32, (F, 2, self.plan.n, self.plan.n), "slopes")
        if ext_init is None:
            ext_init = torch.empty((F, 2, self.plan.N, self.plan.N), dtype=torch.float32, device=slopes.device)
        _need(ext_init, torch.float32, (F, 2, self.plan.N, self.plan.N), "ext_init")
        _check(self._lib.fwr_linws_forward(self._h, _ptr(slopes), F, _ptr(ext_init), _stream(stream)),
               "fwr_linws_forward")
        return ext_init

    def reconstruct(self, slopes, iters, phase=None, plan=None, stream=None):
        """Warm start + `iters` Gerchberg iterations + final filter
        (fwr_linws_reconstruct), the warm start kept in BF16. plan: the one
        given at creation unless another with the same pupil and grid."""
        import torch
        plan = self.plan if plan is None else plan
        F = slopes.shape[0]
        _need(slopes, torch.float32, (F, 2, plan.n, plan.n), "slopes")
        if phase is None:
            phase = torch.empty((F, plan.N, plan.N), dtype=torch.float32, device=slopes.device)
        _need(phase, torch.float32, (F, plan.N, plan.N), "phase")
        _check(self._lib.fwr_linws_reconstruct(self._h, plan._h, _ptr(slopes), F, int(iters), _ptr(phase),
                                               _stream(stream)), "fwr_linws_reconstruct")
        return phase

    def status(self):
        _check(self._lib.fwr_linws_status(self._h), "fwr_linws_status")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fwr_linws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def l2_persist_reset(device=0):
    """Give the whole L2 back to other work: lines that FWR_OPT_L2_PERSIST
    launches left persisting return to normal, and the persisting set-aside to
    its value before the library raised it (fwr_l2_persist_reset)."""
    _check(load().fwr_l2_persist_reset(int(device)), "fwr_l2_persist_reset")


def fp32_fma_peak(stream=None):
    """Measured FP32 FMA throughput of the current device (fwr_fp32_fma_peak):
    (TFLOP/s, ms per timed launch)."""
    lib = load()
    t = ctypes.c_double()
    ms = ctypes.c_double()
    _check(lib.fwr_fp32_fma_peak(ctypes.byref(t), ctypes.byref(ms), _stream(stream)), "fwr_fp32_fma_peak")
    return t.value, ms.value


def gemm_bf16_tc(A, B, out=None, stream=None, wait_cycles=None):
    """D = A B^T (fwr_gemm_bf16_tc): A (M, K), B (N, K) bfloat16 CUDA tensors,
    K a multiple of 8, N of 128; D float32 (M, N). wait_cycles: bound of the
    issuer's and epilogue's waits (fwr_gemm_bf16_tc_limit; for timeout tests)."""
    import torch
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16 or A.dim() != 2 or B.dim() != 2:
        raise ValueError("A and B must be 2-D bfloat16 tensors")
    if A.shape[1] != B.shape[1] or not A.is_cuda or not B.is_cuda:
        raise ValueError("A (M, K) and B (N, K) must be CUDA tensors with the same K")
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    if out is None:
        out = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _need(out, torch.float32, (M, N), "out")
    lib = load()
    if wait_cycles is None:
        _check(lib.fwr_gemm_bf16_tc(_ptr(A), _ptr(B), int(M), int(N), int(K), _ptr(out), _stream(stream)),
               "fwr_gemm_bf16_tc")
    else:
        _check(lib.fwr_gemm_bf16_tc_limit(_ptr(A), _ptr(B), int(M), int(N), int(K), _ptr(out), int(wait_cycles),
                                          _stream(stream)), "fwr_gemm_bf16_tc_limit")
    return out


def dft2_bf16x3(x, inverse=False, out=None, stream=None):
    """Batched 2-D DFT (fwr_dft2_bf16x3) of a (F, N, N) complex64 CUDA tensor,
    N in {32, 64}, through split-BF16 tensor-core products; no scaling."""
    import torch
    if x.dtype != torch.complex64 or x.dim() != 3 or x.shape[1] != x.shape[2] or not x.is_cuda:
        raise ValueError("x must be a (F, N, N) complex64 CUDA tensor")
    x = x.contiguous()
    if out is None:
        out = torch.empty_like(x)
    lib = load()
    _check(lib.fwr_dft2_bf16x3(int(x.shape[1]), _ptr(x), _ptr(out), int(x.shape[0]), int(bool(inverse)),
                               _stream(stream)), "fwr_dft2_bf16x3")
    return out


def fft2(x, inverse=False, out=None, stream=None):
    """Batched 2-D FFT (fwr_fft2) of a (F, N, N) complex64 CUDA tensor; no
    1/N^2 scaling on the inverse."""
    import torch
    if x.dtype != torch.complex64 or x.dim() != 3 or x.shape[1] != x.shape[2] or not x.is_cuda:
        raise ValueError("x must be a (F, N, N) complex64 CUDA tensor")
    x = x.contiguous()
    if out is None:
        out = torch.empty_like(x)
    lib = load()
    _check(lib.fwr_fft2(int(x.shape[1]), _ptr(x), _ptr(out), int(x.shape[0]), int(bool(inverse)),
                        _stream(stream)), "fwr_fft2")
    return out
