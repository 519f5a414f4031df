"""Python binding of libse2n, the C ABI declared in include/se2n.h.

Argument marshalling only: every function here has the name of the C entry
point it calls, turns torch CUDA tensors into device pointers and streams
into cudaStream_t handles, and raises Se2nError on a non-OK status. All
computation happens in the CUDA library; if the library is missing, loading
this module fails (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libse2n.so")

SE2N_OK = 0
SE2N_EINVAL = 1
SE2N_ENOMEM = 2
SE2N_ECUDA = 3
SE2N_ECUFFT = 4
SE2N_EUNSUPPORTED = 5
SE2N_ENUMERIC = 6
SE2N_BIN_FLAT = 255
SE2N_PROJ_MAX = 0
SE2N_PROJ_MEAN = 1
SE2N_DIFFUSE_SM_FP64 = 1
SE2N_DIFFUSE_SPLIT_DIAG = 2
SE2N_DIFFUSE_FULL_CORRECTION = 4
SE2N_DIFFUSE_PROPAGATOR = 8
SE2N_MAX_N = 64
SE2N_BATCH_AUTOTUNE = 1
SE2N_NOALLOC_MAX_VOLUMES = 64
SE2N_NOALLOC_SCRATCH_BYTES = 8192


class Se2nError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {se2n_status_string(status)} (status {status})")


SE2N_STAGES = ("orient", "lift", "fft", "diffuse", "mix", "project", "dr", "propagator")


class se2n_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(SE2N_STAGES)), ("calls", ctypes.c_longlong * len(SE2N_STAGES)),
                ("kernels", ctypes.c_longlong)]


class se2n_image_desc(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("bins", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("N", ctypes.c_int)]


class se2n_volume_desc(ctypes.Structure):
    _fields_ = [("vol_hat", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("N", ctypes.c_int)]


class se2n_batch_info(ctypes.Structure):
    _fields_ = [("images", ctypes.c_int), ("items", ctypes.c_int), ("tile_passes", ctypes.c_int),
                ("block", ctypes.c_int), ("blocks", ctypes.c_int), ("p16", ctypes.c_int), ("p32", ctypes.c_int),
                ("p64", ctypes.c_int), ("fast", ctypes.c_int), ("split", ctypes.c_int),
                ("candidates", ctypes.c_int), ("best_ms", ctypes.c_double), ("worst_ms", ctypes.c_double),
                ("updates_per_run", ctypes.c_double), ("volume_bytes", ctypes.c_double),
                ("prop_images", ctypes.c_int), ("step_updates", ctypes.c_double),
                ("fused_images", ctypes.c_int)]


class se2n_params(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int),
        ("beta", ctypes.c_double),
        ("T", ctypes.c_double),
        ("steps", ctypes.c_int),
        ("rounds", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("sigma_smooth", ctypes.c_double),
        ("flat_tol", ctypes.c_double),
        ("proj", ctypes.c_int),
        ("final_mix", ctypes.c_int),
        ("guard", ctypes.c_double),
        ("diffuse_flags", ctypes.c_int),
        ("reinject", ctypes.c_int),
        ("full_spectrum", ctypes.c_int),
        ("dynamic", ctypes.c_int),
    ]


_P = ctypes.c_void_p
_SIGS = {
    "se2n_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "se2n_params_default": (ctypes.c_int, [ctypes.POINTER(se2n_params)]),
    "se2n_params_from_paper": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "se2n_prop_chain": (ctypes.c_int, [ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_int)]),
    "se2n_plan_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _P]),
    "se2n_plan_destroy": (ctypes.c_int, [_P]),
    "se2n_plan_set_stream": (ctypes.c_int, [_P, _P]),
    "se2n_plan_last_cuda_error": (ctypes.c_int, [_P]),
    "se2n_orient": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_double, _P]),
    "se2n_lift": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "se2n_forward": (ctypes.c_int, [_P, _P]),
    "se2n_inverse": (ctypes.c_int, [_P, _P]),
    "se2n_diffuse": (ctypes.c_int, [_P, _P, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    "se2n_mix": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_double]),
    "se2n_dr_grow": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "se2n_plan_drop_propagators": (ctypes.c_int, [_P, ctypes.c_int]),
    "se2n_project": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "se2n_inpaint": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(se2n_params), _P, _P]),
    "se2n_inpaint_host": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(se2n_params), _P]),
    "se2n_plan_tune_diffuse": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "se2n_plan_profile": (ctypes.c_int, [_P, ctypes.c_int]),
    "se2n_plan_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(se2n_profile), ctypes.c_int]),
    "se2n_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(se2n_image_desc), ctypes.c_int,
                                         ctypes.POINTER(se2n_params), ctypes.c_int, ctypes.c_int, _P]),
    "se2n_batch_run": (ctypes.c_int, [_P]),
    "se2n_batch_run_per_image": (ctypes.c_int, [_P]),
    "se2n_batch_run_diffusion": (ctypes.c_int, [_P]),
    "se2n_batch_get_info": (ctypes.c_int, [_P, ctypes.POINTER(se2n_batch_info)]),
    "se2n_batch_destroy": (ctypes.c_int, [_P]),
    "se2n_diffuse_rows": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int]),
    "se2n_mix_given": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_double, ctypes.c_double]),
    "se2n_diffuse_many_noalloc": (ctypes.c_int, [ctypes.POINTER(se2n_volume_desc), ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "se2n_unet_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "se2n_unet_destroy": (ctypes.c_int, [_P]),
    "se2n_unet_param_count": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "se2n_unet_init": (ctypes.c_int, [_P, ctypes.c_ulonglong]),
    "se2n_unet_set_params": (ctypes.c_int, [_P, _P]),
    "se2n_unet_get_params": (ctypes.c_int, [_P, _P]),
    "se2n_unet_get_grads": (ctypes.c_int, [_P, _P]),
    "se2n_unet_forward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "se2n_unet_backward": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, _P]),
    "se2n_unet_adam": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "se2n_unet_train_step": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_double, _P]),
    "se2n_surrogate_inpaint": (ctypes.c_int, [_P, _P, ctypes.POINTER(se2n_params), _P, _P, ctypes.c_int,
                                              ctypes.c_double, _P, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "se2n_plan_diffuse_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                              ctypes.POINTER(ctypes.c_int)]),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libse2n.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                          "or python paper_1304_2062_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _check(status, where):
    if status != SE2N_OK:
        raise Se2nError(status, where)


def _ptr(x):
    """Device (or host) address of a tensor, a numpy array or a raw int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def se2n_status_string(status):
    return lib.se2n_status_string(int(status)).decode()


def se2n_params_default(**overrides):
    p = se2n_params()
    _check(lib.se2n_params_default(ctypes.byref(p)), "se2n_params_default")
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def se2n_params_from_paper(alpha, T_paper, M, N):
    b = ctypes.c_double()
    t = ctypes.c_double()
    _check(lib.se2n_params_from_paper(alpha, T_paper, M, N, ctypes.byref(b), ctypes.byref(t)),
           "se2n_params_from_paper")
    return b.value, t.value


PROP_CHAIN_MAX = 64
PROP_SQ_P, PROP_SQ_R, PROP_ADD, PROP_COPY = 0, 1, 2, 3


def se2n_prop_chain(steps):
    """The propagator build's powering program for S = steps: (ops, in_r),
    ops a list of PROP_* codes on P (starting as D_1) and R."""
    buf = (ctypes.c_ubyte * PROP_CHAIN_MAX)()
    n = ctypes.c_int()
    in_r = ctypes.c_int()
    _check(lib.se2n_prop_chain(steps, buf, PROP_CHAIN_MAX, ctypes.byref(n), ctypes.byref(in_r)), "se2n_prop_chain")
    return list(buf[:n.value]), in_r.value


class Plan:
    """Owns an se2n_plan*; destroyed on close() or garbage collection."""

    def __init__(self, handle, H, W, N, angle_conv):
        self.handle = handle
        self.H, self.W, self.N, self.angle_conv = H, W, N, angle_conv

    def close(self):
        if self.handle:
            lib.se2n_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _as_parameter_(self):
        return self.handle


def se2n_plan_create(H, W, N, angle_conv=0, stream=None):
    h = _P()
    _check(lib.se2n_plan_create(ctypes.byref(h), H, W, N, angle_conv, _stream(stream)), "se2n_plan_create")
    return Plan(h.value, H, W, N, angle_conv)


def se2n_plan_destroy(plan):
    plan.close()


def se2n_plan_set_stream(plan, stream):
    _check(lib.se2n_plan_set_stream(plan.handle, _stream(stream)), "se2n_plan_set_stream")


def se2n_plan_last_cuda_error(plan):
    return lib.se2n_plan_last_cuda_error(plan.handle)


def se2n_orient(plan, f, mask, sigma, flat_tol, bins):
    _check(lib.se2n_orient(plan.handle, _ptr(f), _ptr(mask), sigma, flat_tol, _ptr(bins)), "se2n_orient")


def se2n_lift(plan, f, mask, bins, vol):
    _check(lib.se2n_lift(plan.handle, _ptr(f), _ptr(mask), _ptr(bins), _ptr(vol)), "se2n_lift")


def se2n_forward(plan, vol):
    _check(lib.se2n_forward(plan.handle, _ptr(vol)), "se2n_forward")


def se2n_inverse(plan, vol):
    _check(lib.se2n_inverse(plan.handle, _ptr(vol)), "se2n_inverse")


def se2n_diffuse(plan, vol_hat, beta, T, steps, flags=0):
    _check(lib.se2n_diffuse(plan.handle, _ptr(vol_hat), beta, T, steps, flags), "se2n_diffuse")


def se2n_diffuse_rows(plan, vol_rows, k0, beta, T, steps, flags=0):
    """vol_rows: complex64 device tensor [N][rows][W], spectrum rows k0 .. k0 + rows - 1."""
    _check(lib.se2n_diffuse_rows(plan.handle, _ptr(vol_rows), k0, vol_rows.shape[1], beta, T, steps, flags),
           "se2n_diffuse_rows")


def se2n_mix_given(plan, vol, f, mask, bins, h_t, eps, guard=0.1):
    _check(lib.se2n_mix_given(plan.handle, _ptr(vol), _ptr(f), _ptr(mask), _ptr(bins), _ptr(h_t), eps, guard),
           "se2n_mix_given")


def se2n_mix(plan, vol, f, mask, bins, eps, guard=0.1):
    _check(lib.se2n_mix(plan.handle, _ptr(vol), _ptr(f), _ptr(mask), _ptr(bins), eps, guard), "se2n_mix")


def se2n_plan_drop_propagators(plan, free_memory=False):
    _check(lib.se2n_plan_drop_propagators(plan.handle, 1 if free_memory else 0), "se2n_plan_drop_propagators")


def se2n_dr_grow(plan, vol, mask_in, mask_out, fref, bins):
    _check(lib.se2n_dr_grow(plan.handle, _ptr(vol), _ptr(mask_in), _ptr(mask_out), _ptr(fref), _ptr(bins)),
           "se2n_dr_grow")


def se2n_project(plan, vol, proj, out):
    _check(lib.se2n_project(plan.handle, _ptr(vol), proj, _ptr(out)), "se2n_project")


def se2n_inpaint(plan, f, mask, bins_in, params, vol, out):
    _check(lib.se2n_inpaint(plan.handle, _ptr(f), _ptr(mask), _ptr(bins_in), ctypes.byref(params), _ptr(vol),
                            _ptr(out)), "se2n_inpaint")


def se2n_inpaint_host(plan, f_host, mask_host, params, out_host):
    _check(lib.se2n_inpaint_host(plan.handle, _ptr(f_host), _ptr(mask_host), ctypes.byref(params),
                                 _ptr(out_host)), "se2n_inpaint_host")


def se2n_plan_tune_diffuse(plan, threads_per_freq=0, block_threads=0, blocks=0):
    _check(lib.se2n_plan_tune_diffuse(plan.handle, threads_per_freq, block_threads, blocks),
           "se2n_plan_tune_diffuse")


def se2n_plan_diffuse_info(plan):
    r, b, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib.se2n_plan_diffuse_info(plan.handle, ctypes.byref(r), ctypes.byref(b), ctypes.byref(p)),
           "se2n_plan_diffuse_info")
    return dict(regs_per_thread=r.value, blocks_per_sm=b.value, threads_per_freq=p.value)


def se2n_plan_profile(plan, enable=True):
    _check(lib.se2n_plan_profile(plan.handle, 1 if enable else 0), "se2n_plan_profile")


def se2n_plan_profile_read(plan, reset=False):
    """Accumulated stage times: {stage: (ms, calls)} plus the own-kernel launch count."""
    prof = se2n_profile()
    _check(lib.se2n_plan_profile_read(plan.handle, ctypes.byref(prof), 1 if reset else 0), "se2n_plan_profile_read")
    out = {name: (prof.ms[i], prof.calls[i]) for i, name in enumerate(SE2N_STAGES)}
    out["kernels"] = prof.kernels
    return out


class Batch:
    """Owns an se2n_batch*; keeps the image descriptors' buffers alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def close(self):
        if self.handle:
            lib.se2n_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def se2n_batch_create(images, params, angle_conv=0, flags=0, stream=None):
    """images: sequence of (f, mask, out, N) or (f, mask, out, N, bins) with
    device tensors f [H][W] float32, mask [H][W] uint8, out [H][W] float32 and
    optionally bins [H][W] uint8."""
    descs = (se2n_image_desc * len(images))()
    keep = []
    for i, img in enumerate(images):
        f, mask, out, N = img[:4]
        bins = img[4] if len(img) > 4 else None
        H, W = f.shape
        descs[i] = se2n_image_desc(_ptr(f), _ptr(mask), _ptr(out), _ptr(bins), H, W, N)
        keep.append(img)
    h = _P()
    _check(lib.se2n_batch_create(ctypes.byref(h), descs, len(images), ctypes.byref(params), angle_conv, flags,
                                 _stream(stream)), "se2n_batch_create")
    return Batch(h.value, keep)


def se2n_batch_run(batch):
    _check(lib.se2n_batch_run(batch.handle), "se2n_batch_run")


def se2n_batch_run_per_image(batch):
    _check(lib.se2n_batch_run_per_image(batch.handle), "se2n_batch_run_per_image")


def se2n_batch_run_diffusion(batch):
    _check(lib.se2n_batch_run_diffusion(batch.handle), "se2n_batch_run_diffusion")


def se2n_batch_get_info(batch):
    info = se2n_batch_info()
    _check(lib.se2n_batch_get_info(batch.handle, ctypes.byref(info)), "se2n_batch_get_info")
    return {name: getattr(info, name) for name, _ in se2n_batch_info._fields_}


def se2n_batch_destroy(batch):
    batch.close()


def se2n_diffuse_many_noalloc(volumes, beta, T, steps, angle_conv=0, flags=0, stream=None):
    """volumes: sequence of complex64 device tensors [N][H][W] (diffused in
    place). Calls the entry point that allocates no device memory."""
    import torch
    descs = (se2n_volume_desc * max(len(volumes), 1))()
    for i, v in enumerate(volumes):
        if v.dtype != torch.complex64 or not v.is_cuda or v.dim() != 3 or not v.is_contiguous():
            raise ValueError(f"volume {i}: a contiguous complex64 CUDA tensor [N][H][W] is required "
                             f"(got {v.dtype}, {tuple(v.shape)}, device {v.device})")
        N, H, W = v.shape
        descs[i] = se2n_volume_desc(_ptr(v), H, W, N)
    _check(lib.se2n_diffuse_many_noalloc(descs, len(volumes), beta, T, steps, angle_conv, flags, _stream(stream)),
           "se2n_diffuse_many_noalloc")


class Unet:
    """Owns an se2n_unet*."""

    def __init__(self, handle, batch, H, W):
        self.handle = handle
        self.batch, self.H, self.W = batch, H, W

    def close(self):
        if self.handle:
            lib.se2n_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def se2n_unet_create(batch, H, W, stream=None):
    h = _P()
    _check(lib.se2n_unet_create(ctypes.byref(h), batch, H, W, _stream(stream)), "se2n_unet_create")
    return Unet(h.value, batch, H, W)


def se2n_unet_destroy(u):
    u.close()


def se2n_unet_param_count(u):
    n = ctypes.c_longlong()
    _check(lib.se2n_unet_param_count(u.handle, ctypes.byref(n)), "se2n_unet_param_count")
    return n.value


def se2n_unet_init(u, seed):
    _check(lib.se2n_unet_init(u.handle, seed), "se2n_unet_init")


def se2n_unet_set_params(u, host):
    _check(lib.se2n_unet_set_params(u.handle, _ptr(host)), "se2n_unet_set_params")


def se2n_unet_get_params(u, host):
    _check(lib.se2n_unet_get_params(u.handle, _ptr(host)), "se2n_unet_get_params")


def se2n_unet_get_grads(u, host):
    _check(lib.se2n_unet_get_grads(u.handle, _ptr(host)), "se2n_unet_get_grads")


def se2n_unet_forward(u, f, mask, count, out):
    _check(lib.se2n_unet_forward(u.handle, _ptr(f), _ptr(mask), count, _ptr(out)), "se2n_unet_forward")


def se2n_unet_backward(u, f, mask, target, count, loss=None):
    _check(lib.se2n_unet_backward(u.handle, _ptr(f), _ptr(mask), _ptr(target), count, _ptr(loss)),
           "se2n_unet_backward")


def se2n_unet_adam(u, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(lib.se2n_unet_adam(u.handle, lr, beta1, beta2, eps), "se2n_unet_adam")


def se2n_unet_train_step(u, f, mask, target, count, lr, loss=None):
    _check(lib.se2n_unet_train_step(u.handle, _ptr(f), _ptr(mask), _ptr(target), count, lr, _ptr(loss)),
           "se2n_unet_train_step")


def se2n_surrogate_inpaint(u, plan, params, f, mask, count, threshold, vol_scratch, out, residual_host=None):
    nf = ctypes.c_int()
    _check(lib.se2n_surrogate_inpaint(u.handle, plan.handle, ctypes.byref(params), _ptr(f), _ptr(mask), count,
                                      threshold, _ptr(vol_scratch), _ptr(out), _ptr(residual_host), ctypes.byref(nf)),
           "se2n_surrogate_inpaint")
    return nf.value
