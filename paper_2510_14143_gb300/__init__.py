"""GB300 (sm_103a) 3D Richardson-Lucy deconvolution: thin Python binding.

Every function here has the name of the C ABI call it wraps
(``include/cubic_rl.h``) and only marshals arguments: torch tensors become
device pointers, ``torch.cuda`` streams become ``cudaStream_t`` handles, and a
non-zero status becomes a ``CubicError``.  All arithmetic runs in the CUDA
kernels of ``libcubic_rl.so``; there is no CPU fallback.  If the library has
not been built, every call raises.

The method is Section 4 of arXiv 2510.14143 ("Richardson-Lucy
deconvolution"): blur the estimate with the PSF, divide the measured volume by
the blur, correlate the quotient with the PSF, multiply the estimate by it.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcubic_rl.so")

_lock = threading.Lock()
_lib = None

STATUS = {
    0: "CUBIC_OK", 1: "CUBIC_ERR_INVALID_ARG", 2: "CUBIC_ERR_UNSUPPORTED_SIZE", 3: "CUBIC_ERR_ALIGNMENT",
    4: "CUBIC_ERR_OUT_OF_MEMORY", 5: "CUBIC_ERR_CUDA", 6: "CUBIC_ERR_TIMEOUT", 7: "CUBIC_ERR_NOT_READY",
}


class CubicError(RuntimeError):
    def __init__(self, status: int, call: str, detail: str):
        self.status = status
        super().__init__(f"{call} failed: {STATUS.get(status, status)}: {detail}")


_vp, _i64, _ci, _cf, _sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_size_t
_SIGS = {
    "cubic_status_string": ([_ci], ctypes.c_char_p),
    "cubic_last_error": ([], ctypes.c_char_p),
    "cubic_rl_supported_length": ([_i64], _ci),
    "cubic_rl_plan": ([ctypes.POINTER(_vp), ctypes.POINTER(_i64), _vp, ctypes.c_uint, _vp], _ci),
    "cubic_rl_plan_linear": ([ctypes.POINTER(_vp), ctypes.POINTER(_i64), ctypes.POINTER(_i64), _vp, ctypes.c_uint,
                              _vp], _ci),
    "cubic_rl_plan_dims": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _ci),
    "cubic_rl_plan_update_psf": ([_vp, _vp, _vp], _ci),
    "cubic_rl_plan_destroy": ([_vp], _ci),
    "cubic_rl_workspace_bytes": ([_vp, ctypes.POINTER(_sz)], _ci),
    "cubic_rl_set_workspace": ([_vp, _vp, _sz], _ci),
    "cubic_rl_deconvolve": ([_vp, _vp, _ci, _cf, _vp, _vp], _ci),
    "cubic_rl_convolve": ([_vp, _vp, _ci, _vp, _vp], _ci),
    "cubic_rl_spectrum_layout": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _ci),
    "cubic_rl_fft3_forward": ([_vp, _vp, _vp, _vp], _ci),
    "cubic_rl_fft3_inverse": ([_vp, _vp, _vp, _vp], _ci),
    "cubic_rl_deconvolve_host": ([_vp, _vp, _ci, _cf, _vp, _vp], _ci),
    "cubic_psf_gaussian": ([ctypes.POINTER(_i64), _cf, _cf, _cf, _vp, _vp], _ci),
    "cubic_rl_stream_status": ([_vp, _vp], _ci),
    "cubic_rl_plan_variants": ([_vp, ctypes.POINTER(_ci), ctypes.POINTER(_ci)], _ci),
    "cubic_rl_plan_set_variants": ([_vp, _ci, _ci, _ci], _ci),
    "cubic_rl_autotune": ([_vp, _vp, _vp, _vp], _ci),
    "cubic_rl_plan_set_chunk": ([_vp, _i64], _ci),
    "cubic_rl_plan_chunk": ([_vp], _i64),
    "cubic_rl_deconvolve_noalloc": ([ctypes.POINTER(_i64), _vp, _vp, _ci, _cf, _vp, _vp], _ci),
    "cubic_rl_noalloc_status": ([_vp], _ci),
    "cubic_rl_plan_set_wait_limit": ([_vp, ctypes.c_uint64], _ci),
    "cubic_test_skip_next_tile_copy": ([ctypes.c_uint64], _ci),
    "cubic_rl_deconvolve_batched": ([ctypes.POINTER(_vp), _ci, ctypes.POINTER(_vp), _ci, _cf, ctypes.POINTER(_vp),
                                     _vp], _ci),
    "cubic_rl_batched_graph_nodes": ([], _i64),
    "cubic_fsc": ([_vp, _vp, _vp, _ci, _vp, _vp], _ci),
    "cubic_fsc_split": ([_vp, _vp, _ci, _vp, _vp], _ci),
    "cubic_rl_deconvolve_auto": ([_vp, _vp, _ci, _cf, _cf, _ci, _vp, ctypes.POINTER(_ci),
                                  ctypes.POINTER(ctypes.c_double), _vp], _ci),
    "cubic_rl_deconvolve_accel": ([_vp, _vp, _ci, _cf, _vp, _vp, _vp], _ci),
    "cubic_rl_deconvolve_monitor": ([_vp, _vp, _vp, _ci, _cf, _ci, ctypes.c_double, _ci, _vp, ctypes.POINTER(_ci),
                                     ctypes.POINTER(ctypes.c_double), _vp], _ci),
    "cubic_rl_deconvolve_ckpt": ([_vp, _vp, _ci, _cf, _ci, _vp, _vp, _vp], _ci),
    "cubic_rl_backward_workspace_bytes": ([_vp, _ci, ctypes.POINTER(_sz)], _ci),
    "cubic_rl_backward": ([_vp, _vp, _ci, _cf, _ci, _vp, _vp, _vp, _vp, _ci, _vp], _ci),
    "cubic_psf_gaussian_backward": ([ctypes.POINTER(_i64), _cf, _cf, _cf, _vp, _vp, _vp], _ci),
    "cubic_rl_kernel_kinds": ([], _ci),
    "cubic_rl_kernel_name": ([_ci], ctypes.c_char_p),
    "cubic_rl_profile": ([_vp, _ci, _ci], _ci),
    "cubic_rl_profile_read": ([_vp, _ci, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i64),
                               ctypes.POINTER(_i64), ctypes.POINTER(ctypes.c_double)], _ci),
}


def lib():
    """The loaded ``libcubic_rl.so`` (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2510_14143_gb300.build`")
            l = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(l, name)
                f.argtypes = args
                f.restype = res
            _lib = l
    return _lib


def _check(status: int, call: str) -> None:
    if status != 0:
        raise CubicError(status, call, lib().cubic_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t, dtype=None, numel=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (checked dtype/size), or an int address."""
    if isinstance(t, int):
        return t
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


class Plan:
    """Owning wrapper of a ``cubic_rl_plan_t``; destroyed with the object."""

    def __init__(self, handle: int, dims):
        self.handle = handle
        self.dims = tuple(int(d) for d in dims)
        self.voxels = self.dims[0] * self.dims[1] * self.dims[2]

    def close(self):
        if self.handle:
            lib().cubic_rl_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cubic_status_string(status: int) -> str:
    return lib().cubic_status_string(status).decode()


def cubic_last_error() -> str:
    return lib().cubic_last_error().decode(errors="replace")


def cubic_rl_supported_length(n: int) -> bool:
    return bool(lib().cubic_rl_supported_length(int(n)))


def cubic_rl_plan(dims, psf, flags: int = 0, stream=None) -> Plan:
    """Plan for volumes of shape dims = (nz, ny, nx) with PSF `psf` (float32, same shape)."""
    import torch
    dims = tuple(int(d) for d in dims)
    d = (_i64 * 3)(*dims)
    h = _vp()
    _check(lib().cubic_rl_plan(ctypes.byref(h), d, _ptr(psf, torch.float32, dims[0] * dims[1] * dims[2], "psf"),
                               flags, _stream(stream)), "cubic_rl_plan")
    return Plan(h.value, dims)


def cubic_rl_plan_linear(dims, psf, flags: int = 0, stream=None) -> Plan:
    """Plan with linear (zero-padded, same-mode) boundaries: image shape dims, PSF box psf.shape."""
    import torch
    dims = tuple(int(d) for d in dims)
    kdims = tuple(int(k) for k in psf.shape)
    h = _vp()
    _check(lib().cubic_rl_plan_linear(ctypes.byref(h), (_i64 * 3)(*dims), (_i64 * 3)(*kdims),
                                      _ptr(psf, torch.float32, kdims[0] * kdims[1] * kdims[2], "psf"), flags,
                                      _stream(stream)), "cubic_rl_plan_linear")
    plan = Plan(h.value, dims)
    plan.psf_voxels = kdims[0] * kdims[1] * kdims[2]
    return plan


def cubic_rl_plan_dims(plan: Plan):
    """((image nz, ny, nx), (transform nz, ny, nx))."""
    im, tr = (_i64 * 3)(), (_i64 * 3)()
    _check(lib().cubic_rl_plan_dims(plan.handle, im, tr), "cubic_rl_plan_dims")
    return tuple(im), tuple(tr)


def cubic_rl_plan_update_psf(plan: Plan, psf, stream=None) -> None:
    import torch
    n = getattr(plan, "psf_voxels", plan.voxels)
    _check(lib().cubic_rl_plan_update_psf(plan.handle, _ptr(psf, torch.float32, n, "psf"),
                                          _stream(stream)), "cubic_rl_plan_update_psf")


def cubic_rl_plan_destroy(plan: Plan) -> None:
    plan.close()


def cubic_rl_workspace_bytes(plan: Plan) -> int:
    n = _sz()
    _check(lib().cubic_rl_workspace_bytes(plan.handle, ctypes.byref(n)), "cubic_rl_workspace_bytes")
    return int(n.value)


def cubic_rl_set_workspace(plan: Plan, workspace) -> None:
    """Hand the plan caller-owned scratch (a CUDA tensor kept alive by the plan object)."""
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib().cubic_rl_set_workspace(plan.handle, _ptr(workspace, name="workspace"), nbytes),
           "cubic_rl_set_workspace")
    plan._workspace = workspace


def cubic_rl_deconvolve(plan: Plan, image, n_iter: int, eps: float, out, stream=None) -> None:
    import torch
    _check(lib().cubic_rl_deconvolve(plan.handle, _ptr(image, torch.float32, plan.voxels, "image"), int(n_iter),
                                     float(eps), _ptr(out, torch.float32, plan.voxels, "out"), _stream(stream)),
           "cubic_rl_deconvolve")


def _host_ptr(a, numel, name):
    import numpy as np
    if isinstance(a, int):
        return a
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous() or a.numel() != numel:
                raise ValueError(f"{name} must be a contiguous float32 host tensor of {numel} elements")
            return a.data_ptr()
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags.c_contiguous or a.size != numel:
        raise ValueError(f"{name} must be a contiguous float32 host array of {numel} elements")
    return a.ctypes.data


def cubic_rl_deconvolve_host(plan: Plan, image, n_iter: int, eps: float, out, stream=None) -> None:
    """Host buffers in and out (numpy arrays or CPU tensors; pin them for async copies)."""
    _check(lib().cubic_rl_deconvolve_host(plan.handle, _host_ptr(image, plan.voxels, "image"), int(n_iter),
                                          float(eps), _host_ptr(out, plan.voxels, "out"), _stream(stream)),
           "cubic_rl_deconvolve_host")


def cubic_psf_gaussian(dims, sigma_xy: float, sigma_z: float, amp: float, psf, stream=None) -> None:
    import torch
    dims = tuple(int(d) for d in dims)
    d = (_i64 * 3)(*dims)
    _check(lib().cubic_psf_gaussian(d, float(sigma_xy), float(sigma_z), float(amp),
                                    _ptr(psf, torch.float32, dims[0] * dims[1] * dims[2], "psf"), _stream(stream)),
           "cubic_psf_gaussian")


def cubic_rl_stream_status(plan: Plan, stream=None) -> None:
    """Raise CubicError(CUBIC_ERR_TIMEOUT) if a kernel's bounded device wait gave up."""
    _check(lib().cubic_rl_stream_status(plan.handle, _stream(stream)), "cubic_rl_stream_status")


def cubic_rl_plan_set_wait_limit(plan: Plan, limit_ns: int) -> None:
    """Limit of every bounded device wait of the plan's kernels, in ns (0: the 2 s default)."""
    _check(lib().cubic_rl_plan_set_wait_limit(plan.handle, int(limit_ns)), "cubic_rl_plan_set_wait_limit")


def cubic_test_skip_next_tile_copy(wait_ns: int) -> None:
    """Test support: the next TMA-pipelined Y launch in this process has its first CTA skip
    its first tile copy and wait at most wait_ns for it (see the C header)."""
    _check(lib().cubic_test_skip_next_tile_copy(int(wait_ns)), "cubic_test_skip_next_tile_copy")


def cubic_rl_plan_variants(plan: Plan):
    """((nx, ny, nz) variant counts, (vx, vy, vz) chosen)."""
    c = (_ci * 3)()
    ch = (_ci * 3)()
    _check(lib().cubic_rl_plan_variants(plan.handle, c, ch), "cubic_rl_plan_variants")
    return tuple(c), tuple(ch)


def cubic_rl_plan_set_variants(plan: Plan, vx: int, vy: int, vz: int) -> None:
    _check(lib().cubic_rl_plan_set_variants(plan.handle, int(vx), int(vy), int(vz)), "cubic_rl_plan_set_variants")


def cubic_rl_plan_set_chunk(plan: Plan, columns: int) -> None:
    _check(lib().cubic_rl_plan_set_chunk(plan.handle, int(columns)), "cubic_rl_plan_set_chunk")


def cubic_rl_plan_chunk(plan: Plan) -> int:
    return int(lib().cubic_rl_plan_chunk(plan.handle))


def cubic_rl_autotune(plan: Plan, image, out, stream=None) -> None:
    import torch
    _check(lib().cubic_rl_autotune(plan.handle, _ptr(image, torch.float32, plan.voxels, "image"),
                                   _ptr(out, torch.float32, plan.voxels, "out"), _stream(stream)),
           "cubic_rl_autotune")


def cubic_rl_deconvolve_noalloc(dims, psf, image, n_iter: int, eps: float, out, stream=None) -> None:
    """Deconvolution that allocates no device memory (for callers that cannot allocate,
    e.g. under another framework's stream capture or a fully reserved memory pool).
    Uses one fixed per-device scratch array shared by all calls: serialise calls."""
    import torch
    dims = tuple(int(d) for d in dims)
    v = dims[0] * dims[1] * dims[2]
    d = (_i64 * 3)(*dims)
    _check(lib().cubic_rl_deconvolve_noalloc(d, _ptr(psf, torch.float32, v, "psf"), _ptr(image, torch.float32, v, "image"),
                                             int(n_iter), float(eps), _ptr(out, torch.float32, v, "out"),
                                             _stream(stream)), "cubic_rl_deconvolve_noalloc")


def cubic_rl_noalloc_status(stream=None) -> None:
    """Raises CubicError (CUBIC_ERR_TIMEOUT) if a bounded device wait of an allocation-free
    call on the current device gave up since the last check; clears the flag."""
    _check(lib().cubic_rl_noalloc_status(_stream(stream)), "cubic_rl_noalloc_status")


def cubic_rl_deconvolve_batched(plans, images, n_iter: int, eps: float, outs, stream=None) -> None:
    """Deconvolve len(plans) volumes (one plan each, distinct) as one CUDA graph."""
    import torch
    n = len(plans)
    if len(images) != n or len(outs) != n:
        raise ValueError("plans, images and outs must have the same length")
    P = (_vp * n)(*[p.handle for p in plans])
    I = (_vp * n)(*[_ptr(im, torch.float32, p.voxels, "image") for im, p in zip(images, plans)])
    O = (_vp * n)(*[_ptr(o, torch.float32, p.voxels, "out") for o, p in zip(outs, plans)])
    _check(lib().cubic_rl_deconvolve_batched(P, n, I, int(n_iter), float(eps), O, _stream(stream)),
           "cubic_rl_deconvolve_batched")


def cubic_rl_batched_graph_nodes() -> int:
    return int(lib().cubic_rl_batched_graph_nodes())


def cubic_rl_deconvolve_auto(plan: Plan, image, max_iter: int, eps: float, tol: float, check_every: int, out,
                             stream=None):
    """Automatic stopping; returns (iterations done, list of per-iteration relative changes)."""
    import torch
    n = _ci(0)
    hist = (ctypes.c_double * max(1, int(max_iter)))()
    _check(lib().cubic_rl_deconvolve_auto(plan.handle, _ptr(image, torch.float32, plan.voxels, "image"),
                                          int(max_iter), float(eps), float(tol), int(check_every),
                                          _ptr(out, torch.float32, plan.voxels, "out"), ctypes.byref(n), hist,
                                          _stream(stream)), "cubic_rl_deconvolve_auto")
    return int(n.value), list(hist[:n.value])


METRIC_REL_CHANGE, METRIC_NLL, METRIC_PSNR = 0, 1, 2


def cubic_rl_deconvolve_monitor(plan: Plan, image, max_iter: int, eps: float, metric: int, tol: float,
                                check_every: int, out, reference=None, stream=None):
    """Metric-guided stopping; returns (iterations done, history as a list of (delta, NLL, PSNR))."""
    import torch
    n = _ci(0)
    hist = (ctypes.c_double * (3 * max(1, int(max_iter))))()
    ref = None if reference is None else _ptr(reference, torch.float32, plan.voxels, "reference")
    _check(lib().cubic_rl_deconvolve_monitor(plan.handle, _ptr(image, torch.float32, plan.voxels, "image"), ref,
                                             int(max_iter), float(eps), int(metric), float(tol), int(check_every),
                                             _ptr(out, torch.float32, plan.voxels, "out"), ctypes.byref(n), hist,
                                             _stream(stream)), "cubic_rl_deconvolve_monitor")
    k = int(n.value)
    return k, [tuple(hist[3 * i:3 * i + 3]) for i in range(k)]


def cubic_rl_deconvolve_accel(plan: Plan, image, n_iter: int, eps: float, out, alpha=None, stream=None) -> None:
    """Accelerated RL (Biggs-Andrews extrapolation); alpha: optional float32 CUDA tensor of n_iter."""
    import torch
    a = None if alpha is None else _ptr(alpha, torch.float32, int(n_iter) if n_iter > 0 else None, "alpha")
    _check(lib().cubic_rl_deconvolve_accel(plan.handle, _ptr(image, torch.float32, plan.voxels, "image"),
                                           int(n_iter), float(eps), _ptr(out, torch.float32, plan.voxels, "out"),
                                           a, _stream(stream)), "cubic_rl_deconvolve_accel")


def cubic_fsc(plan: Plan, a, b, n_shells: int, fsc=None, stream=None):
    """Fourier Shell Correlation of two volumes; returns the float32 CUDA tensor of n_shells values."""
    import torch
    if fsc is None:
        fsc = torch.empty(int(n_shells), dtype=torch.float32, device="cuda")
    _check(lib().cubic_fsc(plan.handle, _ptr(a, torch.float32, plan.voxels, "a"),
                           _ptr(b, torch.float32, plan.voxels, "b"), int(n_shells),
                           _ptr(fsc, torch.float32, int(n_shells), "fsc"), _stream(stream)), "cubic_fsc")
    return fsc


def cubic_fsc_split(half_plan: Plan, image, n_shells: int, fsc=None, stream=None):
    """Single-image FSC of a volume of twice the plan's dims; returns the float32 CUDA tensor."""
    import torch
    if fsc is None:
        fsc = torch.empty(int(n_shells), dtype=torch.float32, device="cuda")
    _check(lib().cubic_fsc_split(half_plan.handle, _ptr(image, torch.float32, 8 * half_plan.voxels, "image"),
                                 int(n_shells), _ptr(fsc, torch.float32, int(n_shells), "fsc"), _stream(stream)),
           "cubic_fsc_split")
    return fsc


def n_checkpoints(n_iter: int, ckpt_every: int) -> int:
    return (int(n_iter) + int(ckpt_every) - 1) // int(ckpt_every)


def shard_volumes(shapes, world: int):
    """Volume indices for each of `world` GPUs, balanced by voxel count.

    A batch of independent volumes needs no exchange between GPUs: each one deconvolves its
    share.  Greedy longest-processing-time order: the largest remaining volume goes to the
    least-loaded GPU (the lower index on ties), so every rank computes the same split on
    its own.  Returns `world` lists of indices, each in increasing order.
    """
    world = int(world)
    if world < 1:
        raise ValueError("world must be >= 1")
    vox = [int(s[0]) * int(s[1]) * int(s[2]) for s in shapes]
    order = sorted(range(len(vox)), key=lambda i: (-vox[i], i))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += vox[i]
    return [sorted(p) for p in parts]


def cubic_rl_deconvolve_ckpt(plan: Plan, image, n_iter: int, eps: float, ckpt_every: int, ckpts, out,
                             stream=None) -> None:
    import torch
    _check(lib().cubic_rl_deconvolve_ckpt(plan.handle, _ptr(image, torch.float32, plan.voxels, "image"), int(n_iter),
                                          float(eps), int(ckpt_every),
                                          _ptr(ckpts, torch.float32, plan.voxels * n_checkpoints(n_iter, ckpt_every),
                                               "ckpts"),
                                          _ptr(out, torch.float32, plan.voxels, "out"), _stream(stream)),
           "cubic_rl_deconvolve_ckpt")


def cubic_rl_backward_workspace_bytes(plan: Plan, ckpt_every: int) -> int:
    n = _sz()
    _check(lib().cubic_rl_backward_workspace_bytes(plan.handle, int(ckpt_every), ctypes.byref(n)),
           "cubic_rl_backward_workspace_bytes")
    return int(n.value)


def cubic_rl_backward(plan: Plan, image, n_iter: int, eps: float, ckpt_every: int, ckpts, grad_out,
                      grad_image=None, grad_psf=None, accumulate_psf: bool = False, stream=None) -> None:
    import torch
    v = plan.voxels
    _check(lib().cubic_rl_backward(plan.handle, _ptr(image, torch.float32, v, "image"), int(n_iter), float(eps),
                                   int(ckpt_every),
                                   _ptr(ckpts, torch.float32, v * n_checkpoints(n_iter, ckpt_every), "ckpts"),
                                   _ptr(grad_out, torch.float32, v, "grad_out"),
                                   None if grad_image is None else _ptr(grad_image, torch.float32, v, "grad_image"),
                                   None if grad_psf is None else _ptr(grad_psf, torch.float32, v, "grad_psf"),
                                   int(bool(accumulate_psf)), _stream(stream)), "cubic_rl_backward")


def cubic_psf_gaussian_backward(dims, sigma_xy: float, sigma_z: float, amp: float, grad_psf, grad_params,
                                stream=None) -> None:
    """grad_params: float32 CUDA tensor of 3 elements <- dL/d(sigma_xy, sigma_z, amp)."""
    import torch
    dims = tuple(int(d) for d in dims)
    d = (_i64 * 3)(*dims)
    _check(lib().cubic_psf_gaussian_backward(d, float(sigma_xy), float(sigma_z), float(amp),
                                             _ptr(grad_psf, torch.float32, dims[0] * dims[1] * dims[2], "grad_psf"),
                                             _ptr(grad_params, torch.float32, 3, "grad_params"), _stream(stream)),
           "cubic_psf_gaussian_backward")


def cubic_rl_kernel_kinds() -> int:
    return int(lib().cubic_rl_kernel_kinds())


def cubic_rl_kernel_name(kind: int) -> str:
    return lib().cubic_rl_kernel_name(int(kind)).decode()


def cubic_rl_profile(plan: Plan, enable: bool, max_events: int = 1 << 15) -> None:
    _check(lib().cubic_rl_profile(plan.handle, int(bool(enable)), int(max_events)), "cubic_rl_profile")


def cubic_rl_profile_read(plan: Plan) -> dict:
    """{kernel name: dict(ms, timed, launches, bytes)} since the last cubic_rl_profile()."""
    n = cubic_rl_kernel_kinds()
    ms = (ctypes.c_double * n)()
    timed = (_i64 * n)()
    launches = (_i64 * n)()
    nbytes = (ctypes.c_double * n)()
    _check(lib().cubic_rl_profile_read(plan.handle, n, ms, timed, launches, nbytes), "cubic_rl_profile_read")
    return {cubic_rl_kernel_name(k): dict(ms=ms[k], timed=int(timed[k]), launches=int(launches[k]),
                                          bytes=nbytes[k]) for k in range(n)}


def cubic_rl_convolve(plan: Plan, x, flipped: bool, out, stream=None) -> None:
    import torch
    _check(lib().cubic_rl_convolve(plan.handle, _ptr(x, torch.float32, plan.voxels, "in"), int(bool(flipped)),
                                   _ptr(out, torch.float32, plan.voxels, "out"), _stream(stream)),
           "cubic_rl_convolve")


def cubic_rl_spectrum_layout(plan: Plan):
    xh, xp = _i64(), _i64()
    _check(lib().cubic_rl_spectrum_layout(plan.handle, ctypes.byref(xh), ctypes.byref(xp)),
           "cubic_rl_spectrum_layout")
    return int(xh.value), int(xp.value)


def _spec_numel(plan: Plan) -> int:
    _, xp = cubic_rl_spectrum_layout(plan)
    return plan.dims[0] * plan.dims[1] * xp


def cubic_rl_fft3_forward(plan: Plan, x, spec, stream=None) -> None:
    import torch
    _check(lib().cubic_rl_fft3_forward(plan.handle, _ptr(x, torch.float32, plan.voxels, "in"),
                                       _ptr(spec, torch.complex64, _spec_numel(plan), "spec"), _stream(stream)),
           "cubic_rl_fft3_forward")


def cubic_rl_fft3_inverse(plan: Plan, spec, out, stream=None) -> None:
    import torch
    _check(lib().cubic_rl_fft3_inverse(plan.handle, _ptr(spec, torch.complex64, _spec_numel(plan), "spec"),
                                       _ptr(out, torch.float32, plan.voxels, "out"), _stream(stream)),
           "cubic_rl_fft3_inverse")


def rl_deconvolve(image, psf, n_iter: int, eps: float = 1e-6, out=None, stream=None):
    """Convenience: plan + deconvolve for one volume (float32 CUDA tensors of one shape)."""
    import torch
    plan = cubic_rl_plan(image.shape, psf, 0, stream)
    if out is None:
        out = torch.empty_like(image)
    cubic_rl_deconvolve(plan, image, n_iter, eps, out, stream)
    out._cubic_plan = plan  # keep the plan (and its buffers) alive until out dies
    return out
