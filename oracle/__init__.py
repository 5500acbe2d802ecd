"""FP64 CPU oracle for 3D Richardson-Lucy deconvolution -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
``paper_2510_14143_gb300``) never imports, links or executes it, and it never
imports the product: the two share no code.  Inputs come from the seeded
generator in ``paper_2510_14143_gb300.synth``, which holds none of the
method's arithmetic.

The arithmetic lives in ``rl_oracle.c`` (plain C, double precision, optional
OpenMP); this module compiles it with gcc on first use and wraps it with
ctypes.  It follows the paper's Section 4 "Richardson-Lucy deconvolution":
each iteration blurs the estimate with the PSF, divides the measured volume by
that blur, correlates the quotient with the PSF and multiplies the estimate by
the result.  The readings taken where the paper is silent (circular
boundaries, PSF centre at floor(n/2), u0 = max(mean(d), eps), denominator
clamp max(b, eps)) are stated in ``rl_oracle.c``.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
in ``tests/test_oracle.py`` (brute-force DFT, direct convolution, closed-form
RL cases, invariants, finite differences).  The paper prints no numerical RL
example, so no pin comes from a value printed in the paper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rl_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile rl_oracle.c into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(ctypes.c_double)
            i64, ci, cd = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            sig = {
                "orc_num_threads": ([], ci),
                "orc_fft1": ([P, i64, ci], ci),
                "orc_dft1_brute": ([P, P, i64, ci], ci),
                "orc_fft3": ([P, i64, i64, i64, ci], ci),
                "orc_center_to_origin": ([P, P, i64, i64, i64], ci),
                "orc_conv3_direct": ([P, P, P, i64, i64, i64], ci),
                "orc_psf_spectrum": ([P, P, i64, i64, i64], ci),
                "orc_convolve": ([P, P, P, i64, i64, i64, ci], ci),
                "orc_initial_value": ([P, i64, cd], cd),
                "orc_rl_iterate": ([P, P, P, cd, i64, i64, i64, P, P, P, P], ci),
                "orc_rl": ([P, P, i64, i64, i64, ci, cd, P], ci),
                "orc_rl_grad": ([P, P, i64, i64, i64, ci, cd, P, P, P], ci),
                "orc_fsc": ([P, P, i64, i64, i64, ci, P, P, P, P], ci),
                "orc_fsc_split": ([P, i64, i64, i64, ci, P], ci),
                "orc_rl_auto": ([P, P, i64, i64, i64, ci, cd, cd, ci, P, ctypes.POINTER(ci), P], ci),
                "orc_rl_accel": ([P, P, i64, i64, i64, ci, cd, P, P], ci),
                "orc_poisson_nll": ([P, P, i64, cd], cd),
                "orc_conv_same": ([P, P, P, i64, i64, i64, i64, i64, i64, ci], ci),
                "orc_rl_same": ([P, P, i64, i64, i64, i64, i64, i64, ci, cd, P], ci),
                "orc_rl_accel_same": ([P, P, i64, i64, i64, i64, i64, i64, ci, cd, P, P], ci),
                "orc_psnr_si": ([P, P, i64], cd),
                "orc_rl_monitor": ([P, P, P, i64, i64, i64, ci, cd, ci, cd, ci, P, ctypes.POINTER(ci), P], ci),
                "orc_rl_monitor_same": ([P, P, P, i64, i64, i64, i64, i64, i64, ci, cd, ci, cd, ci, P,
                                         ctypes.POINTER(ci), P], ci),
                "orc_accel_linear": ([i64, ci, P, P, P, P, P], ci),
                "orc_psf_gaussian": ([i64, i64, i64, cd, cd, cd, P], ci),
                "orc_psf_gaussian_grad": ([i64, i64, i64, cd, cd, cd, P, P], ci),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def num_threads() -> int:
    return int(_load().orc_num_threads())


def fft1(x, inverse: bool = False) -> np.ndarray:
    """Length-n DFT (radix-2, else Bluestein). Inverse carries 1/n."""
    a = _c128(x).copy()
    _check(_load().orc_fft1(_p(a.view(np.float64)), a.size, int(inverse)), "fft1")
    return a


def dft1_brute(x, inverse: bool = False) -> np.ndarray:
    """O(n^2) DFT straight from its definition."""
    a = _c128(x)
    out = np.empty_like(a)
    _check(_load().orc_dft1_brute(_p(a.view(np.float64)), _p(out.view(np.float64)), a.size,
                                  int(inverse)), "dft1_brute")
    return out


def fft3(x, inverse: bool = False) -> np.ndarray:
    """3D DFT of a [nz][ny][nx] array, axis by axis."""
    a = _c128(x).copy()
    nz, ny, nx = a.shape
    _check(_load().orc_fft3(_p(a.view(np.float64)), nz, ny, nx, int(inverse)), "fft3")
    return a


def center_to_origin(p) -> np.ndarray:
    a = _f64(p)
    out = np.empty_like(a)
    _check(_load().orc_center_to_origin(_p(a), _p(out), *a.shape), "center_to_origin")
    return out


def conv3_direct(h0, u) -> np.ndarray:
    """Direct circular convolution out(y) = sum_x h0(x) u(y-x), O(V^2)."""
    h, v = _f64(h0), _f64(u)
    out = np.empty_like(v)
    _check(_load().orc_conv3_direct(_p(h), _p(v), _p(out), *v.shape), "conv3_direct")
    return out


def psf_spectrum(psf) -> np.ndarray:
    """H = DFT3 of the PSF moved from floor(n/2) to the origin."""
    p = _f64(psf)
    H = np.empty(p.shape, np.complex128)
    _check(_load().orc_psf_spectrum(_p(p), _p(H.view(np.float64)), *p.shape), "psf_spectrum")
    return H


def convolve(H, u, flipped: bool = False) -> np.ndarray:
    """Re IDFT3(H . DFT3(u)); with flipped=True uses conj(H) (the flipped PSF)."""
    Hc, v = _c128(H), _f64(u)
    out = np.empty_like(v)
    _check(_load().orc_convolve(_p(Hc.view(np.float64)), _p(v), _p(out), *v.shape, int(flipped)),
           "convolve")
    return out


def initial_value(d, eps: float) -> float:
    a = _f64(d)
    return float(_load().orc_initial_value(_p(a), a.size, float(eps)))


def rl_iterate(H, d, u, eps: float):
    """One RL iteration; returns (u_next, b, r, q)."""
    Hc, dd, uu = _c128(H), _f64(d), _f64(u)
    outs = [np.empty_like(uu) for _ in range(4)]
    _check(_load().orc_rl_iterate(_p(Hc.view(np.float64)), _p(dd), _p(uu), float(eps), *uu.shape,
                                  *[_p(o) for o in outs]), "rl_iterate")
    return tuple(outs)


def rl(d, psf, n_iter: int, eps: float = 1e-6) -> np.ndarray:
    """n_iter RL iterations from u0 = max(mean(d), eps); float64 result."""
    dd, p = _f64(d), _f64(psf)
    if dd.shape != p.shape:
        raise ValueError("image and PSF must have the same shape")
    out = np.empty_like(dd)
    _check(_load().orc_rl(_p(dd), _p(p), *dd.shape, int(n_iter), float(eps), _p(out)), "rl")
    return out


def rl_auto(d, psf, max_iter: int, eps: float, tol: float, check_every: int = 1):
    """RL with automatic stopping; returns (estimate, iterations done, deltas)."""
    dd, p = _f64(d), _f64(psf)
    out = np.empty_like(dd)
    hist = np.zeros(max(1, int(max_iter)), np.float64)
    n = ctypes.c_int(0)
    _check(_load().orc_rl_auto(_p(dd), _p(p), *dd.shape, int(max_iter), float(eps), float(tol), int(check_every),
                               _p(out), ctypes.byref(n), _p(hist)), "rl_auto")
    return out, int(n.value), hist[:n.value].copy()


def conv_same(psf, u, flipped: bool = False) -> np.ndarray:
    """Linear ("same"-mode) convolution of u with a PSF of any box size (peak at floor(k/2));
    flipped=True gives its adjoint."""
    p, v = _f64(psf), _f64(u)
    out = np.empty_like(v)
    _check(_load().orc_conv_same(_p(p), _p(v), _p(out), *v.shape, *p.shape, int(flipped)), "conv_same")
    return out


def rl_same(d, psf, n_iter: int, eps: float = 1e-6) -> np.ndarray:
    """RL with linear boundaries: the PSF box may be smaller than the image."""
    dd, p = _f64(d), _f64(psf)
    out = np.empty_like(dd)
    _check(_load().orc_rl_same(_p(dd), _p(p), *dd.shape, *p.shape, int(n_iter), float(eps), _p(out)), "rl_same")
    return out


def rl_accel_same(d, psf, n_iter: int, eps: float = 1e-6):
    """Accelerated RL with linear boundaries; returns (estimate, alpha_0..alpha_{n-1})."""
    dd, p = _f64(d), _f64(psf)
    out = np.empty_like(dd)
    alpha = np.zeros(max(1, int(n_iter)), np.float64)
    _check(_load().orc_rl_accel_same(_p(dd), _p(p), *dd.shape, *p.shape, int(n_iter), float(eps), _p(out),
                                     _p(alpha)), "rl_accel_same")
    return out, alpha[:int(n_iter)].copy()


def poisson_nll(b, d, eps: float) -> float:
    """sum(c - d ln c), c = max(b, eps)."""
    bb, dd = _f64(b), _f64(d)
    return float(_load().orc_poisson_nll(_p(bb), _p(dd), bb.size, float(eps)))


def psnr_si(x, y) -> float:
    """Scale-invariant PSNR of x against the reference y (best affine fit of x to y)."""
    xx, yy = _f64(x), _f64(y)
    return float(_load().orc_psnr_si(_p(xx), _p(yy), xx.size))


METRIC_REL_CHANGE, METRIC_NLL, METRIC_PSNR = 0, 1, 2


def rl_monitor(d, psf, max_iter: int, eps: float, metric: int, tol: float, check_every: int = 1, ref=None):
    """RL with metric-guided stopping; returns (estimate, iterations done, history[n, 3])."""
    dd, p = _f64(d), _f64(psf)
    rr = None if ref is None else _f64(ref)
    out = np.empty_like(dd)
    hist = np.zeros((max(1, int(max_iter)), 3), np.float64)
    n = ctypes.c_int(0)
    _check(_load().orc_rl_monitor(_p(dd), _p(p), None if rr is None else _p(rr), *dd.shape, int(max_iter),
                                  float(eps), int(metric), float(tol), int(check_every), _p(out), ctypes.byref(n),
                                  _p(hist)), "rl_monitor")
    return out, int(n.value), hist[:n.value].copy()


def rl_monitor_same(d, psf_box, max_iter: int, eps: float, metric: int, tol: float, check_every: int = 1,
                    ref=None):
    """rl_monitor with linear ("same"-mode) boundaries and a PSF box of any size."""
    dd, p = _f64(d), _f64(psf_box)
    rr = None if ref is None else _f64(ref)
    out = np.empty_like(dd)
    hist = np.zeros((max(1, int(max_iter)), 3), np.float64)
    n = ctypes.c_int(0)
    _check(_load().orc_rl_monitor_same(_p(dd), _p(p), None if rr is None else _p(rr), *dd.shape, *p.shape,
                                       int(max_iter), float(eps), int(metric), float(tol), int(check_every), _p(out),
                                       ctypes.byref(n), _p(hist)), "rl_monitor_same")
    return out, int(n.value), hist[:n.value].copy()


def rl_accel(d, psf, n_iter: int, eps: float = 1e-6):
    """Accelerated RL (Biggs-Andrews extrapolation); returns (estimate, alpha_0..alpha_{n-1})."""
    dd, p = _f64(d), _f64(psf)
    if dd.shape != p.shape:
        raise ValueError("image and PSF must have the same shape")
    out = np.empty_like(dd)
    alpha = np.zeros(max(1, int(n_iter)), np.float64)
    _check(_load().orc_rl_accel(_p(dd), _p(p), *dd.shape, int(n_iter), float(eps), _p(out), _p(alpha)),
           "rl_accel")
    return out, alpha[:int(n_iter)].copy()


def accel_linear(xs, lam, x0, n_iter: int):
    """The same extrapolation with the linear step psi(y) = xs + lam (y - xs); returns (x_n, alphas)."""
    a, l, x = _f64(xs).ravel(), _f64(lam).ravel(), _f64(x0).ravel()
    out = np.empty_like(a)
    alpha = np.zeros(max(1, int(n_iter)), np.float64)
    _check(_load().orc_accel_linear(a.size, int(n_iter), _p(a), _p(l), _p(x), _p(out), _p(alpha)), "accel_linear")
    return out, alpha[:int(n_iter)].copy()


def fsc(a, b, n_shells: int):
    """Fourier Shell Correlation per shell; returns (fsc, num, |A|^2 sums, |B|^2 sums)."""
    aa, bb = _f64(a), _f64(b)
    outs = [np.zeros(int(n_shells), np.float64) for _ in range(4)]
    _check(_load().orc_fsc(_p(aa), _p(bb), *aa.shape, int(n_shells), *[_p(o) for o in outs]), "fsc")
    return tuple(outs)


def fsc_split(d, n_shells: int) -> np.ndarray:
    """Single-image FSC: mean FSC of the four opposite-parity pairs of sub-volumes."""
    dd = _f64(d)
    out = np.zeros(int(n_shells), np.float64)
    _check(_load().orc_fsc_split(_p(dd), *dd.shape, int(n_shells), _p(out)), "fsc_split")
    return out


def rl_grad(d, psf, n_iter: int, eps: float, g_out):
    """Reverse mode: returns (dL/dd, dL/dpsf) given dL/du_K = g_out."""
    dd, p, g = _f64(d), _f64(psf), _f64(g_out)
    gd, gp = np.empty_like(dd), np.empty_like(dd)
    _check(_load().orc_rl_grad(_p(dd), _p(p), *dd.shape, int(n_iter), float(eps), _p(g), _p(gd),
                               _p(gp)), "rl_grad")
    return gd, gp


def psf_gaussian(shape, sigma_xy: float, sigma_z: float, amp: float = 1.0) -> np.ndarray:
    """A * g / sum(g), g an anisotropic Gaussian peaked at floor(n/2) per axis."""
    out = np.empty(tuple(shape), np.float64)
    _check(_load().orc_psf_gaussian(*out.shape, float(sigma_xy), float(sigma_z), float(amp), _p(out)),
           "psf_gaussian")
    return out


def psf_gaussian_grad(shape, sigma_xy: float, sigma_z: float, amp: float, grad_psf) -> np.ndarray:
    """(dL/dsigma_xy, dL/dsigma_z, dL/dA) from dL/dpsf."""
    g = _f64(grad_psf)
    out = np.empty(3, np.float64)
    _check(_load().orc_psf_gaussian_grad(*tuple(shape), float(sigma_xy), float(sigma_z), float(amp),
                                         _p(g), _p(out)), "psf_gaussian_grad")
    return out
