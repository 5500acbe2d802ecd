"""Pins for the FP64 oracle, checked against things other than itself.

Each check follows from the definition of the DFT, of circular convolution or
from properties of Richardson-Lucy (RL) iteration that the paper's Section 4
"Richardson-Lucy deconvolution" implies (Poisson maximum likelihood, forward
convolution / ratio / flipped-PSF back-convolution / multiplicative update).
Every check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign or conjugation, an off-by-one PSF centre, a swapped ratio) fails
at least one of them.  No test here needs a GPU.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2510_14143_gb300 import synth

RNG = np.random.default_rng(12345)


def crand(n, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(n) + 1j * r.standard_normal(n)


def dft_matrix(n, sign=-1):
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n)


# ---------------------------------------------------------------- 1D FFT

LENGTHS = [1, 2, 3, 4, 5, 6, 7, 8, 9, 12, 15, 16, 25, 27, 30, 32, 48, 50, 64, 75, 81, 96, 125, 128,
           135, 160]


@pytest.mark.parametrize("n", LENGTHS)
def test_fft1_matches_brute_dft(n):
    x = crand(n, n)
    ref = dft_matrix(n) @ x                          # definition, written here
    assert np.allclose(oracle.fft1(x), ref, rtol=0, atol=1e-11 * max(1, np.abs(ref).max()))
    assert np.allclose(oracle.dft1_brute(x), ref, rtol=0, atol=1e-11 * max(1, np.abs(ref).max()))
    inv = (dft_matrix(n, +1) @ x) / n
    assert np.allclose(oracle.fft1(x, inverse=True), inv, rtol=0, atol=1e-12 * max(1, np.abs(inv).max()))


@pytest.mark.parametrize("n", [8, 12, 75, 128])
def test_fft1_closed_forms(n):
    # delta at m  ->  exp(-2 pi i k m / n)
    m = 3 % n
    x = np.zeros(n, complex)
    x[m] = 1
    k = np.arange(n)
    assert np.allclose(oracle.fft1(x), np.exp(-2j * np.pi * k * m / n), atol=1e-13)
    # pure tone exp(+2 pi i m j / n) -> n * delta(k - m): fixes the sign convention
    tone = np.exp(2j * np.pi * m * k / n)
    out = oracle.fft1(tone)
    expect = np.zeros(n, complex)
    expect[m] = n
    assert np.allclose(out, expect, atol=1e-10)
    # constant -> n at DC
    c = oracle.fft1(np.full(n, 2.5 + 0j))
    assert abs(c[0] - 2.5 * n) < 1e-10 and np.abs(c[1:]).max() < 1e-10


@pytest.mark.parametrize("n", [48, 75, 81, 1024, 160])
def test_fft1_roundtrip_and_parseval(n):
    x = crand(n, 7 * n)
    X = oracle.fft1(x)
    assert np.allclose(oracle.fft1(X, inverse=True), x, atol=1e-12)
    assert np.isclose((np.abs(X) ** 2).sum(), n * (np.abs(x) ** 2).sum(), rtol=1e-12)


def test_fft1_library_cross_check():
    # a special case that reduces to a library routine
    for n in (54, 100, 144, 150, 2160, 2560):
        x = crand(n, n + 1)
        assert np.allclose(oracle.fft1(x), np.fft.fft(x), atol=1e-9 * np.sqrt(n))


# ---------------------------------------------------------------- 3D FFT

@pytest.mark.parametrize("shape", [(4, 6, 5), (3, 5, 7), (8, 8, 8), (1, 1, 6), (2, 1, 3)])
def test_fft3_matches_brute(shape):
    x = crand(int(np.prod(shape)), 99).reshape(shape)
    Fz, Fy, Fx = (dft_matrix(n) for n in shape)
    ref = np.einsum("ai,bj,ck,ijk->abc", Fz, Fy, Fx, x)
    assert np.allclose(oracle.fft3(x), ref, atol=1e-10)
    assert np.allclose(oracle.fft3(ref, inverse=True), x, atol=1e-12)
    # Hermitian symmetry of the transform of a real field
    X = oracle.fft3(x.real)
    idx = tuple(np.ix_(*[(-np.arange(n)) % n for n in shape]))
    assert np.allclose(X, np.conj(X[idx]), atol=1e-10)


# ----------------------------------------------------------- convolution

def direct_circular_conv(h0, u):
    """out(y) = sum_x h0(x) u(y - x), written out with Python loops."""
    nz, ny, nx = u.shape
    out = np.zeros_like(u, dtype=np.float64)
    for (z, y, x) in itertools.product(range(nz), range(ny), range(nx)):
        s = 0.0
        for (a, b, c) in itertools.product(range(nz), range(ny), range(nx)):
            s += h0[a, b, c] * u[(z - a) % nz, (y - b) % ny, (x - c) % nx]
        out[z, y, x] = s
    return out


def test_center_to_origin_definition():
    shape = (3, 4, 5)
    p = np.arange(60, dtype=float).reshape(shape)
    h0 = oracle.center_to_origin(p)
    # the PSF centre floor(n/2) lands on the origin
    assert h0[0, 0, 0] == p[1, 2, 2]
    assert h0[0, 0, 1] == p[1, 2, 3]
    assert h0[0, 0, 4] == p[1, 2, 1]          # x = -1 wraps
    assert h0[2, 3, 0] == p[0, 1, 2]          # z = -1, y = -1


def test_convolution_against_direct_loops():
    shape = (3, 4, 5)
    r = np.random.default_rng(5)
    psf = r.uniform(0.1, 1.0, shape)          # deliberately not symmetric
    u = r.uniform(0.5, 2.0, shape)
    h0 = oracle.center_to_origin(psf)
    ref = direct_circular_conv(h0, u)
    H = oracle.psf_spectrum(psf)
    assert np.allclose(oracle.convolve(H, u), ref, atol=1e-12)
    assert np.allclose(oracle.conv3_direct(h0, u), ref, atol=1e-12)
    # the flipped PSF is the circular flip h0(-x)
    flip = h0[tuple(np.ix_(*[(-np.arange(n)) % n for n in shape]))]
    assert np.allclose(oracle.convolve(H, u, flipped=True), direct_circular_conv(flip, u), atol=1e-12)


def test_delta_psf_centering():
    shape = (4, 6, 5)
    u = np.random.default_rng(2).uniform(size=shape)
    c = tuple(n // 2 for n in shape)
    delta = np.zeros(shape)
    delta[c] = 1.0
    assert np.allclose(oracle.convolve(oracle.psf_spectrum(delta), u), u, atol=1e-13)
    # a delta one voxel right of the centre shifts the image by +1 along x
    delta2 = np.zeros(shape)
    delta2[c[0], c[1], c[2] + 1] = 1.0
    assert np.allclose(oracle.convolve(oracle.psf_spectrum(delta2), u), np.roll(u, 1, axis=2), atol=1e-13)
    # ... and one voxel up in z shifts by +1 along z
    delta3 = np.zeros(shape)
    delta3[c[0] + 1, c[1], c[2]] = 1.0
    assert np.allclose(oracle.convolve(oracle.psf_spectrum(delta3), u), np.roll(u, 1, axis=0), atol=1e-13)


def test_adjoint_identity():
    shape = (6, 5, 4)
    r = np.random.default_rng(11)
    psf = r.uniform(size=shape)
    H = oracle.psf_spectrum(psf)
    x, y = r.standard_normal(shape), r.standard_normal(shape)
    lhs = np.vdot(oracle.convolve(H, x), y)
    rhs = np.vdot(x, oracle.convolve(H, y, flipped=True))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs) * 10


# --------------------------------------------------------------- RL

def brute_rl(d, psf, n_iter, eps):
    """Second RL path: direct spatial convolutions, no FFT."""
    shape = d.shape
    h0 = oracle.center_to_origin(psf)
    flip = h0[tuple(np.ix_(*[(-np.arange(n)) % n for n in shape]))]
    u = np.full(shape, max(d.mean(), eps))
    for _ in range(n_iter):
        b = direct_circular_conv(h0, u)
        r = d / np.maximum(b, eps)
        q = direct_circular_conv(flip, r)
        u = u * q
    return u


def test_rl_matches_spatial_path():
    shape = (3, 4, 5)
    r = np.random.default_rng(21)
    d = r.uniform(1.0, 10.0, shape)
    psf = r.uniform(0.05, 1.0, shape)
    psf /= psf.sum()
    assert np.allclose(oracle.rl(d, psf, 4, 1e-6), brute_rl(d, psf, 4, 1e-6), rtol=1e-12, atol=0)


def test_rl_zero_iterations_is_initial_estimate():
    d = np.random.default_rng(3).uniform(0, 5, (4, 4, 4))
    out = oracle.rl(d, np.ones((4, 4, 4)) / 64, 0, 1e-6)
    assert np.allclose(out, d.mean())
    assert np.allclose(oracle.rl(np.zeros((2, 2, 2)), np.ones((2, 2, 2)), 0, 1e-3), 1e-3)


def test_rl_delta_psf_fixed_point():
    shape = (4, 6, 5)
    d = np.random.default_rng(4).uniform(1, 100, shape)
    psf = np.zeros(shape)
    psf[tuple(n // 2 for n in shape)] = 1.0
    for k in (1, 2, 5):
        assert np.allclose(oracle.rl(d, psf, k, 1e-6), d, rtol=1e-12)


def test_rl_constant_image():
    shape = (4, 5, 6)
    psf = np.random.default_rng(8).uniform(size=shape)
    psf /= psf.sum()
    d = np.full(shape, 7.25)
    assert np.allclose(oracle.rl(d, psf, 5, 1e-6), 7.25, rtol=1e-12)


def test_rl_single_voxel():
    assert np.allclose(oracle.rl(np.array([[[3.5]]]), np.array([[[0.3]]]), 1, 1e-6), 3.5)


def test_rl_first_iterate_closed_form():
    # from a constant start: u1 = (h flipped * d) / sum(h), independent of u0
    shape = (4, 5, 6)
    r = np.random.default_rng(9)
    psf = r.uniform(size=shape)
    d = r.uniform(1, 50, shape)
    h0 = oracle.center_to_origin(psf)
    flip = h0[tuple(np.ix_(*[(-np.arange(n)) % n for n in shape]))]
    expect = direct_circular_conv(flip, d) / psf.sum()
    assert np.allclose(oracle.rl(d, psf, 1, 1e-6), expect, rtol=1e-12)


def test_rl_scale_invariance_flux_nonnegativity():
    d, _ = synth.workload_volume(synth.SMALL)
    psf = oracle.psf_gaussian(d.shape, 1.5, 3.0)
    u = oracle.rl(d, psf, 6, 1e-6)
    u_scaled = oracle.rl(d, 3.0 * psf, 6, 1e-6)
    assert np.allclose(u, u_scaled, rtol=1e-10, atol=1e-9)
    # total flux is conserved for k >= 1 (clamp inactive)
    assert abs(u.sum() - d.astype(np.float64).sum()) <= 1e-10 * d.sum()
    assert u.min() >= 0.0


def test_rl_poisson_likelihood_monotone():
    shape = (8, 12, 10)
    d, _ = synth.make_volume(shape, 4, (1.5, 2.5), 5.0, 1.2, 2.0, 777)
    d = d.astype(np.float64)
    psf = oracle.psf_gaussian(shape, 1.2, 2.0)
    H = oracle.psf_spectrum(psf)
    u = np.full(shape, d.mean())
    prev = np.inf
    for _ in range(15):
        u_next, b, _, _ = oracle.rl_iterate(H, d, u, 1e-6)
        nll = np.sum(b - d * np.log(b))
        assert nll <= prev + 1e-9 * abs(prev if np.isfinite(prev) else 1)
        prev = nll
        u = u_next


def test_rl_separable_slices():
    # a PSF that is a delta along z decouples the slices: 3D RL == 2D RL per slice
    shape = (3, 8, 10)
    r = np.random.default_rng(31)
    d = r.uniform(1, 20, shape)
    p2 = r.uniform(0.1, 1, shape[1:])
    psf = np.zeros(shape)
    psf[shape[0] // 2] = p2
    u3 = oracle.rl(d, psf, 5, 1e-6)
    for z in range(shape[0]):
        u2 = oracle.rl(d[z:z + 1], p2[None], 5, 1e-6)
        assert np.allclose(u3[z], u2[0], rtol=1e-11)


def test_rl_iterate_intermediates():
    shape = (4, 5, 6)
    r = np.random.default_rng(41)
    d = r.uniform(1, 9, shape)
    psf = r.uniform(size=shape)
    H = oracle.psf_spectrum(psf)
    u = r.uniform(1, 2, shape)
    un, b, rr, q = oracle.rl_iterate(H, d, u, 1e-6)
    h0 = oracle.center_to_origin(psf)
    flip = h0[tuple(np.ix_(*[(-np.arange(n)) % n for n in shape]))]
    assert np.allclose(b, direct_circular_conv(h0, u), rtol=1e-12)
    assert np.allclose(rr, d / b, rtol=1e-12)
    assert np.allclose(q, direct_circular_conv(flip, rr), rtol=1e-12)
    assert np.allclose(un, u * q, rtol=1e-12)
    # clamp: a tiny b is replaced by eps
    d2 = np.ones(shape)
    u2 = np.zeros(shape)
    _, b2, r2, _ = oracle.rl_iterate(H, d2, u2, 0.5)
    assert np.allclose(b2, 0.0) and np.allclose(r2, 2.0)


# ----------------------------------------------------------- Gaussian PSF

def test_psf_gaussian_closed_form():
    shape = (9, 12, 11)
    sxy, sz, A = 1.7, 2.6, 1.3
    p = oracle.psf_gaussian(shape, sxy, sz, A)
    c = (4, 6, 5)
    assert np.isclose(p.sum(), A, rtol=1e-14)
    assert np.unravel_index(np.argmax(p), shape) == c
    assert np.isclose(p[4, 6, 6] / p[c], np.exp(-1 / (2 * sxy ** 2)), rtol=1e-14)
    assert np.isclose(p[4, 8, 5] / p[c], np.exp(-4 / (2 * sxy ** 2)), rtol=1e-14)
    assert np.isclose(p[6, 6, 5] / p[c], np.exp(-4 / (2 * sz ** 2)), rtol=1e-14)
    assert np.isclose(p[3, 7, 4] / p[c], np.exp(-2 / (2 * sxy ** 2) - 1 / (2 * sz ** 2)), rtol=1e-14)
    # centred => circularly symmetric about the origin after the shift => real spectrum
    H = oracle.psf_spectrum(oracle.psf_gaussian((8, 10, 6), sxy, sz, A))
    assert np.abs(H.imag).max() < 1e-14


def test_psf_gaussian_grad_fd():
    shape = (5, 7, 6)
    theta = np.array([1.4, 2.1, 0.8])
    w = np.random.default_rng(51).standard_normal(shape)

    def L(t):
        return np.sum(w * oracle.psf_gaussian(shape, *t))

    g = oracle.psf_gaussian_grad(shape, *theta, w)
    h = 1e-3
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (L(theta + e) - L(theta - e)) / (2 * h)
        assert np.isclose(g[i], fd, rtol=1e-5, atol=1e-9)


# -------------------------------------------------------------- gradient

def _loss_parts(shape, seed):
    r = np.random.default_rng(seed)
    d = r.uniform(2.0, 20.0, shape)
    xt = r.uniform(2.0, 20.0, shape)
    return d, xt


def test_rl_grad_image_fd():
    shape = (4, 5, 6)
    d, xt = _loss_parts(shape, 61)
    psf = oracle.psf_gaussian(shape, 1.1, 1.6)
    K, eps = 4, 1e-6

    def L(dd):
        u = oracle.rl(dd, psf, K, eps)
        return np.mean((u - xt) ** 2)

    u = oracle.rl(d, psf, K, eps)
    g_out = 2 * (u - xt) / u.size
    gd, _ = oracle.rl_grad(d, psf, K, eps, g_out)
    r = np.random.default_rng(62)
    h = 1e-3
    for _ in range(3):
        v = r.standard_normal(shape)
        fd = (L(d + h * v) - L(d - h * v)) / (2 * h)
        an = np.sum(gd * v)
        assert np.isclose(an, fd, rtol=1e-5, atol=1e-10)
    # single-voxel directions exercise the per-voxel terms
    for idx in [(0, 0, 0), (2, 3, 1), (3, 4, 5)]:
        v = np.zeros(shape)
        v[idx] = 1.0
        fd = (L(d + h * v) - L(d - h * v)) / (2 * h)
        assert np.isclose(gd[idx], fd, rtol=1e-5, atol=1e-10)


def test_rl_grad_psf_fd():
    shape = (5, 4, 6)
    d, xt = _loss_parts(shape, 71)
    r = np.random.default_rng(72)
    psf = r.uniform(0.2, 1.0, shape)            # not symmetric: exercises both correlation terms
    psf /= psf.sum()
    K, eps = 3, 1e-6

    def L(p):
        return np.mean((oracle.rl(d, p, K, eps) - xt) ** 2)

    u = oracle.rl(d, psf, K, eps)
    _, gp = oracle.rl_grad(d, psf, K, eps, 2 * (u - xt) / u.size)
    h = 1e-6                                    # PSF entries are ~1e-2; error falls as h^2
    for _ in range(3):
        v = r.standard_normal(shape)
        fd = (L(psf + h * v) - L(psf - h * v)) / (2 * h)
        assert np.isclose(np.sum(gp * v), fd, rtol=1e-5, atol=1e-10)
    # scale invariance => the gradient is orthogonal to the PSF itself
    assert abs(np.sum(gp * psf)) <= 1e-10 * np.abs(gp).sum() * np.abs(psf).max() + 1e-14


def test_rl_grad_params_fd():
    # end to end: d L / d(sigma_xy, sigma_z, A) through the Gaussian PSF and RL
    shape = (6, 8, 8)
    d, xt = _loss_parts(shape, 81)
    theta = np.array([1.3, 1.9, 1.0])
    K, eps = 3, 1e-6

    def L(t):
        return np.mean((oracle.rl(d, oracle.psf_gaussian(shape, *t), K, eps) - xt) ** 2)

    psf = oracle.psf_gaussian(shape, *theta)
    u = oracle.rl(d, psf, K, eps)
    _, gp = oracle.rl_grad(d, psf, K, eps, 2 * (u - xt) / u.size)
    g = oracle.psf_gaussian_grad(shape, *theta, gp)
    h = 1e-3
    for i in range(3):
        e = np.zeros(3)
        e[i] = h
        fd = (L(theta + e) - L(theta - e)) / (2 * h)
        assert np.isclose(g[i], fd, rtol=1e-5, atol=1e-11)
    assert abs(g[2]) < 1e-10        # RL is invariant to the PSF amplitude


def test_rl_grad_zero_iterations():
    # n_iter = 0: u = mean(d) everywhere, so dL/dd_i = sum(g_out) / V
    shape = (3, 4, 5)
    d, _ = _loss_parts(shape, 91)
    g = np.random.default_rng(92).standard_normal(shape)
    gd, gp = oracle.rl_grad(d, np.ones(shape) / 60, 0, 1e-6, g)
    assert np.allclose(gd, g.sum() / g.size)
    assert np.allclose(gp, 0.0)


# ------------------------------------------------------- automatic stopping

def test_rl_auto_delta_psf_stops_after_two():
    # delta PSF: u1 = d, u2 = d, so delta_0 = ||d - u0|| / ||u0|| and delta_1 = 0
    shape = (4, 6, 5)
    d = np.random.default_rng(14).uniform(1, 100, shape)
    psf = np.zeros(shape)
    psf[tuple(n // 2 for n in shape)] = 1.0
    out, n, hist = oracle.rl_auto(d, psf, 20, 1e-6, 1e-12, 1)
    u0 = d.mean()
    assert n == 2
    assert np.isclose(hist[0], np.linalg.norm(d - u0) / (u0 * np.sqrt(d.size)), rtol=1e-12)
    assert hist[1] < 1e-13               # zero up to the rounding of the FFT path
    assert np.allclose(out, d, rtol=1e-12)


def test_rl_auto_constant_image_stops_at_once():
    shape = (4, 5, 6)
    psf = np.random.default_rng(8).uniform(size=shape)
    psf /= psf.sum()
    out, n, hist = oracle.rl_auto(np.full(shape, 3.0), psf, 10, 1e-6, 1e-9, 1)
    assert n == 1 and hist[0] < 1e-12 and np.allclose(out, 3.0)


def test_rl_auto_history_and_check_cadence():
    d, _ = synth.workload_volume(synth.SMALL)
    psf = oracle.psf_gaussian(d.shape, 1.5, 3.0)
    _, n_all, hist = oracle.rl_auto(d, psf, 12, 1e-6, 0.0, 1)       # tol 0: never stops early
    assert n_all == 12
    # delta_k from separately computed iterates (a second path through rl())
    for k in (0, 3, 7):
        uk = oracle.rl(d, psf, k, 1e-6)
        uk1 = oracle.rl(d, psf, k + 1, 1e-6)
        assert np.isclose(hist[k], np.linalg.norm(uk1 - uk) / np.linalg.norm(uk), rtol=1e-10)
    # the first delta below a threshold is at index j; a check every 4 iterations stops at the
    # first multiple of 4 whose own delta is below it
    tol = 0.5 * (hist[5] + hist[6]) if hist[6] < hist[5] else hist[6] * 1.01
    out, n, h = oracle.rl_auto(d, psf, 12, 1e-6, tol, 4)
    checks = [k for k in range(4, 13, 4) if hist[k - 1] < tol]
    assert n == (checks[0] if checks else 12)
    assert np.allclose(out, oracle.rl(d, psf, n, 1e-6), rtol=1e-12)


# ------------------------------------------------------- Fourier Shell Correlation

def _tone(shape, k):
    idx = np.indices(shape).astype(float)
    return np.cos(2 * np.pi * sum(k[i] * idx[i] / shape[i] for i in range(3)))


def test_fsc_identity_sign_and_scale():
    shape = (8, 12, 10)
    a = np.random.default_rng(1).standard_normal(shape)
    f, num, da, db = oracle.fsc(a, a, 6)
    nonempty = da > 0
    assert np.allclose(f[nonempty], 1.0, atol=1e-12)
    assert np.allclose(oracle.fsc(a, -2.5 * a, 6)[0][nonempty], -1.0, atol=1e-12)
    assert np.allclose(oracle.fsc(a, 3.0 * a, 6)[0][nonempty], 1.0, atol=1e-12)


def test_fsc_single_tone_closed_forms():
    shape = (8, 16, 12)
    k0 = (1, 3, 2)
    a = _tone(shape, k0)
    V = a.size
    rho = np.sqrt(sum((k0[i] / shape[i]) ** 2 for i in range(3)))
    n_sh = 10
    s0 = int(np.floor(2 * n_sh * rho))
    f, num, da, db = oracle.fsc(a, a, n_sh)
    # all energy in one shell: |A(+-k0)| = V/2, so sum |A|^2 = V^2 / 2
    assert np.isclose(da[s0], V * V / 2, rtol=1e-12)
    assert np.allclose(np.delete(da, s0), 0.0, atol=1e-9 * V * V)
    # a circular shift by s multiplies A by exp(-2 pi i k.s / n): FSC = cos(2 pi k0.s / n)
    s = (2, 5, 1)
    b = np.roll(a, s, axis=(0, 1, 2))
    phase = 2 * np.pi * sum(k0[i] * s[i] / shape[i] for i in range(3))
    assert np.isclose(oracle.fsc(a, b, n_sh)[0][s0], np.cos(phase), atol=1e-12)


def test_fsc_excludes_beyond_nyquist_and_counts_both_halves():
    # a tone at the corner (rho > 1/2) contributes nothing; Parseval over shells for a
    # field with no energy beyond Nyquist
    shape = (8, 8, 8)
    corner = _tone(shape, (4, 4, 4))
    assert np.allclose(oracle.fsc(corner, corner, 4)[2], 0.0, atol=1e-9)
    lowpass = _tone(shape, (1, 0, 0)) + 0.5 * _tone(shape, (0, 2, 1)) + 0.25
    _, _, da, _ = oracle.fsc(lowpass, lowpass, 8)
    assert np.isclose(da.sum(), lowpass.size * (lowpass ** 2).sum(), rtol=1e-12)


def test_fsc_shell_edges_exact():
    # tones sitting exactly on shell edges: rho = 1/4 with 4 shells -> shell 2, rho = 1/8 -> shell 1
    shape = (8, 8, 8)
    for k0, shell in (((0, 2, 0), 2), ((0, 0, 1), 1), ((2, 0, 0), 2)):
        a = _tone(shape, k0)
        _, _, da, _ = oracle.fsc(a, a, 4)
        assert da[shell] > 0 and np.count_nonzero(da > 1e-9) == 1, (k0, da)


# ------------------------------------------------------ accelerated RL (Biggs-Andrews)
#
# The extrapolation is pinned on a linear step psi(y) = xs + lam (y - xs), whose
# iterates follow in closed form:
#   - 0 < lam < 1: the moves are all parallel, alpha_k = lam^(k-1) (k >= 2), and the
#     error after n steps is lam^(1 + n(n-1)/2) e0 (by induction on the exponents);
#   - lam < 0: the ratio of successive changes is lam < 0, so alpha clamps to 0 and the
#     plain iteration remains, error lam^n e0;
#   - lam > 1: the ratio exceeds 1, alpha clamps to 1, and the error coefficient s_n
#     follows s_{n+1} = lam (2 s_n - s_{n-1}) from s_1 = lam, s_2 = lam^2.
# The RL composition is pinned by the cases where RL itself has a closed form.

def test_accel_linear_contraction_closed_form():
    r = np.random.default_rng(71)
    xs = np.full(64, 5.0)
    e0 = r.uniform(-1, 1, 64)
    for lam in (0.3, 0.7, 0.9):
        for n in range(1, 9):
            x, a = oracle.accel_linear(xs, np.full(64, lam), xs + e0, n)
            assert np.allclose(x - xs, lam ** (1 + n * (n - 1) // 2) * e0, rtol=1e-10, atol=1e-14)
            assert np.allclose(a, [0.0, 0.0] + [lam ** (k - 1) for k in range(2, n)][:max(0, n - 2)])


def test_accel_linear_alpha_clamps():
    r = np.random.default_rng(72)
    xs = np.full(32, 5.0)
    e0 = r.uniform(-1, 1, 32)
    # negative ratio: alpha clamps to 0, plain iteration
    x, a = oracle.accel_linear(xs, np.full(32, -0.6), xs + e0, 7)
    assert np.all(a == 0.0)
    assert np.allclose(x - xs, (-0.6) ** 7 * e0, rtol=1e-12)
    # ratio above 1: alpha clamps to 1 from k = 2 on
    lam, n = 1.3, 8
    x, a = oracle.accel_linear(xs, np.full(32, lam), xs + 0.01 * e0, n)
    assert np.all(a[:2] == 0.0) and np.all(a[2:] == 1.0)
    z1, z2 = lam + np.sqrt(lam * lam - lam), lam - np.sqrt(lam * lam - lam)
    # s_k = A z1^k + B z2^k through s_1 = lam, s_2 = lam^2
    A, B = np.linalg.solve([[z1, z2], [z1 ** 2, z2 ** 2]], [lam, lam ** 2])
    assert np.allclose(x - xs, (A * z1 ** n + B * z2 ** n) * 0.01 * e0, rtol=1e-10)


def test_accel_linear_prediction_clamped_at_zero():
    # voxel 0 decays slowly and sets alpha near 0.9; voxel 1 decays fast, so the
    # prediction along its last move is negative at k = 2 and is set to 0, after which
    # psi keeps it at 0 (xs = 0) for good
    xs = np.zeros(2)
    lam = np.array([0.9, 0.2])
    x0 = np.array([1.0, 0.01])
    _, a = oracle.accel_linear(xs, lam, x0, 3)
    assert 0.85 < a[2] < 0.95
    unclamped = 0.2 * 0.01 * (0.2 + a[2] * 0.2 - a[2])
    assert unclamped < 0
    for n in (3, 4, 6):
        x, _ = oracle.accel_linear(xs, lam, x0, n)
        assert x[1] == 0.0 and x[0] > 0.0


def test_rl_accel_first_two_iterates_are_plain_rl():
    d, _ = synth.make_volume((6, 8, 10), 3, (1.0, 2.0), 5.0, 1.0, 1.5, 73)
    psf = oracle.psf_gaussian(d.shape, 1.0, 1.5)
    for n in (0, 1, 2):
        x, a = oracle.rl_accel(d, psf, n, 1e-6)
        assert np.allclose(x, oracle.rl(d, psf, n, 1e-6), rtol=1e-13, atol=0)
        assert np.all(a == 0.0)


def test_rl_accel_delta_and_constant_fixed_points():
    shape = (4, 6, 5)
    d = np.random.default_rng(74).uniform(1, 100, shape)
    psf = np.zeros(shape)
    psf[tuple(n // 2 for n in shape)] = 1.0
    for n in (1, 3, 6):
        x, a = oracle.rl_accel(d, psf, n, 1e-6)
        assert np.allclose(x, d, rtol=1e-12)
        assert np.all(a == 0.0)   # g_1 = 0: no move to extrapolate
    # constant image, normalised PSF: every change is at rounding level, so whatever
    # alpha their ratio gives, the estimate stays at the constant
    psf = np.random.default_rng(75).uniform(size=shape)
    psf /= psf.sum()
    x, a = oracle.rl_accel(np.full(shape, 3.5), psf, 6, 1e-6)
    assert np.allclose(x, 3.5, rtol=1e-12) and np.all((a >= 0) & (a <= 1))
    # exactly zero changes (the 0/0 ratio) give alpha = 0: a linear step at its fixed point
    x, a = oracle.accel_linear(np.full(8, 2.0), np.full(8, 0.5), np.full(8, 2.0), 5)
    assert np.all(x == 2.0) and np.all(a == 0.0)


def test_rl_accel_flux_nonnegativity_and_speedup():
    d, _ = synth.workload_volume(synth.SMALL)
    d = d.astype(np.float64)
    psf = oracle.psf_gaussian(d.shape, 1.5, 3.0)
    n = 20
    x, a = oracle.rl_accel(d, psf, n, 1e-6)
    assert x.min() >= 0.0
    # every RL step conserves the flux of a normalised PSF, whatever point it starts from
    assert abs(x.sum() - d.sum()) <= 1e-10 * d.sum()
    assert np.all((a >= 0) & (a <= 1)) and a[2:].max() > 0.5
    # the point of the method: RL maximises the Poisson likelihood, and the accelerated
    # run gets further in n steps than plain RL in 2n
    H = oracle.psf_spectrum(psf)

    def nll(u):
        b = oracle.convolve(H, u)
        return float(np.sum(b - d * np.log(np.maximum(b, 1e-6))))

    assert nll(x) < nll(oracle.rl(d, psf, 2 * n, 1e-6))


# ---------------------------------------------- metric-guided stopping: NLL, PSNR

def test_poisson_nll_closed_form_and_clamp():
    r = np.random.default_rng(81)
    d = r.uniform(1, 50, 200)
    assert np.isclose(oracle.poisson_nll(d, d, 1e-6), np.sum(d - d * np.log(d)), rtol=1e-14)
    b = d.copy()
    b[:10] = -3.0       # clamped to eps
    expect = np.sum(d[10:] - d[10:] * np.log(d[10:])) + np.sum(0.5 - d[:10] * np.log(0.5))
    assert np.isclose(oracle.poisson_nll(b, d, 0.5), expect, rtol=1e-14)


def test_psnr_si_closed_form_and_invariance():
    r = np.random.default_rng(82)
    y = r.uniform(0, 10, 1000)
    e = r.standard_normal(1000)
    A = np.stack([np.ones_like(y), y], 1)
    e -= A @ np.linalg.lstsq(A, e, rcond=None)[0]      # e orthogonal to 1 and y
    x = y + e
    vy, ve = y.var(), e.var()
    expect = 20 * np.log10((y.max() - y.min()) / np.sqrt(vy * ve / (vy + ve)))
    assert np.isclose(oracle.psnr_si(x, y), expect, rtol=1e-12)
    # invariant under any affine map of the estimate, a sign flip included
    assert np.isclose(oracle.psnr_si(-2.5 * x + 7.0, y), expect, rtol=1e-12)
    assert oracle.psnr_si(3.0 * y + 2.0, y) > 250     # exact up to rounding
    assert oracle.psnr_si(np.full(1000, 4.0), y) == pytest.approx(20 * np.log10((y.max() - y.min()) / y.std()))


def test_rl_monitor_history_recomputed():
    d, xt = synth.workload_volume(synth.SMALL)
    d = d.astype(np.float64)
    psf = oracle.psf_gaussian(d.shape, 1.5, 3.0)
    H = oracle.psf_spectrum(psf)
    _, n, h = oracle.rl_monitor(d, psf, 6, 1e-6, oracle.METRIC_REL_CHANGE, 0.0, 1, xt)
    assert n == 6
    _, _, deltas = oracle.rl_auto(d, psf, 6, 1e-6, 0.0, 1)
    assert np.allclose(h[:, 0], deltas, rtol=1e-12)
    for k in range(6):
        uk = oracle.rl(d, psf, k, 1e-6)
        assert np.isclose(h[k, 1], oracle.poisson_nll(oracle.convolve(H, uk), d, 1e-6), rtol=1e-12)
        assert np.isclose(h[k, 2], oracle.psnr_si(oracle.rl(d, psf, k + 1, 1e-6), xt), rtol=1e-12)
    assert np.all(np.diff(h[:, 1]) <= 1e-9 * np.abs(h[1:, 1]))   # EM: the likelihood never falls
    _, _, h2 = oracle.rl_monitor(d, psf, 3, 1e-6, oracle.METRIC_REL_CHANGE, 0.0, 1, None)
    assert np.all(np.isnan(h2[:, 2]))


def test_rl_monitor_stopping_rules():
    d, xt = synth.workload_volume(synth.SMALL)
    psf = oracle.psf_gaussian(d.shape, 1.5, 3.0)
    _, _, h = oracle.rl_monitor(d, psf, 40, 1e-6, oracle.METRIC_REL_CHANGE, 0.0, 1, xt)
    # PSNR: tol 0 stops after the first iteration whose PSNR is below the previous one
    drop = next(k for k in range(1, 40) if h[k, 2] - h[k - 1, 2] < 0)
    _, n, _ = oracle.rl_monitor(d, psf, 40, 1e-6, oracle.METRIC_PSNR, 0.0, 1, xt)
    assert n == drop + 1
    # NLL: the first check whose relative decrease is under tol
    rel = (h[:-1, 1] - h[1:, 1]) / np.abs(h[1:, 1])
    tol = 0.5 * (rel[10] + rel[11])
    first = next(k for k in range(1, 40) if rel[k - 1] < tol)
    _, n, _ = oracle.rl_monitor(d, psf, 40, 1e-6, oracle.METRIC_NLL, tol, 1, xt)
    assert n == first + 1
    # checks only every third iteration
    _, n, _ = oracle.rl_monitor(d, psf, 40, 1e-6, oracle.METRIC_NLL, tol, 3, xt)
    assert n % 3 == 0 and n >= first + 1 and n - 3 < first + 1


# ------------------------------------------------- linear ("same"-mode) boundaries

def direct_same(psf, u, flipped=False):
    """b(x) = sum_t p(t + c) u(x - t) over x - t inside the box (adjoint: u(x + t))."""
    n, k = u.shape, psf.shape
    c = [kk // 2 for kk in k]
    out = np.zeros(n)
    for x in itertools.product(*[range(v) for v in n]):
        s = 0.0
        for t0 in range(-c[0], k[0] - c[0]):
            for t1 in range(-c[1], k[1] - c[1]):
                for t2 in range(-c[2], k[2] - c[2]):
                    y = (x[0] + t0, x[1] + t1, x[2] + t2) if flipped else (x[0] - t0, x[1] - t1, x[2] - t2)
                    if all(0 <= y[i] < n[i] for i in range(3)):
                        s += psf[t0 + c[0], t1 + c[1], t2 + c[2]] * u[y]
        out[x] = s
    return out


@pytest.mark.parametrize("n,k", [((3, 4, 5), (3, 2, 5)), ((4, 3, 2), (5, 7, 3)), ((2, 5, 6), (1, 1, 1))])
def test_conv_same_against_direct_loops(n, k):
    r = np.random.default_rng(sum(n) + 10 * sum(k))
    psf = r.uniform(0, 1, k)
    u = r.uniform(-1, 1, n)
    for flipped in (False, True):
        assert np.allclose(oracle.conv_same(psf, u, flipped), direct_same(psf, u, flipped), rtol=1e-12, atol=1e-13)


def test_conv_same_adjoint_identity():
    r = np.random.default_rng(91)
    psf = r.uniform(0, 1, (5, 3, 4))
    x = r.standard_normal((6, 7, 9))
    y = r.standard_normal((6, 7, 9))
    lhs = np.vdot(oracle.conv_same(psf, x), y)
    rhs = np.vdot(x, oracle.conv_same(psf, y, True))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_conv_same_equals_circular_away_from_the_border():
    # an object with zero margins of at least the PSF's half-width never meets the border,
    # so zero padding and wrap-around give the same blur
    n, k = (12, 14, 16), (5, 3, 7)
    r = np.random.default_rng(92)
    psf = r.uniform(0, 1, k)
    u = np.zeros(n)
    u[3:-3, 2:-2, 4:-4] = r.uniform(0, 1, (6, 10, 8))
    big = np.zeros(n)
    sl = tuple(slice(nn // 2 - kk // 2, nn // 2 - kk // 2 + kk) for nn, kk in zip(n, k))
    big[sl] = psf            # the same PSF, peak at floor(n/2) of an image-sized box
    H = oracle.psf_spectrum(big)
    assert np.allclose(oracle.conv_same(psf, u), oracle.convolve(H, u), atol=1e-12)
    assert np.allclose(oracle.conv_same(psf, u, True), oracle.convolve(H, u, True), atol=1e-12)


def test_rl_same_matches_direct_path_and_keeps_flux():
    shape, k = (4, 5, 6), (3, 5, 3)
    r = np.random.default_rng(93)
    d = r.uniform(1, 20, shape)
    psf = r.uniform(0.1, 1, k)
    psf /= psf.sum()
    u = np.full(shape, d.mean())
    for _ in range(4):
        b = direct_same(psf, u)
        u = u * direct_same(psf, d / np.maximum(b, 1e-6), True)
    got = oracle.rl_same(d, psf, 4, 1e-6)
    assert np.allclose(got, u, rtol=1e-11)
    # each step keeps the total flux (the adjoint pairs the ratio with the blur it divides)
    assert abs(got.sum() - d.sum()) <= 1e-11 * d.sum()
    # a 1-voxel PSF makes the first iterate the image itself
    assert np.allclose(oracle.rl_same(d, np.array([[[0.7]]]), 1, 1e-6), d, rtol=1e-12)


def test_rl_accel_same_composition():
    # the extrapolation (pinned above) around the same-mode step (pinned by direct loops):
    # the first two iterates are plain same-mode RL, flux stays, alpha stays in [0, 1]
    r = np.random.default_rng(95)
    d = r.uniform(1, 20, (5, 6, 7))
    psf = r.uniform(0.1, 1, (3, 3, 5))
    psf /= psf.sum()
    for n in (0, 1, 2):
        x, a = oracle.rl_accel_same(d, psf, n, 1e-6)
        assert np.allclose(x, oracle.rl_same(d, psf, n, 1e-6), rtol=1e-13, atol=0) and np.all(a == 0)
    x, a = oracle.rl_accel_same(d, psf, 10, 1e-6)
    assert abs(x.sum() - d.sum()) <= 1e-11 * d.sum() and x.min() >= 0
    assert np.all((a >= 0) & (a <= 1)) and a[2:].max() > 0.3


def test_rl_monitor_same_against_direct_loops():
    # every measure of the linear-boundary monitor from the direct loops: delta_k, the
    # likelihood of u_k from its same-mode blur over the image box, the PSNR of u_{k+1}
    shape, k = (4, 5, 6), (3, 5, 3)
    r = np.random.default_rng(96)
    d = r.uniform(1, 20, shape)
    ref = r.uniform(0, 10, shape)
    psf = r.uniform(0.1, 1, k)
    psf /= psf.sum()
    eps = 1e-6
    u = np.full(shape, d.mean())
    rows = []
    for _ in range(5):
        b = direct_same(psf, u)
        c = np.maximum(b, eps)
        un = u * direct_same(psf, d / c, True)
        rows.append((np.linalg.norm(un - u) / np.linalg.norm(u), np.sum(c - d * np.log(c)),
                     oracle.psnr_si(un, ref)))
        u = un
    out, n, h = oracle.rl_monitor_same(d, psf, 5, eps, oracle.METRIC_REL_CHANGE, 0.0, 1, ref)
    assert n == 5 and np.allclose(out, u, rtol=1e-11)
    assert np.allclose(h, np.array(rows), rtol=1e-10, atol=0)
    # the stop rules read the same history as the circular monitor: stop at the first check
    # whose likelihood gain falls under tol
    gain = (h[:-1, 1] - h[1:, 1]) / np.abs(h[1:, 1])
    tol = 0.5 * (gain[1] + gain[2])
    _, n, _ = oracle.rl_monitor_same(d, psf, 5, eps, oracle.METRIC_NLL, tol, 1, ref)
    assert n == 4 and np.allclose(oracle.rl_monitor_same(d, psf, n, eps, 0, 0.0, 1)[0], oracle.rl_same(d, psf, n, eps),
                                  rtol=1e-13, atol=0)


def test_rl_monitor_same_one_voxel_psf_closed_form():
    # a 1-voxel PSF: b = u, so u_1 = d and every later step leaves it there
    d = np.random.default_rng(99).uniform(1, 20, (3, 4, 5))
    u0 = d.mean()
    _, n, h = oracle.rl_monitor_same(d, np.ones((1, 1, 1)), 3, 1e-6, oracle.METRIC_REL_CHANGE, -1.0, 1)
    assert n == 3
    assert np.isclose(h[0, 0], np.linalg.norm(d - u0) / (u0 * np.sqrt(d.size)), rtol=1e-12)
    assert np.isclose(h[0, 1], np.sum(u0 - d * np.log(u0)), rtol=1e-12)
    assert np.allclose(h[1:, 0], 0.0, atol=1e-15)
    assert np.allclose(h[1:, 1], np.sum(d - d * np.log(d)), rtol=1e-12)
    assert np.all(np.isnan(h[:, 2]))


# ------------------------------------------------------------ single-image FSC

def test_fsc_split_block_constant_and_checkerboard():
    r = np.random.default_rng(97)
    # every 2x2x2 block constant: the eight parity sub-volumes are identical
    base = r.uniform(1, 5, (4, 5, 6))
    d = np.repeat(np.repeat(np.repeat(base, 2, 0), 2, 1), 2, 2)
    f = oracle.fsc_split(d, 6)
    _, num, _, _ = oracle.fsc(base, base, 6)
    assert np.allclose(f[num != 0], 1.0, atol=1e-12) and np.all(f[num == 0] == 0.0)
    # c + A (-1)^(z+y+x): each sub-volume is a constant, opposite ones c + A and c - A, so
    # the DC shell holds sign(c^2 - A^2) (the other shells carry only rounding noise)
    z, y, x = np.meshgrid(np.arange(8), np.arange(10), np.arange(12), indexing="ij")
    for c, A, sign in ((3.0, 1.0, 1.0), (1.0, 3.0, -1.0)):
        f = oracle.fsc_split(c + A * (-1.0) ** (z + y + x), 4)
        assert np.isclose(f[0], sign, atol=1e-12) and np.all(np.abs(f) <= 1.0 + 1e-12)


def test_fsc_split_matches_sliced_pairs():
    d = np.random.default_rng(98).uniform(0, 1, (8, 12, 10))
    ref = np.zeros(5)
    for b in (0, 1):
        for c in (0, 1):
            ref += 0.25 * oracle.fsc(d[0::2, b::2, c::2], d[1::2, 1 - b::2, 1 - c::2], 5)[0]
    assert np.allclose(oracle.fsc_split(d, 5), ref, atol=1e-13)
