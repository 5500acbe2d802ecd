"""Linear ("same"-mode, zero-padded) boundaries on the GPU against the FP64 oracle.

The GPU plan transforms on padded lengths m >= max(n + floor(k/2), k), the oracle on
n + k - 1: both give the same "same"-mode result, so the estimates must agree to the
plain path's tolerance (relative L2 <= 1e-4 after 20 iterations) and convolutions to 1e-5.
"""
import numpy as np
import pytest

import oracle
from paper_2510_14143_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cr():
    from paper_2510_14143_gb300 import build
    build.build()
    import paper_2510_14143_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def gaussian_box(k, sxy, sz):
    c = [kk // 2 for kk in k]
    z, y, x = np.meshgrid(*[np.arange(kk) - cc for kk, cc in zip(k, c)], indexing="ij")
    g = np.exp(-(x * x + y * y) / (2 * sxy * sxy) - z * z / (2 * sz * sz))
    return (g / g.sum()).astype(np.float32)


CONV_CASES = [((12, 20, 24), (5, 7, 7)), ((9, 15, 30), (4, 6, 3)), ((8, 10, 6), (11, 13, 9)),
              ((16, 48, 50), (9, 9, 9)), ((1, 24, 40), (1, 5, 5)), ((30, 1, 16), (7, 1, 3))]


@pytest.mark.parametrize("n,k", CONV_CASES)
def test_linear_convolve_matches_oracle(cr, n, k):
    r = np.random.default_rng(sum(n) + sum(k))
    psf = r.uniform(0, 1, k).astype(np.float32)
    x = r.uniform(-1, 1, n).astype(np.float32)
    plan = cr.cubic_rl_plan_linear(n, dev(psf))
    im, tr = cr.cubic_rl_plan_dims(plan)
    assert im == n and all(t >= max(nn + kk // 2, kk) for t, nn, kk in zip(tr, n, k))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    for flipped in (False, True):
        cr.cubic_rl_convolve(plan, dev(x), flipped, out)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), oracle.conv_same(psf, x, flipped)) < 1e-5, flipped


@pytest.mark.parametrize("n,k,n_iter", [((32, 64, 64), (9, 11, 11), 20), ((15, 45, 50), (7, 9, 5), 12),
                                        ((10, 12, 16), (3, 3, 3), 0), ((10, 12, 16), (3, 3, 3), 1),
                                        ((6, 8, 10), (9, 11, 13), 8)])
def test_linear_rl_matches_oracle(cr, n, k, n_iter):
    d, _ = synth.make_volume(n, max(2, int(np.prod(n)) // 20000), (1.5, 3.0), 10.0, 1.5, 3.0, 777 + sum(n))
    psf = gaussian_box(k, 1.5, 2.5)
    plan = cr.cubic_rl_plan_linear(n, dev(psf))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    cr.cubic_rl_deconvolve(plan, dev(d), n_iter, 1e-6, out)
    torch.cuda.synchronize()
    ref = oracle.rl_same(d, psf, n_iter, 1e-6)
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-4


def test_linear_equals_circular_away_from_the_border(cr):
    # zero margins wider than the PSF's half-width: the same-mode blur is the circular one
    n, k = (16, 32, 40), (5, 7, 9)
    r = np.random.default_rng(5)
    psf = r.uniform(0, 1, k).astype(np.float32)
    x = np.zeros(n, np.float32)
    x[3:-3, 4:-4, 5:-5] = r.uniform(0, 1, (10, 24, 30))
    big = np.zeros(n, np.float32)
    big[tuple(slice(nn // 2 - kk // 2, nn // 2 - kk // 2 + kk) for nn, kk in zip(n, k))] = psf
    lin = cr.cubic_rl_plan_linear(n, dev(psf))
    circ = cr.cubic_rl_plan(n, dev(big))
    a = torch.empty(n, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    cr.cubic_rl_convolve(lin, dev(x), False, a)
    cr.cubic_rl_convolve(circ, dev(x), False, b)
    torch.cuda.synchronize()
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy().astype(np.float64)) < 1e-5


def test_linear_paper_shape_properties(cr):
    # the paper's stack shape with a 31 x 33 x 33 PSF box: padded to 45 x 2304 x 2592;
    # flux is conserved by every same-mode step (its adjoint pairs the ratio with the
    # blur it divides), and the estimate stays non-negative
    w = synth.PAPER
    psf = gaussian_box((31, 33, 33), w.psf_sigma_xy, w.psf_sigma_z)
    plan = cr.cubic_rl_plan_linear(w.shape, dev(psf))
    assert cr.cubic_rl_plan_dims(plan) == (w.shape, (45, 2304, 2592))
    g = torch.Generator(device="cuda").manual_seed(9)
    d = torch.poisson(20.0 + 300.0 * torch.rand(w.shape, device="cuda", generator=g) ** 12, generator=g)
    out = torch.empty_like(d)
    cr.cubic_rl_deconvolve(plan, d, 5, 1e-6, out)
    torch.cuda.synchronize()
    flux = d.double().sum().item()
    assert abs(out.double().sum().item() - flux) <= 1e-5 * flux
    assert out.min().item() >= 0.0


def test_linear_autotune_and_update_psf(cr):
    n, k = (24, 40, 48), (7, 9, 9)
    d, _ = synth.make_volume(n, 3, (1.5, 3.0), 10.0, 1.5, 3.0, 31)
    psf = gaussian_box(k, 1.2, 2.0)
    plan = cr.cubic_rl_plan_linear(n, dev(np.ones(k, np.float32) / np.prod(k)))
    cr.cubic_rl_plan_update_psf(plan, dev(psf))
    dd = dev(d)
    out = torch.empty_like(dd)
    cr.cubic_rl_autotune(plan, dd, out)
    cr.cubic_rl_deconvolve(plan, dd, 10, 1e-6, out)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), oracle.rl_same(d, psf, 10, 1e-6)) <= 1e-4


@pytest.mark.parametrize("n,k", [((24, 40, 48), (7, 9, 9)), ((9, 15, 30), (5, 5, 3))])
def test_linear_accelerated_matches_oracle(cr, n, k):
    d, _ = synth.make_volume(n, 3, (1.5, 3.0), 10.0, 1.5, 3.0, 41 + sum(n))
    psf = gaussian_box(k, 1.3, 2.2)
    plan = cr.cubic_rl_plan_linear(n, dev(psf))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    alpha = torch.empty(12, dtype=torch.float32, device="cuda")
    cr.cubic_rl_deconvolve_accel(plan, dev(d), 12, 1e-6, out, alpha)
    torch.cuda.synchronize()
    ref, a_ref = oracle.rl_accel_same(d, psf, 12, 1e-6)
    assert rel_l2(out.cpu().numpy(), ref) <= 1e-4
    assert np.allclose(alpha.cpu().numpy(), a_ref, atol=1e-3)


def test_linear_automatic_stopping(cr):
    n, k = (24, 40, 48), (7, 9, 9)
    d, _ = synth.make_volume(n, 3, (1.5, 3.0), 10.0, 1.5, 3.0, 57)
    psf = gaussian_box(k, 1.3, 2.2)
    plan = cr.cubic_rl_plan_linear(n, dev(psf))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    n_all, hist = cr.cubic_rl_deconvolve_auto(plan, dev(d), 25, 1e-6, 0.0, 1, out)
    assert n_all == 25 and all(h2 < h1 for h1, h2 in zip(hist[1:], hist[2:]))
    tol = 0.5 * (hist[9] + hist[10])
    n_stop, _ = cr.cubic_rl_deconvolve_auto(plan, dev(d), 25, 1e-6, tol, 1, out)
    assert n_stop == 11                      # the first check with delta under tol
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), oracle.rl_same(d, psf, n_stop, 1e-6)) <= 1e-4


@pytest.mark.parametrize("n,k", [((24, 40, 48), (7, 9, 9)), ((9, 15, 30), (5, 5, 3))])
def test_linear_monitor_matches_oracle(cr, n, k):
    # the likelihood counts the image's voxels only (not the blur in the padding), the
    # PSNR is taken on the cropped estimate; thresholds midway between two gains stop both
    # sides at the same iteration
    d, xt = synth.make_volume(n, 3, (1.5, 3.0), 10.0, 1.5, 3.0, 61 + sum(n))
    psf = gaussian_box(k, 1.3, 2.2)
    ref_out, _, h_ref = oracle.rl_monitor_same(d, psf, 12, 1e-6, oracle.METRIC_REL_CHANGE, 0.0, 1, xt)
    plan = cr.cubic_rl_plan_linear(n, dev(psf))
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    dd, rr = dev(d), dev(xt)
    n_done, hist = cr.cubic_rl_deconvolve_monitor(plan, dd, 12, 1e-6, cr.METRIC_REL_CHANGE, 0.0, 1, out, rr)
    h = np.array(hist)
    assert n_done == 12
    assert np.allclose(h[:, 0], h_ref[:, 0], rtol=1e-3)
    assert np.allclose(h[:, 1], h_ref[:, 1], rtol=1e-6, atol=0)
    assert np.allclose(h[:, 2], h_ref[:, 2], atol=1e-3)
    torch.cuda.synchronize()
    assert rel_l2(out.cpu().numpy(), ref_out) <= 1e-4
    gain = (h_ref[:-1, 1] - h_ref[1:, 1]) / np.abs(h_ref[1:, 1])
    tol = 0.5 * (gain[4] + gain[5])
    n_nll, _ = cr.cubic_rl_deconvolve_monitor(plan, dd, 12, 1e-6, cr.METRIC_NLL, tol, 1, out)
    _, n_ref, _ = oracle.rl_monitor_same(d, psf, 12, 1e-6, oracle.METRIC_NLL, tol, 1)
    assert n_nll == n_ref
    torch.cuda.synchronize()        # without a reference, out is cropped once at the stop
    assert rel_l2(out.cpu().numpy(), oracle.rl_same(d, psf, n_nll, 1e-6)) <= 1e-4
    dpsnr = h_ref[1:, 2] - h_ref[:-1, 2]
    tol = 0.5 * (dpsnr[3] + dpsnr[4])
    n_psnr, _ = cr.cubic_rl_deconvolve_monitor(plan, dd, 12, 1e-6, cr.METRIC_PSNR, tol, 2, out, rr)
    _, n_ref, _ = oracle.rl_monitor_same(d, psf, 12, 1e-6, oracle.METRIC_PSNR, tol, 2, xt)
    assert n_psnr == n_ref


def test_linear_plan_errors(cr):
    n, k = (8, 10, 12), (3, 3, 3)
    plan = cr.cubic_rl_plan_linear(n, dev(np.ones(k, np.float32)))
    img = dev(np.ones(n, np.float32))
    out = torch.empty_like(img)
    for call in (lambda: cr.cubic_rl_deconvolve_ckpt(plan, img, 3, 1e-6, 1, torch.empty((3,) + n, device="cuda"), out),
                 lambda: cr.cubic_fsc(plan, img, out, 4)):
        with pytest.raises(cr.CubicError) as e:
            call()
        assert e.value.status == 1
    with pytest.raises(cr.CubicError) as e:   # no supported length for the padded axis
        cr.cubic_rl_plan_linear((8, 10, 3000), dev(np.ones(k, np.float32)))
    assert e.value.status == 2
