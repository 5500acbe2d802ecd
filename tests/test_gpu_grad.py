"""GPU gradients of Richardson-Lucy against the FP64 oracle's reverse mode.

The oracle's gradients are pinned by central finite differences in
tests/test_oracle.py.  Tolerance for the FP32 GPU gradients: relative L2 <= 1e-3
against the oracle (the stated gradient tolerance), parameter gradients to 1e-3
relative (absolute floor for dL/dA, which is zero by PSF-scale invariance).
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu_grads(cr, d, psf, n_iter, ckpt, g_out, eps=1e-6):
    shape = d.shape
    plan = cr.cubic_rl_plan(shape, dev(psf))
    nck = cr.n_checkpoints(n_iter, ckpt)
    ck = torch.empty((nck,) + shape, dtype=torch.float32, device="cuda")
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    dd = dev(d)
    cr.cubic_rl_deconvolve_ckpt(plan, dd, n_iter, eps, ckpt, ck, out)
    gd = torch.empty_like(dd)
    gp = torch.empty_like(dd)
    cr.cubic_rl_backward(plan, dd, n_iter, eps, ckpt, ck, dev(g_out), gd, gp)
    torch.cuda.synchronize()
    return out.cpu().numpy(), gd.cpu().numpy(), gp.cpu().numpy()


@pytest.mark.parametrize("shape,ckpt", [((8, 12, 10), 2), ((5, 9, 15), 3), ((16, 20, 24), 1), ((6, 25, 18), 7)])
def test_backward_matches_oracle(cr, shape, ckpt):
    r = np.random.default_rng(sum(shape) + ckpt)
    d = r.uniform(2.0, 30.0, shape).astype(np.float32)
    psf = r.uniform(0.1, 1.0, shape).astype(np.float32) ** 3      # asymmetric PSF
    psf /= psf.sum()
    g_out = r.standard_normal(shape).astype(np.float32)
    n_iter = 6
    out, gd, gp = gpu_grads(cr, d, psf, n_iter, ckpt, g_out)
    assert rel_l2(out, oracle.rl(d, psf, n_iter, 1e-6)) <= 1e-5
    rd, rp = oracle.rl_grad(d, psf, n_iter, 1e-6, g_out)
    assert rel_l2(gd, rd) <= 1e-3
    assert rel_l2(gp, rp) <= 1e-3


def test_checkpoint_spacing_does_not_change_gradients(cr):
    shape = (8, 16, 12)
    r = np.random.default_rng(3)
    d = r.uniform(2.0, 30.0, shape).astype(np.float32)
    psf = oracle.psf_gaussian(shape, 1.3, 2.0).astype(np.float32)
    g_out = r.standard_normal(shape).astype(np.float32)
    res = [gpu_grads(cr, d, psf, 10, c, g_out) for c in (1, 3, 4, 10)]
    for out, gd, gp in res[1:]:
        assert np.array_equal(out, res[0][0])
        assert np.array_equal(gd, res[0][1])
        assert np.array_equal(gp, res[0][2])


def test_psf_gaussian_backward_matches_oracle(cr):
    for shape, th in [((9, 12, 11), (1.7, 2.6, 1.3)), ((32, 64, 64), (1.5, 3.0, 1.0)), ((64, 128, 128), (2.4, 6.0, 1.0))]:
        w = np.random.default_rng(len(shape) + int(th[0] * 10)).standard_normal(shape).astype(np.float32)
        gp = torch.empty(3, dtype=torch.float32, device="cuda")
        cr.cubic_psf_gaussian_backward(shape, *th, dev(w), gp)
        torch.cuda.synchronize()
        ref = oracle.psf_gaussian_grad(shape, *th, w.astype(np.float64))
        got = gp.cpu().numpy()
        assert np.allclose(got, ref, rtol=1e-3, atol=1e-6 * np.abs(ref).max()), (got, ref)


def test_autograd_function_end_to_end(cr):
    from paper_2510_14143_gb300.autograd import RLDeconvolve
    shape = (12, 24, 20)
    d, xt = synth.make_volume(shape, 4, (1.5, 2.5), 10.0, 1.2, 2.0, 777)
    theta = (1.4, 2.3, 1.0)
    n_iter, ckpt = 8, 3
    dt = dev(d).requires_grad_(True)
    sxy = torch.tensor(theta[0], device="cuda", requires_grad=True)
    sz = torch.tensor(theta[1], device="cuda", requires_grad=True)
    amp = torch.tensor(theta[2], device="cuda", requires_grad=True)
    u = RLDeconvolve.apply(dt, sxy, sz, amp, n_iter, 1e-6, ckpt)
    xt_t = dev(xt)
    loss = ((u - xt_t) ** 2).mean()
    loss.backward()
    # oracle chain: dL/du -> rl_grad -> psf_gaussian_grad
    psf = oracle.psf_gaussian(shape, *theta)
    uo = oracle.rl(d, psf, n_iter, 1e-6)
    g_out = 2 * (uo - xt) / uo.size
    rd, rp = oracle.rl_grad(d, psf, n_iter, 1e-6, g_out)
    gth = oracle.psf_gaussian_grad(shape, *theta, rp)
    assert rel_l2(dt.grad.cpu().numpy(), rd) <= 1e-3
    got = np.array([sxy.grad.item(), sz.grad.item(), amp.grad.item()])
    assert np.allclose(got[:2], gth[:2], rtol=1e-3)
    assert abs(got[2]) <= 1e-3 * np.abs(gth[:2]).max()       # RL is invariant to the PSF amplitude


def test_autograd_batch_over_streams(cr):
    # five volumes over four streams (one stream carries two): per-volume image gradients
    # and the PSF-parameter gradient summed over the batch, against the oracle
    from paper_2510_14143_gb300.autograd import RLDeconvolve
    shape, nb = (8, 12, 10), 5
    vols = [synth.make_volume(shape, 2, (1.2, 2.0), 10.0, 1.2, 2.0, 900 + b) for b in range(nb)]
    d = np.stack([v[0] for v in vols])
    xt = np.stack([v[1] for v in vols])
    theta = (1.3, 2.1, 1.0)
    n_iter, ckpt = 6, 2
    dt = dev(d).requires_grad_(True)
    params = [torch.tensor(v, device="cuda", requires_grad=True) for v in theta]
    u = RLDeconvolve.apply(dt, params[0], params[1], params[2], n_iter, 1e-6, ckpt)
    loss = ((u - dev(xt)) ** 2).mean(dim=(1, 2, 3)).sum()
    loss.backward()
    psf = oracle.psf_gaussian(shape, *theta)
    rp_sum = np.zeros(shape)
    for b in range(nb):
        uo = oracle.rl(d[b], psf, n_iter, 1e-6)
        assert rel_l2(u[b].detach().cpu().numpy(), uo) <= 1e-4
        rd, rp = oracle.rl_grad(d[b], psf, n_iter, 1e-6, 2 * (uo - xt[b]) / uo.size)
        assert rel_l2(dt.grad[b].cpu().numpy(), rd) <= 1e-3
        rp_sum += rp
    gth = oracle.psf_gaussian_grad(shape, *theta, rp_sum)
    got = np.array([p.grad.item() for p in params])
    assert np.allclose(got[:2], gth[:2], rtol=1e-3)


def test_differentiable_workload_sample(cr):
    # one volume of the 16 x 128x128x64 workload, 30 iterations, checkpoints every 6
    d, xt = synth.grad_volume(0)
    shape = d.shape
    th = synth.GRAD_EVAL_PSF
    psf = oracle.psf_gaussian(shape, *th)
    n_iter, ckpt = synth.GRAD_ITERS, synth.GRAD_CKPT
    uo = oracle.rl(d, psf, n_iter, 1e-6)
    g_out = (2 * (uo - xt) / uo.size).astype(np.float32)
    out, gd, gp = gpu_grads(cr, d, psf.astype(np.float32), n_iter, ckpt, g_out)
    rd, rp = oracle.rl_grad(d, psf.astype(np.float32), n_iter, 1e-6, g_out)
    assert rel_l2(out, uo) <= 1e-4
    assert rel_l2(gd, rd) <= 1e-3
    assert rel_l2(gp, rp) <= 1e-3
