"""Every X launch shape of the long lines (including the ratio and update passes that read
their operand rows through an L2 prefetch instead of shared memory) in every Richardson-Lucy
mode that uses them, against the FP64 oracle:

- plain iterations (ratio, in-place update, final update);
- the monitored run (Poisson NLL inside the ratio pass, relative-change sums inside the
  update pass);
- the reverse mode, whose recomputation keeps b, r and q from the same passes.

Tolerances are those of the single-shape tests: relative L2 1e-4 for estimates, 1e-3 for
gradients and relative changes, 1e-6 for the NLL.
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


# x lengths 256 .. 2560 (odd row counts leave the last line pair half empty)
SHAPES = [(6, 9, 256), (4, 10, 512), (3, 9, 1024), (2, 3, 2560)]


def x_variants(cr, plan):
    (nx, _, _), chosen = cr.cubic_rl_plan_variants(plan)
    return nx, chosen


@pytest.mark.parametrize("shape", SHAPES)
def test_every_x_shape_rl(cr, shape):
    d, _ = synth.make_volume(shape, 4, (1.5, 3.0), 10.0, 1.5, 2.5, 91 + sum(shape))
    psf = oracle.psf_gaussian(shape, 1.5, 2.5).astype(np.float32)
    ref = oracle.rl(d, psf, 5, 1e-6)
    plan = cr.cubic_rl_plan(shape, dev(psf))
    nx, chosen = x_variants(cr, plan)
    assert nx >= 4                       # the default split and its three prefetching forms
    dd = dev(d)
    out = torch.empty_like(dd)
    for vx in range(nx):
        cr.cubic_rl_plan_set_variants(plan, vx, chosen[1], chosen[2])
        out.fill_(float("nan"))
        cr.cubic_rl_deconvolve(plan, dd, 5, 1e-6, out)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) <= 1e-4, vx


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_every_x_shape_monitor(cr, shape):
    d, xt = synth.make_volume(shape, 4, (1.5, 3.0), 10.0, 1.5, 2.5, 17 + sum(shape))
    psf = oracle.psf_gaussian(shape, 1.5, 2.5).astype(np.float32)
    _, _, h_ref = oracle.rl_monitor(d, psf, 6, 1e-6, oracle.METRIC_REL_CHANGE, 0.0, 1, xt)
    plan = cr.cubic_rl_plan(shape, dev(psf))
    nx, chosen = x_variants(cr, plan)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    for vx in range(nx):
        cr.cubic_rl_plan_set_variants(plan, vx, chosen[1], chosen[2])
        n, hist = cr.cubic_rl_deconvolve_monitor(plan, dev(d), 6, 1e-6, cr.METRIC_REL_CHANGE, 0.0, 1, out,
                                                 dev(xt))
        h = np.array(hist)
        assert n == 6
        assert np.allclose(h[:, 0], h_ref[:, 0], rtol=1e-3), vx
        assert np.allclose(h[:, 1], h_ref[:, 1], rtol=1e-6, atol=0), vx


@pytest.mark.parametrize("shape", SHAPES[:3])
def test_every_x_shape_backward(cr, shape):
    r = np.random.default_rng(7 + sum(shape))
    d = r.uniform(2.0, 30.0, shape).astype(np.float32)
    psf = r.uniform(0.1, 1.0, shape).astype(np.float32) ** 3      # asymmetric PSF
    psf /= psf.sum()
    g_out = r.standard_normal(shape).astype(np.float32)
    n_iter, ckpt = 4, 2
    rd, rp = oracle.rl_grad(d, psf, n_iter, 1e-6, g_out)
    plan = cr.cubic_rl_plan(shape, dev(psf))
    nx, chosen = x_variants(cr, plan)
    dd = dev(d)
    ck = torch.empty((cr.n_checkpoints(n_iter, ckpt),) + shape, dtype=torch.float32, device="cuda")
    out = torch.empty_like(dd)
    gd = torch.empty_like(dd)
    gp = torch.empty_like(dd)
    for vx in range(nx):
        cr.cubic_rl_plan_set_variants(plan, vx, chosen[1], chosen[2])
        cr.cubic_rl_deconvolve_ckpt(plan, dd, n_iter, 1e-6, ckpt, ck, out)
        cr.cubic_rl_backward(plan, dd, n_iter, 1e-6, ckpt, ck, dev(g_out), gd, gp)
        torch.cuda.synchronize()
        assert rel_l2(gd.cpu().numpy(), rd) <= 1e-3, vx
        assert rel_l2(gp.cpu().numpy(), rp) <= 1e-3, vx
