"""Metric-guided stopping on the GPU (relative change, Poisson NLL, scale-invariant PSNR
against a reference) against the FP64 oracle.

The recorded measures must match the oracle's: relative changes to 1e-3 relative, the NLL
to 1e-6 relative (a sum of float32 terms over the volume), the PSNR to 1e-3 dB.  Each
threshold sits midway between two consecutive improvements, so both sides stop at the same
iteration.
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


@pytest.fixture(scope="module")
def case():
    w = synth.SMALL
    d, xt = synth.workload_volume(w)
    psf = oracle.psf_gaussian(d.shape, w.psf_sigma_xy, w.psf_sigma_z).astype(np.float32)
    _, _, h_ref = oracle.rl_monitor(d, psf, 40, 1e-6, oracle.METRIC_REL_CHANGE, 0.0, 1, xt)
    return d, xt, psf, h_ref


def run(cr, d, psf, xt, metric, tol, check_every, max_iter=40, with_ref=True):
    plan = cr.cubic_rl_plan(d.shape, dev(psf))
    out = torch.empty(d.shape, dtype=torch.float32, device="cuda")
    n, hist = cr.cubic_rl_deconvolve_monitor(plan, dev(d), max_iter, 1e-6, metric, tol, check_every, out,
                                             dev(xt) if with_ref else None)
    return n, np.array(hist), out.cpu().numpy()


def test_monitor_history_matches_oracle(cr, case):
    d, xt, psf, h_ref = case
    n, h, out = run(cr, d, psf, xt, cr.METRIC_REL_CHANGE, 0.0, 1)
    assert n == 40
    assert np.allclose(h[:, 0], h_ref[:, 0], rtol=1e-3)
    assert np.allclose(h[:, 1], h_ref[:, 1], rtol=1e-6, atol=0)
    assert np.allclose(h[:, 2], h_ref[:, 2], atol=1e-3)
    ref_out = oracle.rl(d, psf, 40, 1e-6)
    assert rel_l2(out, ref_out) <= 1e-4
    # without a reference the PSNR column is NaN
    _, h2, _ = run(cr, d, psf, xt, cr.METRIC_NLL, -1.0, 1, max_iter=3, with_ref=False)
    assert np.all(np.isnan(h2[:, 2])) and np.allclose(h2[:, 1], h_ref[:3, 1], rtol=1e-6)


@pytest.mark.parametrize("check_every", [1, 3])
def test_monitor_psnr_stops_where_oracle_does(cr, case, check_every):
    d, xt, psf, h_ref = case
    gain = np.diff(h_ref[:, 2])
    j = int(np.argmax(gain < 0.2))          # first gain under 0.2 dB
    tol = 0.5 * (gain[j] + gain[j - 1]) if gain[j - 1] - gain[j] > 1e-2 else 0.2
    out_ref, n_ref, _ = oracle.rl_monitor(d, psf, 40, 1e-6, oracle.METRIC_PSNR, tol, check_every, xt)
    n, _, out = run(cr, d, psf, xt, cr.METRIC_PSNR, tol, check_every)
    assert n == n_ref
    assert rel_l2(out, out_ref) <= 1e-4


@pytest.mark.parametrize("check_every", [1, 4])
def test_monitor_nll_stops_where_oracle_does(cr, case, check_every):
    d, xt, psf, h_ref = case
    rel = (h_ref[:-1, 1] - h_ref[1:, 1]) / np.abs(h_ref[1:, 1])
    tol = 0.5 * (rel[5] + rel[6])   # consecutive decreases far apart next to the NLL's float error
    out_ref, n_ref, _ = oracle.rl_monitor(d, psf, 40, 1e-6, oracle.METRIC_NLL, tol, check_every, xt)
    n, _, out = run(cr, d, psf, xt, cr.METRIC_NLL, tol, check_every)
    assert n == n_ref and n < 40
    assert rel_l2(out, out_ref) <= 1e-4


def test_monitor_errors(cr, case):
    d, xt, psf, _ = case
    plan = cr.cubic_rl_plan(d.shape, dev(psf))
    out = torch.empty(d.shape, dtype=torch.float32, device="cuda")
    with pytest.raises(cr.CubicError) as e:   # the PSNR measure needs a reference
        cr.cubic_rl_deconvolve_monitor(plan, dev(d), 5, 1e-6, cr.METRIC_PSNR, 0.0, 1, out, None)
    assert e.value.status == 1
    with pytest.raises(cr.CubicError) as e:
        cr.cubic_rl_deconvolve_monitor(plan, dev(d), 5, 1e-6, 7, 0.0, 1, out, None)
    assert e.value.status == 1
    ref = dev(xt)
    with pytest.raises(cr.CubicError) as e:   # out aliases the reference
        cr.cubic_rl_deconvolve_monitor(plan, dev(d), 5, 1e-6, cr.METRIC_PSNR, 0.0, 1, ref, ref)
    assert e.value.status == 1
