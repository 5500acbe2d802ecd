"""Automatic stopping (the paper's Section 4 threshold on the improvement between
consecutive iterations) on the GPU against the FP64 oracle.

The per-iteration relative changes delta_k must match the oracle's to 1e-3 relative
(they are differences of FP32 estimates); the threshold is placed midway between two
consecutive checked deltas so both sides stop at the same iteration.
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


@pytest.mark.parametrize("check_every", [1, 3])
def test_auto_stopping_matches_oracle(cr, check_every):
    w = synth.SMALL
    d, _ = synth.workload_volume(w)
    psf = oracle.psf_gaussian(d.shape, w.psf_sigma_xy, w.psf_sigma_z).astype(np.float32)
    _, n_ref_all, hist_ref = oracle.rl_auto(d, psf, 30, 1e-6, 0.0, 1)
    assert n_ref_all == 30
    plan = cr.cubic_rl_plan(d.shape, dev(psf))
    out = torch.empty(d.shape, dtype=torch.float32, device="cuda")
    n, hist = cr.cubic_rl_deconvolve_auto(plan, dev(d), 30, 1e-6, 0.0, check_every, out)
    assert n == 30
    assert np.allclose(hist, hist_ref, rtol=1e-3)
    # a threshold midway between the deltas at two consecutive checks
    checks = list(range(check_every, 31, check_every))
    j = next(i for i in range(1, len(checks)) if hist_ref[checks[i] - 1] < hist_ref[checks[i - 1] - 1])
    tol = 0.5 * (hist_ref[checks[j] - 1] + hist_ref[checks[j - 1] - 1])
    out_ref, n_ref, _ = oracle.rl_auto(d, psf, 30, 1e-6, tol, check_every)
    n, _ = cr.cubic_rl_deconvolve_auto(plan, dev(d), 30, 1e-6, tol, check_every, out)
    torch.cuda.synchronize()
    assert n == n_ref
    assert rel_l2(out.cpu().numpy(), out_ref) <= 1e-4


def test_auto_stopping_delta_psf(cr):
    shape = (8, 16, 12)
    d = synth.random_field(shape, 9, 1.0, 100.0)
    psf = np.zeros(shape, np.float32)
    psf[4, 8, 6] = 1.0
    plan = cr.cubic_rl_plan(shape, dev(psf))
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    n, hist = cr.cubic_rl_deconvolve_auto(plan, dev(d), 20, 1e-6, 1e-5, 1, out)
    torch.cuda.synchronize()
    assert n == 2 and hist[1] < 1e-5
    assert rel_l2(out.cpu().numpy(), d) < 1e-6
