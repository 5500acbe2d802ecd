"""Fourier Shell Correlation on the GPU against the FP64 oracle (compensated float32
shell sums: FSC values agree to 1e-4 absolute), for two volumes and for the single-image
split."""
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


@pytest.mark.parametrize("shape,n_shells", [((32, 64, 64), 32), ((15, 27, 40), 12), ((8, 8, 8), 4),
                                            ((64, 128, 100), 50)])
def test_fsc_matches_oracle(cr, shape, n_shells):
    d, xt = synth.make_volume(shape, 6, (1.5, 3.0), 10.0, 1.3, 2.0, 77 + sum(shape))
    noise = synth.random_field(shape, 3, -5.0, 5.0)
    a, b = d, (xt + noise).astype(np.float32)
    psf = np.zeros(shape, np.float32)
    psf[tuple(n // 2 for n in shape)] = 1
    plan = cr.cubic_rl_plan(shape, dev(psf))
    got = cr.cubic_fsc(plan, dev(a), dev(b), n_shells).cpu().numpy()
    ref = oracle.fsc(a, b, n_shells)[0]
    assert np.allclose(got, ref, atol=1e-4), (got, ref)
    same = cr.cubic_fsc(plan, dev(a), dev(a), n_shells).cpu().numpy()
    nonempty = oracle.fsc(a, a, n_shells)[2] > 0
    assert np.allclose(same[nonempty], 1.0, atol=1e-5)


def test_fsc_of_deconvolution_against_truth(cr):
    # the paper's use: resolution of an estimate against the object
    # the estimate is the oracle's (both sides take the same volumes)
    w = synth.SMALL
    d, xt = synth.workload_volume(w)
    psf = oracle.psf_gaussian(w.shape, w.psf_sigma_xy, w.psf_sigma_z, 1.0).astype(np.float32)
    plan = cr.cubic_rl_plan(w.shape, dev(psf))
    u = oracle.rl(d, psf, w.n_iter, 1e-6).astype(np.float32)
    got = cr.cubic_fsc(plan, dev(u), dev(xt), 16).cpu().numpy()
    ref = oracle.fsc(u, xt, 16)[0]
    assert np.allclose(got, ref, atol=1e-4)
    with pytest.raises(cr.CubicError):
        cr.cubic_fsc(plan, dev(u), dev(xt), 0)


@pytest.mark.parametrize("half,n_shells", [((8, 12, 10), 6), ((16, 32, 24), 12), ((32, 64, 64), 24)])
def test_fsc_split_matches_oracle(cr, half, n_shells):
    full = tuple(2 * h for h in half)
    d, _ = synth.make_volume(full, 8, (1.5, 3.0), 10.0, 1.3, 2.0, 91 + sum(half))
    psf = np.zeros(half, np.float32)
    psf[tuple(h // 2 for h in half)] = 1
    plan = cr.cubic_rl_plan(half, dev(psf))
    got = cr.cubic_fsc_split(plan, dev(d), n_shells).cpu().numpy()
    ref = oracle.fsc_split(d, n_shells)
    assert np.allclose(got, ref, atol=1e-4), (got, ref)
    with pytest.raises(cr.CubicError) as e:
        cr.cubic_fsc_split(plan, dev(d), 0)
    assert e.value.status == 1
