"""Accelerated Richardson-Lucy (Biggs-Andrews extrapolation) on the GPU against the FP64 oracle.

The estimate must match the oracle's to the plain path's tolerance (relative L2 <= 1e-4
after 20 iterations of the small workload), and the extrapolation weights alpha_k to 1e-3:
they are ratios of float32 dot products of differences of float32 estimates.
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


def run(cr, d, psf, n_iter, vx=None):
    plan = cr.cubic_rl_plan(d.shape, dev(psf))
    if vx is not None:
        counts, chosen = cr.cubic_rl_plan_variants(plan)
        cr.cubic_rl_plan_set_variants(plan, vx, chosen[1], chosen[2])
    out = torch.empty(d.shape, dtype=torch.float32, device="cuda")
    alpha = torch.full((max(1, n_iter),), float("nan"), dtype=torch.float32, device="cuda")
    cr.cubic_rl_deconvolve_accel(plan, dev(d), n_iter, 1e-6, out, alpha[:n_iter] if n_iter else None)
    torch.cuda.synchronize()
    return out.cpu().numpy(), alpha[:n_iter].cpu().numpy(), plan


def test_accel_matches_oracle_small_workload(cr):
    w = synth.SMALL
    d, _ = synth.workload_volume(w)
    psf = oracle.psf_gaussian(d.shape, w.psf_sigma_xy, w.psf_sigma_z).astype(np.float32)
    ref, a_ref = oracle.rl_accel(d, psf, w.n_iter, 1e-6)
    got, a_got, _ = run(cr, d, psf, w.n_iter)
    assert rel_l2(got, ref) <= 1e-4
    assert np.allclose(a_got, a_ref, atol=1e-3), (a_got, a_ref)
    assert a_ref[2:].max() > 0.3   # the extrapolation is active


@pytest.mark.parametrize("shape", [(48, 50, 54), (5, 9, 15), (1, 16, 24), (27, 1, 40), (16, 20, 1), (3, 2, 1)])
def test_accel_ragged_shapes_and_general_psf(cr, shape):
    # a PSF without point symmetry (complex spectrum) and lengths that leave ragged tiles
    r = np.random.default_rng(sum(shape))
    d = r.uniform(1.0, 50.0, shape).astype(np.float32)
    psf = r.uniform(0.0, 1.0, shape).astype(np.float32)
    psf[tuple(n // 2 for n in shape)] += 4.0
    psf /= psf.sum()
    n = 9
    ref, a_ref = oracle.rl_accel(d, psf, n, 1e-6)
    got, a_got, _ = run(cr, d, psf, n)
    assert rel_l2(got, ref) <= 1e-4
    assert np.allclose(a_got, a_ref, atol=1e-3)


def test_accel_every_x_variant(cr):
    # each X launch shape has its own CTA count, so its own number of partial sums
    shape = (16, 24, 256)
    d, _ = synth.make_volume(shape, 6, (1.5, 3.0), 10.0, 1.5, 3.0, 4242)
    psf = oracle.psf_gaussian(shape, 1.5, 3.0).astype(np.float32)
    ref, a_ref = oracle.rl_accel(d, psf, 12, 1e-6)
    plan = cr.cubic_rl_plan(shape, dev(psf))
    counts, _ = cr.cubic_rl_plan_variants(plan)
    for vx in range(counts[0]):
        got, a_got, _ = run(cr, d, psf, 12, vx)
        assert rel_l2(got, ref) <= 1e-4, vx
        assert np.allclose(a_got, a_ref, atol=1e-3), vx


def test_accel_first_two_iterations_are_plain_rl(cr):
    w = synth.SMALL
    d, _ = synth.workload_volume(w)
    psf = oracle.psf_gaussian(d.shape, w.psf_sigma_xy, w.psf_sigma_z).astype(np.float32)
    plan = cr.cubic_rl_plan(d.shape, dev(psf))
    for n in (0, 1, 2):
        got, a_got, _ = run(cr, d, psf, n)
        plain = torch.empty(d.shape, dtype=torch.float32, device="cuda")
        cr.cubic_rl_deconvolve(plan, dev(d), n, 1e-6, plain)
        torch.cuda.synchronize()
        assert rel_l2(got, plain.cpu().numpy()) <= 1e-6
        assert np.all(a_got == 0.0)


def test_accel_delta_psf_fixed_point_and_determinism(cr):
    shape = (8, 12, 10)
    d = np.random.default_rng(5).uniform(1, 100, shape).astype(np.float32)
    psf = np.zeros(shape, np.float32)
    psf[tuple(n // 2 for n in shape)] = 1.0
    got, _, _ = run(cr, d, psf, 6)
    assert rel_l2(got, d) <= 1e-6
    # the dot products merge per-CTA partials in a fixed order: runs repeat bitwise
    w = synth.SMALL
    d, _ = synth.workload_volume(w)
    psf = oracle.psf_gaussian(d.shape, w.psf_sigma_xy, w.psf_sigma_z).astype(np.float32)
    a1, al1, _ = run(cr, d, psf, 15)
    a2, al2, _ = run(cr, d, psf, 15)
    assert np.array_equal(a1, a2) and np.array_equal(al1, al2)


def test_accel_full_size_properties(cr):
    # the 1024x1024x128 volume: flux conservation (every RL step keeps sum(x) = sum(d) for
    # a normalised PSF), nonnegativity and alpha in [0, 1]; values checked at any size
    w = synth.LARGE
    g = torch.Generator(device="cuda").manual_seed(3)
    d = torch.rand(w.shape, device="cuda", generator=g) * 100 + 1
    psf = torch.empty(w.shape, dtype=torch.float32, device="cuda")
    cr.cubic_psf_gaussian(w.shape, w.psf_sigma_xy, w.psf_sigma_z, 1.0, psf)
    plan = cr.cubic_rl_plan(w.shape, psf)
    out = torch.empty_like(d)
    alpha = torch.empty(8, dtype=torch.float32, device="cuda")
    cr.cubic_rl_deconvolve_accel(plan, d, 8, 1e-6, out, alpha)
    torch.cuda.synchronize()
    flux_d = d.double().sum().item()
    assert abs(out.double().sum().item() - flux_d) <= 1e-5 * flux_d
    assert out.min().item() >= 0.0
    a = alpha.cpu().numpy()
    assert a[0] == 0.0 and a[1] == 0.0 and np.all((a >= 0) & (a <= 1))


def test_accel_errors(cr):
    shape = (4, 6, 8)
    d = dev(np.ones(shape))
    psf = dev(np.ones(shape) / 192)
    plan = cr.cubic_rl_plan(shape, psf)
    out = torch.empty_like(d)
    with pytest.raises(cr.CubicError) as e:
        cr.cubic_rl_deconvolve_accel(plan, d, -1, 1e-6, out)
    assert e.value.status == 1
    with pytest.raises(cr.CubicError) as e:
        cr.cubic_rl_deconvolve_accel(plan, d, 3, 0.0, out)
    assert e.value.status == 1
    with pytest.raises(cr.CubicError) as e:
        cr.cubic_rl_deconvolve_accel(plan, d, 3, 1e-6, d)
    assert e.value.status == 1
