"""The allocation-free deconvolution entry point gives the planned path's result.

Some callers cannot call cudaMalloc: a framework whose device memory is fully reserved
by its own pool allocator, plug-in code whose host application does not let it allocate,
or a latency-critical loop that cannot take cudaMalloc's implicit device-wide
synchronisation.  For them cubic_rl_deconvolve_noalloc keeps every internal buffer in
one fixed per-device array.  These tests call it through the C ABI twice in a row -- the
second call reuses the array the first one left behind -- and compare both results with
cubic_rl_plan + cubic_rl_deconvolve, for a Gaussian PSF, a PSF with no symmetry, and a
volume close to the array's size limit.  They also check that a bounded device wait that
runs out inside an allocation-free call is reported by cubic_rl_noalloc_status.  The file
is named to be collected last, so a run that stops at the first failure has run every
other test before it.
"""
import numpy as np
import pytest

from paper_2510_14143_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # float32 rounding: the planned path may multiply by a real PSF spectrum


@pytest.fixture(scope="module")
def cr():
    from paper_2510_14143_gb300 import build
    build.build()
    import paper_2510_14143_gb300 as m
    return m


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def asymmetric_psf(shape, seed):
    """A normalised PSF with no point symmetry: a Gaussian core plus a skewed random tail."""
    rng = np.random.Generator(np.random.PCG64(seed))
    grids = np.meshgrid(*[np.arange(n) - n // 2 for n in shape], indexing="ij")
    r2 = sum((g / s) ** 2 for g, s in zip(grids, (3.0, 1.8, 1.4)))
    p = np.exp(-0.5 * r2) * (1.0 + 0.3 * (grids[2] > 0)) + 1e-3 * rng.random(shape)
    return (p / p.sum()).astype(np.float32)


def compare_twice(cr, shape, psf, image, n_iter):
    plan = cr.cubic_rl_plan(shape, psf)
    ref = torch.empty_like(image)
    cr.cubic_rl_deconvolve(plan, image, n_iter, 1e-6, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    outs = [torch.full(shape, float("nan"), device="cuda") for _ in range(2)]
    free = []
    for out in outs:
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        cr.cubic_rl_deconvolve_noalloc(shape, psf, image, n_iter, 1e-6, out)
        cr.cubic_rl_noalloc_status()
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) <= TOL
    # the second call (set-up done) leaves free device memory unchanged
    assert torch.cuda.mem_get_info()[0] == free[1]


def test_noalloc_matches_planned_path_twice(cr):
    w = synth.SMALL
    d, _ = synth.workload_volume(w)
    image = torch.from_numpy(d).cuda()
    psf = torch.empty(w.shape, dtype=torch.float32, device="cuda")
    cr.cubic_psf_gaussian(w.shape, w.psf_sigma_xy, w.psf_sigma_z, 1.0, psf)
    compare_twice(cr, w.shape, psf, image, w.n_iter)


def test_noalloc_asymmetric_psf_near_the_size_limit(cr):
    # nz * ny * xp = 80 * 80 * 80 complex elements: 98% of the 8 MiB array
    shape = (80, 80, 128)
    d, _ = synth.make_volume(shape, 40, (2.0, 4.0), 10.0, 1.5, 3.0, 777)
    image = torch.from_numpy(d).cuda()
    psf = torch.from_numpy(asymmetric_psf(shape, 778)).cuda()
    compare_twice(cr, shape, psf, image, 12)


def test_noalloc_rejects_volumes_beyond_its_scratch(cr):
    for shape in ((128, 256, 256), (90, 80, 128)):
        x = torch.ones(shape, dtype=torch.float32, device="cuda")
        out = torch.empty_like(x)
        with pytest.raises(cr.CubicError) as e:
            cr.cubic_rl_deconvolve_noalloc(shape, x, x, 1, 1e-6, out)
        assert e.value.status == 2
        assert "scratch" in str(e.value)


def test_noalloc_reports_a_timed_out_wait(cr):
    # ny = 64: the Y pass's first launch shape is TMA-pipelined, which the test setting
    # of cubic_test_skip_next_tile_copy needs (no test autotunes this shape)
    shape = (32, 64, 48)
    d, _ = synth.make_volume(shape, 4, (1.5, 3.0), 10.0, 1.5, 3.0, 4343)
    image = torch.from_numpy(d).cuda()
    psf = torch.empty(shape, dtype=torch.float32, device="cuda")
    cr.cubic_psf_gaussian(shape, 1.5, 3.0, 1.0, psf)
    out = torch.empty_like(image)
    cr.cubic_rl_noalloc_status()  # clean before
    try:
        cr.cubic_test_skip_next_tile_copy(1_000_000)  # 1 ms
        cr.cubic_rl_deconvolve_noalloc(shape, psf, image, 5, 1e-6, out)
        with pytest.raises(cr.CubicError) as e:
            cr.cubic_rl_noalloc_status()
        assert e.value.status == 6  # CUBIC_ERR_TIMEOUT
    finally:
        cr.cubic_test_skip_next_tile_copy(0)
    cr.cubic_rl_noalloc_status()  # cleared
    plan = cr.cubic_rl_plan(shape, psf)
    ref = torch.empty_like(image)
    cr.cubic_rl_deconvolve(plan, image, 5, 1e-6, ref)
    cr.cubic_rl_deconvolve_noalloc(shape, psf, image, 5, 1e-6, out)
    cr.cubic_rl_noalloc_status()
    assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) <= TOL
