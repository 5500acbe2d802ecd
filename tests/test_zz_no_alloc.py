"""The allocation-free deconvolution entry point gives the planned path's result.

Some callers cannot allocate device memory (they run under another framework's
stream capture, or their memory is fully reserved by a pool allocator, or they
cannot afford cudaMalloc's implicit synchronisation).  For them
cubic_rl_deconvolve_noalloc keeps every internal buffer in one fixed
per-device array.  This test calls it through the C ABI twice in a row -- the
second call reuses the array the first one left behind -- and compares both
results with cubic_rl_plan + cubic_rl_deconvolve.  It sits in its own file,
named to be collected last, so a run that stops at the first failure has run
every other test before it.
"""
import numpy as np
import pytest

from paper_2510_14143_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def test_noalloc_matches_planned_path_twice(cr):
    w = synth.SMALL
    d, _ = synth.workload_volume(w)
    image = torch.from_numpy(d).cuda()
    psf = torch.empty(w.shape, dtype=torch.float32, device="cuda")
    cr.cubic_psf_gaussian(w.shape, w.psf_sigma_xy, w.psf_sigma_z, 1.0, psf)
    plan = cr.cubic_rl_plan(w.shape, psf)
    ref = torch.empty_like(image)
    cr.cubic_rl_deconvolve(plan, image, w.n_iter, 1e-6, ref)
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    outs = [torch.full(w.shape, float("nan"), device="cuda") for _ in range(2)]
    free = []
    for out in outs:
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        cr.cubic_rl_deconvolve_noalloc(w.shape, psf, image, w.n_iter, 1e-6, out)
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref) <= 1e-5
    # the second call (set-up done) leaves free device memory unchanged
    assert torch.cuda.mem_get_info()[0] == free[1]


def test_noalloc_rejects_volumes_beyond_its_scratch(cr):
    shape = (128, 256, 256)
    x = torch.ones(shape, dtype=torch.float32, device="cuda")
    out = torch.empty_like(x)
    with pytest.raises(cr.CubicError) as e:
        cr.cubic_rl_deconvolve_noalloc(shape, x, x, 1, 1e-6, out)
    assert e.value.status == 2
    assert "scratch" in str(e.value)
