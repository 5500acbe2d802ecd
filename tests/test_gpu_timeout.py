"""Bounded device waits run out cleanly and are reported: failure detection without a GPU fault.

Every wait of a kernel on an asynchronous tile copy gives up after a limit of the GPU's
global timer, sets the plan's device error word and returns.  To make such a wait run out
without a fault, a hang or a copy left in flight, the one-shot test setting
cubic_test_skip_next_tile_copy(wait_ns) makes the first CTA of the next TMA-pipelined Y
launch not issue the copy of its first tile and wait at most wait_ns for it (an mbarrier
that nothing completes).  The tests check that the status call reports
CUBIC_ERR_TIMEOUT, that the word is clear after it, and that the next call on the same
plan matches the FP64 oracle, i.e. the context and the plan stay usable.
"""
import numpy as np
import pytest

import oracle
from paper_2510_14143_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# ny = 64: the Y pass's first launch shape is the TMA-pipelined one
SHAPE = (32, 64, 48)
N_ITER = 5


@pytest.fixture(scope="module")
def cr():
    from paper_2510_14143_gb300 import build
    build.build()
    import paper_2510_14143_gb300 as m
    return m


@pytest.fixture
def disarm(cr):
    yield
    cr.cubic_test_skip_next_tile_copy(0)  # in case no launch took the setting


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def volume():
    d, _ = synth.make_volume(SHAPE, 4, (1.5, 3.0), 10.0, 1.5, 3.0, 4242)
    psf = oracle.psf_gaussian(SHAPE, 1.5, 3.0).astype(np.float32)
    return d, psf


def test_timed_out_wait_is_reported_and_the_plan_recovers(cr, disarm):
    d, psf = volume()
    plan = cr.cubic_rl_plan(SHAPE, dev(psf))
    cr.cubic_rl_plan_set_variants(plan, 0, 0, 0)
    dd = dev(d)
    out = torch.empty_like(dd)
    cr.cubic_rl_deconvolve(plan, dd, N_ITER, 1e-6, out)
    cr.cubic_rl_stream_status(plan)  # clean before

    cr.cubic_test_skip_next_tile_copy(1_000_000)  # 1 ms
    cr.cubic_rl_deconvolve(plan, dd, N_ITER, 1e-6, out)
    with pytest.raises(cr.CubicError) as e:
        cr.cubic_rl_stream_status(plan)
    assert e.value.status == 6  # CUBIC_ERR_TIMEOUT
    cr.cubic_rl_stream_status(plan)  # the word was cleared

    cr.cubic_rl_deconvolve(plan, dd, N_ITER, 1e-6, out)
    cr.cubic_rl_stream_status(plan)
    assert rel_l2(out.cpu().numpy(), oracle.rl(d, psf, N_ITER, 1e-6)) <= 1e-5


def test_plan_wait_limit_leaves_normal_runs_alone(cr):
    d, psf = volume()
    plan = cr.cubic_rl_plan(SHAPE, dev(psf))
    cr.cubic_rl_plan_set_wait_limit(plan, 100_000_000)  # 100 ms
    dd = dev(d)
    out = torch.empty_like(dd)
    cr.cubic_rl_deconvolve(plan, dd, N_ITER, 1e-6, out)
    cr.cubic_rl_stream_status(plan)
    assert rel_l2(out.cpu().numpy(), oracle.rl(d, psf, N_ITER, 1e-6)) <= 1e-5
    cr.cubic_rl_plan_set_wait_limit(plan, 0)

