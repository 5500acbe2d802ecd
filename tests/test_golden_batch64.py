"""The stored oracle samples of the 64-volume batched workload (tests/golden): complete, and
the oracle's own values.

The file must list every volume with its shape and 48 samples plus the peak; its values for
the first volume are recomputed here with the oracle (a few seconds) and must agree to
double-precision rounding, provided this CPU draws the same image (same exact image sum).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2510_14143_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batch64_oracle_samples.txt")


def load():
    vols, samples = {}, {}
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        j = int(f[1])
        if f[0] == "V":
            vols[j] = ((int(f[2]), int(f[3]), int(f[4])), int(f[5]), int(f[6]), float(f[7]), float(f[8]))
        else:
            samples.setdefault(j, []).append((int(f[2]), float(f[3])))
    return vols, samples


def test_golden_file_is_complete():
    vols, samples = load()
    shapes = synth.batch_shapes()
    assert sorted(vols) == list(range(len(shapes)))
    for j, shape in enumerate(shapes):
        assert vols[j][0] == tuple(shape)
        idx = [i for i, _ in samples[j]]
        assert len(idx) == 48 and len(set(idx)) == 48
        assert all(0 <= i < int(np.prod(shape)) for i in idx)
        peak = vols[j][3]
        assert all(0.0 <= v <= peak for _, v in samples[j])


def test_golden_values_are_the_oracles():
    vols, samples = load()
    j = 0
    shape = synth.batch_shapes()[j]
    d, _ = synth.batch_volume(j, shape)
    if int(np.rint(d.astype(np.float64).sum())) != vols[j][1]:
        pytest.skip("this CPU draws another image for volume 0")
    psf = oracle.psf_gaussian(shape, synth.SMALL.psf_sigma_xy, synth.SMALL.psf_sigma_z, 1.0).astype(np.float32)
    ref = oracle.rl(d, psf, synth.BATCH_ITERS, 1e-6).reshape(-1)
    _, _, peak_index, peak, l2 = vols[j]
    assert int(np.argmax(ref)) == peak_index
    assert ref[peak_index] == pytest.approx(peak, rel=1e-9)
    assert float(np.linalg.norm(ref)) == pytest.approx(l2, rel=1e-9)
    for i, v in samples[j]:
        assert ref[i] == pytest.approx(v, rel=1e-9, abs=1e-12 * peak)
