"""All 64 volumes of the batched workload, one batched call of its 50 iterations, against
the FP64 oracle at sampled voxels.

The oracle's estimates of all 64 volumes take minutes of CPU, so they are stored:
tests/golden/batch64_oracle_samples.txt, written by tests/golden/make_batch64_samples.py
(oracle only), holds per volume 48 seeded voxels, the voxel where the estimate peaks, the
peak value and the estimate's L2 norm.  Each volume must match them within the method's
tolerance (1e-4 of the peak per voxel; the norm within 1e-5, which the relative L2 error
bounds from above).  The images come from numpy's seeded generators, whose floating-point
steps may round differently on another CPU (the blobs' exponentials) and so draw other
Poisson counts: a volume whose image sum differs from the stored one is compared with the
oracle computed on the spot instead, over every voxel.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2510_14143_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batch64_oracle_samples.txt")


@pytest.fixture(scope="module")
def cr():
    from paper_2510_14143_gb300 import build
    build.build()
    import paper_2510_14143_gb300 as m
    return m


def load_golden():
    vols, samples = {}, {}
    for line in open(GOLDEN):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        j = int(f[1])
        if f[0] == "V":
            vols[j] = {"shape": (int(f[2]), int(f[3]), int(f[4])), "sum": int(f[5]), "peak_index": int(f[6]),
                       "peak": float(f[7]), "l2": float(f[8])}
        elif f[0] == "S":
            samples.setdefault(j, []).append((int(f[2]), float(f[3])))
    return vols, samples


def test_all_batched_volumes_at_sampled_voxels(cr):
    vols, samples = load_golden()
    shapes = synth.batch_shapes()
    assert sorted(vols) == list(range(len(shapes)))
    plans, imgs, hosts = [], [], []
    for j, shape in enumerate(shapes):
        assert vols[j]["shape"] == tuple(shape)
        d, _ = synth.batch_volume(j, shape)
        psf = oracle.psf_gaussian(shape, synth.SMALL.psf_sigma_xy, synth.SMALL.psf_sigma_z, 1.0).astype(np.float32)
        plans.append(cr.cubic_rl_plan(shape, torch.from_numpy(psf).cuda()))
        imgs.append(torch.from_numpy(d).cuda())
        hosts.append((d, psf))
    outs = [torch.empty_like(i) for i in imgs]
    cr.cubic_rl_deconvolve_batched(plans, imgs, synth.BATCH_ITERS, 1e-6, outs)
    torch.cuda.synchronize()
    worst, live = 0.0, []
    for j, out in enumerate(outs):
        got = out.cpu().numpy().astype(np.float64).reshape(-1)
        v = vols[j]
        d, psf = hosts[j]
        if int(np.rint(d.astype(np.float64).sum())) == v["sum"]:
            pts = samples[j] + [(v["peak_index"], v["peak"])]
            err = max(abs(got[i] - ref) for i, ref in pts) / v["peak"]
            assert abs(np.linalg.norm(got) - v["l2"]) <= 1e-5 * v["l2"], j
        else:
            # other Poisson counts on this CPU: the oracle on the spot, every voxel
            live.append(j)
            ref = oracle.rl(d, psf, synth.BATCH_ITERS, 1e-6).reshape(-1)
            err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
            assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref), j
        worst = max(worst, err)
        assert err <= 1e-4, (j, err)
    assert len(live) <= len(shapes) // 4, f"stored oracle values unusable for volumes {live}"
    print(f"64 batched volumes, {synth.BATCH_ITERS} iterations: worst error {worst:.3e} of the peak "
          f"(volumes checked against the oracle on the spot: {live})")
