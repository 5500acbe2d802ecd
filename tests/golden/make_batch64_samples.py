"""Writes batch64_oracle_samples.txt: the FP64 oracle's Richardson-Lucy estimate of every
volume of the 64-volume batched workload, at its 50 iterations, at sampled voxels.

Only the oracle computes here (oracle.psf_gaussian, oracle.rl); the inputs come from the
seeded generators of paper_2510_14143_gb300.synth.  The GPU test test_gpu_batched_all.py
compares one batched call over all 64 volumes with these values: 48 seeded voxels per
volume plus the voxel where the estimate peaks, the peak value and the estimate's L2 norm.
The image's sum (exact: Poisson counts) guards against a change of the input generator.

    python tests/golden/make_batch64_samples.py [out_path]

takes about 25 minutes on 8 cores (the oracle's transforms of the non-power-of-two
lengths go through Bluestein's algorithm).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2510_14143_gb300 import synth  # noqa: E402

N_SAMPLES = 48
EPS = 1e-6


def sample_indices(j: int, voxels: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(7000 + j))
    return np.sort(rng.choice(voxels, size=N_SAMPLES, replace=False))


def main(out_path: str) -> None:
    shapes = synth.batch_shapes()
    lines = [
        "# FP64 oracle RL estimates of the 64-volume batched workload at sampled voxels.",
        f"# {synth.BATCH_ITERS} iterations, eps {EPS}; image j = synth.batch_volume(j, synth.batch_shapes()[j]);",
        "# PSF = oracle.psf_gaussian(shape, SMALL.psf_sigma_xy, SMALL.psf_sigma_z, 1) rounded to float32.",
        "# Written by tests/golden/make_batch64_samples.py (oracle only).",
        "# V j nz ny nx image_sum peak_index peak_value l2_norm",
        "# S j flat_index value   (flat index into the C-order [nz][ny][nx] volume)",
    ]
    t0 = time.perf_counter()
    for j, shape in enumerate(shapes):
        d, _ = synth.batch_volume(j, shape)
        psf = oracle.psf_gaussian(shape, synth.SMALL.psf_sigma_xy, synth.SMALL.psf_sigma_z, 1.0).astype(np.float32)
        ref = oracle.rl(d, psf, synth.BATCH_ITERS, EPS)
        flat = ref.reshape(-1)
        peak = int(np.argmax(flat))
        lines.append(f"V {j} {shape[0]} {shape[1]} {shape[2]} {int(np.rint(d.astype(np.float64).sum()))} "
                     f"{peak} {float(flat[peak])!r} {float(np.linalg.norm(flat))!r}")
        for i in sample_indices(j, flat.size):
            lines.append(f"S {j} {int(i)} {float(flat[i])!r}")
        print(f"volume {j} {shape}: {time.perf_counter() - t0:.1f} s", flush=True)
    with open(out_path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(__file__),
                                                            "batch64_oracle_samples.txt"))
