"""Writes tests/golden/full_masks.npz from the FP64 oracle alone (no CUDA):
for the 512 x 512 benchmark view (DeepSDF decoder seed 0, latent 0 of seed
0, first of five seeded viewpoints) and the five 256 x 256 views of seed 0,
every pixel's oracle hit mask and two exclusion sets, bit-packed, and the
oracle's depth at its hits (float32, ``depth_hits``):

* ``sil``: silhouette rays at the 1e-3 |SDF| margin (tests/helpers.
  silhouette_rays: the outcome changes when f is shifted by -/+1e-3, a ray
  near its step budget in any of the three traces, a convergence test within
  5e-6 of eps, a ray grazing the bounding sphere) -- the rays a 16-bit march
  may decide differently;
* ``amb32``: rays whose FP32 trace may take another branch than FP64
  (tests/helpers.ambiguous_rays with tol_f = 1e-5, exit margin 1e-5, grazing
  hits |n . v| < 0.05, step budget).

Run from the repository root: ``python tests/golden/make_full_masks.py``
(a few minutes on 8 cores)."""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import tracer  # noqa: E402
from tests.helpers import (ambiguous_rays, oracle_sdf, shifted_traces,  # noqa: E402
                           silhouette_rays, workload)


def views():
    spec = synth.DEEPSDF_SPEC
    Ws, bs, Z = workload(spec, seed=0, n_shapes=2)
    yield "b512", oracle_sdf(spec, Ws, bs, Z), [
        synth.look_at_camera(synth.random_viewpoints(5, seed=0)[0], 512, 512, shape=0)]
    Ws, bs, Z = workload(spec, seed=0, n_shapes=1)
    yield "v5", oracle_sdf(spec, Ws, bs, Z), [
        synth.look_at_camera(vp, 256, 256) for vp in synth.random_viewpoints(5, seed=0)]


def main():
    out = {}
    for tag, sdf, cams in views():
        orc = tracer.render(sdf, cams, record=True)
        shifted = shifted_traces(lambda f: tracer.render(f, cams, with_normals=False), sdf)
        sil = silhouette_rays(orc, shifted)
        amb32 = ambiguous_rays(orc, tol_f=1e-5, max_steps=50, normals=orc["normal"])
        out[f"{tag}/n"] = np.int64(orc["mask"].size)
        for k, v in (("mask", orc["mask"]), ("sil", sil), ("amb32", amb32)):
            out[f"{tag}/{k}"] = np.packbits(v.astype(bool))
        # the oracle's depth at its hits (pixel order), rounded to float32
        out[f"{tag}/depth_hits"] = orc["depth"][orc["mask"]].astype(np.float32)
        print(tag, orc["mask"].size, int(orc["mask"].sum()), float(sil.mean()), float(amb32.mean()))
    np.savez_compressed(os.path.join(ROOT, "tests", "golden", "full_masks.npz"), **out)


if __name__ == "__main__":
    main()
