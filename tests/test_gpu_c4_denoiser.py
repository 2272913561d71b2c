"""What the trained network gains over the method without it (the learned
denoiser replaces the fixed Savitzky-Golay smoothing of arXiv 2201.13191
Sec. II-C.4 at low photon counts).

On a phantom held out of training (256^3 x 0.25 mm cylinder/rod family, 60 keV,
256^2 x 0.5 mm scatter image), a 1e6-photon scatter image is smoothed by the
paper's filter and denoised by the network trained by
``bench.py --denoise-eval``; both are judged against a 2e9-photon plain Monte
Carlo reference, the error corrected for the reference's own noise (its
20-batch variance).  At equal photons the network's error must be well below
the smoothing's, and the denoised image must stay an image of the same
scatter (its total within 3% of the reference's)."""

import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_denoiser_beats_smoothing_at_equal_photons(gpu):
    torch = pytest.importorskip("torch")
    import bench

    if not os.path.exists(bench.C4_WEIGHTS):
        pytest.skip("trained denoiser weights not present")
    ctx, _ = bench.c4_context(gpu)
    ctx.denoise_load(bench.C4_WEIGHTS, 1)
    v = bench.c4_phantom(bench.C4_HELD_OUT)
    ctx.load_volume(v["mat"], v["rho"], v["spacing"])
    sg = gpu.Context(0)
    errs = {"plain": [], "smoothed": [], "denoised": []}
    for i, ang in enumerate((0.3, 2.2)):
        ref, noise2 = bench.c4_reference(ctx, 2e9, ang, 31 + i)
        img, _ = bench.c4_scatter(ctx, 1e6, ang, 77 + i)
        smooth = sg.smooth_upsample(img[None], [0.0], [0.0], bench.C4_PX, bench.C4_PX)[0]
        den = ctx.denoise_infer(img[None])[0]
        errs["plain"].append(bench.c4_error(img, ref, noise2))
        errs["smoothed"].append(bench.c4_error(smooth, ref, noise2))
        errs["denoised"].append(bench.c4_error(den, ref, noise2))
        assert abs(float(den.double().sum()) / float(ref.sum()) - 1.0) < 0.03
    e = {k: float(np.mean(x)) for k, x in errs.items()}
    print("relative L2 at 1e6 photons vs a 2e9 reference:", e)
    assert e["smoothed"] < e["plain"]
    assert e["denoised"] < 0.5 * e["smoothed"], e
