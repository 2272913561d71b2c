"""Correction plumbing on the GPU (Sec. II-E): FDK parity with the oracle and
an end-to-end scatter correction of synthetic measurements."""

import numpy as np
import pytest

from mc_inputs import cylinder_variant_phantom, mono_spectrum
from oracle import recon

pytestmark = pytest.mark.gpu

SOD, SDD = 300.0, 600.0


def test_fdk_parity(gpu, table_path):
    torch = pytest.importorskip("torch")
    from test_recon_oracle import cylinder_projections

    angles, p = cylinder_projections(48, 40, 24, 3.0, 3.0, 20.0, 50.0, 0.02)
    p += 0.002 * np.random.default_rng(0).normal(size=p.shape)  # break symmetry
    c = gpu.Context(0)
    c.set_geometry(SOD, SDD, 40, 24, 3.0, 3.0)
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.fdk(torch.zeros((48, 24, 40), device="cuda"), angles, 40, 24, (0, 33, 7, 1.1, 0.9, 2.0))
    got = c.fdk(torch.tensor(p, dtype=torch.float32).cuda(), angles, 40, 24, (30, 33, 7, 1.1, 0.9, 2.0)).cpu().numpy()
    ref = recon.fdk(p.astype(np.float32).astype(np.float64), angles.astype(np.float32), 3.0, 3.0, SOD, SDD,
                    (30, 33, 7, 1.1, 0.9, 2.0))
    assert np.abs(got - ref).max() <= 2e-4 * np.abs(ref).max()


def test_scatter_correction_end_to_end(gpu, table_path, tables):
    """Measurements = exact primary + Monte Carlo scatter of a held-out phantom;
    two correction iterations must remove most of the scatter bias of the line
    integrals and of the reconstructed attenuation."""
    torch = pytest.importorskip("torch")
    NU = NV = 96
    n_proj = 64
    angles = (2 * np.pi * np.arange(n_proj) / n_proj).astype(np.float32)
    E, w = mono_spectrum(60.0)
    truth = cylinder_variant_phantom(777)
    c = gpu.Context(0)
    c.load_tables(table_path)
    c.set_spectrum(E, w)
    c.set_geometry(SOD, SDD, NU, NV, 1.2, 1.2)
    c.load_volume(truth["mat"], truth["rho"], truth["spacing"])
    ip_true = c.project(angles, 1, 0.5, 1, scatter=False)["primary"]
    # measured scatter: Monte Carlo on a 48^2 grid at every angle, interpolated to the panel
    c.set_geometry(SOD, SDD, 48, 48, 2.4, 2.4)
    is48 = c.project(angles, 2_000_000, 0.5, 3, primary=False)["scatter"]
    c.set_geometry(SOD, SDD, NU, NV, 1.2, 1.2)
    is_true = c.smooth_upsample(is48, angles, angles, NU, NV) * (48.0 / NU) ** 2  # per-pixel values scale with area
    vac = dict(truth, rho=np.zeros_like(truth["rho"]))
    c.load_volume(vac["mat"], vac["rho"], vac["spacing"])
    I0 = c.project([0.0], 1, 0.5, 1, scatter=False)["primary"][0]
    raw = ip_true + is_true
    a_true = -torch.log(ip_true / I0)
    a_raw = -torch.log(raw / I0)
    errs = {}
    for full, mc_bin in ((1, 0), (0, 0), (1, 2)):
        prm = gpu.binding.CorrectParams(nx=64, ny=64, nz=64, dx=1.0, dy=1.0, dz=1.0, sim_nu=48, sim_nv=48,
                                        sim_angle_stride=2, photons=1_000_000, step_mm=0.5, seed=11, classes=2,
                                        class_material=(0, 1, 1), class_density0=0.001205, e_eff_keV=60.0,
                                        mu_lo=-0.01, mu_hi=0.08, primary_full_res=full, mc_bin=mc_bin)
        out, vol, secs = c.correct_iter(raw, I0, angles, NU, NV, 2, prm)
        errs[(full, mc_bin)] = float(torch.linalg.norm(out - a_true) / torch.linalg.norm(a_true))
        assert len(secs) == 2 and all(s > 0 for s in secs)
        if (full, mc_bin) == (1, 0):
            vol_full = vol
    err_raw = float(torch.linalg.norm(a_raw - a_true) / torch.linalg.norm(a_true))
    print("line-integral error: uncorrected", err_raw, "corrected", errs)
    assert errs[(1, 0)] < 0.35 * err_raw and errs[(0, 0)] < 0.8 * err_raw, (errs, err_raw)
    # the scatter simulated on the volume down-sampled by 2 (the paper's speed-up) corrects as well
    assert errs[(1, 2)] < 0.35 * err_raw, (errs, err_raw)
    vol = vol_full
    # cupping: the reconstructed water attenuation in the central slice, centre vs ring
    v_true = c.fdk(a_true, angles, NU, NV, (64, 64, 64, 1.0, 1.0, 1.0)).cpu().numpy()
    v_raw = c.fdk(a_raw, angles, NU, NV, (64, 64, 64, 1.0, 1.0, 1.0)).cpu().numpy()
    v_cor = vol.cpu().numpy()
    water = truth["mat"] == 1
    d_raw = np.abs(v_raw[water] - v_true[water]).mean()
    d_cor = np.abs(v_cor[water] - v_true[water]).mean()
    assert d_cor < 0.5 * d_raw, (d_cor, d_raw)


def test_bin_volume_matches_oracle(gpu, table_path, tables):
    """The 2x2x2 down-sampling for the Monte Carlo step against oracle/recon.py: the same materials, densities
    within one binary16 unit (FP32 sums on the device, FP64 in the oracle, then rounding to binary16)."""
    torch = pytest.importorskip("torch")
    from oracle.recon import bin_volume

    rng = np.random.default_rng(9)
    mat = rng.choice(np.array([0, 1, 3], np.uint8), size=(10, 12, 16))
    dens = np.where(mat == 0, 0.001205, np.where(mat == 1, 1.0, 2.7)) * rng.uniform(0.7, 1.3, mat.shape)
    rho16 = dens.astype(np.float16)
    c = gpu.Context(0)
    c.load_tables(table_path)
    mo, ro = c.bin_volume(torch.from_numpy(mat).cuda(), torch.from_numpy(rho16.view(np.int16)).cuda(), 60.0)
    murho = np.array([np.interp(60.0, tables.energies, tables.mu_tot[m]) for m in range(tables.n_mat)])
    mb, rb = bin_volume(mat, rho16.astype(np.float64), murho)
    np.testing.assert_array_equal(mo.cpu().numpy(), mb)
    got = ro.cpu().numpy().view(np.float16).astype(np.float64)
    ulp = np.spacing(rb.astype(np.float16)).astype(np.float64)
    assert np.all(np.abs(got - rb) <= ulp), np.max(np.abs(got - rb) / ulp)
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.bin_volume(torch.zeros((3, 4, 4), dtype=torch.uint8, device="cuda"),
                     torch.zeros((3, 4, 4), dtype=torch.int16, device="cuda"), 60.0)
