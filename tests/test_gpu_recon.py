"""Correction plumbing on the GPU (Sec. II-E): each step against the oracle --
line integrals, FDK, the histogram / Otsu thresholds / class map of the
segmentation, the down-sampling for the Monte Carlo step and eq. (Correction)
-- and an end-to-end scatter correction of synthetic measurements."""

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


def _segment_volume(shape, seed):
    """FP32 reconstruction-like volume: air, water and aluminium levels at 60 keV
    with noise, a few values outside [mu_lo, mu_hi) and some on bin edges."""
    rng = np.random.default_rng(seed)
    lvl = rng.choice(3, size=shape, p=[0.5, 0.35, 0.15])
    mu = np.array([0.0002, 0.0206, 0.075])[lvl] + rng.normal(0, 0.004, shape)
    mu.ravel()[:7] = [-0.5, -0.01, 0.09, 0.3, 0.0, 0.05, 0.0890625]
    return mu.astype(np.float32)


@pytest.mark.parametrize("classes,cls_mat", [(2, (0, 1, 1)), (3, (0, 1, 3))])
def test_segmentation_matches_oracle(gpu, table_path, tables, classes, cls_mat):
    """Histogram and Otsu thresholds bit for bit (both take the bin decision in
    FP32), materials bit for bit, densities within one binary16 unit (FP32
    quotient on the device, FP64 in the oracle, both rounded to binary16)."""
    torch = pytest.importorskip("torch")
    vol = _segment_volume((37, 41, 29), 11 + classes)
    lo, hi, e_eff, rho0 = -0.01, 0.09, 60.0, 0.001205
    c = gpu.Context(0)
    c.load_tables(table_path)
    mat, rho, hist, thr = c.segment(torch.from_numpy(vol).cuda(), classes, cls_mat[:classes], rho0, e_eff, lo, hi)
    murho = [np.interp(e_eff, tables.energies, tables.mu_tot[m]) for m in cls_mat]
    m_ref, r_ref, h_ref, t_ref = recon.segment(vol, lo, hi, classes, cls_mat, murho, rho0)
    np.testing.assert_array_equal(hist.astype(np.int64), h_ref)
    assert tuple(int(t) for t in thr) == tuple(t_ref), (thr, t_ref)
    np.testing.assert_array_equal(mat.cpu().numpy(), m_ref)
    got = rho.cpu().numpy().view(np.float16).astype(np.float64)
    ref16 = r_ref.astype(np.float16)
    ulp = np.spacing(ref16).astype(np.float64)
    assert np.all(np.abs(got - ref16.astype(np.float64)) <= ulp), np.max(np.abs(got - ref16) / ulp)
    assert np.mean(got == ref16.astype(np.float64)) > 0.99
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.segment(torch.from_numpy(vol).cuda(), 4, cls_mat, rho0, e_eff, lo, hi)


def test_line_integrals_and_correction_match_oracle(gpu):
    """a = -ln(I/I0) and eq. (Correction) per element against the oracle at FP32
    tolerance: a quotient (2^-24 relative), logf (1 unit in the last place)
    and the final subtraction give |dc| <= 2e-7 (1 + |a| + |c|); the bound
    below is twice that."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    n, NV, NU = 3, 17, 23
    I0 = rng.uniform(0.5, 2.0, (NV, NU)).astype(np.float32)
    I = (I0 * np.exp(-rng.uniform(0, 8, (n, NV, NU)))).astype(np.float32)
    I.ravel()[:3] = [0.0, -1.0, 1e-35]  # clamped to 1e-30
    c = gpu.Context(0)
    a = c.line_integrals(torch.from_numpy(I).cuda(), torch.from_numpy(I0).cuda()).cpu().numpy().astype(np.float64)
    a_ref = recon.line_integrals(I, I0[None])
    assert np.all(np.abs(a - a_ref) <= 4e-7 * (1 + np.abs(a_ref))), np.max(np.abs(a - a_ref) / (1 + np.abs(a_ref)))
    ip = (I0[None] * np.exp(-rng.uniform(0, 8, (n, NV, NU)))).astype(np.float32)
    is_ = (ip * rng.uniform(0, 3, ip.shape)).astype(np.float32)
    is_.ravel()[:2] = [-1.0, 0.0]  # negative scatter clamps to 0: c = a there
    ip.ravel()[2] = 0.0  # clamped to 1e-30
    a32 = a.astype(np.float32)
    for scale in (1.0, 0.0625):
        cc = c.correct_images(torch.from_numpy(a32).cuda(), torch.from_numpy(ip).cuda(), torch.from_numpy(is_).cuda(),
                              scale).cpu().numpy().astype(np.float64)
        ref = recon.correct(a32, ip, is_, scale)
        tol = 4e-7 * (1 + np.abs(a32) + np.abs(ref))
        assert np.all(np.abs(cc - ref) <= tol), np.max(np.abs(cc - ref) / tol)
        assert cc.ravel()[0] == a32.ravel()[0] and cc.ravel()[1] == a32.ravel()[1]
    with pytest.raises(gpu.MCError, match="INVALID_ARG"):
        c.correct_images(torch.from_numpy(a32).cuda(), torch.from_numpy(ip).cuda(), torch.from_numpy(is_).cuda(), -1.0)


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
