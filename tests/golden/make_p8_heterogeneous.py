"""Writes p8_single_scatter_het8.txt: the expected single-scatter (order-1)
image of the point-detector estimator -- eq. (Th) split into pseudo-particles
and summed per eq. (Is) of arXiv 2201.13191 Sec. II-A -- on a two-material
phantom, by deterministic quadrature instead of photon histories.

Phantom: 8^3 voxels of 4 mm, water (binary16 1.0 g/cm^3) with a 2 x 2 x 2
aluminium insert (binary16 2.7) at z 2..3, y 4..5, x 3..4; 60 keV; SOD/SDD
100/250 mm; 8 x 8 panel of 4 mm pixels; beta = 0; fixed step 2 mm.

The estimator's expectation is integrated as the transport defines it
(Sec. II-C.2, the fixed-step march):
  - source point Q uniform on the panel, weight A_det cos(gamma_Q) / (4 pi d^2)
    (composite Gauss-Legendre over the panel's pixels);
  - the source ray's chord through the box cut into n = ceil(L / step) equal
    steps, each with the attenuation of the voxel at its midpoint, so the
    first interaction has the piecewise-exponential density
    mu_k exp(-(tau_k + mu_k (t - t_k))) on step k (Gauss-Legendre per step);
  - at the interaction point X, Compton with probability mu_incoh / mu and
    Rayleigh with mu_coh / mu of the step's voxel material;
  - toward a target point P of pixel j (Gauss-Legendre over the pixel):
    eta(E') p(lambda) cos(gamma_P) / (2 pi d^2) exp(-tau'), p the normalised
    scatter-toward-detector pdfs of eqs. (pmueforIncoherent) and
    (pmueforcoherent), tau' the same fixed-step march from X to P at E'.
The march here is this script's own numpy code (clip, step count, midpoints,
nearest voxel), not the oracle's.  Tables come from mc_inputs, the
Klein-Nishina normalisation from the oracle's closed form (pinned on its
own).  The image is computed at two quadrature orders; the file records the
finer one and the largest per-pixel change between them.

    python tests/golden/make_p8_heterogeneous.py
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

OUT = os.path.join(HERE, "p8_single_scatter_het8.txt")
N_VOX, DV = 8, 4.0
GEO = dict(sod=100.0, sdd=250.0, nu=8, nv=8, pu=4.0, pv=4.0)
E0, STEP = 60.0, 2.0
AL_SLICE = (slice(2, 4), slice(4, 6), slice(3, 5))  # (z, y, x)


def phantom():
    """(mat, rho) arrays [z][y][x] with the densities as binary16 values."""
    from mc_inputs.tables import MAT_AL, MAT_WATER

    mat = np.full((N_VOX,) * 3, MAT_WATER, np.uint8)
    rho = np.full((N_VOX,) * 3, float(np.float16(1.0)))
    mat[AL_SLICE] = MAT_AL
    rho[AL_SLICE] = float(np.float16(2.7))
    return mat, rho


def phantom_volume():
    """The same phantom as an mc_inputs volume dict (binary16 bit patterns)."""
    mat, rho = phantom()
    return dict(mat=mat, rho=rho.astype(np.float16).view(np.uint16), shape=mat.shape, spacing=(DV, DV, DV))


class March:
    """Fixed-step march through the centred voxel box: per-material column
    masses rho * L (g/cm^3 mm) of many rays at once."""

    def __init__(self, mat, rho, n_mat):
        self.mat, self.rho, self.n_mat = mat, rho, n_mat
        self.h = N_VOX * DV / 2.0

    def clip(self, p0, w, t0, t1):
        ta = np.full(p0.shape[:-1], t0, dtype=np.float64)
        tb = np.full(p0.shape[:-1], t1, dtype=np.float64)
        for k in range(3):
            wk, pk = w[..., k], p0[..., k]
            with np.errstate(divide="ignore", invalid="ignore"):
                u = (-self.h - pk) / wk
                v = (self.h - pk) / wk
            lo, hi = np.minimum(u, v), np.maximum(u, v)
            zero = wk == 0
            inside = (pk >= -self.h) & (pk <= self.h)
            lo = np.where(zero, np.where(inside, -np.inf, np.inf), lo)
            hi = np.where(zero, np.where(inside, np.inf, -np.inf), hi)
            ta, tb = np.maximum(ta, lo), np.minimum(tb, hi)
        return ta, tb

    def steps(self, p0, w, t0, t1):
        """ta, h, n and the voxel index of every step midpoint ([..., n_max], -1 past the end)."""
        ta, tb = self.clip(p0, w, t0, t1)
        L = np.where(tb > ta, tb - ta, 0.0)
        n = np.where(L > 0, np.maximum(1, np.ceil(L / STEP)), 0).astype(np.int64)
        h = np.where(n > 0, L / np.maximum(n, 1), 0.0)
        n_max = int(n.max()) if n.size else 0
        k = np.arange(n_max)
        t = ta[..., None] + (k + 0.5) * h[..., None]
        p = p0[..., None, :] + t[..., None] * w[..., None, :]
        ijk = np.clip(np.floor((p + self.h) / DV).astype(np.int64), 0, N_VOX - 1)
        vox = (ijk[..., 2] * N_VOX + ijk[..., 1]) * N_VOX + ijk[..., 0]
        vox = np.where(k < n[..., None], vox, -1)
        return ta, h, n, vox

    def rho_l(self, p0, w, t0, t1):
        _, h, _, vox = self.steps(p0, w, t0, t1)
        valid = vox >= 0
        v = np.where(valid, vox, 0)
        m = self.mat.ravel()[v]
        r = np.where(valid, self.rho.ravel()[v], 0.0) * h[..., None]
        out = np.zeros(p0.shape[:-1] + (self.n_mat,))
        for q in range(self.n_mat):
            out[..., q] = np.sum(np.where(m == q, r, 0.0), axis=-1)
        return out


_CTX = {}


def _setup():
    """Tables, phantom and per-material constants (once per process)."""
    if _CTX:
        return _CTX
    import tempfile

    import oracle
    from mc_inputs import default_table_path, read_tables
    from mc_inputs.tables import HC_KEVA, MEC2_KEV

    T = read_tables(default_table_path("full", os.path.join(tempfile.gettempdir(), "mc_golden_tables")))
    mat, rho = phantom()
    nm = T.n_mat
    en = T.energies
    _CTX.update(
        T=T, mat=mat, rho=rho, nm=nm, mar=March(mat, rho, nm), en=en,
        mu_in=np.array([np.interp(E0, en, T.mu_incoh[m]) for m in range(nm)]) * 0.1,
        mu_co=np.array([np.interp(E0, en, T.mu_coh[m]) for m in range(nm)]) * 0.1,
        icoh=np.array([np.interp(E0, en, T.I_coh[m]) for m in range(nm)]),
        mu0=np.array([np.interp(E0, en, T.mu_tot[m]) * 0.1 for m in range(nm)]),
        jkn=oracle.kn_norm(E0), K=(E0 / HC_KEVA) ** 2, mec2=MEC2_KEV)
    return _CTX


G_S = np.array([GEO["sod"], 0.0, 0.0])
G_C = np.array([GEO["sod"] - GEO["sdd"], 0.0, 0.0])
G_EU, G_EV, G_N = np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])


def panel_nodes(n):
    """Composite Gauss-Legendre nodes over every pixel: points [nv*nu*n*n, 3], weights (area), pixel index."""
    g = GEO
    x, wgt = np.polynomial.legendre.leggauss(n)
    pi, pj = np.meshgrid(np.arange(g["nu"]), np.arange(g["nv"]), indexing="xy")
    shape = (g["nv"], g["nu"], n, n)
    a = np.broadcast_to(pi[..., None, None] + 0.5 * (x[:, None] + 1.0), shape)
    b = np.broadcast_to(pj[..., None, None] + 0.5 * (x[None, :] + 1.0), shape)
    wab = 0.25 * wgt[:, None] * wgt[None, :] * g["pu"] * g["pv"]
    P = G_C + ((a - g["nu"] / 2) * g["pu"])[..., None] * G_EU + ((b - g["nv"] / 2) * g["pv"])[..., None] * G_EV
    pix = np.broadcast_to((pj * g["nu"] + pi)[..., None, None], shape)
    return P.reshape(-1, 3), np.broadcast_to(wab, shape).reshape(-1), pix.reshape(-1)


def _source_node(args):
    """Contribution to the image of one source node Q (weight wq) with nt depth
    nodes per step and npx^2 target nodes per pixel."""
    Q, wq, nt, npx = args
    X_ = _setup()
    T, nm, mar = X_["T"], X_["nm"], X_["mar"]
    en, mu0, mu_in, mu_co, icoh = X_["en"], X_["mu0"], X_["mu_in"], X_["mu_co"], X_["icoh"]
    g = GEO
    Ps, wP, pixP = panel_nodes(npx)
    xt, wt = np.polynomial.legendre.leggauss(nt)
    matv, rhov = X_["mat"].ravel(), X_["rho"].ravel()
    D = Q - G_S
    d = np.linalg.norm(D)
    w = D / d
    wsrc = wq * (g["sdd"] / d) / (4 * np.pi * d * d)
    ta, h, n, vox = mar.steps(G_S[None], w[None], 0.0, np.inf)
    ta, h, n, vox = float(ta[0]), float(h[0]), int(n[0]), vox[0]
    out = np.zeros(g["nu"] * g["nv"])
    if n == 0:
        return out
    ms = matv[vox[:n]]
    mus = rhov[vox[:n]] * mu0[ms]
    tau_k = np.concatenate([[0.0], np.cumsum(mus * h)])[:-1]
    tk = ta + np.arange(n) * h
    t = tk[:, None] + 0.5 * (xt[None, :] + 1.0) * h
    dens = np.exp(-(tau_k[:, None] + mus[:, None] * (t - tk[:, None]))) * 0.5 * h * wt[None, :]
    X = G_S + t.reshape(-1)[:, None] * w
    mX = np.repeat(ms, nt)
    rX = np.repeat(rhov[vox[:n]], nt)
    dX = dens.reshape(-1)
    DD = Ps[None, :, :] - X[:, None, :]
    dd = np.linalg.norm(DD, axis=-1)
    dirs = DD / dd[..., None]
    lam = dirs @ w
    cosg = -(dirs @ G_N)
    rl = mar.rho_l(np.broadcast_to(X[:, None, :], dirs.shape), dirs, 0.0, dd)
    geo = cosg / (2 * np.pi * dd * dd) * wP[None, :]
    # Compton at E' = E / (1 + alpha (1 - lambda)), pdf of eq. (pmueforIncoherent)
    r = 1.0 / (1.0 + E0 / X_["mec2"] * (1.0 - lam))
    Ep = E0 * r
    p_c = r * r * (r + 1.0 / r - 1.0 + lam * lam) / X_["jkn"]
    tau_c = sum(np.interp(Ep, en, T.mu_tot[m]) * 0.1 * rl[..., m] for m in range(nm))
    sc = (rX * mu_in[mX])[:, None] * Ep * p_c * np.exp(-tau_c) * geo
    # Rayleigh at E, pdf of eq. (pmueforcoherent) with the material's form factor
    u = 0.5 * X_["K"] * (1.0 - lam)
    f2 = np.stack([sum(wz * Z * Z / (1.0 + b * u) ** 4 for Z, wz, b in T.comps[m]) for m in range(nm)], 0)
    p_r = (1.0 + lam * lam) * f2[mX, np.arange(len(mX)), :] / icoh[mX][:, None]
    tau_r = sum(mu0[m] * rl[..., m] for m in range(nm))
    sc = sc + (rX * mu_co[mX])[:, None] * E0 * p_r * np.exp(-tau_r) * geo
    contrib = (dX[:, None] * sc).sum(0) * wsrc
    return np.bincount(pixP, weights=contrib, minlength=out.size)


def quadrature(nq, nt, npx, procs=1):
    Qs, wQ, _ = panel_nodes(nq)
    jobs = [(Q, wq, nt, npx) for Q, wq in zip(Qs, wQ)]
    if procs > 1:
        import multiprocessing as mp

        with mp.get_context("spawn").Pool(procs) as pool:
            parts = pool.map(_source_node, jobs, chunksize=8)
    else:
        parts = [_source_node(j) for j in jobs]
    return np.sum(parts, axis=0).reshape(GEO["nv"], GEO["nu"])


def main():
    t0 = time.time()
    procs = int(sys.argv[1]) if len(sys.argv) > 1 else max(1, (os.cpu_count() or 2) - 1)
    coarse = quadrature(4, 4, 4, procs)
    fine = quadrature(8, 6, 6, procs)
    change = np.abs(fine / coarse - 1.0)
    with open(OUT, "w") as f:
        f.write("# Expected single-scatter image (eq. Th / Is, order 1) of the two-material 8^3 phantom by\n")
        f.write("# deterministic quadrature (tests/golden/make_p8_heterogeneous.py): water 8^3 x 4 mm with an\n")
        f.write("# aluminium 2^3 insert at z 2..3, y 4..5, x 3..4; 60 keV; SOD/SDD 100/250 mm; 8 x 8 panel of\n")
        f.write("# 4 mm pixels; beta 0; step 2 mm.  Rows v = 0..7, columns u = 0..7 (keV per source photon).\n")
        f.write(f"# quadrature orders (source, depth, target) 8/6/6; largest per-pixel change from 4/4/4: "
                f"{change.max():.3e}\n")
        for row in fine:
            f.write(" ".join(f"{v:.12e}" for v in row) + "\n")
    print(f"wrote {OUT} in {time.time() - t0:.0f} s; largest per-pixel change between orders {change.max():.3e}, "
          f"total change {abs(fine.sum() / coarse.sum() - 1):.3e}")


if __name__ == "__main__":
    main()
