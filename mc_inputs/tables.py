"""Per-material photon cross-section tables at 1 keV nodes.

The paper takes its cross sections and form factors from Hubbell's tables
(Sec. II-A, eqs. KleinNishina/Thomson and the normalisations of the
scatter-toward-detector pdfs).  Those tables are not available here, so this
module tabulates closed-form stand-ins, in FP64:

* incoherent: the Klein-Nishina cross section of a free electron (S = 1),
  times Z per atom, integrated from its differential form by Gauss-Legendre;
* photoelectric: K_pe * Z^4 / E^3 barn per atom;
* coherent: the Thomson differential cross section times F(x)^2 with the
  analytic atomic form factor F_i(x) = Z_i / (1 + b_i x^2)^2,
  b_i = c_F * Z_i^(-2/3), x = sin(theta/2)/lambda in 1/Angstrom;
* I_coh(E) = sum_i w_i Z_i^2 int_{-1}^{1} (1+mu^2) f_i(x(mu))^2 dmu, the
  normalisation of the Rayleigh scatter-toward-detector pdf, with w_i the
  moles of atoms of element i per gram.

Variant "bound" replaces the free-electron incoherent model by one with an
incoherent scattering function (the S(q,Z) of Sec. II-A, eq. pmueforIncoherent):
d(sigma)/d(Omega) = KN x S_mol(x), S_mol = sum_i w_i S_i, and, consistent with
the form factor above (Z_i electrons sharing one orbital factor
f_i = (1 + b_i x^2)^-2), the Waller-Hartree form S_i(x) = Z_i (1 - f_i(x)^2)
= Z_i (1 - (1 + b_i x^2)^-4).  Its normalisation
I_incoh(E) = sum_i w_i int_{-1}^{1} KN_shape(mu) S_i(x(mu)) dmu, with
KN_shape = r^2 (r + 1/r - 1 + mu^2), r = E'/E, gives mu_incoh = pi r0^2 N_A I_incoh.

File layout (little endian), read independently by the oracle (C) and by the
CUDA library (C++):

  char[8]  magic "MCXTAB01"
  int32    version (1, or 2 for the bound incoherent model), n_mat, n_E, max_comp (8)
  float64  E0_keV, dE_keV
  float64  r0_cm, mec2_keV, hc_keVA, N_A, c_F (A^2), K_pe (barn keV^3)
  n_mat x { char[16] name; float64 density; int32 n_comp; int32 pad;
            max_comp x { float64 Z, w (mol/g), b (A^2) } }
  float64  mu_pe[n_mat][n_E], mu_incoh[n_mat][n_E], mu_coh[n_mat][n_E]  (cm^2/g)
  float64  I_coh[n_mat][n_E]
  version 2 only: float64 I_incoh[n_mat][n_E]
"""

from __future__ import annotations

import os
import struct
from dataclasses import dataclass, field

import numpy as np

MAGIC = b"MCXTAB01"
VERSION = 1
MAX_COMP = 8

# CODATA 2018 constants.
R0_CM = 2.8179403262e-13
MEC2_KEV = 510.99895
HC_KEVA = 12.398419843
N_A = 6.02214076e23
# Model constants of the closed-form stand-ins.
C_F = 12.0  # A^2, form-factor width constant
K_PE = 31.5  # barn keV^3, photoelectric constant

# Element data: Z, standard atomic weight.
ELEMENTS = {
    "H": (1, 1.008),
    "Be": (4, 9.0122),
    "C": (6, 12.011),
    "N": (7, 14.007),
    "O": (8, 15.999),
    "Al": (13, 26.9815),
    "P": (15, 30.9738),
    "Ar": (18, 39.948),
    "S": (16, 32.06),
    "Ca": (20, 40.078),
    "Gd": (64, 157.25),
}

# Materials: name, nominal density (g/cm^3), elemental mass fractions.
MATERIALS = [
    ("air", 0.001205, {"C": 0.000124, "N": 0.755268, "O": 0.231781, "Ar": 0.012827}),
    ("water", 1.0, {"H": 0.111894, "O": 0.888106}),
    ("pmma", 1.19, {"H": 0.080538, "C": 0.599848, "O": 0.319614}),
    ("aluminium", 2.70, {"Al": 1.0}),
    ("bone", 1.85, {"H": 0.034, "C": 0.155, "N": 0.042, "O": 0.435, "P": 0.103, "Ca": 0.231}),
]
MAT_AIR, MAT_WATER, MAT_PMMA, MAT_AL, MAT_BONE = range(5)


@dataclass
class Tables:
    E0: float
    dE: float
    names: list
    density: np.ndarray  # [n_mat]
    comps: list  # per material: array [n_comp, 3] of (Z, w, b)
    mu_pe: np.ndarray  # [n_mat, n_E] cm^2/g
    mu_incoh: np.ndarray
    mu_coh: np.ndarray
    I_coh: np.ndarray
    consts: dict = field(default_factory=dict)
    I_incoh: np.ndarray = None  # bound incoherent model only (version 2)

    @property
    def n_mat(self):
        return len(self.names)

    @property
    def n_E(self):
        return self.mu_pe.shape[1]

    @property
    def energies(self):
        return self.E0 + self.dE * np.arange(self.n_E)

    @property
    def mu_tot(self):
        return self.mu_pe + self.mu_incoh + self.mu_coh

    def mu_rho_at(self, mat, E):
        """Total mass attenuation (cm^2/g) linearly interpolated at E (keV)."""
        return np.interp(E, self.energies, self.mu_tot[mat])


def _gl(n=96):
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def kn_sigma_per_electron(E_keV):
    """Klein-Nishina total cross section per free electron (cm^2).

    Integrates d(sigma)/d(Omega) = r0^2/2 (a'/a)^2 (a'/a + a/a' - sin^2)
    over dOmega = 2 pi dmu with Gauss-Legendre (the integrand is a smooth
    rational function of mu on [-1, 1])."""
    E = np.atleast_1d(np.asarray(E_keV, dtype=np.float64))
    x, w = _gl()
    a = E[:, None] / MEC2_KEV
    ratio = 1.0 / (1.0 + a * (1.0 - x[None, :]))
    integrand = ratio**2 * (ratio + 1.0 / ratio - (1.0 - x[None, :] ** 2))
    return np.pi * R0_CM**2 * (integrand * w[None, :]).sum(axis=1)


def coherent_integral(Z, b, E_keV):
    """int_{-1}^{1} (1+mu^2) (1 + b x^2)^(-4) dmu, x^2 = K (1-mu)/2, K = (E/hc)^2.

    The substitution s = ln(1 + b u), u = x^2 makes the integrand a sum of
    smooth exponentials in s, so Gauss-Legendre converges to FP64 accuracy
    even where the form factor confines it to forward angles."""
    E = np.atleast_1d(np.asarray(E_keV, dtype=np.float64))
    K = (E / HC_KEVA) ** 2
    x, w = _gl()
    smax = np.log1p(b * K)  # [nE]
    s = 0.5 * smax[:, None] * (x[None, :] + 1.0)
    u = np.expm1(s) / b
    mu = 1.0 - 2.0 * u / K[:, None]
    # dmu = -(2/K) du, du = e^s / b ds, (1+bu)^-4 = e^(-4s)
    f = (1.0 + mu**2) * np.exp(-3.0 * s) / b * (2.0 / K[:, None])
    return 0.5 * smax * (f * w[None, :]).sum(axis=1)


def kn_shape_integral(E_keV):
    """int_{-1}^{1} r^2 (r + 1/r - 1 + mu^2) dmu (the free-electron KN total / (pi r0^2))."""
    E = np.atleast_1d(np.asarray(E_keV, dtype=np.float64))
    return kn_sigma_per_electron(E) / (np.pi * R0_CM**2)


def incoherent_deficit(Z, b, E_keV):
    """J = int_{-1}^{1} KN_shape(mu) (1 + b x^2)^(-4) dmu, x^2 = K (1-mu)/2: what the
    bound-electron factor S_i/Z_i = 1 - (1 + b x^2)^-4 removes from the
    free-electron integral.  Same substitution s = ln(1 + b u) as the coherent
    integral, so the forward peak is resolved at every energy."""
    E = np.atleast_1d(np.asarray(E_keV, dtype=np.float64))
    K = (E / HC_KEVA) ** 2
    x, w = _gl()
    smax = np.log1p(b * K)
    s = 0.5 * smax[:, None] * (x[None, :] + 1.0)
    u = np.expm1(s) / b
    mu = 1.0 - 2.0 * u / K[:, None]
    r = 1.0 / (1.0 + (E[:, None] / MEC2_KEV) * (1.0 - mu))
    shape = r * r * (r + 1.0 / r - 1.0 + mu * mu)
    f = shape * np.exp(-3.0 * s) / b * (2.0 / K[:, None])
    return 0.5 * smax * (f * w[None, :]).sum(axis=1)


def incoherent_integral(Z, b, E_keV):
    """int_{-1}^{1} KN_shape(mu) S_i(x(mu)) dmu = Z (I_KN - J) for S_i = Z (1 - (1 + b x^2)^-4)."""
    return Z * (kn_shape_integral(E_keV) - incoherent_deficit(Z, b, E_keV))


def material_components(fracs):
    rows = []
    for el, frac in fracs.items():
        Z, A = ELEMENTS[el]
        rows.append((float(Z), frac / A, C_F * Z ** (-2.0 / 3.0)))
    return np.array(rows, dtype=np.float64)


def composition_attenuation(fracs, E_keV):
    """Mass attenuation (cm^2/g) of an elemental composition by the same closed
    forms as the tables: (photoelectric, incoherent, coherent) at E_keV.  For
    materials outside the table file (source window, detector layers)."""
    E = np.atleast_1d(np.asarray(E_keV, dtype=np.float64))
    kn = kn_sigma_per_electron(E)
    pe = np.zeros_like(E)
    inc = np.zeros_like(E)
    coh = np.zeros_like(E)
    for Z, wmol, b in material_components(fracs):
        n_atoms = wmol * N_A
        pe += n_atoms * K_PE * 1e-24 * Z**4 / E**3
        inc += n_atoms * Z * kn
        coh += np.pi * R0_CM**2 * N_A * wmol * Z**2 * coherent_integral(Z, b, E)
    return pe, inc, coh


def kn_energy_transfer_fraction(E_keV):
    """Mean fraction of the photon energy given to the electron in a free-electron
    Klein-Nishina scatter: int (1 - E'/E) dsigma / int dsigma (Gauss-Legendre in mu)."""
    E = np.atleast_1d(np.asarray(E_keV, dtype=np.float64))
    x, w = _gl()
    a = E[:, None] / MEC2_KEV
    ratio = 1.0 / (1.0 + a * (1.0 - x[None, :]))
    ds = ratio**2 * (ratio + 1.0 / ratio - (1.0 - x[None, :] ** 2))
    return ((1.0 - ratio) * ds * w[None, :]).sum(axis=1) / (ds * w[None, :]).sum(axis=1)


def build_tables(n_E=150, E0=1.0, dE=1.0, materials=None, variant="full"):
    """Tabulate all materials at nodes E0 + k dE.

    variant: "full"; "bound" (all interactions, incoherent with the scattering
    function S); or one of "compton", "rayleigh", "photo" to keep only that
    interaction (the others zeroed) -- used for single-process tests."""
    materials = MATERIALS if materials is None else materials
    E = E0 + dE * np.arange(n_E)
    kn = kn_sigma_per_electron(E)
    names, dens, comps = [], [], []
    mu_pe = np.zeros((len(materials), n_E))
    mu_in = np.zeros_like(mu_pe)
    mu_co = np.zeros_like(mu_pe)
    icoh = np.zeros_like(mu_pe)
    iinc = np.zeros_like(mu_pe) if variant == "bound" else None
    for m, (name, rho, fracs) in enumerate(materials):
        c = material_components(fracs)
        names.append(name)
        dens.append(rho)
        comps.append(c)
        for Z, wmol, b in c:
            n_atoms = wmol * N_A  # atoms per gram
            mu_pe[m] += n_atoms * K_PE * 1e-24 * Z**4 / E**3
            if iinc is None:
                mu_in[m] += n_atoms * Z * kn
            else:
                iinc[m] += wmol * incoherent_integral(Z, b, E)
            ci = Z**2 * coherent_integral(Z, b, E)
            icoh[m] += wmol * ci
        mu_co[m] = np.pi * R0_CM**2 * N_A * icoh[m]
        if iinc is not None:
            mu_in[m] = np.pi * R0_CM**2 * N_A * iinc[m]
    if variant == "compton":
        mu_pe[:] = 0.0
        mu_co[:] = 0.0
    elif variant == "rayleigh":
        mu_pe[:] = 0.0
        mu_in[:] = 0.0
    elif variant == "photo":
        mu_in[:] = 0.0
        mu_co[:] = 0.0
    elif variant not in ("full", "bound"):
        raise ValueError(variant)
    consts = dict(r0=R0_CM, mec2=MEC2_KEV, hc=HC_KEVA, N_A=N_A, c_F=C_F, K_pe=K_PE)
    return Tables(E0, dE, names, np.array(dens), comps, mu_pe, mu_in, mu_co, icoh, consts, I_incoh=iinc)


def write_tables(t: Tables, path):
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<4i", VERSION if t.I_incoh is None else 2, t.n_mat, t.n_E, MAX_COMP))
        f.write(struct.pack("<2d", t.E0, t.dE))
        c = t.consts
        f.write(struct.pack("<6d", c["r0"], c["mec2"], c["hc"], c["N_A"], c["c_F"], c["K_pe"]))
        for m in range(t.n_mat):
            name = t.names[m].encode()[:15].ljust(16, b"\0")
            f.write(name)
            f.write(struct.pack("<d", float(t.density[m])))
            comp = t.comps[m]
            f.write(struct.pack("<2i", comp.shape[0], 0))
            buf = np.zeros((MAX_COMP, 3))
            buf[: comp.shape[0]] = comp
            f.write(buf.astype("<f8").tobytes())
        for arr in (t.mu_pe, t.mu_incoh, t.mu_coh, t.I_coh):
            f.write(np.ascontiguousarray(arr, dtype="<f8").tobytes())
        if t.I_incoh is not None:
            f.write(np.ascontiguousarray(t.I_incoh, dtype="<f8").tobytes())


def read_tables(path) -> Tables:
    with open(path, "rb") as f:
        data = f.read()
    if data[:8] != MAGIC:
        raise ValueError("bad table magic")
    ver, n_mat, n_E, max_comp = struct.unpack_from("<4i", data, 8)
    E0, dE = struct.unpack_from("<2d", data, 24)
    r0, mec2, hc, na, cf, kpe = struct.unpack_from("<6d", data, 40)
    off = 88
    names, dens, comps = [], [], []
    for _ in range(n_mat):
        names.append(data[off : off + 16].split(b"\0")[0].decode())
        (rho,) = struct.unpack_from("<d", data, off + 16)
        (nc, _pad) = struct.unpack_from("<2i", data, off + 24)
        buf = np.frombuffer(data, "<f8", max_comp * 3, off + 32).reshape(max_comp, 3)
        comps.append(buf[:nc].copy())
        dens.append(rho)
        off += 32 + max_comp * 24
    arrs = []
    for _ in range(5 if ver == 2 else 4):
        arrs.append(np.frombuffer(data, "<f8", n_mat * n_E, off).reshape(n_mat, n_E).copy())
        off += n_mat * n_E * 8
    consts = dict(r0=r0, mec2=mec2, hc=hc, N_A=na, c_F=cf, K_pe=kpe)
    iinc = arrs.pop() if ver == 2 else None
    return Tables(E0, dE, names, np.array(dens), comps, *arrs, consts=consts, I_incoh=iinc)


def default_table_path(variant="full", directory=None):
    """Write (once) and return the path of the standard table file."""
    if directory is None:
        directory = os.environ.get(
            "MC_DATA_DIR", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "_data")
        )
    os.makedirs(directory, exist_ok=True)
    path = os.path.join(directory, f"tables_{variant}.bin")
    if not os.path.exists(path):
        tmp = path + f".tmp{os.getpid()}"
        write_tables(build_tables(variant=variant), tmp)
        os.replace(tmp, path)
    return path
