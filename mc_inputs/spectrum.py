"""Source spectra as discrete 1 keV bins (Sec. II-A: polychromatic source by energy bins).

The paper's tube spectrum comes from a Geant4 simulation of its tungsten-target
source behind a 500 um beryllium window and optional aluminium filters
(Sec. II-D.1); that simulation is not available, so Kramers' law filtered by
the window and the filters stands in for it.
"""

from __future__ import annotations

import numpy as np

from .tables import composition_attenuation


def kramers_spectrum(tables, kvp=120, e_min=10, al_mm=2.0, be_mm=0.0):
    """Kramers' law S(E) ~ (kVp - E)/E at integer-keV nodes e_min..kVp, filtered by
    exp(-mu_Al(E) rho_Al t_Al) and, when be_mm > 0, a beryllium window
    exp(-mu_Be(E) rho_Be t_Be) (1.85 g/cm^3).  Returns (energies_keV float32,
    weights float64 summing to 1)."""
    E = np.arange(e_min, kvp + 1, dtype=np.float64)
    al = tables.names.index("aluminium")
    mu = tables.mu_rho_at(al, E) * tables.density[al] * (al_mm * 0.1)
    if be_mm > 0:
        pe, inc, coh = composition_attenuation({"Be": 1.0}, E)
        mu = mu + (pe + inc + coh) * 1.85 * (be_mm * 0.1)
    w = np.clip(kvp - E, 0.0, None) / E * np.exp(-mu)
    w = w / w.sum()
    return E.astype(np.float32), w


def filtered_spectra(tables, kvp=150, al_mm=(0.0, 1.0, 2.0, 4.0), be_mm=0.5):
    """The spectrum variants of one tube setting behind the window with different
    aluminium filters (the paper's Fig. of source spectra): {al_mm: (E, w)}."""
    return {a: kramers_spectrum(tables, kvp=kvp, al_mm=a, be_mm=be_mm) for a in al_mm}


def mono_spectrum(e_kev=60.0):
    return np.array([e_kev], dtype=np.float32), np.array([1.0])
