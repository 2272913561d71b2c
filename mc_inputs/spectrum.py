"""Source spectra as discrete 1 keV bins (Sec. II-A: polychromatic source by energy bins).

The paper's tube spectrum comes from a Geant4 simulation that is not
available; Kramers' law with aluminium filtration stands in for it.
"""

from __future__ import annotations

import numpy as np


def kramers_spectrum(tables, kvp=120, e_min=10, al_mm=2.0):
    """Kramers' law S(E) ~ (kVp - E)/E at integer-keV nodes e_min..kVp, filtered by
    exp(-mu_Al(E) rho_Al t).  Returns (energies_keV float32, weights float64 summing to 1)."""
    E = np.arange(e_min, kvp + 1, dtype=np.float64)
    al = tables.names.index("aluminium")
    mu = tables.mu_rho_at(al, E) * tables.density[al] * (al_mm * 0.1)
    w = np.clip(kvp - E, 0.0, None) / E * np.exp(-mu)
    w = w / w.sum()
    return E.astype(np.float32), w


def mono_spectrum(e_kev=60.0):
    return np.array([e_kev], dtype=np.float32), np.array([1.0])
