"""Flat-panel detector response eta(E) (Sec. II-D.2, "Simulation of the Detector").

The paper simulates its PaxScan 4030E panel -- a 2.86 cm vacuum gap, a 0.25 cm
carbon cover, a thin aluminium foil and a 0.0208 cm gadolinium oxysulfide
scintillator -- with Geant4 and maps each detected photon energy through the
resulting energy-response curve.  Geant4 is not available; this module gives
the analytic counterpart from the closed-form cross sections of `tables`:

  eta(E) = T_C(E) T_Al(E) (1 - exp(-mu_GOS(E) rho t)) E (mu_pe + f_KN(E) mu_incoh) / mu_tot

the mean energy deposited in the scintillator by a photon of energy E at
normal incidence, counting its first interaction only: attenuation by the
carbon cover and the foil, the absorption probability of the screen, and the
share of that interaction's energy left in the screen (all of it for a
photoelectric absorption, the mean electron energy f_KN E for a Compton
scatter, nothing for a coherent one).  Fluorescence escape, scatter inside
the screen and the optical stage are left out.  Readings: the foil is taken
as 0.01 cm; the cover as carbon at 1.7 g/cm^3; the screen at the bulk density
of Gd2O2S, 7.32 g/cm^3.
"""

from __future__ import annotations

import numpy as np

from .tables import composition_attenuation, kn_energy_transfer_fraction

CARBON = {"C": 1.0}
ALUMINIUM = {"Al": 1.0}
# Gd2O2S by mass (2 x 157.25 + 2 x 15.999 + 32.06 = 378.558 g/mol)
GOS = {"Gd": 314.5 / 378.558, "O": 31.998 / 378.558, "S": 32.06 / 378.558}


def flat_panel_response(energies_keV, carbon_cm=0.25, carbon_density=1.7, al_cm=0.01, gos_cm=0.0208,
                        gos_density=7.32):
    """eta(E) in keV per photon of energy E reaching the panel, at the given energies (FP64)."""
    E = np.atleast_1d(np.asarray(energies_keV, dtype=np.float64))
    pc, ic, cc = composition_attenuation(CARBON, E)
    pa, ia, ca = composition_attenuation(ALUMINIUM, E)
    pg, ig, cg = composition_attenuation(GOS, E)
    t_cover = np.exp(-(pc + ic + cc) * carbon_density * carbon_cm - (pa + ia + ca) * 2.70 * al_cm)
    mu_g = pg + ig + cg
    absorbed = 1.0 - np.exp(-mu_g * gos_density * gos_cm)
    share = (pg + kn_energy_transfer_fraction(E) * ig) / mu_g
    return t_cover * absorbed * E * share


def table_response(tables, **kw):
    """eta at the table's energy nodes (what mc_set_detector_response takes)."""
    return flat_panel_response(tables.energies, **kw)
