"""Named synthetic workloads shaped like the paper's scans.

The paper's objects (car engines, cylinder head, cement samples) and its
scanner data are not available; these seeded phantoms stand in for them.
Sizes follow the project's workload list:

  cyl64    64^3 at 1 mm, water cylinder + Al rod, 60 keV, SOD/SDD 300/600,
           128^2 detector at 1 mm, 1e6 photons, step 0.5 mm
  ell256   256^3 at 0.5 mm, 8-16 seeded ellipsoids, 120 kVp Kramers + 2 mm Al,
           SOD/SDD 400/800, 512^2 detector at 0.4 mm, 1e8 photons, step 0.25 mm
  ell512   512^3 at 0.2 mm, same generator, 60 keV, SOD/SDD 300/600,
           1024^2 at 0.2 mm, 360 angles x 1e7 photons
  tiny8    8^3 at 4 mm, 60 keV, SOD/SDD 100/200, 8x8 detector at 8 mm
"""

from __future__ import annotations

import numpy as np

from .phantoms import cylinder_rod_phantom, ellipsoid_phantom, tiny_phantom
from .spectrum import kramers_spectrum, mono_spectrum

WORKLOADS = {
    "cyl64": dict(
        phantom=("cylinder_rod", {}),
        spectrum=("mono", 60.0),
        geometry=dict(sod=300.0, sdd=600.0, nu=128, nv=128, pu=1.0, pv=1.0),
        n_photons=1_000_000,
        step_mm=0.5,
        seed=1,
    ),
    "ell256": dict(
        phantom=("ellipsoids", dict(n=256, dv=0.5, seed=7)),
        spectrum=("kramers", 120),
        geometry=dict(sod=400.0, sdd=800.0, nu=512, nv=512, pu=0.4, pv=0.4),
        n_photons=100_000_000,
        step_mm=0.25,
        seed=1,
    ),
    "ell512": dict(
        phantom=("ellipsoids", dict(n=512, dv=0.2, seed=11)),
        spectrum=("mono", 60.0),
        geometry=dict(sod=300.0, sdd=600.0, nu=1024, nv=1024, pu=0.2, pv=0.2),
        n_photons=10_000_000,
        n_angles=360,
        step_mm=0.2,
        seed=1,
    ),
    "tiny8": dict(
        phantom=("tiny", {}),
        spectrum=("mono", 60.0),
        geometry=dict(sod=100.0, sdd=200.0, nu=8, nv=8, pu=8.0, pv=8.0),
        n_photons=100_000,
        step_mm=0.5,
        seed=1,
    ),
}


def make_workload(name, tables, **override):
    """Build (volume dict, spectrum (E, w), geometry dict, run params) for a named workload."""
    spec = dict(WORKLOADS[name])
    spec.update(override)
    kind, args = spec["phantom"]
    if kind == "cylinder_rod":
        vol = cylinder_rod_phantom(**args)
    elif kind == "ellipsoids":
        vol = ellipsoid_phantom(**args)
    elif kind == "tiny":
        vol = tiny_phantom(**args)
    else:
        raise ValueError(kind)
    sk, sa = spec["spectrum"]
    if sk == "mono":
        E, w = mono_spectrum(sa)
    else:
        E, w = kramers_spectrum(tables, kvp=sa)
    n_angles = spec.get("n_angles", 1)
    angles = (2.0 * np.pi * np.arange(n_angles) / n_angles).astype(np.float32)
    return dict(
        volume=vol,
        energies=E,
        weights=w,
        geometry=spec["geometry"],
        n_photons=spec["n_photons"],
        step_mm=spec["step_mm"],
        seed=spec["seed"],
        angles=angles,
    )
