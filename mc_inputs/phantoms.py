"""Seeded voxel phantoms: uint8 material ids and FP16 densities.

Layout is [nz][ny][nx], x fastest; voxel (ix, iy, iz) has its centre at
((ix - (nx-1)/2) dx, (iy - (ny-1)/2) dy, (iz - (nz-1)/2) dz) mm, so the
volume is centred on the isocentre.  A voxel takes the material of the last
shape (painter's order) that contains its centre; the rest is air.
"""

from __future__ import annotations

import numpy as np

from .tables import MATERIALS, MAT_AIR, MAT_AL, MAT_BONE, MAT_PMMA, MAT_WATER

NOMINAL_DENSITY = np.array([m[1] for m in MATERIALS])


def fp16_bits(x):
    return np.asarray(x, dtype=np.float16).view(np.uint16)


def fp16_values(bits):
    return np.asarray(bits, dtype=np.uint16).view(np.float16).astype(np.float64)


def _centres(n, d):
    return ((np.arange(n) - (n - 1) / 2.0) * d).astype(np.float64)


def _finish(mat, dens=None):
    if dens is None:
        dens = NOMINAL_DENSITY[mat]
    return dict(mat=np.ascontiguousarray(mat, dtype=np.uint8), rho=fp16_bits(dens))


def cylinder_rod_phantom(n=64, dv=1.0, r_cyl=25.0, h_cyl=60.0, r_rod=5.0, rod_x=10.0):
    """Air, a centred water cylinder (axis z) and an aluminium rod parallel to z."""
    c = _centres(n, dv)
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    mat = np.full((n, n, n), MAT_AIR, dtype=np.uint8)
    inz = np.abs(z) <= h_cyl / 2.0
    mat[(x**2 + y**2 <= r_cyl**2) & inz] = MAT_WATER
    mat[((x - rod_x) ** 2 + y**2 <= r_rod**2) & inz] = MAT_AL
    out = _finish(mat)
    out.update(shape=(n, n, n), spacing=(dv, dv, dv))
    return out


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ]
    )


def ellipsoid_params(seed, n_min=8, n_max=16, fov_half=64.0, axis_range=(5.0, 40.0)):
    """Seeded ellipsoid list: (centre, semi-axes, rotation, material)."""
    rng = np.random.default_rng(seed)
    k = int(rng.integers(n_min, n_max + 1))
    out = []
    mats = [MAT_WATER, MAT_PMMA, MAT_AL, MAT_BONE]
    for _ in range(k):
        # uniform in the inscribed sphere
        while True:
            p = rng.uniform(-1.0, 1.0, size=3)
            if p @ p <= 1.0:
                break
        centre = p * fov_half * 0.6
        axes = rng.uniform(axis_range[0], axis_range[1], size=3)
        axes = np.minimum(axes, fov_half * 0.6)
        rot = _random_rotation(rng)
        m = mats[int(rng.integers(0, 4))]
        out.append((centre, axes, rot, m))
    return out


def ellipsoid_phantom(n=256, dv=0.5, seed=0, n_min=8, n_max=16):
    """Air with 8-16 seeded random ellipsoids of water/PMMA/Al/bone."""
    fov_half = n * dv / 2.0
    params = ellipsoid_params(seed, n_min, n_max, fov_half)
    c = _centres(n, dv).astype(np.float32)
    mat = np.full((n, n, n), MAT_AIR, dtype=np.uint8)
    for centre, axes, rot, m in params:
        # bounding box of the rotated ellipsoid
        half = np.sqrt(((rot * axes[None, :]) ** 2).sum(axis=1))
        lo = np.searchsorted(c, centre - half - dv, side="left")
        hi = np.searchsorted(c, centre + half + dv, side="right")
        lo = np.clip(lo, 0, n)
        hi = np.clip(hi, 0, n)
        if np.any(hi <= lo):
            continue
        xs = c[lo[0] : hi[0]] - centre[0]
        ys = c[lo[1] : hi[1]] - centre[1]
        inv = (rot / axes[None, :]).astype(np.float32)  # local = rot^T p / axes
        for iz in range(lo[2], hi[2]):
            zc = c[iz] - centre[2]
            # local coordinates l_j = sum_a rot[a, j] p_a / axes_j
            l0 = xs[None, :] * inv[0, 0] + ys[:, None] * inv[1, 0] + zc * inv[2, 0]
            l1 = xs[None, :] * inv[0, 1] + ys[:, None] * inv[1, 1] + zc * inv[2, 1]
            l2 = xs[None, :] * inv[0, 2] + ys[:, None] * inv[1, 2] + zc * inv[2, 2]
            inside = l0 * l0 + l1 * l1 + l2 * l2 <= 1.0
            sl = mat[iz, lo[1] : hi[1], lo[0] : hi[0]]
            sl[inside] = m
    out = _finish(mat)
    out.update(shape=(n, n, n), spacing=(dv, dv, dv))
    return out


def tiny_phantom(n=8, dv=4.0):
    """8^3 phantom: a water block with an aluminium cube inside, in air."""
    mat = np.full((n, n, n), MAT_AIR, dtype=np.uint8)
    mat[1:7, 1:7, 1:7] = MAT_WATER
    mat[3:5, 2:4, 3:6] = MAT_AL
    dens = NOMINAL_DENSITY[mat].copy()
    dens[mat == MAT_WATER] = 1.0
    out = _finish(mat, dens)
    out.update(shape=(n, n, n), spacing=(dv, dv, dv))
    return out


def slab_phantom(n=(16, 16, 16), dv=(2.0, 2.0, 2.0), material=MAT_WATER, density=None):
    """Homogeneous box of one material filling the volume; n = (nz, ny, nx), dv = (dx, dy, dz)."""
    nz, ny, nx = n
    mat = np.full((nz, ny, nx), material, dtype=np.uint8)
    dens = np.full(mat.shape, NOMINAL_DENSITY[material] if density is None else density)
    out = _finish(mat, dens)
    out.update(shape=(nz, ny, nx), spacing=(dv[0], dv[1], dv[2]))
    return out


def cylinder_variant_phantom(seed, n=64, dv=1.0, physical=False):
    """Seeded variant of the cylinder + rod phantom for denoiser training:
    cylinder radius 18-28 mm and height 40-60 mm (on the 64 mm field of view),
    rod radius 3-8 voxels at a random offset inside the cylinder, rod material
    aluminium, bone or PMMA, and up to three small water/bone/PMMA/aluminium
    ellipsoids (semi-axes 2-8 voxels) inside the cylinder.  physical=True
    reads the rod radius and the semi-axes in mm instead of voxels, so that a
    finer grid over the same field of view (e.g. 256^3 x 0.25 mm) samples the
    same family of objects as 64^3 x 1 mm; at dv = 1 mm both are the same."""
    rng = np.random.default_rng(10_000 + seed)
    unit = 1.0 if physical else dv
    half = n * dv / 2.0
    c = _centres(n, dv)
    r_cyl = rng.uniform(0.56, 0.88) * half * 1.0
    h_cyl = rng.uniform(0.62, 0.94) * 2 * half
    r_rod = rng.uniform(3.0, 8.0) * unit
    ang = rng.uniform(0, 2 * np.pi)
    off = rng.uniform(0.0, max(r_cyl - r_rod - dv, 0.0))
    rx, ry = off * np.cos(ang), off * np.sin(ang)
    # the cylinder and rod are z-invariant inside |z| <= h/2: masks in the x-y plane
    y2, x2 = np.meshgrid(c, c, indexing="ij")
    inz = np.abs(c) <= h_cyl / 2.0
    plane = np.full((n, n), MAT_AIR, dtype=np.uint8)
    plane[x2**2 + y2**2 <= r_cyl**2] = MAT_WATER
    rod_mat = [MAT_AL, MAT_BONE, MAT_PMMA][int(rng.integers(0, 3))]
    plane[(x2 - rx) ** 2 + (y2 - ry) ** 2 <= r_rod**2] = rod_mat
    mat = np.full((n, n, n), MAT_AIR, dtype=np.uint8)
    mat[inz] = plane
    for _ in range(int(rng.integers(0, 4))):
        cx, cy = rng.uniform(-0.6, 0.6, 2) * r_cyl
        cz = rng.uniform(-0.4, 0.4) * h_cyl
        ax = rng.uniform(2.0, 8.0, 3) * unit
        m = [MAT_WATER, MAT_BONE, MAT_PMMA, MAT_AL][int(rng.integers(0, 4))]
        # only the ellipsoid's bounding slab of z is touched
        zs = np.nonzero(np.abs(c - cz) <= ax[2])[0]
        if len(zs) == 0:
            continue
        z3 = c[zs][:, None, None]
        inside = ((x2[None] - cx) / ax[0]) ** 2 + ((y2[None] - cy) / ax[1]) ** 2 + ((z3 - cz) / ax[2]) ** 2 <= 1.0
        sub = mat[zs]
        sub[inside & (sub != MAT_AIR)] = m
        mat[zs] = sub
    out = _finish(mat)
    out.update(shape=(n, n, n), spacing=(dv, dv, dv))
    return out
